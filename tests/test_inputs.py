"""The seeded synthetic inputs follow the stated recipe (no device needed):
workload sizes and densities, the batch and serving distributions, and
that every generator is deterministic in its seed."""
import math

import numpy as np

from paper_1808_00270_gb300 import inputs


def test_single_system_workloads():
    for w, n, rho in ((inputs.MEDIUM, 4096, 0.1), (inputs.LARGE, 262144, 0.1)):
        assert w.n == n and abs(w.density - rho) < 1e-12
    assert inputs.LARGE.m_max == 400 and inputs.LARGE.r_c == 2.5 and inputs.LARGE.tail
    assert inputs.LARGE.r_c <= inputs.LARGE.box / 2


def test_initial_state_is_uniform_and_maxwellian():
    w = inputs.MEDIUM
    pos, vel = inputs.initial_state(w)
    assert pos.shape == (w.n, 3) and pos.min() >= 0 and pos.max() < w.box
    assert abs(pos.mean() / w.box - 0.5) < 0.01
    assert abs(vel.var() - w.kT / w.mass) < 0.03 and abs(vel.mean()) < 0.02
    p2, v2 = inputs.initial_state(w)
    assert np.array_equal(pos, p2) and np.array_equal(vel, v2)


def test_batch_systems_recipe():
    ws = inputs.batch_systems()
    assert len(ws) == 512
    ns = np.array([w.n for w in ws])
    rho = np.array([w.density for w in ws])
    assert ns.min() >= 256 and ns.max() <= 16384
    assert rho.min() >= 0.02 * (1 - 1e-9) and rho.max() <= 0.2 * (1 + 1e-9)
    assert {w.m_max for w in ws} <= {100, 200, 400}
    # log-uniform sizes: the mean of ln N sits mid-range
    assert abs(np.log(ns).mean() - 0.5 * (math.log(256) + math.log(16384))) < 0.2
    assert 1.8e6 < ns.sum() < 2.1e6
    assert [w.n for w in inputs.batch_systems()] == list(ns)


def test_serve_trace_recipe():
    tr = inputs.serve_trace()
    assert len(tr) == 1000
    t = np.array([r.arrival for r in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 1 / 50.0) < 0.003  # Poisson at 50 per second
    ns = np.array([r.w.n for r in tr])
    ms = np.array([r.w.m_max for r in tr])
    steps = np.array([r.steps for r in tr])
    assert ns.min() >= 512 and ns.max() <= 65536
    assert ms.min() >= 64 and ms.max() <= 400
    assert steps.min() >= 2000 and steps.max() <= 20000
    assert [r.w.n for r in inputs.serve_trace()] == list(ns)
