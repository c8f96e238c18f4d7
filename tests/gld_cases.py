"""Shared set-up of GPU/oracle pairs on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1808_00270_gb300 import inputs


def rel_l2(a, b) -> float:
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def kernels(w: inputs.Workload):
    g, f, dr = inputs.pair_kernel_tables(w)
    return inputs.self_kernel_samples(w), g, f, dr


def common_kwargs(w: inputs.Workload, **over):
    kw = dict(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c,
              r_c_min=w.r_c_min, A_cons=w.A_cons, seed=w.seed)
    kw.update(over)
    return kw


def make_gpu(w: inputs.Workload, pos=None, vel=None, pair=True, **over):
    from paper_1808_00270_gb300 import GLD
    if pos is None:
        pos, vel = inputs.initial_state(w)
    gkw = {k: over.pop(k) for k in list(over) if k in ("hist_dtype", "kahan", "noise_block", "use_graphs",
                                                        "psd_clamp", "torch_allocator", "order", "skin")}
    sys_ = GLD(pos=pos, vel=vel, **common_kwargs(w, **over), **gkw)
    ks, g, f, dr = kernels(w)
    if pair:
        sys_.set_kernels(ks, g=g, f=f, dr=dr)
    else:
        sys_.set_kernels(ks)
    return sys_


def make_oracle(w: inputs.Workload, pos=None, vel=None, pair=True, **over):
    if pos is None:
        pos, vel = inputs.initial_state(w)
    s = oracle.System(pos=pos, vel=vel, **common_kwargs(w, **over))
    ks, g, f, dr = kernels(w)
    st = s.set_kernels(ks, g=g, f=f, dr=dr) if pair else s.set_kernels(ks)
    assert st == 0
    return s


def oracle_from_gpu(w: inputs.Workload, gpu, pair=True, **over):
    """An oracle system loaded with the GPU's current FP32 state."""
    from paper_1808_00270_gb300 import ARR_FC, ARR_HIST
    pos, vel = gpu.get_state()
    s = make_oracle(w, pos=pos, vel=vel, pair=pair, **over)
    s.set_state(step=gpu.step_index, pos=pos, vel=vel, fc=gpu.get(ARR_FC), hist=gpu.get(ARR_HIST))
    return s
