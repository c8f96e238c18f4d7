"""Parity at the full sizes (needs a GPU): the 262144-particle, m_max = 400
suspension on sampled particles in the launch configuration bench.py times
(graphs, 64-step noise blocks) -- with the benchmark's kernels and with the
general pair kernel -- and the VACF of the 4096-particle system over
10^4 steps against an independent oracle run."""
import numpy as np
import pytest

import oracle
from gld_cases import make_gpu, make_oracle, oracle_from_gpu, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_large_suspension_sampled_forces():
    from paper_1808_00270_gb300 import ARR_FD, ARR_FR, inputs
    w = inputs.LARGE
    gpu = make_gpu(w)
    gpu.step(448)  # past m_max - 1: every ring slot holds a real displacement
    ref = oracle_from_gpu(w, gpu)
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(w.n, size=1500, replace=False)).astype(np.int32)
    fd_ref, fr_ref = ref.forces_subset(idx)
    gpu.step(1)
    fd, fr = gpu.get(ARR_FD)[idx], gpu.get(ARR_FR)[idx]
    assert rel_l2(fd, fd_ref) < 1e-5
    assert rel_l2(fr, fr_ref) < 1e-5


def test_large_suspension_general_pair_kernel_sampled_forces():
    """The same at full size with the general pair kernel: a self-difference
    term and perpendicular factors on top of the pair term (Sec. II A)."""
    from paper_1808_00270_gb300 import ARR_FC, ARR_FD, ARR_FR, ARR_HIST, GLD, inputs
    w = inputs.LARGE
    g, f, dr = inputs.pair_kernel_tables(w)
    r = np.arange(f.shape[1]) * dr
    fp = (0.8 * np.clip(1 - r / w.r_c, 0, None) * (1 + np.cos(2 * r)))[None]
    ks = inputs.self_kernel_samples(w)
    pos, vel = inputs.initial_state(w)
    kw = dict(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c, A_cons=w.A_cons,
              seed=w.seed)
    gpu = GLD(pos=pos, vel=vel, **kw)
    gpu.set_kernels(ks, g=g, f=f, dr=dr, gs=0.5 * g, fs=0.3 * f)
    gpu.set_perpendicular(fp, 0.25 * fp)
    gpu.step(448)
    p, v = gpu.get_state()
    ref = oracle.System(pos=p, vel=v, **kw)
    assert ref.set_kernels(ks, g=g, f=f, dr=dr, gs=0.5 * g, fs=0.3 * f) == 0
    assert ref.set_perp(fp, 0.25 * fp) == 0
    ref.set_state(step=gpu.step_index, pos=p, vel=v, fc=gpu.get(ARR_FC), hist=gpu.get(ARR_HIST))
    idx = np.sort(np.random.default_rng(12).choice(w.n, size=1500, replace=False)).astype(np.int32)
    fd_ref, fr_ref = ref.forces_subset(idx)
    gpu.step(1)
    assert rel_l2(gpu.get(ARR_FD)[idx], fd_ref) < 1e-5
    assert rel_l2(gpu.get(ARR_FR)[idx], fr_ref) < 1e-5


@pytest.mark.parametrize("wname,L,stride,burn", [("gld_n64_m32", 12, 3, 5), ("gld_n4096_m200", 40, 3, 2)])
def test_vacf_accumulator_definition(wname, L, stride, burn):
    """The VACF accumulator equals the definition evaluated on the recorded
    velocities with the same origin schedule (one or several particle blocks,
    one or several groups of origins)."""
    from paper_1808_00270_gb300 import inputs
    w = inputs.WORKLOADS[wname]
    gpu = make_gpu(w, vacf_len=L, vacf_stride=stride, vacf_burnin=burn)
    V = {0: gpu.get_state()[1]}
    for t in range(1, 60):
        gpu.step(1)
        V[t] = gpu.get_state()[1]
    acc, cnt = np.zeros(L), np.zeros(L)
    for t0 in range(burn, 60, stride):
        for lag in range(L):
            if t0 + lag < 60:
                acc[lag] += (V[t0 + lag] * V[t0]).sum()
                cnt[lag] += 1
    want = acc / (3 * w.n * cnt)
    c, n0 = gpu.vacf()
    assert n0 == len(range(burn, 60, stride))
    assert np.max(np.abs(c - want)) < 1e-6 * np.abs(want).max()


def test_vacf_medium_matches_oracle():
    from paper_1808_00270_gb300 import inputs
    w = inputs.MEDIUM
    kw = dict(vacf_len=200, vacf_stride=10, vacf_burnin=400)
    gpu = make_gpu(w, **kw)
    gpu.step(w.steps)
    c_gpu, n_gpu = gpu.vacf()
    ref = make_oracle(w, **kw)
    ref.step(w.steps)
    c_ref, n_ref = ref.vacf()
    assert n_gpu == n_ref
    dev = np.max(np.abs(c_gpu - c_ref)) / c_ref[0]
    print(f"VACF max deviation / C(0) = {dev:.4f}")
    assert dev <= 0.02
