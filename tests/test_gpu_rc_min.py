"""The lower cutoff r_c,min of the pair kernels (Sec. III B: below r_c,min a
kernel keeps its value at r_c,min) on the GPU (needs a GPU).  A dense
4096-particle system with r_c,min = 0.6 r_c, in which several pairs per
particle are closer than r_c,min: one step against the FP64 oracle with the
one-term pair kernel (fast instance) and with the general kernel (a
self-difference term and perpendicular factors)."""
import numpy as np
import pytest

import oracle
from gld_cases import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RC, RC_MIN = 2.0, 1.2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _w():
    from paper_1808_00270_gb300 import inputs
    return inputs.Workload("rcmin_n4096_rho0.5", n=4096, box=inputs.box_for_density(4096, 0.5), m_max=200,
                           dt=0.005, r_c=RC, tau_s=0.5, tau_p=0.3, steps=1, seed=53, r_c_min=RC_MIN, nr=257)


def _kernels(w, general):
    """The workload's pair kernel f g; for the general form also a
    self-difference term 0.3 f with 0.5 g and perpendicular factors of a
    different radial shape (all varying below r_c,min)."""
    from paper_1808_00270_gb300 import inputs
    g, f, dr = inputs.pair_kernel_tables(w)
    kw = dict(Ks=inputs.self_kernel_samples(w), g=g, f=f, dr=dr)
    perp = None
    if general:
        r = np.arange(f.shape[1]) * dr
        fp = (0.8 * np.clip(1 - r / w.r_c, 0, None) * (1 + np.cos(2 * r)))[None]
        kw.update(gs=0.5 * g, fs=0.3 * f)
        perp = dict(fp=fp, fs=0.25 * fp)
    return kw, perp


def _common(w, rc_min):
    return dict(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c, r_c_min=rc_min,
                A_cons=w.A_cons, seed=w.seed)


def _oracle(w, gpu, kw, perp, rc_min):
    from paper_1808_00270_gb300 import ARR_FC, ARR_HIST
    pos, vel = gpu.get_state()
    s = oracle.System(pos=pos, vel=vel, **_common(w, rc_min))
    assert s.set_kernels(kw["Ks"], g=kw["g"], f=kw["f"], dr=kw["dr"], gs=kw.get("gs"), fs=kw.get("fs")) == 0
    if perp is not None:
        assert s.set_perp(perp["fp"], perp["fs"]) == 0
    s.set_state(step=gpu.step_index, pos=pos, vel=vel, fc=gpu.get(ARR_FC), hist=gpu.get(ARR_HIST))
    return s


@pytest.mark.parametrize("general", [False, True], ids=["one_term", "general_perp"])
def test_rc_min_step_matches_oracle(general):
    """After 150 steps: one step's F^D, F^R and V_{n+1} within 1e-5 of the
    oracle.  The system has more than one pair below r_c,min per particle,
    and the oracle without the cutoff differs by far more than the
    tolerance, so a kernel that ignored r_c,min would fail."""
    from paper_1808_00270_gb300 import ARR_FD, ARR_FR, GLD, inputs
    w = _w()
    kw, perp = _kernels(w, general)
    pos, vel = inputs.initial_state(w)
    gpu = GLD(pos=pos, vel=vel, **_common(w, RC_MIN))
    gpu.set_kernels(kw["Ks"], g=kw["g"], f=kw["f"], dr=kw["dr"], gs=kw.get("gs"), fs=kw.get("fs"))
    if perp is not None:
        gpu.set_perpendicular(perp["fp"], perp["fs"])
    gpu.step(150)
    ref = _oracle(w, gpu, kw, perp, RC_MIN)
    plain = _oracle(w, gpu, kw, perp, 0.0)
    p_now, _ = gpu.get_state()
    close = oracle.pairs_brute(p_now, w.box, RC_MIN).shape[0]
    assert close > w.n, f"only {close} pairs below r_c,min"
    gpu.step(1)
    ref.step(1)
    plain.step(1)
    e_fd = rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD))
    e_fr = rel_l2(gpu.get(ARR_FR), ref.get(oracle.FR))
    e_v = rel_l2(gpu.get_state()[1], ref.get(oracle.VEL))
    gap = rel_l2(plain.get(oracle.FD), ref.get(oracle.FD))
    print(f"pairs below r_c,min {close}; F^D {e_fd:.2e} F^R {e_fr:.2e} V {e_v:.2e}; without the cutoff {gap:.2e}")
    assert e_fd < 1e-5 and e_fr < 1e-5 and e_v < 1e-5
    assert gap > 1e-3
    gpu.close()
