"""Perpendicular components of the pair and self-difference kernels (needs a
GPU): each two-particle tensor K_par(r) e e^T + K_perp(r) (1 - e e^T) of
Sec. II A, against the FP64 oracle -- the step, a batch member, the
pair-correlated noise -- and bit-identical graph forms."""
import numpy as np
import pytest

import oracle
from gld_cases import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _w(n=4096, seed=41):
    from paper_1808_00270_gb300 import inputs
    return inputs.Workload(f"perp_n{n}", n=n, box=inputs.box_for_density(n, 0.1), m_max=200, dt=0.005, r_c=2.0,
                           tau_s=0.5, tau_p=0.3, steps=1, seed=seed, nr=257)


def _kernels(w, self_diff=True, scale=1.0):
    """Pair term f g, self-difference term 0.3 f with 0.5 g, and perpendicular
    factors of a different radial shape."""
    from paper_1808_00270_gb300 import inputs
    g, f, dr = inputs.pair_kernel_tables(w)
    r = np.arange(f.shape[1]) * dr
    fp = (0.8 * np.clip(1 - r / w.r_c, 0, None) * (1 + np.cos(2 * r)))[None]
    kw = dict(Ks=inputs.self_kernel_samples(w), g=g, f=scale * f, dr=dr)
    perp = dict(fp=scale * fp)
    if self_diff:
        kw.update(gs=0.5 * g, fs=0.3 * scale * f)
        perp.update(fs=0.25 * scale * fp)
    return kw, perp


def _gpu(w, kw, perp, **gkw):
    from paper_1808_00270_gb300 import GLD, inputs
    pos, vel = inputs.initial_state(w)
    s = GLD(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c, A_cons=w.A_cons,
            seed=w.seed, pos=pos, vel=vel, **gkw)
    s.set_kernels(kw["Ks"], g=kw["g"], f=kw["f"], dr=kw["dr"], gs=kw.get("gs"), fs=kw.get("fs"))
    if perp is not None:
        s.set_perpendicular(perp["fp"], perp.get("fs"))
    return s


def _oracle_from(w, gpu, kw, perp):
    from paper_1808_00270_gb300 import ARR_FC, ARR_HIST
    pos, vel = gpu.get_state()
    s = oracle.System(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c,
                      A_cons=w.A_cons, seed=w.seed, pos=pos, vel=vel)
    assert s.set_kernels(kw["Ks"], g=kw["g"], f=kw["f"], dr=kw["dr"], gs=kw.get("gs"), fs=kw.get("fs")) == 0
    assert s.set_perp(perp["fp"], perp.get("fs")) == 0
    s.set_state(step=gpu.step_index, pos=pos, vel=vel, fc=gpu.get(ARR_FC), hist=gpu.get(ARR_HIST))
    return s


@pytest.mark.parametrize("self_diff", [False, True])
def test_perpendicular_step_matches_oracle(self_diff):
    """After 150 steps with perpendicular factors: one step's F^D, F^R and
    V_{n+1} within 1e-5 of the oracle (pair term alone, and with the
    self-difference term)."""
    from paper_1808_00270_gb300 import ARR_FD, ARR_FR
    w = _w()
    kw, perp = _kernels(w, self_diff)
    gpu = _gpu(w, kw, perp)
    gpu.step(150)
    ref = _oracle_from(w, gpu, kw, perp)
    gpu.step(1)
    ref.step(1)
    errs = {"fd": rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD)), "fr": rel_l2(gpu.get(ARR_FR), ref.get(oracle.FR)),
            "vel": rel_l2(gpu.get_state()[1], ref.get(oracle.VEL))}
    assert max(errs.values()) < 1e-5, errs


def test_perpendicular_changes_the_force_and_clears():
    """The perpendicular terms are not negligible here, and gld_set_kernels
    (or all-zero factors) returns to the parallel-only force bit for bit."""
    from paper_1808_00270_gb300 import ARR_FD
    w = _w(seed=42)
    kw, perp = _kernels(w)
    a, b = _gpu(w, kw, None), _gpu(w, kw, perp)
    a.step(100)
    b.step(100)
    assert rel_l2(b.get(ARR_FD), a.get(ARR_FD)) > 1e-3
    c, d = _gpu(w, kw, None), _gpu(w, kw, {"fp": 0 * perp["fp"], "fs": 0 * perp["fs"]})
    c.step(70)
    d.step(70)
    assert np.array_equal(c.get_state()[0], d.get_state()[0])


def test_perpendicular_in_a_batch_and_graph_forms():
    """A member with perpendicular factors steps in a batch as alone (to FP32
    rounding of the convolution order); eager and both graph forms agree bit
    for bit."""
    from paper_1808_00270_gb300 import ARR_DISP, Batch
    w = _w(n=2000, seed=43)
    kw, perp = _kernels(w)
    outs = []
    for ug in (0, 1, 2):
        s = _gpu(w, kw, perp, use_graphs=ug)
        s.step(128)
        outs.append(s.get_state()[0])
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    alone, member = _gpu(w, kw, perp), _gpu(w, kw, perp)
    other = _gpu(_w(n=1500, seed=44), *_kernels(_w(n=1500, seed=44)))
    bt = Batch()
    bt.add(member)
    bt.add(other)
    bt.step(128)
    bt.sync()
    alone.step(128)
    assert rel_l2(member.get(ARR_DISP), alone.get(ARR_DISP)) < 1e-5


def test_perpendicular_pair_noise_matches_dense_square_roots():
    """With perpendicular factors the pair matrix has blocks
    f e e^T + fp (1 - e e^T): F^R of one step within 2e-6 of the oracle's
    dense square roots."""
    from paper_1808_00270_gb300 import ARR_FR
    w = _w(n=128, seed=45)
    kw, perp = _kernels(w, self_diff=False, scale=0.3)
    gpu = _gpu(w, kw, perp)
    lam, err = gpu.set_pair_noise(12)
    assert err < 1e-8
    gpu.step(37)
    ref = _oracle_from(w, gpu, kw, perp)
    want = ref.pair_random_force()
    gpu.step(1)
    e = rel_l2(gpu.get(ARR_FR), want)
    print(f"perpendicular pair noise: lambda {lam:.3f}, interpolation {err:.1e}, F^R {e:.2e}")
    assert e < 2e-6
