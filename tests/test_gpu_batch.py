"""Batches of independent GLD systems (needs a GPU).

A member of a batch integrates exactly the system it would integrate alone:
its particles, kernels, noise stream and VACF are its own, the batch only
merges the launches.  Checked against the oracle (trajectory tolerance of the
single-system tests), against the same system stepped alone, and for bitwise
independence of the other members."""
import numpy as np
import pytest

import oracle
from gld_cases import make_gpu, make_oracle, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _workload(name, n, rho, m_max, seed, dt=0.005, tau_s=0.5, tau_p=0.3):
    from paper_1808_00270_gb300 import inputs
    return inputs.Workload(name, n=n, box=inputs.box_for_density(n, rho), m_max=m_max, dt=dt, r_c=2.0,
                           tau_s=tau_s, tau_p=tau_p, steps=1, tail=True, seed=seed)


def _mixed():
    """Uneven members: sizes, densities and memory lengths all differ."""
    from paper_1808_00270_gb300 import inputs
    return [inputs.WORKLOADS["gld_n64_m32"],
            _workload("b_n300_m100", 300, 0.05, 100, 11),
            _workload("b_n4096_m200", 4096, 0.1, 200, 12),
            _workload("b_n1500_m400", 1500, 0.2, 400, 13),
            _workload("b_n700_m64", 700, 0.02, 64, 14)]


def _state(g):
    from paper_1808_00270_gb300 import ARR_DISP
    p, v = g.get_state()
    return p, v, g.get(ARR_DISP)


def test_batch_members_follow_the_oracle():
    """Each member of a mixed batch, 128 steps: unwrapped displacement within
    1e-4 and velocities within 1e-3 relative L2 of the FP64 oracle run alone."""
    from paper_1808_00270_gb300 import ARR_DISP, Batch
    ws = _mixed()
    gs = [make_gpu(w) for w in ws]
    b = Batch()
    for g in gs:
        b.add(g)
    b.step(128)
    b.sync()
    assert b.info()["members"] == len(ws) and b.info()["schedule"] in (0, 1, 2, 3)
    for w, g in zip(ws, gs):
        ref = make_oracle(w)
        ref.step(128)
        assert g.step_index == 128
        assert rel_l2(g.get(ARR_DISP), ref.get(oracle.DISP)) < 1e-4, w.name
        _, v = g.get_state()
        assert rel_l2(v, ref.get(oracle.VEL)) < 1e-3, w.name


def test_member_alone_and_mixed_bit_identical():
    """A system's trajectory does not depend on the other members: stepped in
    a batch of one and in a mixed batch it gives the same bits."""
    from paper_1808_00270_gb300 import Batch
    ws = _mixed()
    target = ws[2]
    alone = make_gpu(target)
    b1 = Batch()
    b1.add(alone)
    b1.step(192)
    b1.sync()
    gs = [make_gpu(w) for w in ws]
    b2 = Batch()
    for g in reversed(gs):
        b2.add(g)
    b2.step(128)
    b2.remove(gs[0])  # composition changes at a block boundary
    b2.step(64)
    b2.sync()
    for x, y in zip(_state(alone), _state(gs[2])):
        assert np.array_equal(x, y)


def test_batch_matches_single_system_path():
    """The batch kernels and the single-system kernels integrate the same
    system: after 128 batched steps plus 70 steps alone the state matches a
    system stepped alone throughout (summation order of the convolution may
    differ, so to FP32 rounding)."""
    from paper_1808_00270_gb300 import Batch
    w = _mixed()[3]
    a = make_gpu(w)
    g = make_gpu(w)
    b = Batch()
    b.add(g)
    b.step(128)
    b.remove(g)
    g.step(70)
    a.step(198)
    for x, y in zip(_state(a), _state(g)):
        assert rel_l2(y, x) < 1e-5


def test_white_noise_ring_changes_form_between_batch_and_alone():
    """Stepped alone, a context keeps its white-noise ring in the FP16 split
    the tensor-core filter multiplies; inside a batch, in FP32 for the batched
    filter.  Each change clears the ring and regenerates the window: F^R of
    the first step alone after a batched block is within 1e-5 of the
    oracle's, and after alone / batch / alone / batch / alone the state
    matches the context stepped alone throughout (FP32 rounding)."""
    from paper_1808_00270_gb300 import ARR_FR, Batch
    from gld_cases import oracle_from_gpu
    w = _mixed()[3]  # 1500 particles, m_max = 400: the tensor-core filter when alone
    a = make_gpu(w)
    g = make_gpu(w)
    g.step(64)
    for _ in range(2):
        b = Batch()
        b.add(g)
        b.step(64)
        b.sync()
        b.remove(g)
        ref = oracle_from_gpu(w, g)
        g.step(1)
        ref.step(1)
        assert rel_l2(g.get(ARR_FR), ref.get(oracle.FR)) < 1e-5
        g.step(63)
    a.step(320)
    for x, y in zip(_state(a), _state(g)):
        assert rel_l2(y, x) < 1e-5


def test_batch_vacf_matches_single_system():
    """The VACF accumulated inside a batch equals the one of the same system
    stepped alone (to FP32 rounding of the trajectory)."""
    from paper_1808_00270_gb300 import Batch
    w = _mixed()[2]
    a = make_gpu(w, vacf_len=100, vacf_stride=20, vacf_burnin=1)
    g = make_gpu(w, vacf_len=100, vacf_stride=20, vacf_burnin=1)
    other = make_gpu(_mixed()[1], vacf_len=50, vacf_stride=50, vacf_burnin=10)
    b = Batch()
    b.add(g)
    b.add(other)
    b.step(256)
    a.step(256)
    ca, na = a.vacf()
    cg, ng = g.vacf()
    assert na == ng and np.array_equal(np.isnan(ca), np.isnan(cg))
    ok = ~np.isnan(ca)
    assert np.max(np.abs(cg[ok] - ca[ok])) <= 1e-4 * abs(ca[0])
    co, no = other.vacf()
    assert no > 0 and np.isfinite(co[0]) and co[0] > 0


def test_batch_preconditions():
    from paper_1808_00270_gb300 import Batch, GLDError
    ws = _mixed()
    b = Batch()
    g = make_gpu(ws[0])
    b.add(g)
    with pytest.raises(GLDError):
        b.add(g)  # twice
    with pytest.raises(GLDError):
        b.step(65)  # not a multiple of 64
    h = make_gpu(ws[1])
    h.step(3)
    with pytest.raises(GLDError):
        b.add(h)  # inside a noise block
    h.step(61)
    b.add(h)
    nopair = make_gpu(ws[4], pair=False)
    with pytest.raises(GLDError):
        b.add(nopair)  # different number of kernel terms
    b.step(64)
    b.sync()
    assert g.step_index == 64 and h.step_index == 128
    b.step(0)
    empty = Batch()
    empty.step(64)
    empty.sync()


def test_batch_history_precision_against_oracle():
    """FP32 and BF16+Kahan history rings in a mixed batch, 128 steps from the
    same initial states, against the FP64 oracle: unwrapped displacement
    relative L2 below 1e-4 (FP32) and 1e-2 (BF16 with compensated sums)."""
    from paper_1808_00270_gb300 import ARR_DISP, Batch
    ws = _mixed()[1:4]
    errs = {}
    for label, kw in (("f32", {}), ("bf16_kahan", dict(hist_dtype="bf16", kahan=True))):
        gs = [make_gpu(w, **kw) for w in ws]
        b = Batch()
        for g in gs:
            b.add(g)
        b.step(128)
        b.sync()
        errs[label] = []
        for w, g in zip(ws, gs):
            ref = make_oracle(w)
            ref.step(128)
            errs[label].append(rel_l2(g.get(ARR_DISP), ref.get(oracle.DISP)))
    print("displacement relative L2 vs FP64 oracle after 128 batched steps:", errs)
    assert max(errs["f32"]) < 1e-4
    assert max(errs["bf16_kahan"]) < 1e-2


def _pn_member(w, degree=0, strength=0.3):
    """A context with the workload's pair kernel scaled by `strength` and, for
    degree > 0, the Chebyshev pair noise on the Gershgorin bound."""
    from paper_1808_00270_gb300 import GLD, inputs
    pos, vel = inputs.initial_state(w)
    g, f, dr = inputs.pair_kernel_tables(w)
    s = GLD(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c, A_cons=w.A_cons,
            seed=w.seed, pos=pos, vel=vel)
    s.set_kernels(inputs.self_kernel_samples(w), g=g, f=strength * f, dr=dr)
    if degree:
        s.set_pair_noise(degree)
    return s


def test_batch_pair_noise_matches_single_system():
    """Members with the Chebyshev pair noise (degrees 8 and 4) beside one
    without: over two noise blocks each follows the same system stepped
    alone (F^R of the last step, positions, velocities and displacements
    within 1e-5; the batch filters on the FP32 pipes, a context alone on the
    tensor cores), and the member without pair noise gets the bits it gets in
    a batch of its own."""
    from paper_1808_00270_gb300 import ARR_FR, Batch
    ws = [_workload("pn_a", 128, 0.1, 200, 21), _workload("pn_b", 500, 0.08, 200, 22),
          _workload("pn_c", 300, 0.05, 100, 23)]
    degs = [8, 4, 0]
    alone = [_pn_member(w, d) for w, d in zip(ws, degs)]
    inb = [_pn_member(w, d) for w, d in zip(ws, degs)]
    b = Batch()
    for g in inb:
        b.add(g)
    b.step(128)
    b.sync()
    for a in alone:
        a.step(128)
    for a, g in zip(alone, inb):
        assert rel_l2(g.get(ARR_FR), a.get(ARR_FR)) < 1e-5
        for x, y in zip(_state(a), _state(g)):
            assert rel_l2(y, x) < 1e-5
    solo = _pn_member(ws[2])
    b2 = Batch()
    b2.add(solo)
    b2.step(128)
    b2.sync()
    for x, y in zip(_state(solo), _state(inb[2])):
        assert np.array_equal(x, y)


def test_batch_refuses_the_estimated_interval_and_lanczos_forms():
    from paper_1808_00270_gb300 import Batch, GLDError
    from paper_1808_00270_gb300.binding import E_INVAL
    w = _workload("pn_d", 128, 0.1, 200, 24)
    for form in ("interval", "lanczos"):
        g = _pn_member(w, strength=1.0)
        if form == "interval":
            g.set_pair_noise_on(8)
        else:
            g.set_pair_noise_krylov(1e-6, 16)
        with pytest.raises(GLDError) as e:
            Batch().add(g)
        assert e.value.status == E_INVAL
