"""Step-level parity of the CUDA path with the FP64 oracle (needs a GPU).

Tolerances: forces 1e-5 relative L2 per force type with the oracle fed the
GPU's FP32 state; unwrapped displacement after 100 steps 1e-4 relative L2;
VACF max |C_gpu - C_oracle| / C_oracle(0) <= 0.02."""
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


def _w(name):
    from paper_1808_00270_gb300 import inputs
    return inputs.WORKLOADS[name]


@pytest.mark.parametrize("wname,warm", [("gld_n64_m32", 0), ("gld_n64_m32", 45), ("gld_n64_m32", 64),
                                        ("gld_n4096_m200", 130), ("gld_n4096_m200", 250)])
def test_one_step_forces(wname, warm):
    """F^D_n, F^R_n, F^C_{n+1} and the new state from one step, oracle fed the
    GPU's FP32 state at step n (history partly or fully populated)."""
    from paper_1808_00270_gb300 import ARR_DISP, ARR_FC, ARR_FD, ARR_FR
    w = _w(wname)
    gpu = make_gpu(w)
    gpu.step(warm)
    ref = oracle_from_gpu(w, gpu)
    d0 = gpu.get(ARR_DISP)
    gpu.step(1)
    ref.step(1)
    assert rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD)) < 1e-5
    assert rel_l2(gpu.get(ARR_FR), ref.get(oracle.FR)) < 1e-5
    assert rel_l2(gpu.get(ARR_FC), ref.get(oracle.FC)) < 1e-5
    assert rel_l2(gpu.get(ARR_DISP) - d0, ref.get(oracle.DISP)) < 1e-5
    _, v = gpu.get_state()
    assert rel_l2(v, ref.get(oracle.VEL)) < 1e-5


def test_long_memory_one_step():
    """m_max = 1000: the noise filter runs over several tap chunks and the
    convolution over 999 slots; one step against the oracle at 1e-5."""
    from paper_1808_00270_gb300 import ARR_FD, ARR_FR, inputs
    w = inputs.Workload("gld_n500_m1000", n=500, box=inputs.box_for_density(500, 0.1), m_max=1000, dt=0.005,
                        r_c=2.0, tau_s=0.5, tau_p=0.3, steps=1, tail=True)
    gpu = make_gpu(w)
    gpu.step(1100)
    ref = oracle_from_gpu(w, gpu)
    gpu.step(1)
    ref.step(1)
    assert rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD)) < 1e-5
    assert rel_l2(gpu.get(ARR_FR), ref.get(oracle.FR)) < 1e-5


@pytest.mark.parametrize("wname", ["gld_n64_m32", "gld_n4096_m200"])
def test_trajectory_100_steps(wname):
    """Independent integrations from the same initial state and noise stream:
    unwrapped displacement after 100 steps within 1e-4 relative L2."""
    from paper_1808_00270_gb300 import ARR_DISP
    w = _w(wname)
    gpu = make_gpu(w)
    ref = make_oracle(w)
    gpu.step(100)
    ref.step(100)
    assert rel_l2(gpu.get(ARR_DISP), ref.get(oracle.DISP)) < 1e-4
    _, v = gpu.get_state()
    assert rel_l2(v, ref.get(oracle.VEL)) < 1e-3


def test_graph_and_eager_paths_identical():
    """Replaying captured graphs gives the same bits as launching eagerly, and
    any chunking of the steps gives the same bits."""
    from paper_1808_00270_gb300 import ARR_DISP
    w = _w("gld_n4096_m200")
    a = make_gpu(w, use_graphs=True)
    b = make_gpu(w, use_graphs=False)
    c = make_gpu(w, use_graphs=True)
    d = make_gpu(w, use_graphs=2)  # gated rebuild kernels instead of a conditional node
    a.step(150)
    b.step(150)
    d.step(150)
    for k in (1, 63, 2, 64, 20):
        c.step(k)
    pa, va = a.get_state()
    pb, vb = b.get_state()
    pc, vc = c.get_state()
    pd, vd = d.get_state()
    assert a.diag()["graph_mode"] in (1, 2) and d.diag()["graph_mode"] == 1
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert np.array_equal(pa, pc) and np.array_equal(va, vc)
    assert np.array_equal(pa, pd) and np.array_equal(va, vd)
    assert np.array_equal(a.get(ARR_DISP), c.get(ARR_DISP))


def test_checkpoint_resume_is_bit_identical():
    """State saved through the array API (with the internal order) and loaded
    into a fresh context created from the snapshot continues exactly as the
    uninterrupted run (noise is counter-based)."""
    from paper_1808_00270_gb300 import ARR_DISP, ARR_FC, ARR_HIST, ARR_POS, ARR_VEL
    w = _w("gld_n4096_m200")
    a = make_gpu(w)
    a.step(77)
    snap = {k: a.get(k) for k in (ARR_POS, ARR_VEL, ARR_FC, ARR_HIST, ARR_DISP)}
    step = a.step_index
    b = make_gpu(w, pos=snap[ARR_POS], vel=snap[ARR_VEL], order=a.order())
    b.set_step(step)
    b.set(ARR_POS, snap[ARR_POS])
    b.set(ARR_VEL, snap[ARR_VEL])
    b.set(ARR_FC, snap[ARR_FC])
    b.set(ARR_HIST, snap[ARR_HIST])
    b.set(ARR_DISP, snap[ARR_DISP])
    a.step(90)
    b.step(90)
    pa, va = a.get_state()
    pb, vb = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)


def test_checkpoint_of_observables_resumes_bit_identical():
    """A checkpoint taken after the VACF burn-in, with ten origins in flight
    and the pair correlations on: the run resumed from the state arrays plus
    gld_save_observables / gld_load_observables returns the VACF and C^a, C^c
    of the uninterrupted run bit for bit; without the observables blob the
    resumed sums differ (they restart at zero)."""
    from paper_1808_00270_gb300 import ARR_DISP, ARR_FC, ARR_HIST, ARR_POS, ARR_VEL
    w = _w("gld_n4096_m200")
    kw = dict(vacf_len=100, vacf_stride=10, vacf_burnin=50)
    a = make_gpu(w, **kw)
    a.set_pair_correlation(8, w.r_c)
    a.step(237)
    snap = {k: a.get(k) for k in (ARR_POS, ARR_VEL, ARR_FC, ARR_HIST, ARR_DISP)}
    blob = a.save_observables()
    _, n_orig = a.vacf()
    assert n_orig == 19  # origins at 50, 60, ..., 230; the last ten in flight
    step = a.step_index

    def resumed(load):
        b = make_gpu(w, pos=snap[ARR_POS], vel=snap[ARR_VEL], order=a.order(), **kw)
        b.set_pair_correlation(8, w.r_c)
        b.set_step(step)
        for k in (ARR_POS, ARR_VEL, ARR_FC, ARR_HIST, ARR_DISP):
            b.set(k, snap[k])
        if load:
            b.load_observables(blob)
        b.step(150)
        return b

    b, c = resumed(True), resumed(False)
    a.step(150)
    (ca, na), (cb, nb), (cc_, nc) = a.vacf(), b.vacf(), c.vacf()
    assert na == nb == 34 and nc == 15
    assert np.array_equal(ca, cb, equal_nan=True)
    assert not np.array_equal(ca, cc_, equal_nan=True)
    for x, y in zip(a.pair_correlation(), b.pair_correlation()):
        assert np.array_equal(x, y, equal_nan=True)
    assert not np.array_equal(a.pair_correlation()[2], c.pair_correlation()[2])


def test_observables_blob_checks_its_configuration():
    from paper_1808_00270_gb300 import GLDError
    from paper_1808_00270_gb300.binding import E_INVAL, E_STATE
    w = _w("gld_n4096_m200")
    a = make_gpu(w, vacf_len=100, vacf_stride=10, vacf_burnin=50)
    a.step(120)
    blob = a.save_observables()
    other = make_gpu(w, vacf_len=50, vacf_stride=10, vacf_burnin=50)
    other.set_step(120)
    with pytest.raises(GLDError) as e:
        other.load_observables(blob)
    assert e.value.status == E_INVAL
    same = make_gpu(w, vacf_len=100, vacf_stride=10, vacf_burnin=50)
    with pytest.raises(GLDError) as e:
        same.load_observables(blob)  # step index not restored first
    assert e.value.status == E_STATE
    same.set_step(120)
    same.load_observables(blob)
    assert same.vacf()[1] == a.vacf()[1]


def test_any_internal_order_matches_oracle():
    """The internal storage order is invisible: a random order gives the same
    one-step forces (to rounding) in the caller's order."""
    from paper_1808_00270_gb300 import ARR_FD, ARR_FR
    w = _w("gld_n4096_m200")
    perm = np.random.default_rng(5).permutation(w.n).astype(np.int32)
    gpu = make_gpu(w, order=perm)
    assert np.array_equal(gpu.order(), perm)
    gpu.step(70)
    ref = oracle_from_gpu(w, gpu)
    gpu.step(1)
    ref.step(1)
    assert rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD)) < 1e-5
    assert rel_l2(gpu.get(ARR_FR), ref.get(oracle.FR)) < 1e-5


def test_edge_cases():
    from paper_1808_00270_gb300 import ARR_FD, GLD, GLDError
    from paper_1808_00270_gb300.binding import E_INVAL, E_STATE
    rng = np.random.default_rng(3)
    # one particle, shortest memory: free GLE particle, no neighbours
    g = GLD(n=1, box=10.0, dt=0.01, m_max=2, r_c=2.0, pos=[[1.0, 2.0, 3.0]], vel=[[0.5, 0.0, 0.0]])
    with pytest.raises(GLDError) as e:
        g.step(1)
    assert e.value.status == E_STATE
    g.set_kernels([3.0, 1.0])
    g.step(0)
    g.step(5)
    ref = oracle.System(n=1, box=10.0, mass=1.0, kT=1.0, dt=0.01, m_max=2, r_c=2.0,
                        pos=[[1.0, 2.0, 3.0]], vel=[[0.5, 0.0, 0.0]])
    ref.set_kernels([3.0, 1.0])
    ref.step(5)
    assert rel_l2(g.get(ARR_FD), ref.get(oracle.FD)) < 1e-5
    # ragged particle count (not a multiple of 32) with pair kernels
    from paper_1808_00270_gb300 import inputs
    w = inputs.Workload("ragged", n=77, box=9.0, m_max=17, dt=0.01, r_c=2.0, tau_s=0.2, tau_p=0.1, steps=1)
    gpu = make_gpu(w)
    gpu.step(20)
    ref = oracle_from_gpu(w, gpu)
    gpu.step(1)
    ref.step(1)
    assert rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD)) < 1e-5
    # invalid parameters
    for bad in (dict(n=0), dict(m_max=1), dict(r_c=6.0), dict(box=-1.0), dict(dt=0.0)):
        kw = dict(n=4, box=10.0, dt=0.01, m_max=4, r_c=2.0, pos=rng.uniform(0, 10, (4, 3)),
                  vel=np.zeros((4, 3)))
        kw.update(bad)
        kw["pos"], kw["vel"] = kw["pos"][: kw["n"]], kw["vel"][: kw["n"]]
        with pytest.raises(GLDError) as e:
            GLD(**kw)
        assert e.value.status == E_INVAL


def test_bf16_and_kahan_errors_against_oracle():
    """F^D error against the FP64 oracle when one FP32 state (history included)
    is loaded into contexts with FP32+Kahan and with BF16 history storage; the
    BF16 contexts round the displacements when they are stored."""
    from paper_1808_00270_gb300 import ARR_DISP, ARR_FC, ARR_FD, ARR_HIST, ARR_POS, ARR_VEL
    w = _w("gld_n4096_m200")
    src = make_gpu(w)
    src.step(250)
    snap = {k: src.get(k) for k in (ARR_POS, ARR_VEL, ARR_FC, ARR_HIST, ARR_DISP)}
    step = src.step_index
    ref = oracle_from_gpu(w, src)
    ref.step(1)
    want = ref.get(oracle.FD)
    errs = {}
    for label, kw in (("f32", {}), ("f32_kahan", dict(kahan=True)), ("bf16", dict(hist_dtype="bf16")),
                      ("bf16_kahan", dict(hist_dtype="bf16", kahan=True))):
        g = make_gpu(w, **kw)
        g.set_step(step)
        for k, v in snap.items():
            g.set(k, v)
        g.step(1)
        errs[label] = rel_l2(g.get(ARR_FD), want)
    print("F^D relative L2 error vs FP64 oracle:", errs)
    assert errs["f32"] < 1e-5 and errs["f32_kahan"] < 1e-5
    assert errs["bf16"] < 1e-2 and errs["bf16_kahan"] < 1e-2, errs
