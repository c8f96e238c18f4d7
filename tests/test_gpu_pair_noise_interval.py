"""Pair-correlated random force by the Chebyshev form on an interval of the
pair matrix's spectrum (needs a GPU): the workloads' full-strength pair
kernel, which the Gershgorin bound refuses, against the FP64 oracle's dense
square roots of the transformed correlation matrices (Sec. II C); the
interval estimated by the device's Lanczos run against the dense
eigenvalues; the check at every noise block; a self-difference term; the
zero kernel; bit-identical graph forms; release and arguments."""
import numpy as np
import pytest

import oracle
from gld_cases import rel_l2
from oracle import pairnoise

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _workload(n=128, seed=31):
    from paper_1808_00270_gb300 import inputs
    return inputs.Workload(f"pairnoise_n{n}", n=n, box=inputs.box_for_density(n, 0.1), m_max=200, dt=0.005,
                           r_c=2.0, tau_s=0.5, tau_p=0.3, steps=1, seed=seed, nr=129)


def _kernels(w, strength=1.0):
    from paper_1808_00270_gb300 import inputs
    g, f, dr = inputs.pair_kernel_tables(w)
    return inputs.self_kernel_samples(w), g, strength * f, dr


def _common(w):
    return dict(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c, A_cons=w.A_cons,
                seed=w.seed)


def _pair(w, strength=1.0, self_diff=False, **gkw):
    from paper_1808_00270_gb300 import GLD, inputs
    pos, vel = inputs.initial_state(w)
    ks, g, f, dr = _kernels(w, strength)
    gpu = GLD(pos=pos, vel=vel, **_common(w), **gkw)
    if self_diff:
        gpu.set_kernels(ks, g=g, f=f, dr=dr, gs=0.5 * g, fs=0.3 * f)
    else:
        gpu.set_kernels(ks, g=g, f=f, dr=dr)
    return gpu


def _oracle_from(w, gpu, strength=1.0, self_diff=False):
    from paper_1808_00270_gb300 import ARR_FC, ARR_HIST
    pos, vel = gpu.get_state()
    s = oracle.System(pos=pos, vel=vel, **_common(w))
    ks, g, f, dr = _kernels(w, strength)
    kw = dict(gs=0.5 * g, fs=0.3 * f) if self_diff else {}
    assert s.set_kernels(ks, g=g, f=f, dr=dr, **kw) == 0
    s.set_state(step=gpu.step_index, pos=pos, vel=vel, fc=gpu.get(ARR_FC), hist=gpu.get(ARR_HIST))
    return s


def _pair_matrix_eigenvalues(w, gpu, strength=1.0, self_diff=False):
    """Eigenvalues of the dense pair matrix (plus the self-difference blocks
    scaled by their time factor's ratio 0.5) at the context's positions."""
    ks, g, f, dr = _kernels(w, strength)
    pos = gpu.get_state()[0]
    kw = dict(gs=0.5 * g, fs=0.3 * f) if self_diff else {}
    terms = pairnoise.matrix_terms(pos, w.box, w.r_c, 0.0, w.m_max, w.dt, ks, g, f, dr, **kw)
    M = terms[1][1] + (0.5 * terms[2][1] if self_diff else 0.0)
    return np.linalg.eigvalsh(M)


@pytest.mark.parametrize("warm", [0, 81])
def test_interval_admits_the_full_strength_kernel(warm):
    """The unscaled pair kernel f = 2 (1 - r/r_c)^2 is refused on the
    Gershgorin bound; on the estimated interval (Ritz extremes within 1 % of
    the dense extremes, widened by 25 % of the spread) one step's F^R is within
    four times the reported interpolation error (1.4e-4 at degree 12 here; 2e-6
    at least) of the oracle's dense square roots, at the start of a noise block
    and inside one."""
    from paper_1808_00270_gb300 import ARR_FR, GLDError
    from paper_1808_00270_gb300.binding import E_NOT_PSD
    w = _workload()
    with pytest.raises(GLDError) as e:
        _pair(w).set_pair_noise(12)
    assert e.value.status == E_NOT_PSD
    gpu = _pair(w)
    ev = _pair_matrix_eigenvalues(w, gpu)
    lo, hi, err = gpu.set_pair_noise_on(12)
    sp = gpu.pair_noise_spectrum()
    spread = ev[-1] - ev[0]
    print(f"dense spectrum [{ev[0]:.4f}, {ev[-1]:.4f}], Ritz [{sp['ritz_min']:.4f}, {sp['ritz_max']:.4f}] "
          f"(Krylov dimension {sp['krylov_dim']}), interval [{lo:.4f}, {hi:.4f}], interpolation {err:.1e}")
    assert abs(sp["ritz_min"] - ev[0]) < 0.01 * spread and abs(sp["ritz_max"] - ev[-1]) < 0.01 * spread
    assert lo < ev[0] and hi > ev[-1] and (sp["lo"], sp["hi"]) == (lo, hi)
    assert ev[0] - lo < 0.27 * spread and hi - ev[-1] < 0.27 * spread
    gpu.step(warm)
    ref = _oracle_from(w, gpu)
    want = ref.pair_random_force()
    gpu.step(1)
    e = rel_l2(gpu.get(ARR_FR), want)
    print(f"full-strength pair noise after {warm} steps: F^R {e:.2e}")
    assert e < max(2e-6, 4 * err), (e, err)


def test_interval_step_matches_oracle():
    """The whole step (F^R, F^D, V) within 1e-5 of the oracle stepping with
    its dense pair noise."""
    from paper_1808_00270_gb300 import ARR_FD, ARR_FR
    w = _workload(seed=32)
    gpu = _pair(w)
    _, _, err = gpu.set_pair_noise_on(14)
    assert err < 2e-6, err
    gpu.step(23)
    ref = _oracle_from(w, gpu)
    gpu.step(1)
    ref.step_pair_noise(1)
    assert rel_l2(gpu.get(ARR_FR), ref.get(oracle.FR)) < 1e-5
    assert rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD)) < 1e-5
    assert rel_l2(gpu.get_state()[1], ref.get(oracle.VEL)) < 1e-5


def test_interval_with_self_difference_term():
    """A self-difference term 0.3 f(r) x 0.5 g(t) joins M on its diagonal
    blocks; the Lanczos run sees it (Ritz extremes against the dense
    spectrum of M_pair + 0.5 D_self) and F^R is within 2e-6 of the oracle."""
    from paper_1808_00270_gb300 import ARR_FR
    w = _workload(seed=36)
    gpu = _pair(w, self_diff=True)
    ev = _pair_matrix_eigenvalues(w, gpu, self_diff=True)
    lo, hi, err = gpu.set_pair_noise_on(12)
    sp = gpu.pair_noise_spectrum()
    assert abs(sp["ritz_min"] - ev[0]) < 0.01 * (ev[-1] - ev[0])
    assert abs(sp["ritz_max"] - ev[-1]) < 0.01 * (ev[-1] - ev[0])
    gpu.step(45)
    ref = _oracle_from(w, gpu, self_diff=True)
    want = ref.pair_random_force()
    gpu.step(1)
    e = rel_l2(gpu.get(ARR_FR), want)
    print(f"self-difference term: interval [{lo:.3f}, {hi:.3f}], F^R {e:.2e}")
    assert e < max(2e-6, 4 * err)


def test_interval_check_latches_when_the_spectrum_leaves():
    """A given interval that misses part of the spectrum (its lower end above
    the smallest eigenvalue, or its upper end below the largest) passes the
    host's test of positive semi-definiteness but not the Lanczos check at
    the first noise block: GLD_E_NOT_PSD, sticky."""
    from paper_1808_00270_gb300 import GLDError
    from paper_1808_00270_gb300.binding import E_NOT_PSD
    w = _workload(seed=38)
    for side in ("low", "high"):
        gpu = _pair(w)
        ev = _pair_matrix_eigenvalues(w, gpu)
        lo, hi = (0.5 * ev[0], 1.1 * ev[-1]) if side == "low" else (1.1 * ev[0], 0.5 * ev[-1])
        assert gpu.set_pair_noise_on(6, lo=lo, hi=hi)[:2] == (lo, hi)
        with pytest.raises(GLDError) as e:
            gpu.step(1)
            gpu.sync()
        assert e.value.status == E_NOT_PSD
        with pytest.raises(GLDError) as e:
            gpu.step(1)
        assert e.value.status == E_NOT_PSD


def test_interval_zero_kernel_gives_the_self_noise():
    from paper_1808_00270_gb300 import ARR_FR
    w = _workload(seed=33)
    a, b = _pair(w, strength=0.0), _pair(w, strength=0.0)
    lo, hi, _ = b.set_pair_noise_on(8)
    assert lo < 0 < hi and hi - lo < 1e-9
    a.step(70)
    b.step(70)
    assert rel_l2(b.get(ARR_FR), a.get(ARR_FR)) < 1e-6


def test_interval_graph_forms_bit_identical():
    """Eager steps, the gated graph and the conditional graph (each noise
    block's Lanczos check captured with it) give the same bits over two
    blocks."""
    from paper_1808_00270_gb300 import ARR_FR
    w = _workload(seed=34)
    outs = []
    for ug in (0, 1, 2):
        g = _pair(w, use_graphs=ug)
        g.set_pair_noise_on(6)
        g.step(128)
        outs.append((g.get_state()[0], g.get(ARR_FR), g.pair_noise_spectrum()))
    for p, fr, sp in outs[1:]:
        assert np.array_equal(p, outs[0][0]) and np.array_equal(fr, outs[0][1]) and sp == outs[0][2]


def test_interval_release_and_arguments():
    from paper_1808_00270_gb300 import Batch, GLDError
    from paper_1808_00270_gb300.binding import E_INVAL, E_STATE
    w = _workload(seed=37)
    g = _pair(w)
    b0 = g.bytes()
    with pytest.raises(GLDError) as e:
        g.pair_noise_spectrum()
    assert e.value.status == E_STATE
    for deg in (-1, 17):
        with pytest.raises(GLDError) as e:
            g.set_pair_noise_on(deg)
        assert e.value.status == E_INVAL
    g.set_pair_noise_on(8)
    assert g.bytes() > b0
    with pytest.raises(GLDError):
        Batch().add(g)
    g.set_pair_noise(0)  # either setter turns the other form off
    assert g.bytes() == b0
    with pytest.raises(GLDError) as e:
        g.pair_noise_spectrum()
    assert e.value.status == E_STATE
    g.set_pair_noise_on(8)
    ks, gg, f, dr = _kernels(w)
    g.set_kernels(ks, g=gg, f=f, dr=dr)  # new kernels release it too
    assert g.bytes() == b0
    Batch().add(g)
