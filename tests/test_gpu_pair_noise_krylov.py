"""Pair-correlated random force by Algorithm 1 of Sec. II C -- a Lanczos
iteration per frequency (needs a GPU) -- against the FP64 oracle, which takes
the square roots of the dense 3N x 3N transformed correlation matrices (the
result the iteration converges to): the workloads' unscaled pair kernel
(whose Gershgorin bound rules out the Chebyshev form), two pair terms, a
self-difference term with a time factor of its own together with
perpendicular factors and the lower cutoff r_c,min, the whole step, the
self-kernel limit, and the rejection of a kernel that is not positive
semi-definite."""
import numpy as np
import pytest

import oracle
from gld_cases import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL, KMAX = 1e-6, 40


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _workload(n=128, seed=31, r_c_min=0.0):
    from paper_1808_00270_gb300 import inputs
    return inputs.Workload(f"krylov_n{n}", n=n, box=inputs.box_for_density(n, 0.1), m_max=200, dt=0.005,
                           r_c=2.0, tau_s=0.5, tau_p=0.3, steps=1, seed=seed, nr=129, r_c_min=r_c_min)


def _kernels(w, form):
    """Kernel descriptions: 'unscaled' (the workloads' f g), 'two' (0.5 f g
    plus 0.3 (1 - r/r_c) exp(-t/0.1)), 'general' (0.5 f g, a self-difference
    term 0.4 f exp(-t/0.05) and perpendicular factors), 'self' (no pair
    term), 'bad' (an oscillating second pair term: not positive definite)."""
    from paper_1808_00270_gb300 import inputs
    g, f, dr = inputs.pair_kernel_tables(w)
    t = np.arange(w.m_max) * w.dt
    r = np.arange(f.shape[1]) * dr
    kw = dict(Ks=inputs.self_kernel_samples(w), dr=dr)
    perp = None
    if form == "unscaled":
        kw.update(g=g, f=f)
    elif form == "two":
        kw.update(g=np.vstack([g[0], np.exp(-t / 0.1)]), f=np.vstack([0.5 * f[0], 0.3 * np.clip(1 - r / w.r_c, 0, None)]))
    elif form == "general":
        kw.update(g=g, f=0.5 * f, gs=np.exp(-t / 0.05)[None], fs=0.4 * f)
        fp = (0.3 * np.clip(1 - r / w.r_c, 0, None) * (1 + np.cos(2 * r)))[None]
        perp = dict(fp=fp, fs=0.5 * fp)
    elif form == "bad":
        kw.update(g=np.vstack([g[0], np.exp(-t / 0.05) * np.cos(8 * t)]),
                  f=np.vstack([f[0], 0.8 * np.clip(1 - r / w.r_c, 0, None)]))
    return kw, perp


def _common(w):
    return dict(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c, r_c_min=w.r_c_min,
                A_cons=w.A_cons, seed=w.seed)


def _gpu(w, form, **gkw):
    from paper_1808_00270_gb300 import GLD, inputs
    pos, vel = inputs.initial_state(w)
    kw, perp = _kernels(w, form)
    s = GLD(pos=pos, vel=vel, **_common(w), **gkw)
    s.set_kernels(kw["Ks"], g=kw.get("g"), f=kw.get("f"), dr=kw["dr"], gs=kw.get("gs"), fs=kw.get("fs"))
    if perp is not None:
        s.set_perpendicular(perp["fp"], perp["fs"])
    return s


def _oracle_from(w, gpu, form):
    from paper_1808_00270_gb300 import ARR_FC, ARR_HIST
    pos, vel = gpu.get_state()
    kw, perp = _kernels(w, form)
    s = oracle.System(pos=pos, vel=vel, **_common(w))
    assert s.set_kernels(kw["Ks"], g=kw.get("g"), f=kw.get("f"), dr=kw["dr"], gs=kw.get("gs"), fs=kw.get("fs")) == 0
    if perp is not None:
        assert s.set_perp(perp["fp"], perp["fs"]) == 0
    s.set_state(step=gpu.step_index, pos=pos, vel=vel, fc=gpu.get(ARR_FC), hist=gpu.get(ARR_HIST))
    return s


@pytest.mark.parametrize("form,warm,rcmin", [("unscaled", 0, 0.0), ("unscaled", 81, 0.0), ("two", 37, 0.0),
                                             ("general", 50, 0.0), ("general", 50, 1.2)])
def test_krylov_pair_noise_matches_dense_square_roots(form, warm, rcmin):
    """One step's F^R within 1e-5 of the oracle's dense evaluation (the
    unscaled workload kernel, two pair terms, a self-difference term with
    its own time factor and perpendicular factors, with and without r_c,min)."""
    from paper_1808_00270_gb300 import ARR_FR
    w = _workload(r_c_min=rcmin)
    gpu = _gpu(w, form)
    gpu.set_pair_noise_krylov(TOL, KMAX)
    gpu.step(warm)
    ref = _oracle_from(w, gpu, form)
    want = ref.pair_random_force()
    gpu.step(1)
    e = rel_l2(gpu.get(ARR_FR), want)
    its = gpu.diag()["krylov_iterations"]
    print(f"{form} r_c,min {rcmin} after {warm} steps: F^R {e:.2e} in {its} Lanczos iterations")
    assert e < 1e-5 and 1 <= its <= KMAX
    gpu.close()


def test_krylov_pair_noise_step_matches_oracle():
    """The whole step with the Lanczos pair noise: F^R, F^D and V_{n+1}
    within 1e-5 of the oracle stepping with its dense pair noise."""
    from paper_1808_00270_gb300 import ARR_FD, ARR_FR
    w = _workload()
    gpu = _gpu(w, "two")
    gpu.set_pair_noise_krylov(TOL, KMAX)
    gpu.step(23)
    ref = _oracle_from(w, gpu, "two")
    gpu.step(1)
    ref.step_pair_noise(1)
    assert rel_l2(gpu.get(ARR_FR), ref.get(oracle.FR)) < 1e-5
    assert rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD)) < 1e-5
    assert rel_l2(gpu.get_state()[1], ref.get(oracle.VEL)) < 1e-5
    gpu.close()


def test_krylov_without_pair_terms_is_the_self_noise():
    """With no pair or self-difference term every hat K_w is a multiple of
    the identity: the iteration stops after one vector per frequency and
    gives the self-kernel moving average of Eq. noise_production."""
    from paper_1808_00270_gb300 import ARR_FR
    w = _workload()
    a = _gpu(w, "self")
    b = _gpu(w, "self")
    b.set_pair_noise_krylov(TOL, KMAX)
    a.step(70)
    b.step(70)
    e = rel_l2(b.get(ARR_FR), a.get(ARR_FR))
    assert e < 1e-5, e
    assert b.diag()["krylov_iterations"] <= 2


def test_krylov_rejects_a_kernel_that_is_not_positive_definite():
    from paper_1808_00270_gb300 import GLDError
    from paper_1808_00270_gb300.binding import E_NOT_PSD
    w = _workload()
    gpu = _gpu(w, "bad")
    gpu.set_pair_noise_krylov(TOL, KMAX)
    with pytest.raises(GLDError) as e:
        gpu.step(1)
    assert e.value.status == E_NOT_PSD


def test_krylov_arguments_and_exclusions():
    from paper_1808_00270_gb300 import Batch, GLDError
    from paper_1808_00270_gb300.binding import E_INVAL, E_STATE
    w = _workload()
    gpu = _gpu(w, "unscaled")
    for tol, kmax in ((1e-8, 1), (1e-8, 65), (2.0, 16)):
        with pytest.raises(GLDError) as e:
            gpu.set_pair_noise_krylov(tol, kmax)
        assert e.value.status == E_INVAL
    gpu.set_pair_noise_krylov(1e-8, 16)
    with pytest.raises(GLDError) as e:
        gpu.profile_steps(64)
    assert e.value.status == E_STATE
    b = Batch()
    with pytest.raises(GLDError) as e:
        b.add(gpu)
    assert e.value.status == E_INVAL
    gpu.set_pair_noise_krylov(0.0, 16)  # off: back to the self-kernel noise
    gpu.step(64)
    assert gpu.diag()["krylov_iterations"] == 0


@pytest.mark.parametrize("form", ["unscaled", "general"])
def test_krylov_window_matches_dense_square_roots(form):
    """The time window after Algorithm 1: at the start of a 64-step noise
    block one Lanczos run per frequency on the cosine and sine transforms of
    the window gives every row of the block; each step's F^R within 1e-5 of
    the oracle's window rows (dense square roots, kernels at the block's
    first configuration), for the unscaled workload kernel and for a
    self-difference term with perpendicular factors."""
    from paper_1808_00270_gb300 import ARR_FR
    w = _workload(seed=35)
    gpu = _gpu(w, form)
    gpu.set_pair_noise_lanczos(TOL, KMAX, window=1)
    gpu.step(64)
    ref = _oracle_from(w, gpu, form)
    want = ref.pair_random_force_window(64)
    worst = 0.0
    for m in range(64):
        gpu.step(1)
        worst = max(worst, rel_l2(gpu.get(ARR_FR), want[m]))
    its = gpu.diag()["krylov_iterations"]
    print(f"window, {form}: worst row F^R {worst:.2e}, Krylov dimension {its}")
    assert worst < 1e-5 and 1 <= its <= KMAX
    gpu.close()


def test_krylov_window_arguments():
    from paper_1808_00270_gb300 import GLDError
    from paper_1808_00270_gb300.binding import E_INVAL
    w = _workload()
    gpu = _gpu(w, "unscaled")
    with pytest.raises(GLDError) as e:
        gpu.set_pair_noise_lanczos(1e-6, 16, window=2)
    assert e.value.status == E_INVAL
    gpu.set_pair_noise_lanczos(1e-6, 16, window=1)
    gpu.step(3)  # a block started: its rows came from one run
    assert gpu.diag()["krylov_iterations"] >= 1
    gpu.set_pair_noise_lanczos(0.0, 16)  # off
    gpu.step(64)
    assert gpu.diag()["krylov_iterations"] == 0
