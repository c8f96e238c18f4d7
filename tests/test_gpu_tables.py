"""Tabulated model inputs on the device (needs a GPU): a conservative force
given as a table of -dU/dr (the form iterative Boltzmann inversion gives,
Sec. III) and a general pair-kernel table K^p(r, t) reduced to separable
terms, each against the FP64 oracle evaluating the table directly."""
import numpy as np
import pytest

import oracle
from gld_cases import make_gpu, oracle_from_gpu, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _w():
    from paper_1808_00270_gb300 import inputs
    return inputs.WORKLOADS["gld_n4096_m200"]


def _force_table(rc, nr=129):
    """Repulsive core plus an attractive well, zero at r_c."""
    dr = rc / (nr - 1)
    r = np.arange(nr) * dr
    x = np.clip(1 - r / rc, 0, None)
    return 30 * x ** 3 - 8 * np.sin(2.5 * r) * x, dr


def _kernel_table(w, nr=33):
    """exp(-t / tau(r)) with tau from 0.2 to 0.3 over [0, r_c]: not separable."""
    dr = w.r_c / (nr - 1)
    r = np.arange(nr) * dr
    t = np.arange(w.m_max) * w.dt
    return 2 * (1 - r[:, None] / w.r_c) ** 2 * np.exp(-t[None, :] / (0.2 + 0.05 * r[:, None])), dr


def _step_errors(gpu, ref):
    from paper_1808_00270_gb300 import ARR_FC, ARR_FD, ARR_FR
    gpu.step(1)
    ref.step(1)
    return {"fc": rel_l2(gpu.get(ARR_FC), ref.get(oracle.FC)), "fd": rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD)),
            "fr": rel_l2(gpu.get(ARR_FR), ref.get(oracle.FR)),
            "vel": rel_l2(gpu.get_state()[1], ref.get(oracle.VEL))}


def test_force_table_matches_oracle_mid_run():
    """Switched from the soft repulsion to a tabulated force after 100 steps:
    F^C at once and the whole next step within 1e-5 of the oracle."""
    from paper_1808_00270_gb300 import ARR_FC
    w = _w()
    gpu = make_gpu(w)
    gpu.step(100)
    f, dr = _force_table(w.r_c)
    gpu.set_conservative_table(f, dr)
    ref = oracle_from_gpu(w, gpu)
    assert ref.set_fc_table(f, dr) == 0
    assert rel_l2(gpu.get(ARR_FC), ref.get(oracle.FC)) < 1e-5
    errs = _step_errors(gpu, ref)
    assert max(errs.values()) < 1e-5, errs


def test_force_table_of_the_soft_repulsion_gives_its_trajectory():
    """The table of the soft repulsion's own force (linear in r, so exact under
    linear interpolation) integrates the same trajectory; nr = 0 restores
    the analytic form."""
    from paper_1808_00270_gb300 import ARR_FC, ARR_DISP
    w = _w()
    a, b = make_gpu(w), make_gpu(w)
    nr = 65
    dr = w.r_c / (nr - 1)
    r = np.arange(nr) * dr
    b.set_conservative_table(2 * w.A_cons / w.r_c * (1 - r / w.r_c), dr)
    a.step(128)
    b.step(128)
    assert rel_l2(b.get(ARR_DISP), a.get(ARR_DISP)) < 1e-5
    b.set_conservative_table(None)
    assert rel_l2(b.get(ARR_FC), a.get(ARR_FC)) < 1e-5


def test_rank_two_kernel_table_is_exact():
    """A table that is a sum of two separable terms: the rank-2 separation
    loses nothing and the step matches the oracle evaluating the table."""
    from paper_1808_00270_gb300 import inputs
    w = _w()
    g, f, dr = inputs.pair_kernel_tables(w)
    r = np.arange(f.shape[1]) * dr
    t = np.arange(w.m_max) * w.dt
    Kp = np.outer(f[0], g[0]) + np.outer((1 - r / w.r_c) * np.sin(3 * r), np.exp(-t / 0.1) * np.cos(t / 0.05))
    gpu = make_gpu(w, pair=False)
    tr = gpu.set_kernels_table(inputs.self_kernel_samples(w), Kp, dr, Q=2)
    assert tr < 1e-6
    gpu.step(150)
    ref = oracle_from_gpu(w, gpu, pair=False)
    assert ref.set_pair_table(Kp, dr) == 0
    errs = _step_errors(gpu, ref)
    assert max(errs.values()) < 1e-5, errs


def test_non_separable_kernel_table_rank_four():
    """exp(-t / tau(r)): the device runs the rank-4 separation, matching the
    oracle given that rank-4 table to 1e-5; against the full table the F^D
    error stays at the reported truncation level."""
    from paper_1808_00270_gb300 import ARR_FD, inputs
    from paper_1808_00270_gb300.binding import separable_terms
    w = _w()
    Kp, dr = _kernel_table(w)
    f4, g4, tr_host = separable_terms(Kp, 4)
    gpu = make_gpu(w, pair=False)
    tr = gpu.set_kernels_table(inputs.self_kernel_samples(w), Kp, dr, Q=4)
    assert abs(tr - tr_host) < 1e-12 and tr < 1e-4
    gpu.step(150)
    ref4 = oracle_from_gpu(w, gpu, pair=False)
    assert ref4.set_pair_table(f4.T @ g4, dr) == 0
    full = oracle_from_gpu(w, gpu, pair=False)
    assert full.set_pair_table(Kp, dr) == 0
    full.step(1)
    errs = _step_errors(gpu, ref4)
    assert max(errs.values()) < 1e-5, errs
    e_full = rel_l2(gpu.get(ARR_FD), full.get(oracle.FD))
    print(f"rank-4 truncation {tr:.2e}; F^D against the full table {e_full:.2e}")
    assert e_full < 1e-5 + 10 * tr


def test_tables_in_a_batch():
    """A member with a tabulated force and a rank-2 kernel table steps in a
    batch exactly as alone (to FP32 rounding of the convolution order)."""
    from paper_1808_00270_gb300 import ARR_DISP, Batch, inputs
    w = _w()
    Kp, dr_k = _kernel_table(w)
    f, dr = _force_table(w.r_c)
    ks = inputs.self_kernel_samples(w)
    a, b = make_gpu(w, pair=False), make_gpu(w, pair=False)
    for s in (a, b):
        s.set_conservative_table(f, dr)
        s.set_kernels_table(ks, Kp, dr_k, Q=2)
    bt = Batch()
    bt.add(b)
    bt.step(128)
    bt.sync()
    a.step(128)
    assert rel_l2(b.get(ARR_DISP), a.get(ARR_DISP)) < 1e-5
    assert rel_l2(b.get_state()[1], a.get_state()[1]) < 1e-4


def test_table_arguments_rejected():
    from paper_1808_00270_gb300 import GLDError, inputs
    from paper_1808_00270_gb300.binding import E_INVAL
    w = _w()
    g = make_gpu(w)
    for f, dr in ((np.ones(1), 0.1), (np.ones(8), 0.0)):
        with pytest.raises(GLDError) as e:
            g.set_conservative_table(f, dr)
        assert e.value.status == E_INVAL
    Kp, dr = _kernel_table(w)
    for Q in (0, 5):
        with pytest.raises(GLDError):
            g.set_kernels_table(inputs.self_kernel_samples(w), Kp, dr, Q=Q)
