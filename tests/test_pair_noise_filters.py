"""Host-side construction of the pair-noise filters (no device needed): with
the taps of gld_pair_noise_filters, F_n = sum_k T_k(M / lambda) Z_k evaluated
in FP64 with the dense pair matrix equals the oracle's dense square roots of
the transformed correlation matrices (Sec. II C) to the reported
interpolation error, which falls with the degree."""
import numpy as np
import pytest

from oracle import pairnoise
from paper_1808_00270_gb300.binding import E_INVAL, E_NOT_PSD, GLDError, pair_noise_filters


def _case(seed=5, n=18, M=24, dt=0.02, kT=0.8):
    rng = np.random.default_rng(seed)
    box, rc = 5.0, 2.0
    pos = rng.uniform(0, box, (n, 3))
    t = np.arange(M) * dt
    Ks = 10.0 * np.exp(-t / 0.2)
    g = np.exp(-t / 0.3)[None]
    r = np.linspace(0, rc, 33)
    f = (0.6 * (1 - r / rc) ** 2)[None]
    terms = pairnoise.matrix_terms(pos, box, rc, 0.0, M, dt, Ks, g, f, r[1])
    W = rng.normal(size=(2 * M - 1, n, 3))
    want = pairnoise.random_force(terms, kT, dt, M, W)
    Mm = terms[1][1]
    blocks = np.abs(Mm).reshape(n, 3, n, 3).max(axis=(1, 3))  # |f| per pair (rank-one blocks)
    lam = 1.25 * blocks.sum(axis=1).max()
    return dict(Kd=pairnoise.discretize(Ks, dt, False), gd=pairnoise.discretize(g[0], dt, False), kT=kT, dt=dt,
                M=Mm, lam=lam, W=W, want=want)


def _chebyshev_force(c, taps):
    n3 = c["M"].shape[0]
    Z = [np.tensordot(tk, c["W"], axes=1).reshape(n3) for tk in taps]
    Mt = c["M"] / c["lam"]
    b1, b2 = np.zeros(n3), np.zeros(n3)
    for k in range(len(Z) - 1, 0, -1):
        b1, b2 = Z[k] + 2 * Mt @ b1 - b2, b1
    return (Z[0] + Mt @ b1 - b2).reshape(-1, 3)


def test_filters_reproduce_the_dense_square_roots():
    c = _case()
    prev = np.inf
    for K in (2, 4, 8, 12):
        taps, err = pair_noise_filters(c["Kd"], c["gd"], c["kT"], c["dt"], c["lam"], K)
        got = _chebyshev_force(c, taps)
        e = np.linalg.norm(got - c["want"]) / np.linalg.norm(c["want"])
        assert e <= 4 * err + 1e-12, (K, e, err)
        assert err < prev or err < 1e-13, (K, err, prev)  # falls until rounding
        prev = err
    assert e < 1e-9


def test_degree_zero_part_is_the_self_noise_filter():
    """lambda -> 0: T_0 carries everything and its taps are the self-kernel
    moving average A_s (the inverse transform of sqrt(hat C), 1/(2 m_max - 1))."""
    c = _case(seed=6)
    taps, _ = pair_noise_filters(c["Kd"], c["gd"], c["kT"], c["dt"], 1e-9, 4)
    import oracle
    st, _, _, A, _ = oracle.noise_coefs(c["Kd"], c["kT"], c["dt"])
    assert st == 0
    assert np.abs(taps[0] - A).max() < 1e-9 * np.abs(A).max()
    assert np.abs(taps[1:]).max() < 1e-6 * np.abs(A).max()


def test_filter_arguments():
    c = _case()
    with pytest.raises(GLDError) as e:
        pair_noise_filters(c["Kd"], c["gd"], c["kT"], c["dt"], 1e4, 8)
    assert e.value.status == E_NOT_PSD
    pair_noise_filters(c["Kd"], c["gd"], c["kT"], c["dt"], 1e4, 8, psd_clamp=True)
    for K, lam in ((0, 1.0), (17, 1.0), (8, 0.0)):
        with pytest.raises(GLDError) as e:
            pair_noise_filters(c["Kd"], c["gd"], c["kT"], c["dt"], lam, K)
        assert e.value.status == E_INVAL


def _dense_case(amp, seed=5, n=40, box=4.0, M=24, dt=0.02, kT=0.8):
    """40 particles in a box of 4 (about 10 neighbours within r_c = 2), pair
    kernel amp (1 - r/r_c)^2 exp(-t/0.3): an asymmetric pair-matrix spectrum."""
    rng = np.random.default_rng(seed)
    rc = 2.0
    pos = rng.uniform(0, box, (n, 3))
    t = np.arange(M) * dt
    Ks = 10.0 * np.exp(-t / 0.2)
    g = np.exp(-t / 0.3)[None]
    r = np.linspace(0, rc, 33)
    f = (amp * (1 - r / rc) ** 2)[None]
    terms = pairnoise.matrix_terms(pos, box, rc, 0.0, M, dt, Ks, g, f, r[1])
    W = rng.normal(size=(2 * M - 1, n, 3))
    want = pairnoise.random_force(terms, kT, dt, M, W)
    return dict(Kd=pairnoise.discretize(Ks, dt, False), gd=pairnoise.discretize(g[0], dt, False), kT=kT, dt=dt,
                M=terms[1][1], W=W, want=want)


def _chebyshev_force_on(c, taps, lo, hi):
    """Clenshaw's recurrence for sum_k T_k((M - cen) / rad) Z_k in FP64."""
    n3 = c["M"].shape[0]
    cen, rad = 0.5 * (lo + hi), 0.5 * (hi - lo)
    Z = [np.tensordot(tk, c["W"], axes=1).reshape(n3) for tk in taps]
    Mt = (c["M"] - cen * np.eye(n3)) / rad
    b1, b2 = np.zeros(n3), np.zeros(n3)
    for k in range(len(Z) - 1, 0, -1):
        b1, b2 = Z[k] + 2 * Mt @ b1 - b2, b1
    return (Z[0] + Mt @ b1 - b2).reshape(-1, 3)


def test_interval_filters_reproduce_the_dense_square_roots():
    """On the interval of the actual spectrum (widened by 5 % of its spread)
    the form reproduces the oracle's dense square roots to the reported error,
    for a pair kernel whose symmetric bound (1.25 x the spectral radius) the
    positive semi-definiteness test refuses: h_w + g_w mu >= 0 holds on the
    eigenvalues but not on [-1.25 rho, 1.25 rho]."""
    from paper_1808_00270_gb300.binding import pair_noise_filters_on
    c = _dense_case(5.9)
    ev = np.linalg.eigvalsh(c["M"])
    assert ev[-1] > 1.2 * -ev[0]  # asymmetric
    with pytest.raises(GLDError) as e:
        pair_noise_filters(c["Kd"], c["gd"], c["kT"], c["dt"], 1.25 * np.abs(ev).max(), 8)
    assert e.value.status == E_NOT_PSD
    w = ev[-1] - ev[0]
    lo, hi = ev[0] - 0.05 * w, ev[-1] + 0.05 * w
    prev = np.inf
    for K in (4, 8, 12, 16):
        taps, err = pair_noise_filters_on(c["Kd"], c["gd"], c["kT"], c["dt"], lo, hi, K)
        got = _chebyshev_force_on(c, taps, lo, hi)
        e = np.linalg.norm(got - c["want"]) / np.linalg.norm(c["want"])
        assert e <= 4 * err + 1e-12, (K, e, err)
        assert err < prev, (K, err, prev)
        prev = err
    assert e < 1e-5, e


def test_symmetric_interval_is_the_lambda_form():
    from paper_1808_00270_gb300.binding import pair_noise_filters_on
    c = _case()
    a, ea = pair_noise_filters(c["Kd"], c["gd"], c["kT"], c["dt"], c["lam"], 8)
    b, eb = pair_noise_filters_on(c["Kd"], c["gd"], c["kT"], c["dt"], -c["lam"], c["lam"], 8)
    assert np.array_equal(a, b) and ea == eb


def test_interval_arguments():
    """The test of positive semi-definiteness takes both ends of the interval
    (h_w + g_w mu is linear in mu); an empty or non-finite interval is invalid."""
    from paper_1808_00270_gb300.binding import pair_noise_filters_on
    c = _dense_case(5.9)
    ev = np.linalg.eigvalsh(c["M"])
    pair_noise_filters_on(c["Kd"], c["gd"], c["kT"], c["dt"], ev[0], 10 * ev[-1], 8)  # far above: still fine
    with pytest.raises(GLDError) as e:
        pair_noise_filters_on(c["Kd"], c["gd"], c["kT"], c["dt"], 2 * ev[0], ev[-1], 8)  # far below: not PSD
    assert e.value.status == E_NOT_PSD
    pair_noise_filters_on(c["Kd"], c["gd"], c["kT"], c["dt"], 2 * ev[0], ev[-1], 8, psd_clamp=True)
    for lo, hi in ((1.0, 1.0), (2.0, 1.0), (np.nan, 1.0), (-np.inf, 1.0)):
        with pytest.raises(GLDError) as e:
            pair_noise_filters_on(c["Kd"], c["gd"], c["kT"], c["dt"], lo, hi, 8)
        assert e.value.status == E_INVAL
