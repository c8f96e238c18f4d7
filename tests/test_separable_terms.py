"""Host-side separation of a general pair-kernel table into separable terms
(no device needed): against singular values and vectors fixed by
construction, on both table shapes."""
import numpy as np
import pytest

from paper_1808_00270_gb300.binding import GLDError, separable_terms


def _known(nr, m, sig, seed=3):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.normal(size=(nr, len(sig))))
    V, _ = np.linalg.qr(rng.normal(size=(m, len(sig))))
    return U @ np.diag(sig) @ V.T


@pytest.mark.parametrize("nr,m", [(40, 200), (300, 60)])
def test_truncation_of_a_known_spectrum(nr, m):
    """Singular values 1, 0.5, 0.1, 1e-3, 1e-5: the rank-Q part is the
    leading Q terms, the reported remainder is sqrt(sum_{q>Q} s^2 / sum s^2)
    and equals the actual Frobenius error; the full rank reproduces the table."""
    sig = np.array([1.0, 0.5, 0.1, 1e-3, 1e-5])
    T = _known(nr, m, sig)
    for Q in (1, 2, 3, 4, 5):
        f, g, tr = separable_terms(T, Q)
        want = np.sqrt((sig[Q:] ** 2).sum() / (sig ** 2).sum())
        err = np.linalg.norm(T - f.T @ g) / np.linalg.norm(T)
        assert abs(err - want) <= 1e-9 + 1e-6 * want, (Q, err, want)
        assert abs(tr - want) <= 1e-7 + 1e-6 * want, (Q, tr, want)
        # the terms are the singular triplets: g rows orthonormal or f rows orthonormal
        gn, fn = np.linalg.norm(g, axis=1), np.linalg.norm(f, axis=1)
        assert np.allclose(np.sort(gn * fn)[::-1], sig[:Q], rtol=1e-6)


def test_rank_one_and_non_separable_kernels():
    """f(r) g(t) separates exactly with one term; exp(-t / tau(r)) with
    tau from 0.2 to 0.4 needs several, with the remainder falling with Q."""
    r = np.linspace(0, 2, 33)
    t = np.arange(200) * 0.005
    T1 = np.outer(2 * (1 - r / 2) ** 2, np.exp(-t / 0.3))
    f, g, tr = separable_terms(T1, 1)
    assert np.abs(f.T @ g - T1).max() < 1e-12 * np.abs(T1).max() and tr < 1e-6
    T = 2 * (1 - r[:, None] / 2) ** 2 * np.exp(-t[None, :] / (0.2 + 0.1 * r[:, None]))
    trs = [separable_terms(T, Q)[2] for Q in (1, 2, 3, 4)]
    s = np.linalg.svd(T, compute_uv=False)
    for Q, tr in zip((1, 2, 3, 4), trs):
        assert abs(tr - np.sqrt((s[Q:] ** 2).sum() / (s ** 2).sum())) < 1e-7
    assert trs == sorted(trs, reverse=True) and trs[3] < 1e-3


def test_invalid_rank():
    T = np.ones((4, 3))
    for Q in (0, 4):
        with pytest.raises(GLDError):
            separable_terms(T, Q)
