"""Pair-correlated random force of Sec. II C (TEST INFRASTRUCTURE).

Part of the FP64 oracle: only the test-suite, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import it.  It evaluates, for one time step n,
the quantity that Algorithm 1 approximates with a Lanczos iteration per
frequency, by its plain definition with dense matrices:

  * the 3N x 3N correlation matrices K_m of Eq. correlation_matrix, built from
    the right-hand side of Eq. stochastic_force2 under the time-scale
    separation remarked on after Algorithm 1 (all kernels at the current
    configuration R_n):  K_m = kT a_m / dt * ( K^s_m 1
        + blocks (i, j != i): K^p_m(R_ij)
        + blocks (i, i):      sum_k dK^s_m(R_ik) ),
    each pair tensor K(R) = K_par(R) e e^T + K_perp(R) (1 - e e^T) (Sec. II A),
    a_0 = 2, a_m = 1 (Eq. FDT_discretized);
  * their transform over the 2 m_max - 1 points of Eq. FT,
    hat K_w = K_0 + 2 sum_{m>=1} K_m cos(2 pi w m / (2 m_max - 1));
  * hat F_w = sqrt(hat K_w) hat W_w with the symmetric square root taken from
    an eigen-decomposition (the result the Lanczos iteration converges to);
  * F_n = inverse transform at time 0, scaled by 1 / (2 m_max - 1) (the same
    reading as for the self-kernel noise; Algorithm 1 prints 1/m_max).

Because K_{-m} = K_m, hat K_{-w} = hat K_w and hat W_{-w} = conj(hat W_w), so
F_n = (hat K_0^{1/2} hat W_0 + 2 sum_{w>=1} hat K_w^{1/2} Re hat W_w) / (2 m_max - 1)
with Re hat W_w = sum_m W_{n+m} cos(2 pi w m / (2 m_max - 1)).

Radial factors use max(r, r_c,min) and linear interpolation on r = k dr with
the last value held (as the dissipative force of the oracle); pairs are those
with r < r_c.

With the window of the remark after Algorithm 1 (``random_force_window``),
one window W_{n-H} .. W_{n+H} gives F at the times n .. n + rows - 1 through
the whole inverse transform of hat F_w (its sine part too).

Deliberate mistakes for the pin test (``variant``): 11 the sign of the pair
blocks flipped; 12 the inverse transform scaled by 1 / m_max; 17 the radial
factors read at the unclamped distance (r_c,min ignored); 18 the sine part of
the window's inverse transform with the wrong sign.
"""
from __future__ import annotations

import numpy as np


def discretize(samples, dt: float, discrete: bool) -> np.ndarray:
    """K_m from continuous samples K(m dt): K_0 = dt K(0)/2, K_m = dt K(m dt)
    (Eq. k-discrete with trapezoid weights), or the weights themselves."""
    s = np.asarray(samples, dtype=float)
    if discrete:
        return s.copy()
    out = dt * s
    out[..., 0] *= 0.5
    return out


def radial(table, dr: float, r):
    """Linear interpolation on r = k dr, constant past the last entry."""
    t = np.asarray(table, dtype=float)
    return np.interp(np.asarray(r, dtype=float), np.arange(t.size) * dr, t)


def pair_geometry(pos, box: float, rc: float):
    """(i, j, r, e) for all unordered pairs i < j with minimum-image distance
    r < rc; e = (R_i - R_j) / r."""
    pos = np.asarray(pos, dtype=float)
    d = pos[:, None, :] - pos[None, :, :]
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(-1))
    i, j = np.nonzero(np.triu(r < rc, k=1))
    return i, j, r[i, j], d[i, j] / r[i, j][:, None]


def matrix_terms(pos, box, rc, rc_min, m_max, dt, Ks, g=None, f=None, dr=1.0, gs=None, fs=None,
                 discrete=False, variant=0, fp=None, fsp=None):
    """The memory kernel as a list of (time weights w[m], 3N x 3N matrix X),
    K_m = sum w[m] X (before the factor kT a_m / dt).  Each pair block is
    f(r) e e^T + fp(r) (1 - e e^T) (perpendicular factors fp, fsp: None = 0)."""
    n = np.asarray(pos).shape[0]
    terms = [(discretize(Ks, dt, discrete), np.eye(3 * n))]
    i, j, r, e = pair_geometry(pos, box, rc)
    rt = r if variant == 17 else np.maximum(r, rc_min)
    ee = e[:, :, None] * e[:, None, :]
    perp = np.eye(3)[None] - ee
    g = np.zeros((0, m_max)) if g is None else np.reshape(g, (-1, m_max))
    f = np.zeros((0, 2)) if f is None or g.shape[0] == 0 else np.reshape(f, (g.shape[0], -1))
    fp = np.zeros_like(f) if fp is None else np.reshape(fp, f.shape)
    for gq, fq, fpq in zip(g, f, fp):
        X = np.zeros((n, 3, n, 3))
        w = radial(fq, dr, rt)[:, None, None] * ee + radial(fpq, dr, rt)[:, None, None] * perp
        if variant == 11:
            w = -w
        X[i, :, j, :] = w
        X[j, :, i, :] = w
        terms.append((discretize(gq, dt, discrete), X.reshape(3 * n, 3 * n)))
    if gs is not None and fs is not None and np.size(gs) > 0:
        gs = np.reshape(gs, (-1, m_max))
        fs = np.reshape(fs, (gs.shape[0], -1))
        fsp = np.zeros_like(fs) if fsp is None else np.reshape(fsp, fs.shape)
        for gq, fq, fpq in zip(gs, fs, fsp):
            X = np.zeros((n, 3, n, 3))
            w = radial(fq, dr, rt)[:, None, None] * ee + radial(fpq, dr, rt)[:, None, None] * perp
            np.add.at(X, (i, slice(None), i, slice(None)), w)
            np.add.at(X, (j, slice(None), j, slice(None)), w)
            terms.append((discretize(gq, dt, discrete), X.reshape(3 * n, 3 * n)))
    return terms


def correlation_matrix(terms, kT: float, dt: float, m: int) -> np.ndarray:
    """K_m of Eq. correlation_matrix: kT a_m / dt * sum_terms w[m] X."""
    a = 2.0 if m == 0 else 1.0
    return kT * a / dt * sum(w[abs(m)] * X for w, X in terms)


def transformed(terms, kT: float, dt: float, m_max: int, w: int) -> np.ndarray:
    """hat K_w = K_0 + 2 sum_{m>=1} K_m cos(2 pi w m / L), L = 2 m_max - 1
    (Eq. FT), each term's scalar transform times its matrix."""
    L = 2 * m_max - 1
    c = np.cos(2.0 * np.pi * ((w * np.arange(1, m_max)) % L) / L)
    return sum(kT / dt * (2.0 * wt[0] + 2.0 * (wt[1:m_max] * c).sum()) * X for wt, X in terms)


def sqrt_psd(Kh: np.ndarray, clamp: bool = False):
    """Symmetric square root; returns (root, most negative eigenvalue / max |eig|)."""
    lam, U = np.linalg.eigh(0.5 * (Kh + Kh.T))
    scale = max(np.abs(lam).max(), 1e-300)
    worst = lam.min() / scale
    if worst < -1e-12 and not clamp:
        raise ValueError(f"correlation matrix not positive semi-definite (eigenvalue {worst:.3e} of max)")
    return (U * np.sqrt(np.clip(lam, 0.0, None))) @ U.T, worst


def random_force_window(terms, kT: float, dt: float, m_max: int, Wwin, rows: int, clamp: bool = False,
                        variant: int = 0):
    """F_{n+m} [rows, N, 3] for m = 0 .. rows - 1 from ONE window
    Wwin[s + m_max - 1] = W_{n+s}: the time window of the remark after
    Algorithm 1 (kernels held at R_n).  hat F_w = sqrt(hat K_w) hat W_w with
    the complex transform hat W_w = sum_s W_{n+s} exp(-2 pi i w s / L) =
    C_w - i S_w, and the whole inverse transform at the first `rows` times,
    F_{n+m} = (1/L) sum_{w=-(m_max-1)}^{m_max-1} hat F_w exp(2 pi i w m / L)
            = (X^c_0 + 2 sum_{w>=1} (X^c_w cos(2 pi w m / L) + X^s_w sin(2 pi w m / L))) / L,
    X^c_w = sqrt(hat K_w) C_w, X^s_w = sqrt(hat K_w) S_w (hat K_{-w} = hat K_w
    is real).  Row 0 is random_force's F_n.  variant 18 flips the sign of the
    sine part (a time-reversed window)."""
    L = 2 * m_max - 1
    Wwin = np.asarray(Wwin, dtype=float)
    n = Wwin.shape[1]
    shifts = np.arange(-(m_max - 1), m_max)
    m = np.arange(rows)
    F = np.zeros((rows, 3 * n))
    for w in range(m_max):
        ph = 2.0 * np.pi * ((w * shifts) % L) / L
        C = np.tensordot(np.cos(ph), Wwin, axes=1).reshape(3 * n)
        S = np.tensordot(np.sin(ph), Wwin, axes=1).reshape(3 * n)
        R, _ = sqrt_psd(transformed(terms, kT, dt, m_max, w), clamp)
        th = 2.0 * np.pi * ((w * m) % L) / L
        sgn = -1.0 if variant == 18 else 1.0
        F += (1.0 if w == 0 else 2.0) * (np.outer(np.cos(th), R @ C) + sgn * np.outer(np.sin(th), R @ S))
    return (F / L).reshape(rows, n, 3)


def random_force(terms, kT: float, dt: float, m_max: int, Wwin, clamp: bool = False, variant: int = 0):
    """F_n [N, 3] from the window Wwin[s + m_max - 1] = W_{n+s} [N, 3]."""
    L = 2 * m_max - 1
    Wwin = np.asarray(Wwin, dtype=float)
    n = Wwin.shape[1]
    shifts = np.arange(-(m_max - 1), m_max)
    F = np.zeros(3 * n)
    for w in range(m_max):
        ReW = np.tensordot(np.cos(2.0 * np.pi * ((w * shifts) % L) / L), Wwin, axes=1).reshape(3 * n)
        S, _ = sqrt_psd(transformed(terms, kT, dt, m_max, w), clamp)
        F += (1.0 if w == 0 else 2.0) * (S @ ReW)
    return (F / (m_max if variant == 12 else L)).reshape(n, 3)
