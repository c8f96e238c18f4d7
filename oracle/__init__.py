"""FP64 CPU oracle of the GLD time step (TEST INFRASTRUCTURE).

This package is the slow, plain reference that the CUDA path is checked
against.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
product path never does.  The arithmetic lives in ``gldref.c`` (plain C,
double precision, OpenMP over particles) and, for the pair-correlated noise
with its dense matrix square roots, in ``pairnoise.py`` (numpy); this module
compiles the C part and marshals arrays through ctypes.

Paper: Jung, Hanke & Schmid, arXiv:1808.00270.  Sections followed are listed
in the header of ``gldref.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gldref.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict = {}

POS, VEL, FC, FD, FR, DISP, HIST = range(7)
NOT_PSD = -3


def _lib_path(variant: int) -> str:
    return os.path.join(_BUILD, "libgldref.so" if variant == 0 else f"libgldref_plant{variant}.so")


def build(force: bool = False, variant: int = 0) -> str:
    """Compile gldref.c into a shared library (gcc, OpenMP when available).

    ``variant`` > 0 builds a deliberately wrong oracle (see OR_PLANT in
    gldref.c); only the test that checks the pins uses those."""
    path = _lib_path(variant)
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = f"{path}.{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", f"-DOR_PLANT={int(variant)}", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, path)
    return path


def lib(variant: int = 0):
    with _lock:
        if variant not in _libs:
            L = C.CDLL(build(variant=variant))
            d, i32, i64, u32, u64, vp = C.c_double, C.c_int, C.c_int64, C.c_uint32, C.c_uint64, C.c_void_p
            L.or_philox4x32_10.argtypes = [vp, vp, vp]
            L.or_gauss3.argtypes = [u64, u32, i64, u32, vp]
            L.or_noise_coefs.argtypes = [i32, d, d, vp, i32, vp, vp, vp, vp]
            L.or_noise_coefs.restype = i32
            L.or_integrator_factors.argtypes = [d, d, d, vp, vp]
            L.or_pairs_brute.argtypes = [vp, i32, d, d, vp, i64]
            L.or_pairs_brute.restype = i64
            L.or_pairs_brute_f32.argtypes = [vp, i32, C.c_float, C.c_float, vp, i64]
            L.or_pairs_brute_f32.restype = i64
            L.or_pairs_cells.argtypes = [vp, i32, d, d, vp, i64]
            L.or_pairs_cells.restype = i64
            L.or_create.argtypes = [i32, d, d, d, d, i32, d, d, d, u64, i32, i32, i64, vp, vp]
            L.or_create.restype = vp
            L.or_destroy.argtypes = [vp]
            L.or_set_kernels.argtypes = [vp, vp, i32, vp, vp, i32, d, i32, vp, vp, i32, i32]
            L.or_set_kernels.restype = i32
            L.or_step.argtypes = [vp, i64]
            L.or_step.restype = i32
            L.or_forces_subset.argtypes = [vp, vp, i32, vp, vp]
            L.or_get.argtypes = [vp, i32, vp]
            L.or_get.restype = i32
            L.or_set.argtypes = [vp, i32, vp]
            L.or_set.restype = i32
            L.or_set_step.argtypes = [vp, i64]
            L.or_get_step.argtypes = [vp]
            L.or_get_step.restype = i64
            L.or_recompute_fc.argtypes = [vp]
            L.or_get_coefs.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.or_get_vacf.argtypes = [vp, vp]
            L.or_get_vacf.restype = i64
            L.or_set_fc_table.argtypes = [vp, vp, i32, C.c_double]
            L.or_set_fc_table.restype = i32
            L.or_set_pair_table.argtypes = [vp, vp, i32, C.c_double, i32]
            L.or_set_pair_table.restype = i32
            L.or_set_paircorr.argtypes = [vp, i32, C.c_double]
            L.or_set_paircorr.restype = i32
            L.or_get_paircorr.argtypes = [vp, vp, vp, vp]
            L.or_white_window.argtypes = [vp, i64, vp]
            L.or_set_perp.argtypes = [vp, vp, vp]
            L.or_set_perp.restype = i32
            L.or_set_fr_override.argtypes = [vp, vp]
            L.or_set_threads.argtypes = [i32]
            L.or_get_threads.restype = i32
            _libs[variant] = L
    return _libs[variant]


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(t: int) -> None:
    lib().or_set_threads(int(t))


def threads() -> int:
    return int(lib().or_get_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block: 4 uint32 counter words, 2 key words -> 4 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def gauss3(seed: int, particle: int, time: int, stream: int = 0) -> np.ndarray:
    """The three Gaussian components W_{i,k} of particle i at time k."""
    z = np.zeros(3)
    lib().or_gauss3(seed, particle, time, stream, _p(z))
    return z


def noise_coefs(Kd, kT: float, dt: float, clamp: bool = False, variant: int = 0):
    """A_s from discrete K_m (Sec. II C).  Returns (status, C, Chat, A, clamped_mass)."""
    Kd = _f64(Kd)
    M = Kd.size
    Cm, Ch, A = np.zeros(M), np.zeros(M), np.zeros(2 * M - 1)
    mass = C.c_double(0.0)
    st = lib(variant).or_noise_coefs(M, kT, dt, _p(Kd), int(clamp), _p(Cm), _p(Ch), _p(A), C.byref(mass))
    return st, Cm, Ch, A, mass.value


def integrator_factors(K0: float, dt: float, mass: float):
    a, b = C.c_double(), C.c_double()
    lib().or_integrator_factors(K0, dt, mass, C.byref(a), C.byref(b))
    return a.value, b.value


def _pairs(fn, *args, n):
    cap = max(64, 64 * n)
    while True:
        out = np.zeros((cap, 2), dtype=np.int32)
        np_ = fn(*args, _p(out), cap)
        if np_ <= cap:
            return out[:np_].copy()
        cap = int(np_)


def pairs_brute(pos, box: float, rc: float) -> np.ndarray:
    pos = _f64(pos)
    return _pairs(lib().or_pairs_brute, _p(pos), pos.shape[0], box, rc, n=pos.shape[0])


def pairs_brute_f32(pos32, box: float, rc2_f32: float) -> np.ndarray:
    """Pair set from FP32 positions with the fixed single-precision distance test."""
    p = np.ascontiguousarray(pos32, dtype=np.float32)
    return _pairs(lib().or_pairs_brute_f32, _p(p), p.shape[0], float(np.float32(box)),
                  float(np.float32(rc2_f32)), n=p.shape[0])


def pairs_cells(pos, box: float, rc: float) -> np.ndarray:
    pos = _f64(pos)
    return _pairs(lib().or_pairs_cells, _p(pos), pos.shape[0], box, rc, n=pos.shape[0])


class System:
    """An oracle GLD system (FP64).  Mirrors the CUDA library's model API."""

    def __init__(self, *, n, box, mass, kT, dt, m_max, r_c, r_c_min=0.0, A_cons=0.0, seed=1,
                 vacf_len=0, vacf_stride=1, vacf_burnin=-1, pos, vel, variant=0):
        self._L = lib(variant)
        self.n, self.m_max = int(n), int(m_max)
        pos, vel = _f64(pos).reshape(n, 3), _f64(vel).reshape(n, 3)
        self._h = self._L.or_create(self.n, box, mass, kT, dt, self.m_max, r_c, r_c_min, A_cons,
                                    int(seed), int(vacf_len), int(vacf_stride),
                                    int(vacf_burnin) if vacf_burnin >= 0 else 2 * int(m_max),
                                    _p(pos), _p(vel))
        if not self._h:
            raise ValueError("oracle: invalid parameters")
        self.vacf_len = int(vacf_len)
        self._geom = dict(box=float(box), rc=float(r_c), rc_min=float(r_c_min), kT=float(kT), dt=float(dt))
        self._variant = int(variant)
        self._kern = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_destroy(h)
            self._h = None

    def set_kernels(self, Ks, g=None, f=None, dr=1.0, gs=None, fs=None, discrete=False, clamp=False):
        M = self.m_max
        Ks = _f64(Ks)
        g = np.zeros((0, M)) if g is None else _f64(g).reshape(-1, M)
        gs = np.zeros((0, M)) if gs is None else _f64(gs).reshape(-1, M)
        nr = (f.shape[-1] if f is not None else (fs.shape[-1] if fs is not None else 2))
        f = np.zeros((0, nr)) if f is None else _f64(f).reshape(-1, nr)
        fs = np.zeros((0, nr)) if fs is None else _f64(fs).reshape(-1, nr)
        self._kern = dict(Ks=Ks, g=g, f=f, dr=float(dr), gs=gs, fs=fs, discrete=bool(discrete), fp=None, fsp=None)
        return int(self._L.or_set_kernels(self._h, _p(Ks), g.shape[0], _p(g), _p(f), nr, dr,
                                          gs.shape[0], _p(gs), _p(fs), int(discrete), int(clamp)))

    def set_perp(self, fp=None, fsp=None) -> int:
        """Perpendicular radial factors fp[Q, nr], fsp[Qs, nr] of the kernel
        terms already set (None: zero)."""
        k = self._kern
        fp = None if fp is None else _f64(fp).reshape(k["g"].shape[0], -1)
        fsp = None if fsp is None else _f64(fsp).reshape(k["gs"].shape[0], -1)
        k["fp"], k["fsp"] = fp, fsp
        return int(self._L.or_set_perp(self._h, None if fp is None else _p(fp), None if fsp is None else _p(fsp)))

    def white_window(self, step=None) -> np.ndarray:
        """W_{i,n+s} for s = -(m_max-1) .. m_max-1: [2 m_max - 1, N, 3]."""
        n = self.step_index if step is None else int(step)
        out = np.zeros((2 * self.m_max - 1, self.n, 3))
        self._L.or_white_window(self._h, n, _p(out))
        return out

    def pair_random_force(self, clamp: bool = False) -> np.ndarray:
        """F^R of the coming step with the pair-correlated noise (Sec. II C,
        Algorithm 1 evaluated exactly; see pairnoise.py)."""
        from . import pairnoise
        k, G = self._kern, self._geom
        terms = pairnoise.matrix_terms(self.get(POS), G["box"], G["rc"], G["rc_min"], self.m_max, G["dt"],
                                       k["Ks"], k["g"], k["f"], k["dr"], k["gs"], k["fs"], k["discrete"],
                                       variant=self._variant, fp=k["fp"], fsp=k["fsp"])
        return pairnoise.random_force(terms, G["kT"], G["dt"], self.m_max, self.white_window(), clamp=clamp,
                                      variant=self._variant)

    def pair_random_force_window(self, rows: int, clamp: bool = False) -> np.ndarray:
        """F^R of the coming `rows` steps [rows, N, 3] from the one window of
        the coming step with the kernels at the current configuration (the
        time window of the remark after Algorithm 1; see pairnoise.py)."""
        from . import pairnoise
        k, G = self._kern, self._geom
        terms = pairnoise.matrix_terms(self.get(POS), G["box"], G["rc"], G["rc_min"], self.m_max, G["dt"],
                                       k["Ks"], k["g"], k["f"], k["dr"], k["gs"], k["fs"], k["discrete"],
                                       variant=self._variant, fp=k["fp"], fsp=k["fsp"])
        return pairnoise.random_force_window(terms, G["kT"], G["dt"], self.m_max, self.white_window(), rows,
                                             clamp=clamp, variant=self._variant)

    def step_pair_noise(self, nsteps: int = 1, clamp: bool = False) -> None:
        """Steps with the pair-correlated random force instead of the
        self-kernel noise."""
        for _ in range(int(nsteps)):
            F = _f64(self.pair_random_force(clamp))
            self._L.or_set_fr_override(self._h, _p(F))
            self.step(1)

    def step(self, nsteps: int = 1) -> None:
        st = self._L.or_step(self._h, int(nsteps))
        if st != 0:
            raise RuntimeError(f"oracle step failed ({st})")

    def get(self, which: int) -> np.ndarray:
        shape = (self.m_max - 1, self.n, 3) if which == HIST else (self.n, 3)
        out = np.zeros(shape)
        self._L.or_get(self._h, which, _p(out))
        return out

    def set(self, which: int, values) -> None:
        v = _f64(values)
        self._L.or_set(self._h, which, _p(v))

    @property
    def step_index(self) -> int:
        return int(self._L.or_get_step(self._h))

    def set_step(self, step: int) -> None:
        self._L.or_set_step(self._h, int(step))

    def recompute_fc(self) -> None:
        self._L.or_recompute_fc(self._h)

    def set_state(self, *, step, pos, vel, fc=None, hist=None) -> None:
        """Load a state (e.g. the GPU's FP32 state promoted to FP64)."""
        self.set_step(step)
        self.set(POS, pos)
        self.set(VEL, vel)
        if hist is not None:
            self.set(HIST, hist)
        if fc is None:
            self.recompute_fc()
        else:
            self.set(FC, fc)

    def coefs(self) -> dict:
        M = self.m_max
        Kd, A, Cm, Ch, ab = np.zeros(M), np.zeros(2 * M - 1), np.zeros(M), np.zeros(M), np.zeros(2)
        mass = C.c_double()
        self._L.or_get_coefs(self._h, _p(Kd), _p(A), _p(Cm), _p(Ch), _p(ab), C.byref(mass))
        return dict(Kd=Kd, A=A, C=Cm, Chat=Ch, a=ab[0], b=ab[1], clamped_mass=mass.value)

    def set_fc_table(self, f, dr: float) -> int:
        """Conservative force magnitude -dU/dr tabulated on r = k dr (None: the
        soft repulsion); F^C is recomputed."""
        if f is None:
            return self._L.or_set_fc_table(self._h, None, 0, 1.0)
        f = _f64(f)
        return self._L.or_set_fc_table(self._h, _p(f), int(f.size), float(dr))

    def set_pair_table(self, Kp, dr: float, discrete: bool = False) -> int:
        """A general pair kernel Kp[k, m] = K^p(k dr, m dt) (None: off)."""
        if Kp is None:
            return self._L.or_set_pair_table(self._h, None, 0, 1.0, 0)
        Kp = _f64(Kp).reshape(-1, self.m_max)
        return self._L.or_set_pair_table(self._h, _p(Kp), int(Kp.shape[0]), float(dr), int(bool(discrete)))

    def set_paircorr(self, nbins: int, rmax: float) -> int:
        """Enables C^a(R, t), C^c(R, t) (Sec. III A) on nbins distance bins of
        [0, rmax), sampled with the VACF's origins; rmax <= r_c."""
        st = self._L.or_set_paircorr(self._h, int(nbins), float(rmax))
        if st == 0:
            self._pc_nbins = int(nbins)
        return st

    def paircorr(self):
        """(C^a, C^c, counts), each [vacf_len, nbins]."""
        L, nb = self.vacf_len, self._pc_nbins
        ca, cc = np.zeros((L, nb)), np.zeros((L, nb))
        cnt = np.zeros((L, nb), dtype=np.int64)
        self._L.or_get_paircorr(self._h, _p(ca), _p(cc), _p(cnt))
        return ca, cc, cnt

    def vacf(self):
        out = np.zeros(max(self.vacf_len, 1))
        n0 = self._L.or_get_vacf(self._h, _p(out))
        return out[: self.vacf_len], int(n0)

    def forces_subset(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        fd, fr = np.zeros((idx.size, 3)), np.zeros((idx.size, 3))
        self._L.or_forces_subset(self._h, _p(idx), idx.size, _p(fd), _p(fr))
        return fd, fr


def history_projections(hist, coef) -> np.ndarray:
    """The history sums of Eq. dissipative_force2 written out in FP64:
    out[a, i, c] = sum_{m=1}^{m_max-1} coef[a, m] * hist[m-1, i, c],
    where hist[m-1] holds dR_{n-m}.  Used as the reference of the
    history-convolution kernel on identical FP32 inputs."""
    hist = np.asarray(hist, dtype=np.float64)
    coef = np.asarray(coef, dtype=np.float64)
    out = np.zeros((coef.shape[0],) + hist.shape[1:])
    for a in range(coef.shape[0]):
        for m in range(1, coef.shape[1]):
            out[a] += coef[a, m] * hist[m - 1]
    return out
