"""ctypes binding of the GLD CUDA library (include/gld.h).

Argument marshalling only: every step of the integrator runs in the CUDA
kernels of libgld.so.  PyTorch supplies device memory (its caching allocator,
handed to the library as an allocation callback) and streams.  If the
library is missing the import fails; there is no CPU or other fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, E_INVAL, E_NOMEM, E_NOT_PSD, E_CUDA, E_NONFINITE, E_TIMEOUT, E_STATE, E_CANCELLED = 0, -1, -2, -3, -4, -5, -6, -7, -8
HIST_F32, HIST_BF16 = 0, 1
KCONT, KDISCRETE = 0, 1
ARR_POS, ARR_VEL, ARR_FC, ARR_FD, ARR_FR, ARR_DISP, ARR_HIST, ARR_CONV = range(8)
_NAMES = {OK: "GLD_OK", E_INVAL: "GLD_E_INVAL", E_NOMEM: "GLD_E_NOMEM", E_NOT_PSD: "GLD_E_NOT_PSD",
          E_CUDA: "GLD_E_CUDA", E_NONFINITE: "GLD_E_NONFINITE", E_TIMEOUT: "GLD_E_TIMEOUT",
          E_STATE: "GLD_E_STATE", E_CANCELLED: "GLD_E_CANCELLED"}


class GLDError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        self.status = status
        super().__init__(f"{_NAMES.get(status, status)}: {message}")


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Params(C.Structure):
    _fields_ = [("n", C.c_int32), ("box", C.c_double), ("mass", C.c_double), ("kT", C.c_double),
                ("dt", C.c_double), ("m_max", C.c_int32), ("r_c", C.c_double), ("r_c_min", C.c_double),
                ("A_cons", C.c_double), ("skin", C.c_double), ("seed", C.c_uint64), ("hist_dtype", C.c_int32),
                ("kahan", C.c_int32), ("vacf_len", C.c_int32), ("vacf_stride", C.c_int32),
                ("vacf_burnin", C.c_int64), ("noise_block", C.c_int32), ("psd_clamp", C.c_int32),
                ("use_graphs", C.c_int32), ("order", C.c_void_p), ("stream", C.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class ServerParams(C.Structure):
    _fields_ = [("hbm_budget", C.c_int64), ("max_members", C.c_int32), ("in_flight", C.c_int32),
                ("tuning", C.c_int32), ("stream", C.c_void_p)]


class Request(C.Structure):
    _fields_ = [("params", Params), ("pos", C.c_void_p), ("vel", C.c_void_p), ("Ks", C.c_void_p),
                ("Q", C.c_int32), ("g", C.c_void_p), ("f", C.c_void_p), ("nr", C.c_int32), ("dr", C.c_double),
                ("dKs_g", C.c_void_p), ("dKs_f", C.c_void_p), ("Qs", C.c_int32),
                ("kernel_convention", C.c_int32), ("steps", C.c_int64), ("arrival", C.c_double),
                ("keep_state", C.c_int32), ("pair_noise", C.c_int32)]


SRV_STATS = ["queued", "active", "retiring", "done", "failed", "blocks", "particle_steps", "bytes", "bytes_peak",
             "members_peak", "budget"]

_lib = None


def lib():
    """Loads libgld.so (building it with nvcc if it is absent or stale)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError("libgld.so is missing and could not be built")
        L = C.CDLL(path)
        vp, i32, i64, d, u32, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint32, C.c_uint64
        sig = {
            "gld_params_default": (None, [C.POINTER(Params)]),
            "gld_create": (i32, [C.POINTER(Params), vp, vp, C.POINTER(vp)]),
            "gld_set_kernels": (i32, [vp, vp, i32, vp, vp, i32, d, vp, vp, i32, i32]),
            "gld_step": (i32, [vp, i64]),
            "gld_sync": (i32, [vp]),
            "gld_vacf": (i32, [vp, vp, C.POINTER(i64)]),
            "gld_get_state": (i32, [vp, vp, vp]),
            "gld_get_array": (i32, [vp, i32, vp]),
            "gld_set_array": (i32, [vp, i32, vp]),
            "gld_get_step": (i32, [vp, C.POINTER(i64)]),
            "gld_set_step": (i32, [vp, i64]),
            "gld_get_coefs": (i32, [vp, vp, vp, vp, vp]),
            "gld_get_pairs": (i32, [vp, vp, i64, C.POINTER(i64)]),
            "gld_get_order": (i32, [vp, vp]),
            "gld_get_diag": (i32, [vp, vp, i32]),
            "gld_profile_steps": (i32, [vp, i64, vp, vp]),
            "gld_last_error": (C.c_char_p, [vp]),
            "gld_destroy": (i32, [vp]),
            "gld_philox_dev": (i32, [vp, vp, vp, i64, vp]),
            "gld_gauss3_dev": (i32, [u64, vp, vp, u32, vp, i64, vp]),
            "gld_hist_conv_dev": (i32, [vp, i32, i32, i32, i64, vp, i32, vp, i32, vp]),
            "gld_pairs_noalloc": (i32, [vp, i32, d, d, vp, i64, vp, vp]),
            "gld_get_bytes": (i32, [vp, C.POINTER(i64)]),
            "gld_set_pair_correlation": (i32, [vp, i32, d]),
            "gld_set_memory_modes": (i32, [vp, i32, vp, vp]),
            "gld_set_conservative_table": (i32, [vp, vp, i32, C.c_double]),
            "gld_set_pair_noise": (i32, [vp, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "gld_set_perpendicular": (i32, [vp, vp, vp]),
            "gld_set_pair_noise_krylov": (i32, [vp, C.c_double, i32]),
            "gld_set_pair_noise_lanczos": (i32, [vp, C.c_double, i32, i32]),
            "gld_set_pair_noise_on": (i32, [vp, i32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]),
            "gld_pair_noise_spectrum": (i32, [vp, vp]),
            "gld_pair_noise_filters_on": (i32, [vp, vp, i32, C.c_double, C.c_double, C.c_double, C.c_double, i32,
                                                i32, vp, C.POINTER(C.c_double)]),
            "gld_pair_noise_filters": (i32, [vp, vp, i32, C.c_double, C.c_double, C.c_double, i32, i32, vp,
                                             C.POINTER(C.c_double)]),
            "gld_set_kernels_table": (i32, [vp, vp, vp, i32, C.c_double, i32, i32, C.POINTER(C.c_double)]),
            "gld_separable_terms": (i32, [vp, i32, i32, i32, vp, vp, C.POINTER(C.c_double)]),
            "gld_pair_correlation": (i32, [vp, vp, vp, vp]),
            "gld_save_observables": (i32, [vp, vp, i64, C.POINTER(i64)]),
            "gld_load_observables": (i32, [vp, vp, i64]),
            "gld_bytes_needed": (i32, [C.POINTER(Params), i32, i32, i32, C.POINTER(i64)]),
            "gld_batch_set_tuning": (i32, [vp, i32]),
            "gld_server_params_default": (None, [C.POINTER(ServerParams)]),
            "gld_server_create": (i32, [C.POINTER(ServerParams), C.POINTER(vp)]),
            "gld_server_submit": (i32, [vp, C.POINTER(Request), C.POINTER(i64)]),
            "gld_server_pump": (i32, [vp, C.POINTER(i32)]),
            "gld_server_drain": (i32, [vp, d]),
            "gld_server_clock": (i32, [vp, C.POINTER(d)]),
            "gld_server_result": (i32, [vp, i64, vp, C.POINTER(i64), vp, vp, vp]),
            "gld_server_stats": (i32, [vp, vp, i32]),
            "gld_server_cancel": (i32, [vp, i64]),
            "gld_server_last_error": (C.c_char_p, [vp]),
            "gld_server_destroy": (i32, [vp]),
            "gld_batch_create": (i32, [vp, C.POINTER(vp)]),
            "gld_batch_add": (i32, [vp, vp]),
            "gld_batch_remove": (i32, [vp, vp]),
            "gld_batch_step": (i32, [vp, i64]),
            "gld_batch_sync": (i32, [vp]),
            "gld_batch_info": (i32, [vp, C.POINTER(i32), C.POINTER(i32), vp]),
            "gld_batch_last_error": (C.c_char_p, [vp]),
            "gld_batch_destroy": (i32, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    """Names of the C entry points the binding expects the library to export."""
    return ["gld_params_default", "gld_create", "gld_set_kernels", "gld_step", "gld_sync", "gld_vacf",
            "gld_get_state", "gld_get_array", "gld_set_array", "gld_get_step", "gld_set_step",
            "gld_get_coefs", "gld_get_pairs", "gld_get_order", "gld_get_diag", "gld_profile_steps", "gld_last_error", "gld_destroy", "gld_philox_dev",
            "gld_gauss3_dev", "gld_hist_conv_dev", "gld_pairs_noalloc", "gld_batch_create", "gld_batch_add",
            "gld_batch_remove", "gld_batch_step", "gld_batch_sync", "gld_batch_info", "gld_batch_last_error",
            "gld_batch_destroy", "gld_get_bytes", "gld_bytes_needed", "gld_batch_set_tuning",
            "gld_server_params_default", "gld_server_create", "gld_server_submit", "gld_server_pump",
            "gld_server_drain", "gld_server_clock", "gld_server_result", "gld_server_stats",
            "gld_server_last_error", "gld_server_destroy", "gld_server_cancel", "gld_set_pair_correlation",
            "gld_pair_correlation", "gld_set_memory_modes", "gld_set_conservative_table",
            "gld_set_kernels_table", "gld_separable_terms", "gld_set_pair_noise",
            "gld_set_perpendicular", "gld_pair_noise_filters", "gld_save_observables", "gld_load_observables",
            "gld_set_pair_noise_krylov", "gld_set_pair_noise_lanczos", "gld_set_pair_noise_on",
            "gld_pair_noise_spectrum",
            "gld_pair_noise_filters_on"]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _current_stream() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, passed as C callbacks."""

    def __init__(self):
        import torch
        self._torch = torch
        self._device = torch.cuda.current_device()

        def _alloc(nbytes, stream, user):
            try:
                return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self._device,
                                                                    int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, stream, user):
            if ptr:
                self._torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


class GLD:
    """One GLD system on the current CUDA device (wraps a gld_ctx)."""

    def __init__(self, *, n, box, dt, m_max, r_c, pos, vel, mass=1.0, kT=1.0, r_c_min=0.0,
                 A_cons=0.0, skin=0.0, seed=1, hist_dtype="f32", kahan=False, vacf_len=0, vacf_stride=1,
                 vacf_burnin=-1, noise_block=64, psd_clamp=False, use_graphs=True, stream=None,
                 torch_allocator=True, order=None):
        L = lib()
        p = Params()
        L.gld_params_default(C.byref(p))
        p.n, p.box, p.mass, p.kT, p.dt = int(n), float(box), float(mass), float(kT), float(dt)
        p.m_max, p.r_c, p.r_c_min, p.A_cons = int(m_max), float(r_c), float(r_c_min), float(A_cons)
        p.skin = float(skin)
        p.seed = int(seed)
        p.hist_dtype = HIST_BF16 if hist_dtype in ("bf16", HIST_BF16) else HIST_F32
        p.kahan = int(bool(kahan))
        p.vacf_len, p.vacf_stride, p.vacf_burnin = int(vacf_len), int(vacf_stride), int(vacf_burnin)
        p.noise_block, p.psd_clamp = int(noise_block), int(bool(psd_clamp))
        p.use_graphs = int(use_graphs) if not isinstance(use_graphs, bool) else int(use_graphs)
        self.stream = _current_stream() if stream is None else int(stream)
        p.stream = self.stream
        self._alloc = _TorchAllocator() if torch_allocator else None
        if self._alloc is not None:
            p.alloc, p.free = self._alloc.alloc, self._alloc.free
        self._order = None
        if order is not None:
            self._order = np.ascontiguousarray(order, dtype=np.int32)
            p.order = _ptr(self._order)
        self._params = p
        self.n, self.m_max, self.vacf_len = int(n), int(m_max), int(vacf_len)
        pos, vel = _f64(pos).reshape(self.n, 3), _f64(vel).reshape(self.n, 3)
        h = C.c_void_p()
        st = L.gld_create(C.byref(p), _ptr(pos), _ptr(vel), C.byref(h))
        if st != OK:
            raise GLDError(st, "gld_create failed")
        self._h = h
        self.nacc = 1

    # -- life cycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().gld_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != OK:
            raise GLDError(st, lib().gld_last_error(self._h).decode())

    # -- model ----------------------------------------------------------------
    def set_kernels(self, Ks, g=None, f=None, dr=1.0, gs=None, fs=None, discrete=False):
        M = self.m_max
        Ks = _f64(Ks)
        g = None if g is None else _f64(g).reshape(-1, M)
        gs = None if gs is None else _f64(gs).reshape(-1, M)
        Q = 0 if g is None else g.shape[0]
        Qs = 0 if gs is None else gs.shape[0]
        nr = 2
        if f is not None:
            f = _f64(f).reshape(Q, -1)
            nr = f.shape[1]
        if fs is not None:
            fs = _f64(fs).reshape(Qs, -1)
            nr = fs.shape[1]
        keep = (Ks, g, f, gs, fs)
        st = lib().gld_set_kernels(self._h, _ptr(Ks), Q, None if g is None else _ptr(g),
                                   None if f is None else _ptr(f), nr, float(dr),
                                   None if gs is None else _ptr(gs), None if fs is None else _ptr(fs),
                                   Qs, KDISCRETE if discrete else KCONT)
        del keep
        self._check(st)
        self.nacc = 1 + Q + Qs

    def step(self, nsteps: int = 1):
        self._check(lib().gld_step(self._h, int(nsteps)))

    def sync(self):
        self._check(lib().gld_sync(self._h))

    def vacf(self):
        out = np.zeros(max(self.vacf_len, 1))
        n0 = C.c_int64()
        self._check(lib().gld_vacf(self._h, _ptr(out), C.byref(n0)))
        return out[: self.vacf_len], int(n0.value)

    def get_state(self):
        pos, vel = np.zeros((self.n, 3)), np.zeros((self.n, 3))
        self._check(lib().gld_get_state(self._h, _ptr(pos), _ptr(vel)))
        return pos, vel

    def get(self, which: int) -> np.ndarray:
        if which == ARR_HIST:
            shape = (self.m_max - 1, self.n, 3)
        elif which == ARR_CONV:
            shape = (self.nacc, self.n, 3)
        else:
            shape = (self.n, 3)
        out = np.zeros(shape)
        self._check(lib().gld_get_array(self._h, int(which), _ptr(out)))
        return out

    def set(self, which: int, values) -> None:
        v = _f64(values)
        self._check(lib().gld_set_array(self._h, int(which), _ptr(v)))

    @property
    def step_index(self) -> int:
        s = C.c_int64()
        self._check(lib().gld_get_step(self._h, C.byref(s)))
        return int(s.value)

    def set_step(self, step: int) -> None:
        self._check(lib().gld_set_step(self._h, int(step)))

    def diag(self) -> dict:
        out = np.zeros(5, dtype=np.int64)
        self._check(lib().gld_get_diag(self._h, _ptr(out), 5))
        return dict(graph_mode=int(out[0]), rebuilds=int(out[1]), maxnb=int(out[2]), cells_per_edge=int(out[3]),
                    krylov_iterations=int(out[4]))

    def set_memory_modes(self, rates, omegas):
        """Carries the memory sums in auxiliary-variable form for kernels that
        are sums of the modes exp((-rate + i omega) t); empty: the ring."""
        r, o = _f64(rates).ravel(), _f64(omegas).ravel()
        self._check(lib().gld_set_memory_modes(self._h, int(r.size), _ptr(r), _ptr(o)))

    def set_conservative_table(self, f, dr: float = 1.0):
        """F^C from a tabulated -dU/dr on r = k dr (None: the soft repulsion)."""
        if f is None:
            self._check(lib().gld_set_conservative_table(self._h, None, 0, 1.0))
            return
        f = _f64(f).ravel()
        self._check(lib().gld_set_conservative_table(self._h, _ptr(f), int(f.size), float(dr)))

    def set_kernels_table(self, Ks, Kp, dr: float, Q: int = 4, discrete: bool = False) -> float:
        """Self kernel Ks and a general pair kernel Kp[k, m] = K^p(k dr, m dt),
        reduced to its best rank-Q separable form; returns the relative
        Frobenius norm of the discarded part."""
        Ks, Kp = _f64(Ks), _f64(Kp).reshape(-1, self.m_max)
        tr = C.c_double()
        self._check(lib().gld_set_kernels_table(self._h, _ptr(Ks), _ptr(Kp), int(Kp.shape[0]), float(dr), int(Q),
                                                KDISCRETE if discrete else KCONT, C.byref(tr)))
        self.nacc = 1 + min(int(Q), Kp.shape[0], self.m_max)
        return float(tr.value)

    def set_perpendicular(self, fp=None, fs=None):
        """Perpendicular radial factors fp[Q, nr], fs[Qs, nr] of the kernel
        terms already set (acting through 1 - e e^T); None: zero."""
        fp = None if fp is None else _f64(fp).ravel()
        fs = None if fs is None else _f64(fs).ravel()
        keep = (fp, fs)
        self._check(lib().gld_set_perpendicular(self._h, None if fp is None else _ptr(fp),
                                                None if fs is None else _ptr(fs)))
        del keep

    def set_pair_noise(self, degree: int = 12, lam: float = 0.0):
        """Pair-correlated random force by a degree-`degree` Chebyshev form of
        the matrix square root (0: self-kernel noise only).  lam: bound on the
        pair matrix's spectrum (<= 0: automatic).  Returns (lam used,
        relative interpolation error)."""
        lv, err = C.c_double(float(lam)), C.c_double()
        self._check(lib().gld_set_pair_noise(self._h, int(degree), C.byref(lv), C.byref(err)))
        return float(lv.value), float(err.value)

    def set_pair_noise_on(self, degree: int = 12, lo: float | None = None, hi: float | None = None):
        """Chebyshev pair noise on an interval [lo, hi] of the pair matrix's
        spectrum (None: estimated by a Lanczos run, widened by 25 % of its
        spread each side within the positive semi-definite range; re-checked
        at every noise block).  Returns (lo, hi,
        relative interpolation error)."""
        l = C.c_double(float(lo) if lo is not None else 0.0)
        h = C.c_double(float(hi) if hi is not None else 0.0)
        err = C.c_double()
        self._check(lib().gld_set_pair_noise_on(self._h, int(degree), C.byref(l), C.byref(h), C.byref(err)))
        return float(l.value), float(h.value), float(err.value)

    def pair_noise_spectrum(self) -> dict:
        """The last Lanczos run of set_pair_noise_on: Ritz extremes, the
        Krylov dimension used, and the interval."""
        out = np.zeros(5)
        self._check(lib().gld_pair_noise_spectrum(self._h, _ptr(out)))
        return dict(ritz_min=float(out[0]), ritz_max=float(out[1]), krylov_dim=int(out[2]), lo=float(out[3]),
                    hi=float(out[4]))

    def set_pair_noise_lanczos(self, tol: float = 1e-6, kmax: int = 32, window: int = 0):
        """Pair-correlated noise by Algorithm 1: window 0 every step, window 1
        one run per 64-step noise block giving all its rows (the time window
        after Algorithm 1); tol <= 0 turns it off."""
        self._check(lib().gld_set_pair_noise_lanczos(self._h, float(tol), int(kmax), int(window)))

    def set_pair_noise_krylov(self, tol: float = 1e-6, kmax: int = 32):
        """Pair-correlated noise by a Lanczos iteration per frequency
        (Algorithm 1); tol <= 0 turns it off."""
        self._check(lib().gld_set_pair_noise_krylov(self._h, float(tol), int(kmax)))

    def set_pair_correlation(self, nbins: int, r_max: float):
        """Enables C^a(R, t), C^c(R, t) on nbins distance bins of [0, r_max)."""
        self._check(lib().gld_set_pair_correlation(self._h, int(nbins), float(r_max)))
        self._pc_nbins = int(nbins)

    def pair_correlation(self):
        """(C^a, C^c, counts), each [vacf_len, nbins]."""
        L, nb = self.vacf_len, self._pc_nbins
        ca, cc = np.zeros((L, nb)), np.zeros((L, nb))
        cnt = np.zeros((L, nb), dtype=np.int64)
        self._check(lib().gld_pair_correlation(self._h, _ptr(ca), _ptr(cc), _ptr(cnt)))
        return ca, cc, cnt

    def save_observables(self) -> bytes:
        """The VACF and pair-correlation accumulators as an opaque blob."""
        size = C.c_int64()
        self._check(lib().gld_save_observables(self._h, None, 0, C.byref(size)))
        buf = C.create_string_buffer(int(size.value))
        self._check(lib().gld_save_observables(self._h, buf, int(size.value), C.byref(size)))
        return buf.raw[: int(size.value)]

    def load_observables(self, blob: bytes) -> None:
        buf = C.create_string_buffer(bytes(blob), len(blob))
        self._check(lib().gld_load_observables(self._h, buf, len(blob)))

    def bytes(self) -> int:
        """Device bytes this system holds."""
        b = C.c_int64()
        self._check(lib().gld_get_bytes(self._h, C.byref(b)))
        return b.value

    def order(self) -> np.ndarray:
        """Internal storage order: entry k is the caller's index stored at k."""
        out = np.zeros(self.n, dtype=np.int32)
        self._check(lib().gld_get_order(self._h, _ptr(out)))
        return out

    def coefs(self) -> dict:
        M = self.m_max
        Kd, A, ab, spec = np.zeros(M), np.zeros(2 * M - 1), np.zeros(2), np.zeros(2)
        self._check(lib().gld_get_coefs(self._h, _ptr(Kd), _ptr(A), _ptr(ab), _ptr(spec)))
        return dict(Kd=Kd, A=A, a=ab[0], b=ab[1], spec_min=spec[0], clamped_mass=spec[1])

    PROF_NAMES = ("noise", "hist_conv", "pair_force_integrate", "cell_build", "cforce", "vacf", "pcorr",
                  "pair_noise")

    def profile_steps(self, nsteps: int):
        """Runs nsteps steps with per-kernel CUDA-event timing; returns
        {family: (milliseconds, launches)}."""
        ms, n = np.zeros(len(self.PROF_NAMES)), np.zeros(len(self.PROF_NAMES), dtype=np.int64)
        self._check(lib().gld_profile_steps(self._h, int(nsteps), _ptr(ms), _ptr(n)))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.PROF_NAMES)}

    def pairs(self) -> np.ndarray:
        cnt = C.c_int64()
        self._check(lib().gld_get_pairs(self._h, None, 0, C.byref(cnt)))
        cap = int(cnt.value)
        out = np.zeros((max(cap, 1), 2), dtype=np.int32)
        self._check(lib().gld_get_pairs(self._h, _ptr(out), cap, C.byref(cnt)))
        return out[: int(cnt.value)]


# ---- single kernels on torch device tensors ------------------------------------
def _dptr(t) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return int(t.data_ptr())


def bytes_needed(*, n, box, m_max, r_c, dt=0.005, skin=0.0, hist_dtype="f32", vacf_len=0, vacf_stride=1,
                 Q=1, Qs=0, nr=1024) -> int:
    """Device bytes a GLD system of these parameters holds once its kernels
    (Q pair terms, Qs self-difference terms on nr table points) are set."""
    p = Params()
    lib().gld_params_default(C.byref(p))
    p.n, p.box, p.m_max, p.r_c, p.dt, p.skin = int(n), float(box), int(m_max), float(r_c), float(dt), float(skin)
    p.hist_dtype = HIST_BF16 if hist_dtype in ("bf16", HIST_BF16) else HIST_F32
    p.vacf_len, p.vacf_stride = int(vacf_len), int(vacf_stride)
    b = C.c_int64()
    st = lib().gld_bytes_needed(C.byref(p), int(Q), int(Qs), int(nr), C.byref(b))
    if st != OK:
        raise GLDError(st, "gld_bytes_needed")
    return b.value


class Batch:
    """Independent GLD systems stepped together (wraps a gld_batch): each kernel
    family is one launch over all members, a 64-step block of the whole batch
    is one CUDA graph.  Members stay ordinary GLD objects."""

    def __init__(self, stream=None):
        self.stream = _current_stream() if stream is None else int(stream)
        h = C.c_void_p()
        st = lib().gld_batch_create(C.c_void_p(self.stream), C.byref(h))
        if st != OK:
            raise GLDError(st, "gld_batch_create failed")
        self._h = h
        self.members = []

    def _check(self, st: int):
        if st != OK:
            raise GLDError(st, lib().gld_batch_last_error(self._h).decode())

    def add(self, g: "GLD"):
        self._check(lib().gld_batch_add(self._h, g._h))
        self.members.append(g)

    def remove(self, g: "GLD"):
        self._check(lib().gld_batch_remove(self._h, g._h))
        self.members.remove(g)

    def step(self, nsteps: int):
        """Steps every member by nsteps (a multiple of 64) without waiting."""
        self._check(lib().gld_batch_step(self._h, int(nsteps)))

    def sync(self):
        st = lib().gld_batch_sync(self._h)
        if st != OK:
            raise GLDError(st, lib().gld_batch_last_error(self._h).decode())

    def set_tuning(self, policy: int):
        """0: re-time the convolution schedules at every composition change;
        1: only when the total column count moved by more than 2x."""
        self._check(lib().gld_batch_set_tuning(self._h, int(policy)))

    def info(self) -> dict:
        m, sc = C.c_int32(), C.c_int32()
        ms = np.zeros(4)
        self._check(lib().gld_batch_info(self._h, C.byref(m), C.byref(sc), _ptr(ms)))
        return {"members": m.value, "schedule": sc.value, "schedule_ms": ms.tolist()}

    def close(self):
        if getattr(self, "_h", None):
            lib().gld_batch_destroy(self._h)
            self._h = None
        self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop over GLD simulation requests (wraps a gld_server):
    admission by device bytes, continuous batching in 64-step blocks,
    results (VACF, optionally the final state) per request."""

    def __init__(self, *, hbm_budget=0, max_members=0, in_flight=2, tuning=1, stream=None):
        L = lib()
        p = ServerParams()
        L.gld_server_params_default(C.byref(p))
        p.hbm_budget, p.max_members, p.in_flight, p.tuning = int(hbm_budget), int(max_members), int(in_flight), int(tuning)
        p.stream = None if stream is None else int(stream)
        h = C.c_void_p()
        st = L.gld_server_create(C.byref(p), C.byref(h))
        if st != OK:
            raise GLDError(st, "gld_server_create failed")
        self._h = h
        self._meta = {}

    def _check(self, st: int):
        if st != OK:
            raise GLDError(st, lib().gld_server_last_error(self._h).decode())

    def submit(self, *, n, box, dt, m_max, r_c, pos, vel, Ks, g=None, f=None, dr=1.0, gs=None, fs=None,
               discrete=False, steps, arrival=0.0, keep_state=False, mass=1.0, kT=1.0, r_c_min=0.0, A_cons=0.0,
               skin=0.0, seed=1, hist_dtype="f32", kahan=False, vacf_len=0, vacf_stride=1, vacf_burnin=-1,
               pair_noise=0) -> int:
        L = lib()
        r = Request()
        p = r.params
        L.gld_params_default(C.byref(p))
        p.n, p.box, p.mass, p.kT, p.dt = int(n), float(box), float(mass), float(kT), float(dt)
        p.m_max, p.r_c, p.r_c_min, p.A_cons, p.skin = int(m_max), float(r_c), float(r_c_min), float(A_cons), float(skin)
        p.seed = int(seed)
        p.hist_dtype = HIST_BF16 if hist_dtype in ("bf16", HIST_BF16) else HIST_F32
        p.kahan = int(bool(kahan))
        p.vacf_len, p.vacf_stride, p.vacf_burnin = int(vacf_len), int(vacf_stride), int(vacf_burnin)
        M = int(m_max)
        pos, vel, Ks = _f64(pos).reshape(-1, 3), _f64(vel).reshape(-1, 3), _f64(Ks)
        g = None if g is None else _f64(g).reshape(-1, M)
        gs = None if gs is None else _f64(gs).reshape(-1, M)
        Q = 0 if g is None else g.shape[0]
        Qs = 0 if gs is None else gs.shape[0]
        nr = 2
        if f is not None:
            f = _f64(f).reshape(Q, -1)
            nr = f.shape[1]
        if fs is not None:
            fs = _f64(fs).reshape(Qs, -1)
            nr = fs.shape[1]
        keep = (pos, vel, Ks, g, f, gs, fs)
        r.pos, r.vel, r.Ks = pos.ctypes.data, vel.ctypes.data, Ks.ctypes.data
        r.Q, r.Qs, r.nr, r.dr = Q, Qs, nr, float(dr)
        r.g = None if g is None else g.ctypes.data
        r.f = None if f is None else f.ctypes.data
        r.dKs_g = None if gs is None else gs.ctypes.data
        r.dKs_f = None if fs is None else fs.ctypes.data
        r.kernel_convention = KDISCRETE if discrete else KCONT
        r.steps, r.arrival, r.keep_state = int(steps), float(arrival), int(bool(keep_state))
        r.pair_noise = int(pair_noise)
        rid = C.c_int64()
        st = L.gld_server_submit(self._h, C.byref(r), C.byref(rid))
        del keep
        self._check(st)
        self._meta[rid.value] = (int(n), int(vacf_len), bool(keep_state))
        return rid.value

    def pump(self) -> int:
        a = C.c_int32()
        self._check(lib().gld_server_pump(self._h, C.byref(a)))
        return a.value

    def drain(self, timeout: float = 0.0):
        self._check(lib().gld_server_drain(self._h, float(timeout)))

    def clock(self) -> float:
        t = C.c_double()
        self._check(lib().gld_server_clock(self._h, C.byref(t)))
        return t.value

    def result(self, rid: int) -> dict:
        """{'status', 'vacf', 'n_origins', 'arrival', 'admitted', 'done'[, 'pos', 'vel']};
        status is 0 when finished, E_STATE while pending, else the error."""
        n, L, keep_state = self._meta[rid]
        vacf = np.zeros(max(L, 1))
        no = C.c_int64()
        times = np.full(3, -1.0)
        pos = np.zeros((n, 3)) if keep_state else None
        vel = np.zeros((n, 3)) if keep_state else None
        st = lib().gld_server_result(self._h, int(rid), _ptr(vacf), C.byref(no),
                                     None if pos is None else _ptr(pos), None if vel is None else _ptr(vel),
                                     _ptr(times))
        out = {"status": st, "vacf": vacf[:L], "n_origins": no.value, "arrival": times[0], "admitted": times[1],
               "done": times[2]}
        if keep_state:
            out["pos"], out["vel"] = pos, vel
        return out

    def cancel(self, rid: int):
        self._check(lib().gld_server_cancel(self._h, int(rid)))

    def stats(self) -> dict:
        out = np.zeros(len(SRV_STATS), dtype=np.int64)
        self._check(lib().gld_server_stats(self._h, _ptr(out), len(SRV_STATS)))
        return dict(zip(SRV_STATS, out.tolist()))

    def close(self):
        if getattr(self, "_h", None):
            lib().gld_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox_dev(ctr, key, out, stream=None):
    """ctr: uint32-valued int32/uint32 CUDA tensor [n, 4]; out: same shape."""
    k = (C.c_uint32 * 2)(int(key[0]) & 0xffffffff, int(key[1]) & 0xffffffff)
    st = lib().gld_philox_dev(_dptr(ctr), k, _dptr(out), int(ctr.shape[0]),
                              _current_stream() if stream is None else stream)
    if st != OK:
        raise GLDError(st, "gld_philox_dev")


def gauss3_dev(seed, particle, time, out, stream_id=0, stream=None):
    """particle: int32 [n]; time: int64 [n]; out: float32 [n, 3] (CUDA tensors)."""
    st = lib().gld_gauss3_dev(int(seed), _dptr(particle), _dptr(time), int(stream_id), _dptr(out),
                              int(particle.shape[0]), _current_stream() if stream is None else stream)
    if st != OK:
        raise GLDError(st, "gld_gauss3_dev")


def hist_conv_dev(ring, n_pad, m_max, step, coef, nacc, out, bf16=False, kahan=False, stream=None):
    st = lib().gld_hist_conv_dev(_dptr(ring), int(bool(bf16)), int(n_pad), int(m_max), int(step),
                                 _dptr(coef), int(nacc), _dptr(out), int(bool(kahan)),
                                 _current_stream() if stream is None else stream)
    if st != OK:
        raise GLDError(st, "gld_hist_conv_dev")


NOALLOC_MAX_N = 65536


def pairs_noalloc(pos4, box, r_c, pairs, count, stream=None):
    """Neighbour pairs with no device allocation (scratch in a static device
    array).  pos4: float32 CUDA tensor [n, 4]; pairs: int32 [cap, 2];
    count: int64 [1]; all caller-owned."""
    st = lib().gld_pairs_noalloc(_dptr(pos4), int(pos4.shape[0]), float(box), float(r_c), _dptr(pairs),
                                 int(pairs.shape[0]), _dptr(count),
                                 _current_stream() if stream is None else stream)
    if st != OK:
        raise GLDError(st, "gld_pairs_noalloc")


def separable_terms(table, Q: int):
    """Host-side rank-Q separation of table[nr, m] ~ f^T g: (f[Q, nr], g[Q, m],
    relative Frobenius norm of the remainder)."""
    t = _f64(table)
    nr, m = t.shape
    f, g, tr = np.zeros((Q, nr)), np.zeros((Q, m)), C.c_double()
    st = lib().gld_separable_terms(_ptr(t), nr, m, int(Q), _ptr(f), _ptr(g), C.byref(tr))
    if st != 0:
        raise GLDError(st, "gld_separable_terms failed")
    return f, g, float(tr.value)


def pair_noise_filters(ks_weights, g_weights, kT: float, dt: float, lam: float, degree: int, psd_clamp=False):
    """Host-side filters of the pair-correlated noise: (taps[degree + 1,
    2 m_max - 1], relative interpolation error) from discrete weights."""
    ks, g = _f64(ks_weights).ravel(), _f64(g_weights).ravel()
    M = ks.size
    taps, err = np.zeros((int(degree) + 1, 2 * M - 1)), C.c_double()
    st = lib().gld_pair_noise_filters(_ptr(ks), _ptr(g), M, float(kT), float(dt), float(lam), int(degree),
                                      int(bool(psd_clamp)), _ptr(taps), C.byref(err))
    if st != 0:
        raise GLDError(st, "gld_pair_noise_filters failed")
    return taps, float(err.value)


def pair_noise_filters_on(ks_weights, g_weights, kT: float, dt: float, lo: float, hi: float, degree: int,
                          psd_clamp=False):
    """pair_noise_filters on the spectral interval [lo, hi]:
    F_n = sum_k T_k((M - c) / rho) Z_k, c and rho its centre and half-width."""
    ks, g = _f64(ks_weights).ravel(), _f64(g_weights).ravel()
    M = ks.size
    taps, err = np.zeros((int(degree) + 1, 2 * M - 1)), C.c_double()
    st = lib().gld_pair_noise_filters_on(_ptr(ks), _ptr(g), M, float(kT), float(dt), float(lo), float(hi),
                                         int(degree), int(bool(psd_clamp)), _ptr(taps), C.byref(err))
    if st != 0:
        raise GLDError(st, "gld_pair_noise_filters_on failed")
    return taps, float(err.value)
