"""FP64 CPU oracle for the detector-tomography solver (arXiv 2404.02844).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library and
its Python binding never import this package, and this package never imports
them.

This module is a thin ctypes wrapper around ``tomo_oracle.c`` (plain C, double
precision, OpenMP).  Every function of the C file cites the passage of the
paper it follows; see the header comment there for the readings of points the
paper leaves open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tomo_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

c_i64 = ctypes.c_int64
c_dbl = ctypes.c_double
c_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile tomo_oracle.c with gcc (OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    # -ffp-contract=off: products and sums are rounded as written (no fused
    # multiply-add), so integer decisions such as the band bounds are those of
    # the plain IEEE evaluation on every host architecture
    cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Opts(ctypes.Structure):
    _fields_ = [("eps_kkt", c_dbl), ("eps_bar", c_dbl), ("beta", c_dbl), ("c", c_dbl),
                ("switch_tol", c_dbl), ("f_target", c_dbl), ("max_newton", c_i64),
                ("max_stage1", c_i64), ("max_cg", c_i64), ("ls_max", c_i64),
                ("start_stage", c_i64), ("warm_start", c_i64), ("stall_iters", c_i64),
                ("cg_eta_max", c_dbl), ("cg_eta_pow", c_dbl)]


class _Report(ctypes.Structure):
    _fields_ = [("f", c_dbl), ("kkt", c_dbl), ("iters_s1", c_i64), ("iters_s2", c_i64),
                ("cg_total", c_i64), ("ls_total", c_i64), ("status", c_i64),
                ("stage_end", c_i64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_poisson.restype = c_dbl
        L.orc_poisson.argtypes = [c_i64, c_dbl]
        L.orc_band.argtypes = [c_i64, c_dbl, c_dbl, c_ptr, c_ptr]
        L.orc_create.restype = c_ptr
        L.orc_create.argtypes = [c_i64, c_i64, c_i64, c_ptr, c_dbl, c_dbl, ctypes.c_int]
        L.orc_destroy.argtypes = [c_ptr]
        L.orc_band_nnz.restype = c_i64
        L.orc_band_nnz.argtypes = [c_ptr]
        L.orc_bands.argtypes = [c_ptr, c_ptr, c_ptr]
        for name in ("orc_apply_F", "orc_apply_Ft", "orc_hvp"):
            getattr(L, name).argtypes = [c_ptr, c_ptr, c_ptr]
        L.orc_dense_F.argtypes = [c_ptr, c_ptr]
        L.orc_apply_F_rows.argtypes = [c_ptr, c_ptr, c_ptr, c_i64, c_ptr]
        L.orc_apply_Ft_rows.argtypes = [c_ptr, c_ptr, c_ptr, c_i64, c_ptr]
        L.orc_regulariser.restype = c_dbl
        L.orc_regulariser.argtypes = [c_ptr, c_ptr]
        L.orc_objective.restype = c_dbl
        L.orc_objective.argtypes = [c_ptr, c_ptr, c_ptr, c_ptr]
        L.orc_gradient.restype = c_dbl
        L.orc_gradient.argtypes = [c_ptr, c_ptr, c_ptr, c_ptr]
        L.orc_hess_diag.argtypes = [c_ptr, c_ptr]
        L.orc_project_simplex_sort.argtypes = [c_ptr, c_i64, c_ptr]
        L.orc_project_simplex_condat.argtypes = [c_ptr, c_i64, c_ptr]
        L.orc_project_rows.argtypes = [c_ptr, c_ptr, c_ptr]
        L.orc_smooth.argtypes = [c_ptr, c_ptr, c_ptr, c_i64, c_dbl]
        L.orc_fw_gap.restype = c_dbl
        L.orc_fw_gap.argtypes = [c_ptr, c_ptr, c_ptr]
        L.orc_kkt.restype = c_dbl
        L.orc_kkt.argtypes = [c_ptr, c_ptr, c_ptr]
        L.orc_default_opts.argtypes = [ctypes.POINTER(_Opts)]
        L.orc_fit.restype = c_i64
        L.orc_fit.argtypes = [c_ptr, c_ptr, c_ptr, ctypes.POINTER(_Opts),
                              ctypes.POINTER(_Report), c_ptr]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def poisson(i: int, lam: float) -> float:
    """F_{d,i} of Eq. Fmatrix for one (i, lambda)."""
    return lib().orc_poisson(int(i), float(lam))


def band(M: int, band_k: float, lam: float):
    lo = ctypes.c_int64()
    hi = ctypes.c_int64()
    lib().orc_band(M, band_k, lam, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def project_simplex(x, method: str = "sort") -> np.ndarray:
    x = _f64(x)
    y = np.empty_like(x)
    fn = lib().orc_project_simplex_sort if method == "sort" else lib().orc_project_simplex_condat
    fn(_p(x), x.shape[0], _p(y))
    return y


def num_threads() -> int:
    return lib().orc_num_threads()


class Problem:
    """One tomography problem: probes lambda (D), cutoff M, outcomes N,
    band half-width k (<= 0: dense F) and regularisation gamma."""

    def __init__(self, M: int, N: int, lam, band_k: float, gamma: float,
                 store_F: bool = True):
        self.M, self.N = int(M), int(N)
        self.lam = _f64(lam)
        self.D = int(self.lam.shape[0])
        self.band_k, self.gamma = float(band_k), float(gamma)
        self._h = lib().orc_create(self.M, self.N, self.D, _p(self.lam), self.band_k,
                                   self.gamma, 1 if store_F else 0)
        if not self._h:
            raise MemoryError("orc_create failed")

    @classmethod
    def from_workload(cls, w, store_F: bool = True):
        return cls(w.M, w.N, w.lam, w.band_k, w.gamma, store_F=store_F)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    # --- structure -----------------------------------------------------
    def nnz(self) -> int:
        return lib().orc_band_nnz(self._h)

    def bands(self):
        lo = np.empty(self.D, np.int64)
        hi = np.empty(self.D, np.int64)
        lib().orc_bands(self._h, _p(lo), _p(hi))
        return lo, hi

    def dense_F(self) -> np.ndarray:
        """F as a dense D x M array (Eq. Fmatrix, zero outside the bands)."""
        out = np.empty((self.D, self.M))
        lib().orc_dense_F(self._h, _p(out))
        return out

    # --- products ------------------------------------------------------
    def apply_F(self, X) -> np.ndarray:
        X = _f64(X)
        O = np.empty((self.D, self.N))
        lib().orc_apply_F(self._h, _p(X), _p(O))
        return O

    def apply_Ft(self, Y) -> np.ndarray:
        Y = _f64(Y)
        Z = np.empty((self.M, self.N))
        lib().orc_apply_Ft(self._h, _p(Y), _p(Z))
        return Z

    def apply_F_rows(self, X, rows) -> np.ndarray:
        """Selected rows of F X (X must be C-contiguous M x N float64)."""
        X = _f64(X)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty((rows.shape[0], self.N))
        lib().orc_apply_F_rows(self._h, _p(X), _p(rows), rows.shape[0], _p(out))
        return out

    def apply_Ft_rows(self, Y, rows) -> np.ndarray:
        Y = _f64(Y)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty((rows.shape[0], self.N))
        lib().orc_apply_Ft_rows(self._h, _p(Y), _p(rows), rows.shape[0], _p(out))
        return out

    def regulariser(self, X) -> float:
        return lib().orc_regulariser(self._h, _p(_f64(X)))

    def objective(self, P, Theta) -> float:
        return lib().orc_objective(self._h, _p(_f64(P)), _p(_f64(Theta)), None)

    def residual(self, P, Theta) -> np.ndarray:
        R = np.empty((self.D, self.N))
        lib().orc_objective(self._h, _p(_f64(P)), _p(_f64(Theta)), _p(R))
        return R

    def gradient(self, P, Theta):
        G = np.empty((self.M, self.N))
        f = lib().orc_gradient(self._h, _p(_f64(P)), _p(_f64(Theta)), _p(G))
        return f, G

    def hvp(self, V) -> np.ndarray:
        V = _f64(V)
        HV = np.empty((self.M, self.N))
        lib().orc_hvp(self._h, _p(V), _p(HV))
        return HV

    def hess_diag(self) -> np.ndarray:
        h = np.empty(self.M)
        lib().orc_hess_diag(self._h, _p(h))
        return h

    def project_rows(self, X) -> np.ndarray:
        X = _f64(X)
        Y = np.empty_like(X)
        lib().orc_project_rows(self._h, _p(X), _p(Y))
        return Y

    def kkt(self, Theta, G) -> float:
        return lib().orc_kkt(self._h, _p(_f64(Theta)), _p(_f64(G)))

    def smooth(self, X, exclude: int = 100, div: float = 50.0) -> np.ndarray:
        """Long-range smoothing of Eq. smoothing (window floor(i/div), rows
        below `exclude` unchanged)."""
        X = _f64(X)
        Y = np.empty_like(X)
        lib().orc_smooth(self._h, _p(X), _p(Y), int(exclude), float(div))
        return Y

    def fit_smoothed(self, P, exclude: int = 100, div: float = 50.0, **opts):
        """Sec. Regularisation and smoothing: Algorithm 3 from 1/N, long-range
        smoothing of the result, then stage 2 only from the smoothed POVM."""
        Th, rep1, _ = self.fit(P, **opts)
        Ts = self.smooth(Th, exclude, div)
        Th2, rep2, hist = self.fit(P, Theta0=Ts, start_stage=2, **opts)
        return Th2, rep1, rep2, Ts

    def fw_gap(self, Theta, G) -> float:
        """Upper bound of f(Theta) - f* for a feasible Theta (convexity)."""
        return lib().orc_fw_gap(self._h, _p(_f64(Theta)), _p(_f64(G)))

    # --- solver --------------------------------------------------------
    @staticmethod
    def default_opts() -> dict:
        o = _Opts()
        lib().orc_default_opts(ctypes.byref(o))
        return {k: getattr(o, k) for k, _ in _Opts._fields_}

    def fit(self, P, Theta0=None, **opts):
        """Algorithm 3 (or stage 2 only with start_stage=2).  Returns
        (Theta, report dict, f history)."""
        o = _Opts()
        lib().orc_default_opts(ctypes.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        Th = np.empty((self.M, self.N))
        if Theta0 is not None:
            Th[:] = Theta0
            o.warm_start = 1
        hist = np.empty(int(o.max_newton) + 2)
        rep = _Report()
        nh = lib().orc_fit(self._h, _p(_f64(P)), _p(Th), ctypes.byref(o),
                           ctypes.byref(rep), _p(hist))
        r = {k: getattr(rep, k) for k, _ in _Report._fields_}
        return Th, r, hist[:nh].copy()


def infidelity(Theta, Theta_ref):
    """Per-outcome infidelity 1 - F_n of Eq. fidelities for phase-insensitive
    (diagonal) POVMs: the operators commute, so
    Tr((sqrt(pi) pi_ref sqrt(pi))^(1/2)) = sum_i sqrt(Theta_in Theta_ref_in) and
    F_n = (sum_i sqrt(Theta_in Theta_ref_in))^2 / (sum_i Theta_in sum_i Theta_ref_in).
    Outcomes with an all-zero column on either side give nan."""
    A = np.asarray(Theta, dtype=np.float64)
    B = np.asarray(Theta_ref, dtype=np.float64)
    num = np.sum(np.sqrt(A * B), axis=0) ** 2
    den = A.sum(axis=0) * B.sum(axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        return 1.0 - num / den
