"""GB300 detector-tomography solver: Python binding of the C ABI in
include/tomo.h (libtomo.so, hand-written CUDA for sm_103a).

This module only marshals arguments: every step of the solve runs in the
library's kernels.  There is no CPU fallback -- if libtomo.so is missing or a
call fails, an exception is raised.

The functions ``tomo_plan``, ``tomo_objective``, ``tomo_fit``, ... carry the
names of the C entry points; :class:`Plan` wraps them for torch CUDA tensors
(float64, contiguous; device memory) and numpy arrays (host memory).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

__all__ = ["Plan", "TomoError", "lib", "tomo_plan", "tomo_plan_destroy", "tomo_objective",
           "tomo_fit", "tomo_fit_opts_default", "tomo_apply_F", "tomo_apply_Ft", "tomo_hvp",
           "tomo_hess_diag", "tomo_project_simplex", "tomo_kkt", "tomo_poisson_weights",
           "tomo_bands", "tomo_kernel_launches", "tomo_last_error", "PREC_FP64", "PREC_FP32",
           "STATUS", "STOP", "WarmStart", "fit_warm", "tomo_smooth"]

PREC_FP64 = 0
PREC_FP32 = 1
PREC_MIXED = 2
PREC_TC = 3
STATUS = {0: "TOMO_OK", 1: "TOMO_EINVAL", 2: "TOMO_ENOMEM", 3: "TOMO_ECUDA",
          4: "TOMO_ENOTCONV", 5: "TOMO_ETIMEOUT", 6: "TOMO_ENONFINITE"}
STOP = {0: "kkt", 1: "f_target", 2: "iteration_cap", 3: "stagnated"}

c_i32, c_i64, c_u32, c_dbl, c_ptr = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                     ctypes.c_double, ctypes.c_void_p)


class tomo_desc(ctypes.Structure):
    _fields_ = [("M", c_i64), ("N", c_i64), ("D", c_i64), ("lambda_", c_ptr),
                ("band_k", c_dbl), ("gamma", c_dbl), ("precision", c_i32),
                ("reserved", c_i32), ("stream", c_ptr), ("flags", c_u32)]


class tomo_fit_opts(ctypes.Structure):
    _fields_ = [("eps_kkt", c_dbl), ("eps_bar", c_dbl), ("beta", c_dbl), ("c", c_dbl),
                ("switch_tol", c_dbl), ("f_target", c_dbl), ("max_newton", c_i32),
                ("max_stage1", c_i32), ("max_cg", c_i32), ("ls_max", c_i32),
                ("start_stage", c_i32), ("warm_start", c_i32), ("stall_iters", c_i32),
                ("refresh_every", c_i32), ("profile", c_i32), ("trace_len", c_i32),
                ("cg_eta_max", c_dbl), ("cg_eta_pow", c_dbl), ("max_seconds", c_dbl),
                ("trace", c_ptr)]

TRACE_COLS = 11
TRACE_NAMES = ("stage", "f", "kkt", "cg", "cg_rel_res", "alpha", "ls", "ms", "ls_neg", "cg_end", "cg_ms")


class tomo_fit_report(ctypes.Structure):
    _fields_ = [("f", c_dbl), ("kkt", c_dbl), ("time_ms", c_dbl), ("iters_s1", c_i32),
                ("iters_s2", c_i32), ("cg_total", c_i32), ("ls_total", c_i32),
                ("refreshes", c_i32), ("stop", c_i32), ("stage_end", c_i32),
                ("kernels", c_i32), ("fwd_count", c_i32), ("adj_count", c_i32),
                ("fwd_ms", c_dbl), ("adj_ms", c_dbl)]


PLAN_AUTOTUNE = 1


class tomo_plan_info_t(ctypes.Structure):
    _fields_ = [("autotuned", c_i32), ("from_cache", c_i32), ("tensor_cores", c_i32),
                ("density", c_i32), ("hvp_ms", c_dbl), ("units_fwd", c_i32), ("units_adj", c_i32),
                ("ctas_fwd", c_i32), ("ctas_adj", c_i32)]


class tomo_ws_desc(ctypes.Structure):
    _fields_ = [("D", c_i64), ("C0", c_i64), ("M", c_i64), ("C1", c_i64), ("C2", c_i64),
                ("K", c_i64), ("S1", c_i64), ("S2", c_i64), ("H", c_i64), ("max_batch", c_i64),
                ("seed", ctypes.c_uint64), ("stream", c_ptr)]


# (name, restype, argtypes) of every entry point of include/tomo.h
EXPORTS = [
    ("tomo_plan", c_i32, [ctypes.POINTER(c_ptr), ctypes.POINTER(tomo_desc)]),
    ("tomo_plan_destroy", None, [c_ptr]),
    ("tomo_objective", c_i32, [c_ptr, c_ptr, c_ptr, ctypes.POINTER(c_dbl), c_ptr]),
    ("tomo_fit_opts_default", None, [ctypes.POINTER(tomo_fit_opts)]),
    ("tomo_fit", c_i32, [c_ptr, c_ptr, c_ptr, ctypes.POINTER(tomo_fit_opts),
                         ctypes.POINTER(tomo_fit_report)]),
    ("tomo_fit_batched", c_i32, [ctypes.POINTER(tomo_desc), ctypes.POINTER(c_ptr),
                                 ctypes.POINTER(c_ptr), c_i32, ctypes.POINTER(tomo_fit_opts),
                                 ctypes.POINTER(tomo_fit_report), ctypes.POINTER(c_i32), c_i32]),
    ("tomo_apply_F", c_i32, [c_ptr, c_ptr, c_ptr]),
    ("tomo_apply_Ft", c_i32, [c_ptr, c_ptr, c_ptr]),
    ("tomo_hvp", c_i32, [c_ptr, c_ptr, c_ptr]),
    ("tomo_hess_diag", c_i32, [c_ptr, c_ptr]),
    ("tomo_plan_info", c_i32, [c_ptr, ctypes.POINTER(tomo_plan_info_t)]),
    ("tomo_selftest_tc_timeout", c_i32, [c_ptr]),
    ("tomo_plan_tc_units", c_i64, [c_ptr, c_ptr, c_i32, c_i32, c_i64, c_i64, c_ptr, c_i64, c_ptr, c_ptr,
                                   ctypes.POINTER(c_i32)]),
    ("tomo_project_simplex", c_i32, [c_ptr, c_ptr, c_ptr]),
    ("tomo_smooth", c_i32, [c_ptr, c_ptr, c_ptr, c_i64, c_dbl]),
    ("tomo_infidelity", c_i32, [c_ptr, c_ptr, c_ptr, c_ptr]),
    ("tomo_kkt", c_i32, [c_ptr, c_ptr, c_ptr, ctypes.POINTER(c_dbl)]),
    ("tomo_poisson_weights", c_i32, [c_ptr, c_ptr, c_ptr, c_i64, c_ptr]),
    ("tomo_bands", c_i32, [c_ptr, c_ptr, c_ptr]),
    ("tomo_objective_noalloc", c_i32, [c_i64, c_i64, c_i64, c_ptr, c_dbl, c_dbl, c_ptr, c_ptr,
                                       c_ptr, c_ptr]),
    ("tomo_ws_create", c_i32, [ctypes.POINTER(c_ptr), ctypes.POINTER(tomo_ws_desc)]),
    ("tomo_ws_destroy", None, [c_ptr]),
    ("tomo_ws_param_count", c_i64, [c_ptr]),
    ("tomo_ws_get_params", c_i32, [c_ptr, c_ptr]),
    ("tomo_ws_set_params", c_i32, [c_ptr, c_ptr]),
    ("tomo_ws_loss_grad", c_i32, [c_ptr, c_ptr, c_ptr, c_ptr, c_i32, ctypes.POINTER(ctypes.c_float), c_ptr]),
    ("tomo_ws_train_step", c_i32, [c_ptr, c_ptr, c_ptr, c_ptr, c_i32, ctypes.c_float,
                                   ctypes.POINTER(ctypes.c_float)]),
    ("tomo_ws_infer", c_i32, [c_ptr, c_ptr, c_i64, c_ptr]),
    ("tomo_fit_warm", c_i32, [c_ptr, c_ptr, c_ptr, c_ptr, c_dbl, ctypes.POINTER(tomo_fit_opts),
                              ctypes.POINTER(tomo_fit_report), ctypes.POINTER(c_i32)]),
    ("tomo_ws_save", c_i32, [c_ptr, ctypes.c_char_p]),
    ("tomo_ws_load", c_i32, [c_ptr, ctypes.c_char_p]),
    ("tomo_kernel_launches", c_i64, []),
    ("tomo_last_error", ctypes.c_char_p, []),
]

_lib = None


class TomoError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


def lib(path: str | None = None) -> ctypes.CDLL:
    """Loads libtomo.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"libtomo.so not built ({p}); run paper_2404_02844_gb300.build.build()")
        L = ctypes.CDLL(p)
        for name, res, args in EXPORTS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st: int, where: str, allow=(0,)):
    if st not in allow:
        raise TomoError(st, where, lib().tomo_last_error().decode())
    return st


# --------------------------------------------------------------- C-named API
def tomo_plan(desc: tomo_desc) -> int:
    h = c_ptr()
    _check(lib().tomo_plan(ctypes.byref(h), ctypes.byref(desc)), "tomo_plan")
    return h.value


def tomo_plan_destroy(h: int) -> None:
    lib().tomo_plan_destroy(h)


def tomo_objective(h: int, P: int, Theta: int, grad: int | None = None) -> float:
    f = c_dbl()
    _check(lib().tomo_objective(h, P, Theta, ctypes.byref(f), grad), "tomo_objective")
    return f.value


def tomo_fit_opts_default() -> tomo_fit_opts:
    o = tomo_fit_opts()
    lib().tomo_fit_opts_default(ctypes.byref(o))
    return o


def tomo_fit(h: int, P: int, Theta: int, opts: tomo_fit_opts | None = None):
    rep = tomo_fit_report()
    st = lib().tomo_fit(h, P, Theta, ctypes.byref(opts) if opts is not None else None,
                        ctypes.byref(rep))
    _check(st, "tomo_fit", allow=(0, 4))
    return st, rep


def tomo_fit_batched(descs, P_ptrs, Theta_ptrs, opts=None, concurrency=8):
    """Solves len(descs) independent problems; returns (statuses, reports)."""
    n = len(descs)
    D = (tomo_desc * n)(*descs)
    Pp = (c_ptr * n)(*P_ptrs)
    Tp = (c_ptr * n)(*Theta_ptrs)
    reps = (tomo_fit_report * n)()
    sts = (c_i32 * n)()
    st = lib().tomo_fit_batched(D, Pp, Tp, n, ctypes.byref(opts) if opts is not None else None,
                                reps, sts, concurrency)
    _check(st, "tomo_fit_batched", allow=(0,))
    return [int(x) for x in sts], [_fit_dict(r) for r in reps]


def fit_batched(problems, precision="fp32", concurrency=8, autotune=False, **opts):
    """problems: list of (M, N, lam, band_k, gamma, P, Theta) with P, Theta
    float64 CUDA tensors (Theta receives the result).  Returns (statuses,
    reports).  autotune: plan every instance with TOMO_PLAN_AUTOTUNE."""
    prec = {"fp64": PREC_FP64, "fp32": PREC_FP32, "mixed": PREC_MIXED, "tc": PREC_TC}[precision]
    o = tomo_fit_opts_default()
    for k, v in opts.items():
        setattr(o, k, v)
    keep, descs, Pp, Tp = [], [], [], []
    stream = None
    try:
        import torch
        if torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    for (M, N, lam, band_k, gamma, P, Theta) in problems:
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        keep.append(lam)
        descs.append(tomo_desc(int(M), int(N), lam.shape[0], lam.ctypes.data, float(band_k),
                               float(gamma), prec, 0, stream or None, PLAN_AUTOTUNE if autotune else 0))
        Pp.append(_ptr(P))
        Tp.append(_ptr(Theta))
    return tomo_fit_batched(descs, Pp, Tp, o, concurrency)


def tomo_apply_F(h, X, O):
    _check(lib().tomo_apply_F(h, X, O), "tomo_apply_F")


def tomo_apply_Ft(h, Y, Z):
    _check(lib().tomo_apply_Ft(h, Y, Z), "tomo_apply_Ft")


def tomo_hvp(h, V, HV):
    _check(lib().tomo_hvp(h, V, HV), "tomo_hvp")


def tomo_hess_diag(h, out):
    _check(lib().tomo_hess_diag(h, out), "tomo_hess_diag")


def tomo_project_simplex(h, X, Y):
    _check(lib().tomo_project_simplex(h, X, Y), "tomo_project_simplex")


def tomo_smooth(h, X, Y, exclude=100, div=50.0):
    _check(lib().tomo_smooth(h, X, Y, int(exclude), float(div)), "tomo_smooth")


def tomo_kkt(h, Theta, G) -> float:
    k = c_dbl()
    _check(lib().tomo_kkt(h, Theta, G, ctypes.byref(k)), "tomo_kkt")
    return k.value


def tomo_poisson_weights(h, d, i, count, out):
    _check(lib().tomo_poisson_weights(h, d, i, count, out), "tomo_poisson_weights")


def tomo_bands(h, lo, hi):
    _check(lib().tomo_bands(h, lo, hi), "tomo_bands")


def tomo_kernel_launches() -> int:
    return lib().tomo_kernel_launches()


def tomo_last_error() -> str:
    return lib().tomo_last_error().decode()


# ------------------------------------------------------------------ wrapper
def _ptr(a):
    """Address of a torch tensor (device) or numpy array (host), float64 and
    contiguous."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy arrays must be float64 and C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be float64 and contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _fit_dict(rep: tomo_fit_report) -> dict:
    d = {k: getattr(rep, k) for k, _ in tomo_fit_report._fields_}
    d["stop_name"] = STOP.get(rep.stop, rep.stop)
    return d


class Plan:
    """A planned problem: probes ``lam`` (sorted, >= 0), cutoff M, outcomes N,
    Poisson band half-width ``band_k`` (<= 0: dense F), regularisation
    ``gamma`` and contraction precision ('fp64' or 'fp32').

    Work is ordered on torch's current CUDA stream at construction unless a
    raw ``stream`` handle is given."""

    def __init__(self, M, N, lam, band_k=10.0, gamma=0.0, precision="fp64", stream=None,
                 autotune=False):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        self.M, self.N, self.D = int(M), int(N), int(lam.shape[0])
        self.band_k, self.gamma = float(band_k), float(gamma)
        self.precision = {"fp64": PREC_FP64, "fp32": PREC_FP32, "mixed": PREC_MIXED, "tc": PREC_TC}[precision] \
            if isinstance(precision, str) else int(precision)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        self._lam = lam
        desc = tomo_desc(self.M, self.N, self.D, lam.ctypes.data, self.band_k, self.gamma,
                         self.precision, 0, stream or None, PLAN_AUTOTUNE if autotune else 0)
        self._h = tomo_plan(desc)

    def info(self) -> dict:
        """The schedule of the CG Hessian product (tomo_plan_info)."""
        i = tomo_plan_info_t()
        _check(lib().tomo_plan_info(self._h, ctypes.byref(i)), "tomo_plan_info")
        return {k: getattr(i, k) for k, _ in i._fields_}

    @classmethod
    def from_workload(cls, w, precision="fp64", **kw):
        return cls(w.M, w.N, w.lam, w.band_k, w.gamma, precision=precision, **kw)

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            tomo_plan_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- helpers
    def _dev_empty(self, *shape):
        import torch
        return torch.empty(*shape, dtype=torch.float64, device="cuda")

    def objective(self, P, Theta, want_grad=False):
        G = None
        if want_grad:
            G = np.empty((self.M, self.N)) if isinstance(Theta, np.ndarray) \
                else self._dev_empty(self.M, self.N)
        f = tomo_objective(self._h, _ptr(P), _ptr(Theta), _ptr(G) if G is not None else None)
        return (f, G) if want_grad else f

    def fit(self, P, Theta=None, **opts):
        """Algorithm 3.  Returns (Theta, report dict).  Theta (if given) is
        the warm start and is overwritten with the result."""
        o = tomo_fit_opts_default()
        trace = opts.pop("trace", 0)
        for k, v in opts.items():
            if not hasattr(o, k) or k in ("trace", "trace_len"):
                raise KeyError(k)
            setattr(o, k, v)
        tr = None
        if trace:
            tr = np.zeros((int(trace), TRACE_COLS))
            o.trace, o.trace_len = tr.ctypes.data, int(trace)
        if Theta is None:
            Theta = np.empty((self.M, self.N)) if isinstance(P, np.ndarray) \
                else self._dev_empty(self.M, self.N)
        else:
            o.warm_start = 1 if "warm_start" not in opts else opts["warm_start"]
        st, rep = tomo_fit(self._h, _ptr(P), _ptr(Theta), o)
        d = _fit_dict(rep)
        d["status"] = STATUS[st]
        if tr is not None:
            d["trace"] = tr[:rep.iters_s1 + rep.iters_s2]
        return Theta, d

    def apply_F(self, X):
        O = self._dev_empty(self.D, self.N)
        tomo_apply_F(self._h, _ptr(X), _ptr(O))
        return O

    def apply_Ft(self, Y):
        Z = self._dev_empty(self.M, self.N)
        tomo_apply_Ft(self._h, _ptr(Y), _ptr(Z))
        return Z

    def hvp(self, V):
        HV = self._dev_empty(self.M, self.N)
        tomo_hvp(self._h, _ptr(V), _ptr(HV))
        return HV

    def hess_diag(self):
        h = np.empty(self.M)
        tomo_hess_diag(self._h, h.ctypes.data)
        return h

    def project_simplex(self, X):
        Y = self._dev_empty(*tuple(X.shape))
        tomo_project_simplex(self._h, _ptr(X), _ptr(Y))
        return Y

    def smooth(self, X, exclude=100, div=50.0, out=None):
        """Long-range smoothing of Eq. smoothing (window floor(i/div), rows
        below `exclude` unchanged)."""
        Y = self._dev_empty(self.M, self.N) if out is None else out
        tomo_smooth(self._h, _ptr(X), _ptr(Y), exclude, div)
        return Y

    def fit_smoothed(self, P, exclude=100, div=50.0, **opts):
        """Sec. Regularisation and smoothing: Algorithm 3 from 1/N, the
        long-range smoothing of its result (in place), then a stage-2-only
        refit started from the smoothed POVM.  Returns (Theta, first report,
        refit report)."""
        Th, rep1 = self.fit(P, **opts)
        self.smooth(Th, exclude, div, out=Th)
        o = dict(opts)
        o["start_stage"] = 2
        Th, rep2 = self.fit(P, Th, **o)
        return Th, rep1, rep2

    def infidelity(self, Theta, Theta_ref) -> np.ndarray:
        """Per-outcome infidelity 1 - F_n (Eq. fidelities) of two POVMs."""
        out = np.empty(self.N)
        _check(lib().tomo_infidelity(self._h, _ptr(Theta), _ptr(Theta_ref), out.ctypes.data),
               "tomo_infidelity")
        return out

    def kkt(self, Theta, G):
        return tomo_kkt(self._h, _ptr(Theta), _ptr(G))

    def poisson_weights(self, d, i):
        d = np.ascontiguousarray(d, dtype=np.int64)
        i = np.ascontiguousarray(i, dtype=np.int64)
        out = np.empty(d.shape[0])
        tomo_poisson_weights(self._h, d.ctypes.data, i.ctypes.data, d.shape[0], out.ctypes.data)
        return out

    def bands(self):
        lo = np.empty(self.D, np.int64)
        hi = np.empty(self.D, np.int64)
        tomo_bands(self._h, lo.ctypes.data, hi.ctypes.data)
        return lo, hi


# ---------------------------------------------------------------------------
# learned warm start
# ---------------------------------------------------------------------------
class WarmStart:
    """Handle of the learned warm start (tomo_ws_*): a conv1d encoder over the
    probes, an MLP and a per-row softmax giving a feasible Theta0.  Batches
    are float64 torch CUDA tensors: P (B, D, C0) and targets (B, M, C0),
    padded with zero columns beyond each sample's ncols."""

    def __init__(self, D, C0, M, C1=32, C2=32, K=5, S1=2, S2=4, H=32, max_batch=32, seed=1,
                 stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        d = tomo_ws_desc(D, C0, M, C1, C2, K, S1, S2, H, max_batch, seed, c_ptr(stream))
        h = c_ptr()
        _check(lib().tomo_ws_create(ctypes.byref(h), ctypes.byref(d)), "tomo_ws_create")
        self._h = h.value
        self.shape = dict(D=D, C0=C0, M=M, C1=C1, C2=C2, K=K, S1=S1, S2=S2, H=H)
        self.max_batch = max_batch

    def close(self):
        if getattr(self, "_h", None):
            lib().tomo_ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def param_count(self) -> int:
        return int(lib().tomo_ws_param_count(self._h))

    def params(self) -> np.ndarray:
        out = np.empty(self.param_count, dtype=np.float32)
        _check(lib().tomo_ws_get_params(self._h, out.ctypes.data), "tomo_ws_get_params")
        return out

    def set_params(self, values) -> None:
        v = np.ascontiguousarray(values, dtype=np.float32)
        if v.size != self.param_count:
            raise ValueError("parameter vector of the wrong length")
        _check(lib().tomo_ws_set_params(self._h, v.ctypes.data), "tomo_ws_set_params")

    @staticmethod
    def _ncols(ncols):
        return np.ascontiguousarray(ncols, dtype=np.int32)

    def loss_grad(self, P, T, ncols):
        nc = self._ncols(ncols)
        loss = ctypes.c_float()
        g = np.empty(self.param_count, dtype=np.float32)
        _check(lib().tomo_ws_loss_grad(self._h, _ptr(P), _ptr(T), nc.ctypes.data, int(nc.size),
                                       ctypes.byref(loss), g.ctypes.data), "tomo_ws_loss_grad")
        return float(loss.value), g

    def train_step(self, P, T, ncols, lr=1e-3) -> float:
        nc = self._ncols(ncols)
        loss = ctypes.c_float()
        _check(lib().tomo_ws_train_step(self._h, _ptr(P), _ptr(T), nc.ctypes.data, int(nc.size),
                                        float(lr), ctypes.byref(loss)), "tomo_ws_train_step")
        return float(loss.value)

    def infer(self, P):
        """Theta0 (M x N) for one problem's P (D x N, float64 CUDA tensor)."""
        import torch
        N = int(P.shape[1])
        out = torch.empty(self.shape["M"], N, dtype=torch.float64, device="cuda")
        _check(lib().tomo_ws_infer(self._h, _ptr(P), N, _ptr(out)), "tomo_ws_infer")
        return out

    def save(self, path) -> None:
        _check(lib().tomo_ws_save(self._h, str(path).encode()), "tomo_ws_save")

    def load(self, path) -> None:
        _check(lib().tomo_ws_load(self._h, str(path).encode()), "tomo_ws_load")


def fit_warm(plan, ws, P, zero_below=0.0, **opts):
    """tomo_fit_warm: Algorithm 3 started from the learned Theta0, falling
    back to 1/N when f(Theta0) >= f(1/N) or when the warm-started fit fails
    (the rule runs in the library); zero_below > 0 first sets the entries of
    each row of Theta0 below zero_below x the row's largest to 0 and rescales
    the row.  P: float64 CUDA tensor.  Returns (Theta, report,
    used_warm_start)."""
    import torch
    o = tomo_fit_opts_default()
    for k, v in opts.items():
        if not hasattr(o, k) or k in ("trace", "trace_len"):
            raise KeyError(k)
        setattr(o, k, v)
    Th = torch.empty(plan.M, plan.N, dtype=torch.float64, device="cuda")
    rep = tomo_fit_report()
    used = c_i32(0)
    st = lib().tomo_fit_warm(plan._h, ws._h, _ptr(P), _ptr(Th), float(zero_below), ctypes.byref(o), ctypes.byref(rep),
                             ctypes.byref(used))
    _check(st, "tomo_fit_warm", allow=(0, 4))
    d = _fit_dict(rep)
    d["status"] = STATUS[st]
    return Th, d, bool(used.value)


def plan_tc_units(st, en, align=64, max_unit=1024, ctas=152):
    """Host-only tensor-core work-unit planning (tomo_plan_tc_units): returns
    (units as an (n, 4) int32 array of tile, chunk, k0, k1 in CTA order,
    CTA boundaries, units per tile)."""
    st = np.ascontiguousarray(st, dtype=np.int64)
    en = np.ascontiguousarray(en, dtype=np.int64)
    tiles = st.shape[0]
    cap = int(np.sum(np.maximum(en - st, 0)) // align + 2 * tiles + 8)
    units = np.empty((cap, 4), dtype=np.int32)
    cta_first = np.empty(ctas + 1, dtype=np.int32)
    nsplit = np.empty(tiles, dtype=np.int32)
    nc = c_i32()
    n = lib().tomo_plan_tc_units(st.ctypes.data, en.ctypes.data, tiles, align, max_unit, ctas,
                                 units.ctypes.data, cap, cta_first.ctypes.data, nsplit.ctypes.data,
                                 ctypes.byref(nc))
    if n < 0:
        raise TomoError(1, "tomo_plan_tc_units", tomo_last_error())
    return units[:n].copy(), cta_first[:nc.value + 1].copy(), nsplit
