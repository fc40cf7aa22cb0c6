"""ctypes binding of libpichol (C ABI in include/pichol.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libpichol.so.  Functions named ``pichol_*`` are the raw C entry
points; ``Context`` owns one C context plus its device workspace (a torch
uint8 tensor) and exposes the same calls with torch tensors.

There is no fallback: if the library has not been built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import pathlib
from dataclasses import dataclass

_PKG = pathlib.Path(__file__).resolve().parent
# PICHOL_DEBUG=1 in the environment loads the bounds-checked build instead
LIB_PATH = _PKG / ("libpichol_debug.so" if os.environ.get("PICHOL_DEBUG") == "1" else "libpichol.so")
INTERFACE = (2, 0)          # PICHOL_VERSION_MAJOR, _MINOR of include/pichol.h

PICHOL_MODE_FP64, PICHOL_MODE_MIXED = 0, 1
PICHOL_STATE_HESSIAN, PICHOL_STATE_FACTORS, PICHOL_STATE_FIT = 1, 2, 4
PICHOL_BASIS_MONO, PICHOL_BASIS_CHEB_LOG = 0, 1
REFINE_TARGETS = {"interpolated": 0, "exact": 1}
RESIDUALS = {"tensor": 0, "double_float": 1}
BASES = {"mono": PICHOL_BASIS_MONO, "cheb_log": PICHOL_BASIS_CHEB_LOG}
MODES = {"fp64": PICHOL_MODE_FP64, "mixed": PICHOL_MODE_MIXED}


def _choice(what: str, value, table: dict) -> int:
    if value not in table:
        raise ValueError(f"{what} must be one of {sorted(table)}, got {value!r}")
    return table[value]
STATUS = {0: "PICHOL_OK", 1: "PICHOL_ERR_INVALID_ARG", 2: "PICHOL_ERR_NOT_SPD", 3: "PICHOL_ERR_CUDA",
          4: "PICHOL_ERR_WORKSPACE", 5: "PICHOL_ERR_TIMEOUT", 6: "PICHOL_ERR_UNSUPPORTED", 7: "PICHOL_ERR_STATE"}

# every symbol include/pichol.h declares
EXPORTS = [
    "pichol_config_default", "pichol_create", "pichol_workspace_size", "pichol_set_workspace",
    "pichol_hessian", "pichol_factor_samples", "pichol_fit", "pichol_eval_holdout",
    "pichol_eval_holdout_exact", "pichol_get_lambdas", "pichol_export_factor", "pichol_export_theta",
    "pichol_export_hessian", "pichol_get_info", "pichol_clear_status", "pichol_launch_count",
    "pichol_destroy", "pichol_status_string", "pichol_set_timing", "pichol_stage_times",
    "pichol_fold_rhs_noalloc", "pichol_holdout_grad",
    "pichol_batch_create", "pichol_batch_workspace_size", "pichol_batch_set_workspace", "pichol_batch_set_streams",
    "pichol_batch_run", "pichol_batch_get_info", "pichol_batch_launch_count", "pichol_batch_destroy",
    "pichol_batch_set_timing", "pichol_batch_stage_times",
    "pichol_get_tuning", "pichol_set_tuning", "pichol_batch_set_tuning", "pichol_check_timeout",
    "pichol_check_wave_timeout",
    "pichol_mchol", "pichol_mchol_levels", "pichol_check_rsqrt", "pichol_eval_pinrmse", "pichol_probe_fma", "pichol_probe_mma",
    "pichol_get_state", "pichol_resume", "pichol_version", "pichol_debug_guards", "pichol_debug_build",
]
STAGES = ["gram", "xty", "setup", "chol_init", "chol_diag", "chol_panel", "chol_update", "fit",
          "diag_inv", "solve", "resid", "score", "select", "misc"]


class Tuning(ctypes.Structure):
    _fields_ = [("update_strip", ctypes.c_int32), ("diag_threads", ctypes.c_int32),
                ("diag_exclusive", ctypes.c_int32), ("eval_overlap", ctypes.c_int32), ("update_engine", ctypes.c_int32),
                ("solve_engine", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class Config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int64), ("c", ctypes.c_int64),
                ("k", ctypes.c_int32), ("g", ctypes.c_int32), ("r", ctypes.c_int32), ("q", ctypes.c_int32),
                ("lam_lo", ctypes.c_double), ("lam_hi", ctypes.c_double),
                ("scale_by_trace", ctypes.c_int32), ("basis", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("refine_steps", ctypes.c_int32), ("gram_passes", ctypes.c_int32),
                ("exact_batch", ctypes.c_int32), ("refine_target", ctypes.c_int32),
                ("warm_samples", ctypes.c_int32), ("refine_residual", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class Info(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int), ("fold", ctypes.c_int32), ("index", ctypes.c_int32),
                ("pivot", ctypes.c_int64), ("unusable", ctypes.c_int32)]


class PicholError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


_lib = None


def lib():
    """Load libpichol.so (raises if it was not built; there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1404_0466_gb300.build.build()")
    L = ctypes.CDLL(str(LIB_PATH))
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    sig = {
        "pichol_config_default": ([ctypes.POINTER(Config)], None),
        "pichol_create": ([ctypes.POINTER(Config), ctypes.POINTER(vp)], ctypes.c_int),
        "pichol_workspace_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "pichol_set_workspace": ([vp, vp, ctypes.c_size_t], ctypes.c_int),
        "pichol_hessian": ([vp, vp, vp, vp, vp], ctypes.c_int),
        "pichol_factor_samples": ([vp, vp, vp], ctypes.c_int),
        "pichol_fit": ([vp, vp, vp], ctypes.c_int),
        "pichol_eval_holdout": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "pichol_eval_holdout_exact": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "pichol_get_lambdas": ([vp, vp, vp], ctypes.c_int),
        "pichol_export_factor": ([vp, i32, i32, vp, vp], ctypes.c_int),
        "pichol_export_theta": ([vp, i32, vp, vp], ctypes.c_int),
        "pichol_export_hessian": ([vp, i32, vp, vp, vp], ctypes.c_int),
        "pichol_get_info": ([vp, ctypes.POINTER(Info), vp], ctypes.c_int),
        "pichol_clear_status": ([vp, vp], ctypes.c_int),
        "pichol_launch_count": ([vp], i64),
        "pichol_destroy": ([vp], None),
        "pichol_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "pichol_set_timing": ([vp, i32], ctypes.c_int),
        "pichol_fold_rhs_noalloc": ([i32, vp, vp, i64, i64, i64, i32, vp, vp, vp], ctypes.c_int),
        "pichol_holdout_grad": ([vp, ctypes.c_double, vp, vp, vp], ctypes.c_int),
        "pichol_mchol": ([vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp, vp], ctypes.c_int),
        "pichol_mchol_levels": ([ctypes.c_double, ctypes.c_double, ctypes.POINTER(i32)], ctypes.c_int),
        "pichol_check_rsqrt": ([i64, ctypes.c_uint64, vp, vp], ctypes.c_int),
        "pichol_eval_pinrmse": ([vp, vp, vp, vp], ctypes.c_int),
        "pichol_probe_fma": ([i32, i64, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "pichol_probe_mma": ([i32, i64, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "pichol_get_state": ([vp, ctypes.POINTER(i32)], ctypes.c_int),
        "pichol_resume": ([vp, i32], ctypes.c_int),
        "pichol_version": ([], i32),
        "pichol_debug_guards": ([vp, ctypes.POINTER(i64), i32, ctypes.POINTER(i32)], ctypes.c_int),
        "pichol_debug_build": ([], i32),
        "pichol_batch_create": ([ctypes.POINTER(Config), i32, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "pichol_batch_workspace_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "pichol_batch_set_workspace": ([vp, vp, ctypes.c_size_t], ctypes.c_int),
        "pichol_batch_set_streams": ([vp, i32], ctypes.c_int),
        "pichol_batch_run": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp], ctypes.c_int),
        "pichol_batch_get_info": ([vp, i32, ctypes.POINTER(Info), vp], ctypes.c_int),
        "pichol_batch_launch_count": ([vp], i64),
        "pichol_batch_destroy": ([vp], None),
        "pichol_batch_set_timing": ([vp, i32], ctypes.c_int),
        "pichol_get_tuning": ([vp, ctypes.POINTER(Tuning)], ctypes.c_int),
        "pichol_check_timeout": ([vp, i64, vp], ctypes.c_int),
        "pichol_check_wave_timeout": ([vp, i64, vp], ctypes.c_int),
        "pichol_set_tuning": ([vp, ctypes.POINTER(Tuning)], ctypes.c_int),
        "pichol_batch_set_tuning": ([vp, ctypes.POINTER(Tuning)], ctypes.c_int),
        "pichol_batch_stage_times": ([vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i32,
                                      vp], ctypes.c_int),
        "pichol_stage_times": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i32, vp],
                               ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    del dp
    v = L.pichol_version()
    if v // 100 != INTERFACE[0] or v % 100 < INTERFACE[1]:
        raise RuntimeError(f"{LIB_PATH} implements interface {v // 100}.{v % 100}, this binding needs "
                           f"{INTERFACE[0]}.{INTERFACE[1]}: rebuild it with paper_1404_0466_gb300.build.build()")
    _lib = L
    return L


def __getattr__(name):
    # raw C entry points: binding.pichol_hessian(...) etc.
    if name.startswith("pichol_"):
        return getattr(lib(), name)
    raise AttributeError(name)


def _check(code: int, where: str):
    if code != 0:
        raise PicholError(code, where)


def _require(t, name: str, shape, dtype):
    """Raise unless ``t`` is a contiguous CUDA tensor of ``dtype`` and
    ``shape``: the kernels read and write exactly that many elements.  Only
    tensor metadata is read, so this is safe during CUDA-graph capture."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclass
class CVOutput:
    E: "object"          # torch float64 (k, q) on device
    t_star: "object"     # torch int32 (1,) on device
    W: "object" = None   # torch (k, q, d, c) or None


class Context:
    """One piCholesky cross-validation problem on the current CUDA device."""

    def __init__(self, *, n, d, c, k, g, r, q, lam_lo=1e-3, lam_hi=1e1, basis="mono", mode="fp64",
                 refine_steps=0, gram_passes=3, exact_batch=0, scale_by_trace=True, refine_target="interpolated",
                 warm_samples=0, refine_residual="tensor"):
        import torch
        L = lib()
        cfg = Config()
        L.pichol_config_default(ctypes.byref(cfg))
        cfg.n, cfg.d, cfg.c, cfg.k, cfg.g, cfg.r, cfg.q = n, d, c, k, g, r, q
        cfg.lam_lo, cfg.lam_hi = lam_lo, lam_hi
        cfg.scale_by_trace = 1 if scale_by_trace else 0
        cfg.basis = _choice("basis", basis, BASES)
        cfg.mode = _choice("mode", mode, MODES)
        cfg.refine_steps, cfg.gram_passes, cfg.exact_batch = refine_steps, gram_passes, exact_batch
        cfg.refine_target = _choice("refine_target", refine_target, REFINE_TARGETS)
        cfg.warm_samples = warm_samples
        cfg.refine_residual = _choice("refine_residual", refine_residual, RESIDUALS)
        self.cfg = cfg
        self.dtype = torch.float64 if mode == "fp64" else torch.float32
        h = ctypes.c_void_p()
        _check(L.pichol_create(ctypes.byref(cfg), ctypes.byref(h)), "pichol_create")
        self._h = h
        nbytes = ctypes.c_size_t()
        _check(L.pichol_workspace_size(h, ctypes.byref(nbytes)), "pichol_workspace_size")
        self.workspace_bytes = nbytes.value
        self._ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device="cuda")
        _check(L.pichol_set_workspace(h, ctypes.c_void_p(self._ws.data_ptr()), self._ws.numel()),
               "pichol_set_workspace")

    # -- steps -------------------------------------------------------------
    def _host_doubles(self, values, count, name):
        """A caller's lambdas as a C array of `count` doubles (kept alive on self), or None."""
        if values is None:
            return None
        import numpy as np
        a = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(-1))
        if a.shape[0] != count:
            raise ValueError(f"{name}: expected {count} values, got {a.shape[0]}")
        return a

    def hessian(self, X, Y, fold_offsets=None, stream=None):
        """Normal-equation blocks (pichol_hessian); ``fold_offsets`` = k+1 row
        offsets of the folds (host), None for the contiguous floor split."""
        import numpy as np
        _require(X, "X", (self.cfg.n, self.cfg.d), self.dtype)
        _require(Y, "Y", (self.cfg.n, self.cfg.c), self.dtype)
        offs = None
        if fold_offsets is not None:
            offs = np.ascontiguousarray(np.asarray(fold_offsets, dtype=np.int64).reshape(-1))
            if offs.shape[0] != self.cfg.k + 1:
                raise ValueError(f"fold_offsets: expected {self.cfg.k + 1} values, got {offs.shape[0]}")
        self._X, self._Y = X, Y   # keep alive while kernels may read them
        _check(lib().pichol_hessian(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                    ctypes.c_void_p(offs.ctypes.data if offs is not None else 0),
                                    ctypes.c_void_p(_stream_ptr(stream))), "pichol_hessian")

    def factor_samples(self, lam_s=None, stream=None):
        """Exact factors at the g sampled lambdas: ``lam_s`` (absolute values,
        host) or None for the grid samples."""
        a = self._host_doubles(lam_s, self.cfg.g, "lam_s")
        _check(lib().pichol_factor_samples(self._h, ctypes.c_void_p(a.ctypes.data if a is not None else 0),
                                           ctypes.c_void_p(_stream_ptr(stream))), "pichol_factor_samples")

    def fit(self, theta_out=None, stream=None):
        """Algorithm 1's fit; ``theta_out`` (device tensor of theta_elems() values
        of the mode's type) also receives the tile-major coefficients."""
        if theta_out is not None:
            _require(theta_out, "theta_out", (self.theta_elems(),), self.dtype)
        _check(lib().pichol_fit(self._h, ctypes.c_void_p(theta_out.data_ptr() if theta_out is not None else 0),
                                ctypes.c_void_p(_stream_ptr(stream))), "pichol_fit")

    def theta_elems(self) -> int:
        """Values pichol_fit writes to theta_out: k * T * (r+1) * 64 * 64, T = nt (nt+1)/2."""
        nt = (self.cfg.d + 63) // 64
        return self.cfg.k * (nt * (nt + 1) // 2) * (self.cfg.r + 1) * 64 * 64

    def _outputs(self, want_w):
        import torch
        cfg = self.cfg
        E = torch.empty((cfg.k, cfg.q), dtype=torch.float64, device="cuda")
        t = torch.empty((1,), dtype=torch.int32, device="cuda")
        W = torch.empty((cfg.k, cfg.q, cfg.d, cfg.c), dtype=self.dtype, device="cuda") if want_w else None
        return E, t, W

    def _given_outputs(self, out, want_w):
        """A caller's (E, t_star, W) buffers, checked; new ones if ``out`` is None."""
        if out is None:
            return self._outputs(want_w)
        import torch
        E, t, W = out
        cfg = self.cfg
        _require(E, "E", (cfg.k, cfg.q), torch.float64)
        _require(t, "t_star", (1,), torch.int32)
        if W is not None:
            _require(W, "W", (cfg.k, cfg.q, cfg.d, cfg.c), self.dtype)
        return E, t, W

    def eval_holdout(self, want_w=False, out=None, stream=None, lam_t=None) -> CVOutput:
        """Interpolated solves and hold-out errors at the q evaluation lambdas:
        ``lam_t`` (absolute values, host) or None for the grid."""
        E, t, W = self._given_outputs(out, want_w)
        a = self._host_doubles(lam_t, self.cfg.q, "lam_t")
        _check(lib().pichol_eval_holdout(self._h, ctypes.c_void_p(a.ctypes.data if a is not None else 0),
                                         ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                         ctypes.c_void_p(W.data_ptr() if W is not None else 0),
                                         ctypes.c_void_p(_stream_ptr(stream))), "pichol_eval_holdout")
        return CVOutput(E, t, W)

    def eval_holdout_exact(self, want_w=False, out=None, stream=None, lam_t=None) -> CVOutput:
        E, t, W = self._given_outputs(out, want_w)
        a = self._host_doubles(lam_t, self.cfg.q, "lam_t")
        _check(lib().pichol_eval_holdout_exact(self._h, ctypes.c_void_p(a.ctypes.data if a is not None else 0),
                                               ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                               ctypes.c_void_p(W.data_ptr() if W is not None else 0),
                                               ctypes.c_void_p(_stream_ptr(stream))), "pichol_eval_holdout_exact")
        return CVOutput(E, t, W)

    def run(self, X, Y, want_w=False, out=None, stream=None, fold_offsets=None, lam_s=None,
            lam_t=None) -> CVOutput:
        """The whole hot path: hessian, factor_samples, fit, eval_holdout."""
        self.hessian(X, Y, fold_offsets, stream)
        self.factor_samples(lam_s, stream)
        self.fit(stream=stream)
        return self.eval_holdout(want_w, out, stream, lam_t=lam_t)

    def holdout_grad(self, log_lam: float, stream=None):
        """(E, dE/dlog(lambda)) per fold at lambda = exp(log_lam), through the
        interpolated factor; device float64 tensors of k entries."""
        import torch
        E = torch.empty((self.cfg.k,), dtype=torch.float64, device="cuda")
        dE = torch.empty((self.cfg.k,), dtype=torch.float64, device="cuda")
        _check(lib().pichol_holdout_grad(self._h, float(log_lam), ctypes.c_void_p(E.data_ptr()),
                                         ctypes.c_void_p(dE.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
               "pichol_holdout_grad")
        return E, dE

    def eval_pinrmse(self, out=None, stream=None) -> CVOutput:
        """PINRMSE after ``factor_samples``: the exact hold-out errors at the g
        sampled lambdas interpolated over the grid (pichol_eval_pinrmse)."""
        E, t, _ = self._given_outputs(out, False)
        _check(lib().pichol_eval_pinrmse(self._h, ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                         ctypes.c_void_p(_stream_ptr(stream))), "pichol_eval_pinrmse")
        return CVOutput(E, t, None)

    def mchol(self, c: float, s: float, s_min: float, trace=True, stream=None):
        """Multi-level range narrowing (pichol_mchol) after ``hessian``; the
        grid then spans the final range, so ``factor_samples``, ``fit`` and
        ``eval_holdout`` run piCholesky over it.  Returns the device trace
        (levels x 8 float64: three lambdas, their mean errors, c, s) or None."""
        import torch
        levels = mchol_levels(s, s_min)
        tr = torch.empty((levels, 8), dtype=torch.float64, device="cuda") if trace else None
        _check(lib().pichol_mchol(self._h, float(c), float(s), float(s_min),
                                  ctypes.c_void_p(tr.data_ptr() if tr is not None else 0),
                                  ctypes.c_void_p(_stream_ptr(stream))), "pichol_mchol")
        return tr

    # -- inspection ----------------------------------------------------------
    def lambdas(self, stream=None):
        import torch
        lam = torch.empty((self.cfg.q,), dtype=torch.float64, device="cuda")
        _check(lib().pichol_get_lambdas(self._h, ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
               "pichol_get_lambdas")
        return lam

    def export_factor(self, f, s, stream=None):
        import torch
        d = self.cfg.d
        L = torch.empty((d, d), dtype=torch.float64, device="cuda")
        _check(lib().pichol_export_factor(self._h, f, s, ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
               "pichol_export_factor")
        return L

    def export_theta(self, f, stream=None):
        import torch
        d = self.cfg.d
        T = torch.empty((self.cfg.r + 1, d, d), dtype=torch.float64, device="cuda")
        _check(lib().pichol_export_theta(self._h, f, ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
               "pichol_export_theta")
        return T

    def export_hessian(self, f, stream=None):
        import torch
        d, c = self.cfg.d, self.cfg.c
        H = torch.empty((d, d), dtype=torch.float64, device="cuda")
        B = torch.empty((d, c), dtype=torch.float64, device="cuda")
        _check(lib().pichol_export_hessian(self._h, f, ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                           ctypes.c_void_p(_stream_ptr(stream))), "pichol_export_hessian")
        return H, B

    def info(self, stream=None) -> Info:
        inf = Info()
        _check(lib().pichol_get_info(self._h, ctypes.byref(inf), ctypes.c_void_p(_stream_ptr(stream))), "pichol_get_info")
        return inf

    def check(self, stream=None) -> None:
        """Synchronise ``stream`` and raise PicholError if a device error was
        latched (pichol_get_info), naming the fold, index and pivot."""
        inf = self.info(stream)
        if inf.code != 0:
            raise PicholError(inf.code, f"device (fold {inf.fold}, index {inf.index}, pivot {inf.pivot})")

    def check_timeout(self, cycles: int, stream=None):
        """One bounded wait that runs out after `cycles` clocks (latches PICHOL_ERR_TIMEOUT)."""
        _check(lib().pichol_check_timeout(self._h, cycles, ctypes.c_void_p(_stream_ptr(stream))),
               "pichol_check_timeout")

    def check_wave_timeout(self, cycles: int, stream=None):
        """One wavefront pass whose waits run out after `cycles` clocks (latches PICHOL_ERR_TIMEOUT)."""
        _check(lib().pichol_check_wave_timeout(self._h, cycles, ctypes.c_void_p(_stream_ptr(stream))),
               "pichol_check_wave_timeout")

    def clear_status(self, stream=None):
        _check(lib().pichol_clear_status(self._h, ctypes.c_void_p(_stream_ptr(stream))), "pichol_clear_status")

    def set_timing(self, max_launches: int):
        _check(lib().pichol_set_timing(self._h, max_launches), "pichol_set_timing")

    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().pichol_get_tuning(self._h, ctypes.byref(t)), "pichol_get_tuning")
        return {"update_strip": t.update_strip, "diag_threads": t.diag_threads, "diag_exclusive": t.diag_exclusive,
                "eval_overlap": t.eval_overlap, "update_engine": t.update_engine, "solve_engine": t.solve_engine}

    def set_tuning(self, **kw):
        """Change launch shapes and scheduling (results are bit-identical under every tuning)."""
        cur = self.tuning()
        cur.update(kw)
        t = Tuning(cur["update_strip"], cur["diag_threads"], cur["diag_exclusive"], cur["eval_overlap"],
                   cur["update_engine"], cur["solve_engine"])
        _check(lib().pichol_set_tuning(self._h, ctypes.byref(t)), "pichol_set_tuning")

    def state(self) -> int:
        """Which results the workspace holds (PICHOL_STATE_* bits)."""
        st = ctypes.c_int32(0)
        _check(lib().pichol_get_state(self._h, ctypes.byref(st)), "pichol_get_state")
        return int(st.value)

    def guard_offsets(self) -> list:
        """Debug build: byte offsets of the guard bands in the workspace (empty otherwise)."""
        n = ctypes.c_int32(0)
        arr = (ctypes.c_int64 * 128)()
        _check(lib().pichol_debug_guards(self._h, arr, 128, ctypes.byref(n)), "pichol_debug_guards")
        return [int(arr[i]) for i in range(min(n.value, 128))]

    def state_dict(self, stream=None) -> dict:
        """A checkpoint: the configuration, the tuning, which results the
        workspace holds, and a copy of the workspace made on ``stream`` (default:
        the current one) after the work enqueued there.  torch.save can store it."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(s):
            ws = self._ws.clone()
        return {"config": bytes(self.cfg), "tuning": self.tuning(), "state": self.state(), "workspace": ws}

    def load_state_dict(self, sd: dict, stream=None):
        """Resume from ``state_dict()`` of a context with an identical
        configuration: copy the workspace in, apply the tuning, and declare the
        results it holds (pichol_resume)."""
        import torch
        if bytes(self.cfg) != sd["config"]:
            raise ValueError("the checkpoint was saved from a context with another configuration")
        ws = sd["workspace"]
        if ws.dtype != self._ws.dtype or ws.numel() != self._ws.numel():
            raise ValueError("the checkpoint's workspace does not match this context's")
        s = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(s):
            self._ws.copy_(ws, non_blocking=False)
        self.set_tuning(**sd["tuning"])
        _check(lib().pichol_resume(self._h, int(sd["state"])), "pichol_resume")

    def autotune(self, X, Y, *, reps=2, stream=None, cache=None, pg=None):
        """Time the launch-shape candidates on (X, Y), apply the fastest and
        return an ``autotune.TuneResult``.  No choice changes a result."""
        from . import autotune
        return autotune.tune_context(self, X, Y, reps=reps, stream=stream, cache=cache, pg=pg)

    def stage_times(self, stream=None):
        """{stage: (total ms, launches)} since the last call; needs set_timing."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        rc = lib().pichol_stage_times(self._h, ms, cnt, n, ctypes.c_void_p(_stream_ptr(stream)))
        if rc not in (0, 4):
            _check(rc, "pichol_stage_times")
        return {STAGES[i]: (ms[i], int(cnt[i])) for i in range(n)}, rc == 0

    def launch_count(self) -> int:
        return int(lib().pichol_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().pichol_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_rsqrt(n: int, seed: int = 1, stream=None) -> float:
    """Largest relative difference of the pivots' 1/sqrt from the library's
    1 / sqrt over n sampled values (pichol_check_rsqrt)."""
    import torch
    out = torch.empty((1,), dtype=torch.float64, device="cuda")
    _check(lib().pichol_check_rsqrt(int(n), int(seed), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(_stream_ptr(stream))), "pichol_check_rsqrt")
    return float(out.cpu().item())


def probe_fma(fp64: bool, iters: int = 1 << 14) -> float:
    """Measured FMA throughput of the FP32 or FP64 pipes in TFLOP/s (pichol_probe_fma)."""
    out = ctypes.c_double(0.0)
    _check(lib().pichol_probe_fma(1 if fp64 else 0, int(iters), ctypes.byref(out)), "pichol_probe_fma")
    return float(out.value)


def probe_mma(n_cols: int = 128, iters: int = 1 << 15) -> float:
    """Measured tcgen05.mma kind::tf32 rate (M = 128, K = 8, N = n_cols) in TFLOP/s (pichol_probe_mma)."""
    out = ctypes.c_double(0.0)
    _check(lib().pichol_probe_mma(int(n_cols), int(iters), ctypes.byref(out)), "pichol_probe_mma")
    return float(out.value)


def mchol_levels(s: float, s_min: float) -> int:
    """Levels pichol_mchol runs from half-width s down to s_min."""
    n = ctypes.c_int32(0)
    _check(lib().pichol_mchol_levels(float(s), float(s_min), ctypes.byref(n)), "pichol_mchol_levels")
    return int(n.value)


def holdout_loss(ctx: "Context", log_lam):
    """Mean hold-out error over the folds as a differentiable function of a
    scalar log(lambda) tensor: the forward pass and the derivative both come
    from pichol_holdout_grad (one call), the backward pass scales it."""
    import torch

    class _HoldoutLoss(torch.autograd.Function):
        @staticmethod
        def forward(fctx, ll):
            E, dE = ctx.holdout_grad(float(ll.detach().cpu()))
            fctx.save_for_backward(dE.mean().to(ll.device, ll.dtype))
            return E.mean().to(ll.device, ll.dtype)

        @staticmethod
        def backward(fctx, g):
            (dEbar,) = fctx.saved_tensors
            return g * dEbar

    return _HoldoutLoss.apply(log_lam)


class Batch:
    """Independent problems of uneven size run by one call (pichol_batch_run),
    capturable into a CUDA graph.  ``problems`` is a list of dicts with the
    Context keyword arguments (n, d, c, k, g, r, q, ...)."""

    def __init__(self, problems, nstreams=8):
        import torch
        L = lib()
        n = len(problems)
        cfgs = (Config * n)()
        self.mode = problems[0].get("mode", "fp64")
        for i, pr in enumerate(problems):
            L.pichol_config_default(ctypes.byref(cfgs[i]))
            cfg = cfgs[i]
            cfg.n, cfg.d, cfg.c, cfg.k, cfg.g, cfg.r, cfg.q = (pr[x] for x in ("n", "d", "c", "k", "g", "r", "q"))
            cfg.lam_lo, cfg.lam_hi = pr.get("lam_lo", 1e-3), pr.get("lam_hi", 1e1)
            cfg.basis = _choice("basis", pr.get("basis", "mono"), BASES)
            cfg.mode = _choice("mode", pr.get("mode", "fp64"), MODES)
            cfg.refine_steps = pr.get("refine_steps", 0)
            cfg.refine_target = _choice("refine_target", pr.get("refine_target", "interpolated"), REFINE_TARGETS)
            cfg.exact_batch = pr.get("exact_batch", cfg.g)
            cfg.warm_samples = pr.get("warm_samples", 0)
            cfg.refine_residual = _choice("refine_residual", pr.get("refine_residual", "tensor"), RESIDUALS)
        self.cfgs = cfgs
        self.n = n
        h = ctypes.c_void_p()
        _check(L.pichol_batch_create(cfgs, n, nstreams, ctypes.byref(h)), "pichol_batch_create")
        self._h = h
        nbytes = ctypes.c_size_t()
        _check(L.pichol_batch_workspace_size(h, ctypes.byref(nbytes)), "pichol_batch_workspace_size")
        self.workspace_bytes = nbytes.value
        self._ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device="cuda")
        _check(L.pichol_batch_set_workspace(h, ctypes.c_void_p(self._ws.data_ptr()), self._ws.numel()),
               "pichol_batch_set_workspace")
        dt = torch.float64 if self.mode == "fp64" else torch.float32
        self.dtype = dt
        self.E = [torch.empty((c.k, c.q), dtype=torch.float64, device="cuda") for c in cfgs]
        self.t_star = torch.empty((n,), dtype=torch.int32, device="cuda")

    def set_streams(self, nstreams):
        _check(lib().pichol_batch_set_streams(self._h, nstreams), "pichol_batch_set_streams")

    def set_tuning(self, update_strip=4, diag_threads=512, diag_exclusive=0, eval_overlap=0, update_engine=1,
                   solve_engine=2):
        """Launch shapes and scheduling for every problem (results are bit-identical)."""
        t = Tuning(update_strip, diag_threads, diag_exclusive, eval_overlap, update_engine, solve_engine)
        _check(lib().pichol_batch_set_tuning(self._h, ctypes.byref(t)), "pichol_batch_set_tuning")

    def autotune(self, Xs, Ys, *, reps=2, stream=None, cache=None, pg=None):
        """Time concurrent streams x update strip on (Xs, Ys), apply the
        fastest and return an ``autotune.TuneResult``."""
        from . import autotune
        return autotune.tune_batch(self, Xs, Ys, reps=reps, stream=stream, cache=cache, pg=pg)

    def run(self, Xs, Ys, stream=None):
        if len(Xs) != self.n or len(Ys) != self.n:
            raise ValueError(f"expected {self.n} X and Y tensors, got {len(Xs)} and {len(Ys)}")
        import torch
        for i, (x, y, c) in enumerate(zip(Xs, Ys, self.cfgs)):
            dt = torch.float64 if c.mode == PICHOL_MODE_FP64 else torch.float32
            _require(x, f"X[{i}]", (c.n, c.d), dt)
            _require(y, f"Y[{i}]", (c.n, c.c), dt)
        P = ctypes.c_void_p * self.n
        self._keep = (Xs, Ys)
        xp = P(*[x.data_ptr() for x in Xs])
        yp = P(*[y.data_ptr() for y in Ys])
        ep = P(*[e.data_ptr() for e in self.E])
        self._ptrs = (xp, yp, ep)
        _check(lib().pichol_batch_run(self._h, xp, yp, ep, ctypes.c_void_p(self.t_star.data_ptr()),
                                      ctypes.c_void_p(_stream_ptr(stream))), "pichol_batch_run")
        return self.E, self.t_star

    def info(self, i, stream=None) -> Info:
        inf = Info()
        _check(lib().pichol_batch_get_info(self._h, i, ctypes.byref(inf), ctypes.c_void_p(_stream_ptr(stream))),
               "pichol_batch_get_info")
        return inf

    def launch_count(self) -> int:
        return int(lib().pichol_batch_launch_count(self._h))

    def set_timing(self, max_launches: int):
        _check(lib().pichol_batch_set_timing(self._h, max_launches), "pichol_batch_set_timing")

    def stage_times(self, i, stream=None):
        """Problem i's {stage: (total ms, launches)} since the last call; needs set_timing."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        rc = lib().pichol_batch_stage_times(self._h, i, ms, cnt, n, ctypes.c_void_p(_stream_ptr(stream)))
        if rc not in (0, 4):
            _check(rc, "pichol_batch_stage_times")
        return {STAGES[j]: (ms[j], int(cnt[j])) for j in range(n)}, rc == 0

    def close(self):
        if getattr(self, "_h", None):
            lib().pichol_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
