"""ctypes binding of the C ABI in include/svm_gb300.h.

Argument marshalling only: numpy arrays are passed as host pointers, CUDA
torch tensors as device pointers. Every step of training and prediction runs
in the CUDA library; when the library cannot be built or loaded, every call
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

SVM_OK, SVM_NOT_CONVERGED, SVM_PENDING = 0, 1, 2
SVM_ERR_ARG, SVM_ERR_OOM, SVM_ERR_BUDGET, SVM_ERR_TIMEOUT = -1, -2, -3, -4
SVM_ERR_CUDA, SVM_ERR_CANCELLED, SVM_ERR_UNSUPPORTED = -5, -6, -7
SVM_FP64, SVM_MIXED_BF16, SVM_MIXED_BF16_SIMT = 0, 1, 2
SVM_SHRINK_NONE, SVM_SHRINK_FIXED, SVM_SHRINK_FRACTION = 0, 1, 2
SVM_RECON_SINGLE, SVM_RECON_MULTI = 0, 1
SVM_FLAG_STREAM_ROWS = 1
SVM_FLAG_PHASE_TIMES = 2
SVM_FLAG_NO_CLUSTERS = 4
SVM_FLAG_CSR_ROWS = 8
SVM_FLAG_WSS2 = 16
SVM_FLAG_NO_RELAYOUT = 32
SVM_FLAG_CUDA_CORE_ROWS = 64
SVM_FLAG_TENSOR_ROWS = 128
SVM_FLAG_FULL_RECON = 256
SVM_KERNEL_RBF, SVM_KERNEL_LINEAR, SVM_KERNEL_POLY, SVM_KERNEL_SIGMOID = 0, 1, 2, 3

STATUS_NAMES = {0: "SVM_OK", 1: "SVM_NOT_CONVERGED", 2: "SVM_PENDING", -1: "SVM_ERR_ARG",
                -2: "SVM_ERR_OOM", -3: "SVM_ERR_BUDGET", -4: "SVM_ERR_TIMEOUT",
                -5: "SVM_ERR_CUDA", -6: "SVM_ERR_CANCELLED", -7: "SVM_ERR_UNSUPPORTED"}


class svm_csr(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("d", ct.c_int64), ("indptr", ct.c_void_p),
                ("indices", ct.c_void_p), ("values", ct.c_void_p),
                ("on_device", ct.c_int32), ("reserved", ct.c_int32)]


class svm_params(ct.Structure):
    _fields_ = [("C", ct.c_double), ("gamma", ct.c_double), ("tau", ct.c_double),
                ("max_iter", ct.c_int64), ("precision", ct.c_int32), ("tie_break", ct.c_int32),
                ("stream", ct.c_void_p), ("trace", ct.c_void_p), ("trace_len", ct.c_int64),
                ("flags", ct.c_int32), ("ctas", ct.c_int32),
                ("lanes_per_row", ct.c_int32), ("cache_mb", ct.c_int32),
                ("kernel", ct.c_int32), ("degree", ct.c_int32), ("coef0", ct.c_double),
                ("active_trace", ct.c_void_p), ("active_trace_len", ct.c_int64),
                ("alpha0", ct.c_void_p)]


class svm_kernel(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("degree", ct.c_int32), ("gamma", ct.c_double),
                ("coef0", ct.c_double)]


class svm_shrink_policy(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("recon", ct.c_int32), ("value", ct.c_double),
                ("first_factor", ct.c_double)]


class svm_stats(ct.Structure):
    _fields_ = [("iters", ct.c_int64), ("shrink_events", ct.c_int64),
                ("reconstructions", ct.c_int64), ("final_active", ct.c_int64),
                ("n_sv", ct.c_int64), ("n_bound", ct.c_int64), ("row_visits", ct.c_int64),
                ("b_up", ct.c_double), ("b_low", ct.c_double), ("objective", ct.c_double),
                ("ms_total", ct.c_double), ("ms_smo", ct.c_double), ("ms_recon", ct.c_double),
                ("binary_input", ct.c_int32), ("launches", ct.c_int32),
                ("resident", ct.c_int32), ("ctas", ct.c_int32), ("lanes_per_row", ct.c_int32),
                ("cluster_size", ct.c_int32), ("phase_ms", ct.c_double * 8),
                ("cta_busy_ms_min", ct.c_double), ("cta_busy_ms_max", ct.c_double),
                ("bit_rows", ct.c_int32), ("cache_slots", ct.c_int32),
                ("cache_hits", ct.c_int64), ("cache_misses", ct.c_int64), ("relayouts", ct.c_int64),
                ("row_tiles", ct.c_int32), ("incremental_recons", ct.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "phase_ms"}
        d["phase_ms"] = list(self.phase_ms)
        return d


_lock = threading.Lock()
_lib = None


class SvmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsvmgb.so (building it with nvcc when missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("CUDA library libsvmgb.so is missing and could not be built")
            lib = ct.CDLL(_build.LIB)
            P = ct.c_void_p
            lib.svm_train.restype = ct.c_int
            lib.svm_train.argtypes = [P, P, P, P, P, P, P, P]
            lib.svm_decision.restype = ct.c_int
            lib.svm_decision.argtypes = [P, P, P, ct.c_double, ct.c_double, P, ct.c_int32, P, P]
            lib.svm_decision_kernel.restype = ct.c_int
            lib.svm_decision_kernel.argtypes = [P, P, P, ct.c_double, P, P, ct.c_int32, P, P]
            lib.svm_last_error.restype = ct.c_char_p
            lib.svm_last_error.argtypes = []
            lib.svm_version.restype = ct.c_char_p
            lib.svm_version.argtypes = []
            lib.svm_kernel_launches.restype = ct.c_int64
            lib.svm_kernel_launches.argtypes = []
            lib.svm_train_fixed_workspace.restype = ct.c_int
            lib.svm_train_fixed_workspace.argtypes = [P, P, P, P, P, P]
            lib.svm_diag_wait_timeout.restype = ct.c_int
            lib.svm_diag_wait_timeout.argtypes = [ct.c_int64, P]
            lib.svm_diag_sfu_rate.restype = ct.c_int
            lib.svm_diag_sfu_rate.argtypes = [P, P]
            lib.svm_model_create.restype = ct.c_int
            lib.svm_model_create.argtypes = [P, P, P, ct.c_double, P, ct.c_int32, P, P]
            lib.svm_model_decision.restype = ct.c_int
            lib.svm_model_decision.argtypes = [P, P, P, P]
            lib.svm_model_info.restype = ct.c_int
            lib.svm_model_info.argtypes = [P, P, P, P]
            lib.svm_model_free.restype = ct.c_int
            lib.svm_model_free.argtypes = [P]
            _lib = lib
    return _lib


def svm_kernel_launches() -> int:
    return int(load().svm_kernel_launches())


def svm_diag_sfu_rate(stream=None) -> float:
    """SFU exp2 instructions per second over the whole device (measured)."""
    v = ct.c_double(0.0)
    rc = load().svm_diag_sfu_rate(ct.byref(v), _stream_ptr(stream))
    if rc != SVM_OK:
        raise SvmError(rc, svm_last_error())
    return v.value


def svm_diag_wait_timeout(limit_ns: int, stream=None) -> int:
    """Runs the library's bounded device-side wait on a barrier that nothing
    completes; returns the status (SVM_ERR_TIMEOUT expected)."""
    return int(load().svm_diag_wait_timeout(int(limit_ns), _stream_ptr(stream)))


def svm_last_error() -> str:
    return load().svm_last_error().decode()


def svm_version() -> str:
    return load().svm_version().decode()


# ------------------------------------------------------------ marshalling
def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


class _Hold:
    """Keeps the buffers behind raw pointers alive during a call."""

    def __init__(self):
        self.keep = []

    def np(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.keep.append(a)
        return a.ctypes.data

    def tensor(self, t, dtype_name: str):
        import torch
        dt = getattr(torch, dtype_name)
        if t.dtype != dt or not t.is_contiguous():
            t = t.to(dt).contiguous()
        self.keep.append(t)
        return t.data_ptr()


@dataclass
class DeviceCSR:
    """CSR matrix whose arrays are CUDA torch tensors."""
    n: int
    d: int
    indptr: object
    indices: object
    values: object  # or None for binary rows


def to_device(X, device="cuda") -> DeviceCSR:
    """Copy a host CSR (numpy) into CUDA tensors."""
    import torch
    vals = None if X.values is None else torch.as_tensor(np.ascontiguousarray(X.values, np.float32), device=device)
    return DeviceCSR(int(X.n), int(X.d),
                     torch.as_tensor(np.ascontiguousarray(X.indptr, np.int64), device=device),
                     torch.as_tensor(np.ascontiguousarray(X.indices, np.int32), device=device),
                     vals)


def _csr(h: _Hold, X) -> tuple:
    if isinstance(X, DeviceCSR) or _is_torch_cuda(getattr(X, "indptr", None)):
        c = svm_csr(int(X.n), int(X.d), h.tensor(X.indptr, "int64"), h.tensor(X.indices, "int32"),
                    None if X.values is None else h.tensor(X.values, "float32"), 1, 0)
        return c, True
    c = svm_csr(int(X.n), int(X.d), h.np(X.indptr, np.int64), h.np(X.indices, np.int32),
                None if X.values is None else h.np(X.values, np.float32), 0, 0)
    return c, False


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ct.c_void_p(stream.cuda_stream)
    return ct.c_void_p(int(stream))


def svm_train(X, y, C: float, gamma: float, tau: float = 1e-3, *, max_iter: int = 0,
              precision: int = SVM_FP64, shrink: tuple | None = None, stream=None,
              trace_len: int = 0, alpha_out=None, flags: int = 0, ctas: int = 0,
              lanes_per_row: int = 0, cache_mb: int = 0, kernel: int = SVM_KERNEL_RBF,
              degree: int = 3, coef0: float = 0.0, active_trace_len: int = 0,
              alpha0=None, check: bool = True) -> dict:
    """Train by SMO. ``shrink`` = (kind, value, recon[, first_factor]) or None.
    ``active_trace_len``: record (step, active rows) after each of the first
    so many shrink events (returned as ``active_trace``, one row per event).
    ``cache_mb``: kernel-row cache budget in MiB (0 automatic, < 0 off).
    ``kernel``: SVM_KERNEL_* (RBF default; polynomial uses degree, coef0;
    sigmoid uses coef0).
    X is a host CSR (numpy arrays) or a DeviceCSR; y matches X's memory space.
    Returns dict(status, alpha, b, iters, stats, trace)."""
    lib = load()
    h = _Hold()
    cx, dev = _csr(h, X)
    n = int(X.n)
    if dev:
        import torch
        yp = h.tensor(y, "int8")
        if alpha_out is None:
            alpha_out = torch.empty(n, dtype=torch.float64, device=X.indptr.device)
        ap = alpha_out.data_ptr()
    else:
        yp = h.np(y, np.int8)
        if alpha_out is None:
            alpha_out = np.zeros(n)
        ap = alpha_out.ctypes.data
    trace = np.full((max(trace_len, 0), 2), -1, dtype=np.int32)
    p = svm_params(float(C), float(gamma), float(tau), int(max_iter), int(precision), 0,
                   _stream_ptr(stream), trace.ctypes.data if trace_len else None, int(trace_len),
                   int(flags), int(ctas), int(lanes_per_row), int(cache_mb), int(kernel), int(degree),
                   float(coef0))
    if alpha0 is not None:   # warm start, in X's memory space
        p.alpha0 = h.tensor(alpha0, "float64") if dev else h.np(alpha0, np.float64)
    atrace = np.full((max(active_trace_len, 0), 2), -1, dtype=np.int64)
    if active_trace_len:
        p.active_trace = atrace.ctypes.data
        p.active_trace_len = int(active_trace_len)
    pol = None
    if shrink is not None:
        kind, value, recon = shrink[:3]
        ff = shrink[3] if len(shrink) > 3 else 20.0
        pol = svm_shrink_policy(int(kind), int(recon), float(value), float(ff))
    b = ct.c_double(0.0)
    it = ct.c_int64(0)
    st = svm_stats()
    rc = lib.svm_train(ct.byref(cx), yp, ct.byref(p), ct.byref(pol) if pol is not None else None,
                       ap, ct.byref(b), ct.byref(it), ct.byref(st))
    if check and rc < 0:
        raise SvmError(rc, svm_last_error())
    out = {"status": rc, "alpha": alpha_out, "b": b.value, "iters": it.value, "stats": st.as_dict()}
    if trace_len:
        out["trace"] = trace[: min(trace_len, it.value)]
    if active_trace_len:
        out["active_trace"] = atrace[atrace[:, 0] >= 0]
    return out


def svm_decision(X, y, alpha, b: float, gamma: float, Z, *, precision: int = SVM_FP64,
                 stream=None, out=None, kernel: int = SVM_KERNEL_RBF, degree: int = 3,
                 coef0: float = 0.0, check: bool = True):
    """Eq. (classi) before the sign for the rows of Z (any kernel)."""
    lib = load()
    h = _Hold()
    cx, devx = _csr(h, X)
    cz, devz = _csr(h, Z)
    if devx:
        yp = h.tensor(y, "int8")
        ap = h.tensor(alpha, "float64")
    else:
        yp = h.np(y, np.int8)
        ap = h.np(alpha, np.float64)
    m = int(Z.n)
    if devz:
        import torch
        if out is None:
            out = torch.empty(m, dtype=torch.float64, device=Z.indptr.device)
        op = out.data_ptr()
    else:
        if out is None:
            out = np.zeros(m)
        op = out.ctypes.data
    if kernel == SVM_KERNEL_RBF:
        rc = lib.svm_decision(ct.byref(cx), yp, ap, float(b), float(gamma), ct.byref(cz),
                              int(precision), _stream_ptr(stream), op)
    else:
        k = svm_kernel(int(kernel), int(degree), float(gamma), float(coef0))
        rc = lib.svm_decision_kernel(ct.byref(cx), yp, ap, float(b), ct.byref(k), ct.byref(cz),
                                     int(precision), _stream_ptr(stream), op)
    if check and rc < 0:
        raise SvmError(rc, svm_last_error())
    return out


class Model:
    """A trained model resident on the device (svm_model_* of the C ABI): the
    support vectors, alpha y, b and the kernel, for repeated decisions."""

    def __init__(self, X, y, alpha, b: float, gamma: float, *, precision: int = SVM_FP64,
                 kernel: int = SVM_KERNEL_RBF, degree: int = 3, coef0: float = 0.0, stream=None):
        lib = load()
        h = _Hold()
        cx, devx = _csr(h, X)
        if devx:
            yp = h.tensor(y, "int8")
            ap = h.tensor(alpha, "float64")
        else:
            yp = h.np(y, np.int8)
            ap = h.np(alpha, np.float64)
        k = svm_kernel(int(kernel), int(degree), float(gamma), float(coef0))
        handle = ct.c_void_p(None)
        rc = lib.svm_model_create(ct.byref(cx), yp, ap, float(b), ct.byref(k), int(precision),
                                  _stream_ptr(stream), ct.byref(handle))
        if rc < 0:
            raise SvmError(rc, svm_last_error())
        self._h = handle
        self._lib = lib

    def decision(self, Z, *, stream=None, out=None):
        h = _Hold()
        cz, devz = _csr(h, Z)
        m = int(Z.n)
        if devz:
            import torch
            if out is None:
                out = torch.empty(m, dtype=torch.float64, device=Z.indptr.device)
            op = out.data_ptr()
        else:
            if out is None:
                out = np.zeros(m)
            op = out.ctypes.data
        rc = self._lib.svm_model_decision(self._h, ct.byref(cz), _stream_ptr(stream), op)
        if rc < 0:
            raise SvmError(rc, svm_last_error())
        return out

    def info(self) -> dict:
        n_sv, d, b = ct.c_int64(0), ct.c_int64(0), ct.c_double(0.0)
        rc = self._lib.svm_model_info(self._h, ct.byref(n_sv), ct.byref(d), ct.byref(b))
        if rc < 0:
            raise SvmError(rc, svm_last_error())
        return {"n_sv": n_sv.value, "d": d.value, "b": b.value}

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value is not None:
            self._lib.svm_model_free(self._h)
            self._h = ct.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


def svm_train_fixed_workspace(X, y, C: float, gamma: float, tau: float = 1e-3, *,
                              max_iter: int = 0, stream=None, alpha_out=None,
                              flags: int = 0, check: bool = True) -> dict:
    """Plain FP64 solve that allocates no device memory (see the header for
    who needs it and its limits). X, y and alpha_out are device buffers."""
    import torch
    lib = load()
    h = _Hold()
    cx, dev = _csr(h, X)
    if not dev:
        raise ValueError("svm_train_fixed_workspace takes a DeviceCSR")
    yp = h.tensor(y, "int8")
    if alpha_out is None:
        alpha_out = torch.empty(int(X.n), dtype=torch.float64, device=X.indptr.device)
    p = svm_params(float(C), float(gamma), float(tau), int(max_iter), SVM_FP64, 0,
                   _stream_ptr(stream), None, 0, int(flags), 0, 0, 0)
    b = ct.c_double(0.0)
    it = ct.c_int64(0)
    rc = lib.svm_train_fixed_workspace(ct.byref(cx), yp, ct.byref(p), alpha_out.data_ptr(),
                                       ct.byref(b), ct.byref(it))
    if check and rc < 0:
        raise SvmError(rc, svm_last_error())
    return {"status": rc, "alpha": alpha_out, "b": b.value, "iters": it.value}


class svm_job(ct.Structure):
    _fields_ = [("n_rows", ct.c_int64), ("rows", ct.c_void_p), ("y", ct.c_void_p),
                ("C", ct.c_double), ("gamma", ct.c_double), ("tau", ct.c_double),
                ("max_iter", ct.c_int64), ("alpha_out", ct.c_void_p)]


class svm_result(ct.Structure):
    _fields_ = [("b", ct.c_double), ("b_up", ct.c_double), ("b_low", ct.c_double),
                ("objective", ct.c_double), ("iters", ct.c_int64), ("status", ct.c_int32),
                ("n_sv", ct.c_int32)]


class svm_batch_config(ct.Structure):
    _fields_ = [("precision", ct.c_int32), ("cluster_size", ct.c_int32),
                ("lanes_per_row", ct.c_int32), ("clusters", ct.c_int32), ("stream", ct.c_void_p),
                ("ms_kernel", ct.c_double), ("ms_total", ct.c_double), ("iters_total", ct.c_int64),
                ("clusters_used", ct.c_int32), ("reserved", ct.c_int32)]


def _batch_args(X, jobs, precision, cluster_size, lanes_per_row, clusters, stream, h, alloc_alpha):
    cx, dev = _csr(h, X)
    arr = (svm_job * len(jobs))()
    alphas = []
    for k, jb in enumerate(jobs):
        y = jb["y"]
        n = len(y)
        rows = jb.get("rows")
        if dev:
            import torch
            yp = h.tensor(y, "int8")
            rp = None if rows is None else h.tensor(rows, "int32")
            a = torch.empty(n, dtype=torch.float64, device=X.indptr.device) if alloc_alpha else None
            ap = a.data_ptr() if a is not None else None
        else:
            yp = h.np(y, np.int8)
            rp = None if rows is None else h.np(rows, np.int32)
            a = np.zeros(n) if alloc_alpha else None
            ap = a.ctypes.data if a is not None else None
        alphas.append(a)
        arr[k] = svm_job(n, rp, yp, float(jb["C"]), float(jb["gamma"]), float(jb.get("tau", 1e-3)),
                         int(jb.get("max_iter", 0)), ap)
    cfg = svm_batch_config(int(precision), int(cluster_size), int(lanes_per_row), int(clusters),
                           _stream_ptr(stream), 0.0, 0.0, 0, 0, 0)
    return cx, arr, cfg, alphas


def svm_train_batch(X, jobs, *, precision: int = SVM_FP64, cluster_size: int = 0,
                    lanes_per_row: int = 0, clusters: int = 0, stream=None, check: bool = True) -> dict:
    """Train every job of ``jobs`` (dicts with rows, y, C, gamma[, tau, max_iter])
    over the shared matrix X in one persistent launch."""
    lib = load()
    if not hasattr(lib, "_batch_bound"):
        P = ct.c_void_p
        lib.svm_train_batch.restype = ct.c_int
        lib.svm_train_batch.argtypes = [P, P, ct.c_int32, P, P]
        lib.svm_batch_autotune.restype = ct.c_int
        lib.svm_batch_autotune.argtypes = [P, P, ct.c_int32, P]
        lib._batch_bound = True
    h = _Hold()
    cx, arr, cfg, alphas = _batch_args(X, jobs, precision, cluster_size, lanes_per_row, clusters,
                                       stream, h, True)
    res = (svm_result * len(jobs))()
    rc = lib.svm_train_batch(ct.byref(cx), arr, len(jobs), ct.byref(cfg), res)
    if check and rc < 0:
        raise SvmError(rc, svm_last_error())
    out = [{"b": r.b, "b_up": r.b_up, "b_low": r.b_low, "objective": r.objective,
            "iters": r.iters, "status": r.status, "n_sv": r.n_sv, "alpha": a}
           for r, a in zip(res, alphas)]
    return {"status": rc, "results": out, "cluster_size": cfg.cluster_size,
            "lanes_per_row": cfg.lanes_per_row, "clusters": cfg.clusters_used,
            "ms_kernel": cfg.ms_kernel, "ms_total": cfg.ms_total, "iters_total": cfg.iters_total}


def svm_batch_autotune(X, jobs, *, precision: int = SVM_FP64, cluster_size: int = 0,
                       lanes_per_row: int = 0, stream=None) -> dict:
    """Pick cluster_size / lanes_per_row for a batch by timing candidates."""
    lib = load()
    if not hasattr(lib, "_batch_bound"):
        P = ct.c_void_p
        lib.svm_train_batch.restype = ct.c_int
        lib.svm_train_batch.argtypes = [P, P, ct.c_int32, P, P]
        lib.svm_batch_autotune.restype = ct.c_int
        lib.svm_batch_autotune.argtypes = [P, P, ct.c_int32, P]
        lib._batch_bound = True
    h = _Hold()
    cx, arr, cfg, _ = _batch_args(X, jobs, precision, cluster_size, lanes_per_row, 0, stream, h, False)
    rc = lib.svm_batch_autotune(ct.byref(cx), arr, len(jobs), ct.byref(cfg))
    if rc < 0:
        raise SvmError(rc, svm_last_error())
    return {"cluster_size": cfg.cluster_size, "lanes_per_row": cfg.lanes_per_row}


class svm_server_config(ct.Structure):
    _fields_ = [("budget_bytes", ct.c_size_t), ("max_slots", ct.c_int32), ("precision", ct.c_int32),
                ("cluster_size", ct.c_int32), ("lanes_per_row", ct.c_int32), ("max_d", ct.c_int32),
                ("reserved", ct.c_int32)]


class svm_server_times(ct.Structure):
    _fields_ = [("submit_to_admit_ms", ct.c_double), ("admit_to_done_ms", ct.c_double),
                ("submit_to_done_ms", ct.c_double)]


class svm_server_info(ct.Structure):
    _fields_ = [("bytes_in_use", ct.c_size_t), ("budget_bytes", ct.c_size_t), ("queued", ct.c_int32),
                ("running", ct.c_int32), ("clusters", ct.c_int32), ("cluster_size", ct.c_int32),
                ("engine_launches", ct.c_int64)]


def _bind_server(lib):
    if getattr(lib, "_server_bound", False):
        return
    P = ct.c_void_p
    lib.svm_server_create.restype = ct.c_int
    lib.svm_server_create.argtypes = [P, P]
    lib.svm_server_submit.restype = ct.c_int
    lib.svm_server_submit.argtypes = [P, P, P, P, P]
    lib.svm_server_poll.restype = ct.c_int
    lib.svm_server_poll.argtypes = [P, ct.c_uint64, P, P, P]
    lib.svm_server_wait.restype = ct.c_int
    lib.svm_server_wait.argtypes = [P, ct.c_uint64, ct.c_double, P, P, P]
    lib.svm_server_cancel.restype = ct.c_int
    lib.svm_server_cancel.argtypes = [P, ct.c_uint64]
    lib.svm_server_stats.restype = ct.c_int
    lib.svm_server_stats.argtypes = [P, P]
    lib.svm_server_destroy.restype = ct.c_int
    lib.svm_server_destroy.argtypes = [P]
    lib._server_bound = True


class Server:
    """Continuous-batching training server (svm_server_* of the C ABI)."""

    def __init__(self, budget_bytes: int, max_slots: int = 0, precision: int = SVM_MIXED_BF16,
                 cluster_size: int = 0, lanes_per_row: int = 0, max_d: int = 0):
        self.lib = load()
        _bind_server(self.lib)
        cfg = svm_server_config(int(budget_bytes), int(max_slots), int(precision), int(cluster_size),
                                int(lanes_per_row), int(max_d), 0)
        self.h = ct.c_void_p()
        rc = self.lib.svm_server_create(ct.byref(cfg), ct.byref(self.h))
        if rc < 0:
            raise SvmError(rc, svm_last_error())
        self.n = {}

    def submit(self, X, y, C: float, gamma: float, tau: float = 1e-3, max_iter: int = 0,
               check: bool = True):
        h = _Hold()
        cx, dev = _csr(h, X)
        if dev:
            raise ValueError("submit takes host arrays")
        p = svm_params(float(C), float(gamma), float(tau), int(max_iter), 0, 0, None, None, 0, 0, 0, 0, 0)
        t = ct.c_uint64(0)
        rc = self.lib.svm_server_submit(self.h, ct.byref(cx), h.np(y, np.int8), ct.byref(p), ct.byref(t))
        if rc < 0:
            if check:
                raise SvmError(rc, svm_last_error())
            return rc
        self.n[t.value] = int(X.n)
        return t.value

    def _out(self, rc, ticket, r, a, tm):
        if rc == SVM_PENDING:
            return None
        self.n.pop(ticket, None)
        return {"status": rc, "b": r.b, "b_up": r.b_up, "b_low": r.b_low, "objective": r.objective,
                "iters": r.iters, "n_sv": r.n_sv, "alpha": a,
                "time_to_model_ms": tm.submit_to_done_ms, "queue_ms": tm.submit_to_admit_ms,
                "run_ms": tm.admit_to_done_ms, "error": svm_last_error() if rc < 0 else ""}

    def poll(self, ticket: int):
        r, tm = svm_result(), svm_server_times()
        a = np.zeros(self.n.get(ticket, 0))
        rc = self.lib.svm_server_poll(self.h, ticket, ct.byref(r), a.ctypes.data if len(a) else None,
                                      ct.byref(tm))
        return self._out(rc, ticket, r, a, tm)

    def wait(self, ticket: int, timeout: float = 600.0):
        r, tm = svm_result(), svm_server_times()
        a = np.zeros(self.n.get(ticket, 0))
        rc = self.lib.svm_server_wait(self.h, ticket, float(timeout), ct.byref(r),
                                      a.ctypes.data if len(a) else None, ct.byref(tm))
        return self._out(rc, ticket, r, a, tm)

    def cancel(self, ticket: int) -> int:
        return self.lib.svm_server_cancel(self.h, ticket)

    def stats(self) -> dict:
        i = svm_server_info()
        self.lib.svm_server_stats(self.h, ct.byref(i))
        return {k: getattr(i, k) for k, _ in i._fields_}

    def close(self):
        if self.h:
            self.lib.svm_server_destroy(self.h)
            self.h = ct.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
