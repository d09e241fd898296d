"""FP64 CPU oracle for the SVM training method of arXiv:1406.5161.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users. The CUDA library never
imports, links or calls anything here, and this package imports nothing from
the library (inputs come from the seeded generators in
``paper_1406_5161_gb300.synth``, which hold no solver arithmetic).

The arithmetic lives in ``smo_oracle.c`` (plain C, FP64, ``-ffp-contract=off``
so x86 and Arm produce the same bits); this module compiles it with gcc on
first use and wraps it with ctypes.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  smo            two-point closed form; brute-force dual QP (n <= 12);
                 invariants (sum y a = 0, box, monotone objective, f equal
                 to f recomputed from scratch); KKT gap at exit.
  smo_shrink     reaches the no-shrink optimum (structural fact of the paper:
                 shrinking changes the path, never the optimum); equals smo
                 with shrinking off; keeps the plain run's pairs until late;
                 its schedule (the step of every shrink test and
                 reconstruction, the counter h = k or ceil(p N), the reset to
                 min(h, |active|), the 20 tau / 2 tau phase thresholds, the
                 Multi restart and the Single stop) equals the one derived
                 from Algorithms 4 and 5 and Table 3 in the tests.
  dot / kernel   dense numpy inner product; closed forms.
  gradient,
  reconstruct    recomputation from the definition (Eq. fcache) with numpy.
  decision       decision at training points equals f + y - b; free support
                 vectors sit on the margin.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smo_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsmo_oracle.so")
_lock = threading.Lock()
_lib = None

SHRINK_NONE, SHRINK_FIXED, SHRINK_FRACTION = 0, 1, 2
RECON_SINGLE, RECON_MULTI = 0, 1


class _CSR(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("d", ct.c_int64),
                ("indptr", ct.c_void_p), ("indices", ct.c_void_p),
                ("values", ct.c_void_p)]


class _Result(ct.Structure):
    _fields_ = [("iters", ct.c_int64), ("b", ct.c_double), ("b_up", ct.c_double),
                ("b_low", ct.c_double), ("objective", ct.c_double),
                ("n_shrink", ct.c_int64), ("n_recon", ct.c_int64),
                ("final_active", ct.c_int64), ("status", ct.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-std=c99", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    """Load a build of the oracle and declare its C signatures."""
    lib = ct.CDLL(path)
    P = ct.c_void_p
    lib.or_dot.restype = ct.c_double
    lib.or_dot.argtypes = [P, ct.c_int64, P, ct.c_int64]
    lib.or_kernel.restype = ct.c_double
    lib.or_kernel.argtypes = [ct.c_double] * 4
    lib.or_sqnorm.restype = ct.c_double
    lib.or_sqnorm.argtypes = [P, ct.c_int64]
    lib.or_smo.restype = ct.c_int
    lib.or_smo.argtypes = [P, P, ct.c_double, ct.c_double, ct.c_double, ct.c_int64,
                           P, P, P, P, P, P, ct.c_int64]
    lib.or_smo_wss2.restype = ct.c_int
    lib.or_smo_wss2.argtypes = [P, P, ct.c_double, ct.c_double, ct.c_double, ct.c_int64,
                                P, P, P, P, P, ct.c_int64]
    lib.or_smo_shrink.restype = ct.c_int
    lib.or_smo_shrink.argtypes = [P, P, ct.c_double, ct.c_double, ct.c_double,
                                  ct.c_int64, ct.c_int, ct.c_double, ct.c_int,
                                  ct.c_double, P, P, P, P, ct.c_int64, P, ct.c_int,
                                  P, P, P, ct.c_int64, P]
    lib.or_gradient.restype = None
    lib.or_gradient.argtypes = [P, P, P, ct.c_double, P]
    lib.or_reconstruct.restype = None
    lib.or_reconstruct.argtypes = [P, P, P, ct.c_double, ct.c_int64, P, P]
    lib.or_kkt.restype = None
    lib.or_kkt.argtypes = [P, P, P, ct.c_double, ct.c_double, P, P]
    lib.or_decision.restype = None
    lib.or_decision.argtypes = [P, P, P, ct.c_double, ct.c_double, P, P]
    lib.or_set_kernel.restype = None
    lib.or_set_kernel.argtypes = [ct.c_int, ct.c_double, ct.c_int]
    lib.or_set_threads.restype = None
    lib.or_set_threads.argtypes = [ct.c_int]
    lib.or_max_threads.restype = ct.c_int
    lib.or_max_threads.argtypes = []
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


def load_variant(path: str):
    """Bind another build of the oracle source (used by the tests that plant
    a mistake in a copy of the oracle and check that the pins catch it)."""
    return _bind(path)


class _Keep:
    """Holds contiguous copies alive for the duration of a call."""

    def __init__(self):
        self.arrs = []

    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.arrs.append(a)
        return a

    def csr(self, X):
        ip = self.arr(X.indptr, np.int64)
        ix = self.arr(X.indices, np.int32)
        vv = self.arr(X.values, np.float32)
        c = _CSR(int(X.n), int(X.d), ip.ctypes.data, ix.ctypes.data, vv.ctypes.data)
        self.arrs.append(c)
        return ct.byref(c)


def _ptr(a):
    return None if a is None else a.ctypes.data


KERNEL_RBF, KERNEL_LINEAR, KERNEL_POLY, KERNEL_SIGMOID = 0, 1, 2, 3


def set_kernel(kind: int = KERNEL_RBF, coef0: float = 0.0, degree: int = 3, lib=None) -> None:
    """Select the kernel of later calls: RBF exp(-gamma ||x-z||^2) (default),
    linear <x,z>, polynomial (gamma <x,z> + coef0)^degree, sigmoid
    tanh(gamma <x,z> + coef0)."""
    (lib or _load()).or_set_kernel(int(kind), float(coef0), int(degree))


class kernel_spec:
    """Context manager: the oracle uses the given kernel inside the block."""

    def __init__(self, kind: int, coef0: float = 0.0, degree: int = 3, lib=None):
        self.args = (kind, coef0, degree)
        self.lib = lib

    def __enter__(self):
        set_kernel(*self.args, lib=self.lib)
        return self

    def __exit__(self, *exc):
        set_kernel(KERNEL_RBF, lib=self.lib)
        return False


def set_threads(t: int, lib=None) -> None:
    (lib or _load()).or_set_threads(int(t))


def max_threads(lib=None) -> int:
    return int((lib or _load()).or_max_threads())


def dot(X, i: int, Z, j: int, lib=None) -> float:
    k = _Keep()
    return (lib or _load()).or_dot(k.csr(X), i, k.csr(Z), j)


def sqnorm(X, i: int, lib=None) -> float:
    k = _Keep()
    return (lib or _load()).or_sqnorm(k.csr(X), i)


def kernel(gamma: float, nx: float, nz: float, dp: float, lib=None) -> float:
    return (lib or _load()).or_kernel(gamma, nx, nz, dp)


def _result(r: _Result) -> dict:
    return {"iters": r.iters, "b": r.b, "b_up": r.b_up, "b_low": r.b_low,
            "objective": r.objective, "n_shrink": r.n_shrink, "n_recon": r.n_recon,
            "final_active": r.final_active, "status": r.status}


def smo(X, y, C: float, gamma: float, tau: float, max_iter: int = 10**9,
        trace_len: int = 0, record_objective: bool = False, lib=None) -> dict:
    """Algorithm 1 without shrinking. Returns alpha, f, b, b_up, b_low, iters,
    objective, and when ``trace_len`` > 0 the first (i_up, i_low) pairs with
    their selection margins (second best minus best on each side)."""
    k = _Keep()
    n = int(X.n)
    alpha = np.zeros(n)
    f = np.zeros(n)
    res = _Result()
    trace = np.full((max(trace_len, 0), 2), -1, dtype=np.int64)
    margin = np.zeros((max(trace_len, 0), 2))
    objs = np.full(max(trace_len, 0), np.nan) if record_objective else None
    (lib or _load()).or_smo(k.csr(X), _ptr(k.arr(y, np.int8)), C, gamma, tau, int(max_iter),
                   _ptr(alpha), _ptr(f), ct.byref(res),
                   _ptr(trace) if trace_len else None,
                   _ptr(margin) if trace_len else None,
                   _ptr(objs) if objs is not None else None, int(trace_len))
    out = _result(res)
    out.update(alpha=alpha, f=f)
    if trace_len:
        m = min(trace_len, res.iters)
        out["trace"] = trace[:m]
        out["margin"] = margin[:m]
        if objs is not None:
            out["objectives"] = objs[:m]
    return out


def smo_wss2(X, y, C: float, gamma: float, tau: float, max_iter: int = 10**9,
             trace_len: int = 0, lib=None) -> dict:
    """SMO with the second-order choice of i_low (no shrinking). The trace's
    margins are, per step, the I_up margin (second best minus best f) and the
    chosen gain's relative lead over the runner-up."""
    k = _Keep()
    n = int(X.n)
    alpha = np.zeros(n)
    f = np.zeros(n)
    res = _Result()
    trace = np.full((max(trace_len, 0), 2), -1, dtype=np.int64)
    margin = np.zeros((max(trace_len, 0), 2))
    (lib or _load()).or_smo_wss2(k.csr(X), _ptr(k.arr(y, np.int8)), C, gamma, tau, int(max_iter),
                                 _ptr(alpha), _ptr(f), ct.byref(res),
                                 _ptr(trace) if trace_len else None,
                                 _ptr(margin) if trace_len else None, int(trace_len))
    out = _result(res)
    out.update(alpha=alpha, f=f)
    if trace_len:
        m = min(trace_len, res.iters)
        out["trace"] = trace[:m]
        out["margin"] = margin[:m]
    return out


def smo_shrink(X, y, C: float, gamma: float, tau: float, kind: int, value: float,
               recon: int, first_factor: float = 20.0, max_iter: int = 10**9,
               trace_len: int = 0, wss: int = 1, events: int = 0, lib=None) -> dict:
    """Algorithms 4/5 (+ the multiple-reconstruction variant) with Algorithm 6.
    ``wss=2`` chooses i_low by the second-order gain over the active rows.
    ``trace_len`` > 0 records per step the pair, the active-set size and the
    active-set gap (``trace``, ``active``, ``gap``); ``events`` > 0 records up
    to that many schedule events as rows (steps completed, kind 1 = shrink /
    2 = reconstruction, active rows after, triggering gap, gap over all rows
    after a reconstruction) in ``events`` (``n_events`` counts all)."""
    k = _Keep()
    n = int(X.n)
    alpha = np.zeros(n)
    f = np.zeros(n)
    res = _Result()
    trace = np.full((max(trace_len, 0), 2), -1, dtype=np.int64)
    act = np.zeros(max(trace_len, 0), dtype=np.int64)
    gap = np.full(max(trace_len, 0), np.nan)
    ev = np.full((max(events, 0), 3), -1, dtype=np.int64)
    evg = np.full((max(events, 0), 2), np.nan)
    nev = ct.c_int64(0)
    (lib or _load()).or_smo_shrink(k.csr(X), _ptr(k.arr(y, np.int8)), C, gamma, tau, int(max_iter),
                          int(kind), float(value), int(recon), float(first_factor),
                          _ptr(alpha), _ptr(f), ct.byref(res),
                          _ptr(trace) if trace_len else None, int(trace_len),
                          _ptr(act) if trace_len else None, int(wss),
                          _ptr(gap) if trace_len else None,
                          _ptr(ev) if events else None, _ptr(evg) if events else None,
                          int(events), ct.byref(nev))
    out = _result(res)
    out.update(alpha=alpha, f=f)
    if trace_len:
        m = min(trace_len, res.iters)
        out["trace"] = trace[:m]
        out["active"] = act[:m]
        out["gap"] = gap[:m]
    if events:
        m = min(events, nev.value)
        out["events"] = [{"step": int(ev[e, 0]), "kind": int(ev[e, 1]), "active": int(ev[e, 2]),
                          "gap": float(evg[e, 0]), "gap_all": float(evg[e, 1])} for e in range(m)]
        out["n_events"] = int(nev.value)
    return out


def gradient(X, y, alpha, gamma: float, lib=None) -> np.ndarray:
    """Eq. (fcache) from scratch."""
    k = _Keep()
    f = np.zeros(int(X.n))
    (lib or _load()).or_gradient(k.csr(X), _ptr(k.arr(y, np.int8)), _ptr(k.arr(alpha, np.float64)),
                        gamma, _ptr(f))
    return f


def reconstruct(X, y, alpha, gamma: float, rows, f_in, lib=None) -> np.ndarray:
    """Algorithm 6 on ``rows``; other entries of ``f_in`` are kept."""
    k = _Keep()
    f = np.array(f_in, dtype=np.float64, copy=True)
    rows = k.arr(rows, np.int64)
    (lib or _load()).or_reconstruct(k.csr(X), _ptr(k.arr(y, np.int8)), _ptr(k.arr(alpha, np.float64)),
                           gamma, len(rows), _ptr(rows), _ptr(f))
    return f


def kkt(X, y, alpha, C: float, gamma: float, lib=None) -> dict:
    """Recompute f from alpha and report b_up, b_low, gap, b and objective."""
    k = _Keep()
    f = np.zeros(int(X.n))
    res = _Result()
    (lib or _load()).or_kkt(k.csr(X), _ptr(k.arr(y, np.int8)), _ptr(k.arr(alpha, np.float64)),
                   C, gamma, _ptr(f), ct.byref(res))
    out = _result(res)
    out["f"] = f
    out["gap"] = res.b_low - res.b_up
    return out


def decision(X, y, alpha, b: float, gamma: float, Z, lib=None) -> np.ndarray:
    """Eq. (classi) before the sign."""
    k = _Keep()
    out = np.zeros(int(Z.n))
    (lib or _load()).or_decision(k.csr(X), _ptr(k.arr(y, np.int8)), _ptr(k.arr(alpha, np.float64)),
                        b, gamma, k.csr(Z), _ptr(out))
    return out
