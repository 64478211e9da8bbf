"""CPU oracle for EAPrunedDTW subsequence search (test infrastructure only).

This package wraps ``oracle.c``, a plain sequential FP64 restatement of the
method of Herrmann & Webb, "Early Abandoning PrunedDTW and its application to
similarity search" (Eq. 1-5, Algorithms 1-3, Section 5).  It is used by the
test-suite, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``.  The CUDA library never imports it and shares no code with it.

``build()`` compiles ``oracle.c`` with gcc into ``oracle/_build``; the other
functions call it through ctypes and take/return numpy float64 arrays.

The ``o7_*`` functions wrap ``oracle_f32.c``, the FP32-emulating mode: the same
search with the GPU's FP32/FP64 rounding reproduced operation by operation, so
that integer outcomes (pruning decisions, completed/abandoned DTWs, indices)
and FP32 distances compare bit for bit.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC_F32 = os.path.join(_HERE, "oracle_f32.c")
_LIB_F32 = os.path.join(_BUILD, "liboracle_f32.so")
_lib = None
_lib_f32 = None

_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


class EapTrace(C.Structure):
    _fields_ = [
        ("cells", C.c_int64),
        ("rows", C.c_int64),
        ("abandon_row", C.c_int64),
        ("next_start", _I64),
        ("pruning_point", _I64),
    ]


def _compile(src: str, out: str, force: bool) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call([
        "gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
        "-fPIC", "-shared", "-o", tmp, src, "-lpthread", "-lm",
    ])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c and oracle_f32.c (gcc, no FMA contraction); returns
    the path of the FP64 oracle's .so."""
    _compile(_SRC_F32, _LIB_F32, force)
    return _compile(_SRC, _LIB_PATH, force)


def _bind(L):
    L.orc_dtw_matrix.restype = C.c_double
    L.orc_dtw_matrix.argtypes = [_D, C.c_int64, _D, C.c_int64, C.c_int64, _D]
    L.orc_dtw_tworow.restype = C.c_double
    L.orc_dtw_tworow.argtypes = [_D, C.c_int64, _D, C.c_int64, C.c_int64]
    L.orc_dtw_prune_left.restype = C.c_double
    L.orc_dtw_prune_left.argtypes = [_D, C.c_int64, _D, C.c_int64, C.c_double, _I64]
    L.orc_eapruned_dtw.restype = C.c_double
    L.orc_eapruned_dtw.argtypes = [_D, C.c_int64, _D, C.c_int64, C.c_int64, C.c_double,
                                   C.POINTER(EapTrace)]
    L.orc_znorm.restype = None
    L.orc_znorm.argtypes = [_D, C.c_int64, _D]
    L.orc_mean_std.restype = None
    L.orc_mean_std.argtypes = [_D, C.c_int64, _D, _D]
    L.orc_envelope.restype = None
    L.orc_envelope.argtypes = [_D, C.c_int64, C.c_int64, _D, _D]
    L.orc_lb_kim_fl.restype = C.c_double
    L.orc_lb_kim_fl.argtypes = [_D, _D, C.c_int64]
    L.orc_lb_keogh.restype = C.c_double
    L.orc_lb_keogh.argtypes = [_D, _D, _D, C.c_int64]
    L.orc_search_brute.restype = C.c_int
    L.orc_search_brute.argtypes = [_D, C.c_int64, _D, C.c_int64, C.c_int64, C.c_int32,
                                   _I64, _D]
    L.orc_search_cascade.restype = C.c_int
    L.orc_search_cascade.argtypes = [_D, C.c_int64, _D, C.c_int64, C.c_int64, C.c_int32,
                                     C.c_int, C.c_double, C.c_int, _I64, _D, _I64]
    L.orc_window_stats.restype = None
    L.orc_window_stats.argtypes = [_D, C.c_int64, C.c_int64, _D, _D]
    if hasattr(L, "orc_dtw_cost"):
        L.orc_dtw_cost.restype = C.c_double
        L.orc_dtw_cost.argtypes = [_D, C.c_int64, _D, C.c_int64, C.c_int64, C.c_int]
        L.orc_search_brute_cost.restype = C.c_int
        L.orc_search_brute_cost.argtypes = [_D, C.c_int64, _D, C.c_int64, C.c_int64, C.c_int32, C.c_int,
                                            _I64, _D]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def compile_variant(src_text: str, out_dir: str) -> str:
    """Compile a modified copy of oracle.c (used by the tests that plant a
    mistake in the oracle to show that its pins catch it)."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "oracle_variant.c")
    so = os.path.join(out_dir, "liboracle_variant.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                           "-fPIC", "-shared", "-o", so, src, "-lpthread", "-lm"])
    return so


class use_library:
    """Context manager: route this module's functions to another build of oracle.c."""

    def __init__(self, so_path: str):
        self.so_path = so_path

    def __enter__(self):
        global _lib
        self._saved = _lib
        _lib = _bind(C.CDLL(self.so_path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def dtw_matrix(S, T, w: int | None = None):
    """Eq. 1-5: (DTW, full (lS+1)x(lT+1) matrix with borders)."""
    S, T = _f64(S), _f64(T)
    if w is None:
        w = max(len(S), len(T))
    M = np.empty((len(S) + 1, len(T) + 1), dtype=np.float64)
    d = lib().orc_dtw_matrix(_p(S), len(S), _p(T), len(T), int(w), _p(M))
    return d, M


def dtw(S, T, w: int | None = None) -> float:
    """Algorithm 1 (two rows), banded |i-j| <= w; w=None is unconstrained."""
    S, T = _f64(S), _f64(T)
    if w is None:
        w = max(len(S), len(T))
    return lib().orc_dtw_tworow(_p(S), len(S), _p(T), len(T), int(w))


def dtw_prune_left(S, T, ub: float):
    """Algorithm 2 (no window): (value, 1-based abandon row or 0)."""
    S, T = _f64(S), _f64(T)
    row = C.c_int64(0)
    d = lib().orc_dtw_prune_left(_p(S), len(S), _p(T), len(T), float(ub), C.byref(row))
    return d, row.value


def eapruned_dtw(S, T, w: int | None = None, ub: float = np.inf, trace: bool = False):
    """Algorithm 3 (EAPrunedDTW).  Returns the value, or (value, info) with
    trace=True where info has cells, rows, abandon_row, next_start[], pruning_point[]."""
    S, T = _f64(S), _f64(T)
    if w is None:
        w = max(len(S), len(T))
    rows = max(len(S), len(T))
    ns = np.zeros(rows, dtype=np.int64)
    pp = np.zeros(rows, dtype=np.int64)
    tr = EapTrace(0, 0, 0, ns.ctypes.data_as(_I64), pp.ctypes.data_as(_I64))
    d = lib().orc_eapruned_dtw(_p(S), len(S), _p(T), len(T), int(w), float(ub), C.byref(tr))
    if not trace:
        return d
    n = tr.rows
    return d, {"cells": tr.cells, "rows": tr.rows, "abandon_row": tr.abandon_row,
               "next_start": ns[:n].copy(), "pruning_point": pp[:n].copy()}


def znorm(x) -> np.ndarray:
    x = _f64(x)
    z = np.empty_like(x)
    lib().orc_znorm(_p(x), len(x), _p(z))
    return z


def mean_std(x):
    x = _f64(x)
    mu, sd = C.c_double(0), C.c_double(0)
    lib().orc_mean_std(_p(x), len(x), C.byref(mu), C.byref(sd))
    return mu.value, sd.value


def window_stats(R, m: int):
    R = _f64(R)
    nw = len(R) - m + 1
    mu = np.empty(nw)
    sd = np.empty(nw)
    lib().orc_window_stats(_p(R), len(R), int(m), _p(mu), _p(sd))
    return mu, sd


def envelope(x, w: int):
    x = _f64(x)
    U = np.empty_like(x)
    L = np.empty_like(x)
    lib().orc_envelope(_p(x), len(x), int(w), _p(U), _p(L))
    return U, L


def lb_kim_fl(zc, zq) -> float:
    zc, zq = _f64(zc), _f64(zq)
    return lib().orc_lb_kim_fl(_p(zc), _p(zq), len(zq))


def lb_keogh(x, U, L) -> float:
    x, U, L = _f64(x), _f64(U), _f64(L)
    return lib().orc_lb_keogh(_p(x), _p(U), _p(L), len(x))


def search_brute(Q, R, w: int, k: int = 1):
    """O5: every window, z-normalised, full banded DTW; k smallest (idx, dist)."""
    Q, R = _f64(Q), _f64(R)
    idx = np.empty(k, dtype=np.int64)
    dist = np.empty(k, dtype=np.float64)
    rc = lib().orc_search_brute(_p(Q), len(Q), _p(R), len(R), int(w), int(k),
                                idx.ctypes.data_as(_I64), _p(dist))
    if rc != 0:
        raise ValueError("invalid arguments")
    return idx, dist


COUNTER_NAMES = ("windows", "kim_pruned", "eq_pruned", "ec_pruned",
                 "dtw_abandoned", "dtw_completed", "cells")



COST_SQUARED, COST_ABSOLUTE = 0, 1


def dtw_cost(S, T, w: int | None = None, cost: int = COST_SQUARED) -> float:
    """DTW of Eq. 1-4 with the pointwise cost (a-b)^2 (cost 0) or |a-b| (cost 1)."""
    S, T = _f64(S), _f64(T)
    if w is None:
        w = max(len(S), len(T))
    return float(lib().orc_dtw_cost(_p(S), len(S), _p(T), len(T), int(w), int(cost)))


def search_brute_cost(Q, R, w: int, k: int = 1, cost: int = COST_SQUARED):
    """Brute-force k-NN subsequence search with the given pointwise cost."""
    Q, R = _f64(Q), _f64(R)
    idx = np.empty(k, dtype=np.int64)
    dist = np.empty(k)
    rc = lib().orc_search_brute_cost(_p(Q), len(Q), _p(R), len(R), int(w), int(k), int(cost),
                                     idx.ctypes.data_as(_I64), _p(dist))
    if rc != 0:
        raise ValueError("search_brute_cost: invalid arguments")
    return idx, dist

def search_cascade(Q, R, w: int, k: int = 1, use_lb: bool = True, ub_fixed: float = np.nan,
                   nthreads: int = 1):
    """O6: LB_Kim -> LB_Keogh EQ -> EC -> EAPrunedDTW.  Returns (idx, dist, counters)."""
    Q, R = _f64(Q), _f64(R)
    idx = np.empty(k, dtype=np.int64)
    dist = np.empty(k, dtype=np.float64)
    cnt = np.zeros(7, dtype=np.int64)
    rc = lib().orc_search_cascade(_p(Q), len(Q), _p(R), len(R), int(w), int(k), int(use_lb),
                                  float(ub_fixed), int(nthreads),
                                  idx.ctypes.data_as(_I64), _p(dist),
                                  cnt.ctypes.data_as(_I64))
    if rc != 0:
        raise ValueError("invalid arguments")
    return idx, dist, dict(zip(COUNTER_NAMES, (int(c) for c in cnt)))


# ---------------------------------------------------------------------------
# FP32-emulating mode (oracle_f32.c)
# ---------------------------------------------------------------------------
_F = C.POINTER(C.c_float)
_I32 = C.POINTER(C.c_int32)


def _bind_f32(L):
    L.o7_rsqrt_rn.restype = C.c_float
    L.o7_rsqrt_rn.argtypes = [C.c_float]
    L.o7_ref_prefix.restype = None
    L.o7_ref_prefix.argtypes = [_F, C.c_int64, _D, _D, _D, _D, _F]
    L.o7_window_coeffs.restype = None
    L.o7_window_coeffs.argtypes = [_F, C.c_int64, _D, _D, _D, _D, _F, C.c_int64, C.c_int64, _F, _F, _F]
    L.o7_query_prep.restype = None
    L.o7_query_prep.argtypes = [_F, C.c_int64, C.c_int64, _F, _F, _F, _F, _I32]
    L.o7_dtw_f32.restype = C.c_float
    L.o7_dtw_f32.argtypes = [_F, _F, C.c_int64, C.c_int64]
    L.o7_search.restype = C.c_int
    L.o7_search.argtypes = [_F, C.c_int64, _F, C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_float, C.c_int,
                            _I64, _I64, _D, C.POINTER(C.c_int8)]
    return L


def lib_f32():
    global _lib_f32
    if _lib_f32 is None:
        build()
        _lib_f32 = _bind_f32(C.CDLL(_LIB_F32))
    return _lib_f32


def compile_variant_f32(src_text: str, out_dir: str):
    """A modified copy of oracle_f32.c, bound like lib_f32() (mutation tests)."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "oracle_f32_variant.c")
    so = os.path.join(out_dir, "liboracle_f32_variant.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                           "-fPIC", "-shared", "-o", so, src, "-lm"])
    return _bind_f32(C.CDLL(so))


def source_text_f32() -> str:
    with open(_SRC_F32) as f:
        return f.read()


def _f32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def _pf(a: np.ndarray):
    return a.ctypes.data_as(_F)


O7_COUNTER_NAMES = ("windows", "kim_pruned", "eq_pruned", "ec_pruned", "dtw_abandoned", "dtw_completed")


def o7_rsqrt_rn(v: float, L=None) -> float:
    """Correctly rounded FP32 1/sqrt(v) (v > 0 finite)."""
    return float((L or lib_f32()).o7_rsqrt_rn(C.c_float(v)))


def o7_ref_prefix(R, L=None):
    """Chunk-anchored prefix sums in the GPU's order: (P1, P2, T1, T2, A)."""
    R = _f32(R)
    n = len(R)
    nch = (n + 4095) // 4096
    P1, P2 = np.empty(n), np.empty(n)
    T1, T2 = np.empty(nch), np.empty(nch)
    A = np.empty(nch, dtype=np.float32)
    (L or lib_f32()).o7_ref_prefix(_pf(R), n, _p(P1), _p(P2), _p(T1), _p(T2), _pf(A))
    return P1, P2, T1, T2, A


def o7_window_coeffs(R, m: int, windows=None, L=None):
    """(a, cw, isd) FP32 arrays of the given windows (default: all)."""
    L = L or lib_f32()
    R = _f32(R)
    P1, P2, T1, T2, A = o7_ref_prefix(R, L)
    idx = range(len(R) - m + 1) if windows is None else windows
    out = np.empty((len(idx), 3), dtype=np.float32)
    a, cw, isd = C.c_float(), C.c_float(), C.c_float()
    for r, i in enumerate(idx):
        L.o7_window_coeffs(_pf(R), len(R), _p(P1), _p(P2), _p(T1), _p(T2), _pf(A), int(i), int(m),
                           C.byref(a), C.byref(cw), C.byref(isd))
        out[r] = (a.value, cw.value, isd.value)
    return out


def o7_query_prep(Q, w: int, L=None):
    """(zq, uq, lq, zq in LB order, order) as the GPU prepares the query."""
    Q = _f32(Q)
    m = len(Q)
    zq, uq, lq, zqo = (np.empty(m, dtype=np.float32) for _ in range(4))
    ord_ = np.empty(m, dtype=np.int32)
    (L or lib_f32()).o7_query_prep(_pf(Q), m, int(w), _pf(zq), _pf(uq), _pf(lq), _pf(zqo),
                                   ord_.ctypes.data_as(_I32))
    return zq, uq, lq, zqo, ord_


def o7_dtw_f32(z, q, w: int, L=None) -> float:
    """FP32 DTW of Eq. 1-5 (fma cells) of two equal-length normalised series."""
    z, q = _f32(z), _f32(q)
    return float((L or lib_f32()).o7_dtw_f32(_pf(z), _pf(q), len(z), int(w)))


def o7_search(Q, R, w: int, k: int = 1, audit_ub: float | None = None, use_lb: bool = True, L=None,
              return_why: bool = False):
    """FP32-emulated search: exact top-k (audit_ub None) or the audit cascade under
    the fixed bound audit_ub.  Returns (idx, dist, counters dict), plus with
    return_why each window's outcome (int8: 1 LB_Kim, 2 LB_Keogh EQ, 3 LB_Keogh
    EC, 4 abandoned, 5 completed)."""
    Q, R = _f32(Q), _f32(R)
    idx = np.empty(k, dtype=np.int64)
    dist = np.empty(k)
    cnt = np.zeros(6, dtype=np.int64)
    audit = audit_ub is not None
    why = np.zeros(len(R) - len(Q) + 1, dtype=np.int8) if return_why else None
    rc = (L or lib_f32()).o7_search(_pf(Q), len(Q), _pf(R), len(R), int(w), int(k), int(audit),
                                    C.c_float(float(audit_ub) if audit else 0.0), int(bool(use_lb)),
                                    cnt.ctypes.data_as(_I64), idx.ctypes.data_as(_I64), _p(dist),
                                    why.ctypes.data_as(C.POINTER(C.c_int8)) if return_why else None)
    if rc != 0:
        raise ValueError("o7_search: invalid arguments")
    out = (idx, dist, dict(zip(O7_COUNTER_NAMES, (int(c) for c in cnt))))
    return out + (why,) if return_why else out
