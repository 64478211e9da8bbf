"""CPU oracle for EAPrunedDTW subsequence search (test infrastructure only).

This package wraps ``oracle.c``, a plain sequential FP64 restatement of the
method of Herrmann & Webb, "Early Abandoning PrunedDTW and its application to
similarity search" (Eq. 1-5, Algorithms 1-3, Section 5).  It is used by the
test-suite, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``.  The CUDA library never imports it and shares no code with it.

``build()`` compiles ``oracle.c`` with gcc into ``oracle/_build``; the other
functions call it through ctypes and take/return numpy float64 arrays.
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
_lib = None

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


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, no FMA contraction) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call([
        "gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
        "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread", "-lm",
    ])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


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
