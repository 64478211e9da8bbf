"""Python binding of libeapdtw.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/eapdtw.h; all
computation runs in the library's CUDA kernels.  Device-array functions take
CUDA float32 tensors; the *_host functions take numpy arrays.  If the library
is not built, the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import re

import numpy as np

from . import build as _build

_lib = None

_HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                       "eapdtw.h")

NCOUNTERS = 18
COUNTER_NAMES = ("windows", "kim_pruned", "eq_pruned", "ec_pruned", "dtw_abandoned",
                 "dtw_completed", "cells", "lb_recheck", "overflow", "steps", "ns_main",
                 "ns_wider", "ns_prep", "ns_seed", "ns_total", "launches", "probe_overflow",
                 "first_tile")


class SearchOpts(C.Structure):
    _fields_ = [
        ("no_lb", C.c_int32),
        ("tile", C.c_int32),
        ("no_seed", C.c_int32),
        ("audit", C.c_int32),
        ("ub_fixed", C.c_double),
        ("counters", C.POINTER(C.c_int64)),
        ("tighten", C.c_int32),
        ("cost", C.c_int32),
        ("reserved", C.c_int32 * 6),
    ]


class Item(C.Structure):
    """eapdtw_item of include/eapdtw.h."""
    _fields_ = [
        ("Q", C.c_void_p),
        ("lQ", C.c_int64),
        ("w", C.c_int64),
        ("ref_id", C.c_int32),
        ("k", C.c_int32),
        ("no_lb", C.c_int32),
        ("reserved", C.c_int32),
    ]


PENDING = 1
SERVE_STAT_NAMES = ("completed", "cancelled", "queued", "admitted", "rounds", "windows", "p50_ns", "p99_ns",
                    "reruns", "error")

CTX_INFO_NAMES = ("bytes_held", "budget", "live_refs", "arena_bytes", "batches", "items_run",
                  "items_rerun", "graph_captured")


class EapDtwError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libeapdtw.so (it must have been built by build.build())."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2010_05371_gb300.build.build()")
        L = C.CDLL(path)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        L.eapdtw_strerror.restype = C.c_char_p
        L.eapdtw_strerror.argtypes = [i32]
        L.eapdtw_version.restype = C.c_char_p
        L.eapdtw_version.argtypes = []
        L.eap_dtw.restype = i32
        L.eap_dtw.argtypes = [vp, i64, vp, i64, i64, dbl, vp, vp]
        L.eap_dtw_host.restype = i32
        L.eap_dtw_host.argtypes = [vp, i64, vp, i64, i64, dbl, C.POINTER(dbl)]
        L.subseq_search.restype = i32
        L.subseq_search.argtypes = [vp, i64, vp, i64, i64, i32, vp, vp, vp]
        L.subseq_search_ex.restype = i32
        L.subseq_search_ex.argtypes = [vp, i64, vp, i64, i64, i32, C.POINTER(SearchOpts), vp, vp, vp]
        L.subseq_search_host.restype = i32
        L.subseq_search_host.argtypes = [vp, i64, vp, i64, i64, i32, C.POINTER(SearchOpts), vp, vp]
        L.eapdtw_release_scratch.restype = i32
        L.eapdtw_release_scratch.argtypes = []
        L.subseq_search_noalloc.restype = i32
        L.subseq_search_noalloc.argtypes = [vp, i64, vp, i64, i64, i32, vp, vp, vp]
        L.eapdtw_cell_peak.restype = i32
        L.eapdtw_cell_peak.argtypes = [i32, i64, C.POINTER(dbl), C.POINTER(dbl)]
        pi32 = C.POINTER(i32)
        L.eapdtw_ctx_create.restype = i32
        L.eapdtw_ctx_create.argtypes = [i32, i64, C.POINTER(vp)]
        L.eapdtw_ctx_destroy.restype = i32
        L.eapdtw_ctx_destroy.argtypes = [vp]
        L.eapdtw_ref_register.restype = i32
        L.eapdtw_ref_register.argtypes = [vp, vp, i64, pi32, vp]
        L.eapdtw_ref_unregister.restype = i32
        L.eapdtw_ref_unregister.argtypes = [vp, i32]
        L.eapdtw_ref_info.restype = i32
        L.eapdtw_ref_info.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(i64)]
        L.eapdtw_ctx_info.restype = i32
        L.eapdtw_ctx_info.argtypes = [vp, C.POINTER(i64), i32]
        L.eapdtw_search_batch.restype = i32
        L.eapdtw_search_batch.argtypes = [vp, C.POINTER(Item), i32, i32, vp, vp, C.POINTER(i64), vp]
        L.eapdtw_set_first_tile.restype = i32
        L.eapdtw_set_first_tile.argtypes = [vp, i32, i32, i32, i32]
        L.eapdtw_get_first_tile.restype = i32
        L.eapdtw_get_first_tile.argtypes = [vp, i32, i32, i32, pi32]
        L.eapdtw_set_tuning.restype = i32
        L.eapdtw_set_tuning.argtypes = [vp, i32, i32, i32, i32, i32]
        L.eapdtw_get_tuning.restype = i32
        L.eapdtw_get_tuning.argtypes = [vp, i32, i32, i32, pi32, pi32]
        L.eapdtw_autotune.restype = i32
        L.eapdtw_autotune.argtypes = [vp, C.POINTER(Item), i32, i64, vp, pi32]
        pi64 = C.POINTER(i64)
        L.eapdtw_pairwise.restype = i32
        L.eapdtw_pairwise.argtypes = [vp, i64, vp, i64, i64, i64, i32, vp, vp]
        L.eapdtw_nn.restype = i32
        L.eapdtw_nn.argtypes = [vp, i64, vp, i64, i64, i64, i32, i32, vp, vp, vp]
        L.eapdtw_serve_start.restype = i32
        L.eapdtw_serve_start.argtypes = [vp, i32, i64]
        L.eapdtw_serve_stop.restype = i32
        L.eapdtw_serve_stop.argtypes = [vp]
        L.eapdtw_serve_submit.restype = i32
        L.eapdtw_serve_submit.argtypes = [vp, vp, i64, i32, i64, i32, i32, pi64]
        L.eapdtw_serve_poll.restype = i32
        L.eapdtw_serve_poll.argtypes = [vp, i64, vp, vp, pi64, i32]
        L.eapdtw_serve_cancel.restype = i32
        L.eapdtw_serve_cancel.argtypes = [vp, i64]
        L.eapdtw_serve_stats.restype = i32
        L.eapdtw_serve_stats.argtypes = [vp, pi64, i32]
        _lib = L
    return _lib


def header_functions(path: str = _HEADER):
    """Names of the functions declared in include/eapdtw.h."""
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                      text, flags=re.M)


def strerror(code: int) -> str:
    return lib().eapdtw_strerror(int(code)).decode()


def version() -> str:
    return lib().eapdtw_version().decode()


def _check(rc: int, what: str):
    if rc != 0:
        raise EapDtwError(rc, what)


def _dev_f32(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous")
    return t


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def eap_dtw(S, T, w: int | None = None, ub: float = math.inf, out=None, stream=None):
    """DTW_w(S, T) if <= ub else +inf (Algorithm 3), on raw CUDA float32 series.
    Returns a 0-d float64 CUDA tensor (asynchronous on the stream)."""
    import torch
    S, T = _dev_f32(S, "S"), _dev_f32(T, "T")
    if w is None:
        w = max(S.numel(), T.numel())
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=S.device)
    rc = lib().eap_dtw(C.c_void_p(S.data_ptr()), S.numel(), C.c_void_p(T.data_ptr()), T.numel(),
                       int(w), float(ub), C.c_void_p(out.data_ptr()), _stream_ptr(stream))
    _check(rc, "eap_dtw")
    return out


def eap_dtw_host(S, T, w: int | None = None, ub: float = math.inf) -> float:
    S = np.ascontiguousarray(S, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    if w is None:
        w = max(len(S), len(T))
    out = C.c_double(0.0)
    rc = lib().eap_dtw_host(S.ctypes.data, len(S), T.ctypes.data, len(T), int(w), float(ub),
                            C.byref(out))
    _check(rc, "eap_dtw_host")
    return out.value


COST_SQUARED, COST_ABSOLUTE = 0, 1


def _opts(no_lb, tile, no_seed, audit_ub, counters, tighten=False, cost=0):
    o = SearchOpts()
    o.no_lb = int(bool(no_lb))
    o.tighten = int(bool(tighten))
    o.cost = int(cost)
    o.tile = int(tile)
    o.no_seed = int(bool(no_seed))
    o.audit = int(audit_ub is not None)
    o.ub_fixed = float(audit_ub) if audit_ub is not None else 0.0
    o.counters = counters.ctypes.data_as(C.POINTER(C.c_int64))
    return o


def subseq_search(Q, R, w: int, k: int = 1, *, no_lb: bool = False, tile: int = 0,
                  no_seed: bool = False, audit_ub: float | None = None, out=None, stream=None,
                  return_counters: bool = False, tighten: bool = False, cost: int = 0):
    """k nearest z-normalised subsequences of R to Q under DTW_w (Section 5).

    Q, R: CUDA float32 tensors.  Returns (idx int64[k], dist float64[k]) CUDA
    tensors, plus a counter dict when return_counters=True.  Blocking."""
    import torch
    Q, R = _dev_f32(Q, "Q"), _dev_f32(R, "R")
    if out is None:
        idx = torch.empty(k, dtype=torch.int64, device=Q.device)
        dist = torch.empty(k, dtype=torch.float64, device=Q.device)
    else:
        idx, dist = out
    cnt = np.zeros(NCOUNTERS, dtype=np.int64)
    o = _opts(no_lb, tile, no_seed, audit_ub, cnt, tighten, cost)
    rc = lib().subseq_search_ex(C.c_void_p(Q.data_ptr()), Q.numel(), C.c_void_p(R.data_ptr()),
                                R.numel(), int(w), int(k), C.byref(o), C.c_void_p(idx.data_ptr()),
                                C.c_void_p(dist.data_ptr()), _stream_ptr(stream))
    _check(rc, "subseq_search")
    if return_counters:
        return idx, dist, dict(zip(COUNTER_NAMES, (int(c) for c in cnt)))
    return idx, dist


def subseq_search_host(Q, R, w: int, k: int = 1, *, no_lb: bool = False, tile: int = 0,
                       no_seed: bool = False, audit_ub: float | None = None,
                       return_counters: bool = False):
    """subseq_search on host (numpy) arrays: copies in, searches, copies out."""
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    R = np.ascontiguousarray(R, dtype=np.float32)
    idx = np.empty(k, dtype=np.int64)
    dist = np.empty(k, dtype=np.float64)
    cnt = np.zeros(NCOUNTERS, dtype=np.int64)
    o = _opts(no_lb, tile, no_seed, audit_ub, cnt)
    rc = lib().subseq_search_host(Q.ctypes.data, len(Q), R.ctypes.data, len(R), int(w), int(k),
                                  C.byref(o), idx.ctypes.data, dist.ctypes.data)
    _check(rc, "subseq_search_host")
    if return_counters:
        return idx, dist, dict(zip(COUNTER_NAMES, (int(c) for c in cnt)))
    return idx, dist


def subseq_search_noalloc(Q, R, w: int, idx, dist, stream=None):
    """subseq_search into caller-provided idx (int64[k]) and dist (float64[k])
    CUDA tensors, through the entry point that allocates nothing (for callers
    that cannot allocate device memory).  k = idx.numel().  Blocking."""
    Q, R = _dev_f32(Q, "Q"), _dev_f32(R, "R")
    k = idx.numel()
    rc = lib().subseq_search_noalloc(C.c_void_p(Q.data_ptr()), Q.numel(), C.c_void_p(R.data_ptr()),
                                     R.numel(), int(w), int(k), C.c_void_p(idx.data_ptr()),
                                     C.c_void_p(dist.data_ptr()), _stream_ptr(stream))
    _check(rc, "subseq_search_noalloc")
    return idx, dist


def cell_peak(mode: int, steps: int = 1 << 18):
    """Measured DP-cell throughput ceiling (eapdtw_cell_peak): (cells/s, ms)."""
    rate, ms = C.c_double(), C.c_double()
    _check(lib().eapdtw_cell_peak(int(mode), int(steps), C.byref(rate), C.byref(ms)), "eapdtw_cell_peak")
    return rate.value, ms.value


def _series_2d(X, name):
    import torch
    X = _dev_f32(X, name)
    if X.dim() != 2:
        raise TypeError(f"{name} must be a 2-D tensor (series x points)")
    return X


def pairwise(A, B, w: int | None = None, *, znorm: bool = True, stream=None):
    """DTW_w of every pair of rows (A_i, B_j) as a (len(A), len(B)) float64 CUDA
    tensor; each pair pruned under its own diagonal cost (no external bound)."""
    import torch
    A, B = _series_2d(A, "A"), _series_2d(B, "B")
    if A.shape[1] != B.shape[1]:
        raise ValueError("A and B rows must have the same length")
    L = A.shape[1]
    out = torch.empty((A.shape[0], B.shape[0]), dtype=torch.float64, device=A.device)
    rc = lib().eapdtw_pairwise(C.c_void_p(A.data_ptr()), A.shape[0], C.c_void_p(B.data_ptr()), B.shape[0], L,
                               int(L if w is None else w), int(bool(znorm)), C.c_void_p(out.data_ptr()),
                               _stream_ptr(stream))
    _check(rc, "eapdtw_pairwise")
    return out


def nearest_series(train, test, w: int | None = None, k: int = 1, *, znorm: bool = True, stream=None):
    """The k nearest rows of train (by DTW_w) of every row of test: (idx, dist)
    CUDA tensors of shape (len(test), k); 1-NN classification for k = 1."""
    import torch
    train, test = _series_2d(train, "train"), _series_2d(test, "test")
    if train.shape[1] != test.shape[1]:
        raise ValueError("train and test rows must have the same length")
    L = train.shape[1]
    idx = torch.empty((test.shape[0], k), dtype=torch.int64, device=test.device)
    dist = torch.empty((test.shape[0], k), dtype=torch.float64, device=test.device)
    rc = lib().eapdtw_nn(C.c_void_p(train.data_ptr()), train.shape[0], C.c_void_p(test.data_ptr()), test.shape[0],
                         L, int(L if w is None else w), int(k), int(bool(znorm)), C.c_void_p(idx.data_ptr()),
                         C.c_void_p(dist.data_ptr()), _stream_ptr(stream))
    _check(rc, "eapdtw_nn")
    return idx, dist


def release_scratch():
    _check(lib().eapdtw_release_scratch(), "eapdtw_release_scratch")


class Context:
    """A context of include/eapdtw.h: references resident on one device and the
    batched search over many (query, reference) items."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        h = C.c_void_p()
        _check(lib().eapdtw_ctx_create(int(device), int(mem_budget), C.byref(h)), "eapdtw_ctx_create")
        self._h = h
        self.device = int(device)
        self._refs = {}

    def close(self):
        if self._h is not None and self._h.value:
            _check(lib().eapdtw_ctx_destroy(self._h), "eapdtw_ctx_destroy")
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, R, stream=None) -> int:
        """Copy the CUDA float32 series R into the context; returns its id."""
        R = _dev_f32(R, "R")
        rid = C.c_int32(-1)
        _check(lib().eapdtw_ref_register(self._h, C.c_void_p(R.data_ptr()), R.numel(), C.byref(rid),
                                         _stream_ptr(stream)), "eapdtw_ref_register")
        self._refs[rid.value] = R.numel()
        return rid.value

    def unregister(self, ref_id: int):
        _check(lib().eapdtw_ref_unregister(self._h, int(ref_id)), "eapdtw_ref_unregister")
        self._refs.pop(int(ref_id), None)

    def ref_length(self, ref_id: int) -> int:
        n = C.c_int64(0)
        _check(lib().eapdtw_ref_info(self._h, int(ref_id), None, C.byref(n)), "eapdtw_ref_info")
        return n.value

    def info(self) -> dict:
        out = (C.c_int64 * len(CTX_INFO_NAMES))()
        _check(lib().eapdtw_ctx_info(self._h, out, len(CTX_INFO_NAMES)), "eapdtw_ctx_info")
        return dict(zip(CTX_INFO_NAMES, (int(v) for v in out)))

    @staticmethod
    def _items(items):
        """items: sequence of (Q, ref_id, w, k) or (Q, ref_id, w, k, no_lb)."""
        arr = (Item * len(items))()
        keep = []
        for i, t in enumerate(items):
            Q = _dev_f32(t[0], "Q")
            keep.append(Q)
            arr[i].Q = Q.data_ptr()
            arr[i].lQ = Q.numel()
            arr[i].ref_id = int(t[1])
            arr[i].w = int(t[2])
            arr[i].k = int(t[3])
            arr[i].no_lb = int(bool(t[4])) if len(t) > 4 else 0
            arr[i].reserved = 0
        return arr, keep

    def search_batch(self, items, kstride: int | None = None, *, out=None, stream=None,
                     return_counters: bool = False):
        """Run every item; returns (idx int64[n, kstride], dist float64[n, kstride])
        CUDA tensors (row i: item i's k results, then (-1, +inf)).  Blocking."""
        import torch
        n = len(items)
        if n == 0:
            raise ValueError("empty batch")
        arr, keep = self._items(items)
        if kstride is None:
            kstride = max(int(t[3]) for t in items)
        if out is None:
            dev = torch.device("cuda", self.device)
            idx = torch.empty((n, kstride), dtype=torch.int64, device=dev)
            dist = torch.empty((n, kstride), dtype=torch.float64, device=dev)
        else:
            idx, dist = out
        cnt = np.zeros(NCOUNTERS, dtype=np.int64)
        rc = lib().eapdtw_search_batch(self._h, arr, n, int(kstride), C.c_void_p(idx.data_ptr()),
                                       C.c_void_p(dist.data_ptr()), cnt.ctypes.data_as(C.POINTER(C.c_int64)),
                                       _stream_ptr(stream))
        del keep
        _check(rc, "eapdtw_search_batch")
        if return_counters:
            return idx, dist, dict(zip(COUNTER_NAMES, (int(c) for c in cnt)))   # 0..9 summed, ns_total timed
        return idx, dist

    def autotune(self, items, sample_windows: int = 1 << 18, stream=None) -> int:
        """Time the first-level tile choices for the items' signatures (see
        eapdtw_autotune); returns the number of signatures entered."""
        arr, keep = self._items(items)
        nt = C.c_int32(0)
        rc = lib().eapdtw_autotune(self._h, arr, len(items), int(sample_windows), _stream_ptr(stream),
                                   C.byref(nt))
        del keep
        _check(rc, "eapdtw_autotune")
        return nt.value

    def set_first_tile(self, log2_m: int, ratio_tenths: int, band: int, tile: int):
        _check(lib().eapdtw_set_first_tile(self._h, int(log2_m), int(ratio_tenths), int(band), int(tile)),
               "eapdtw_set_first_tile")

    def get_first_tile(self, log2_m: int, ratio_tenths: int, band: int) -> int:
        t = C.c_int32(0)
        _check(lib().eapdtw_get_first_tile(self._h, int(log2_m), int(ratio_tenths), int(band), C.byref(t)),
               "eapdtw_get_first_tile")
        return t.value

    # ---- serving loop -----------------------------------------------------
    def serve_start(self, max_active: int = 64, chunk_windows: int = 1 << 22):
        """Start the context's server thread (continuous batching in rounds)."""
        _check(lib().eapdtw_serve_start(self._h, int(max_active), int(chunk_windows)), "eapdtw_serve_start")

    def serve_stop(self):
        _check(lib().eapdtw_serve_stop(self._h), "eapdtw_serve_stop")

    def submit(self, Q, ref_id: int, w: int, k: int = 1, no_lb: bool = False) -> int:
        """Queue a request (Q: host array, copied); returns its id."""
        q = np.ascontiguousarray(Q, dtype=np.float32)
        rid = C.c_int64(0)
        _check(lib().eapdtw_serve_submit(self._h, q.ctypes.data, len(q), int(ref_id), int(w), int(k),
                                         int(bool(no_lb)), C.byref(rid)), "eapdtw_serve_submit")
        return rid.value

    def poll(self, req_id: int, k: int, timeout_ms: int = 0):
        """None while the request runs; else (idx[k], dist[k], latency_ns), releasing it.
        Raises EapDtwError if the request failed or was cancelled."""
        idx = np.empty(k, dtype=np.int64)
        dist = np.empty(k, dtype=np.float64)
        lat = C.c_int64(0)
        rc = lib().eapdtw_serve_poll(self._h, int(req_id), idx.ctypes.data, dist.ctypes.data, C.byref(lat),
                                     int(timeout_ms))
        if rc == PENDING:
            return None
        _check(rc, "eapdtw_serve_poll")
        return idx, dist, lat.value

    def cancel(self, req_id: int):
        _check(lib().eapdtw_serve_cancel(self._h, int(req_id)), "eapdtw_serve_cancel")

    def serve_stats(self) -> dict:
        out = (C.c_int64 * len(SERVE_STAT_NAMES))()
        _check(lib().eapdtw_serve_stats(self._h, out, len(SERVE_STAT_NAMES)), "eapdtw_serve_stats")
        return dict(zip(SERVE_STAT_NAMES, (int(v) for v in out)))

    # ---- autotuner table: persisted per GPU model ---------------------------
    def set_tuning(self, log2_m: int, ratio_tenths: int, band: int, tile: int, check_double: int):
        """The autotuner's choice for a signature: first-level tile and check interval (0/1)."""
        _check(lib().eapdtw_set_tuning(self._h, log2_m, ratio_tenths, band, tile, check_double),
               "eapdtw_set_tuning")

    def get_tuning(self, log2_m: int, ratio_tenths: int, band: int):
        t, c = C.c_int32(), C.c_int32()
        _check(lib().eapdtw_get_tuning(self._h, log2_m, ratio_tenths, band, C.byref(t), C.byref(c)),
               "eapdtw_get_tuning")
        return t.value, c.value

    def tuning_table(self) -> dict:
        """The choices in effect: {(log2_m, ratio_tenths, band): (tile, check_double)}."""
        out = {}
        for lg in range(13):
            for tenth in range(11):
                for band in (0, 1):
                    t, c = self.get_tuning(lg, tenth, band)
                    if t or c:
                        out[(lg, tenth, band)] = (t, c)
        return out

    def save_tuning(self, path: str):
        """Write the tuning table to a JSON file, keyed by this device's name."""
        import json
        import torch
        entries = [[lg, tenth, band, tile, chk] for (lg, tenth, band), (tile, chk) in sorted(self.tuning_table().items())]
        with open(path, "w") as f:
            json.dump({"device": torch.cuda.get_device_name(self.device), "entries": entries}, f, indent=1)

    def load_tuning(self, path: str) -> int:
        """Load a table written by save_tuning on the same GPU model; returns the
        number of entries set (0 if the file was written on another model)."""
        import json
        import torch
        with open(path) as f:
            data = json.load(f)
        if data.get("device") != torch.cuda.get_device_name(self.device):
            return 0
        for e in data.get("entries", []):
            lg, tenth, band, tile = e[:4]
            self.set_tuning(lg, tenth, band, tile, e[4] if len(e) > 4 else 0)
        return len(data.get("entries", []))
