"""The search entry point for callers that cannot allocate memory.

subseq_search_noalloc keeps its scratch in one fixed device array of the
library instead of allocating it.  Its results must be those of subseq_search
(the entry point that allocates its scratch), within the tolerance of the
other GPU tests, and a second call must not be affected by what the first one
left in the shared array.  This file is collected last so that a run stopping
at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import dist_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2010_05371_gb300 import api, synth  # noqa: E402


def _call_noalloc(Q, R, w, k):
    idx = torch.empty(k, dtype=torch.int64, device="cuda")
    dist = torch.empty(k, dtype=torch.float64, device="cuda")
    L = api.lib()
    rc = L.subseq_search_noalloc(ctypes.c_void_p(Q.data_ptr()), Q.numel(), ctypes.c_void_p(R.data_ptr()),
                                 R.numel(), w, k, ctypes.c_void_p(idx.data_ptr()),
                                 ctypes.c_void_p(dist.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, api.strerror(rc)
    return idx.cpu().numpy(), dist.cpu().numpy()


def _same(a, b, m):
    ai, ad = a
    bi, bd = b
    for x, y in zip(ad, bd):
        assert dist_close(float(x), float(y), m)
    assert list(ai) == list(bi) or all(dist_close(float(x), float(y), m) for x, y in zip(ad, bd))


def test_noalloc_matches_allocating_entry_point_twice():
    cases = [
        (synth.random_walk(300_000, 21), synth.random_walk(256, 22), 26, 3),
        (synth.ecg_like(200_000, 23), synth.ecg_query(128, 24), 13, 5),
    ]
    for R_np, Q_np, w, k in cases:  # two calls in a row, different inputs
        R = torch.tensor(R_np, dtype=torch.float32, device="cuda")
        Q = torch.tensor(Q_np, dtype=torch.float32, device="cuda")
        got = _call_noalloc(Q, R, w, k)
        ref_i, ref_d = api.subseq_search(Q, R, w, k)
        _same(got, (ref_i.cpu().numpy(), ref_d.cpu().numpy()), len(Q_np))


def test_noalloc_rejects_sizes_beyond_its_array():
    L = api.lib()
    big = torch.zeros((1 << 20) + 1, dtype=torch.float32, device="cuda")
    q = torch.zeros(16, dtype=torch.float32, device="cuda")
    idx = torch.empty(1, dtype=torch.int64, device="cuda")
    dist = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = L.subseq_search_noalloc(ctypes.c_void_p(q.data_ptr()), 16, ctypes.c_void_p(big.data_ptr()),
                                 big.numel(), 2, 1, ctypes.c_void_p(idx.data_ptr()),
                                 ctypes.c_void_p(dist.data_ptr()), None)
    assert rc == -6
