"""The search entry point for callers that cannot allocate memory.

subseq_search_noalloc keeps its scratch in one fixed device array of the
library instead of allocating it (for callers inside an allocator or memory
pool they do not own, or under a no-allocation-after-start-up policy).  Each
call's result must be the oracle's (distances within the GPU tests' tolerance;
an index that differs must carry, in the oracle, a distance within the same
tolerance of the best) and the allocating entry point's.  The calls run small,
large, small, so that what a larger call left in the shared array cannot
affect the next one, and they reach every path: the sampled seed, the
no-seed path (fewer than 2048 windows), the widest re-run level (queries
longer than 1024 points) and k larger than the number of windows.  This file
is collected last so that a run stopping at its first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from gpu_util import check_topk, dist_close

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


# (reference, query, w, k); windows = len(R) - len(Q) + 1
SMALL_1 = (synth.random_walk(2000, 21), synth.random_walk(128, 22), 13, 3)            # 1873 windows: no seed
LARGE = (synth.random_walk(1_000_000, 23), synth.random_walk(256, 24), 26, 5)         # seeded, 999,745 windows
SMALL_2 = (synth.random_walk(2600, 25), synth.random_walk(1100, 26), 1100, 2)         # no seed, widest level
TINY = (synth.ecg_like(131, 27), synth.ecg_query(128, 28), 20, 6)                     # 4 windows, k = 6


def test_noalloc_matches_the_oracle_small_large_small():
    for R_np, Q_np, w, k in (SMALL_1, LARGE, SMALL_2, TINY, SMALL_1):
        R = torch.tensor(R_np, dtype=torch.float32, device="cuda")
        Q = torch.tensor(Q_np, dtype=torch.float32, device="cuda")
        gi, gd = _call_noalloc(Q, R, w, k)
        oi, od, _ = O.search_cascade(Q_np, R_np, w, k, nthreads=8)
        check_topk(gi, gd, oi, od, Q_np, R_np, w)
        nw = len(R_np) - len(Q_np) + 1
        if k > nw:   # the slots past the last window
            assert list(gi[nw:]) == [-1] * (k - nw) and np.all(np.isinf(gd[nw:]))
        # and the allocating entry point's result
        ri, rd = api.subseq_search(Q, R, w, k)
        for x, y in zip(gd, rd.cpu().numpy()):
            assert dist_close(float(x), float(y), len(Q_np))


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
