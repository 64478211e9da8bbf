"""One subsequence search sharded by window range across the ranks of a
process group (host logic; every rank's search runs in the library's kernels).

The windows of a search are independent (Section 5: each candidate window is
z-normalised on its own and compared with the query), so the search splits
into contiguous window ranges, one per rank.  Rank r searches windows
[lo_r, hi_r) of R through the slice R[lo_r : hi_r + lQ - 1) (the range plus
an lQ - 1 halo: the last window of the range ends there), shifts its local
indices by lo_r, and the ranks merge their k-best lists: a k-best list orders
windows by (distance, index), which packed keys (FP32 distance bits << 32 |
index) order the same way, since non-negative floats order like their bits.
k = 1 merges with one all-reduce MIN of the packed key; k > 1 all-gathers the
ranks' k keys and keeps the k smallest distinct ones.  No rank reads another
rank's data, and there is no exchange before the merge.

Each rank's window statistics come from its own slice (prefix sums anchored in
the slice), so a distance may differ from the one-rank search's in the last
FP32 bits; both stay within the oracle tolerance.
"""
from __future__ import annotations

import numpy as np

EMPTY_KEY = np.iinfo(np.int64).max   # sorts after every real key


def window_ranges(nw: int, world: int):
    """Contiguous window ranges [lo, hi) covering [0, nw), one per rank, as
    even as possible (the first nw % world ranks get one more window)."""
    if nw < 0 or world < 1:
        raise ValueError("nw >= 0 and world >= 1")
    base, extra = divmod(nw, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def slice_bounds(lo: int, hi: int, m: int):
    """Points of R that windows [lo, hi) of length m read: [lo, hi + m - 1)
    (empty for an empty range)."""
    return (lo, hi + m - 1) if hi > lo else (lo, lo)


def pack_keys(idx, dist) -> np.ndarray:
    """Packed int64 keys of a k-best list: FP32 bits of the distance << 32 |
    index; empty slots (index < 0 or distance +inf with no window) sort last."""
    idx = np.asarray(idx, dtype=np.int64)
    d32 = np.asarray(dist, dtype=np.float64).astype(np.float32)
    bits = d32.view(np.uint32).astype(np.int64)
    keys = (bits << 32) | (idx & 0xFFFFFFFF)
    return np.where(idx >= 0, keys, EMPTY_KEY).astype(np.int64)


def unpack_keys(keys, k: int):
    """(idx int64[k], dist float64[k]) of the k smallest distinct keys,
    (-1, +inf) past the last real one."""
    keys = np.unique(np.asarray(keys, dtype=np.int64))   # sorted, distinct
    keys = keys[keys != EMPTY_KEY][:k]
    idx = np.full(k, -1, dtype=np.int64)
    dist = np.full(k, np.inf)
    idx[:len(keys)] = keys & 0xFFFFFFFF
    dist[:len(keys)] = (keys >> 32).astype(np.uint32).view(np.float32).astype(np.float64)
    return idx, dist


def merge_local(lists, k: int):
    """Merge k-best lists [(idx, dist), ...] with global indices (the host
    form of the collective merge)."""
    return unpack_keys(np.concatenate([pack_keys(i, d) for i, d in lists]), k)


def sharded_search(search, Q, R, w: int, k: int, rank: int, world: int, group=None, device=None):
    """k nearest windows of R to Q, sharded over `world` ranks of the current
    process group.  search(Q, R_slice, w, k) -> (idx, dist) runs one rank's
    part (for example api.subseq_search on a device slice) and returns local
    indices.  Every rank returns the merged (idx, dist) as numpy arrays."""
    import torch
    import torch.distributed as dist

    m = len(Q)
    nw = len(R) - m + 1
    lo, hi = window_ranges(nw, world)[rank]
    a, b = slice_bounds(lo, hi, m)
    if hi > lo:
        li, ld = search(Q, R[a:b], w, k)
        li = np.asarray(li.cpu() if hasattr(li, "cpu") else li, dtype=np.int64)
        ld = np.asarray(ld.cpu() if hasattr(ld, "cpu") else ld, dtype=np.float64)
        gi = np.where(li >= 0, li + lo, -1)
    else:
        gi, ld = np.full(k, -1, dtype=np.int64), np.full(k, np.inf)
    keys = torch.from_numpy(pack_keys(gi, ld))
    if device is not None:
        keys = keys.to(device)
    if world == 1:
        return unpack_keys(keys.cpu().numpy(), k)
    if k == 1:
        dist.all_reduce(keys, op=dist.ReduceOp.MIN, group=group)
        return unpack_keys(keys.cpu().numpy(), 1)
    parts = [torch.empty_like(keys) for _ in range(world)]
    dist.all_gather(parts, keys, group=group)
    return unpack_keys(torch.cat(parts).cpu().numpy(), k)
