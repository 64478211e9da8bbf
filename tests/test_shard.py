"""One search sharded by window range (paper_2010_05371_gb300/shard.py): the
partition with its lQ - 1 halo, the packed-key merge, and the collective merge
on two gloo ranks on CPU, each rank searching its slice with the oracle
(Section 5: every window's distance is independent of the others), against
the oracle's search of the whole reference."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle as O
from gpu_util import dist_close
from paper_2010_05371_gb300 import shard, synth

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("nw,world", [(10, 1), (10, 3), (7, 7), (5, 8), (1_000_003, 4)])
def test_window_ranges_partition_the_windows(nw, world):
    rs = shard.window_ranges(nw, world)
    assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == nw
    assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
    sizes = [hi - lo for lo, hi in rs]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def test_slices_hold_every_window_of_their_range():
    m = 37
    R = np.arange(1000.0)
    nw = len(R) - m + 1
    for lo, hi in shard.window_ranges(nw, 3):
        a, b = shard.slice_bounds(lo, hi, m)
        S = R[a:b]
        for i in (lo, hi - 1):
            j = i - a
            np.testing.assert_array_equal(S[j:j + m], R[i:i + m])
        assert b <= len(R) and len(S) - m + 1 == hi - lo


def test_packed_keys_order_by_distance_then_index():
    idx = np.array([5, 3, 9, -1, 4])
    dist = np.array([2.0, 2.0, 0.5, np.inf, np.float32(2.0000002)])
    i, d = shard.unpack_keys(shard.pack_keys(idx, dist), 6)
    assert list(i) == [9, 3, 5, 4, -1, -1]
    assert d[0] == 0.5 and d[1] == d[2] == 2.0 and np.isinf(d[4])


def test_local_merge_of_oracle_shards_equals_the_whole_search():
    R = synth.random_walk(30_000, 3)
    Q = synth.random_walk(128, 4)
    m, w, k = len(Q), 13, 5
    oi, od, _ = O.search_cascade(Q, R, w, k, nthreads=4)
    lists = []
    for lo, hi in shard.window_ranges(len(R) - m + 1, 3):
        a, b = shard.slice_bounds(lo, hi, m)
        li, ld, _ = O.search_cascade(Q, R[a:b], w, k, nthreads=4)
        lists.append((np.where(li >= 0, li + lo, -1), ld))
    gi, gd = shard.merge_local(lists, k)
    for x, y in zip(gd, od):
        assert dist_close(float(x), float(y), m)
    assert list(gi) == list(oi)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q, k):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle as O2
    from paper_2010_05371_gb300 import shard as S, synth as Y
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        R = Y.random_walk(20_000, 11)
        Q = Y.random_walk(200, 12)

        def oracle_part(Qp, Rp, w, kk):
            i, d, _ = O2.search_cascade(Qp, Rp, w, kk, nthreads=2)
            return i, d

        gi, gd = S.sharded_search(oracle_part, Q, R, 40, k, rank, world)
        q.put((rank, list(gi), list(gd)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("k", [1, 5])
def test_two_gloo_ranks_merge_to_the_one_rank_answer(k):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, k)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=240) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    R = synth.random_walk(20_000, 11)
    Q = synth.random_walk(200, 12)
    oi, od, _ = O.search_cascade(Q, R, 40, k, nthreads=4)
    for rank, gi, gd in out:
        assert gi == out[0][1] and gd == out[0][2]   # every rank holds the merged answer
        for x, y in zip(gd, od):
            assert dist_close(float(x), float(y), len(Q))
        assert gi == list(oi)
