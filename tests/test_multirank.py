"""The N > 1 host logic of bench.py, on CPU with two gloo ranks.

Multi-GPU runs shard each search by window range (paper_2010_05371_gb300/
shard.py, tested in test_shard.py): every window is searched by one rank, and
the job's time per step is the slowest rank's.  These tests run bench.py's
side of that on two gloo ranks: each rank's environment, the max of the step
time over ranks, and the whole-job rate (the job's units over that time)."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        ms = bench.max_over_ranks(100.0 + 50.0 * r, w)   # rank 1 is the slower replica
        dist.barrier()
        q.put((r, w, local, ms, bench.job_rate(2000.0, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert [o[0] for o in out] == [0, 1] and [o[2] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[3] == 150.0 for o in out)                       # both see the slowest rank
    assert all(abs(o[4] - 2000.0 / 0.150) < 1e-6 for o in out)  # the job's units / that time


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(10.0, 1000.0) == 10.0
