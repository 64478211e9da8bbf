"""The serving loop (continuous batching in rounds): every request's result
equals the one-query search of the same (Q, R, w, k), alone and in a mix of
requests that arrive while others run; cancellation, errors and admission."""
import math
import threading
import time

import numpy as np
import pytest

import oracle as O
from gpu_util import check_topk

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2010_05371_gb300 import api, synth  # noqa: E402


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float32), device="cuda")


def plain(Q, R, w, k, no_lb=False):
    idx, dist = api.subseq_search(dev(Q), R, w, k, no_lb=no_lb)
    return idx.cpu().numpy(), dist.cpu().numpy()


def wait(ctx, rid, k, timeout_s=120.0):
    t0 = time.time()
    while time.time() - t0 < timeout_s:
        r = ctx.poll(rid, k, timeout_ms=200)
        if r is not None:
            return r
    raise AssertionError(f"request {rid} did not finish")


def requests(rng, nreq, m_lo, m_hi, seed):
    out = []
    for q in range(nreq):
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        w = int(math.ceil(rng.uniform(0.0, 0.5) * m))
        k = 1 if rng.random() < 0.5 else 5
        out.append((synth.random_walk(m, seed + q), w, k))
    return out


def test_alone_and_in_the_mix_are_identical():
    R_np = synth.random_walk(400_000, 17)
    R = dev(R_np)
    rng = np.random.default_rng(4)
    reqs = requests(rng, 12, 64, 1500, 2000)
    with api.Context(0) as ctx:
        rid = ctx.register(R)
        ctx.serve_start(max_active=4, chunk_windows=1 << 15)   # several rounds per request
        # alone
        alone = []
        for Q, w, k in reqs[:3]:
            h = ctx.submit(Q, rid, w, k)
            alone.append(wait(ctx, h, k))
        # in the mix: arrivals from two threads while earlier requests run
        handles = [None] * len(reqs)

        def producer(idxs, gap):
            for i in idxs:
                Q, w, k = reqs[i]
                handles[i] = ctx.submit(Q, rid, w, k)
                time.sleep(gap)

        t1 = threading.Thread(target=producer, args=(range(0, len(reqs), 2), 0.01))
        t2 = threading.Thread(target=producer, args=(range(1, len(reqs), 2), 0.017))
        t1.start(); t2.start(); t1.join(); t2.join()
        mixed = [wait(ctx, handles[i], reqs[i][2]) for i in range(len(reqs))]
        st = ctx.serve_stats()
        assert st["completed"] == 3 + len(reqs)
        assert st["p50_ns"] > 0 and st["p99_ns"] >= st["p50_ns"]
        assert st["rounds"] > 3 and st["error"] == 0
        for j in range(3):
            np.testing.assert_array_equal(alone[j][0], mixed[j][0])
            np.testing.assert_array_equal(alone[j][1], mixed[j][1])
        for i, (Q, w, k) in enumerate(reqs):
            pi, pd = plain(Q, R, w, k)
            np.testing.assert_array_equal(mixed[i][1], pd, err_msg=f"request {i}")
        ctx.serve_stop()


def test_served_results_against_the_oracle():
    R_np = synth.ecg_like(8_000, 3)
    R = dev(R_np)
    rng = np.random.default_rng(9)
    reqs = requests(rng, 4, 20, 200, 70)
    with api.Context(0) as ctx:
        rid = ctx.register(R)
        ctx.serve_start(max_active=2, chunk_windows=1000)
        hs = [ctx.submit(Q, rid, w, k) for Q, w, k in reqs]
        for h, (Q, w, k) in zip(hs, reqs):
            gi, gd, lat = wait(ctx, h, k)
            oi, od = O.search_brute(Q, R_np, w, k)
            check_topk(gi, gd, oi, od, Q, R_np, w)
            assert lat > 0


def test_cancel_and_errors():
    R = dev(synth.random_walk(2_000_000, 5))
    with api.Context(0) as ctx:
        rid = ctx.register(R)
        ctx.serve_start(max_active=1, chunk_windows=1 << 14)
        long_q = synth.random_walk(2048, 6)
        h1 = ctx.submit(long_q, rid, 2048, 1, no_lb=True)   # long: many rounds
        h2 = ctx.submit(synth.random_walk(64, 7), rid, 6, 1)  # queued behind it
        ctx.cancel(h2)
        with pytest.raises(api.EapDtwError) as e:
            wait(ctx, h2, 1)
        assert e.value.code == -9
        ctx.cancel(h1)
        with pytest.raises(api.EapDtwError) as e:
            wait(ctx, h1, 1)
        assert e.value.code == -9
        bad = synth.random_walk(100, 8)
        bad[10] = np.nan
        h3 = ctx.submit(bad, rid, 10, 1)
        with pytest.raises(api.EapDtwError) as e:
            wait(ctx, h3, 1)
        assert e.value.code == -2
        # the loop keeps serving after both
        h4 = ctx.submit(synth.random_walk(100, 9), rid, 10, 2)
        assert wait(ctx, h4, 2)[0].shape == (2,)
        assert ctx.serve_stats()["cancelled"] == 2


def test_admission_by_memory():
    """A request whose envelope table does not fit the budget is refused; the
    ones that need no new memory are served."""
    n = 1_000_000
    R = dev(synth.random_walk(n, 11))
    with api.Context(0) as probe:
        probe.register(R)
        probe.serve_start(max_active=2, chunk_windows=1 << 16)
        need = probe.info()["bytes_held"]
    with api.Context(0, mem_budget=need + (1 << 20)) as ctx:
        rid = ctx.register(R)
        ctx.serve_start(max_active=2, chunk_windows=1 << 16)
        Q = synth.random_walk(128, 12)
        ok1 = ctx.submit(Q, rid, 0, 1)                 # radius 0: R itself is the envelope
        ok2 = ctx.submit(Q, rid, 13, 1, no_lb=True)    # no envelope
        refused = ctx.submit(Q, rid, 13, 1)            # needs 4 levels of 8 MB
        wait(ctx, ok1, 1)
        wait(ctx, ok2, 1)
        with pytest.raises(api.EapDtwError) as e:
            wait(ctx, refused, 1)
        assert e.value.code == -3
