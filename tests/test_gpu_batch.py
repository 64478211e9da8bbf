"""The batched search (contexts, resident references, eapdtw_search_batch):
every item equals the one-query search of the same (Q, R, w, k), and a sample
of items is checked against the oracle."""
import math

import numpy as np
import pytest

import oracle as O
from gpu_util import check_topk, dist_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2010_05371_gb300 import api, synth  # noqa: E402


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float32), device="cuda")


def plain(Q, R, w, k, no_lb=False):
    idx, dist = api.subseq_search(Q, R, w, k, no_lb=no_lb)
    return idx.cpu().numpy(), dist.cpu().numpy()


def mixed_items(rng, refs, nq, m_lo, m_hi, seed):
    """Queries of log-uniform lengths, window ratios uniform in [0, 1], random
    walk or ECG-like by a coin flip, k in {1, 5}, each against every reference."""
    items = []
    for q in range(nq):
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        ratio = rng.uniform(0.0, 1.0)
        w = int(math.ceil(ratio * m))
        Q = synth.random_walk(m, seed + q) if rng.random() < 0.5 else synth.ecg_query(m, seed + q)
        k = 1 if rng.random() < 0.5 else 5
        for rid, R in refs:
            if m <= len(R):
                items.append((Q, rid, w, k))
    return items


def compare_with_plain(ctx, items, Rs, kstride=None):
    Qd = {}
    dev_items = []
    for Q, rid, w, k in items:
        key = id(Q)
        if key not in Qd:
            Qd[key] = dev(Q)
        dev_items.append((Qd[key], rid, w, k))
    bi, bd = ctx.search_batch(dev_items, kstride)
    bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
    ks = bi.shape[1]
    for i, (Q, rid, w, k) in enumerate(items):
        pi, pd = plain(Qd[id(Q)], Rs[rid], w, k)
        # same FP32 arithmetic on both paths: equal distances, equal indices up to ties
        np.testing.assert_array_equal(bd[i, :k], pd, err_msg=f"item {i} (m={len(Q)}, w={w}, k={k})")
        for j in range(k):
            if bi[i, j] != pi[j]:
                assert bd[i, j] == pd[j], f"item {i} rank {j}"
        assert np.all(bi[i, k:ks] == -1) and np.all(np.isinf(bd[i, k:ks]))
    return bi, bd


def test_mixed_batch_equals_plain_search():
    rng = np.random.default_rng(7)
    lens = [30_000, 120_000, 9_000]
    refs_np = [synth.random_walk(n, 300 + j) for j, n in enumerate(lens)]
    Rs = [dev(R) for R in refs_np]
    with api.Context(0) as ctx:
        ids = [ctx.register(R) for R in Rs]
        assert ids == [0, 1, 2]
        items = mixed_items(rng, list(zip(ids, refs_np)), 10, 16, 1500, 500)
        compare_with_plain(ctx, items, dict(zip(ids, Rs)))
        info = ctx.info()
        assert info["live_refs"] == 3 and info["batches"] == 1 and info["graph_captured"] == 1


def test_batch_items_against_the_oracle():
    """A sample of items checked against the FP64 oracle's exact search."""
    rng = np.random.default_rng(11)
    R1 = synth.random_walk(6_000, 41)
    R2 = synth.ecg_like(5_000, 42)
    with api.Context(0) as ctx:
        r1, r2 = ctx.register(dev(R1)), ctx.register(dev(R2))
        refs = {r1: R1, r2: R2}
        items = []
        for q in range(6):
            m = int(rng.integers(20, 300))
            w = int(rng.integers(0, m + 1))
            Q = synth.random_walk(m, 600 + q)
            items.append((Q, r1 if q % 2 == 0 else r2, w, 1 + q % 3))
        Qs = [dev(t[0]) for t in items]
        bi, bd = ctx.search_batch([(Qs[i],) + t[1:] for i, t in enumerate(items)])
        bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
        for i, (Q, rid, w, k) in enumerate(items):
            oi, od = O.search_brute(Q, refs[rid], w, k)
            check_topk(bi[i, :k], bd[i, :k], oi, od, Q, refs[rid], w)


def test_graph_replay_and_growth():
    """Several batches in a row on one context: the captured launch sequence is
    replayed with new tables, and captured again when the arena grows."""
    rng = np.random.default_rng(3)
    R_np = synth.random_walk(50_000, 77)
    R = dev(R_np)
    with api.Context(0) as ctx:
        rid = ctx.register(R)
        for rnd, nq in enumerate([2, 3, 90]):
            items = mixed_items(rng, [(rid, R_np)], nq, 32, 700, 900 + 100 * rnd)
            compare_with_plain(ctx, items, {rid: R}, kstride=6)
        assert ctx.info()["batches"] == 3


def test_shared_query_and_no_lb():
    """Items sharing one query tensor (one preparation), with and without the
    lower bounds, and k up to the row length."""
    R_np = synth.random_walk(40_000, 5)
    R = dev(R_np)
    Q_np = synth.random_walk(256, 6)
    Q = dev(Q_np)
    with api.Context(0) as ctx:
        rid = ctx.register(R)
        items = [(Q, rid, 26, 3), (Q, rid, 26, 3, True), (Q, rid, 256, 8), (Q, rid, 0, 1)]
        bi, bd = ctx.search_batch(items, 8)
        bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
        np.testing.assert_array_equal(bd[0], bd[1])
        for i, t in enumerate(items):
            pi, pd = plain(Q, R, t[2], t[3], no_lb=len(t) > 4)
            np.testing.assert_array_equal(bd[i, :t[3]], pd)


def test_wide_queries_reach_the_four_window_level():
    """Unconstrained queries longer than 1024 columns overflow up to the last level."""
    R_np = synth.random_walk(8_000, 51)
    Q_np = synth.random_walk(1800, 52)
    R, Q = dev(R_np), dev(Q_np)
    with api.Context(0) as ctx:
        rid = ctx.register(R)
        bi, bd, cnt = ctx.search_batch([(Q, rid, 1800, 2, True), (Q, rid, 400, 1)], return_counters=True)
        oi, od = O.search_brute(Q_np, R_np, 1800, 2)
        check_topk(bi[0, :2].cpu().numpy(), bd[0, :2].cpu().numpy(), oi, od, Q_np, R_np, 1800)
        pi, pd = plain(Q, R, 400, 1)
        assert dist_close(float(bd[1, 0]), float(pd[0]), 1800)


def test_full_rerun_lists_fall_back_to_single_searches(monkeypatch):
    """A re-run list too small for the overflowing windows marks the items; they
    are searched again alone and the results are still exact."""
    monkeypatch.setenv("EAPDTW_RERUN_LIST_CAP", "4")
    R_np = synth.random_walk(20_000, 61)
    Q_np = synth.random_walk(900, 62)
    R, Q = dev(R_np), dev(Q_np)
    with api.Context(0) as ctx:
        rid = ctx.register(R)
        bi, bd = ctx.search_batch([(Q, rid, 900, 1, True)])
        assert ctx.info()["items_rerun"] == 1
        pi, pd = plain(Q, R, 900, 1, no_lb=True)
        np.testing.assert_array_equal(bd.cpu().numpy()[0], pd)


def test_errors():
    R = dev(synth.random_walk(5_000, 1))
    with api.Context(0) as ctx:
        rid = ctx.register(R)
        Q = dev(synth.random_walk(64, 2))
        bad = Q.clone()
        bad[3] = float("nan")
        with pytest.raises(api.EapDtwError) as e:
            ctx.search_batch([(bad, rid, 5, 1)])
        assert e.value.code == -2
        with pytest.raises(api.EapDtwError) as e:
            ctx.search_batch([(Q, rid + 7, 5, 1)])
        assert e.value.code == -1
        with pytest.raises(api.EapDtwError) as e:
            ctx.search_batch([(Q, rid, 5, 4)], kstride=2)
        assert e.value.code == -1
        Rn = R.clone()
        Rn[10] = float("inf")
        with pytest.raises(api.EapDtwError) as e:
            ctx.register(Rn)
        assert e.value.code == -2
        ctx.unregister(rid)
        with pytest.raises(api.EapDtwError):
            ctx.search_batch([(Q, rid, 5, 1)])
    with api.Context(0, mem_budget=1 << 20) as small:
        with pytest.raises(api.EapDtwError) as e:
            small.register(dev(synth.random_walk(200_000, 3)))
        assert e.value.code == -3


def test_autotune_keeps_results():
    R_np = synth.random_walk(300_000, 81)
    R = dev(R_np)
    rng = np.random.default_rng(5)
    with api.Context(0) as ctx:
        rid = ctx.register(R)
        items = mixed_items(rng, [(rid, R_np)], 4, 100, 1200, 1000)
        Qd = {id(t[0]): dev(t[0]) for t in items}
        n = ctx.autotune([(Qd[id(t[0])],) + t[1:] for t in items], sample_windows=1 << 15)
        assert n >= 1
        compare_with_plain(ctx, items, {rid: R})


def test_tuning_table_round_trip(tmp_path):
    with api.Context(0) as ctx:
        ctx.set_first_tile(7, 3, 1, 16)
        ctx.set_tuning(10, 10, 0, 8, 1)
        ctx.set_tuning(9, 5, 1, 0, 1)      # the check interval alone
        assert ctx.tuning_table() == {(7, 3, 1): (16, 0), (10, 10, 0): (8, 1), (9, 5, 1): (0, 1)}
        assert ctx.get_first_tile(10, 10, 0) == 8
        path = str(tmp_path / "tuning.json")
        ctx.save_tuning(path)
    with api.Context(0) as ctx2:
        assert ctx2.load_tuning(path) == 3
        assert ctx2.tuning_table() == {(7, 3, 1): (16, 0), (10, 10, 0): (8, 1), (9, 5, 1): (0, 1)}
        ctx2.set_first_tile(7, 3, 1, 0)
        ctx2.set_tuning(9, 5, 1, 0, 0)
        assert ctx2.tuning_table() == {(10, 10, 0): (8, 1)}


def test_doubled_check_interval_changes_work_not_results():
    """Every signature of a mixed batch at twice the wavefront's check interval:
    bit-identical to the built-in interval (and so to the one-query path)."""
    rng = np.random.default_rng(23)
    R_np = np.asarray(synth.random_walk(60_000, 24), np.float32)
    with api.Context(0) as ctx:
        R = dev(R_np)
        rid = ctx.register(R)
        items = mixed_items(rng, [(rid, R_np)], 6, 64, 1300, 1000)
        Qd = {id(t[0]): dev(t[0]) for t in items}
        dev_items = [(Qd[id(t[0])],) + t[1:] for t in items]
        bi0, bd0 = ctx.search_batch(dev_items, 5)
        for lg in range(13):
            for tenth in range(11):
                for band in (0, 1):
                    ctx.set_tuning(lg, tenth, band, 0, 1)
        bi1, bd1 = ctx.search_batch(dev_items, 5)
        assert torch.equal(bd0, bd1) and torch.equal(bi0, bi1)


def test_elastic_and_one_warp_first_levels_agree():
    """Every signature of a mixed batch (unconstrained and banded items, short
    and long queries) forced to the elastic first level (tile 1; queries it
    cannot run fall back to the built-in rule) and to the one-warp K = 32
    level: bit-identical results, equal to the built-in choice's."""
    rng = np.random.default_rng(29)
    R_np = np.asarray(synth.random_walk(80_000, 30), np.float32)
    with api.Context(0) as ctx:
        R = dev(R_np)
        rid = ctx.register(R)
        items = mixed_items(rng, [(rid, R_np)], 8, 64, 2000, 1500)
        Qd = {id(t[0]): dev(t[0]) for t in items}
        dev_items = [(Qd[id(t[0])],) + t[1:] for t in items]
        bi0, bd0 = ctx.search_batch(dev_items, 5)
        for tile in (1, 32):
            for lg in range(13):
                for tenth in range(11):
                    for band in (0, 1):
                        ctx.set_first_tile(lg, tenth, band, tile)
            assert ctx.get_first_tile(10, 10, 0) == tile
            bi1, bd1 = ctx.search_batch(dev_items, 5)
            assert torch.equal(bd0, bd1) and torch.equal(bi0, bi1), tile
        compare_with_plain(ctx, items, {rid: R})


def test_batched_mix_sample_against_the_oracle():
    """64 items of the batched mix (1,024 queries x 8 references, drawn among the
    four shortest references) as one batch, against the FP64 oracle's k nearest
    windows written by oracle/batched_reference.py."""
    import json
    import os
    from oracle import batched_reference as B
    path = os.path.join(os.path.dirname(__file__), "golden", "batched_mix_oracle.json")
    if not os.path.exists(path):
        pytest.skip("golden file not written")
    with open(path) as f:
        gold = json.load(f)["items"]
    lens, qs = B.mix()
    refs_np = {}
    with api.Context(0) as ctx:
        rid = {}
        items = []
        for e in gold:
            j = e["ref"]
            if j not in rid:
                refs_np[j] = np.asarray(synth.random_walk(lens[j], 100 + j), np.float32)
                rid[j] = ctx.register(dev(refs_np[j]))
            m, w, ecg, k = qs[e["query"]]
            assert (m, w, ecg, k) == (e["m"], e["w"], e["ecg"], e["k"])
            Q = B.query_values(e["query"], m, ecg)
            items.append((dev(Q), rid[j], w, k))
        ctx.autotune(items, sample_windows=1 << 15)
        bi, bd = ctx.search_batch(items, 5)
        bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
    for r, e in enumerate(gold):
        m, k, w = e["m"], e["k"], e["w"]
        Q = B.query_values(e["query"], m, e["ecg"])
        R = refs_np[e["ref"]]
        check_topk(bi[r, :k], bd[r, :k], np.array(e["idx"]), np.array(e["dist"]), Q, R, w)
