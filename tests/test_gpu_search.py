"""subseq_search (the full hot path through the C ABI) against the oracle."""
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


def run(Q, R, w, k, **kw):
    idx, dist = api.subseq_search(dev(Q), dev(R), w, k, **kw)
    return idx.cpu().numpy(), dist.cpu().numpy()


SMALL = [
    # (n, m, w, k, seed)
    (3000, 16, 0, 1, 1),
    (3000, 16, 2, 3, 2),
    (3000, 16, 15, 1, 3),
    (2500, 64, 6, 5, 4),
    (2500, 64, 64, 2, 5),
    (4099, 128, 13, 1, 6),
    (1000, 100, 30, 4, 7),
    (777, 33, 7, 1, 8),
]


@pytest.mark.parametrize("n,m,w,k,seed", SMALL)
@pytest.mark.parametrize("no_lb", [False, True])
def test_small_vs_brute_force(n, m, w, k, seed, no_lb):
    R = synth.random_walk(n, seed)
    Q = synth.random_walk(m, seed + 100)
    oi, od = O.search_brute(Q, R, w, k)
    gi, gd = run(Q, R, w, k, no_lb=no_lb)
    check_topk(gi, gd, oi, od, Q, R, w)


@pytest.mark.parametrize("tile", [4, 8, 16, 32])
def test_every_tile_width(tile):
    R = synth.random_walk(3000, 11)
    Q = synth.random_walk(96, 12)
    for w in (0, 5, 40, 96):
        oi, od = O.search_brute(Q, R, w, 2)
        gi, gd = run(Q, R, w, 2, tile=tile)
        check_topk(gi, gd, oi, od, Q, R, w)


def test_small_config_full_size():
    """Random walk of 100,000 points, query of 128, w = 13, k = 1 and 5."""
    R = synth.random_walk(100_000, 0)
    Q = synth.random_walk(128, 1)
    for k in (1, 5):
        oi, od, _ = O.search_cascade(Q, R, 13, k, nthreads=8)
        gi, gd = run(Q, R, 13, k)
        check_topk(gi, gd, oi, od, Q, R, 13)
        gi2, gd2 = run(Q, R, 13, k, no_lb=True)
        check_topk(gi2, gd2, oi, od, Q, R, 13)


def test_ecg_like():
    R = synth.ecg_like(60_000, 0)
    Q = synth.ecg_query(256, 1)
    for w in (13, 52, 128):
        oi, od, _ = O.search_cascade(Q, R, w, 3, nthreads=8)
        gi, gd = run(Q, R, w, 3)
        check_topk(gi, gd, oi, od, Q, R, w)


def test_edge_cases():
    R = synth.random_walk(500, 3)
    # one window
    Q = R[100:300].copy()
    oi, od = O.search_brute(Q, R[100:300], 10, 1)
    gi, gd = run(Q, R[100:300], 10, 1)
    check_topk(gi, gd, oi, od, Q, R[100:300], 10)
    # k larger than the number of windows
    gi, gd = run(R[:40], R[:45], 3, 8)
    assert list(gi[6:]) == [-1, -1] and all(math.isinf(x) for x in gd[6:])
    # query of length 1: every window normalises to 0 -> all distances 0, ties by index
    gi, gd = run(R[:1], R, 0, 3)
    assert list(gi) == [0, 1, 2] and list(gd) == [0, 0, 0]
    # constant stretch: constant windows normalise to zeros
    Rc = R.copy()
    Rc[200:320] = 7.25
    Q = synth.random_walk(50, 9)
    oi, od = O.search_brute(Q, Rc, 5, 4)
    gi, gd = run(Q, Rc, 5, 4)
    check_topk(gi, gd, oi, od, Q, Rc, 5)
    # the query itself is in the reference: distance 0 at its position
    Rl = synth.random_walk(5000, 4)
    gi, gd = run(Rl[1234:1234 + 77], Rl, 7, 1)
    assert gi[0] == 1234 and dist_close(gd[0], 0.0, 77)


def test_large_offset_series():
    """A random walk far from zero: window statistics stay accurate (chunk anchors)."""
    R = synth.f32(synth.random_walk(20_000, 5) + 3.0e4)
    Q = synth.random_walk(64, 6)
    oi, od = O.search_brute(Q, R, 6, 3)
    gi, gd = run(Q, R, 6, 3)
    check_topk(gi, gd, oi, od, Q, R, 6)


def test_nan_input_is_an_error():
    R = synth.random_walk(1000, 1)
    R[500] = np.nan
    with pytest.raises(api.EapDtwError) as e:
        run(R[:20], R, 2, 1)
    assert e.value.code == -2


def test_host_entry_point_matches_device():
    R = synth.random_walk(50_000, 2)
    Q = synth.random_walk(128, 3)
    gi, gd = run(Q, R, 13, 3)
    hi, hd = api.subseq_search_host(Q, R, 13, 3)
    assert list(hi) == list(gi) and list(hd) == list(gd)


def test_repeatable_and_seed_independent():
    R = synth.random_walk(80_000, 8)
    Q = synth.random_walk(200, 9)
    a = run(Q, R, 20, 5)
    b = run(Q, R, 20, 5)
    c = run(Q, R, 20, 5, no_seed=True)
    assert list(a[0]) == list(b[0]) == list(c[0])
    assert list(a[1]) == list(b[1]) == list(c[1])


def test_wide_query_without_seed():
    """m = 1500, unconstrained, no seed: the first candidates run with ub = +inf,
    their live regions exceed 1024 columns and go to the four-window level."""
    R = synth.random_walk(2500, 31)
    Q = synth.random_walk(1500, 32)
    oi, od = O.search_brute(Q, R, 1500, 2)
    gi, gd = run(Q, R, 1500, 2, no_seed=True, no_lb=True)
    check_topk(gi, gd, oi, od, Q, R, 1500)
    gi, gd = run(Q, R, 1500, 2, no_seed=True)
    check_topk(gi, gd, oi, od, Q, R, 1500)


@pytest.mark.parametrize("m,w,k", [(128, 13, 1), (256, 40, 5), (512, 512, 2), (1500, 300, 1)])
def test_tightening_changes_work_not_results(m, w, k):
    """Upper-bound tightening with the LB_Keogh EQ terms: bit-identical results
    and audit decisions, no more DTW steps than without it."""
    R = synth.random_walk(120_000, 70 + m)
    Q = synth.random_walk(m, 71 + m)
    Rd, Qd = dev(R), dev(Q)
    i1, d1, c1 = api.subseq_search(Qd, Rd, w, k, return_counters=True, tighten=True)
    i0, d0, c0 = api.subseq_search(Qd, Rd, w, k, return_counters=True)
    np.testing.assert_array_equal(d1.cpu().numpy(), d0.cpu().numpy())
    np.testing.assert_array_equal(i1.cpu().numpy(), i0.cpu().numpy())
    ub = float(d0.cpu().numpy()[-1])
    _, a1, e1 = api.subseq_search(Qd, Rd, w, k, audit_ub=ub, return_counters=True, tighten=True)
    _, a0, e0 = api.subseq_search(Qd, Rd, w, k, audit_ub=ub, return_counters=True)
    np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
    for key in ("kim_pruned", "eq_pruned", "ec_pruned", "dtw_abandoned", "dtw_completed"):
        assert e1[key] == e0[key], key
    # steps compare on the same first level (tightening keeps the one-window
    # wavefront, where an unconstrained search would otherwise take the elastic one)
    _, _, e0 = api.subseq_search(Qd, Rd, w, k, audit_ub=ub, return_counters=True, tile=e1["first_tile"])
    assert e1["steps"] <= e0["steps"]


@pytest.mark.parametrize("n,m,w,k", [(3000, 32, 4, 1), (4000, 200, 200, 3), (3000, 600, 600, 2),
                                     (2600, 1300, 1300, 1), (5000, 128, 20, 5)])
def test_absolute_cost_search_vs_brute_force(n, m, w, k):
    """Another elastic distance with DTW's recurrence: cost |a - b|, searched
    without lower bounds, across the re-run levels (m up to 1300 unconstrained)."""
    R = synth.random_walk(n, 90 + m)
    Q = synth.random_walk(m, 91 + m)
    oi, od = O.search_brute_cost(Q, R, w, k, O.COST_ABSOLUTE)
    gi, gd = run(Q, R, w, k, no_lb=True, cost=api.COST_ABSOLUTE)
    zq = O.znorm(Q)
    for j in range(k):
        assert dist_close(float(gd[j]), float(od[j]), m), (j, gd[j], od[j])
        if gi[j] != oi[j]:
            rescored = O.dtw_cost(O.znorm(R[gi[j]:gi[j] + m]), zq, w, O.COST_ABSOLUTE)
            assert dist_close(rescored, float(od[j]), m)


def test_absolute_cost_needs_no_lower_bounds():
    R, Q = dev(synth.random_walk(2000, 1)), dev(synth.random_walk(50, 2))
    with pytest.raises(api.EapDtwError) as e:
        api.subseq_search(Q, R, 5, 1, cost=api.COST_ABSOLUTE)
    assert e.value.code == -1


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


def _check_nn(gi, gd, nn_index, nn_dist, Q, R, w):
    m = len(Q)
    assert dist_close(gd, nn_dist, m), (gd, nn_dist)
    if gi != nn_index:  # tie-equivalent: the oracle's own distance at the GPU's index
        rescored = O.dtw(O.znorm(np.asarray(R[gi:gi + m], np.float64)), O.znorm(np.asarray(Q, np.float64)), w)
        assert dist_close(rescored, nn_dist, m), (gi, rescored, nn_index, nn_dist)


def test_large_configs_at_full_size():
    """The large random-walk and ECG-like configurations at full size (2e7
    points), against the FP64 oracle's nearest neighbours written by
    oracle/bench_reference.py and oracle/ecg_reference.py."""
    g = _golden("bench_large_oracle.json")
    R = np.asarray(synth.random_walk(20_000_000, 0), np.float32)
    Rd = dev(R)
    for e in g["searches"]:
        Q = synth.random_walk(e["m"], e["query_seed"])
        gi, gd = api.subseq_search(dev(Q), Rd, e["w"], 1, no_lb=not e["lower_bounds"])
        _check_nn(int(gi.cpu()[0]), float(gd.cpu()[0]), e["nn_index"], e["nn_dist"], Q, R, e["w"])
    del Rd
    g = _golden("ecg_large_oracle.json")
    R = np.asarray(synth.ecg_like(20_000_000, 0), np.float32)
    Rd = dev(R)
    for e in g["searches"]:
        Q = synth.ecg_query(e["m"], e["query_seed"])
        gi, gd = api.subseq_search(dev(Q), Rd, e["w"], 1)
        _check_nn(int(gi.cpu()[0]), float(gd.cpu()[0]), e["nn_index"], e["nn_dist"], Q, R, e["w"])
