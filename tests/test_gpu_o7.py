"""Bit-exact parity with the FP32-emulating oracle mode: the GPU search's
distances and indices equal the emulation's exactly, and under a fixed upper
bound (audit mode) so do its integer outcomes -- the windows pruned by
LB_Kim, LB_Keogh EQ and LB_Keogh EC, and the EAPrunedDTW runs completed and
abandoned."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2010_05371_gb300 import api, synth  # noqa: E402

CASES = [
    # (series, n, m, w, k, seed)
    ("walk", 100_000, 128, 13, 1, 0),
    ("walk", 60_000, 128, 13, 5, 1),
    ("walk", 30_000, 64, 0, 3, 2),
    ("walk", 20_000, 200, 200, 2, 3),
    ("ecg", 40_000, 256, 26, 1, 4),
    ("walk", 9_000, 600, 150, 1, 5),
    # edges of the per-lane corner check (rows and columns 1..16): the shortest
    # query and the narrowest band it runs with, and a query just too short
    ("walk", 20_000, 16, 15, 2, 6),
    ("walk", 20_000, 16, 16, 1, 7),
    ("walk", 20_000, 15, 15, 1, 8),
    ("walk", 20_000, 40, 14, 3, 9),
]
AUDIT_KEYS = ("windows", "kim_pruned", "eq_pruned", "ec_pruned", "dtw_abandoned", "dtw_completed")


def inputs(kind, n, m, seed):
    if kind == "ecg":
        R, Q = synth.ecg_like(n, seed), synth.ecg_query(m, seed + 50)
    else:
        R, Q = synth.random_walk(n, seed), synth.random_walk(m, seed + 50)
    return np.asarray(R, np.float32), np.asarray(Q, np.float32)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("kind,n,m,w,k,seed", CASES)
def test_results_and_audit_counts_bit_exact(kind, n, m, w, k, seed):
    R, Q = inputs(kind, n, m, seed)
    ei, ed, _ = O.o7_search(Q, R, w, k)
    Rd, Qd = dev(R), dev(Q)
    gi, gd = api.subseq_search(Qd, Rd, w, k)
    np.testing.assert_array_equal(gd.cpu().numpy(), ed)
    np.testing.assert_array_equal(gi.cpu().numpy(), ei)
    ub = float(np.float32(ed[-1]))
    for use_lb in (True, False):
        ai, ad, oc = O.o7_search(Q, R, w, k, audit_ub=ub, use_lb=use_lb)
        gi2, gd2, gc = api.subseq_search(Qd, Rd, w, k, audit_ub=ub, no_lb=not use_lb, return_counters=True)
        assert {c: gc[c] for c in AUDIT_KEYS} == oc, (use_lb, gc)
        np.testing.assert_array_equal(gd2.cpu().numpy(), ad)
        np.testing.assert_array_equal(gi2.cpu().numpy(), ai)


def test_batched_results_bit_exact():
    items, expect = [], []
    with api.Context(0) as ctx:
        refs = {}
        for kind, n, m, w, k, seed in CASES[:4]:
            R, Q = inputs(kind, n, m, seed)
            rid = ctx.register(dev(R))
            items.append((dev(Q), rid, w, k))
            expect.append(O.o7_search(Q, R, w, k)[:2])
        bi, bd = ctx.search_batch(items, 5)
        bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
        for j, (ei, ed) in enumerate(expect):
            k = len(ei)
            np.testing.assert_array_equal(bd[j, :k], ed)
            np.testing.assert_array_equal(bi[j, :k], ei)


@pytest.mark.parametrize("kind,m,seed", [("walk", 1024, 11), ("ecg", 512, 12)])
def test_dominant_shape_audit_counts_bit_exact(kind, m, seed):
    """The benchmark's dominant path: an unconstrained search without lower
    bounds (the elastic first level and its re-run levels), and the same search
    with the first level forced to the one-window wavefront at K = 16.  Under a
    fixed bound just above the FP64 oracle's nearest-neighbour distance, the
    audit counts and the k-best list equal the FP32 emulation's bit for bit,
    and the free search returns the emulation's nearest window (4,001 windows,
    so that the emulation of every window's DTW finishes)."""
    R, Q = inputs(kind, 4_000 + m, m, seed)
    _, od, _ = O.search_cascade(Q, R, m, 1, nthreads=8)
    ub = float(np.float32(od[0] * (1 + 1e-4)))
    ai, ad, oc = O.o7_search(Q, R, m, 3, audit_ub=ub, use_lb=False)
    assert oc["dtw_completed"] >= 1
    Rd, Qd = dev(R), dev(Q)
    for tile in (0, 16):
        gi, gd = api.subseq_search(Qd, Rd, m, 1, no_lb=True, tile=tile)
        assert float(gd.cpu()[0]) == ad[0] and int(gi.cpu()[0]) == ai[0], (tile, gi, gd, ai, ad)
        gi2, gd2, gc = api.subseq_search(Qd, Rd, m, 3, audit_ub=ub, no_lb=True, tile=tile, return_counters=True)
        assert {c: gc[c] for c in AUDIT_KEYS} == oc, (tile, gc, oc)
        np.testing.assert_array_equal(gd2.cpu().numpy(), ad)
        np.testing.assert_array_equal(gi2.cpu().numpy(), ai)


GROUP_CASES = [
    # (series, n, m, w, k, seed, tile): the group of warps as the first level
    # (tile = 512), or as the re-run level after the one-warp levels (tile 0)
    ("walk", 3_000, 300, 40, 2, 20, 512),     # one warp per group
    ("ecg", 4_000, 700, 200, 3, 21, 512),     # two warps
    ("walk", 2_300, 1500, 900, 1, 22, 512),   # three warps
    ("ecg", 2_800, 2500, 1500, 2, 23, 512),   # five warps
    ("ecg", 2_800, 2500, 1500, 2, 23, 0),     # the same through the one-warp levels and re-runs
    ("walk", 4_300, 4096, 4096, 1, 24, 512),  # eight warps, unconstrained
    # the elastic wavefront on a wide band as the first level (w >= 64 and a
    # quarter of m), handing candidates near the band's edges to the banded levels
    ("walk", 30_000, 300, 200, 2, 30, 0),
    ("ecg", 20_000, 500, 130, 1, 31, 0),
    ("walk", 12_000, 900, 300, 3, 32, 0),
]


@pytest.mark.parametrize("kind,n,m,w,k,seed,tile", GROUP_CASES)
def test_group_and_banded_elastic_levels_bit_exact(kind, n, m, w, k, seed, tile):
    """The group wavefront as the first level (its warp 0 runs the
    lower-bound cascade of each tile, the group the survivors) or as the
    re-run level, and the banded elastic first level: results equal the FP32
    emulation's, and under a fixed bound so do the prune, abandon and
    completion counts, with and without lower bounds."""
    R, Q = inputs(kind, n, m, seed)
    ei, ed, _ = O.o7_search(Q, R, w, k)
    Rd, Qd = dev(R), dev(Q)
    gi, gd = api.subseq_search(Qd, Rd, w, k, tile=tile)
    np.testing.assert_array_equal(gd.cpu().numpy(), ed)
    np.testing.assert_array_equal(gi.cpu().numpy(), ei)
    ub = float(np.float32(ed[-1] * 1.05))
    for use_lb in (True, False):
        ai, ad, oc = O.o7_search(Q, R, w, k, audit_ub=ub, use_lb=use_lb)
        gi2, gd2, gc = api.subseq_search(Qd, Rd, w, k, audit_ub=ub, no_lb=not use_lb, tile=tile,
                                         return_counters=True)
        assert {c: gc[c] for c in AUDIT_KEYS} == oc, (use_lb, gc, oc)
        if tile == 0 and 128 < m <= 1024 and w >= 64 and 4 * w >= m and w < m - 1:
            assert gc["first_tile"] == 4, gc   # the elastic wavefront ran first
        np.testing.assert_array_equal(gd2.cpu().numpy(), ad)
        np.testing.assert_array_equal(gi2.cpu().numpy(), ai)
