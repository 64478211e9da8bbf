"""The per-lane corner check's rule, pinned against the oracle's EAPrunedDTW.

Before the warp wavefront, each lane computes rows and columns 1..16 of its
window's cost matrix and drops the window when some row r of that corner is
entirely > ub while column 16 has been > ub in every row up to r.  The claim
is that Algorithm 3 then abandons the window (every cell of row r is > ub, so
no warping path stays within ub).  These tests restate the rule from that
definition, in FP64, and check the claim against the oracle on random-walk
windows, unconstrained and banded, and that the rule is not vacuous."""
import numpy as np
import pytest

import oracle as O
from paper_2010_05371_gb300 import synth

CORNER = 16   # the kernel's default corner size (EAPDTW_CORNER)


def corner_dead_row(z, q, ub, w, absolute=False):
    """The first corner row r that makes the rule fire, or 0."""
    D = np.full((CORNER + 1, CORNER + 1), np.inf)
    D[0, 0] = 0.0
    edge = True
    for r in range(1, CORNER + 1):
        for c in range(1, CORNER + 1):
            if abs(r - c) > w:
                continue
            d = z[r - 1] - q[c - 1]
            D[r, c] = (abs(d) if absolute else d * d) + min(D[r - 1, c], D[r - 1, c - 1], D[r, c - 1])
        edge = edge and D[r, CORNER] > ub
        if edge and np.all(D[r, 1:] > ub):
            return r
    return 0


@pytest.mark.parametrize("m,w,seed", [(32, 32, 1), (64, 64, 2), (64, 20, 3), (128, 15, 4)])
def test_caught_windows_are_abandoned_by_eapruned_dtw(m, w, seed):
    R = synth.random_walk(60_000, seed)
    zq = O.znorm(synth.random_walk(m, seed + 100))
    rng = np.random.default_rng(seed)
    caught = 0
    for ub in (2.0, 6.0, 20.0):
        for i in rng.integers(0, len(R) - m, 120):
            z = O.znorm(R[i:i + m])
            r = corner_dead_row(z, zq, ub, w)
            if not r:
                continue
            caught += 1
            d, info = O.eapruned_dtw(z, zq, w, ub, trace=True)
            assert d == np.inf, (i, ub, r)
            # Algorithm 3 gives up no later than the corner's dead row
            assert 1 <= info["abandon_row"] <= r, (i, ub, r, info["abandon_row"])
    assert caught >= 60, caught   # the rule fires on a good share of random windows


def test_rule_never_fires_on_the_nearest_neighbour():
    """At ub = the exact nearest-neighbour distance, the best window survives."""
    m, w = 48, 48
    R = synth.random_walk(5_000, 11)
    Q = synth.random_walk(m, 12)
    idx, dist = O.search_brute(Q, R, w, 1)
    z = O.znorm(R[idx[0]:idx[0] + m])
    assert corner_dead_row(z, O.znorm(Q), float(dist[0]), w) == 0


@pytest.mark.parametrize("m,w", [(64, 64), (100, 20)])
def test_caught_windows_exceed_ub_under_the_absolute_cost(m, w):
    """The same rule with cost |a - b| (any non-negative cost keeps the argument)."""
    R = synth.random_walk(40_000, 60 + m)
    zq = O.znorm(synth.random_walk(m, 61 + m))
    rng = np.random.default_rng(m)
    caught = 0
    for ub in (3.0, 10.0, 30.0):
        for i in rng.integers(0, len(R) - m, 100):
            z = O.znorm(R[i:i + m])
            if corner_dead_row(z, zq, ub, w, absolute=True):
                caught += 1
                assert O.dtw_cost(z, zq, w, O.COST_ABSOLUTE) > ub, (i, ub)
    assert caught >= 30, caught
