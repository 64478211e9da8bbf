"""Pins of the oracle's other pointwise costs (Section 6: elastic distances that
share DTW's recurrence): the absolute cost |a - b| against every warping path on
tiny inputs, its closed forms, and the squared cost's consistency with Eq. 1-5."""
import numpy as np
import pytest

import oracle as O

INF = float("inf")


def paths_min(S, T, w, cost):
    """Minimum over every warping path within the band of the summed cost."""
    n, m = len(S), len(T)
    best = INF
    stack = [(0, 0, cost(S[0], T[0]))]
    while stack:
        i, j, acc = stack.pop()
        if i == n - 1 and j == m - 1:
            best = min(best, acc)
            continue
        for di, dj in ((1, 0), (0, 1), (1, 1)):
            a, b = i + di, j + dj
            if a < n and b < m and abs(a - b) <= w:
                stack.append((a, b, acc + cost(S[a], T[b])))
    return best


@pytest.mark.parametrize("mode,fn", [(O.COST_ABSOLUTE, lambda a, b: abs(a - b)),
                                     (O.COST_SQUARED, lambda a, b: (a - b) ** 2)])
def test_every_warping_path(mode, fn):
    rng = np.random.default_rng(31)
    for _ in range(120):
        n, m = int(rng.integers(1, 7)), int(rng.integers(1, 7))
        w = int(rng.integers(0, 7))
        S, T = rng.normal(size=n), rng.normal(size=m)
        got = O.dtw_cost(S, T, w, mode)
        ref = paths_min(S, T, w, fn) if w >= abs(n - m) else INF
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-12) or (got == INF and ref == INF)


def test_absolute_cost_closed_forms():
    rng = np.random.default_rng(32)
    for _ in range(50):
        m = int(rng.integers(1, 60))
        S, T = rng.normal(size=m), rng.normal(size=m)
        l1 = float(np.abs(S - T).sum())
        assert O.dtw_cost(S, T, 0, O.COST_ABSOLUTE) == pytest.approx(l1, rel=1e-12)   # w = 0: L1 distance
        assert O.dtw_cost(S, S, m, O.COST_ABSOLUTE) == 0.0                            # identity
        w = int(rng.integers(0, m + 1))
        d = O.dtw_cost(S, T, w, O.COST_ABSOLUTE)
        assert d == O.dtw_cost(T, S, w, O.COST_ABSOLUTE)                               # symmetry
        assert d <= l1 + 1e-12                                                          # the diagonal is a path
        assert O.dtw_cost(S, T, w, O.COST_SQUARED) == pytest.approx(O.dtw(S, T, w), rel=1e-12)


def test_brute_force_search_with_a_cost():
    rng = np.random.default_rng(33)
    R = np.cumsum(rng.normal(size=800))
    Q = np.cumsum(rng.normal(size=40))
    i0, d0 = O.search_brute_cost(Q, R, 5, 3, O.COST_SQUARED)
    i1, d1 = O.search_brute(Q, R, 5, 3)
    np.testing.assert_array_equal(i0, i1)
    np.testing.assert_allclose(d0, d1, rtol=1e-12)
    ia, da = O.search_brute_cost(Q, R, 5, 3, O.COST_ABSOLUTE)
    zq = O.znorm(Q)
    every = [O.dtw_cost(O.znorm(R[i:i + 40]), zq, 5, O.COST_ABSOLUTE) for i in range(len(R) - 39)]
    order = np.lexsort((np.arange(len(every)), every))[:3]
    np.testing.assert_array_equal(ia, order)
