"""eap_dtw (Algorithm 3 on one pair, through the C ABI) against the oracle."""
import math

import numpy as np
import pytest

import oracle as O
import pins
from gpu_util import dist_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2010_05371_gb300 import api  # noqa: E402


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float32), device="cuda")


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def test_worked_example():
    g = pins.load_golden()
    S = [float(x) for x in g["S"].split()]
    T = [float(x) for x in g["T"].split()]
    assert api.eap_dtw(dev(S), dev(T)).item() == float(g["dtw"])
    assert api.eap_dtw(dev(S), dev(T), ub=9).item() == float(g["ub9_result"])
    assert math.isinf(api.eap_dtw(dev(S), dev(T), ub=6).item())
    assert api.eap_dtw_host(S, T, ub=9) == 9.0


def _pair_cases(seed, count, lmax):
    rng = np.random.default_rng(seed)
    for c in range(count):
        n = int(rng.integers(1, lmax + 1))
        m = n if c % 3 else int(rng.integers(1, lmax + 1))
        if c % 4 == 0:
            S = rng.integers(0, 5, n).astype(np.float64)
            T = rng.integers(0, 5, m).astype(np.float64)
        else:
            S = f32(np.cumsum(rng.standard_normal(n)))
            T = f32(np.cumsum(rng.standard_normal(m)))
        w = int(rng.integers(0, max(n, m) + 2))
        yield S, T, w, rng


@pytest.mark.parametrize("seed,count,lmax", [(1, 300, 40), (2, 120, 300), (3, 30, 1024)])
def test_random_pairs(seed, count, lmax):
    for S, T, w, rng in _pair_cases(seed, count, lmax):
        d = O.dtw(S, T, w)
        ubs = [math.inf]
        if math.isfinite(d):
            ubs += [d * 0.9, d * 1.1, d * float(rng.uniform(0.3, 3.0))]
        else:
            ubs += [1e9]
        for ub in ubs:
            got = api.eap_dtw(dev(S), dev(T), w, ub).item()
            if math.isfinite(d) and abs(d - ub) <= 1e-4 * max(d, 1e-6):
                continue  # FP32 vs FP64 decides this one
            exp = d if d <= ub else math.inf
            assert dist_close(got, exp, max(len(S), len(T))), (len(S), len(T), w, ub, got, exp)


def test_no_admissible_path_and_degenerate():
    assert math.isinf(api.eap_dtw(dev([1, 2, 3, 4, 5]), dev([1, 2]), 2).item())
    assert api.eap_dtw(dev([1, 2, 3, 4, 5]), dev([1, 2]), 3).item() == O.dtw([1, 2, 3, 4, 5], [1, 2], 3)
    assert api.eap_dtw(dev([2.5]), dev([0.5]), 0).item() == 4.0
    x = dev(np.linspace(-1, 1, 200))
    assert api.eap_dtw(x, x, 5).item() == 0.0
    assert api.eap_dtw(x, x, 5, ub=0.0).item() == 0.0


def test_ties_are_not_abandoned():
    """A DTW exactly equal to ub is returned (strict > ub abandons, Section 2.2)."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        S = rng.integers(0, 4, 30).astype(np.float64)
        T = rng.integers(0, 4, 30).astype(np.float64)
        d = O.dtw(S, T, 5)
        assert api.eap_dtw(dev(S), dev(T), 5, d).item() == d
        if d > 0:
            assert math.isinf(api.eap_dtw(dev(S), dev(T), 5, d - 0.5).item())


@pytest.mark.parametrize("n,m,w", [(1100, 1100, None), (2500, 2300, None), (4000, 4000, None),
                                   (3000, 3000, 800), (3500, 3100, 1500)])
def test_wide_live_region(n, m, w):
    """ub = +inf keeps every cell alive: the live region is the whole band, wider
    than one window of K = 32 blocks, so the four-window level must finish it."""
    rng = np.random.default_rng(n + m)
    S = f32(np.cumsum(rng.standard_normal(n)) * 0.05)
    T = f32(np.cumsum(rng.standard_normal(m)) * 0.05)
    d = O.dtw(S, T, w)
    got = api.eap_dtw(dev(S), dev(T), w, math.inf).item()
    assert dist_close(got, d, max(n, m)), (got, d)
    got2 = api.eap_dtw(dev(S), dev(T), w, d * 1.01).item()
    assert dist_close(got2, d, max(n, m))


def test_lone_diagonal_path_is_not_abandoned():
    """S = T = 0, 1, 2, ...: only the diagonal is within ub = 0.5 (every other
    cell costs at least 1), so the live region is one cell wide and crosses
    every block boundary diagonally; the wavefront must not take such a
    crossing for a dead row."""
    for m in (33, 50, 70, 100, 300, 1000):
        S = np.arange(m, dtype=np.float32)
        for w in (m, 10, 3):
            assert api.eap_dtw(dev(S), dev(S), w=w, ub=0.5).item() == 0.0, (m, w)
