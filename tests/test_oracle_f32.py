"""Pins of the FP32-emulating oracle mode (oracle_f32.c) against what does not
depend on it: correctly rounded arithmetic computed with Python's decimal
module, sums that are exact on integer data, the FP64 oracle's definitions of
DTW and z-normalisation, and invariants of the audit cascade."""
import math
import random
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle as O
from paper_2010_05371_gb300 import synth


def f32_neighbours(f):
    f = np.float32(f)
    return [np.nextafter(f, np.float32(0)), f, np.nextafter(f, np.float32(np.inf))]


def rsqrt_reference(v: float) -> np.float32:
    """The float32 nearest to v^(-1/2), decided in 60-digit decimal arithmetic."""
    getcontext().prec = 60
    r = Decimal(1) / Decimal(float(v)).sqrt()
    cand = f32_neighbours(np.float32(1.0 / math.sqrt(float(v))))
    return min(cand, key=lambda c: abs(Decimal(float(c)) - r))


def test_rsqrt_is_correctly_rounded():
    rnd = random.Random(5)
    vals = [4.0, 1.0, 0.25, 2.0, 3.0, 1e-30, 3.4e38, 1.17549435e-38, 0.999999940, 1.00000012]
    vals += [math.ldexp(rnd.uniform(1.0, 2.0), rnd.randint(-120, 120)) for _ in range(3000)]
    for v in vals:
        v32 = float(np.float32(v))
        got = np.float32(O.o7_rsqrt_rn(v32))
        assert got == rsqrt_reference(v32), v32


def test_prefix_sums_exact_on_integer_data():
    """Integer-valued series: every FP64 sum is exact, so the emulated block
    scan must give exactly the exclusive prefix sums of (x - anchor) per chunk."""
    rng = np.random.default_rng(2)
    n = 3 * 4096 + 777
    R = rng.integers(-50, 50, size=n).astype(np.float32)
    P1, P2, T1, T2, A = O.o7_ref_prefix(R)
    for c in range((n + 4095) // 4096):
        lo, hi = c * 4096, min(n, (c + 1) * 4096)
        a = int(R[lo])
        d = [int(x) - a for x in R[lo:hi]]
        assert A[c] == R[lo]
        e1 = np.concatenate([[0], np.cumsum(d)[:-1]])
        e2 = np.concatenate([[0], np.cumsum(np.square(d))[:-1]])
        np.testing.assert_array_equal(P1[lo:hi], e1)
        np.testing.assert_array_equal(P2[lo:hi], e2)
        assert T1[c] == sum(d) and T2[c] == sum(x * x for x in d)


def test_prefix_sums_close_on_random_walk():
    R = synth.random_walk(10_000, 3).astype(np.float32)
    P1, P2, T1, T2, A = O.o7_ref_prefix(R)
    for c in range(3):
        lo, hi = c * 4096, min(len(R), (c + 1) * 4096)
        d = R[lo:hi].astype(np.float64) - float(R[lo])
        np.testing.assert_allclose(P1[lo + 1:hi], np.cumsum(d)[:-1], rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(P2[lo + 1:hi], np.cumsum(d * d)[:-1], rtol=1e-12, atol=1e-9)


def test_window_coefficients_match_the_definition():
    R = synth.random_walk(12_000, 4).astype(np.float32)
    m = 300
    wins = [0, 1, 4000, 4095 - 150, 8191, len(R) - m]
    co = O.o7_window_coeffs(R, m, wins)
    for (a, cw, isd), i in zip(co, wins):
        x = R[i:i + m].astype(np.float64)
        mu, sd = x.mean(), x.std()
        assert a == R[i]
        assert abs(float(cw) - (mu - float(a))) <= 1e-6 * max(1.0, abs(mu - float(a)))
        assert abs(float(isd) * sd - 1.0) <= 1e-6
    # zero variance normalises to zeros; a large offset takes the two-pass path
    flat = np.full(500, 7.25, dtype=np.float32)
    assert tuple(O.o7_window_coeffs(flat, 100, [3])[0][1:]) == (0.0, 0.0)
    # far from its chunk's anchor (var <= 1e-6 of the anchored second moment)
    jump = np.concatenate([np.zeros(100), 1000.0 + np.random.default_rng(1).normal(0, 0.5, 900)])
    jump = jump.astype(np.float32)
    a, cw, isd = O.o7_window_coeffs(jump, 200, [500])[0]
    x = jump[500:700].astype(np.float64)
    assert abs(float(isd) * x.std() - 1.0) <= 1e-6
    assert abs(float(cw) - (x.mean() - float(a))) <= 1e-5


def test_query_prep_matches_the_definition():
    Q = synth.random_walk(300, 6).astype(np.float32)
    for w in (0, 7, 299, 1000):
        zq, uq, lq, zqo, order = O.o7_query_prep(Q, w)
        np.testing.assert_allclose(zq, O.znorm(Q.astype(np.float64)), rtol=0, atol=2e-6)
        mag = np.abs(zq)
        assert sorted(order.tolist()) == list(range(300))
        for p in range(299):
            a, b = order[p], order[p + 1]
            assert mag[a] > mag[b] or (mag[a] == mag[b] and a < b)
        r = min(w, 299)
        for p, j in enumerate(order):
            lo, hi = max(0, j - r), min(299, j + r)
            assert uq[p] == zq[lo:hi + 1].max() and lq[p] == zq[lo:hi + 1].min()
            assert zqo[p] == zq[j]


def test_dtw_f32_exact_on_integer_data_and_close_otherwise():
    rng = np.random.default_rng(8)
    for trial in range(40):
        m = int(rng.integers(1, 30))
        w = int(rng.integers(0, m + 1))
        z = rng.integers(-4, 5, size=m).astype(np.float32)
        q = rng.integers(-4, 5, size=m).astype(np.float32)
        assert O.o7_dtw_f32(z, q, w) == O.dtw(z.astype(np.float64), q.astype(np.float64), w)
    for trial in range(20):
        m = int(rng.integers(20, 120))
        w = int(rng.integers(0, m))
        z, q = rng.normal(size=m).astype(np.float32), rng.normal(size=m).astype(np.float32)
        ref = O.dtw(z.astype(np.float64), q.astype(np.float64), w)
        assert abs(O.o7_dtw_f32(z, q, w) - ref) <= 1e-5 * ref


@pytest.mark.parametrize("m,w,k", [(64, 6, 1), (96, 96, 3), (50, 0, 2)])
def test_exact_search_agrees_with_fp64_brute_force(m, w, k):
    R = synth.random_walk(3000, 11).astype(np.float32)
    Q = synth.random_walk(m, 12).astype(np.float32)
    gi, gd, _ = O.o7_search(Q, R, w, k)
    oi, od = O.search_brute(Q.astype(np.float64), R.astype(np.float64), w, k)
    for j in range(k):
        assert abs(gd[j] - od[j]) <= 1e-4 * od[j]
        if gi[j] != oi[j]:
            z = O.znorm(R[gi[j]:gi[j] + m].astype(np.float64))
            assert abs(O.dtw(z, O.znorm(Q.astype(np.float64)), w) - od[j]) <= 1e-4 * od[j]


def test_audit_cascade_invariants():
    """Counts partition the windows; a window is completed iff its FP32 DTW is
    within the bound (checked window by window); no lower bound prunes a window
    whose DTW is within the bound; with the bound at the exact k-th distance the
    audit result is the exact result."""
    R = synth.random_walk(2500, 21).astype(np.float32)
    Q = synth.random_walk(60, 22).astype(np.float32)
    w, k = 9, 3
    ei, ed, _ = O.o7_search(Q, R, w, k)
    ub = np.float32(ed[-1])
    ai, ad, c = O.o7_search(Q, R, w, k, audit_ub=float(ub))
    assert sum(c[x] for x in O.O7_COUNTER_NAMES[1:]) == c["windows"] == len(R) - len(Q) + 1
    np.testing.assert_array_equal(ai, ei)
    np.testing.assert_array_equal(ad, ed)
    co = O.o7_window_coeffs(R, len(Q))
    zq = O.o7_query_prep(Q, w)[0]
    within = 0
    for i, (a, cw, isd) in enumerate(co):
        z = ((R[i:i + len(Q)] - a) - cw) * isd
        within += O.o7_dtw_f32(z.astype(np.float32), zq, w) <= ub
    assert c["dtw_completed"] == within
    _, _, c0 = O.o7_search(Q, R, w, k, audit_ub=float(ub), use_lb=False)
    assert c0["dtw_completed"] == within and c0["kim_pruned"] == 0


MUTANTS_F32 = [
    # (description, text to replace, replacement)
    ("rsqrt of the square", "float y = (float)(1.0 / sqrt((double)v));", "float y = (float)(1.0 / (double)v);"),
    ("prefix of the wrong chunk anchor", "const float anchor = R[base];", "const float anchor = R[base] + 1.0f;"),
    ("inclusive prefix stored instead of exclusive", "P1[base + j] = r1;", "P1[base + j] = r1 + d[j];"),
    ("dropped diagonal", "fminf(fminf(prev[c], prev[c - 1]), curr[c - 1])", "fminf(prev[c], curr[c - 1])"),
    ("ties in the LB order by descending position", "return p->j < q->j ? -1 : (p->j > q->j);",
     "return p->j > q->j ? -1 : (p->j < q->j);"),
    ("query envelope radius w + 1", "const int64_t wc = w < m - 1 ? w : m - 1;",
     "const int64_t wc = w + 1 < m - 1 ? w + 1 : m - 1;"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS_F32, ids=[m[0] for m in MUTANTS_F32])
def test_pins_catch_planted_mistakes(desc, old, new, tmp_path):
    src = O.source_text_f32()
    assert old in src, desc
    L = O.compile_variant_f32(src.replace(old, new, 1), str(tmp_path))
    caught = []
    for test in (lambda: _rsqrt_pin(L), lambda: _prefix_pin(L), lambda: _dtw_pin(L), lambda: _query_pin(L)):
        try:
            test()
        except AssertionError:
            caught.append(True)
    assert caught, f"no pin caught: {desc}"


def _rsqrt_pin(L):
    rnd = random.Random(3)
    for _ in range(400):
        v = float(np.float32(math.ldexp(rnd.uniform(1.0, 2.0), rnd.randint(-60, 60))))
        assert np.float32(O.o7_rsqrt_rn(v, L)) == rsqrt_reference(v)


def _prefix_pin(L):
    R = np.random.default_rng(2).integers(-50, 50, size=5000).astype(np.float32)
    P1, P2, T1, T2, A = O.o7_ref_prefix(R, L)
    d = R[:4096].astype(np.int64) - int(R[0])
    np.testing.assert_array_equal(P1[:4096], np.concatenate([[0], np.cumsum(d)[:-1]]))
    assert A[0] == R[0]


def _dtw_pin(L):
    rng = np.random.default_rng(8)
    for _ in range(20):
        m = int(rng.integers(2, 20))
        w = int(rng.integers(0, m + 1))
        z = rng.integers(-4, 5, size=m).astype(np.float32)
        q = rng.integers(-4, 5, size=m).astype(np.float32)
        assert O.o7_dtw_f32(z, q, w, L) == O.dtw(z.astype(np.float64), q.astype(np.float64), w)


def _query_pin(L):
    Q = np.array([3, -1, 2, -2, 1, 0, 0, 5, -5, 1], dtype=np.float32)  # ties in |zq|
    for w in (0, 2):
        zq, uq, lq, zqo, order = O.o7_query_prep(Q, w, L)
        mag = np.abs(zq)
        for p in range(len(Q) - 1):
            a, b = order[p], order[p + 1]
            assert mag[a] > mag[b] or (mag[a] == mag[b] and a < b)
        for p, j in enumerate(order):
            lo, hi = max(0, j - w), min(len(Q) - 1, j + w)
            assert uq[p] == zq[lo:hi + 1].max()
