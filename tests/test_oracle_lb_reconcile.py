"""The FP32-emulating oracle's lower-bound decisions against the FP64
definitions, window by window.

Section 2.2: a lower bound skips a candidate only when it exceeds the upper
bound; Section 5 runs LB_Kim, then LB_Keogh EQ, then LB_Keogh EC, then
EAPrunedDTW.  The FP64 side here is the cascade restated in Python from the
oracle's own definitions (two-pass z-normalisation, lb_kim_fl, lb_keogh over
the query envelope, lb_keogh of the query over the window's normalised raw
envelope of radius min(w, m - 1), full DTW), pinned to orc_search_cascade's
audit counts.  The FP32-emulating mode (oracle_f32.c, which the GPU must match
bit for bit) decides each window under the same fixed bound ub but prunes only
above fl32(ub (1 + 1e-4)) and rounds its sums to FP32.  So the two may
disagree only on windows whose deciding FP64 bound lies within the margin of
ub, or whose FP64 and FP32 DTW straddle ub.  Every other window must get the
same outcome (the same bound, or the same DTW decision), and the exceptions
are listed and bounded.  Two mistakes that leave every bound valid, and so
pass the other pins, must be caught: the EC envelope over radius w instead of
min(w, m - 1), and LB_Keogh EQ reading the window in natural order against the
envelope in LB order."""
import numpy as np
import pytest

import oracle as O
from paper_2010_05371_gb300 import synth

MARGIN = 2e-4   # the 1e-4 pruning margin plus FP32 rounding of the bounds


def fp64_outcomes(Q, R, w, ub):
    """(outcome per window: 1 Kim, 2 EQ, 3 EC, 4 abandoned, 5 completed;
    the FP64 value each window was decided on)."""
    m = len(Q)
    nw = len(R) - m + 1
    zq = O.znorm(Q)
    uq, lq = O.envelope(zq, w)
    ur, lr = O.envelope(R, min(w, m - 1))
    mu, sd = O.window_stats(R, m)
    why = np.zeros(nw, np.int8)
    val = np.zeros(nw)
    for i in range(nw):
        s = sd[i]
        zc = (R[i:i + m] - mu[i]) / s if s > 0 else np.zeros(m)
        kim = O.lb_kim_fl(zc, zq)
        if kim > ub:
            why[i], val[i] = 1, kim
            continue
        eq = O.lb_keogh(zc, uq, lq)
        if eq > ub:
            why[i], val[i] = 2, eq
            continue
        uc = (ur[i:i + m] - mu[i]) / s if s > 0 else np.zeros(m)
        lc = (lr[i:i + m] - mu[i]) / s if s > 0 else np.zeros(m)
        ec = O.lb_keogh(zq, uc, lc)
        if ec > ub:
            why[i], val[i] = 3, ec
            continue
        d = O.dtw(zc, zq, w)
        why[i], val[i] = (5 if d <= ub else 4), d
    return why, val


def _bounds64(Q, R, w, i):
    """The three FP64 bounds and the DTW of window i."""
    m = len(Q)
    zq = O.znorm(Q)
    uq, lq = O.envelope(zq, w)
    ur, lr = O.envelope(R, min(w, m - 1))
    mu, sd = O.mean_std(R[i:i + m])
    zc = (R[i:i + m] - mu) / sd
    uc = (ur[i:i + m] - mu) / sd
    lc = (lr[i:i + m] - mu) / sd
    return {1: O.lb_kim_fl(zc, zq), 2: O.lb_keogh(zc, uq, lq), 3: O.lb_keogh(zq, uc, lc),
            4: O.dtw(zc, zq, w)}


def unexplained(Q, R, w, ub, why64, why32):
    """Windows whose outcomes differ for a reason other than the margin: the
    first stage where the two disagree must have its FP64 value within the
    margin of ub (a bound) or straddle ub (the DTW)."""
    bad, explained = [], []
    for i in np.nonzero(why64 != why32)[0]:
        b = _bounds64(Q, R, w, int(i))
        stage = min(int(why64[i]), int(why32[i]), 4)
        v = b[stage]
        tol = MARGIN if stage <= 3 else 1e-4
        (explained if abs(v - ub) <= tol * ub else bad).append((int(i), int(why64[i]), int(why32[i]), v))
    return bad, explained


CASES = [  # (series, n, m, w, ub factor over the nearest-neighbour distance)
    ("walk", 12_000, 128, 13, 1.0),
    ("walk", 12_000, 128, 128, 1.0),
    ("walk", 12_000, 96, 96, 1.4),
    ("ecg", 12_000, 200, 20, 1.2),
    ("ecg", 12_000, 200, 200, 1.0),
]


def _case(series, n, m, w, f, seed):
    if series == "walk":
        R = synth.random_walk(n, 300 + seed)
        Q = synth.random_walk(m, 400 + seed)
    else:
        R = synth.ecg_like(n, 300 + seed)
        Q = synth.ecg_query(m, 400 + seed)
    _, d, _ = O.search_cascade(Q, R, w, 1, nthreads=4)
    return Q, R, float(d[0]) * f


@pytest.mark.parametrize("series,n,m,w,f", CASES)
def test_fp64_restatement_matches_the_c_cascade(series, n, m, w, f):
    """The Python FP64 outcomes reproduce orc_search_cascade's audit counts."""
    Q, R, ub = _case(series, n, m, w, f, 0)
    why64, _ = fp64_outcomes(Q, R, w, ub)
    _, _, c = O.search_cascade(Q, R, w, 1, use_lb=True, ub_fixed=ub, nthreads=4)
    got = [int(np.sum(why64 == s)) for s in (1, 2, 3, 4, 5)]
    assert got == [c["kim_pruned"], c["eq_pruned"], c["ec_pruned"], c["dtw_abandoned"], c["dtw_completed"]], (got, c)


@pytest.mark.parametrize("series,n,m,w,f", CASES)
def test_fp32_lower_bound_decisions_agree_with_fp64(series, n, m, w, f):
    Q, R, ub = _case(series, n, m, w, f, 1)
    why64, _ = fp64_outcomes(Q, R, w, ub)
    _, _, _, why32 = O.o7_search(Q, R, w, 1, audit_ub=ub, return_why=True)
    bad, explained = unexplained(Q, R, w, ub, why64, why32)
    assert not bad, bad[:10]
    assert len(explained) <= max(3, len(why64) // 500), explained
    # every stage decides windows in both, so each bound is exercised
    for s in (1, 2, 3):
        assert np.sum(why32 == s) > 0 and np.sum(why64 == s) > 0, (s, np.bincount(why32))


MUTANTS = [
    ("EC envelope over radius w instead of min(w, m - 1)",
     "const int64_t re = wi < m - 1 ? wi : m - 1;", "const int64_t re = wi;"),
    ("LB_Keogh EQ reads the window in natural order against the envelope in LB order",
     "const float zz = znorm1(R[i + ord[p]], a, cw, isd);", "const float zz = znorm1(R[i + p], a, cw, isd);"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS)
def test_reconciliation_catches_planted_mistakes(desc, old, new, tmp_path):
    src = O.source_text_f32()
    assert old in src, desc
    L = O.compile_variant_f32(src.replace(old, new, 1), str(tmp_path))
    caught = False
    for series, n, m, w, f in CASES:
        if "radius" in desc and w < m:
            continue   # the radius differs only when w >= m
        Q, R, ub = _case(series, n, m, w, f, 1)
        why64, _ = fp64_outcomes(Q, R, w, ub)
        _, _, _, why32 = O.o7_search(Q, R, w, 1, audit_ub=ub, return_why=True, L=L)
        bad, explained = unexplained(Q, R, w, ub, why64, why32)
        if bad or len(explained) > max(3, len(why64) // 500):
            caught = True
            break
    assert caught, desc
