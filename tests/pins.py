"""Checks that pin the oracle to facts fixed by the paper and by mathematics.

Each check returns a list of failure messages (empty = pass).  They are used
by tests/test_oracle.py directly, and by the planted-mistake tests, which build
a deliberately broken copy of oracle.c and require at least one check to fail.

Pins (none of them re-types the oracle's own formula):
  - the worked example of the paper (tests/golden/worked_example.txt);
  - DTW by enumerating every warping path on tiny inputs (Section 2: the
    optimal warping path is the cheapest continuous monotone path);
  - closed forms: w = 0 is the squared Euclidean distance (Section 2.1),
    DTW(S, S) = 0, symmetry, unconstrained windows, no admissible path;
  - EAPrunedDTW returns DTW when DTW <= ub and +inf only when DTW > ub
    (Section 2.2, Algorithm 3);
  - lower bounds never exceed DTW (Section 2.2);
  - z-normalisation against numpy's mean/std;
  - the w = 0 search against an FFT sliding-dot-product z-normalised
    Euclidean profile (d^2 = 2m(1 - rho)), an independent method.
"""
from __future__ import annotations

import math
import os

import numpy as np

import oracle as O

INF = math.inf
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "worked_example.txt")


def load_golden(path: str = GOLDEN) -> dict:
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            out[k] = v
    return out


def _cells(s: str):
    return [tuple(int(x) for x in p.split(",")) for p in s.split()]


def path_enumeration_dtw(S, T, w) -> float:
    """Minimum cost over every warping path within the band (no recurrence)."""
    n, m = len(S), len(T)
    best = INF
    stack = [(0, 0, (S[0] - T[0]) ** 2)]
    while stack:
        i, j, acc = stack.pop()
        if i == n - 1 and j == m - 1:
            best = min(best, acc)
            continue
        for di, dj in ((1, 0), (0, 1), (1, 1)):
            a, b = i + di, j + dj
            if a < n and b < m and abs(a - b) <= w:
                stack.append((a, b, acc + (S[a] - T[b]) ** 2))
    return best


def check_worked_example() -> list:
    g = load_golden()
    fails = []
    S = [float(x) for x in g["S"].split()]
    T = [float(x) for x in g["T"].split()]
    d, M = O.dtw_matrix(S, T)
    if d != float(g["dtw"]):
        fails.append(f"worked example: Eq.1-5 DTW {d} != {g['dtw']}")
    if O.dtw(S, T) != float(g["dtw"]):
        fails.append("worked example: Algorithm 1 DTW mismatch")
    if M[3, 4] != float(g["cell_3_4"]):
        fails.append(f"worked example: cell (3,4) {M[3, 4]}")
    if M[2, 2] != float(g["cell_2_2"]):
        fails.append(f"worked example: cell (2,2) {M[2, 2]}")
    for (i, j) in _cells(g["ub9_discard"]) + _cells(g["ub9_above_ub"]):
        if not M[i, j] > 9:
            fails.append(f"worked example: cell ({i},{j}) = {M[i, j]} should exceed ub = 9")
    v, tr = O.eapruned_dtw(S, T, ub=9, trace=True)
    if v != float(g["ub9_result"]) or tr["abandon_row"] != 0:
        fails.append(f"worked example: EAPrunedDTW(ub=9) = {v}, abandon row {tr['abandon_row']}")
    v2, row = O.dtw_prune_left(S, T, 6)
    if v2 != INF or row != int(g["alg2_ub6_abandon_row"]):
        fails.append(f"worked example: Algorithm 2 (ub=6) = {v2}, abandon row {row}")
    v, tr = O.eapruned_dtw(S, T, ub=6, trace=True)
    pp = tr["pruning_point"]
    for (i, j) in _cells(g["ub6_pruning_points"]):
        if i > len(pp) or pp[i - 1] != j:
            fails.append(f"worked example: pruning point of row {i} is "
                         f"{pp[i - 1] if i <= len(pp) else None}, expected {j}")
    ci, cj = _cells(g["ub6_collision"])[0]
    if v != INF or tr["abandon_row"] != ci or tr["next_start"][ci - 1] != cj or not M[ci, cj] > 6:
        fails.append(f"worked example: EAPrunedDTW(ub=6) = {v}, abandon row {tr['abandon_row']}")
    return fails


def check_path_enumeration(ncases: int = 150, seed: int = 11) -> list:
    rng = np.random.default_rng(seed)
    fails = []
    for _ in range(ncases):
        n, m = int(rng.integers(1, 7)), int(rng.integers(1, 7))
        S = rng.integers(0, 5, n).astype(float)
        T = rng.uniform(-2, 2, m).round(2)
        w = int(rng.integers(0, 7))
        ref = path_enumeration_dtw(S, T, w)
        for name, got in (("Eq.1-5", O.dtw_matrix(S, T, w)[0]), ("Alg.1", O.dtw(S, T, w)),
                          ("Alg.3", O.eapruned_dtw(S, T, w, INF))):
            if not (got == ref or (math.isfinite(ref) and abs(got - ref) <= 1e-12 * max(1, ref))):
                fails.append(f"path enumeration: {name} {got} != {ref} (n={n} m={m} w={w})")
                break
        if len(fails) > 5:
            break
    return fails


def check_eapruned(ncases: int = 400, seed: int = 12) -> list:
    """Algorithm 3 returns DTW iff DTW <= ub, else +inf (Sections 2.2 and 4)."""
    rng = np.random.default_rng(seed)
    fails = []
    for c in range(ncases):
        n, m = int(rng.integers(1, 14)), int(rng.integers(1, 14))
        if c % 2:
            S = rng.integers(0, 5, n).astype(float)
            T = rng.integers(0, 5, m).astype(float)
        else:
            S = rng.standard_normal(n)
            T = rng.standard_normal(m)
        w = int(rng.integers(0, 15))
        d = O.dtw_matrix(S, T, w)[0]
        ubs = [INF, 0.0, float(rng.uniform(0, 40))]
        if math.isfinite(d):
            ubs += [d, d - 1, d + 1, math.nextafter(d, -INF), math.nextafter(d, INF)]
        for ub in ubs:
            got = O.eapruned_dtw(S, T, w, ub)
            exp = d if d <= ub else INF
            if got != exp:
                fails.append(f"EAPrunedDTW {got} != {exp} (n={n} m={m} w={w} ub={ub})")
        v2, _ = O.dtw_prune_left(S, T, ub=INF)
        if w >= max(n, m) and v2 != d:
            fails.append("Algorithm 2 with ub=inf differs from DTW")
        if len(fails) > 5:
            break
    return fails


def check_closed_forms(seed: int = 13) -> list:
    rng = np.random.default_rng(seed)
    fails = []
    for _ in range(60):
        n = int(rng.integers(1, 30))
        S, T = rng.standard_normal(n), rng.standard_normal(n)
        ed = float(np.sum((S - T) ** 2))
        if abs(O.dtw(S, T, 0) - ed) > 1e-12 * max(1, ed):
            fails.append("w = 0 is not the squared Euclidean distance")
        if abs(O.eapruned_dtw(S, T, 0, INF) - ed) > 1e-12 * max(1, ed):
            fails.append("EAPrunedDTW(w = 0) is not the squared Euclidean distance")
        w = int(rng.integers(0, n + 1))
        if O.dtw(S, S, w) != 0.0 or O.eapruned_dtw(S, S, w, 0.0) != 0.0:
            fails.append("DTW(S, S) != 0")
        m = int(rng.integers(1, 30))
        U = rng.standard_normal(m)
        wu = int(rng.integers(0, 32))
        if O.dtw(S, U, wu) != O.dtw(U, S, wu):
            fails.append("DTW is not symmetric")
        big = max(n, m) + 5
        if O.dtw(S, U, max(n, m) - 1) != O.dtw(S, U, big):
            fails.append("w = max(l) - 1 differs from unconstrained DTW")
        if abs(n - m) > 0 and O.dtw(S, U, abs(n - m) - 1) != INF:
            fails.append("w < |lS - lT| should admit no path")
        if O.dtw(S, U, wu + 1) > O.dtw(S, U, wu):
            fails.append("DTW increases with a wider window")
    return fails


def check_lower_bounds(seed: int = 14) -> list:
    rng = np.random.default_rng(seed)
    fails = []
    for _ in range(150):
        m = int(rng.integers(2, 40))
        w = int(rng.integers(0, m + 1))
        q = O.znorm(np.cumsum(rng.standard_normal(m)))
        raw = np.cumsum(rng.standard_normal(m + 2 * w + 6))
        off = w + 3
        mu, sd = O.mean_std(raw[off:off + m])
        c = (raw[off:off + m] - mu) / sd
        d = O.dtw(c, q, w)
        kim = O.lb_kim_fl(c, q)
        uq, lq = O.envelope(q, w)
        eq = O.lb_keogh(c, uq, lq)
        ur, lr = O.envelope(raw, w)
        uc, lc = (ur[off:off + m] - mu) / sd, (lr[off:off + m] - mu) / sd
        ec = O.lb_keogh(q, uc, lc)
        for name, lb in (("LB_Kim", kim), ("LB_Keogh EQ", eq), ("LB_Keogh EC", ec)):
            if lb > d * (1 + 1e-12) + 1e-12:
                fails.append(f"{name} {lb} > DTW {d} (m={m} w={w})")
        if w + 1 <= m:
            uq1, lq1 = O.envelope(q, w + 1)
            if O.lb_keogh(c, uq1, lq1) > eq + 1e-12:
                fails.append("LB_Keogh increases with a wider window")
        u0, l0 = O.envelope(q, 0)
        ed = float(np.sum((c - q) ** 2))
        if abs(O.lb_keogh(c, u0, l0) - ed) > 1e-12 * max(1, ed):
            fails.append("LB_Keogh(w = 0) is not the squared Euclidean distance")
    # LB_Kim <= LB_Keogh does not hold in general: q = (0, 5), c = (5, 5), w = 1.
    q, c = np.array([0.0, 5.0]), np.array([5.0, 5.0])
    uq, lq = O.envelope(q, 1)
    if not (O.lb_kim_fl(c, q) == 25.0 and O.lb_keogh(c, uq, lq) == 0.0 and O.dtw(c, q, 1) == 25.0):
        fails.append("LB_Kim / LB_Keogh counterexample changed")
    return fails


def check_znorm(seed: int = 15) -> list:
    rng = np.random.default_rng(seed)
    fails = []
    for _ in range(30):
        m = int(rng.integers(2, 200))
        x = rng.standard_normal(m) * rng.uniform(0.1, 100) + rng.uniform(-1e3, 1e3)
        ref = (x - x.mean()) / x.std()
        if np.max(np.abs(O.znorm(x) - ref)) > 1e-9:
            fails.append("z-normalisation differs from numpy mean/std")
        mu, sd = O.mean_std(x)
        if abs(mu - x.mean()) > 1e-9 * abs(x.mean()) + 1e-12 or abs(sd - x.std()) > 1e-9 * x.std():
            fails.append("mean/std differ from numpy")
    if np.any(O.znorm(np.full(17, 3.25)) != 0.0):
        fails.append("a constant window must normalise to zeros")
    return fails


def mass_zed2_profile(Q, R):
    """Squared z-normalised Euclidean distance of Q to every window of R via an
    FFT sliding dot product: d^2 = 2m(1 - rho) (textbook identity)."""
    Q = np.asarray(Q, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    m, n = len(Q), len(R)
    L = 1 << int(math.ceil(math.log2(n + m)))
    qt = np.fft.irfft(np.fft.rfft(R, L) * np.fft.rfft(Q[::-1], L), L)[m - 1:n]
    cs = np.concatenate([[0.0], np.cumsum(R)])
    cs2 = np.concatenate([[0.0], np.cumsum(R * R)])
    mu = (cs[m:] - cs[:-m]) / m
    sd = np.sqrt(np.maximum((cs2[m:] - cs2[:-m]) / m - mu * mu, 0))
    rho = (qt - m * Q.mean() * mu) / (m * Q.std() * sd)
    return 2 * m * (1 - rho)


def check_search(seed: int = 16, quick: bool = False) -> list:
    rng = np.random.default_rng(seed)
    fails = []
    cases = [(1200, 16, 0, 1), (1500, 24, 3, 3), (900, 20, 20, 2)]
    if not quick:
        cases += [(2500, 32, 4, 5), (1000, 12, 11, 1), (700, 40, 8, 4)]
    for n, m, w, k in cases:
        R = np.cumsum(rng.standard_normal(n))
        Q = np.cumsum(rng.standard_normal(m))
        bi, bd = O.search_brute(Q, R, w, k)
        # top-k against an explicit sort of every window's distance
        zq = O.znorm(Q)
        allv = np.array([O.dtw_matrix(O.znorm(R[i:i + m]), zq, w)[0] for i in range(n - m + 1)])
        order = np.lexsort((np.arange(len(allv)), allv))[:k]
        if list(bi) != list(order) or not np.allclose(bd, allv[order], rtol=0, atol=0):
            fails.append(f"brute-force top-{k} differs from sorting every window (n={n} m={m} w={w})")
        for use_lb in (True, False):
            for nthreads in (1, 3):
                ci, cd, cnt = O.search_cascade(Q, R, w, k, use_lb=use_lb, nthreads=nthreads)
                if list(ci) != list(bi) or list(cd) != list(bd):
                    fails.append(f"cascade (lb={use_lb}, threads={nthreads}) differs from brute force")
                tot = sum(cnt[x] for x in ("kim_pruned", "eq_pruned", "ec_pruned",
                                           "dtw_abandoned", "dtw_completed"))
                if tot != cnt["windows"] or cnt["windows"] != n - m + 1:
                    fails.append("cascade counters do not add up")
        ai, ad, _ = O.search_cascade(Q, R, w, k, ub_fixed=bd[-1])
        if list(ai) != list(bi) or list(ad) != list(bd):
            fails.append("audit-mode cascade differs from brute force")
    # w = 0 against the FFT profile
    R = np.cumsum(rng.standard_normal(3000))
    Q = np.cumsum(rng.standard_normal(64))
    prof = mass_zed2_profile(Q, R)
    bi, bd = O.search_brute(Q, R, 0, 3)
    ref = np.sort(prof)[:3]
    if not np.allclose(bd, ref, rtol=1e-7, atol=1e-9):
        fails.append(f"w = 0 search {bd} differs from the FFT z-ED profile {ref}")
    for i, d in zip(bi, bd):
        if abs(prof[i] - d) > 1e-7 * max(d, 1e-6):
            fails.append("w = 0 search index is not a minimiser of the FFT profile")
    # exact distance ties: a periodic reference repeats the query's window, and
    # equal distances must come back in ascending window order
    pat = np.round(rng.standard_normal(50), 3)
    R = np.tile(pat, 8)
    Q = pat[5:25].copy()
    bi, bd = O.search_brute(Q, R, 2, 3)
    if list(bi) != [5, 55, 105] or list(bd) != [0.0, 0.0, 0.0]:
        fails.append(f"distance ties must go to the smaller window start, got {list(bi)}")
    # k larger than the number of windows
    idx, dist = O.search_brute(Q[:10], R[:12], 2, 5)
    if list(idx[3:]) != [-1, -1] or not all(math.isinf(x) for x in dist[3:]):
        fails.append("extra k slots must be (-1, inf)")
    return fails


ALL = (check_worked_example, check_path_enumeration, check_eapruned, check_closed_forms,
       check_lower_bounds, check_znorm, check_search)


def all_checks(quick: bool = False) -> list:
    fails = []
    for chk in ALL:
        if chk is check_search:
            fails += chk(quick=quick)
        elif quick and chk in (check_path_enumeration, check_eapruned):
            fails += chk(ncases=60)
        else:
            fails += chk()
    return fails
