"""A lane-by-lane model of the narrow-block elastic wavefront's schedule
(csrc/dtw_elastic.cuh), checked against the oracle's DTW.

The model restates, in numpy, the wavefront's control logic: 32 lanes per
window, up to J windows of blocks of 4 columns, two rows per step computed
along anti-diagonals, left inputs passed one lane per step (lane 0 of window j
from lane 31 of window j - 1), NaN rows before and after the window's rows and
NaN columns after the query's, checks every 8 steps (all blocks dead at two
consecutive steps abandons; retirable leading blocks; windows switched on
when an alive block comes within 9 blocks of the end of the last one, off when
they are no longer needed; lazy slides; an overflow when J windows do not
suffice), the rows written on demand 64 at a time before the interval that
first reads them, and the final step's capture of cell (nr, nc).  It asserts every
index it reads from the row and column buffers, as the kernel's shared-memory
buffers are sized, and its outcomes must agree with Eq. 1-5 (the oracle's DTW):
a finished value equals DTW when DTW <= ub, an abandoned candidate has
DTW > ub.  Cells are rounded to FP32 after an exact product and sum (the
kernel's fma)."""
import numpy as np
import pytest

import oracle as O
from paper_2010_05371_gb300 import synth

f32 = np.float32
INF = f32(np.inf)
NAN = f32(np.nan)
FMAX = f32(3.402823466e38)
FULL = 0xffffffff
K, R = 4, 2
CE = 8   # the kernel's default check interval; the tests also run 4


def _ballot(pred):
    return int(np.sum(np.asarray(pred, dtype=np.int64) << np.arange(32, dtype=np.int64)))


def _clz(x):
    return 32 - int(x).bit_length()


def _ffs(x):
    return (x & -x).bit_length() if x else 0


def emu(rows, cols, ub, J=3, ub_sched=None, CE=CE, w=None):
    nr, nc = len(rows), len(cols)
    padr = R * 32 * J
    padc = 32 * J * K
    rowf = (2 * padr + nr + R + 3) // 4 * 4
    colf = (nc + padc + 3) // 4 * 4
    zr = np.full(rowf, NAN, f32)
    zr[padr:padr + nr] = -np.asarray(rows, f32)   # the kernel keeps -z: d = q + (-z)
    zq = np.full(colf, NAN, f32)
    zq[:nc] = cols
    lanes = np.arange(32)

    p = np.full((J, 32, K), INF, f32)
    q = np.zeros((J, 32, K), f32)
    lo0 = np.full((J, 32), INF, f32)
    lo1 = np.full((J, 32), INF, f32)
    dg = np.full((J, 32), INF, f32)
    st = {"B0": 0, "jact": 1}

    def load_q(j):
        base = (st["B0"] + 32 * j + lanes) * K
        assert base.min() >= 0 and base.max() + K <= colf, ("column read", base.max(), colf)
        for k in range(K):
            q[j, :, k] = zq[base + k]

    def reset(j):
        p[j] = INF; lo0[j] = INF; lo1[j] = INF; dg[j] = INF

    load_q(0)
    dg[0, 0] = 0.0
    ub = f32(min(ub, FMAX))
    ub_next = ub
    bm = (nc - 1) // K
    km = (nc - 1) - bm * K
    t_end = bm + 1 + (nr - 1) // 2
    last_first = nr % 2 == 1
    nre = (nr + 1) & ~1
    zoff = np.zeros((J, 32), np.int64)

    def set_zoff(tnow):
        for j in range(J):
            o = -2 * (1 + st["B0"] + 32 * j + lanes)
            zoff[j] = np.minimum(o, nre - 2 * (tnow + 1))

    set_zoff(0)
    FILL = 64   # rows written ahead (the kernel's kElFillRows)
    fl = {"filled": min(nr, FILL)}

    def fill_to(need):
        need = min(need, nr)
        if need > fl["filled"]:
            fl["filled"] = min(nr, max(need, fl["filled"] + FILL))

    def cost(qv, nz, mn):
        d = (qv + nz).astype(f32)
        with np.errstate(invalid="ignore"):
            return (d.astype(np.float64) * d.astype(np.float64) + mn.astype(np.float64)).astype(f32)

    def fmin3(a, b, c):
        return np.fmin(np.fmin(a, b), c)

    def step(s, which, cap, bma, bmb, capture):
        jact = st["jact"]
        l0 = np.empty((J, 32), f32); l1 = np.empty((J, 32), f32)
        for j in range(jact):
            s0 = lo0[j].copy(); s1 = lo1[j].copy()
            s0[31] = lo0[j - 1][31] if j > 0 else INF
            s1[31] = lo1[j - 1][31] if j > 0 else INF
            src = (lanes + 31) & 31
            l0[j] = s0[src]; l1[j] = s1[src]
        for j in range(jact):
            idx = zoff[j] + 2 * s
            assert (padr + idx).min() >= 0 and (padr + idx + 1).max() < rowf, ("row read", idx.min(), idx.max())
            for r in (idx, idx + 1):   # a row inside the window's rows has been written
                inside = (r >= 0) & (r < nr)
                assert np.all(r[inside] < fl["filled"]), ("row read before it was written", r.max(), fl["filled"])
            z0 = zr[padr + idx]; z1 = zr[padr + idx + 1]
            a0 = cost(q[j, :, 0], z0, fmin3(p[j, :, 0], dg[j], l0[j]))
            a1 = cost(q[j, :, 1], z0, fmin3(p[j, :, 1], p[j, :, 0], a0))
            b0 = cost(q[j, :, 0], z1, fmin3(a0, l0[j], l1[j]))
            a2 = cost(q[j, :, 2], z0, fmin3(p[j, :, 2], p[j, :, 1], a1))
            b1 = cost(q[j, :, 1], z1, fmin3(a1, a0, b0))
            a3 = cost(q[j, :, 3], z0, fmin3(p[j, :, 3], p[j, :, 2], a2))
            b2 = cost(q[j, :, 2], z1, fmin3(a2, a1, b1))
            b3 = cost(q[j, :, 3], z1, fmin3(a3, a2, b2))
            if cap >= 0 and j == cap >> 5:
                ra = [a0, a1, a2, a3][km]; rb = [b0, b1, b2, b3][km]
                capture[:] = ra if last_first else rb
            p[j, :, 0] = b0; p[j, :, 1] = b1; p[j, :, 2] = b2; p[j, :, 3] = b3
            lo0[j] = a3; lo1[j] = b3; dg[j] = l1[j]
            mn = fmin3(fmin3(b0, b1, b2), b3, a3)
            if which == 1: bma[j] = mn
            if which == 2: bmb[j] = mn
            if w is not None:
                # banded: every alive cell computed lies in the band
                b = st["B0"] + 32 * j + lanes
                for row_off, vals in ((1, (a0, a1, a2, a3)), (2, (b0, b1, b2, b3))):
                    r = 2 * (s - 1 - b) + row_off
                    for k, v in enumerate(vals):
                        c = 4 * b + 1 + k
                        bad = (v <= ub) & (r >= 1) & (r <= nr) & (c <= nc) & (np.abs(r - c) > w)
                        assert not bad.any(), ("alive cell outside the band", s, int(np.argmax(bad)))

    if w is not None and w < 4 * CE:
        return ("ovf", 0), None
    t = 0
    while True:
        jact = st["jact"]
        if t + CE < t_end:
            fill_to(2 * (t + CE))
            bma = np.full((J, 32), INF, f32); bmb = np.full((J, 32), INF, f32)
            for s in range(1, CE + 1):
                step(t + s, 1 if s == CE - 1 else (2 if s == CE else 0), -1, bma, bmb, None)
            t += CE
            ub = f32(min(ub, ub_next))
            if ub_sched is not None:
                ub_next = f32(min(ub_next, ub_sched(t)))
            da = [FULL] * J; db = [FULL] * J
            all_dead = True; hi = -1
            for j in range(jact):
                da[j] = _ballot([not (x <= ub) for x in bma[j]])
                db[j] = _ballot([not (x <= ub) for x in bmb[j]])
                al = (~(da[j] & db[j])) & FULL
                all_dead = all_dead and al == 0
                if al: hi = 32 * j + 31 - _clz(al)
            cond = db[0] & (((da[0] << 1) | 1) & FULL)
            if all_dead or (jact == 1 and cond == FULL):
                return ("abandon", t), None
            d = 32 if cond == FULL else _ffs(~cond & FULL) - 1
            B0 = st["B0"]
            if w is not None and (6 * (B0 + hi) - 2 * t + 4 * CE + 5 > w or 2 * (t + CE) - 6 * (B0 + d) - 1 > w):
                return ("ovf", t), None   # an alive cell may leave the band: the banded levels re-run it

            def need(shift):
                nd = int((hi - shift + CE + 1) / 32) + 1   # C integer division truncates toward zero
                cap_w = (bm - (B0 + shift)) // 32 + 1
                nd = min(nd, cap_w)
                return max(nd, 1)

            n0 = need(0); nnew = n0; shift = 0
            if d > 0:
                nd = need(d)
                if nd < jact or n0 > jact:
                    shift = d; nnew = nd
            if nnew > J:
                return ("ovf", t), None
            if shift > 0:
                st["B0"] += shift
                src = (lanes + shift) & 31
                nxt = lanes < shift
                for j in range(jact):
                    on = j + 1 < jact
                    for arr in (p, lo0, lo1, dg):
                        nx = arr[j + 1] if on else np.full_like(arr[j], INF)
                        if arr.ndim == 3:
                            send = np.where(nxt[:, None], nx, arr[j])
                        else:
                            send = np.where(nxt, nx, arr[j])
                        arr[j] = send[src]
                    load_q(j)
            for j in range(J):
                if jact <= j < nnew:   # switched on: +inf state (switched-off windows keep stale values)
                    reset(j)
                    load_q(j)
            st["jact"] = nnew
            if shift > 0 or t + 2 * CE >= st["B0"] + (nre >> 1):
                set_zoff(t)
            continue
        src = bm - st["B0"]
        fill_to(nr)
        fin = np.full(32, INF, f32)
        for s in range(t + 1, t_end + 1):
            step(s, 0, src if (s == t_end and src >= 0) else -1, None, None, fin)
        val = fin[src & 31]
        if src < 0 or src >= 32 * st["jact"]:
            val = INF
        val = val if val <= INF else INF
        return ("done", t_end), val


def _check(s, val, d, ub, eff_ub, tag):
    if s == "done":
        if d <= ub * (1 - 1e-3):
            assert abs(val - d) <= 1e-3 * max(d, 1e-6), (tag, val, d)
        else:
            assert not (val <= ub) or abs(val - d) <= 1e-3 * d, (tag, val, d)
    elif s == "abandon":
        assert d > eff_ub * (1 - 1e-3), (tag, s, d)
    else:
        assert s == "ovf", s   # a valid outcome: the caller re-runs it wider


@pytest.mark.parametrize("ce", [8, 4])
@pytest.mark.parametrize("seed", range(6))
def test_schedule_outcomes_agree_with_dtw(seed, ce):
    rng = np.random.default_rng(seed)
    R = synth.random_walk(50_000, 60 + seed)
    counts = {}
    for trial in range(6):
        m = int(rng.choice([5, 17, 64, 129, 200, 300, 420]))
        J = int(rng.choice([1, 2, 3, 4]))
        zq = O.znorm(synth.random_walk(m, 700 + 10 * seed + trial)).astype(np.float32)
        i = int(rng.integers(0, len(R) - m))
        zr = O.znorm(R[i:i + m]).astype(np.float32)
        d = O.dtw(zr.astype(np.float64), zq.astype(np.float64), m)
        for f in (np.inf, 2.0, 1.02, 0.98, 0.6):
            ub = d * f if np.isfinite(f) else np.inf
            sched = None
            if f == 2.0 and trial % 2:   # the bound drops to 1.02 DTW mid-candidate
                sched = lambda t, d=d: d * 1.02 if t >= 12 else np.inf
            (s, _), val = emu(zr, zq, ub, J, sched, ce)
            counts[s] = counts.get(s, 0) + 1
            eff_ub = min(ub, d * 1.02) if sched else ub
            _check(s, val, d, ub, eff_ub, (m, J, f))
    assert counts.get("done", 0) > 0 and counts.get("abandon", 0) > 0, counts


@pytest.mark.parametrize("seed", range(3))
def test_unequal_shapes_of_the_live_region(seed):
    """Windows from an ECG-like series against a random-walk query and the
    reverse: live regions that widen, drift and narrow, with the windows
    switched on and off and slid; plus a candidate equal to the query (its
    diagonal costs 0)."""
    rng = np.random.default_rng(100 + seed)
    E = synth.ecg_like(40_000, 10 + seed)
    for m in (150, 333):
        zq = O.znorm(synth.random_walk(m, 900 + seed)).astype(np.float32)
        for _ in range(3):
            i = int(rng.integers(0, len(E) - m))
            zr = O.znorm(E[i:i + m]).astype(np.float32)
            d = O.dtw(zr.astype(np.float64), zq.astype(np.float64), m)
            for f in (1.5, 1.0001, 0.9):
                (s, _), val = emu(zr, zq, d * f)
                _check(s, val, d, d * f, d * f, (m, f))
        (s, _), val = emu(zq, zq, 0.25)
        assert s == "done" and val == 0.0, (m, s, val)


@pytest.mark.parametrize("m", [33, 130, 257, 400])
def test_lone_diagonal_path_survives_block_crossings(m):
    """S = T = 0, 1, 2, ...: the diagonal costs 0 and every other cell at least
    1, so at ub = 0.5 the live region is one cell wide and leaves each block
    diagonally into the next, across window boundaries and slides; the result
    must be 0."""
    x = np.arange(m, dtype=np.float32)
    for J in (1, 2, 3):
        (s, _), val = emu(x, x, 0.5, J)
        assert s == "done" and val == 0.0, (m, J, s, val)


def test_everything_alive_overflows_or_finishes():
    """ub = +inf keeps every cell alive: a query wider than the windows can hold
    must overflow (never abandon), a narrow one must finish with the DTW."""
    rng = np.random.default_rng(5)
    for m, J in ((100, 1), (300, 3), (700, 3), (700, 2)):
        a = rng.standard_normal(m).astype(np.float32)
        b = rng.standard_normal(m).astype(np.float32)
        d = O.dtw(a.astype(np.float64), b.astype(np.float64), m)
        (s, _), val = emu(a, b, np.inf, J)
        if 32 * J * K - (CE + 1) * K >= m + 2 * 32:
            assert s == "done" and abs(val - d) <= 1e-3 * d, (m, J, s)
        else:
            assert s in ("done", "ovf"), (m, J, s)
            if s == "done":
                assert abs(val - d) <= 1e-3 * d


def test_benchmark_shape_near_the_nearest_neighbour():
    """The benchmark's unconstrained search shape: m = 1024 random-walk windows
    (reference seed 0) against query seed 2, under a bound 1.3 times that
    query's nearest-neighbour distance (6.1956, window 2798147): windows around
    the nearest neighbour finish, random ones are abandoned after their live
    regions have widened, slid and narrowed."""
    R = synth.random_walk(2_800_200, 0)
    zq = O.znorm(synth.random_walk(1024, 2)).astype(np.float32)
    ub = 1.3 * 6.1956
    rng = np.random.default_rng(11)
    starts = list(range(2798140, 2798156)) + [int(x) for x in rng.integers(0, len(R) - 1024, size=16)]
    outcomes = {}
    for i in starts:
        zr = O.znorm(R[i:i + 1024]).astype(np.float32)
        d = O.dtw(zr.astype(np.float64), zq.astype(np.float64), 1024)
        (s, _), val = emu(zr, zq, ub)
        outcomes[s] = outcomes.get(s, 0) + 1
        _check(s, val, d, ub, ub, i)
    assert outcomes.get("done", 0) >= 4 and outcomes.get("abandon", 0) >= 8, outcomes


@pytest.mark.parametrize("seed", range(4))
def test_banded_handover_keeps_alive_cells_in_the_band(seed):
    """The banded elastic wavefront: unconstrained cells, and a hand-over to the
    banded levels when an alive cell could leave |r - c| <= w before the next
    check.  Every alive cell the model computes lies in the band (asserted
    cell by cell), a finished value equals the banded DTW, an abandoned
    candidate's banded DTW exceeds ub, and both outcomes and hand-overs occur."""
    rng = np.random.default_rng(40 + seed)
    R = synth.random_walk(60_000, 80 + seed)
    E = synth.ecg_like(60_000, 20 + seed)
    counts = {}
    for trial in range(8):
        m = int(rng.choice([150, 300, 512]))
        w = int(rng.choice([40, 64, m // 4, m // 2, int(0.9 * m)]))
        src = E if trial % 2 else R
        q = synth.random_walk(m, 500 + 10 * seed + trial)
        zq = O.znorm(q).astype(np.float32)
        if trial % 4 < 2:   # a near copy of the query: a small DTW, a narrow live region
            zr = O.znorm(q + rng.normal(0.0, 0.5, m)).astype(np.float32)
        else:
            i = int(rng.integers(0, len(src) - m))
            zr = O.znorm(src[i:i + m]).astype(np.float32)
        d = O.dtw(zr.astype(np.float64), zq.astype(np.float64), w)
        for f in (np.inf, 1.5, 1.0005, 0.8):
            ub = d * f if np.isfinite(f) else np.inf
            (s, _), val = emu(zr, zq, ub, 3, None, CE, w)
            counts[s] = counts.get(s, 0) + 1
            _check(s, val, d, ub, ub, (m, w, f))
    assert counts.get("done", 0) > 0 and counts.get("abandon", 0) > 0 and counts.get("ovf", 0) > 0, counts


@pytest.mark.parametrize("lead", [1, -1])
def test_banded_handover_with_paths_along_a_band_edge(lead):
    """Candidates that lead or lag the query by about the band's width: the
    warping path runs along one edge of the band (r - c near +w or -w), so the
    hand-over is decided by that edge's rule; every alive cell stays in the
    band and the outcomes agree with the banded DTW."""
    rng = np.random.default_rng(7 if lead > 0 else 8)
    counts = {}
    for m, w in ((300, 80), (400, 160), (512, 200)):
        x = synth.random_walk(m + 400, 900 + m)
        for shift in (20, w // 2, w - 20, w - 4):
            q = x[200:200 + m]
            r = x[200 - lead * shift:200 - lead * shift + m] + rng.normal(0.0, 0.2, m)
            zq, zr = O.znorm(q).astype(np.float32), O.znorm(r).astype(np.float32)
            d = O.dtw(zr.astype(np.float64), zq.astype(np.float64), w)
            for f in (1.2, 1.0005):
                (s, _), val = emu(zr, zq, d * f, 3, None, CE, w)
                counts[s] = counts.get(s, 0) + 1
                _check(s, val, d, d * f, d * f, (m, w, shift, f))
    # paths near an edge are handed over (the rule keeps a margin of about
    # 2 kElCE rows and a block's extent); a path 20 cells inside finishes
    assert counts.get("done", 0) > 0 and counts.get("ovf", 0) > 0, counts
