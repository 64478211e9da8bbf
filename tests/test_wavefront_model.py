"""A lane-by-lane model of the one-window warp wavefront's schedule, checked
against the oracle's DTW.

The model restates, in numpy, the control logic of the EAPrunedDTW wavefront
with one window of 32 blocks: K columns per lane, row r of block b at step
r + b, left inputs shifted one lane per step, checks every 16 steps in the
unconstrained case and every 8 otherwise (two consecutive dead steps abandon;
the last lane passing an alive value out of the window is an overflow), lazy
retirement of dead leading blocks, lanes that have not started computing +inf
cells on the fast path, and the band's two forced cells per row.  It asserts
every row index it reads and that unstarted lanes hold +inf only, and its
outcomes must agree with Eq. 1-5 (the oracle's DTW): a finished value equals
DTW when DTW <= ub, an abandoned candidate has DTW > ub.  Cells are rounded
to FP32 after an exact product and sum (the kernel's fma)."""
import numpy as np
import pytest

import oracle as O
from paper_2010_05371_gb300 import synth

INF = np.float32(np.inf); FMAX = np.float32(3.402823466e38); NAN = np.float32(np.nan)
FULL = 0xffffffff


def emu(rows, cols, nr, nc, w, K, BAND, ub, ub_sched=None):
    f32 = np.float32
    CE = 16 if BAND == 0 else 8
    near = (FULL << (31 - CE)) & FULL
    lanes = np.arange(32)
    st = dict(B0=0)
    prv = np.full((32, K), INF, f32)
    zc = np.zeros((32, K), f32)

    def load_cols():
        cb = (st['B0'] + lanes) * K
        for l in range(32):
            for k in range(K):
                c = cb[l] + k
                zc[l, k] = cols[c] if c < nc else NAN
    load_cols()
    lout = np.full(32, INF, f32); lprev = np.full(32, INF, f32); lprev[0] = 0
    omin = np.full(32, INF, f32)
    dead_a = FULL
    ub = f32(min(ub, FMAX)); ub_next = ub
    bm = (nc - 1) // K; km = (nc - 1) - bm * K; t_end = nr + bm

    def cells(l, z, lin, f1):
        diag = lprev[l]; left = lin
        kf = kf2 = -1
        if BAND != 0:
            f2 = f1 + 2 * w + 2
            kf = f1 if 0 <= f1 < K else f2; kf2 = f2
        for k in range(K):
            top = prv[l, k]
            d = f32(z - zc[l, k])
            m = np.fmin(np.fmin(top, diag), left)
            v = f32(np.float64(d) * np.float64(d) + np.float64(m)) if not np.isnan(m) else NAN
            if BAND == 1 and k == kf: v = INF
            if BAND == 2 and (k == kf or k == kf2): v = INF
            diag = top; left = v; prv[l, k] = v
        lout[l] = prv[l, K - 1]; lprev[l] = lin
        omin[l] = np.fmin(omin[l], lout[l])

    def ballot(pred):
        b = 0
        for l in range(32):
            if pred[l]: b |= 1 << l
        return b

    def check(bmin_b, t):
        nonlocal ub, ub_next, dead_a, prv, lout, lprev, omin
        ub = f32(min(ub, ub_next))
        db = ballot([not (bmin_b[l] <= ub) for l in range(32)])
        if omin[31] <= ub and st['B0'] + 31 < bm:
            return ('ovf', t)
        cond = db & (((dead_a << 1) | 1) & FULL)
        if (dead_a == FULL and db == FULL) or cond == FULL:
            return ('abandon', t)
        d = 0
        while d < 32 and (cond >> d) & 1: d += 1
        if d > 0 and ((~(dead_a & db)) & near) == 0:
            d = 0   # lazy retirement
        if ub_sched is not None:
            ub_next = f32(min(ub_next, ub_sched(t)))
        omin[:] = INF
        if d > 0:
            st['B0'] += d
            src = lanes + d; fresh = src >= 32; src = np.minimum(src, 31)
            prv = np.where(fresh[:, None], INF, prv[src]).astype(f32)
            lprev = np.where(fresh, INF, lprev[src]).astype(f32)
            lout = np.where(fresh, INF, lout[src]).astype(f32)
            load_cols()
        return None

    def shfl_up(x):
        y = np.empty_like(x); y[1:] = x[:-1]; y[0] = INF
        return y

    t = 0
    while True:
        B0 = st['B0']
        if t % CE == 0 and t + CE - B0 <= nr and t + CE < t_end:
            bmin_a = bmin_b = None
            for s in range(1, CE + 1):
                lin = shfl_up(lout)
                for l in range(32):
                    bj = B0 + l
                    r = t + s - bj
                    rr = max(r, 1)
                    assert 1 <= rr <= nr, ('fast row', r)
                    if r < 1:
                        assert np.all(~(prv[l] <= FMAX)) and not (lin[l] <= FMAX) and not (lprev[l] <= FMAX), ('unstarted lane not inf', l, t, s)
                    cells(l, rows[rr - 1], lin[l], r - w - 1 - (bj * K + 1))
                if s == CE - 1: bmin_a = np.fmin.reduce(prv, axis=1)
                if s == CE: bmin_b = np.fmin.reduce(prv, axis=1)
            t += CE
            dead_a = ballot([not (bmin_a[l] <= ub) for l in range(32)])
            res = check(bmin_b, t)
            if res: return res, None
            continue
        t += 1
        phase = t % CE
        lin = shfl_up(lout)
        bmin = np.full(32, INF, f32)
        for l in range(32):
            bj = B0 + l; r = t - bj
            if 1 <= r <= nr:
                cells(l, rows[r - 1], lin[l], r - w - 1 - (bj * K + 1))
                if phase == 0 or phase == CE - 1: bmin[l] = np.fmin.reduce(prv[l])
            else:
                if r < 1: lout[l] = INF
                lprev[l] = lin[l]
        if t == t_end:
            src = bm - B0
            if 0 <= src < 32: return ('done', t), prv[src, km]
            if src >= 32: return ('ovf_end', t), None
            return ('done_retired', t), INF
        if phase == CE - 1:
            dead_a = ballot([not (bmin[l] <= ub) for l in range(32)])
        elif phase == 0:
            res = check(bmin, t)
            if res: return res, None




def _band(m, w, K):
    return 0 if w >= m - 1 else (1 if K <= 2 * w + 2 else 2)


@pytest.mark.parametrize("seed", range(6))
def test_schedule_outcomes_agree_with_dtw(seed):
    rng = np.random.default_rng(seed)
    R = synth.random_walk(50_000, 40 + seed)
    counts = {}
    for trial in range(6):
        m = int(rng.choice([5, 16, 17, 40, 64, 150, 300]))
        w = min(m, int(rng.choice([m, m - 1, max(1, m // 10), 15, 3])))
        K = int(rng.choice([4, 8]) if m >= 150 else rng.choice([4, 8, 16, 32]))
        BAND = _band(m, w, K)
        zq = O.znorm(synth.random_walk(m, 500 + 10 * seed + trial)).astype(np.float32)
        i = int(rng.integers(0, len(R) - m))
        zr = O.znorm(R[i:i + m]).astype(np.float32)
        d = O.dtw(zr.astype(np.float64), zq.astype(np.float64), w)
        for f in (np.inf, 2.0, 1.02, 0.98, 0.6):
            ub = d * f if np.isfinite(f) else np.inf
            sched = None
            if f == 2.0 and trial % 2:   # the bound drops to 1.02 DTW mid-candidate
                sched = lambda t, d=d: d * 1.02 if t >= 24 else np.inf
            (s, _), val = emu(zr, zq, m, m, w, K, BAND, ub, sched)
            counts[s] = counts.get(s, 0) + 1
            eff_ub = min(ub, d * 1.02) if sched else ub
            if s == "done":
                if d <= ub * (1 - 1e-3):
                    assert abs(val - d) <= 1e-3 * max(d, 1e-6), (m, w, K, f, val, d)
                else:
                    assert not (val <= ub) or abs(val - d) <= 1e-3 * d, (m, w, K, f, val, d)
            elif s in ("abandon", "done_retired"):
                assert d > eff_ub * (1 - 1e-3), (m, w, K, f, s, d)
            else:
                assert s == "ovf", s   # a valid outcome: the caller re-runs it wider
    assert counts.get("done", 0) > 0 and counts.get("abandon", 0) > 0, counts


@pytest.mark.parametrize("m", [33, 50, 70, 100])
def test_lone_diagonal_path_survives_block_crossings(m):
    """S = T = 0, 1, 2, ...: the diagonal costs 0 and every other cell at least
    1, so at ub = 0.5 the live region is one cell wide and leaves each block
    diagonally into the next.  A step at which every block is dead can still
    hand an alive diagonal input to the next block, which is why abandoning
    needs two consecutive dead steps; the result must be 0."""
    x = np.arange(m, dtype=np.float32)
    for K in (4, 8, 16, 32):
        for w in (m, 10, 3):
            (s, _), val = emu(x, x, m, m, w, K, _band(m, w, K), 0.5)
            assert s == "done" and val == 0.0, (m, K, w, s, val)
