"""A lane-by-lane model of the group wavefront's protocol (csrc/dtw_group.cuh),
checked against the oracle's DTW.

The model restates, in numpy, what each warp of a group does: 32 lanes of
blocks of 16 columns per warp (warp g owns columns 512 g + 1 .. 512 g + 512),
one row per step pipelined across the lanes, the edge column passed through
each warp's ring of 64 slots, published every 8 steps (prog, cons), the skip of
steps whose blocks and inputs are all dead, the dead-for-good marks (dead), the
band's two forced cells per row, the row reads clamped into 1..nr and the
final capture of cell (nr, nc).  Warps run in a random order, one round of 8
steps at a time, each only when its waits are satisfied, so every
interleaving the waits allow can occur; the rings start filled with garbage,
so that a read of an entry nobody wrote changes the result.  The model asserts
that some warp can always go on (no deadlock) and that no ring entry is
overwritten before its reader has read it, and its outcomes must agree with
Eq. 1-5 (the oracle's DTW): a finished value equals DTW when DTW <= ub, and an
abandoned candidate has DTW > ub."""
import numpy as np
import pytest

import oracle as O
from paper_2010_05371_gb300 import synth

f32 = np.float32
INF = f32(np.inf)
FMAX = f32(3.402823466e38)
K, LANES, CE, RING = 16, 32, 8, 64
BIG = 2 ** 31 - 1


def _cell(q, z, mn):
    d = (q + (-z)).astype(f32)
    with np.errstate(invalid="ignore"):
        return (d.astype(np.float64) * d.astype(np.float64) + mn.astype(np.float64)).astype(f32)


class Warp:
    def __init__(self, g, ge, rows, cols, nr, nc, w, band, ub):
        self.g, self.last = g, g == ge - 1
        self.rows, self.nr, self.nc, self.w, self.band = rows, nr, nc, w, band
        self.b = 32 * g + np.arange(LANES)
        self.bm = (nc - 1) // K
        self.km = (nc - 1) - self.bm * K
        self.t_fin = nr + self.bm if self.last else nr + 32 * g + 31
        c = self.b[:, None] * K + np.arange(K)[None, :]
        self.zc = np.where(c < nc, cols[np.minimum(c, nc - 1)], np.nan).astype(f32)
        self.prv = np.full((LANES, K), INF, f32)
        self.lout = np.full(LANES, INF, f32)
        self.lprev = np.full(LANES, INF, f32)
        if g == 0:
            self.lprev[0] = 0.0
        self.ub = f32(min(ub, FMAX))
        self.own_dead = g > 0
        self.t, self.done, self.dist, self.busy = 0, False, INF, 0

    def step(self, s, lin0):
        r = s - self.b
        rr = np.clip(r, 1, self.nr)
        z = self.rows[rr - 1]
        lin = np.empty(LANES, f32)
        lin[0] = lin0
        lin[1:] = self.lout[:-1]
        diag, left = self.lprev.copy(), lin.copy()
        f1 = r - self.w - 1 - (self.b * K + 1)
        f2 = f1 + 2 * self.w + 2
        kf = np.where((f1 >= 0) & (f1 < K), f1, f2)
        for k in range(K):
            top = self.prv[:, k].copy()
            v = _cell(self.zc[:, k], z, np.fmin(np.fmin(top, diag), left))
            if self.band == 1:
                v = np.where(kf == k, INF, v)
            elif self.band == 2:
                v = np.where((kf == k) | (f2 == k), INF, v)
            diag, left = top, v
            self.prv[:, k] = v
        self.lout = self.prv[:, K - 1].copy()
        self.lprev = lin
        return int(np.sum((r >= 1) & (r <= self.nr)))

    def bmin(self):
        return np.fmin.reduce(self.prv, axis=1)


def run_group(rows, cols, w, ub, rng):
    nr, nc = len(rows), len(cols)
    band = 0 if w >= max(nr, nc) - 1 else (1 if 32 <= 2 * w + 2 else 2)
    ge = (nc - 1) // 512 + 1
    W = [Warp(g, ge, rows, cols, nr, nc, w, band, ub) for g in range(ge)]
    ring = rng.uniform(-1, 50, size=(ge, RING)).astype(f32)   # garbage
    written = np.full((ge, RING), -1, np.int64)               # step held by each slot
    prog, cons, dead = [0] * ge, [0] * ge, [BIG] * ge

    def ready(x):
        g, t_next = x.g, min(x.t + CE, x.t_fin)
        if g > 0 and not (prog[g - 1] >= t_next - 1 or dead[g - 1] <= t_next - 1):
            return False
        if not x.last and not (cons[g + 1] >= t_next - RING + 1):
            return False
        return True

    def round_(x):
        g, t = x.g, x.t
        t_next = min(t + CE, x.t_fin)
        ns = t_next - t
        dd = dead[g - 1] if g > 0 else 0

        def inp(s):
            if not (s >= 2 and s - 1 < dd):
                return INF
            slot = (s - 1) % RING
            assert written[g - 1][slot] == s - 1, ("ring entry read before it was written or after reuse",
                                                   g, s - 1, written[g - 1][slot])
            return ring[g - 1][slot]

        def put(s, v):
            slot = s % RING
            old = written[g][slot]
            if old >= 0 and not x.last:
                # its reader (warp g+1) must have read step old: it reads entry
                # old at its step old + 1, completed by cons[g + 1]
                assert cons[g + 1] >= old + 1, ("ring entry overwritten before it was read", g, old, cons[g + 1])
            ring[g][slot] = v
            written[g][slot] = s

        skip = False
        if x.own_dead:
            ind = not (x.lprev[0] <= x.ub)
            for i in range(1, CE + 1):
                ind = ind and (i > ns or not (inp(t + i) <= x.ub))
            skip = ind
        ba = bb = np.full(LANES, INF, f32)
        if skip:
            x.prv[:] = INF
            x.lout[:] = INF
            x.lprev[:] = INF
            for i in range(ns):
                put(t + 1 + i, INF)
        else:
            fin = INF
            for s in range(t + 1, t_next + 1):
                x.busy += x.step(s, inp(s))
                put(s, x.lout[31])
                if s == t_next - 1:
                    ba = x.bmin()
                if s == t_next:
                    bb = x.bmin()
                if x.last and s == x.t_fin:
                    fin = x.prv[x.bm - 32 * g, x.km]
            if x.last and t_next == x.t_fin:
                x.dist = fin
        x.t = t_next
        prog[g] = x.t
        cons[g] = x.t
        if x.t == x.t_fin:
            if not x.last:
                dead[g] = x.t + 1
            if x.last and not (x.dist <= INF):
                x.dist = INF
            x.done = True
            return
        da, db = ~(ba <= x.ub), ~(bb <= x.ub)
        x.own_dead = bool(np.all(da) and np.all(db))
        if x.own_dead:
            d0 = dead[g - 1] if g > 0 else 0
            if d0 <= x.t - 1:
                dead[g] = x.t - 1
                x.dist = INF
                x.done = True

    while not W[-1].done:
        cand = [x for x in W if not x.done and ready(x)]
        assert cand, ("no warp can go on", [(x.g, x.t, x.done) for x in W], prog, cons, dead)
        round_(cand[rng.integers(len(cand))])
    return W[-1].dist, sum(x.busy for x in W)


def _check(val, d, ub, tag):
    if d <= ub * (1 - 1e-3):
        assert abs(val - d) <= 1e-3 * max(d, 1e-6), (tag, val, d)
    elif d > ub * (1 + 1e-3):
        assert not (val <= ub), (tag, val, d)


@pytest.mark.parametrize("seed", range(3))
def test_group_outcomes_agree_with_dtw(seed):
    """Random-walk and ECG-like windows against random-walk queries; short
    windows against long queries (the live region crosses every warp within
    few rows) and square ones; unconstrained and banded (the band edges cross
    the warps); bounds from +inf (nothing pruned) to below the DTW."""
    rng = np.random.default_rng(seed)
    R = synth.random_walk(20_000, 300 + seed)
    E = synth.ecg_like(20_000, 40 + seed)
    outcomes = {}
    for trial, (nr, nc) in enumerate([(60, 1030), (150, 1600), (600, 600), (520, 1030)]):
        src = E if (trial + seed) % 2 else R
        zq = O.znorm(synth.random_walk(nc, 900 + 10 * seed + trial)).astype(np.float32)
        i = int(rng.integers(0, len(src) - nr))
        zr = O.znorm(src[i:i + nr]).astype(np.float32)
        for w in (max(nr, nc), nc - nr + 20):
            d = O.dtw(zr.astype(np.float64), zq.astype(np.float64), w)
            for f in (np.inf, 1.0005, 0.7):
                ub = d * f if np.isfinite(f) else np.inf
                val, _ = run_group(zr, zq, w, ub, rng)
                key = "done" if val <= ub else "inf"
                outcomes[key] = outcomes.get(key, 0) + 1
                _check(val, d, ub, (nr, nc, w, f))
    assert outcomes.get("done", 0) > 0 and outcomes.get("inf", 0) > 0, outcomes


def test_equal_series_finish_at_zero():
    """S = T: the diagonal costs 0; at a bound of 0.5 the live region is a thin
    diagonal that leaves each warp into the next, and the result must be 0."""
    rng = np.random.default_rng(1)
    x = O.znorm(synth.random_walk(1100, 5)).astype(np.float32)
    val, _ = run_group(x, x, 1100, 0.5, rng)
    assert val == 0.0, val


def test_eight_warp_group():
    """The largest group (4096 columns, eight warps, the batch's level 5 and
    the one-query search's queries of up to 4096 points): short windows
    against a 4096-point query, unconstrained and banded, bounds from +inf to
    below the DTW; every interleaving the waits allow, in random order."""
    rng = np.random.default_rng(17)
    R = synth.random_walk(10_000, 71)
    zq = O.znorm(synth.random_walk(4096, 72)).astype(np.float32)
    outcomes = {}
    for nr in (40, 90):
        i = int(rng.integers(0, len(R) - nr))
        zr = O.znorm(R[i:i + nr]).astype(np.float32)
        for w in (4096, 4096 - nr + 30):
            d = O.dtw(zr.astype(np.float64), zq.astype(np.float64), w)
            for f in (np.inf, 1.0005, 0.7):
                ub = d * f if np.isfinite(f) else np.inf
                val, _ = run_group(zr, zq, w, ub, rng)
                key = "done" if val <= ub else "inf"
                outcomes[key] = outcomes.get(key, 0) + 1
                _check(val, d, ub, (nr, w, f))
    assert outcomes.get("done", 0) > 0 and outcomes.get("inf", 0) > 0, outcomes
