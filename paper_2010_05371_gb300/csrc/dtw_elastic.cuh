// EAPrunedDTW as a narrow-block elastic warp wavefront (sm_103a), for the
// unconstrained search.
//
// What is computed: the DTW recurrence of Eq. 1-5 without a window, with early
// abandoning against an upper bound ub (Section 2.2): DTW if DTW <= ub, else
// +inf, exactly the contract of Algorithm 3 (EAPrunedDTW).
//
// Why a second wavefront.  The live region of Algorithm 3, the columns between
// next_start (Section 3) and pruning_point (Section 4), is on the benchmark's
// unconstrained searches about 100-190 columns wide for the windows that live
// past the first rows, and changes over a candidate's life.  The one-window
// wavefront (dtw_wavefront.cuh) must cover the widest moment with 32 blocks of
// K columns, so with K = 16 about three quarters of its lane-steps compute
// dead cells right of the live region.  Here each lane owns blocks of only
// K = 4 columns, and the warp holds up to J windows of 32 blocks, switched on
// and off as the live region widens and narrows:
//  * Layout.  Lane l of window j owns block b = B0 + 32 j + l (columns
//    4b+1 .. 4b+4).  Each step a block computes two rows: block b at step t
//    holds rows 2(t-1-b)+1 and 2(t-1-b)+2, so the left neighbour's last column
//    of the same two rows was produced one step earlier by lane l-1 (or by lane
//    31 of window j-1) and arrives by two shuffles.  The two rows are computed
//    along anti-diagonals, (r, k) beside (r+1, k-1): two independent chains.
//  * Rows.  The candidate's z-normalised rows sit in the warp's shared-memory
//    buffer with NaN rows before and after.  A block that has not started, or
//    has passed the last row, reads NaN rows and computes NaN cells, which fmin
//    ignores and which are never alive: no per-lane range tests.
//  * Left border (next_start).  A leading block dead at this check whose left
//    neighbour was dead at the previous step can never revive (its top, left and
//    diagonal inputs are dead), so it is retired.  Retired blocks are dropped by
//    sliding the windows right, lazily: only when the slide lets a window switch
//    off or saves switching one on.
//  * Right border (pruning_point).  Cells right of the live region are computed
//    as dead values.  The live region grows by at most one block per step, so a
//    window is switched on at a check when an alive block of the last active
//    window lies within kElCE + 1 blocks of its end; when that happens with J
//    windows active the candidate overflows and is re-run wider.
//  * Early abandoning.  Every active block dead at two consecutive steps means
//    every later cell has dead inputs only: the result is +inf (the border
//    collision and full discard line of Algorithm 3).
// Arithmetic: each cell is fma(d, d, min(top, diag, left)) with d = q - z in
// FP32, the same operations as the other wavefront: every alive cell equals the
// sequential FP32 DP value.
#pragma once

#include "dtw_wavefront.cuh"

namespace eapdtw {

constexpr int kElK = 4;    // columns per block
constexpr int kElR = 2;    // rows per step
constexpr int kElCE = 4;   // steps between checks
#ifndef EAPDTW_ELASTIC_WINDOWS
#define EAPDTW_ELASTIC_WINDOWS 3
#endif
constexpr int kElJ = EAPDTW_ELASTIC_WINDOWS;
static_assert(kElJ >= 1 && kElJ <= 4, "1 to 4 windows");
// NaN rows before the first row and after the last one: a block reads rows
// 2(t-1-b)+1, +2 with -(32 J - 1) <= t-1-b (blocks of the active windows, B0 <
// t) and t-1-b <= 32 J - 1 + (nr - 1) / 2 (up to the final step).
constexpr int kElPadRows = kElR * 32 * kElJ;
// NaN columns after the last one: blocks up to B0 + 32 J - 1 with B0 <= the
// last column's block.
constexpr int kElPadCols = 32 * kElJ * kElK;

// Floats of the per-warp row buffer (rows start at offset kElPadRows) and of
// the query buffer (NaN past the last column) for queries of m points.
__host__ __device__ inline int elastic_row_floats(int m) { return (2 * kElPadRows + m + kElR + 3) / 4 * 4; }
__host__ __device__ inline int elastic_col_floats(int m) { return (m + kElPadCols + 3) / 4 * 4; }
// Cells one busy lane-step computes.
constexpr int kElCellsPerStep = kElK * kElR;

// zr: row r (1-based) at zr[r - 1], NaN at zr[-kElPadRows .. -1] and
// zr[nr .. nr + kElPadRows + 2); zq: column c at zq[c - 1], NaN from zq[nc]
// through zq[nc + kElPadCols - 1], 16-byte aligned.  All 32 lanes call it
// with identical arguments.  Returns busy = lane-steps whose rows started.
template <int J, int COST>
__device__ __forceinline__ DtwOut dtw_elastic(const float* __restrict__ zr, const float* __restrict__ zq, int nr,
                                              int nc, const BestSoFar bsf, float ub) {
    constexpr int K = kElK;
    constexpr int CE = kElCE;
    const int lane = threadIdx.x & 31;
    const float INF = f_inf();
    float p[J][K];          // the block's values at its second row of the last step
    float q[J][K];          // its columns
    float lo0[J], lo1[J];   // its last column at the two rows of the last step
    float dg[J];            // diagonal input of its first cell: D(r - 1, 4b)
    int B0 = 0, jact = 1;

    auto reset = [&](int j) {
#pragma unroll
        for (int k = 0; k < K; ++k) p[j][k] = INF;
        lo0[j] = INF;
        lo1[j] = INF;
        dg[j] = INF;
    };
    auto load_q = [&](int j) {
        const float4 v = *reinterpret_cast<const float4*>(zq + (B0 + 32 * j + lane) * K);
        q[j][0] = v.x; q[j][1] = v.y; q[j][2] = v.z; q[j][3] = v.w;
    };
#pragma unroll
    for (int j = 0; j < J; ++j) reset(j);
    load_q(0);
    if (lane == 0) dg[0] = 0.0f;   // D(0, 0) = 0: diagonal of cell (1, 1)

    ub = fminf(ub, 3.402823466e38f);   // +inf cells (borders, retired blocks) are dead
    BestSoFar::Raw ub_raw = BestSoFar::of(ub);
    const int bm = (nc - 1) / K;              // block of the last column
    const int km = (nc - 1) - bm * K;
    const int t_end = bm + 1 + (nr - 1) / 2;  // step holding row nr of block bm
    const bool last_first = (nr & 1) != 0;    // row nr is the first of its step's two rows
    DtwOut out{INF, 0, 0, 0};
    int busy = 0;
    // Rows of window j at step s: zr + zoff[j] + 2 s, i.e. rows 2(s-1-b)+1, +2
    // of block b.  At every check the offset is capped so that no block reads
    // past the first NaN row after the last one for the next CE steps: a block
    // that has passed the last row reads NaN rows (at most 2 CE + 2 floats
    // beyond it).  Unstarted blocks read the NaN rows before the first.
    const int nre = (nr + 1) & ~1;
    int zoff[J];
    auto set_zoff = [&](int tnow) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int o = -2 * (1 + B0 + 32 * j + lane);
            const int cap = nre - 2 * (tnow + 1);
            zoff[j] = o < cap ? o : cap;
        }
    };
    set_zoff(0);

    auto cost = [&](float qv, float z, float mn) -> float {
        const float d = __fsub_rn(qv, z);
        return COST == kCostAbsolute ? __fadd_rn(fabsf(d), mn) : __fmaf_rn(d, d, mn);
    };
    // One step of every active window.  which = 1 or 2: bma[j] or bmb[j]
    // receives the min of the block's outputs (its second row and the first
    // row's last column); cap >= 0 asks for row nr's column km of this lane's
    // block of window cap >> 5, into fin.
    float bma[J], bmb[J];
    float fin = INF;
    auto step = [&](int s, int which, int cap) {
        float l0[J], l1[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (j < jact) {
                const float s0 = (lane == 31) ? (j > 0 ? lo0[j > 0 ? j - 1 : 0] : INF) : lo0[j];
                const float s1 = (lane == 31) ? (j > 0 ? lo1[j > 0 ? j - 1 : 0] : INF) : lo1[j];
                l0[j] = __shfl_sync(kFull, s0, (lane + 31) & 31);
                l1[j] = __shfl_sync(kFull, s1, (lane + 31) & 31);
            }
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (j < jact) {
                const float2 zz = *reinterpret_cast<const float2*>(zr + zoff[j] + 2 * s);
                const float z0 = zz.x, z1 = zz.y;
                const float a0 = cost(q[j][0], z0, fmin3(p[j][0], dg[j], l0[j]));
                const float a1 = cost(q[j][1], z0, fmin3(p[j][1], p[j][0], a0));
                const float b0 = cost(q[j][0], z1, fmin3(a0, l0[j], l1[j]));
                const float a2 = cost(q[j][2], z0, fmin3(p[j][2], p[j][1], a1));
                const float b1 = cost(q[j][1], z1, fmin3(a1, a0, b0));
                const float a3 = cost(q[j][3], z0, fmin3(p[j][3], p[j][2], a2));
                const float b2 = cost(q[j][2], z1, fmin3(a2, a1, b1));
                const float b3 = cost(q[j][3], z1, fmin3(a3, a2, b2));
                if (cap >= 0 && j == (cap >> 5)) {
                    const float ra = km == 0 ? a0 : (km == 1 ? a1 : (km == 2 ? a2 : a3));
                    const float rb = km == 0 ? b0 : (km == 1 ? b1 : (km == 2 ? b2 : b3));
                    fin = last_first ? ra : rb;
                }
                p[j][0] = b0; p[j][1] = b1; p[j][2] = b2; p[j][3] = b3;
                lo0[j] = a3;
                lo1[j] = b3;
                dg[j] = l1[j];
                if (which == 1) bma[j] = fmin3(fmin3(b0, b1, b2), b3, a3);
                if (which == 2) bmb[j] = fmin3(fmin3(b0, b1, b2), b3, a3);
            }
        }
    };
    // lane-steps with started rows among steps (t0, t1] of this lane's blocks
    auto count_busy = [&](int t0, int t1) {
        const int half = (nr + 1) >> 1;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (j < jact) {
                const int b = B0 + 32 * j + lane;
                const int lo = t0 > b ? t0 : b;
                const int hi = t1 < b + half ? t1 : b + half;
                busy += hi > lo ? hi - lo : 0;
            }
        }
    };

    int t = 0;   // steps completed
    for (;;) {
        if (t + CE < t_end) {
#pragma unroll
            for (int s = 1; s <= CE; ++s) step(t + s, s == CE - 1 ? 1 : (s == CE ? 2 : 0), -1);
            count_busy(t, t + CE);
            t += CE;
            // ---- check ----
            ub = fminf(ub, __shfl_sync(kFull, BestSoFar::finish(ub_raw), 0));   // one reading for the warp
            ub_raw = bsf.issue();
            unsigned da[J], db[J];
            bool all_dead = true;
            int hi = -1;   // highest block (relative to B0) alive at step t - 1 or t
#pragma unroll
            for (int j = 0; j < J; ++j) {
                da[j] = kFull;
                db[j] = kFull;
                if (j < jact) {
                    da[j] = __ballot_sync(kFull, !(bma[j] <= ub));
                    db[j] = __ballot_sync(kFull, !(bmb[j] <= ub));
                    const unsigned al = ~(da[j] & db[j]);
                    all_dead = all_dead && al == 0u;
                    if (al) hi = 32 * j + 31 - __clz(al);
                }
            }
            const unsigned cond = db[0] & ((da[0] << 1) | 1u);   // retirable leading blocks of window 0
            if (all_dead || (jact == 1 && cond == kFull)) {
                out.steps = t;
                break;
            }
            const int d = (cond == kFull) ? 32 : (__ffs(~cond) - 1);
            // windows needed with and without the slide (an alive block needs
            // CE + 1 blocks after it), capped by the window holding the last column
            auto need = [&](int shift) {
                int nd = (hi - shift + CE + 1) / 32 + 1;
                const int cap_w = (bm - (B0 + shift)) / 32 + 1;
                nd = nd < cap_w ? nd : cap_w;
                return nd < 1 ? 1 : nd;
            };
            const int n0 = need(0);
            int nnew = n0;
            int shift = 0;
            if (d > 0) {
                const int nd = need(d);
                if (nd < jact || n0 > jact) {
                    shift = d;
                    nnew = nd;
                }
            }
            // the last active window's end is near an alive block and no
            // window is left: the live region is wider than J windows
            if (nnew > J) {
                out.status = 1;
                out.steps = t;
                break;
            }
            if (shift > 0) {
                // lane l of window j takes block B0 + shift + 32 j + l: from lane
                // l + shift of window j, or lane l + shift - 32 of window j + 1
                // (+inf past the active windows); each lane sends the value its
                // receiver needs.  shift = 32 drops window 0 (every lane takes
                // its own lane of the next window).
                B0 += shift;
                const int src = (lane + shift) & 31;
                const bool nxt = lane < shift;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    if (j < jact) {
                        const bool on = j + 1 < jact;
                        const int jn = j + 1 < J ? j + 1 : j;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const float nx = on ? p[jn][k] : INF;
                            p[j][k] = __shfl_sync(kFull, nxt ? nx : p[j][k], src);
                        }
                        const float n0v = on ? lo0[jn] : INF;
                        const float n1v = on ? lo1[jn] : INF;
                        const float ndv = on ? dg[jn] : INF;
                        lo0[j] = __shfl_sync(kFull, nxt ? n0v : lo0[j], src);
                        lo1[j] = __shfl_sync(kFull, nxt ? n1v : lo1[j], src);
                        dg[j] = __shfl_sync(kFull, nxt ? ndv : dg[j], src);
                        load_q(j);
                    }
                }
            }
            // switch windows on (state +inf, columns loaded) or off (state reset)
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (j >= jact && j < nnew) load_q(j);
                if (j >= nnew && j < jact) reset(j);
            }
            jact = nnew;
            set_zoff(t);
            continue;
        }
        // the last steps up to t_end (fewer than CE: no check falls before it)
        const int src = bm - B0;
        // Every lane takes every step (the steps shuffle); each captures its
        // own block of the window holding the last column, and the lane of
        // block bm passes it on.  If that block lies beyond the active windows
        // no alive value ever reached it (the switch-on rule): the result is +inf.
        for (int s = t + 1; s <= t_end; ++s) step(s, 0, (s == t_end && src >= 0) ? src : -1);
        count_busy(t, t_end);
        fin = __shfl_sync(kFull, fin, src & 31);
        if (src < 0 || src >= 32 * jact) fin = INF;
        out.dist = (fin <= INF) ? fin : INF;   // NaN (no path through started rows) is +inf
        out.steps = t_end;
        break;
    }
    int bs = busy;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bs += __shfl_xor_sync(kFull, bs, o);
    out.busy = bs;
    return out;
}

}  // namespace eapdtw
