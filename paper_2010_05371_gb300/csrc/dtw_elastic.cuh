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
//    window lies within kElCE + 1 blocks of its end (checks every kElCE
//    steps); when that happens with J
//    windows active the candidate overflows and is re-run wider.
//  * Early abandoning.  Every active block dead at two consecutive steps means
//    every later cell has dead inputs only: the result is +inf (the border
//    collision and full discard line of Algorithm 3).
// Arithmetic: each cell is fma(d, d, min(top, diag, left)) with d = q - z in
// FP32, the same operations as the other wavefront: every alive cell equals the
// sequential FP32 DP value.
#pragma once

#include <type_traits>

#include "dtw_wavefront.cuh"

namespace eapdtw {

constexpr int kElK = 4;    // columns per block
constexpr int kElR = 2;    // rows per step
// Steps between checks (a power of 2; a compile-time knob for tuning
// experiments).  Measured on the large workload's unconstrained searches: 4
// steps 75.9 ms, 8 steps 66.8 ms, 16 steps 97.8 ms per search (the switch-on
// margin of CE + 1 blocks keeps more windows on as CE grows, while the checks'
// own instructions shrink).
#ifndef EAPDTW_ELASTIC_CE
#define EAPDTW_ELASTIC_CE 8
#endif
constexpr int kElCE = EAPDTW_ELASTIC_CE;
// 1: the anti-diagonal cell pairs (r, k), (r + 1, k - 1) share packed f32x2
// adds and fused multiply-adds (identical values, fewer issue slots, two more
// registers per window; 65.2 against 66.8 ms per search); 0: scalar
// operations.  A knob for tuning experiments.
#ifndef EAPDTW_ELASTIC_PAIRED
#define EAPDTW_ELASTIC_PAIRED 1
#endif
constexpr bool kElPaired = EAPDTW_ELASTIC_PAIRED != 0;
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
// (after the NaN rows past the last row, 8 floats hold the survivor's
// z-normalisation coefficients and window pointer for the on-demand fill)
__host__ __device__ constexpr int elastic_row_floats(int m) { return (2 * kElPadRows + m + 12 + 3) / 4 * 4; }
// Offset, from row 1, of those 8 floats.
__host__ __device__ constexpr int elastic_fill_slot(int m) { return m + kElPadRows + 4; }
__host__ __device__ constexpr int elastic_col_floats(int m) { return (m + kElPadCols + 3) / 4 * 4; }
// Cells one busy lane-step computes.
constexpr int kElCellsPerStep = kElK * kElR;

// Rows written ahead of the steps that read them (a multiple of 32; a
// compile-time knob for tuning experiments).
#ifndef EAPDTW_ELASTIC_FILL
#define EAPDTW_ELASTIC_FILL 64
#endif
constexpr int kElFillRows = EAPDTW_ELASTIC_FILL;
static_assert(kElFillRows >= 32 && kElFillRows % 32 == 0, "whole warps of rows");

// zr: minus row r (1-based), -z_r, at zr[r - 1] (so that d = q + (-z) is one
// add, packed or not), NaN at zr[-kElPadRows .. -1] and
// zr[nr .. nr + kElPadRows + 2); zq: column c at zq[c - 1] (c <= nc; see QPAD).  All 32 lanes call it
// with identical arguments.  Returns busy = lane-steps executed by the
// active windows (started or not).
//
// The rows are written on demand: fill(r0, r1), called by all lanes with
// identical arguments, writes zr[r0 .. r1) and synchronises the warp.  Steps
// up to s read rows below 2 s only, and most candidates are abandoned long
// before their last row, so the rows are filled kElFillRows at a time before
// the interval that first reads them.
//
// The steps and the check between them are compiled once per number of
// active windows (1..J), so that a step computes only the active windows and
// inactive ones hold no live state: a window's state is reset when it is
// switched on.
//
// BANDED: the window |r - c| <= w (Section 2.1) without forcing any cell: the
// recurrence runs unconstrained, and at every check the candidate is handed to
// the banded levels (status 1, as an overflow) unless no alive cell of the
// next kElCE steps can lie outside the band.  Block b at step s holds cells
// with c - r <= 6 b - 2 s + 5 and r - c <= 2 s - 6 b - 1; the highest alive
// block grows by at most one per step and no block left of the retirable
// leading ones revives, so with H the highest alive block and L the first
// non-retirable one at check t, the next steps keep c - r <= 6 H - 2 t +
// 4 kElCE + 5 and r - c <= 2 (t + kElCE) - 6 L - 1.  While both stay within w,
// every alive cell's optimal path lies in the band, so its value is the banded
// DP's (the same operations on the same inputs; dead out-of-band values lose
// every min to the alive ones), and the result is the banded EAPrunedDTW's.
//
// QPAD: zq holds NaN from zq[nc] through zq[nc + kElPadCols - 1] and is
// 16-byte aligned (the one-query kernel's shared copy), so the column loads
// need no test; otherwise (the batch's query in global memory) columns past nc
// are NaN by a test.
template <int J, int COST, bool BANDED, bool QPAD, typename FillF>
__device__ __forceinline__ DtwOut dtw_elastic(const float* __restrict__ zr, const float* __restrict__ zq, int nr,
                                              int nc, const BestSoFar bsf, float ub, int w, FillF fill) {
    constexpr int K = kElK;
    constexpr int CE = kElCE;
    const int lane = threadIdx.x & 31;
    const float INF = f_inf();
    float p[J][K];          // the block's values at its second row of the last step
    float q[J][K];          // its columns
    float2 qp[kElPaired ? J : 1][kElPaired ? K - 1 : 1];   // pairs (q[k], q[k - 1]), k = 1..3
    float lo0[J], lo1[J];   // its last column at the two rows of the last step
    float dg[J];            // diagonal input of its first cell: D(r - 1, 4b)
    const float* zp[J];     // rows of window j at step s: zp[j] + 2 s
    int B0 = 0, jact = 1, t = 0;

    auto reset = [&](int j) {
#pragma unroll
        for (int k = 0; k < K; ++k) p[j][k] = INF;
        lo0[j] = INF;
        lo1[j] = INF;
        dg[j] = INF;
    };
    // columns past nc are NaN: read from the array only below nc (it may hold
    // just nc values, in shared or global memory)
    auto load_q = [&](int j) {
        const int c0 = (B0 + 32 * j + lane) * K;
        float4 v;
        if (QPAD || (c0 + K <= nc && (reinterpret_cast<uintptr_t>(zq + c0) & 15) == 0)) {
            v = *reinterpret_cast<const float4*>(zq + c0);
        } else {
            const float nan = f_nan();
            v.x = c0 < nc ? zq[c0] : nan;
            v.y = c0 + 1 < nc ? zq[c0 + 1] : nan;
            v.z = c0 + 2 < nc ? zq[c0 + 2] : nan;
            v.w = c0 + 3 < nc ? zq[c0 + 3] : nan;
        }
        q[j][0] = v.x; q[j][1] = v.y; q[j][2] = v.z; q[j][3] = v.w;
        if (kElPaired) {
            qp[kElPaired ? j : 0][0] = make_float2(v.y, v.x);
            qp[kElPaired ? j : 0][kElPaired ? 1 : 0] = make_float2(v.z, v.y);
            qp[kElPaired ? j : 0][kElPaired ? 2 : 0] = make_float2(v.w, v.z);
        }
    };
    // zp[j] + 2 s points at rows 2(s-1-b)+1, +2 of block b.  The offset is
    // capped so that for the CE steps after step tnow no block reads past the
    // first NaN row after the last one: a block that has passed the last row
    // reads NaN rows (at most 2 CE + 2 floats beyond it).  Unstarted blocks
    // read the NaN rows before the first.
    const int nre = (nr + 1) & ~1;
    auto set_zp = [&](int tnow) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int o = -2 * (1 + B0 + 32 * j + lane);
            const int cap = nre - 2 * (tnow + 1);
            zp[j] = zr + (o < cap ? o : cap);
        }
    };
    // rows below `filled` are written; the steps of an interval starting after
    // step t read rows below 2 (t + CE)
    int filled = nr < kElFillRows ? nr : kElFillRows;
    fill(0, filled);
    auto fill_to = [&](int need) {
        if (need > nr) need = nr;
        if (need > filled) {
            int to = filled + kElFillRows;
            to = to > need ? to : need;
            to = to < nr ? to : nr;
            fill(filled, to);
            filled = to;
        }
    };
    reset(0);
    load_q(0);
    if (lane == 0) dg[0] = 0.0f;   // D(0, 0) = 0: diagonal of cell (1, 1)
    set_zp(0);

    ub = fminf(ub, 3.402823466e38f);   // +inf cells (borders, retired blocks) are dead
    BestSoFar::Raw ub_raw = BestSoFar::of(ub);
    const int bm = (nc - 1) / K;              // block of the last column
    const int km = (nc - 1) - bm * K;
    const int t_end = bm + 1 + (nr - 1) / 2;  // step holding row nr of block bm
    const bool last_first = (nr & 1) != 0;    // row nr is the first of its step's two rows
    DtwOut out{INF, 0, 0, 0};
    int busy = 0;   // window-steps (the same on every lane)
    if (BANDED && w < 4 * CE) {   // the first steps, before any check, need c - r <= 4 CE - 1
        out.status = 1;
        return out;
    }

    // nz = -z: d = q + nz = q - z exactly
    auto cost = [&](float qv, float nz, float mn) -> float {
        const float d = __fadd_rn(qv, nz);
        return COST == kCostAbsolute ? __fadd_rn(fabsf(d), mn) : __fmaf_rn(d, d, mn);
    };
    auto cost2 = [&](float2 qv, float2 nz, float2 mn) -> float2 {
        const float2 d = __fadd2_rn(qv, nz);
        if (COST == kCostAbsolute) return __fadd2_rn(make_float2(fabsf(d.x), fabsf(d.y)), mn);
        return __ffma2_rn(d, d, mn);
    };
    // Window j's step s given its left inputs: the two rows along
    // anti-diagonals.  Returns the min of the block's outputs (its second row
    // and the first row's last column); with cap, row nr's column km into fin.
    float fin = INF;
    auto cells = [&](int j, int s, float l0, float l1, bool cap) -> float {
        const float2 zz = *reinterpret_cast<const float2*>(zp[j] + 2 * s);   // (-z_r, -z_r+1)
        const float z0 = zz.x, z1 = zz.y;
        float a0, a1, a2, a3, b0, b1, b2, b3;
        a0 = cost(q[j][0], z0, fmin3(p[j][0], dg[j], l0));
        if (kElPaired) {
            const int jq = kElPaired ? j : 0;
            float2 v = cost2(qp[jq][0], zz, make_float2(fmin3(p[j][1], p[j][0], a0), fmin3(a0, l0, l1)));
            a1 = v.x; b0 = v.y;
            v = cost2(qp[jq][kElPaired ? 1 : 0], zz, make_float2(fmin3(p[j][2], p[j][1], a1), fmin3(a1, a0, b0)));
            a2 = v.x; b1 = v.y;
            v = cost2(qp[jq][kElPaired ? 2 : 0], zz, make_float2(fmin3(p[j][3], p[j][2], a2), fmin3(a2, a1, b1)));
            a3 = v.x; b2 = v.y;
        } else {
            a1 = cost(q[j][1], z0, fmin3(p[j][1], p[j][0], a0));
            b0 = cost(q[j][0], z1, fmin3(a0, l0, l1));
            a2 = cost(q[j][2], z0, fmin3(p[j][2], p[j][1], a1));
            b1 = cost(q[j][1], z1, fmin3(a1, a0, b0));
            a3 = cost(q[j][3], z0, fmin3(p[j][3], p[j][2], a2));
            b2 = cost(q[j][2], z1, fmin3(a2, a1, b1));
        }
        b3 = cost(q[j][3], z1, fmin3(a3, a2, b2));
        if (cap) {
            const float ra = km == 0 ? a0 : (km == 1 ? a1 : (km == 2 ? a2 : a3));
            const float rb = km == 0 ? b0 : (km == 1 ? b1 : (km == 2 ? b2 : b3));
            fin = last_first ? ra : rb;
        }
        p[j][0] = b0; p[j][1] = b1; p[j][2] = b2; p[j][3] = b3;
        lo0[j] = a3;
        lo1[j] = b3;
        dg[j] = l1;
        return fmin3(fmin3(b0, b1, b2), b3, a3);
    };
    // Left inputs of window j: lane l takes lane l-1's last column; lane 0
    // takes lane 31's of window j-1 (+inf for window 0).  All windows' inputs
    // are read before any window computes.
    auto left = [&](int j, float& l0, float& l1) {
        const bool last = lane == 31;
        const float s0 = last ? (j > 0 ? lo0[j > 0 ? j - 1 : 0] : INF) : lo0[j];
        const float s1 = last ? (j > 0 ? lo1[j > 0 ? j - 1 : 0] : INF) : lo1[j];
        l0 = __shfl_sync(kFull, s0, (lane + 31) & 31);
        l1 = __shfl_sync(kFull, s1, (lane + 31) & 31);
    };

    // CE steps with ja active windows, then the check.  Returns 0 to go on,
    // 1 when every active block was dead at the last two steps (+inf), 2 on
    // overflow.
    auto interval = [&](auto ja) -> int {
        constexpr int JA = decltype(ja)::value;
        float bma[JA], bmb[JA];
#pragma unroll
        for (int s = 1; s <= CE; ++s) {
            float l0[JA], l1[JA];
#pragma unroll
            for (int j = 0; j < JA; ++j) left(j, l0[j], l1[j]);
#pragma unroll
            for (int j = 0; j < JA; ++j) {
                const float mn = cells(j, t + s, l0[j], l1[j], false);
                if (s == CE - 1) bma[j] = mn;
                if (s == CE) bmb[j] = mn;
            }
        }
        t += CE;
        busy += JA * CE;
        // ---- check ----
        ub = fminf(ub, __shfl_sync(kFull, BestSoFar::finish(ub_raw), 0));   // one reading for the warp
        ub_raw = bsf.issue();
        unsigned da[JA], db[JA];
        bool all_dead = true;
        int hi = -1;   // highest block (relative to B0) alive at step t - 1 or t
#pragma unroll
        for (int j = 0; j < JA; ++j) {
            da[j] = __ballot_sync(kFull, !(bma[j] <= ub));
            db[j] = __ballot_sync(kFull, !(bmb[j] <= ub));
            const unsigned al = ~(da[j] & db[j]);
            all_dead = all_dead && al == 0u;
            if (al) hi = 32 * j + 31 - __clz(al);
        }
        const unsigned cond = db[0] & ((da[0] << 1) | 1u);   // retirable leading blocks of window 0
        if (all_dead || (JA == 1 && cond == kFull)) return 1;
        const int d = (cond == kFull) ? 32 : (__ffs(~cond) - 1);
        if (BANDED && (6 * (B0 + hi) - 2 * t + 4 * CE + 5 > w || 2 * (t + CE) - 6 * (B0 + d) - 1 > w))
            return 2;   // an alive cell may leave the band: the banded levels re-run it
        // windows needed without and with the slide (an alive block needs
        // CE + 1 blocks after it), capped by the window holding the last column
        auto need = [&](int sh) {
            int nd = (hi - sh + CE + 1) / 32 + 1;
            const int cap_w = (bm - (B0 + sh)) / 32 + 1;
            nd = nd < cap_w ? nd : cap_w;
            return nd < 1 ? 1 : nd;
        };
        const int n0 = need(0);
        int nnew = n0, shift = 0;
        if (d > 0) {
            const int nd = need(d);
            if (nd < JA || n0 > JA) {
                shift = d;
                nnew = nd;
            }
        }
        if (nnew > J) return 2;   // the live region is wider than J windows
        if (shift > 0) {
            // lane l of window j takes block B0 + shift + 32 j + l: from lane
            // l + shift of window j, or lane l + shift - 32 of window j + 1
            // (+inf past the active windows); each lane sends the value its
            // receiver needs.  shift = 32 drops window 0 (every lane takes its
            // own lane of the next window).
            B0 += shift;
            const int src = (lane + shift) & 31;
            const bool nxt = lane < shift;
#pragma unroll
            for (int j = 0; j < JA; ++j) {
                const bool on = j + 1 < JA;
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
        // windows switched on start with +inf state; switched-off ones are dropped
#pragma unroll
        for (int j = JA; j < J; ++j) {
            if (j < nnew) {
                reset(j);
                load_q(j);
            }
        }
        jact = nnew;
        // the row pointers move with a slide; near the last row they are capped
        if (shift > 0 || t + 2 * CE >= B0 + (nre >> 1)) set_zp(t);
        return 0;
    };

    for (;;) {
        if (t + CE < t_end) {
            fill_to(2 * (t + CE));
            int r;
            if (jact == 1) r = interval(std::integral_constant<int, 1>{});
            else if (J >= 2 && jact == 2) r = interval(std::integral_constant<int, (J >= 2 ? 2 : 1)>{});
            else if (J >= 3 && jact == 3) r = interval(std::integral_constant<int, (J >= 3 ? 3 : 1)>{});
            else r = interval(std::integral_constant<int, J>{});
            if (r == 0) continue;
            out.status = r == 2 ? 1 : 0;
            out.steps = t;
            break;
        }
        // The last steps up to t_end (at most CE: no check falls before it).
        // Every lane takes every step (the steps shuffle); each captures its
        // own block of the window holding the last column, and the lane of
        // block bm passes it on.  If that block lies beyond the active windows
        // no alive value ever reached it (the switch-on rule): the result is +inf.
        const int src = bm - B0;
        fill_to(nr);
        for (int s = t + 1; s <= t_end; ++s) {
            float l0[J], l1[J];
#pragma unroll
            for (int j = 0; j < J; ++j)
                if (j < jact) left(j, l0[j], l1[j]);
#pragma unroll
            for (int j = 0; j < J; ++j)
                if (j < jact) cells(j, s, l0[j], l1[j], s == t_end && src >= 0 && j == (src >> 5));
        }
        busy += jact * (t_end - t);
        fin = __shfl_sync(kFull, fin, src & 31);
        if (src < 0 || src >= 32 * jact) fin = INF;
        out.dist = (fin <= INF) ? fin : INF;   // NaN (no path through started rows) is +inf
        out.steps = t_end;
        break;
    }
    out.busy = 32 * busy;
    return out;
}

}  // namespace eapdtw
