// EAPrunedDTW as a warp wavefront (sm_103a).
//
// What is computed: the DTW recurrence of Eq. 1-5 (cost (a - b)^2) restricted
// to the band |r - c| <= w (Section 2.1), with early abandoning against an
// upper bound ub (Section 2.2).  The result is DTW if DTW <= ub, else +inf:
// exactly the contract of Algorithm 3 (EAPrunedDTW).
//
// How (a GPU restatement of Algorithm 3's borders, not its loop structure):
//  * Layout.  The DP row is held in registers: lane l owns K consecutive
//    columns ("block" b = B0 + l, columns b*K+1 .. b*K+K).  Rows are pipelined
//    across lanes: block b computes row r at step t = r + b, so the left
//    neighbour of its first column (last column of block b-1, same row) was
//    produced by lane l-1 one step earlier and arrives by one warp shuffle.
//    Top and diagonal neighbours stay in the lane's registers.  One shuffle
//    per K cells.
//  * Left border (next_start, Section 3).  Cells above ub are "dead": every
//    path through them costs more than ub.  When the leftmost block of the
//    warp's window is dead and its left neighbour is retired, no later row of
//    it can be alive, so it is retired and the window slides right (the
//    discard points of Algorithm 3 moving next_start; the band's left edge
//    retires blocks the same way).
//  * Right border (pruning_point, Section 4).  Cells right of the last alive
//    cell only receive dead inputs from above, so they are dead unless the
//    left chain keeps them alive; no bookkeeping is needed: they are computed
//    as dead values inside the window.  A live chain reaching past the
//    window's last block is an overflow: the caller re-runs the candidate
//    with a wider block (larger K).
//  * Early abandoning (border collision / full discard line).  When every
//    block of the window is dead at two consecutive steps, every later cell
//    has dead inputs only: the result is +inf.
//  * Band.  Only two cells per row must be forced to +inf: the one just left
//    of the band (it is the left neighbour of the first band cell) and the one
//    just right of it (it is the top neighbour of the next row's last band
//    cell); every other out-of-band cell then only ever sees +inf inputs and
//    stays +inf by induction from the +inf border row.
//  * Columns past the end (c > nc) hold NaN: fminf ignores NaN operands, so
//    such cells act as +inf and never count as alive.
//
// Arithmetic: each cell is fma(d, d, min(top, diag, left)) with d = z - q in
// FP32; min is exact, so every alive cell equals the sequential FP32 DP value
// regardless of the order in which cells are computed.
#pragma once

#include "common.cuh"

namespace eapdtw {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCheckEvery = 8;  // steps between border / abandon checks (power of 2)

struct DtwOut {
    float dist;     // DTW value or +inf
    int status;     // 0 = done, 1 = overflow (live region wider than the window)
    int steps;      // wavefront steps executed
    int busy;       // lane-steps that computed a block (cells = busy * K)
};

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }
__device__ __forceinline__ float f_nan() { return __int_as_float(0x7fffffff); }

// Rows r = 1..nr take values znorm1(rows[r-1], a, cw, isd); columns c = 1..nc
// take cols[c-1] (already normalised; cols must be 16-byte aligned).
// BAND = 0: unconstrained (only valid when w >= max(nr, nc) - 1);
// BAND = 1: banded with K <= 2w + 2 (at most one forced cell per block and row);
// BAND = 2: banded, any w (two forced cells may share a block).
// All 32 lanes call it with identical arguments.
template <int K, int BAND>
__device__ __forceinline__ DtwOut dtw_warp(const float* __restrict__ rows, float a, float cw,
                                           float isd, const float* __restrict__ cols, int nr,
                                           int nc, int w, const BestSoFar bsf, float ub) {
    static_assert(K % 4 == 0, "K must be a multiple of 4");
    const int lane = threadIdx.x & 31;
    const float INF = f_inf();
    float prv[K];
    float zc[K];
    int B0 = 0;

    auto load_cols = [&]() {
        const int cb = (B0 + lane) * K;
        if (cb + K <= nc && (reinterpret_cast<uintptr_t>(cols + cb) & 15) == 0) {
            const float4* p = reinterpret_cast<const float4*>(cols + cb);
#pragma unroll
            for (int q = 0; q < K / 4; ++q) {
                const float4 v = p[q];
                zc[4 * q] = v.x; zc[4 * q + 1] = v.y; zc[4 * q + 2] = v.z; zc[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) zc[k] = (cb + k < nc) ? cols[cb + k] : f_nan();
        }
    };
    load_cols();
#pragma unroll
    for (int k = 0; k < K; ++k) prv[k] = INF;

    float lout = INF;                         // my block's last cell, previous step
    float lprev = (lane == 0) ? 0.0f : INF;   // left input of the previous step; D(0,0) = 0
    float omin = INF;                         // min of lout since the last check
    float ub_next = ub;
    unsigned dead_a = 0;
    const int bm = (nc - 1) / K;              // block of the last column
    const int km = (nc - 1) - bm * K;
    const int t_end = nr + bm;                // step computing cell (nr, nc)
    DtwOut out{INF, 0, 0, 0};
    int busy = 0;

    // One wavefront step for row r of this lane's block.  f1 is the position,
    // in the block, of the column just left of the band (the one just right of
    // it is f1 + 2w + 2); both are forced to +inf.
    auto cells = [&](float z, float lin, int f1) {
        float diag = lprev;
        float left = lin;
        int kf = -1, kf2 = -1;
        if (BAND != 0) {
            const int f2 = f1 + 2 * w + 2;
            kf = (static_cast<unsigned>(f1) < static_cast<unsigned>(K)) ? f1 : f2;
            kf2 = f2;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float top = prv[k];
            const float d = __fsub_rn(z, zc[k]);
            float v = __fmaf_rn(d, d, fminf(fminf(top, diag), left));
            if (BAND == 1) v = (k == kf) ? INF : v;
            if (BAND == 2) v = (k == kf || k == kf2) ? INF : v;
            diag = top;
            left = v;
            prv[k] = v;
        }
        lout = prv[K - 1];
        omin = fminf(omin, lout);
    };
    auto block_min = [&]() {
        float bmin = prv[0];
#pragma unroll
        for (int k = 1; k < K; ++k) bmin = fminf(bmin, prv[k]);
        return bmin;
    };
    // Border / abandon checks after step t (t a multiple of kCheckEvery):
    // returns true when the candidate is finished (abandoned or overflowed).
    auto check = [&](float bmin_b, int t) -> bool {
        ub = fminf(ub, ub_next);
        const unsigned dead_b = __ballot_sync(kFull, !(bmin_b <= ub));
        // Overflow: the last block of the window passed an alive value to a
        // block outside the window.
        const bool ovf = __shfl_sync(kFull, omin <= ub, 31) && (B0 + 31 < bm);
        if (ovf) {
            out.status = 1;
            out.steps = t;
            return true;
        }
        // Retire leading blocks: block 0 of the window needs to be dead now;
        // block j >= 1 also needs block j-1 dead one step earlier (that value
        // is its diagonal input at the next row).
        const unsigned cond = dead_b & ((dead_a << 1) | 1u);
        const int d = (cond == kFull) ? 32 : (__ffs(~cond) - 1);
        if (d == 32 || (dead_a == kFull && dead_b == kFull)) {
            out.dist = INF;  // every cell of the frontier is above ub
            out.steps = t;
            return true;
        }
        ub_next = bsf.load();
        omin = INF;
        if (d > 0) {
            B0 += d;
            const bool fresh = lane >= 32 - d;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float v = __shfl_down_sync(kFull, prv[k], d);
                prv[k] = fresh ? INF : v;
            }
            const float lp = __shfl_down_sync(kFull, lprev, d);
            const float lo = __shfl_down_sync(kFull, lout, d);
            lprev = fresh ? INF : lp;
            lout = fresh ? INF : lo;
            load_cols();
        }
        return false;
    };

    int t = 0;  // last completed step
    for (;;) {
        // Fast path: the next kCheckEvery steps keep every lane's row inside
        // [1, nr] and stop short of the final step, so no per-lane range test.
        if ((t & (kCheckEvery - 1)) == 0 && t + 1 - (B0 + 31) >= 1 && t + kCheckEvery - B0 <= nr &&
            t + kCheckEvery < t_end) {
            const int b = B0 + lane;
            const float* rp = rows + (t - b - 1);  // rp[s] = rows[r - 1], r = t + s - b
            const int f1base = t - b - w - 1 - b * K - 1;
            float bmin_a = INF, bmin_b = INF;
#pragma unroll
            for (int s = 1; s <= kCheckEvery; ++s) {
                float lin = __shfl_up_sync(kFull, lout, 1);
                lin = (lane == 0) ? INF : lin;
                cells(znorm1(rp[s], a, cw, isd), lin, f1base + s);
                lprev = lin;
                if (s == kCheckEvery - 1) bmin_a = block_min();
                if (s == kCheckEvery) bmin_b = block_min();
            }
            busy += kCheckEvery;
            t += kCheckEvery;
            dead_a = __ballot_sync(kFull, !(bmin_a <= ub));
            if (check(bmin_b, t)) break;
            continue;
        }
        // General step with per-lane range tests (pipeline fill and drain).
        ++t;
        const int b = B0 + lane;
        const int r = t - b;
        float lin = __shfl_up_sync(kFull, lout, 1);
        if (lane == 0) lin = INF;
        const int phase = t & (kCheckEvery - 1);
        float bmin = INF;
        if (r >= 1 && r <= nr) {
            cells(znorm1(rows[r - 1], a, cw, isd), lin, r - w - 1 - (b * K + 1));
            ++busy;
            if (phase == 0 || phase == kCheckEvery - 1) bmin = block_min();
        } else if (r < 1) {
            lout = INF;
        }
        lprev = lin;

        if (t == t_end) {
            const int src = bm - B0;
            float fin = INF;
            if (src >= 0 && src < 32) {
                float mine = prv[0];
#pragma unroll
                for (int k = 1; k < K; ++k) mine = (k == km) ? prv[k] : mine;
                fin = __shfl_sync(kFull, mine, src);
            } else if (src >= 32) {
                out.status = 1;
            }
            out.dist = fin;
            out.steps = t;
            break;
        }
        if (phase == kCheckEvery - 1) {
            dead_a = __ballot_sync(kFull, !(bmin <= ub));
        } else if (phase == 0) {
            if (check(bmin, t)) break;
        }
    }
    // warp totals of busy lane-steps
    int bs = busy;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bs += __shfl_xor_sync(kFull, bs, o);
    out.busy = bs;
    return out;
}

}  // namespace eapdtw
