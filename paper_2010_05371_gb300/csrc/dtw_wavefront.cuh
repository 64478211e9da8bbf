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
//    retires blocks the same way).  With one window the slide is lazy: dead
//    leading blocks stay in place until the live region nears the window's end.
//  * Right border (pruning_point, Section 4).  Cells right of the last alive
//    cell only receive dead inputs from above, so they are dead unless the
//    left chain keeps them alive; no bookkeeping is needed: they are computed
//    as dead values inside the window.  The window is elastic: up to J
//    windows of 32 blocks follow one another (lane l also owns block
//    B0 + 32j + l of window j); window j+1 is switched on when an alive cell
//    comes within 9 blocks of the end of window j (the live region grows by
//    at most one block per step, and the checks come every 8 steps), and off
//    again when it and the end of window j are dead.  A live chain reaching
//    past the last of the J windows is an overflow: the caller re-runs the
//    candidate with wider blocks (larger K).
//  * Early abandoning (border collision / full discard line).  When every
//    block of the window is dead at two consecutive steps, every later cell
//    has dead inputs only: the result is +inf.  These checks come every 16
//    steps with one window in the unconstrained case and every 8 otherwise.
//  * Upper bound tightening (optional, the UCR Suite's use of LB_Keogh that
//    Section 5 keeps).  Every warping path visits every row, and a row's cells
//    cost at least that row's LB_Keogh EQ term, so a cell of row r whose value
//    plus the terms of rows r+1..nr exceeds ub is dead too.  The threshold
//    rises with the row, and the retirement and abandon arguments hold with it:
//    a cell derived from dead cells of row r pays at least the terms of the
//    rows in between, so it stays above its own row's threshold.
//  * Band.  Only two cells per row must be forced to +inf: the one just left
//    of the band (it is the left neighbour of the first band cell) and the one
//    just right of it (it is the top neighbour of the next row's last band
//    cell); every other out-of-band cell then only ever sees +inf inputs and
//    stays +inf by induction from the +inf border row.
//  * Columns past the end (c > nc) hold NaN: fminf ignores NaN operands, so
//    such cells act as +inf and never count as alive.
//
// Arithmetic: each cell is fma(d, d, min(top, diag, left)) with d = q - z in
// FP32 (two adjacent columns per packed f32x2 add); min is exact, so every
// alive cell equals the sequential FP32 DP value regardless of the order in
// which cells are computed.
#pragma once

#include "common.cuh"

namespace eapdtw {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCostSquared = 0;   // cost(a, b) = (a - b)^2
constexpr int kCostAbsolute = 1;  // cost(a, b) = |a - b|
// Steps between border / abandon checks (a power of 2; a compile-time knob for
// tuning experiments).
#ifndef EAPDTW_CHECK_EVERY
#define EAPDTW_CHECK_EVERY 8
#endif
constexpr int kCheckEvery = EAPDTW_CHECK_EVERY;
// The same for the unconstrained one-window kernels.  There the per-lane
// corner check always runs first and removes the windows that die within a
// few rows, so the survivors live long enough that checking half as often
// pays.  Banded searches (where the corner check may not run, and short
// queries abound) and the multi-window levels (whose window switch-on margin
// is sized for 8) keep 8.
#ifndef EAPDTW_CHECK_EVERY_ONE
#define EAPDTW_CHECK_EVERY_ONE 16
#endif
constexpr int kCheckEveryOne = EAPDTW_CHECK_EVERY_ONE;

struct DtwOut {
    float dist;     // DTW value or +inf
    int status;     // 0 = done, 1 = overflow (live region wider than the window)
    int steps;      // wavefront steps executed
    int busy;       // lane-steps that computed a block (cells = busy * K)
};

// Windows of 32 blocks a candidate may use.  A second window for narrow blocks
// of the unconstrained case (EAPDTW_WIDE_WINDOWS=2) executes fewer cells on
// wide candidates but needs about 120 registers per thread, which halves the
// resident warps; measured on GB300 it ran about 2x slower, so one window is
// the default and wide live regions are re-run with wider blocks instead.
#ifndef EAPDTW_WIDE_WINDOWS
#define EAPDTW_WIDE_WINDOWS 1
#endif
__host__ __device__ constexpr int dtw_windows(int K, int BAND) {
    return (BAND == 0 && K <= 8) ? EAPDTW_WIDE_WINDOWS : 1;
}

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }
__device__ __forceinline__ float f_nan() { return __int_as_float(0x7fffffff); }

// Rows r = 1..nr take values znorm1(rows[r-1], a, cw, isd); columns c = 1..nc
// take cols[c-1] (already normalised).
// BAND = 0: unconstrained (only valid when w >= max(nr, nc) - 1);
// BAND = 1: banded with K <= 2w + 2 (at most one forced cell per block and row);
// BAND = 2: banded, any w (two forced cells may share a block).
// J: windows of 32 blocks available to the live region.
// CS: read the column values from `cols` at every step instead of holding them
// in registers (for the widest windows, whose registers would not fit).
// All 32 lanes call it with identical arguments.
// TIGHT: upper-bound tightening with cb (see thr below); compiled out otherwise.
// COST: the pointwise cost of the recurrence: kCostSquared, (a - b)^2 (Eq. 5, the
// paper's); kCostAbsolute, |a - b| (another elastic distance with the same
// recurrence, Section 6).  Both are non-negative, so the pruning and abandoning
// arguments hold unchanged.
// check2: 1 checks borders and the bound at twice the built-in interval (the
// autotuner's poll-interval choice; the retirement and switch-on margins grow
// with it), 0 at the built-in one.  Results are the same either way.
template <int K, int BAND, int J = 1, bool CS = false, bool TIGHT = false, int COST = 0>
__device__ __forceinline__ DtwOut dtw_warp(const float* __restrict__ rows, float a, float cw,
                                           float isd, const float* __restrict__ cols, int nr,
                                           int nc, int w, const BestSoFar bsf, float ub,
                                           int* dbg = nullptr, const float* __restrict__ cb = nullptr,
                                           int check2 = 0) {
    static_assert(K % 4 == 0, "K must be a multiple of 4");
    static_assert(J >= 1 && J <= 4, "1 to 4 windows");
    (void)dbg;
    const int lane = threadIdx.x & 31;
    const float INF = f_inf();
    float prv[J][K];
    float zc[CS ? 1 : J][K];
    float lout[J];    // each window's last cell of this lane's block, previous step
    float lprev[J];   // left input of the previous step (diagonal of cell 0)
    float omin[J];    // min of lout since the last check
    unsigned dead_a[J];
    int B0 = 0;
    int jact = 1;     // active windows

    // Column values of window j's block into q[0..K) (+NaN past the last column).
    auto fetch_cols = [&](int j, float* q) {
        const int cb = (B0 + 32 * j + lane) * K;
        if (cb + K <= nc && (reinterpret_cast<uintptr_t>(cols + cb) & 15) == 0) {
            const float4* p = reinterpret_cast<const float4*>(cols + cb);
#pragma unroll
            for (int u = 0; u < K / 4; ++u) {
                const float4 v = p[u];
                q[4 * u] = v.x; q[4 * u + 1] = v.y; q[4 * u + 2] = v.z; q[4 * u + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) q[k] = (cb + k < nc) ? cols[cb + k] : f_nan();
        }
    };
    auto load_cols = [&](int j) {
        if (!CS) fetch_cols(j, zc[CS ? 0 : j]);
    };
    auto reset = [&](int j) {
#pragma unroll
        for (int k = 0; k < K; ++k) prv[j][k] = INF;
        lout[j] = INF;
        lprev[j] = INF;
        omin[j] = INF;
        dead_a[j] = kFull;
    };
#pragma unroll
    for (int j = 0; j < J; ++j) {
        reset(j);
        load_cols(j);
    }
    if (lane == 0) lprev[0] = 0.0f;   // D(0,0) = 0: diagonal of cell (1,1)

    // A cell is alive iff v <= ub.  +inf marks cells that do not exist (the
    // border, out-of-band cells, retired blocks), so ub is kept finite: with
    // ub = +inf, a +inf cell would otherwise count as alive.
    ub = fminf(ub, 3.402823466e38f);
    constexpr int kCE = (J == 1 && BAND == 0) ? kCheckEveryOne : kCheckEvery;   // steps between checks
    // lanes 31-ce .. 31 for the effective interval ce: an alive cell there can
    // reach the window's end before the next check
    const int ce_eff = check2 ? 2 * kCE : kCE;
    const unsigned near_mask = ce_eff >= 31 ? kFull : (kFull << (31 - ce_eff));
    // The bound read at the last check, applied at the next one (its loads
    // complete meanwhile).
    BestSoFar::Raw ub_raw = BestSoFar::of(ub);
    const int bm = (nc - 1) / K;       // block of the last column
    const int km = (nc - 1) - bm * K;
    const int t_end = nr + bm;         // step computing cell (nr, nc)
    DtwOut out{INF, 0, 0, 0};
    int busy = 0;

    // Left inputs of every active window, read before any lout changes.
    auto left_inputs = [&](float* lin) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (j < jact) {
                const float up = __shfl_up_sync(kFull, lout[j], 1);
                float from_prev = INF;
                if (j > 0) from_prev = __shfl_sync(kFull, lout[j - 1], 31);
                lin[j] = (lane == 0) ? from_prev : up;
            }
        }
    };
    // One wavefront step of window j for row r of this lane's block.  f1 is
    // the position, in the block, of the column just left of the band (the one
    // just right of it is f1 + 2w + 2); both are forced to +inf.
    auto cells = [&](int j, float z, float lin, int f1) {
        float qs[CS ? K : 1];
        if (CS) fetch_cols(j, qs);
        float diag = lprev[j];
        float left = lin;
        int kf = -1, kf2 = -1;
        if (BAND != 0) {
            const int f2 = f1 + 2 * w + 2;
            kf = (static_cast<unsigned>(f1) < static_cast<unsigned>(K)) ? f1 : f2;
            kf2 = f2;
        }
        // d = q - z for two adjacent columns per packed f32x2 add; the cost
        // squares d or takes its absolute value, so the sign is immaterial and
        // fl(q - z) = -fl(z - q) gives the scalar form's values exactly.
        const float2 nz = make_float2(-z, -z);
#pragma unroll
        for (int k = 0; k < K; k += 2) {
            const float2 dd = __fadd2_rn(CS ? make_float2(qs[CS ? k : 0], qs[CS ? k + 1 : 0])
                                            : make_float2(zc[CS ? 0 : j][k], zc[CS ? 0 : j][k + 1]),
                                         nz);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float top = prv[j][k + u];
                const float d = u ? dd.y : dd.x;
                const float mn = fmin3(top, diag, left);
                float v = (COST == kCostAbsolute) ? __fadd_rn(fabsf(d), mn) : __fmaf_rn(d, d, mn);
                if (BAND == 1) v = (k + u == kf) ? INF : v;
                if (BAND == 2) v = (k + u == kf || k + u == kf2) ? INF : v;
                diag = top;
                left = v;
                prv[j][k + u] = v;
            }
        }
        lout[j] = prv[j][K - 1];
        lprev[j] = lin;
        omin[j] = fminf(omin[j], lout[j]);
    };
    auto block_min = [&](int j) {
        float bmin = fminf(prv[j][0], prv[j][K - 1]);
#pragma unroll
        for (int k = 1; k + 1 < K - 1; k += 2) bmin = fmin3(bmin, prv[j][k], prv[j][k + 1]);
        return bmin;
    };
    // Death threshold of window j's block at step `step` (its row r = step - block).
    // Without tightening: ub.  With it (cb[r] = a lower bound of the cost of rows r+1..nr,
    // the suffix sums of the window's LB_Keogh EQ terms): a cell of row r is dead
    // when even the cheapest completion exceeds ub, v > ub (1 + 1e-4) - cb[r]
    // (the margin absorbs FP32 rounding of v and cb); never looser than ub.
    auto thr = [&](int j, int step) -> float {
        if (!TIGHT) return ub;
        int r = step - (B0 + 32 * j + lane);
        r = r < 0 ? 0 : (r > nr ? nr : r);
        return fminf(ub, __fsub_rn(__fmul_rn(ub, 1.0001f), cb[r]));
    };
    // Border / abandon checks after step t (t a multiple of kCE);
    // dead_a holds the dead lanes of the step before.  Returns true when the
    // candidate is finished (abandoned or overflowed).
    auto check = [&](const float* bmin_b, int t) -> bool {
        const float ub_next = __shfl_sync(kFull, BestSoFar::finish(ub_raw), 0);  // one reading for the whole warp
#ifdef EAPDTW_DEVICE_CHECKS
        EAPDTW_CHECK(dbg, __shfl_sync(kFull, t, 0) == t, 13, t);
        EAPDTW_CHECK(dbg, __shfl_sync(kFull, B0, 0) == B0, 14, B0);
        EAPDTW_CHECK(dbg, __shfl_sync(kFull, jact, 0) == jact, 15, jact);
        EAPDTW_CHECK(dbg, __shfl_sync(kFull, __float_as_int(ub), 0) == __float_as_int(ub), 16, 0);
        EAPDTW_CHECK(dbg, __shfl_sync(kFull, __float_as_int(ub_next), 0) == __float_as_int(ub_next), 17, 0);
#endif
        ub = fminf(ub, ub_next);
        unsigned db[J];
#pragma unroll
        for (int j = 0; j < J; ++j)
            db[j] = (j < jact) ? __ballot_sync(kFull, !(bmin_b[j] <= thr(j, t))) : kFull;
        // Overflow: the last active window passed an alive value beyond itself.
        float om = omin[0];
#pragma unroll
        for (int j = 1; j < J; ++j) om = (j == jact - 1) ? omin[j] : om;
        if (__shfl_sync(kFull, om <= ub, 31) && B0 + 32 * jact - 1 < bm) {
            out.status = 1;
            out.steps = t;
            return true;
        }
        // Every active block dead at two consecutive steps: abandon.
        bool all_dead = true;
#pragma unroll
        for (int j = 0; j < J; ++j) all_dead &= (j >= jact) || (dead_a[j] == kFull && db[j] == kFull);
        // Retire leading blocks of window 0: block 0 needs to be dead now;
        // block j >= 1 also needs block j-1 dead one step earlier (that value
        // is its diagonal input at the next row).
        const unsigned cond = db[0] & ((dead_a[0] << 1) | 1u);
        if (all_dead || (jact == 1 && cond == kFull)) {
            out.dist = INF;
            out.steps = t;
            return true;
        }
        int d = (cond == kFull) ? 31 : (__ffs(~cond) - 1);
        // One window: retire lazily.  Dead leading blocks stay dead, so the
        // slide (two shuffles per DP value and a reload of the column values)
        // waits until an alive cell comes within kCE + 1 blocks of the
        // window's end.  An alive block at step s+1 needs an alive input at
        // step s or s-1 one block to its left at most, so with nothing alive
        // in lanes 31-kCE..31 at steps t-1 and t, nothing alive reaches the
        // last lane before the next check.
        if (J == 1 && d > 0 && (~(dead_a[0] & db[0]) & near_mask) == 0) d = 0;
        // Switch the next window on when an alive cell came within 9 blocks
        // of the end of the last active one; off when the last one and the
        // end of the one before are dead.
        if (J > 1) {
            const unsigned kNear = near_mask;   // lanes 31-ce .. 31 (23..31 at 8 steps)
            unsigned near_last = 0, near_prev = 0, dead_last = 0;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (j == jact - 1) {
                    near_last = ~(dead_a[j] & db[j]) & kNear;
                    dead_last = (dead_a[j] == kFull && db[j] == kFull) ? 1u : 0u;
                }
                if (j == jact - 2) near_prev = ~(dead_a[j] & db[j]) & kNear;
            }
            if (jact < J && near_last) {
                ++jact;  // its state is +inf (reset when it was switched off)
            } else if (jact > 1 && dead_last && !near_prev) {
#pragma unroll
                for (int j = 1; j < J; ++j)
                    if (j == jact - 1) reset(j);
                --jact;
            }
        }
        ub_raw = bsf.issue();
#pragma unroll
        for (int j = 0; j < J; ++j) omin[j] = INF;
        if (d > 0) {
            // Slide every active window d blocks right: lane l of window j
            // takes block B0 + d + 32j + l from lane l + d of window j, or from
            // lane l + d - 32 of window j + 1 (+inf past the active windows).
            B0 += d;
            const int src = (lane + d) & 31;
            const bool from_next = lane < d;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (j < jact) {
                    const bool nxt_on = j + 1 < jact;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float nx = (j + 1 < J && nxt_on) ? prv[j + 1 < J ? j + 1 : j][k] : INF;
                        prv[j][k] = __shfl_sync(kFull, from_next ? nx : prv[j][k], src);
                    }
                    const float nlo = (j + 1 < J && nxt_on) ? lout[j + 1 < J ? j + 1 : j] : INF;
                    const float nlp = (j + 1 < J && nxt_on) ? lprev[j + 1 < J ? j + 1 : j] : INF;
                    lout[j] = __shfl_sync(kFull, from_next ? nlo : lout[j], src);
                    lprev[j] = __shfl_sync(kFull, from_next ? nlp : lprev[j], src);
                }
                load_cols(j);
            }
        }
        return false;
    };

    int t = 0;  // last completed step
    for (;;) {
        // Fast path: the next kCE steps keep every active lane's row at most
        // nr and stop short of the final step: no per-lane tests.  A lane
        // whose row is still below 1 (the pipeline filling) computes too: its
        // own values and its left input (the previous lane's output for the
        // same row) are all +inf, so its cells stay +inf (NaN past the last
        // column), exactly the state it would keep by waiting.
        if ((t & (kCE - 1)) == 0 && t + kCE - B0 <= nr && t + kCE < t_end) {
            float bmin_a[J], bmin_b[J];
#pragma unroll
            for (int s = 1; s <= kCE; ++s) {
                float lin[J];
                left_inputs(lin);
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    if (j < jact) {
                        const int bj = B0 + 32 * j + lane;
                        const int r = t + s - bj;
                        const int rr = r < 1 ? 1 : r;   // rows below 1 read row 1 (their cells stay +inf)
                        const float x = EAPDTW_CHECK(dbg, rr <= nr, 11, r) ? rows[rr - 1] : 0.0f;
                        cells(j, znorm1(x, a, cw, isd), lin[j], r - w - 1 - (bj * K + 1));
                        if (s == kCE - 1) bmin_a[j] = block_min(j);
                        if (s == kCE) bmin_b[j] = block_min(j);
                    }
                }
            }
            // lane-steps whose row was in [1, nr]
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (j < jact) {
                    const int started = t + kCE - (B0 + 32 * j + lane);
                    busy += started < kCE ? (started > 0 ? started : 0) : kCE;
                }
            }
            t += kCE;
#pragma unroll
            for (int j = 0; j < J; ++j)
                dead_a[j] = (j < jact) ? __ballot_sync(kFull, !(bmin_a[j] <= thr(j, t - 1))) : kFull;
            if (check2 && (t & kCE)) continue;   // every other check is skipped
            if (check(bmin_b, t)) break;
            continue;
        }
        // General step with per-lane range tests (pipeline fill and drain).
        ++t;
        const int phase = t & (kCE - 1);
        float lin[J], bmin[J];
        left_inputs(lin);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            bmin[j] = INF;
            if (j < jact) {
                const int bj = B0 + 32 * j + lane;
                const int r = t - bj;
                if (r >= 1 && r <= nr) {
                    const float x = EAPDTW_CHECK(dbg, r - 1 < nr, 12, r) ? rows[r - 1] : 0.0f;
                    cells(j, znorm1(x, a, cw, isd), lin[j], r - w - 1 - (bj * K + 1));
                    ++busy;
                    if (phase == 0 || phase == kCE - 1) bmin[j] = block_min(j);
                } else {
                    if (r < 1) lout[j] = INF;
                    lprev[j] = lin[j];
                }
            }
        }
        if (t == t_end) {
            const int src = bm - B0;
            float fin = INF;
            if (src >= 0 && src < 32 * jact) {
                float mine = INF;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    if (j == (src >> 5)) {
#pragma unroll
                        for (int k = 0; k < K; ++k) mine = (k == km) ? prv[j][k] : mine;
                    }
                }
                fin = __shfl_sync(kFull, mine, src & 31);
            } else if (src >= 32 * jact) {
                out.status = 1;
            }
            out.dist = fin;
            out.steps = t;
            break;
        }
        if (phase == kCE - 1) {
#pragma unroll
            for (int j = 0; j < J; ++j)
                dead_a[j] = (j < jact) ? __ballot_sync(kFull, !(bmin[j] <= thr(j, t))) : kFull;
        } else if (phase == 0 && !(check2 && (t & kCE))) {
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

// EAPrunedDTW's first rows, one candidate per lane (Algorithm 3, abandoning).
// Most windows are abandoned within a few rows, while their live cells still
// sit in the top-left corner of the cost matrix.  corner_dead computes rows
// and columns 1..kCorner of one window with the wavefront's own operations
// (the same FP32 values) and reports whether some row r of the corner is
// entirely > ub while column kCorner has been > ub in every row up to r.
// Then no cell right of the corner is alive in rows 1..r either: row 1 only
// grows to the right, and a later cell right of the corner has only dead
// inputs.  So all of row r is > ub, and Algorithm 3 abandons the window.
// Needs m >= kCorner and every corner cell inside the band (w >= kCorner - 1).
// The corner's size is a compile-time knob for tuning experiments.  Up to 16
// columns the query values sit in registers; a wider corner reads them from
// memory at each cell, since the registers would spill.
#ifndef EAPDTW_CORNER
#define EAPDTW_CORNER 16
#endif
constexpr int kCorner = EAPDTW_CORNER;
static_assert(kCorner >= 2 && kCorner <= 32 && kCorner % 2 == 0, "corner of 2 to 32 rows and columns, even");
constexpr bool kCornerQInRegs = kCorner <= 16;
// Run it only when this many lanes of the tile are alive (a knob for tuning
// experiments).
#ifndef EAPDTW_CORNER_MIN_LANES
#define EAPDTW_CORNER_MIN_LANES 8
#endif
constexpr int kCornerMinLanes = EAPDTW_CORNER_MIN_LANES;

template <int COST>
__device__ __forceinline__ bool corner_dead(const float* x, float a, float cw, float isd, const float* zq, float ub) {
    const float INF = f_inf();
    float q[kCornerQInRegs ? kCorner : 1], prv[kCorner];
#pragma unroll
    for (int c = 0; c < kCorner; ++c) {
        if (kCornerQInRegs) q[kCornerQInRegs ? c : 0] = zq[c];
        prv[c] = INF;   // row 0
    }
    bool edge = true;   // column kCorner > ub in every row so far
    for (int r = 0; r < kCorner; ++r) {
        const float z = znorm1(x[r], a, cw, isd);
        float diag = r == 0 ? 0.0f : INF;   // D(0, 0) = 0; D(r, 0) = +inf
        float left = INF;
        const float2 nz = make_float2(-z, -z);   // packed d = q - z, as in dtw_warp
#pragma unroll
        for (int c = 0; c < kCorner; c += 2) {
            const float2 dd = __fadd2_rn(kCornerQInRegs ? make_float2(q[kCornerQInRegs ? c : 0], q[kCornerQInRegs ? c + 1 : 0])
                                                        : make_float2(zq[c], zq[c + 1]),
                                         nz);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float top = prv[c + u];
                const float d = u ? dd.y : dd.x;
                const float mn = fmin3(top, diag, left);
                const float v = (COST == kCostAbsolute) ? __fadd_rn(fabsf(d), mn) : __fmaf_rn(d, d, mn);
                diag = top;
                left = v;
                prv[c + u] = v;
            }
        }
        float rmin = prv[0];
#pragma unroll
        for (int c = 1; c + 1 < kCorner; c += 2) rmin = fmin3(rmin, prv[c], prv[c + 1]);
        rmin = fminf(rmin, prv[kCorner - 1]);
        edge = edge && !(prv[kCorner - 1] <= ub);
        if (edge && !(rmin <= ub)) return true;
    }
    return false;
}

}  // namespace eapdtw
