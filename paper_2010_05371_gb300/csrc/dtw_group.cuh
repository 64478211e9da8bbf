// EAPrunedDTW on a group of warps (sm_103a): the widest re-run level.
//
// What is computed: as dtw_warp (dtw_wavefront.cuh): the DTW recurrence of
// Eq. 1-5 inside the band |r - c| <= w (Section 2.1), early abandoned against
// an upper bound ub (Section 2.2): DTW if DTW <= ub, else +inf.
//
// Why.  A live region wider than one warp's registers can hold (the widest
// re-run level, queries of more than 1024 points) used to run one warp with
// the column values streamed from shared memory at every step.  Here G warps
// of one block share the candidate instead, each holding its own slice of the
// DP row and of the columns in registers:
//  * Layout.  Warp g owns the fixed columns 512 g + 1 .. 512 g + 512 as 32
//    blocks of K = 16 (lane l: block b = 32 g + l), in the one-window
//    wavefront's pipeline: block b computes row r at step t = r + b.  So lane 0
//    of warp g needs at step t the last column of block 32 g - 1 at step
//    t - 1, which lane 31 of warp g - 1 computed; everything else comes from
//    the lane itself or from lane l - 1 by a shuffle, as in dtw_warp.
//  * Edges.  Lane 31 of warp g writes its last column of every step into the
//    warp's ring in shared memory (slot t mod kGrpRing).  Every kGrpCE steps a
//    warp publishes the last step it has written (prog, after a block-scope
//    fence) and the last step it has completed (cons).  Warp g starts the
//    steps t + 1 .. t + kGrpCE once warp g - 1 has published step
//    t + kGrpCE - 1, and warp g - 1 overwrites a slot only after warp g has
//    read it (cons).  A warp is then at most kGrpRing - kGrpCE - 1 steps ahead
//    of its right neighbour and never behind it; the two waits cannot block
//    each other (that would need the producer both ahead of the consumer by
//    more than kGrpRing - kGrpCE and by less than kGrpCE).
//  * Pruning (Sections 3-4).  A warp whose blocks were all dead at the last
//    two steps it checked, and whose left inputs for its next steps are dead
//    too, keeps +inf and skips those steps (a dead value and +inf lead to the
//    same alive cells: none).  This covers both the columns the live region has
//    not reached yet and those it has left behind.
//  * Early abandoning.  A warp dead at two consecutive steps whose left inputs
//    are dead from then on is dead for good: it publishes that (dead) and
//    leaves.  Warp 0's left inputs are the +inf border, so the chain starts
//    there; the candidate is abandoned when the warp holding the last column
//    is dead for good.
//  * Bounded waits.  Every wait polls at most kGrpSpinLimit times; a wait that
//    runs out sets the group's abort flag and the caller's error flag, and
//    every warp of the group leaves the candidate.
// Arithmetic: the one-window wavefront's cells (fma(d, d, min(top, diag,
// left)), d = q - z in FP32, the same two forced cells per row in the band), so
// every alive cell equals the sequential FP32 DP value.
#pragma once

#include "dtw_wavefront.cuh"

namespace eapdtw {

constexpr int kGrpK = 16;                 // columns per block
constexpr int kGrpCols = 32 * kGrpK;      // columns per warp
constexpr int kGrpMaxWarps = 8;           // warps per group: up to 4096 columns
constexpr int kGrpCE = 8;                 // steps between checks (and publications)
constexpr int kGrpRing = 64;              // ring slots per warp (a power of 2)
static_assert(kGrpRing > 2 * kGrpCE, "the producer may run kGrpRing - kGrpCE - 1 steps ahead");
constexpr int kGrpSpinLimit = 1 << 23;    // polls per wait (about half a second)

// Resident blocks per SM the group kernels are compiled for (a compile-time
// knob for tuning experiments).
#ifndef EAPDTW_MINB_GROUP
#define EAPDTW_MINB_GROUP 3
#endif

// Warps a candidate of nc columns uses.
__host__ __device__ constexpr int group_warps(int nc) { return (nc - 1) / kGrpCols + 1; }

// Shared state of one group (one per group of warps in the block).
struct GroupSync {
    float ring[kGrpMaxWarps][kGrpRing];  // warp g's last column at step s in ring[g][s % kGrpRing]
    int prog[kGrpMaxWarps];   // warp g has written its ring entries of steps <= prog[g]
    int cons[kGrpMaxWarps];   // warp g has completed its steps <= cons[g] (read warp g-1's entries < cons[g])
    int dead[kGrpMaxWarps];   // warp g's entries of steps >= dead[g] are dead or past the last row (INT_MAX: none)
    int abort_flag;           // a wait ran out: every warp leaves the candidate
    long long unit;           // the group's current work unit
    // the tile's survivors of the lower-bound stage (lane bits) and their statistics
    unsigned surv;
    int cand;                 // the survivor the group runs next (-1: skipped by the recheck)
    float ub;                 // the bound the leader read for it
    float sa[32], scw[32], sisd[32], slb[32];
};

// Lane 31's store of v to a shared-memory float at the 32-bit shared address
// a, as one predicated instruction (no branch around it).
__device__ __forceinline__ void st_shared_lane31(unsigned a, float v, int lane) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %0, 31;\n\t@p st.volatile.shared.f32 [%1], %2;\n\t}"
                 ::"r"(lane), "r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ float ld_shared_volatile(unsigned a) {
    float v;
    asm volatile("ld.volatile.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}

// Ready for the next candidate: nothing written, nothing dead (one thread).
__device__ __forceinline__ void group_reset(GroupSync& gs) {
    volatile GroupSync& v = gs;
#pragma unroll
    for (int g = 0; g < kGrpMaxWarps; ++g) {
        v.prog[g] = 0;
        v.cons[g] = 0;
        v.dead[g] = 0x7fffffff;
    }
}

// Named barrier 1 + gi of group gi's warps (barrier 0 is __syncthreads); the
// ids are immediates so that the kernel reserves only the barriers it uses.
__device__ __forceinline__ void group_bar(int gi, int nwarps) {
    const int n = nwarps * 32;
    switch (gi) {
        case 0: asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); break;
        case 1: asm volatile("bar.sync 2, %0;" ::"r"(n) : "memory"); break;
        case 2: asm volatile("bar.sync 3, %0;" ::"r"(n) : "memory"); break;
        default: asm volatile("bar.sync 4, %0;" ::"r"(n) : "memory"); break;
    }
}

// Warp g's part of the candidate.  All 32 lanes of each of the candidate's
// group_warps(nc) warps call it with identical arguments (only g differs);
// rows: the window's raw points, in shared or global memory (row r is
// znorm1(rows[r - 1], a, cw, isd));
// cols: the z-normalised query (columns 1..nc); err: err_bit is or-ed into
// it when a wait runs out.  The warp holding the last column returns the result (status 0,
// or 2 when the group was aborted); the others return +inf with their steps
// and busy lane-steps.
template <int BAND, int COST>
__device__ __forceinline__ DtwOut dtw_group(GroupSync& gs, int g, const float* __restrict__ rows, float a, float cw,
                                            float isd, const float* __restrict__ cols, int nr, int nc, int w,
                                            const BestSoFar bsf, float ub, int* err, int err_bit) {
    constexpr int K = kGrpK;
    constexpr int CE = kGrpCE;
    const int lane = threadIdx.x & 31;
    const float INF = f_inf();
    volatile GroupSync& vs = gs;
    const int ge = group_warps(nc);
    const bool last = g == ge - 1;
    const int b = 32 * g + lane;               // this lane's block
    const int bm = (nc - 1) / K;               // block of the last column
    const int km = (nc - 1) - bm * K;
    const int t_fin = last ? nr + bm : nr + 32 * g + 31;   // this warp's last step (its last lane at row nr)

    float prv[K], zc[K];
    {
        const int c0 = b * K;
        if (c0 + K <= nc && (reinterpret_cast<uintptr_t>(cols + c0) & 15) == 0) {
            const float4* p = reinterpret_cast<const float4*>(cols + c0);
#pragma unroll
            for (int u = 0; u < K / 4; ++u) {
                const float4 v = p[u];
                zc[4 * u] = v.x; zc[4 * u + 1] = v.y; zc[4 * u + 2] = v.z; zc[4 * u + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) zc[k] = (c0 + k < nc) ? cols[c0 + k] : f_nan();
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) prv[k] = INF;
    float lout = INF;                                      // last column of the block, previous step
    float lprev = (g == 0 && lane == 0) ? 0.0f : INF;      // D(0, 0) = 0: diagonal of cell (1, 1)
    ub = fminf(ub, 3.402823466e38f);                       // +inf cells (border, band) are dead
    BestSoFar::Raw ub_raw = BestSoFar::of(ub);
    bool own_dead = g > 0;   // every block dead at the last two checked steps (warps g > 0 start at +inf)
    int busy = 0;
    int t = 0;               // last completed step
    DtwOut out{INF, 0, 0, 0};
    const unsigned rin_s = static_cast<unsigned>(__cvta_generic_to_shared(&gs.ring[g > 0 ? g - 1 : 0][0]));
    const unsigned rout_s = static_cast<unsigned>(__cvta_generic_to_shared(&gs.ring[g][0]));
    auto put = [&](int s, float v) {   // lane 31's last column at step s into this warp's ring
        st_shared_lane31(rout_s + 4u * static_cast<unsigned>(s & (kGrpRing - 1)), v, lane);
    };

    // Polls until ready() (lane 0's reading, broadcast); false when the group
    // was aborted or this wait ran out (then the group is aborted).
    auto wait = [&](auto ready) -> bool {
        int ok = 1;
        if (lane == 0) {
            int n = 0;
            while (!ready()) {
                if (vs.abort_flag) { ok = 0; break; }
                if (++n > kGrpSpinLimit) {
                    vs.abort_flag = 1;
                    atomicOr(err, err_bit);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        return __shfl_sync(kFull, ok, 0) != 0;
    };
    // One step of this lane's block at row r (clamped into 1..nr for the
    // read: rows below 1 hold +inf state and inputs, rows past nr only feed
    // rows past nr); f1 positions the band's forced cells as in dtw_warp.
    auto row_at = [&](int r) -> float {   // shared or global memory
        const int rr = r < 1 ? 1 : (r > nr ? nr : r);
        return rows[rr - 1];
    };
    auto cells = [&](int r, float x, float lin) {
        const float z = znorm1(x, a, cw, isd);
        const int f1 = r - w - 1 - (b * K + 1);
        float diag = lprev;
        float left = lin;
        int kf = -1, kf2 = -1;
        if (BAND != 0) {
            const int f2 = f1 + 2 * w + 2;
            kf = (static_cast<unsigned>(f1) < static_cast<unsigned>(K)) ? f1 : f2;
            kf2 = f2;
        }
        const float2 nz = make_float2(-z, -z);
#pragma unroll
        for (int k = 0; k < K; k += 2) {
            const float2 dd = __fadd2_rn(make_float2(zc[k], zc[k + 1]), nz);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float top = prv[k + u];
                const float d = u ? dd.y : dd.x;
                const float mn = fmin3(top, diag, left);
                float v = (COST == kCostAbsolute) ? __fadd_rn(fabsf(d), mn) : __fmaf_rn(d, d, mn);
                if (BAND == 1) v = (k + u == kf) ? INF : v;
                if (BAND == 2) v = (k + u == kf || k + u == kf2) ? INF : v;
                diag = top;
                left = v;
                prv[k + u] = v;
            }
        }
        lout = prv[K - 1];
        lprev = lin;
    };
    auto block_min = [&]() {
        float m = fminf(prv[0], prv[K - 1]);
#pragma unroll
        for (int k = 1; k + 1 < K - 1; k += 2) m = fmin3(m, prv[k], prv[k + 1]);
        return m;
    };
    // lane-steps of steps t0+1 .. t0+n whose row is in 1..nr
    auto rows_in = [&](int t0, int n) {
        const int lo = max(t0 + 1 - b, 1);
        const int hi = min(t0 + n - b, nr);
        return hi >= lo ? hi - lo + 1 : 0;
    };

    for (;;) {
        const int t_next = min(t + CE, t_fin);
        const int ns = t_next - t;
        // left inputs of steps t+1 .. t_next: warp g-1's last column at steps
        // t .. t_next-1 (ring entries below dd; +inf from dd on)
        int dd = 0;
        if (g > 0) {
            if (!wait([&] { return vs.prog[g - 1] >= t_next - 1 || vs.dead[g - 1] <= t_next - 1; })) {
                out.status = 2;
                break;
            }
            __threadfence_block();
            dd = vs.dead[g - 1];
        }
        // lane 0's left input at step s (nothing at step 0); the slot is read
        // unconditionally (it is in bounds) and the value selected
        auto input = [&](int s) -> float {
            const float v = ld_shared_volatile(rin_s + 4u * static_cast<unsigned>((s - 1) & (kGrpRing - 1)));
            return (s >= 2 && s - 1 < dd) ? v : INF;
        };
        // room: warp g+1 has read the entries these steps overwrite (step
        // s reuses the slot of step s - kGrpRing, read before warp g+1
        // completed step s - kGrpRing + 1)
        if (!last && !wait([&] { return vs.cons[g + 1] >= t_next - kGrpRing + 1; })) {
            out.status = 2;
            break;
        }
        bool skip = false;
        if (own_dead) {
            bool in_dead = !(lprev <= ub);   // lane 0: the diagonal of its first cell
#pragma unroll
            for (int i = 1; i <= CE; ++i) in_dead = in_dead && (i > ns || !(input(t + i) <= ub));
            skip = __shfl_sync(kFull, in_dead, 0);
        }
        float bmin_a = INF, bmin_b = INF;
        if (skip) {
#pragma unroll
            for (int k = 0; k < K; ++k) prv[k] = INF;
            lout = INF;
            lprev = INF;
            if (lane < ns) vs.ring[g][(t + 1 + lane) & (kGrpRing - 1)] = INF;
        } else if (t_next < t_fin) {
            // CE steps, no capture; lane 0's input and each lane's row read
            // one step ahead
            float nxt = input(t + 1);
            float xn = row_at(t + 1 - b);
#pragma unroll
            for (int s = 1; s <= CE; ++s) {
                const float cur = nxt;
                const float x = xn;
                if (s < CE) {
                    nxt = input(t + s + 1);
                    xn = row_at(t + s + 1 - b);
                }
                const float up = __shfl_up_sync(kFull, lout, 1);
                cells(t + s - b, x, lane == 0 ? cur : up);
                put(t + s, lout);
                if (s == CE - 1) bmin_a = block_min();
                if (s == CE) bmin_b = block_min();
            }
            busy += rows_in(t, CE);
        } else {
            // the last steps of this warp; the warp holding the last column
            // captures cell (nr, nc) at its final step
            float fin = INF;
            for (int s = t + 1; s <= t_next; ++s) {
                const float in0 = input(s);
                const float up = __shfl_up_sync(kFull, lout, 1);
                cells(s - b, row_at(s - b), lane == 0 ? in0 : up);
                put(s, lout);
                if (last && s == t_fin && b == bm) {
#pragma unroll
                    for (int k = 0; k < K; ++k) fin = (k == km) ? prv[k] : fin;
                }
            }
            busy += rows_in(t, ns);
            if (last) out.dist = __shfl_sync(kFull, fin, bm & 31);
        }
        t = t_next;
        // publish this warp's entries up to step t and its progress
        __syncwarp();
        if (lane == 31) {
            __threadfence_block();
            vs.prog[g] = t;
        }
        if (lane == 0) vs.cons[g] = t;
        if (t == t_fin) {
            // past its last row: what it would still send feeds rows past nr only
            if (!last && lane == 31) vs.dead[g] = t + 1;
            out.steps = t;
            if (last && !(out.dist <= INF)) out.dist = INF;   // NaN (no path) is +inf
            break;
        }
        // check: the bound, then this warp's blocks at steps t - 1 and t
        ub = fminf(ub, __shfl_sync(kFull, BestSoFar::finish(ub_raw), 0));
        ub_raw = bsf.issue();
        const unsigned da = __ballot_sync(kFull, !(bmin_a <= ub));
        const unsigned db = __ballot_sync(kFull, !(bmin_b <= ub));
        own_dead = da == kFull && db == kFull;
        if (own_dead) {
            // inputs dead from step t - 1 on (the diagonal of the next step
            // included): dead for good from step t - 1
            int dd = 0;
            if (g > 0 && lane == 0) dd = vs.dead[g - 1];
            dd = __shfl_sync(kFull, dd, 0);
            if (dd <= t - 1) {
                if (lane == 31) vs.dead[g] = t - 1;
                out.dist = INF;
                out.steps = t;
                break;
            }
        }
        int ab = 0;
        if (lane == 0) ab = vs.abort_flag;
        if (__shfl_sync(kFull, ab, 0)) {
            out.status = 2;
            break;
        }
    }
    int bs = busy;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bs += __shfl_xor_sync(kFull, bs, o);
    out.busy = bs;
    return out;
}

}  // namespace eapdtw
