// Subsequence search kernel: the UCR-Suite loop of Section 5 run over all
// candidate windows in parallel (sm_103a).
//
// Persistent warps take tiles of 32 consecutive windows from a global counter.
//  1. The warp streams R[i0 .. i0+31+m) into its shared-memory tile with
//     coalesced 16-byte loads.
//  2. Lane l owns window i0 + l: window statistics from the chunk-anchored
//     prefix sums, then LB_Kim (first/last points), LB_Keogh EQ (window vs
//     query envelope) and LB_Keogh EC (query vs the window's normalised
//     reference envelope), each skipping the window if above the current
//     upper bound (Section 2.2).  Terms are visited in decreasing |zq| order
//     with early exit every 8 terms.
//  3. Surviving windows are run one after another by the whole warp through
//     the EAPrunedDTW wavefront (dtw_wavefront.cuh) against the current k-th
//     best distance, re-read every few steps; a value <= ub enters the k-best
//     list by atomicMin.
// List mode (ovf_in != nullptr) re-runs single windows whose live region did
// not fit the window of blocks of a narrower launch.
#pragma once

#include "common.cuh"
#include "dtw_wavefront.cuh"
#include "dtw_elastic.cuh"

namespace eapdtw {

constexpr int kWarpsPerBlock = 8;
// 1: the elastic wavefront's on-demand row fill keeps its inputs in shared
// memory instead of registers (a compile-time knob for tuning experiments).
// Measured on the large workload's unconstrained searches: spills fell from
// 84 / 152 bytes (stores / loads) to 52 / 88, and the search from 65.8 to
// 65.3 ms.
#ifndef EAPDTW_ELASTIC_FILL_SMEM
#define EAPDTW_ELASTIC_FILL_SMEM 1
#endif
// LB_Keogh terms per early-exit test (a compile-time knob for tuning
// experiments; the query arrays are padded to a multiple of it with neutral
// terms).  A window is pruned iff its whole sum exceeds the bound, whatever
// the spacing of the tests, so the spacing changes work, not results.
#ifndef EAPDTW_LB_UNROLL
#define EAPDTW_LB_UNROLL 8
#endif
constexpr int kLbUnroll = EAPDTW_LB_UNROLL;

struct SearchArgs {
    RefView ref;
    QueryView q;
    const float* ur;   // reference envelope (upper) over +-w_env, raw values [n]
    const float* lr;   // lower
    BestSoFar bsf;
    int64_t nw;        // number of windows n - m + 1
    int w;             // warping window
    int use_lb;
    float lb_scale;    // prune iff lb > ub * lb_scale (lb_scale = 1 + slack)
    int* work_counter; // tile / list-item counter
    unsigned long long* counters;
    long long* ovf_out;  // windows whose live region overflowed (re-run wider)
    int* ovf_out_count;
    int ovf_cap;
    const long long* ovf_in;  // list mode input
    const int* ovf_in_count;
    int ovf_in_cap;           // entries beyond the capacity were dropped by the producer
    float* cb;                // upper-bound tightening scratch: cb_stride floats per warp of the grid, or nullptr
    int cb_stride;
    int64_t tile_lo, tile_hi; // tile mode: tiles [tile_lo, tile_hi) of 32 windows (tile_hi 0: all)
    // Gate (or nullptr): the launch runs only if (*gate_count > gate_threshold) == gate_wider,
    // a decision every block reads from device memory written by an earlier launch.
    const int* gate_count;
    int gate_threshold;
    int gate_wider;
    int* dbg;                 // device self-check record (EAPDTW_DEVICE_CHECKS builds only)
    int* err;                 // set to 1 when a device-side wait ran out (the group level), or nullptr
};

__host__ __device__ inline int query_pad(int m) { return (m + kLbUnroll - 1) / kLbUnroll * kLbUnroll; }
__host__ __device__ inline int tile_floats(int m) { return (m + 31 + 3) / 4 * 4 + 4; }

// Warps per block: up to kWarpsPerBlock, fewer when long queries fill shared memory.
__host__ inline int search_warps(int m) {
    const size_t budget = 227 * 1024;
    const size_t q = sizeof(float) * 5 * static_cast<size_t>(query_pad(m));
    const size_t t = sizeof(float) * static_cast<size_t>(tile_floats(m));
    if (q + t > budget) return 0;
    size_t w = (budget - q) / t;
    return static_cast<int>(w < kWarpsPerBlock ? w : kWarpsPerBlock);
}

__host__ inline size_t search_smem_bytes(int m) {
    const int mp = query_pad(m);
    return sizeof(float) * (5 * static_cast<size_t>(mp) + search_warps(m) * static_cast<size_t>(tile_floats(m)));
}

// Everything one work item needs: where the reference, the query and the
// best-so-far bound live.  The query arrays may be in shared memory (one
// query per launch) or in global memory (a batch of queries).
struct TileCtx {
    RefView ref;
    const float* zq;      // [>= m] z-normalised query (NaN past m)
    const float* uq;      // [mp] LB order
    const float* lq;
    const float* zqo;
    const int* ord;
    int m;
    int w;
    int use_lb;           // LB_Kim and LB_Keogh EQ
    int use_ec;           // LB_Keogh EC
    const float* ur;      // envelope arrays U[t], L[t] of R over +-w (ECM = 1)
    const float* lr;
    const float* eu;      // sparse-table level of running maxima / minima (ECM = 2): eu[t] =
    const float* el;      // max R[t .. t + 2^p), clipped at the end; U[t] = max(eu[t - ec_w], eu[t + ec_d])
    int ec_w;             // envelope radius
    int ec_d;             // ec_w - 2^p + 1, with 2^p <= 2 ec_w + 1 < 2^(p+1)
    float lb_scale;
    BestSoFar bsf;
    int64_t nw;
    long long* ovf_out;   // overflow list: entries (tag | window)
    int* ovf_out_count;
    int ovf_cap;
    long long tag;        // high bits of the overflow entries (batch item << 32)
    int* lost;            // set to 1 when an overflow entry did not fit the list (or nullptr)
    float* cbw;           // this warp's scratch for upper-bound tightening (>= m + 1 floats), or nullptr
    float* zr;            // elastic wavefront: this warp's row buffer (row 1 at zr[0], NaN pads around)
    int check2;           // one-window wavefront: 1 checks at twice its built-in interval (the autotuner's choice)
    int* dbg;
};

// Suffix sums of a window's LB_Keogh EQ terms by position, cb[r] = sum of the
// terms of rows r+1..m (1-based; cb[m] = 0), into the warp's scratch: a row
// costs at least its term on any warping path, so cb[r] bounds the cost still
// to come after row r (upper bound tightening, see dtw_wavefront.cuh).
__device__ __forceinline__ void tightening_terms(const TileCtx& C, const float* x, float a, float cw, float isd) {
    const int lane = threadIdx.x & 31;
    const int m = C.m;
    float* cb = C.cbw;
    for (int p = lane; p < m; p += 32) {
        const int j = C.ord[p];
        const float z = znorm1(x[j], a, cw, isd);
        const float e = fmaxf(fmaxf(__fsub_rn(z, C.uq[p]), __fsub_rn(C.lq[p], z)), 0.0f);
        cb[j] = __fmul_rn(e, e);
    }
    __syncwarp();
    // lane l owns positions [l S, (l + 1) S): suffix sums inside, then the
    // totals of the lanes to its right
    const int S = (m + 31) >> 5;
    const int lo = lane * S;
    const int hi = lo + S < m ? lo + S : m;
    float acc = 0.0f;
    for (int j = hi - 1; j >= lo; --j) {
        acc = __fadd_rn(acc, cb[j]);
        cb[j] = acc;
    }
    float v = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float u = __shfl_down_sync(kFull, v, o);
        if (lane + o < 32) v = __fadd_rn(v, u);
    }
    float add = __shfl_down_sync(kFull, v, 1);
    if (lane == 31) add = 0.0f;
    for (int j = lo; j < hi; ++j) cb[j] = __fadd_rn(cb[j], add);
    // cb[j] now sums the terms of positions j..m-1, i.e. of rows j+1..m
    if (lane == 0) cb[m] = 0.0f;
    __syncwarp();
}

// The first half of process_tile: per-lane window statistics (a, cw, isd),
// the lower-bound cascade (lb: the largest bound computed) with its counts,
// and the corner check.  The tile's points are at s_r (window lane at
// s_r + lane; list mode: the single window at s_r).  Returns whether this
// lane's window is still alive.  All 32 lanes call it.
template <int BAND, bool LB, int ECM, int COST, typename CountF>
__device__ __forceinline__ bool tile_lanes(const TileCtx& C, const float* s_r, bool list_mode, int64_t i0, int nlanes,
                                           CountF count, float& a, float& cw, float& isd, float& lb) {
    const int lane = threadIdx.x & 31;
    const int m = C.m;
    const int mp = query_pad(m);
    (void)mp;
    // ---- per-lane window statistics and lower bounds ----------------------
    const int my = list_mode ? 0 : lane;
    const bool valid = lane < nlanes || list_mode;
    const int64_t i = i0 + my;
    a = 0.0f;
    cw = 0.0f;
    isd = 0.0f;
    if (valid) window_coeffs(C.ref, i, m, s_r + my, a, cw, isd);
    lb = 0.0f;
    bool alive = valid && (!list_mode || lane == 0);
    int why = 0;  // 1, 2, 3: pruned by LB_Kim, LB_Keogh EQ, LB_Keogh EC
    if (LB && C.use_lb && alive && !list_mode) {
        const float ub = C.bsf.load() * C.lb_scale;
        const float* x = s_r + my;
        const float z0 = znorm1(x[0], a, cw, isd);
        const float d0 = __fsub_rn(z0, C.zq[0]);
        float kim = __fmul_rn(d0, d0);
        if (m > 1) {
            const float dl = __fsub_rn(znorm1(x[m - 1], a, cw, isd), C.zq[m - 1]);
            kim = __fmaf_rn(dl, dl, kim);
        }
        lb = kim;
        if (kim > ub) {
            alive = false;
            why = 1;
        } else {
            // LB_Keogh EQ: the normalised window against the query envelope.
            float s = 0.0f;
            for (int p = 0; p < mp; p += kLbUnroll) {
#pragma unroll
                for (int u = 0; u < kLbUnroll; ++u) {
                    const int j = C.ord[p + u];
                    const float z = znorm1(EAPDTW_CHECK(C.dbg, j >= 0 && j < m, 22, j) ? x[j] : 0.0f, a, cw, isd);
                    const float e = fmaxf(fmaxf(__fsub_rn(z, C.uq[p + u]), __fsub_rn(C.lq[p + u], z)), 0.0f);
                    s = __fmaf_rn(e, e, s);
                }
                if (s > ub) break;
            }
            lb = fmaxf(lb, s);
            if (s > ub) {
                alive = false;
                why = 2;
            } else if (C.use_ec) {
                // LB_Keogh EC: the query against the window's envelope.
                float s2 = 0.0f;
                if (ECM == 1) {
                    const float* ur = C.ur + i;
                    const float* lr = C.lr + i;
                    for (int p = 0; p < mp; p += kLbUnroll) {
#pragma unroll
                        for (int u = 0; u < kLbUnroll; ++u) {
                            const int j = C.ord[p + u];
                            const bool okj = EAPDTW_CHECK(C.dbg, j >= 0 && j < m && i + j < C.ref.n, 23, j);
                            const float uu = znorm1(okj ? __ldg(ur + j) : 0.0f, a, cw, isd);
                            const float ll = znorm1(okj ? __ldg(lr + j) : 0.0f, a, cw, isd);
                            const float qv = C.zqo[p + u];
                            const float e = fmaxf(fmaxf(__fsub_rn(qv, uu), __fsub_rn(ll, qv)), 0.0f);
                            s2 = __fmaf_rn(e, e, s2);
                        }
                        if (s2 > ub) break;
                    }
                } else {
                    const int64_t nlast = C.ref.n - 1;
                    const bool interior = i - C.ec_w >= 0 && i + (m - 1) + C.ec_w <= nlast;
                    for (int p = 0; p < mp; p += kLbUnroll) {
#pragma unroll
                        for (int u = 0; u < kLbUnroll; ++u) {
                            const int j = C.ord[p + u];
                            int64_t x1 = i + j - C.ec_w, x2 = i + j + C.ec_d;
                            if (!interior) {
                                x1 = x1 < 0 ? 0 : (x1 > nlast ? nlast : x1);
                                x2 = x2 < 0 ? 0 : (x2 > nlast ? nlast : x2);
                            }
                            const float uu = znorm1(fmaxf(__ldg(C.eu + x1), __ldg(C.eu + x2)), a, cw, isd);
                            const float ll = znorm1(fminf(__ldg(C.el + x1), __ldg(C.el + x2)), a, cw, isd);
                            const float qv = C.zqo[p + u];
                            const float e = fmaxf(fmaxf(__fsub_rn(qv, uu), __fsub_rn(ll, qv)), 0.0f);
                            s2 = __fmaf_rn(e, e, s2);
                        }
                        if (s2 > ub) break;
                    }
                }
                lb = fmaxf(lb, s2);
                if (s2 > ub) {
                    alive = false;
                    why = 3;
                }
            }
        }
    }

    if (!list_mode) {
        const unsigned b1 = __ballot_sync(kFull, why == 1);
        const unsigned b2 = __ballot_sync(kFull, why == 2);
        const unsigned b3 = __ballot_sync(kFull, why == 3);
        if (lane == 0) {
            count(kCntWindows, nlanes);
            count(kCntKim, __popc(b1));
            count(kCntEq, __popc(b2));
            count(kCntEc, __popc(b3));
        }
    }

    // ---- EAPrunedDTW's first rows, lane by lane -----------------------------
    if (!list_mode && m >= kCorner && (BAND == 0 || C.w >= kCorner - 1)) {
        const unsigned am = __ballot_sync(kFull, alive);
        if (__popc(am) >= kCornerMinLanes) {
            bool ab = false;
            if (alive) ab = corner_dead<COST>(s_r + my, a, cw, isd, C.zq, C.bsf.load());
            const unsigned bab = __ballot_sync(kFull, ab);
            if (lane == 0) {
                count(kCntAbandoned, __popc(bab));
                count(kCntCells, static_cast<unsigned long long>(__popc(am)) * (kCorner * kCorner));
            }
            alive = alive && !ab;
        }
    }

    return alive;
}

// One work item on one warp: a tile of nlanes (<= 32) consecutive windows
// starting at i0, or (list_mode) the single window i0.  STAGE: copy the
// windows' points into the warp's shared-memory tile s_r first (one query per
// launch); otherwise read them from the reference in global memory through L1
// (a batch, whose query lengths differ from item to item).  Then the lower
// bounds lane by lane (tile mode), then EAPrunedDTW for every survivor on the
// whole warp.
// ECM: where LB_Keogh EC reads the reference envelope: 1 = arrays over the
// window's own radius; 2 = a sparse table of running maxima / minima (any
// radius, two reads per bound; windows within the radius of either end of the
// reference use a slightly wider envelope, which is still a valid bound).
// JW: 0 = the DP columns' query values held in registers, one window of 32
// blocks; JW >= 1 = the values streamed from C.zq at every step, JW windows of
// 32 blocks (fewer registers per thread, more resident warps).
// TIGHT: upper-bound tightening for the survivors (needs C.cbw and the lower
// bounds; compiled out otherwise).
// EL: run the survivors through the narrow-block elastic wavefront
// (dtw_elastic.cuh; K = kElK, C.zr padded as it needs; ELQPAD: C.zq padded
// with NaN and 16-byte aligned too).
template <int K, int BAND, bool LB, int JW, bool STAGE = true, int ECM = 1, bool TIGHT = false, int COST = 0,
          bool EL = false, bool ELQPAD = true, typename CountF>
__device__ __forceinline__ void process_tile(const TileCtx& C, float* s_r, bool list_mode, int64_t i0,
                                             int nlanes, CountF count) {
    const int lane = threadIdx.x & 31;
    const int m = C.m;
    const int mp = query_pad(m);
    const int len = nlanes - 1 + m;
    if (!EAPDTW_CHECK(C.dbg, i0 >= 0 && i0 + len <= C.ref.n, 21, len)) return;
    if (STAGE) {
        // R[i0 .. i0 + nlanes - 1 + m) into the warp's tile.
        if (!EAPDTW_CHECK(C.dbg, len <= tile_floats(m), 26, len)) return;
        if ((reinterpret_cast<uintptr_t>(C.ref.R + i0) & 15) == 0 && !list_mode) {
            const float4* src = reinterpret_cast<const float4*>(C.ref.R + i0);
            const int nv = len / 4;
            for (int v = lane; v < nv; v += 32) reinterpret_cast<float4*>(s_r)[v] = __ldg(src + v);
            for (int j = nv * 4 + lane; j < len; j += 32) s_r[j] = __ldg(C.ref.R + i0 + j);
        } else {
            for (int j = lane; j < len; j += 32) s_r[j] = __ldg(C.ref.R + i0 + j);
        }
        __syncwarp();
    } else {
        s_r = const_cast<float*>(C.ref.R + i0);
    }

    float a, cw, isd, lb;
    bool alive = tile_lanes<BAND, LB, ECM, COST>(C, s_r, list_mode, i0, nlanes, count, a, cw, isd, lb);

    // ---- EAPrunedDTW on the survivors, one warp per window ----------------
    unsigned mask = __ballot_sync(kFull, alive);
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const float a_s = __shfl_sync(kFull, a, src);
        const float cw_s = __shfl_sync(kFull, cw, src);
        const float isd_s = __shfl_sync(kFull, isd, src);
        const float lb_s = __shfl_sync(kFull, lb, src);
        const int off = list_mode ? 0 : src;
        const int64_t iw = i0 + off;
        // ub steers warp-wide control flow (the recheck below skips the DTW
        // for the whole warp): take lane 0's reading, because other warps
        // lower the bound concurrently and lanes that load it at slightly
        // different times may see different values.
        float ub = __shfl_sync(kFull, C.bsf.load(), 0);
#ifdef EAPDTW_DEVICE_CHECKS
        EAPDTW_CHECK(C.dbg, __shfl_sync(kFull, __float_as_int(ub), 0) == __float_as_int(ub), 24, 0);
        EAPDTW_CHECK(C.dbg, off >= 0 && off < 32 && iw < C.nw, 25, off);
#endif
        if (LB && C.use_lb && !list_mode && lb_s > ub * C.lb_scale) {
            if (lane == 0) count(kCntRecheck, 1);
            continue;
        }
        if (TIGHT) tightening_terms(C, s_r + off, a_s, cw_s, isd_s);
        DtwOut o;
        if constexpr (EL) {
            static_assert(BAND <= 1 && !TIGHT, "the elastic wavefront: unconstrained or banded, without tightening");
            // the window's z-normalised rows, negated, into the warp's buffer
            // as the wavefront reaches them (the same znorm1 values the other
            // wavefront computes row by row)
            const float* xw = s_r + off;
            float* zr = C.zr;
#if EAPDTW_ELASTIC_FILL_SMEM
            // the coefficients and the window pointer wait in shared memory
            // (elastic_fill_slot) while the wavefront runs, instead of
            // occupying registers through it
            if (lane == 0) {
                float* slot = zr + elastic_fill_slot(m);
                const unsigned long long pw = reinterpret_cast<unsigned long long>(xw);
                slot[0] = a_s;
                slot[1] = cw_s;
                slot[2] = isd_s;
                slot[4] = __uint_as_float(static_cast<unsigned>(pw));
                slot[5] = __uint_as_float(static_cast<unsigned>(pw >> 32));
            }
            __syncwarp();
            auto fill = [zr, m, lane](int r0, int r1) {
                const float* slot = zr + elastic_fill_slot(m);
                const float fa = slot[0], fcw = slot[1], fisd = slot[2];
                const unsigned long long pw = static_cast<unsigned long long>(__float_as_uint(slot[4])) |
                                              (static_cast<unsigned long long>(__float_as_uint(slot[5])) << 32);
                const float* x = reinterpret_cast<const float*>(pw);
                for (int i = r0 + lane; i < r1; i += 32) zr[i] = -znorm1(x[i], fa, fcw, fisd);
                __syncwarp();
            };
#else
            auto fill = [&](int r0, int r1) {
                for (int i = r0 + lane; i < r1; i += 32) zr[i] = -znorm1(xw[i], a_s, cw_s, isd_s);
                __syncwarp();
            };
#endif
            o = dtw_elastic<kElJ, COST, (BAND != 0), ELQPAD>(C.zr, C.zq, m, m, C.bsf, ub, C.w, fill);
            __syncwarp();   // every lane is done with the rows before the next survivor's
        } else {
            constexpr int kJ = JW > 0 ? JW : dtw_windows(K, BAND);
            o = dtw_warp<K, BAND, kJ, (JW > 0), TIGHT, COST>(s_r + off, a_s, cw_s, isd_s, C.zq, m, m, C.w, C.bsf,
                                                             ub, C.dbg, TIGHT ? C.cbw : nullptr, C.check2);
        }
        if (lane == 0) {
            count(kCntSteps, static_cast<unsigned long long>(o.steps));
            count(kCntCells, static_cast<unsigned long long>(o.busy) * (EL ? kElCellsPerStep : K));
        }
        if (o.status != 0) {
            if (lane == 0) {
                count(kCntOverflow, 1);
                const int slot = C.ovf_out_count ? atomicAdd(C.ovf_out_count, 1) : C.ovf_cap;
                if (slot < C.ovf_cap) C.ovf_out[slot] = C.tag | static_cast<long long>(iw);
                else if (C.lost) atomicOr(C.lost, 1);
            }
            continue;
        }
        ub = __shfl_sync(kFull, C.bsf.load(), 0);
        if (o.dist <= ub && o.dist < f_inf()) {
            if (lane == 0) {
                C.bsf.insert(o.dist, static_cast<uint32_t>(iw));
                count(kCntCompleted, 1);
            }
        } else if (lane == 0) {
            count(kCntAbandoned, 1);
        }
    }
    __syncwarp();
}

// Resident blocks per SM the register allocation is sized for (registers per
// thread <= 65536 / (256 * blocks)): the DP row takes 2K registers per lane.
#ifndef EAPDTW_MINB16
#define EAPDTW_MINB16 3
#endif
__host__ __device__ constexpr int search_min_blocks(int K, int BAND) {
    return dtw_windows(K, BAND) > 1 ? (K <= 4 ? 3 : 2) : (K <= 8 ? 4 : (K <= 16 ? EAPDTW_MINB16 : 2));
}
// Same for the streamed-column variants (JW windows).
#ifndef EAPDTW_MINB_CS1
#define EAPDTW_MINB_CS1 3
#endif
__host__ __device__ constexpr int mode_min_blocks(int K, int BAND, int JW) {
    return JW == 0 ? search_min_blocks(K, BAND) : (JW == 1 ? EAPDTW_MINB_CS1 : (JW == 2 ? 2 : 1));
}


// LB: compile the lower-bound cascade in (true) or out (false, the "nolb"
// variant and the list-mode re-runs); leaving it out frees registers.
// JW: 0 for the column values in registers (every level built by default);
// JW >= 1 streams them from the query in shared memory with JW windows of 32
// blocks (kept for tuning experiments through EAPDTW_KJW; the widest re-run
// level is the group wavefront, search_wide.cu).
// COST: see dtw_warp (the absolute cost is built for the no-lower-bound search only).
template <int K, int BAND, bool LB, int JW = 0, bool TIGHT = false, int COST = 0>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, mode_min_blocks(K, BAND, JW))
search_kernel(const SearchArgs A) {
    extern __shared__ __align__(16) float smem[];
    if (A.gate_count && ((*A.gate_count > A.gate_threshold) ? 1 : 0) != A.gate_wider) return;  // uniform
    const int m = A.q.m;
    const int mp = query_pad(m);
    float* s_zq = smem;
    float* s_uq = s_zq + mp;
    float* s_lq = s_uq + mp;
    float* s_zqo = s_lq + mp;
    int* s_ord = reinterpret_cast<int*>(s_zqo + mp);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float* s_r = reinterpret_cast<float*>(s_ord + mp) + warp * tile_floats(m);

    // block-level counters (shared 64-bit atomics), flushed to global at the end
    __shared__ unsigned long long s_cnt[10];
    if (threadIdx.x < 10) s_cnt[threadIdx.x] = 0;
    for (int j = threadIdx.x; j < mp; j += blockDim.x) {
        s_zq[j] = j < m ? A.q.zq[j] : f_nan();
        s_uq[j] = A.q.uq_o[j];
        s_lq[j] = A.q.lq_o[j];
        s_zqo[j] = A.q.zq_o[j];
        s_ord[j] = A.q.ord[j];
    }
    __syncthreads();

    const bool list_mode = A.ovf_in != nullptr;
    const int64_t tile_lo = A.tile_lo;
    const int64_t tile_hi = A.tile_hi > 0 ? A.tile_hi : (A.nw + 31) / 32;
    int64_t nitems = tile_hi - tile_lo;
    if (list_mode) {
        const int c = *A.ovf_in_count;
        nitems = c < A.ovf_in_cap ? c : A.ovf_in_cap;
    }
    auto count = [&](int c, unsigned long long v) { if (v) atomicAdd(s_cnt + c, v); };
    TileCtx C;
    C.ref = A.ref;
    C.zq = s_zq;
    C.uq = s_uq;
    C.lq = s_lq;
    C.zqo = s_zqo;
    C.ord = s_ord;
    C.m = m;
    C.w = A.w;
    C.use_lb = A.use_lb;
    C.use_ec = A.use_lb;
    C.ur = A.ur;
    C.lr = A.lr;
    C.eu = nullptr;
    C.el = nullptr;
    C.ec_w = 0;
    C.ec_d = 0;
    C.lb_scale = A.lb_scale;
    C.bsf = A.bsf;
    C.nw = A.nw;
    C.ovf_out = A.ovf_out;
    C.ovf_out_count = A.ovf_out_count;
    C.ovf_cap = A.ovf_cap;
    C.tag = 0;
    C.lost = nullptr;
    C.cbw = A.cb ? A.cb + (static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp) * A.cb_stride : nullptr;
    C.zr = nullptr;
    C.check2 = 0;
    C.dbg = A.dbg;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(A.work_counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= nitems) break;
        if (!list_mode) {
            const int64_t i0 = (tile_lo + item) * 32;
            process_tile<K, BAND, LB, JW, true, 1, TIGHT, COST>(C, s_r, false, i0,
                                                          static_cast<int>(A.nw - i0 < 32 ? A.nw - i0 : 32),
                                            count);
        } else {
            process_tile<K, BAND, LB, JW, true, 1, TIGHT, COST>(C, s_r, true, A.ovf_in[item] & 0xffffffffll, 1,
                                                                count);
        }
    }

    __syncthreads();
    if (threadIdx.x < 10 && s_cnt[threadIdx.x]) atomicAdd(A.counters + threadIdx.x, s_cnt[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// The first level with the narrow-block elastic wavefront (dtw_elastic.cuh):
// unconstrained (BAND = 0), or banded (BAND = 1: candidates whose live region
// may leave the band go to the banded levels).  Tile mode only (the re-runs
// of overflowed windows use search_kernel's list mode).  Windows are read through L1 from the
// reference (no staged tile); shared memory holds the query, NaN-padded past
// its last column, the lower-bound arrays when LB, and one row buffer per warp
// with its NaN pads.
__host__ __device__ inline int elastic_query_floats(int m, bool lb) {
    return elastic_col_floats(m) + (lb ? 4 * query_pad(m) : 0);
}
__host__ inline int elastic_warps(int m, bool lb) {
    const size_t budget = 227 * 1024 - 1024;   // the kernel's static shared memory fits in the rest
    const size_t q = sizeof(float) * static_cast<size_t>(elastic_query_floats(m, lb));
    const size_t r = sizeof(float) * static_cast<size_t>(elastic_row_floats(m));
    if (q + r > budget) return 0;
    const size_t w = (budget - q) / r;
    return static_cast<int>(w < kWarpsPerBlock ? w : kWarpsPerBlock);
}
__host__ inline size_t elastic_smem_bytes(int m, bool lb) {
    return sizeof(float) * (static_cast<size_t>(elastic_query_floats(m, lb)) +
                            static_cast<size_t>(elastic_warps(m, lb)) * elastic_row_floats(m));
}

#ifndef EAPDTW_MINB_ELASTIC
#define EAPDTW_MINB_ELASTIC 3
#endif
template <bool LB, int BAND, int COST>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, EAPDTW_MINB_ELASTIC) search_elastic_kernel(const SearchArgs A) {
    extern __shared__ __align__(16) float smem[];
    const int m = A.q.m;
    const int mp = query_pad(m);
    const int ecf = elastic_col_floats(m);
    const int erf = elastic_row_floats(m);
    float* s_zq = smem;
    float* s_uq = s_zq + ecf;
    float* s_lq = s_uq + (LB ? mp : 0);
    float* s_zqo = s_lq + (LB ? mp : 0);
    int* s_ord = reinterpret_cast<int*>(s_zqo + (LB ? mp : 0));
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float* s_rows = reinterpret_cast<float*>(s_ord + (LB ? mp : 0)) + warp * erf;

    __shared__ unsigned long long s_cnt[10];
    if (threadIdx.x < 10) s_cnt[threadIdx.x] = 0;
    for (int j = threadIdx.x; j < ecf; j += blockDim.x) s_zq[j] = j < m ? A.q.zq[j] : f_nan();
    if (LB) {
        for (int j = threadIdx.x; j < mp; j += blockDim.x) {
            s_uq[j] = A.q.uq_o[j];
            s_lq[j] = A.q.lq_o[j];
            s_zqo[j] = A.q.zq_o[j];
            s_ord[j] = A.q.ord[j];
        }
    }
    // the row buffer's NaN pads (its rows are written per survivor)
    for (int j = lane; j < erf; j += 32)
        if (j < kElPadRows || j >= kElPadRows + m) s_rows[j] = f_nan();
    __syncthreads();

    const int64_t tile_lo = A.tile_lo;
    const int64_t tile_hi = A.tile_hi > 0 ? A.tile_hi : (A.nw + 31) / 32;
    const int64_t nitems = tile_hi - tile_lo;
    auto count = [&](int c, unsigned long long v) { if (v) atomicAdd(s_cnt + c, v); };
    TileCtx C;
    C.ref = A.ref;
    C.zq = s_zq;
    C.uq = s_uq;
    C.lq = s_lq;
    C.zqo = s_zqo;
    C.ord = s_ord;
    C.m = m;
    C.w = A.w;
    C.use_lb = LB ? A.use_lb : 0;
    C.use_ec = LB ? A.use_lb : 0;
    C.ur = A.ur;
    C.lr = A.lr;
    C.eu = nullptr;
    C.el = nullptr;
    C.ec_w = 0;
    C.ec_d = 0;
    C.lb_scale = A.lb_scale;
    C.bsf = A.bsf;
    C.nw = A.nw;
    C.ovf_out = A.ovf_out;
    C.ovf_out_count = A.ovf_out_count;
    C.ovf_cap = A.ovf_cap;
    C.tag = 0;
    C.lost = nullptr;
    C.cbw = nullptr;
    C.zr = s_rows + kElPadRows;
    C.check2 = 0;
    C.dbg = A.dbg;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(A.work_counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= nitems) break;
        const int64_t i0 = (tile_lo + item) * 32;
        process_tile<kElK, BAND, LB, 0, false, 1, false, COST, true>(
            C, nullptr, false, i0, static_cast<int>(A.nw - i0 < 32 ? A.nw - i0 : 32), count);
    }

    __syncthreads();
    if (threadIdx.x < 10 && s_cnt[threadIdx.x]) atomicAdd(A.counters + threadIdx.x, s_cnt[threadIdx.x]);
}

}  // namespace eapdtw
