// Device-side tables of a batched search: many (query, reference) items in
// one launch sequence (eapdtw_search_batch).
//
// Work is cut into units that persistent warps take from one 64-bit counter
// per launch:
//  * seed units: the exact DTW of the sampled windows with the smallest
//    z-normalised Euclidean distance (they seed each item's k-best list);
//  * re-run units: single windows whose live region overflowed the warp's
//    window of blocks at the previous (narrower) level;
//  * tile units: 32 consecutive windows of one item, through the lower-bound
//    cascade and EAPrunedDTW.
// Items are grouped into classes by their first level (block width K) and
// band mode; a class launch serves the seed and tile units of its items and
// the re-run units its level receives.
#pragma once

#include <cstdint>

#include "common.cuh"
#include "eapdtw.h"
#include "search_kernel.cuh"

namespace eapdtw {

// Levels: K = 4, 8, 16, 32 with one window of 32 blocks, then the group
// wavefront with groups of 4 warps (queries up to 2048 points) or 8 (longer
// queries).  Before them, for unconstrained and wide-band items of up to 2048
// points, the elastic first level (launched before level 0).
constexpr int kBatchLevels = 6;
constexpr int kElLevel = 6;          // the elastic first level
constexpr int kElClasses = 4;        // band mode 0 / 1 x queries up to 1024 / 2048 points
constexpr int kElClass0 = 12;
constexpr int kElMaxM = 2048;
constexpr int kTileElastic = 1;      // the tuning table's first-level tile for the elastic level
constexpr int kBatchClasses = 12 + kElClasses;   // tile classes: first levels 0..3 x band modes 0..2, then the elastic ones
constexpr int kSeedClasses = 9;      // seed passes at levels 3, 4, 5 x band modes
constexpr int kRerunBuffers = 3;     // re-run lists of level L live in buffer L % 3
constexpr int kAllClasses = kBatchClasses + kSeedClasses;
constexpr int kBatchSeedBest = 32;   // sampled windows per item run through exact DTW
constexpr int kBatchSeedSamples = 4096;
constexpr int kBatchSlots = 64;      // k-best slots per item (k <= 64)
// Bits of an item's flags.
constexpr int kFlagLost = 1;         // an overflow entry did not fit a re-run list
constexpr int kFlagTimeout = 2;      // a device-side wait of the group level ran out
// Block width a level's band mode is chosen for: the one-warp levels' K, and
// 32 for the group levels (a band mode valid at K = 32 is valid at their 16).
__host__ __device__ constexpr int batch_level_K(int level) { return level < 4 ? (4 << level) : 32; }
// The widest level a query of m points needs (3 for m <= 1024).
__host__ __device__ constexpr int batch_last_level(int m) { return m <= 1024 ? 3 : (m <= 2048 ? 4 : 5); }

struct BatchItem {
    RefView ref;
    const float* zq;     // query slot arrays (global memory; see TileCtx)
    const float* uq;
    const float* lq;
    const float* zqo;
    const int* ord;
    int64_t nw;          // windows n - m + 1
    int64_t win0;        // this launch sequence covers windows [win0, win0 + nwin)
    int64_t nwin;
    int64_t seed_off;    // first sample of this item in the seed sample arrays
    int state;           // slot of the item's resident state (k-best list, seed bound, flags)
    int fresh;           // 1: the state starts from empty in this launch sequence
    int m, w, k, use_lb;
    int seed_ns;         // sampled windows (0: no seed)
    int check2;          // 1: the wavefront checks at twice its built-in interval (autotuner)
    int level0;          // first level
    int next_level[kBatchLevels + 1];  // level that re-runs windows overflowing level L (-1: none;
                                       // index kElLevel: the elastic first level)
    int next_band[kBatchLevels + 1];   // its band mode
    const float* eu;     // sparse-table level of the reference for LB_Keogh EC (see TileCtx)
    const float* el;
    int ec_w, ec_d;
};

struct BatchClass {
    int item_off;   // citems[item_off .. item_off + nitems) are the items of the class
    int nitems;
    // cprefix[item_off + cls .. item_off + cls + nitems]: tile prefix over the class's items
};

struct QuerySlot {
    const float* Q;  // raw query (caller's device memory)
    int m, w;
    int off;         // float offset of the slot's arrays in the query arena
    int pad;
};

// Fixed device addresses of a context's batch arena.
struct BatchDev {
    const int* nitems;           // [1]
    const int* nslots;           // [1]
    const int* kstride;          // [1] result row length
    const BatchItem* items;      // [cap_items]
    const BatchClass* classes;   // [kAllClasses]
    const int* citems;           // [2 * cap_items]: tile classes, then seed classes
    const int64_t* cprefix;      // [cap_items + kBatchClasses]
    const int64_t* sprefix;      // [cap_items + 1] seed sample prefix
    const QuerySlot* qslots;     // [cap_slots]
    float* qarena;               // 5 arrays of mp floats per slot (ord stored as int)
    int* qbad;                   // [cap_slots] non-finite query values
    // resident per-state arrays (indexed by BatchItem::state)
    unsigned long long* slots;   // [cap_states * kBatchSlots]
    float* ub_seed;              // [cap_states]
    int* nbest;                  // [cap_states]
    long long* best;             // [cap_states * kBatchSeedBest]
    int* flags;                  // [cap_states] kFlagLost | kFlagTimeout
    unsigned long long* cost;    // [cap_states] SM clock cycles the warps spent on the state's
                                 // work units in this launch sequence (the serving loop's cost estimate)
    float* seed_ed;              // [cap_samples]
    int* seed_idx;               // [cap_samples]
    int64_t* res_idx;            // [cap_items * kstride]
    double* res_dist;
};

// One class launch of level `level` and band mode `band`.
struct BatchLaunch {
    BatchDev D;
    int level;
    int band;
    int cls;                    // class of items whose first level this is (-1: none)
    int scls;                   // seed class whose seed windows this launch runs (-1: none)
    const long long* rr_in;     // re-run entries (item << 32 | window) for this level and band
    const int* rr_in_count;
    long long* rr;              // every re-run list: rr + (buffer * 3 + band) * rr_cap
    int* rr_count;              // [kRerunBuffers * 3]
    int rr_cap;
    unsigned long long* work;   // unit counter of this launch
    unsigned long long* counters;
    float lb_scale;
};

// Persistent batch kernel of the one-warp levels: the cascade and wavefront
// of process_tile, the windows and the query read from global memory through
// L1 (items differ in length).  A seed launch (scls >= 0) runs the seed
// windows of its class, before any tile: their exact distances tighten each
// item's bound, as the one-query search's seed pass does.  It runs at the
// item's widest level, where no live region overflows (K = 32 here for
// queries of up to 1024 points; the group levels run the longer ones).
template <int K, int BAND>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, mode_min_blocks(K, BAND, 0))
batch_kernel(const BatchLaunch L) {
    __shared__ unsigned long long s_cnt[kNumCounters];
    if (threadIdx.x < kNumCounters) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int cn = 0, c0 = 0, sn = 0, s0 = 0;
    int64_t ntiles = 0;
    const int64_t* P = nullptr;
    if (L.cls >= 0) {
        const BatchClass c = L.D.classes[L.cls];
        cn = c.nitems;
        c0 = c.item_off;
        P = L.D.cprefix + c.item_off + L.cls;
        ntiles = P[cn];
    }
    if (L.scls >= 0) {
        const BatchClass c = L.D.classes[L.scls];
        sn = c.nitems;
        s0 = c.item_off;
    }
    const int64_t nseed = static_cast<int64_t>(sn) * kBatchSeedBest;
    int nrr = 0;
    if (L.rr_in) {
        const int c = *L.rr_in_count;
        nrr = c < L.rr_cap ? c : L.rr_cap;
    }
    auto count = [&](int c, unsigned long long v) { if (v) atomicAdd(s_cnt + c, v); };
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(L.work, 1ull);
        u = __shfl_sync(kFull, u, 0);
        int item;
        int64_t i0;
        bool list;
        int nl = 1;
        const int64_t su = static_cast<int64_t>(u);
        if (su < nseed) {
            const int j = static_cast<int>(su / kBatchSeedBest);
            const int s = static_cast<int>(su % kBatchSeedBest);
            item = L.D.citems[s0 + j];
            const int st = L.D.items[item].state;
            if (s >= L.D.nbest[st]) continue;
            i0 = L.D.best[static_cast<int64_t>(st) * kBatchSeedBest + s] & 0xffffffffll;
            list = true;
        } else if (su < nseed + nrr) {
            const long long e = L.rr_in[su - nseed];
            item = static_cast<int>(e >> 32);
            i0 = e & 0xffffffffll;
            list = true;
        } else {
            const int64_t t = su - nseed - nrr;
            if (t >= ntiles) break;
            int lo = 0, hi = cn;  // P[lo] <= t < P[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (P[mid] <= t) lo = mid;
                else hi = mid;
            }
            item = L.D.citems[c0 + lo];
            i0 = L.D.items[item].win0 + (t - P[lo]) * 32;
            list = false;
        }
        const BatchItem& it = L.D.items[item];
        if (!list) {
            const int64_t end = it.win0 + it.nwin;
            nl = static_cast<int>(end - i0 < 32 ? end - i0 : 32);
        }
        TileCtx C;
        C.ref = it.ref;
        C.zq = it.zq;
        C.uq = it.uq;
        C.lq = it.lq;
        C.zqo = it.zqo;
        C.ord = it.ord;
        C.m = it.m;
        C.w = it.w;
        C.use_lb = it.use_lb;
        C.use_ec = it.use_lb;
        C.ur = nullptr;
        C.lr = nullptr;
        C.eu = it.eu;
        C.el = it.el;
        C.ec_w = it.ec_w;
        C.ec_d = it.ec_d;
        C.lb_scale = L.lb_scale;
        C.bsf = BestSoFar{L.D.slots + static_cast<int64_t>(it.state) * kBatchSlots, L.D.ub_seed + it.state, it.k, 0,
                          0.0f};
        C.nw = it.nw;
        const bool seed = su < nseed;
        const int nx = seed ? -1 : it.next_level[L.level];
        const int rl = nx >= 0 ? (nx % kRerunBuffers) * 3 + it.next_band[L.level] : -1;
        C.ovf_out = rl >= 0 ? L.rr + static_cast<int64_t>(rl) * L.rr_cap : nullptr;
        C.ovf_out_count = rl >= 0 ? L.rr_count + rl : nullptr;
        C.ovf_cap = rl >= 0 ? L.rr_cap : 0;
        C.tag = static_cast<long long>(item) << 32;
        C.cbw = nullptr;
        C.zr = nullptr;
        C.check2 = it.check2;
        C.lost = seed ? nullptr : L.D.flags + it.state;   // a seed is only a hint: nothing is lost
        C.dbg = nullptr;
        const long long c0 = clock64();
        process_tile<K, BAND, true, 0, false, 2>(C, nullptr, list, i0, nl, count);
        if (lane == 0) atomicAdd(L.D.cost + it.state, static_cast<unsigned long long>(clock64() - c0));
    }
    __syncthreads();
    if (threadIdx.x < 10 && s_cnt[threadIdx.x]) atomicAdd(L.counters + threadIdx.x, s_cnt[threadIdx.x]);
}

}  // namespace eapdtw
