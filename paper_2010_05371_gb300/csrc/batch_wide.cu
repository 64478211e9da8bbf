// The batch kernel at the widest levels (4: queries of up to 2048 points, 5:
// up to 4096): single windows (seed windows and re-runs of candidates whose
// live region overflowed K = 32) run by groups of warps of one block
// (dtw_group.cuh).  Level 4 forms groups of 4 warps, level 5 one group of 8;
// an item of m points uses the first group_warps(m) warps of its group.
//
// Compiled once per (level, band mode) pair with EAPDTW_UNIT_LEVEL and
// EAPDTW_UNIT_BAND defined, and once without them for the dispatcher (see
// build.py).
#include "batch.cuh"
#include "dtw_group.cuh"
#include "kernels.h"

namespace eapdtw {

// Warps per group at the widest levels.
__host__ __device__ constexpr int batch_group_warps(int level) { return level == 4 ? 4 : 8; }

template <int BAND, int GW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, EAPDTW_MINB_GROUP) batch_group_kernel(const BatchLaunch L) {
    constexpr int kGroups = kWarpsPerBlock / GW;
    constexpr int kTile = GW * kGrpCols;   // the longest window a group runs
    __shared__ GroupSync s_gs[kGroups];
    __shared__ __align__(16) float s_win[kGroups][kTile];   // each group's window, staged once per candidate
    __shared__ unsigned long long s_cnt[kNumCounters];
    if (threadIdx.x < kNumCounters) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gi = warp / GW;
    const int g = warp - gi * GW;
    int sn = 0, s0 = 0;
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
    const int64_t nunits = nseed + nrr;
    auto count = [&](int c, unsigned long long v) { if (v) atomicAdd(s_cnt + c, v); };
    GroupSync& gs = s_gs[gi];
    volatile GroupSync& vs = gs;
    if (g == 0 && lane == 0) {
        group_reset(gs);
        vs.abort_flag = 0;
    }
    for (;;) {
        if (g == 0 && lane == 0)
            vs.unit = vs.abort_flag ? nunits : static_cast<long long>(atomicAdd(L.work, 1ull));
        group_bar(gi, GW);
        const int64_t su = vs.unit;   // the same reading on every warp of the group
        if (su >= nunits) break;
        int item;
        int64_t i0;
        bool run = true;
        if (su < nseed) {
            const int j = static_cast<int>(su / kBatchSeedBest);
            const int s = static_cast<int>(su % kBatchSeedBest);
            item = L.D.citems[s0 + j];
            const int st = L.D.items[item].state;
            run = s < L.D.nbest[st];
            i0 = run ? (L.D.best[static_cast<int64_t>(st) * kBatchSeedBest + s] & 0xffffffffll) : 0;
        } else {
            const long long e = L.rr_in[su - nseed];
            item = static_cast<int>(e >> 32);
            i0 = e & 0xffffffffll;
        }
        const BatchItem& it = L.D.items[item];
        const int ge = group_warps(it.m);
        const bool go = run && ge <= GW && it.m <= kTile;
        if (go) {   // the window's points into the group's tile, by all its warps
            const float* src = it.ref.R + i0;
            for (int j = g * 32 + lane; j < it.m; j += GW * 32) s_win[gi][j] = __ldg(src + j);
        }
        group_bar(gi, GW);
        if (go && g < ge) {
            const long long c0 = clock64();
            const BestSoFar bsf{L.D.slots + static_cast<int64_t>(it.state) * kBatchSlots, L.D.ub_seed + it.state,
                                it.k, 0, 0.0f};
            const float* x = s_win[gi];
            float a = 0.0f, cw = 0.0f, isd = 0.0f;
            if (lane == 0) window_coeffs(it.ref, i0, it.m, x, a, cw, isd);
            a = __shfl_sync(kFull, a, 0);
            cw = __shfl_sync(kFull, cw, 0);
            isd = __shfl_sync(kFull, isd, 0);
            const float ub = __shfl_sync(kFull, bsf.load(), 0);
            const DtwOut o = dtw_group<BAND, kCostSquared>(gs, g, x, a, cw, isd, it.zq, it.m, it.m, it.w, bsf, ub,
                                                           L.D.flags + it.state, kFlagTimeout);
            if (lane == 0) {
                count(kCntCells, static_cast<unsigned long long>(o.busy) * kGrpK);
                if (g == ge - 1 && o.status == 0) {
                    count(kCntSteps, static_cast<unsigned long long>(o.steps));
                    const float ubn = bsf.load();
                    if (o.dist <= ubn && o.dist < f_inf()) {
                        bsf.insert(o.dist, static_cast<uint32_t>(i0));
                        count(kCntCompleted, 1);
                    } else {
                        count(kCntAbandoned, 1);
                    }
                }
                atomicAdd(L.D.cost + it.state, static_cast<unsigned long long>(clock64() - c0));
            }
        }
        group_bar(gi, GW);   // every warp is done with the group's state
        if (g == 0 && lane == 0) group_reset(gs);
    }
    __syncthreads();
    if (threadIdx.x < 10 && s_cnt[threadIdx.x]) atomicAdd(L.counters + threadIdx.x, s_cnt[threadIdx.x]);
}

template <int BAND, int LEVEL>
cudaError_t launch_bwide_unit(const BatchLaunch& args, int blocks, cudaStream_t s) {
    batch_group_kernel<BAND, batch_group_warps(LEVEL)><<<blocks, kWarpsPerBlock * 32, 0, s>>>(args);
    return cudaGetLastError();
}

template <int BAND, int LEVEL>
int blocks_bwide_unit() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_group_kernel<BAND, batch_group_warps(LEVEL)>,
                                                      kWarpsPerBlock * 32, 0) != cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}

#if defined(EAPDTW_UNIT_LEVEL) && defined(EAPDTW_UNIT_BAND)

template cudaError_t launch_bwide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_LEVEL>(const BatchLaunch&, int, cudaStream_t);
template int blocks_bwide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_LEVEL>();

#else

#define EAPDTW_BWIDE_EXTERN(B, LV)                                                                 \
    extern template cudaError_t launch_bwide_unit<B, LV>(const BatchLaunch&, int, cudaStream_t); \
    extern template int blocks_bwide_unit<B, LV>();
EAPDTW_BWIDE_EXTERN(0, 4)
EAPDTW_BWIDE_EXTERN(1, 4)
EAPDTW_BWIDE_EXTERN(2, 4)
EAPDTW_BWIDE_EXTERN(0, 5)
EAPDTW_BWIDE_EXTERN(1, 5)
EAPDTW_BWIDE_EXTERN(2, 5)
#undef EAPDTW_BWIDE_EXTERN

namespace {
template <int LEVEL>
cudaError_t launch_l(int band, const BatchLaunch& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_bwide_unit<0, LEVEL>(args, blocks, s);
    if (band == 1) return launch_bwide_unit<1, LEVEL>(args, blocks, s);
    return launch_bwide_unit<2, LEVEL>(args, blocks, s);
}
template <int LEVEL>
int blocks_l(int band) {
    if (band == 0) return blocks_bwide_unit<0, LEVEL>();
    if (band == 1) return blocks_bwide_unit<1, LEVEL>();
    return blocks_bwide_unit<2, LEVEL>();
}
}  // namespace

cudaError_t launch_batch_wide(int level, int band, const BatchLaunch& args, int blocks, cudaStream_t s) {
    return level == 4 ? launch_l<4>(band, args, blocks, s) : launch_l<5>(band, args, blocks, s);
}

int batch_blocks_wide(int level, int band) { return level == 4 ? blocks_l<4>(band) : blocks_l<5>(band); }

// The group kernels use static shared memory only.
cudaError_t batch_attributes_wide() { return cudaSuccess; }

#endif

}  // namespace eapdtw
