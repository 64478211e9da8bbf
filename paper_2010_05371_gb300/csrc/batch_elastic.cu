// The batch's elastic first level: tiles of the items whose first level is
// the narrow-block elastic wavefront (dtw_elastic.cuh), unconstrained
// (BAND = 0) or banded with the hand-over of candidates that near the band's
// edges (BAND = 1), through the lower-bound cascade (process_tile, windows and
// query read through L1).  Overflows and hand-overs go to the re-run list of
// each item's next level.  MMAX: the longest query of the class (1024 or
// 2048); each warp's row buffer in dynamic shared memory is sized for it.
// Two resident blocks per SM: at three (80 registers) the cascade's and the
// batch's per-item state spill several hundred bytes per thread.
#include "batch.cuh"
#include "kernels.h"

namespace eapdtw {

template <int MMAX>
__host__ __device__ constexpr size_t batch_elastic_smem() {
    return sizeof(float) * kWarpsPerBlock * static_cast<size_t>(elastic_row_floats(MMAX));
}

template <int BAND, int MMAX>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2) batch_elastic_kernel(const BatchLaunch L) {
    extern __shared__ __align__(16) float s_rows[];
    __shared__ unsigned long long s_cnt[kNumCounters];
    constexpr int kRowF = elastic_row_floats(MMAX);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float* rows = s_rows + warp * kRowF;
    if (threadIdx.x < kNumCounters) s_cnt[threadIdx.x] = 0;
    for (int j = lane; j < kElPadRows; j += 32) rows[j] = f_nan();   // the pad before the first row
    __syncthreads();
    const BatchClass c = L.D.classes[L.cls];
    const int64_t* P = L.D.cprefix + c.item_off + L.cls;
    const int64_t ntiles = P[c.nitems];
    auto count = [&](int k, unsigned long long v) { if (v) atomicAdd(s_cnt + k, v); };
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(L.work, 1ull);
        u = __shfl_sync(kFull, u, 0);
        const int64_t t = static_cast<int64_t>(u);
        if (t >= ntiles) break;
        int lo = 0, hi = c.nitems;   // P[lo] <= t < P[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (P[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int item = L.D.citems[c.item_off + lo];
        const BatchItem& it = L.D.items[item];
        const int64_t i0 = it.win0 + (t - P[lo]) * 32;
        const int64_t end = it.win0 + it.nwin;
        const int nl = static_cast<int>(end - i0 < 32 ? end - i0 : 32);
        if (it.m > MMAX) {   // not planned (the class holds queries of up to MMAX points): run it alone
            if (lane == 0) atomicOr(L.D.flags + it.state, kFlagLost);
            continue;
        }
        // NaN rows after this item's last row (the rows are written per survivor)
        __syncwarp();
        for (int j = lane; j < kElPadRows + 4; j += 32) rows[kElPadRows + it.m + j] = f_nan();
        __syncwarp();
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
        const int nx = it.next_level[kElLevel];
        const int rl = nx >= 0 ? (nx % kRerunBuffers) * 3 + it.next_band[kElLevel] : -1;
        C.ovf_out = rl >= 0 ? L.rr + static_cast<int64_t>(rl) * L.rr_cap : nullptr;
        C.ovf_out_count = rl >= 0 ? L.rr_count + rl : nullptr;
        C.ovf_cap = rl >= 0 ? L.rr_cap : 0;
        C.tag = static_cast<long long>(item) << 32;
        C.lost = L.D.flags + it.state;
        C.cbw = nullptr;
        C.zr = rows + kElPadRows;
        C.check2 = 0;
        C.dbg = nullptr;
        const long long c0 = clock64();
        process_tile<kElK, BAND, true, 0, false, 2, false, 0, true, false>(C, nullptr, false, i0, nl, count);
        if (lane == 0) atomicAdd(L.D.cost + it.state, static_cast<unsigned long long>(clock64() - c0));
    }
    __syncthreads();
    if (threadIdx.x < 10 && s_cnt[threadIdx.x]) atomicAdd(L.counters + threadIdx.x, s_cnt[threadIdx.x]);
}

namespace {
template <int BAND, int MMAX>
cudaError_t launch_e(const BatchLaunch& args, int blocks, cudaStream_t s) {
    batch_elastic_kernel<BAND, MMAX><<<blocks, kWarpsPerBlock * 32, batch_elastic_smem<MMAX>(), s>>>(args);
    return cudaGetLastError();
}
template <int BAND, int MMAX>
int blocks_e() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_elastic_kernel<BAND, MMAX>, kWarpsPerBlock * 32,
                                                      batch_elastic_smem<MMAX>()) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}
template <int BAND, int MMAX>
cudaError_t attributes_e() {
    return cudaFuncSetAttribute(batch_elastic_kernel<BAND, MMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(batch_elastic_smem<MMAX>()));
}
}  // namespace

// e = 2 x (queries longer than 1024 points) + band mode (0, 1): the class
// kElClass0 + e.
cudaError_t launch_batch_elastic(int e, const BatchLaunch& args, int blocks, cudaStream_t s) {
    switch (e) {
        case 0: return launch_e<0, 1024>(args, blocks, s);
        case 1: return launch_e<1, 1024>(args, blocks, s);
        case 2: return launch_e<0, kElMaxM>(args, blocks, s);
        default: return launch_e<1, kElMaxM>(args, blocks, s);
    }
}

int batch_blocks_elastic(int e) {
    switch (e) {
        case 0: return blocks_e<0, 1024>();
        case 1: return blocks_e<1, 1024>();
        case 2: return blocks_e<0, kElMaxM>();
        default: return blocks_e<1, kElMaxM>();
    }
}

cudaError_t batch_attributes_elastic() {
    cudaError_t e = attributes_e<0, 1024>();
    if (e == cudaSuccess) e = attributes_e<1, 1024>();
    if (e == cudaSuccess) e = attributes_e<0, kElMaxM>();
    if (e == cudaSuccess) e = attributes_e<1, kElMaxM>();
    return e;
}

}  // namespace eapdtw
