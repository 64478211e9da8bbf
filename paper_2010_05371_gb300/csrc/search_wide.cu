// The widest re-run level of the one-query search: candidates whose live
// region overflowed one warp's window at K = 32 (queries of more than 1024
// points), each run by a group of warps of one block (dtw_group.cuh: warp g
// owns columns 512 g + 1 .. 512 g + 512 in registers, the edge columns pass
// through shared memory).  List mode only: the re-run list of the previous
// level, or the seed windows.  Groups of group_warps(m) warps; the block's
// eight warps hold as many groups as fit (warps left over stay idle).
//
// Each (band mode, cost) pair is compiled as its own unit (build.py defines
// EAPDTW_UNIT_BAND and EAPDTW_UNIT_COST and this file is compiled once per
// pair, plus once without them for the dispatcher).
#include "dtw_group.cuh"
#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {

constexpr int kMaxGroupsPerBlock = kWarpsPerBlock / 2;

template <int BAND, int COST>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 3) search_group_kernel(const SearchArgs A) {
    __shared__ GroupSync s_gs[kMaxGroupsPerBlock];
    __shared__ unsigned long long s_cnt[10];
    if (threadIdx.x < 10) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int m = A.q.m;
    const int G = group_warps(m);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int gi = warp / G;
    const int g = warp - gi * G;
    auto count = [&](int c, unsigned long long v) { if (v) atomicAdd(s_cnt + c, v); };
    if (G >= 2 && G <= kGrpMaxWarps && gi < kWarpsPerBlock / G && gi < kMaxGroupsPerBlock) {
        GroupSync& gs = s_gs[gi];
        volatile GroupSync& vs = gs;
        const int c = *A.ovf_in_count;
        const int nitems = c < A.ovf_in_cap ? c : A.ovf_in_cap;
        if (g == 0 && lane == 0) {
            group_reset(gs);
            vs.abort_flag = 0;
        }
        for (;;) {
            if (g == 0 && lane == 0) vs.unit = vs.abort_flag ? nitems : atomicAdd(A.work_counter, 1);
            group_bar(gi, G);
            const int item = static_cast<int>(vs.unit);
            if (item >= nitems) break;   // the same reading on every warp of the group
            const int64_t iw = A.ovf_in[item] & 0xffffffffll;
            const float* x = A.ref.R + iw;
            float a = 0.0f, cw = 0.0f, isd = 0.0f;
            if (lane == 0) window_coeffs(A.ref, iw, m, x, a, cw, isd);
            a = __shfl_sync(kFull, a, 0);
            cw = __shfl_sync(kFull, cw, 0);
            isd = __shfl_sync(kFull, isd, 0);
            const float ub = __shfl_sync(kFull, A.bsf.load(), 0);
            const DtwOut o = dtw_group<BAND, COST>(gs, g, x, a, cw, isd, A.q.zq, m, m, A.w, A.bsf, ub, A.err, 1);
            if (lane == 0) count(kCntCells, static_cast<unsigned long long>(o.busy) * kGrpK);
            if (g == G - 1 && lane == 0 && o.status == 0) {
                count(kCntSteps, static_cast<unsigned long long>(o.steps));
                const float ubn = A.bsf.load();
                if (o.dist <= ubn && o.dist < f_inf()) {
                    A.bsf.insert(o.dist, static_cast<uint32_t>(iw));
                    count(kCntCompleted, 1);
                } else {
                    count(kCntAbandoned, 1);
                }
            }
            group_bar(gi, G);   // every warp is done with the group's state
            if (g == 0 && lane == 0) group_reset(gs);
        }
    }
    __syncthreads();
    if (threadIdx.x < 10 && s_cnt[threadIdx.x]) atomicAdd(A.counters + threadIdx.x, s_cnt[threadIdx.x]);
}

template <int BAND, int COST>
cudaError_t launch_wide_unit(const SearchArgs& args, int blocks, cudaStream_t s) {
    search_group_kernel<BAND, COST><<<blocks, kWarpsPerBlock * 32, 0, s>>>(args);
    return cudaGetLastError();
}

template <int BAND, int COST>
int blocks_wide_unit() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_group_kernel<BAND, COST>, kWarpsPerBlock * 32,
                                                      0) != cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}

#if defined(EAPDTW_UNIT_BAND) && defined(EAPDTW_UNIT_COST)

template cudaError_t launch_wide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_COST>(const SearchArgs&, int, cudaStream_t);
template int blocks_wide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_COST>();

#else

#define EAPDTW_WIDE_EXTERN(B, C)                                                                  \
    extern template cudaError_t launch_wide_unit<B, C>(const SearchArgs&, int, cudaStream_t); \
    extern template int blocks_wide_unit<B, C>();
EAPDTW_WIDE_EXTERN(0, 0)
EAPDTW_WIDE_EXTERN(1, 0)
EAPDTW_WIDE_EXTERN(2, 0)
EAPDTW_WIDE_EXTERN(0, 1)
EAPDTW_WIDE_EXTERN(1, 1)
EAPDTW_WIDE_EXTERN(2, 1)
#undef EAPDTW_WIDE_EXTERN

namespace {
template <int COST>
cudaError_t launch_c(int band, const SearchArgs& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_wide_unit<0, COST>(args, blocks, s);
    if (band == 1) return launch_wide_unit<1, COST>(args, blocks, s);
    return launch_wide_unit<2, COST>(args, blocks, s);
}
template <int COST>
int blocks_c(int band) {
    if (band == 0) return blocks_wide_unit<0, COST>();
    if (band == 1) return blocks_wide_unit<1, COST>();
    return blocks_wide_unit<2, COST>();
}
}  // namespace

cudaError_t launch_search_wide(int band, const SearchArgs& args, int blocks, cudaStream_t s, int cost) {
    if (group_warps(args.q.m) > kGrpMaxWarps || group_warps(args.q.m) < 2) return cudaErrorInvalidValue;
    return cost == kCostAbsolute ? launch_c<kCostAbsolute>(band, args, blocks, s) : launch_c<0>(band, args, blocks, s);
}

int search_blocks_wide(int band, int m, int cost) {
    (void)m;
    return cost == kCostAbsolute ? blocks_c<kCostAbsolute>(band) : blocks_c<0>(band);
}

#endif

}  // namespace eapdtw
