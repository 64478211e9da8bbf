// Instantiations of the search kernel for K = 32 DP cells per lane.
#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {


namespace {
template <int BAND, bool LB>
cudaError_t launch_band(const SearchArgs& args, int blocks, cudaStream_t s) {
    const size_t sm = search_smem_bytes(args.q.m);
    cudaError_t e = cudaFuncSetAttribute(search_kernel<32, BAND, LB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    search_kernel<32, BAND, LB><<<blocks, search_warps(args.q.m) * 32, sm, s>>>(args);
    return cudaGetLastError();
}
template <int BAND, bool LB>
int occupancy_blocks(int m) {
    const size_t sm = search_smem_bytes(m);
    cudaFuncSetAttribute(search_kernel<32, BAND, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sm));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<32, BAND, LB>,
                                                      search_warps(m) * 32, sm) != cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}
}  // namespace

cudaError_t launch_search_k32(int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s) {
    if (lb) {
        if (band == 0) return launch_band<0, true>(args, blocks, s);
        if (band == 1) return launch_band<1, true>(args, blocks, s);
        return launch_band<2, true>(args, blocks, s);
    }
    if (band == 0) return launch_band<0, false>(args, blocks, s);
    if (band == 1) return launch_band<1, false>(args, blocks, s);
    return launch_band<2, false>(args, blocks, s);
}

int search_blocks_k32(int band, bool lb, int m) {
    if (lb) {
        if (band == 0) return occupancy_blocks<0, true>(m);
        if (band == 1) return occupancy_blocks<1, true>(m);
        return occupancy_blocks<2, true>(m);
    }
    if (band == 0) return occupancy_blocks<0, false>(m);
    if (band == 1) return occupancy_blocks<1, false>(m);
    return occupancy_blocks<2, false>(m);
}

}  // namespace eapdtw
