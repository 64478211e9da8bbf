// Instantiations of the widest re-run level of the search kernel: K = 32,
// four windows of 32 blocks (4096 columns), column values streamed from
// shared memory.
#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {

namespace {
template <int BAND>
cudaError_t launch_band(const SearchArgs& args, int blocks, cudaStream_t s) {
    const size_t sm = search_smem_bytes(args.q.m);
    cudaError_t e = cudaFuncSetAttribute(search_kernel<32, BAND, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    search_kernel<32, BAND, false, true><<<blocks, search_warps(args.q.m) * 32, sm, s>>>(args);
    return cudaGetLastError();
}
template <int BAND>
int occupancy_blocks(int m) {
    const size_t sm = search_smem_bytes(m);
    cudaFuncSetAttribute(search_kernel<32, BAND, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sm));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<32, BAND, false, true>,
                                                      search_warps(m) * 32, sm) != cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}
}  // namespace

cudaError_t launch_search_wide(int band, const SearchArgs& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_band<0>(args, blocks, s);
    if (band == 1) return launch_band<1>(args, blocks, s);
    return launch_band<2>(args, blocks, s);
}

int search_blocks_wide(int band, int m) {
    if (band == 0) return occupancy_blocks<0>(m);
    if (band == 1) return occupancy_blocks<1>(m);
    return occupancy_blocks<2>(m);
}

}  // namespace eapdtw
