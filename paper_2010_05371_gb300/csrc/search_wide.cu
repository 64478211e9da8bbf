// Instantiations of the widest re-run level of the search kernel: K = 32 with
// the column values streamed from the query in shared memory, two windows of
// 32 blocks (2048 columns, two resident blocks per SM) for queries up to 2048
// points, four windows (4096 columns, one block per SM) beyond.
#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {

namespace {
template <int BAND, int JW>
cudaError_t launch_band(const SearchArgs& args, int blocks, cudaStream_t s) {
    const size_t sm = search_smem_bytes(args.q.m);
    cudaError_t e = cudaFuncSetAttribute(search_kernel<32, BAND, false, JW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    search_kernel<32, BAND, false, JW><<<blocks, search_warps(args.q.m) * 32, sm, s>>>(args);
    return cudaGetLastError();
}
template <int BAND, int JW>
int occupancy_blocks(int m) {
    const size_t sm = search_smem_bytes(m);
    cudaFuncSetAttribute(search_kernel<32, BAND, false, JW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sm));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<32, BAND, false, JW>,
                                                      search_warps(m) * 32, sm) != cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}
template <int JW>
cudaError_t launch_j(int band, const SearchArgs& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_band<0, JW>(args, blocks, s);
    if (band == 1) return launch_band<1, JW>(args, blocks, s);
    return launch_band<2, JW>(args, blocks, s);
}
template <int JW>
int blocks_j(int band, int m) {
    if (band == 0) return occupancy_blocks<0, JW>(m);
    if (band == 1) return occupancy_blocks<1, JW>(m);
    return occupancy_blocks<2, JW>(m);
}
}  // namespace

cudaError_t launch_search_wide(int band, const SearchArgs& args, int blocks, cudaStream_t s) {
    return args.q.m <= 2 * 1024 ? launch_j<2>(band, args, blocks, s) : launch_j<4>(band, args, blocks, s);
}

int search_blocks_wide(int band, int m) { return m <= 2 * 1024 ? blocks_j<2>(band, m) : blocks_j<4>(band, m); }

}  // namespace eapdtw
