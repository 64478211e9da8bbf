// Instantiations of the batch kernel for the four-window level (K = 32, 4096 columns).
#include "batch.cuh"
#include "kernels.h"

namespace eapdtw {

namespace {
template <int BAND>
cudaError_t launch_band(const BatchLaunch& args, int blocks, cudaStream_t s) {
    batch_kernel<32, BAND, true><<<blocks, kWarpsPerBlock * 32, kWideSmem, s>>>(args);
    return cudaGetLastError();
}
template <int BAND>
int occupancy_blocks() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<32, BAND, true>, kWarpsPerBlock * 32,
                                                      kWideSmem) !=
        cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}
template <int BAND>
cudaError_t attributes() {
    // the query copies of the eight warps live in dynamic shared memory
    return cudaFuncSetAttribute(batch_kernel<32, BAND, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kWideSmem));
}
}  // namespace

cudaError_t launch_batch_wide(int band, const BatchLaunch& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_band<0>(args, blocks, s);
    if (band == 1) return launch_band<1>(args, blocks, s);
    return launch_band<2>(args, blocks, s);
}

int batch_blocks_wide(int band) {
    if (band == 0) return occupancy_blocks<0>();
    if (band == 1) return occupancy_blocks<1>();
    return occupancy_blocks<2>();
}

cudaError_t batch_attributes_wide() {
    cudaError_t e = attributes<0>();
    if (e == cudaSuccess) e = attributes<1>();
    if (e == cudaSuccess) e = attributes<2>();
    return e;
}

}  // namespace eapdtw
