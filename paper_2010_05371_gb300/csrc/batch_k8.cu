// Instantiations of the batch kernel for K = 8 DP cells per lane.
#include "batch.cuh"
#include "kernels.h"

namespace eapdtw {

namespace {
template <int BAND>
cudaError_t launch_band(const BatchLaunch& args, int blocks, cudaStream_t s) {
    batch_kernel<8, BAND, 0><<<blocks, kWarpsPerBlock * 32, 0, s>>>(args);
    return cudaGetLastError();
}
template <int BAND>
int occupancy_blocks() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<8, BAND, 0>, kWarpsPerBlock * 32, 0) !=
        cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}
template <int BAND>
cudaError_t attributes() {
    // the windows and the query are read through L1: give it the whole carveout
    return cudaFuncSetAttribute(batch_kernel<8, BAND, 0>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
}
}  // namespace

cudaError_t launch_batch_k8(int band, const BatchLaunch& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_band<0>(args, blocks, s);
    if (band == 1) return launch_band<1>(args, blocks, s);
    return launch_band<2>(args, blocks, s);
}

int batch_blocks_k8(int band) {
    if (band == 0) return occupancy_blocks<0>();
    if (band == 1) return occupancy_blocks<1>();
    return occupancy_blocks<2>();
}

cudaError_t batch_attributes_k8() {
    cudaError_t e = attributes<0>();
    if (e == cudaSuccess) e = attributes<1>();
    if (e == cudaSuccess) e = attributes<2>();
    return e;
}

}  // namespace eapdtw
