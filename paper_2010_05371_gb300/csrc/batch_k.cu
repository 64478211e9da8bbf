// Instantiations of the batch kernel for K DP cells per lane, compiled once
// per K (build.py defines EAPDTW_UNIT_K = 4, 8, 16, 32); the dispatcher
// (launch_batch and friends in ctx.cu) declares them extern.
#include "batch.cuh"
#include "kernels.h"

#ifndef EAPDTW_UNIT_K
#error "batch_k.cu is compiled once per K with -DEAPDTW_UNIT_K=4|8|16|32"
#endif

#define EAPDTW_PASTE2(a, b) a##b
#define EAPDTW_PASTE(a, b) EAPDTW_PASTE2(a, b)

namespace eapdtw {

namespace {
constexpr int K = EAPDTW_UNIT_K;

template <int BAND>
cudaError_t launch_band(const BatchLaunch& args, int blocks, cudaStream_t s) {
    batch_kernel<K, BAND><<<blocks, kWarpsPerBlock * 32, 0, s>>>(args);
    return cudaGetLastError();
}
template <int BAND>
int occupancy_blocks() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<K, BAND>, kWarpsPerBlock * 32, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}
template <int BAND>
cudaError_t attributes() {
    // the windows and the query are read through L1: give it the whole carveout
    return cudaFuncSetAttribute(batch_kernel<K, BAND>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
}
}  // namespace

cudaError_t EAPDTW_PASTE(launch_batch_k, EAPDTW_UNIT_K)(int band, const BatchLaunch& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_band<0>(args, blocks, s);
    if (band == 1) return launch_band<1>(args, blocks, s);
    return launch_band<2>(args, blocks, s);
}

int EAPDTW_PASTE(batch_blocks_k, EAPDTW_UNIT_K)(int band) {
    if (band == 0) return occupancy_blocks<0>();
    if (band == 1) return occupancy_blocks<1>();
    return occupancy_blocks<2>();
}

cudaError_t EAPDTW_PASTE(batch_attributes_k, EAPDTW_UNIT_K)() {
    cudaError_t e = attributes<0>();
    if (e == cudaSuccess) e = attributes<1>();
    if (e == cudaSuccess) e = attributes<2>();
    return e;
}

}  // namespace eapdtw
