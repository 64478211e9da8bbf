// The batch kernel at the widest levels: K = 32, the column values streamed
// from each warp's copy of the query in shared memory, two windows of 32
// blocks (level 4, queries up to 2048 points) or four (level 5, longer ones).
//
// Compiled once per (windows, band mode) pair with EAPDTW_UNIT_JW and
// EAPDTW_UNIT_BAND defined, and once without them for the dispatcher (see
// build.py), so that the six large kernels compile in parallel.
#include "batch.cuh"
#include "kernels.h"

namespace eapdtw {

template <int BAND, int JW>
cudaError_t launch_bwide_unit(const BatchLaunch& args, int blocks, cudaStream_t s) {
    batch_kernel<32, BAND, JW><<<blocks, kWarpsPerBlock * 32, wide_smem(JW), s>>>(args);
    return cudaGetLastError();
}

template <int BAND, int JW>
int blocks_bwide_unit() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<32, BAND, JW>, kWarpsPerBlock * 32,
                                                      wide_smem(JW)) != cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}

template <int BAND, int JW>
cudaError_t attributes_bwide_unit() {
    return cudaFuncSetAttribute(batch_kernel<32, BAND, JW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(wide_smem(JW)));
}

#if defined(EAPDTW_UNIT_JW) && defined(EAPDTW_UNIT_BAND)

template cudaError_t launch_bwide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_JW>(const BatchLaunch&, int, cudaStream_t);
template int blocks_bwide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_JW>();
template cudaError_t attributes_bwide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_JW>();

#else

#define EAPDTW_BWIDE_EXTERN(B, J)                                                                 \
    extern template cudaError_t launch_bwide_unit<B, J>(const BatchLaunch&, int, cudaStream_t); \
    extern template int blocks_bwide_unit<B, J>();                                             \
    extern template cudaError_t attributes_bwide_unit<B, J>();
EAPDTW_BWIDE_EXTERN(0, 2)
EAPDTW_BWIDE_EXTERN(1, 2)
EAPDTW_BWIDE_EXTERN(2, 2)
EAPDTW_BWIDE_EXTERN(0, 4)
EAPDTW_BWIDE_EXTERN(1, 4)
EAPDTW_BWIDE_EXTERN(2, 4)
#undef EAPDTW_BWIDE_EXTERN

namespace {
template <int JW>
cudaError_t launch_j(int band, const BatchLaunch& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_bwide_unit<0, JW>(args, blocks, s);
    if (band == 1) return launch_bwide_unit<1, JW>(args, blocks, s);
    return launch_bwide_unit<2, JW>(args, blocks, s);
}
template <int JW>
int blocks_j(int band) {
    if (band == 0) return blocks_bwide_unit<0, JW>();
    if (band == 1) return blocks_bwide_unit<1, JW>();
    return blocks_bwide_unit<2, JW>();
}
template <int JW>
cudaError_t attributes_j() {
    cudaError_t e = attributes_bwide_unit<0, JW>();
    if (e == cudaSuccess) e = attributes_bwide_unit<1, JW>();
    if (e == cudaSuccess) e = attributes_bwide_unit<2, JW>();
    return e;
}
}  // namespace

cudaError_t launch_batch_wide(int level, int band, const BatchLaunch& args, int blocks, cudaStream_t s) {
    return level == 4 ? launch_j<2>(band, args, blocks, s) : launch_j<4>(band, args, blocks, s);
}

int batch_blocks_wide(int level, int band) { return level == 4 ? blocks_j<2>(band) : blocks_j<4>(band); }

cudaError_t batch_attributes_wide() {
    cudaError_t e = attributes_j<2>();
    if (e == cudaSuccess) e = attributes_j<4>();
    return e;
}

#endif

}  // namespace eapdtw
