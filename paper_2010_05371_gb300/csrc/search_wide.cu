// The widest re-run level of the search kernel: K = 32 with the column values
// streamed from the query in shared memory, two windows of 32 blocks (2048
// columns, two resident blocks per SM) for queries up to 2048 points, four
// windows (4096 columns, one block per SM) beyond.
//
// Each (windows, band mode) pair is compiled as its own unit (build.py defines
// EAPDTW_UNIT_JW and EAPDTW_UNIT_BAND and this file is compiled once per
// pair, plus once without them for the dispatcher), so that the six large
// kernels compile in parallel.
#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {

template <int BAND, int JW>
cudaError_t launch_wide_unit(const SearchArgs& args, int blocks, cudaStream_t s) {
    const size_t sm = search_smem_bytes(args.q.m);
    cudaError_t e = cudaFuncSetAttribute(search_kernel<32, BAND, false, JW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    search_kernel<32, BAND, false, JW><<<blocks, search_warps(args.q.m) * 32, sm, s>>>(args);
    return cudaGetLastError();
}

template <int BAND, int JW>
int blocks_wide_unit(int m) {
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

#if defined(EAPDTW_UNIT_JW) && defined(EAPDTW_UNIT_BAND)

template cudaError_t launch_wide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_JW>(const SearchArgs&, int, cudaStream_t);
template int blocks_wide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_JW>(int);

#else

#define EAPDTW_WIDE_EXTERN(B, J)                                                                 \
    extern template cudaError_t launch_wide_unit<B, J>(const SearchArgs&, int, cudaStream_t); \
    extern template int blocks_wide_unit<B, J>(int);
EAPDTW_WIDE_EXTERN(0, 2)
EAPDTW_WIDE_EXTERN(1, 2)
EAPDTW_WIDE_EXTERN(2, 2)
EAPDTW_WIDE_EXTERN(0, 4)
EAPDTW_WIDE_EXTERN(1, 4)
EAPDTW_WIDE_EXTERN(2, 4)
#undef EAPDTW_WIDE_EXTERN

cudaError_t launch_search_wide(int band, const SearchArgs& args, int blocks, cudaStream_t s) {
    if (args.q.m <= 2 * 1024) {
        if (band == 0) return launch_wide_unit<0, 2>(args, blocks, s);
        if (band == 1) return launch_wide_unit<1, 2>(args, blocks, s);
        return launch_wide_unit<2, 2>(args, blocks, s);
    }
    if (band == 0) return launch_wide_unit<0, 4>(args, blocks, s);
    if (band == 1) return launch_wide_unit<1, 4>(args, blocks, s);
    return launch_wide_unit<2, 4>(args, blocks, s);
}

int search_blocks_wide(int band, int m) {
    if (m <= 2 * 1024) {
        if (band == 0) return blocks_wide_unit<0, 2>(m);
        if (band == 1) return blocks_wide_unit<1, 2>(m);
        return blocks_wide_unit<2, 2>(m);
    }
    if (band == 0) return blocks_wide_unit<0, 4>(m);
    if (band == 1) return blocks_wide_unit<1, 4>(m);
    return blocks_wide_unit<2, 4>(m);
}

#endif

}  // namespace eapdtw
