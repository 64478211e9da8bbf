// The widest re-run level of the search kernel: K = 32 with the column values
// streamed from the query in shared memory, two windows of 32 blocks (2048
// columns, two resident blocks per SM) for queries up to 2048 points, four
// windows (4096 columns, one block per SM) beyond.
//
// Each (windows, band mode, cost) triple is compiled as its own unit (build.py
// defines EAPDTW_UNIT_JW, EAPDTW_UNIT_BAND and EAPDTW_UNIT_COST and this file is
// compiled once per triple, plus once without them for the dispatcher), so that
// the large kernels compile in parallel.
#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {

template <int BAND, int JW, int COST>
cudaError_t launch_wide_unit(const SearchArgs& args, int blocks, cudaStream_t s) {
    const size_t sm = search_smem_bytes(args.q.m);
    cudaError_t e = cudaFuncSetAttribute(search_kernel<32, BAND, false, JW, false, COST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    search_kernel<32, BAND, false, JW, false, COST><<<blocks, search_warps(args.q.m) * 32, sm, s>>>(args);
    return cudaGetLastError();
}

template <int BAND, int JW, int COST>
int blocks_wide_unit(int m) {
    const size_t sm = search_smem_bytes(m);
    cudaFuncSetAttribute(search_kernel<32, BAND, false, JW, false, COST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sm));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<32, BAND, false, JW, false, COST>,
                                                      search_warps(m) * 32, sm) != cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}

#if defined(EAPDTW_UNIT_JW) && defined(EAPDTW_UNIT_BAND) && defined(EAPDTW_UNIT_COST)

template cudaError_t launch_wide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_JW, EAPDTW_UNIT_COST>(const SearchArgs&, int,
                                                                                         cudaStream_t);
template int blocks_wide_unit<EAPDTW_UNIT_BAND, EAPDTW_UNIT_JW, EAPDTW_UNIT_COST>(int);

#else

#define EAPDTW_WIDE_EXTERN(B, J, C)                                                                  \
    extern template cudaError_t launch_wide_unit<B, J, C>(const SearchArgs&, int, cudaStream_t); \
    extern template int blocks_wide_unit<B, J, C>(int);
#define EAPDTW_WIDE_EXTERN_BANDS(J, C) \
    EAPDTW_WIDE_EXTERN(0, J, C)         \
    EAPDTW_WIDE_EXTERN(1, J, C)         \
    EAPDTW_WIDE_EXTERN(2, J, C)
EAPDTW_WIDE_EXTERN_BANDS(2, 0)
EAPDTW_WIDE_EXTERN_BANDS(4, 0)
EAPDTW_WIDE_EXTERN_BANDS(2, 1)
EAPDTW_WIDE_EXTERN_BANDS(4, 1)
#undef EAPDTW_WIDE_EXTERN_BANDS
#undef EAPDTW_WIDE_EXTERN

namespace {
template <int JW, int COST>
cudaError_t launch_jc(int band, const SearchArgs& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_wide_unit<0, JW, COST>(args, blocks, s);
    if (band == 1) return launch_wide_unit<1, JW, COST>(args, blocks, s);
    return launch_wide_unit<2, JW, COST>(args, blocks, s);
}
template <int JW, int COST>
int blocks_jc(int band, int m) {
    if (band == 0) return blocks_wide_unit<0, JW, COST>(m);
    if (band == 1) return blocks_wide_unit<1, JW, COST>(m);
    return blocks_wide_unit<2, JW, COST>(m);
}
}  // namespace

cudaError_t launch_search_wide(int band, const SearchArgs& args, int blocks, cudaStream_t s, int cost) {
    const bool two = args.q.m <= 2 * 1024;
    if (cost == kCostAbsolute)
        return two ? launch_jc<2, kCostAbsolute>(band, args, blocks, s) : launch_jc<4, kCostAbsolute>(band, args, blocks, s);
    return two ? launch_jc<2, 0>(band, args, blocks, s) : launch_jc<4, 0>(band, args, blocks, s);
}

int search_blocks_wide(int band, int m, int cost) {
    const bool two = m <= 2 * 1024;
    if (cost == kCostAbsolute) return two ? blocks_jc<2, kCostAbsolute>(band, m) : blocks_jc<4, kCostAbsolute>(band, m);
    return two ? blocks_jc<2, 0>(band, m) : blocks_jc<4, 0>(band, m);
}

#endif

}  // namespace eapdtw
