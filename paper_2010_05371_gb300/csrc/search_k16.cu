// Instantiations of the search kernel for K = 16 DP cells per lane: band modes
// 0-2, with and without the lower bounds, the first-level variants with
// upper-bound tightening, and the no-lower-bound variants with the absolute cost.
#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {

// Column values of the K = 16 kernels: 0 in registers, 1 streamed from the
// query in shared memory (a tuning knob; 0 is the measured choice).
#ifndef EAPDTW_K16_JW
#define EAPDTW_K16_JW 0
#endif

namespace {
// Per device: the shared-memory size the kernel is currently allowed, and the
// resident blocks for the last query length asked (host-side caches, so that a
// launch does not repeat the attribute and occupancy calls).
template <int BAND, bool LB, bool TIGHT, int COST>
struct LaunchCache {
    static int smem_allowed[64];
    static int last_m[64];
    static int last_blocks[64];
};
template <int BAND, bool LB, bool TIGHT, int COST> int LaunchCache<BAND, LB, TIGHT, COST>::smem_allowed[64] = {};
template <int BAND, bool LB, bool TIGHT, int COST> int LaunchCache<BAND, LB, TIGHT, COST>::last_m[64] = {};
template <int BAND, bool LB, bool TIGHT, int COST> int LaunchCache<BAND, LB, TIGHT, COST>::last_blocks[64] = {};

inline int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev & 63;
}

template <int BAND, bool LB, bool TIGHT, int COST>
cudaError_t allow_smem(size_t sm, int dev) {
    using C = LaunchCache<BAND, LB, TIGHT, COST>;
    if (static_cast<int>(sm) <= C::smem_allowed[dev]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(search_kernel<16, BAND, LB, EAPDTW_K16_JW, TIGHT, COST>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e == cudaSuccess) C::smem_allowed[dev] = static_cast<int>(sm);
    return e;
}

template <int BAND, bool LB, bool TIGHT, int COST>
cudaError_t launch_band(const SearchArgs& args, int blocks, cudaStream_t s) {
    const size_t sm = search_smem_bytes(args.q.m);
    const cudaError_t e = allow_smem<BAND, LB, TIGHT, COST>(sm, current_device());
    if (e != cudaSuccess) return e;
    search_kernel<16, BAND, LB, EAPDTW_K16_JW, TIGHT, COST><<<blocks, search_warps(args.q.m) * 32, sm, s>>>(args);
    return cudaGetLastError();
}
template <int BAND, bool LB, bool TIGHT, int COST>
int occupancy_blocks(int m) {
    using C = LaunchCache<BAND, LB, TIGHT, COST>;
    const int dev = current_device();
    if (C::last_m[dev] == m && C::last_blocks[dev] > 0) return C::last_blocks[dev];
    const size_t sm = search_smem_bytes(m);
    allow_smem<BAND, LB, TIGHT, COST>(sm, dev);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<16, BAND, LB, EAPDTW_K16_JW, TIGHT, COST>,
                                                      search_warps(m) * 32, sm) != cudaSuccess)
        per_sm = 1;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (per_sm > 0 ? per_sm : 1) * sms;
    C::last_m[dev] = m;
    C::last_blocks[dev] = blocks;
    return blocks;
}
template <bool LB, bool TIGHT, int COST>
cudaError_t launch_lb(int band, const SearchArgs& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_band<0, LB, TIGHT, COST>(args, blocks, s);
    if (band == 1) return launch_band<1, LB, TIGHT, COST>(args, blocks, s);
    return launch_band<2, LB, TIGHT, COST>(args, blocks, s);
}
template <bool LB, bool TIGHT, int COST>
int blocks_lb(int band, int m) {
    if (band == 0) return occupancy_blocks<0, LB, TIGHT, COST>(m);
    if (band == 1) return occupancy_blocks<1, LB, TIGHT, COST>(m);
    return occupancy_blocks<2, LB, TIGHT, COST>(m);
}
}  // namespace

cudaError_t launch_search_k16(int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s, bool tight,
                             int cost) {
    if (cost == kCostAbsolute) return lb ? cudaErrorInvalidValue : launch_lb<false, false, kCostAbsolute>(band, args, blocks, s);
    if (lb) return tight ? launch_lb<true, true, 0>(band, args, blocks, s) : launch_lb<true, false, 0>(band, args, blocks, s);
    return launch_lb<false, false, 0>(band, args, blocks, s);
}

int search_blocks_k16(int band, bool lb, int m, bool tight, int cost) {
    if (cost == kCostAbsolute) return blocks_lb<false, false, kCostAbsolute>(band, m);
    if (lb) return tight ? blocks_lb<true, true, 0>(band, m) : blocks_lb<true, false, 0>(band, m);
    return blocks_lb<false, false, 0>(band, m);
}

}  // namespace eapdtw
