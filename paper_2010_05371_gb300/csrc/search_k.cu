// Instantiations of the search kernel for K DP cells per lane: band modes 0-2,
// with and without the lower bounds, the first-level variants with upper-bound
// tightening, and the no-lower-bound variants with the absolute cost.
//
// Compiled once per K (build.py defines EAPDTW_UNIT_K = 4, 8, 16, 32), so that
// the instantiations compile in parallel; the dispatcher (launch_search,
// search_blocks in api.cu) declares them extern.
#include <mutex>

#include "kernels.h"
#include "search_kernel.cuh"

#ifndef EAPDTW_UNIT_K
#error "search_k.cu is compiled once per K with -DEAPDTW_UNIT_K=4|8|16|32"
#endif

// launch_search_k4 etc.: the unit's K pasted onto the name
#define EAPDTW_PASTE2(a, b) a##b
#define EAPDTW_PASTE(a, b) EAPDTW_PASTE2(a, b)

namespace eapdtw {

// Column values of the kernels: 0 in registers, 1 streamed from the query in
// shared memory (a tuning knob; 0 is the measured choice).
#ifndef EAPDTW_KJW
#define EAPDTW_KJW 0
#endif

namespace {
constexpr int K = EAPDTW_UNIT_K;

// Per device: the shared-memory size the kernel is currently allowed, and the
// resident blocks for the last query length asked (host-side caches, so that a
// launch does not repeat the attribute and occupancy calls).  One mutex guards
// them: launches may come from several host threads at once (the one-query
// API, the no-allocation entry point, a context's serving thread).
std::mutex g_cache_mu;
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
cudaError_t allow_smem(size_t sm, int dev) {   // caller holds g_cache_mu
    using C = LaunchCache<BAND, LB, TIGHT, COST>;
    if (static_cast<int>(sm) <= C::smem_allowed[dev]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(search_kernel<K, BAND, LB, EAPDTW_KJW, TIGHT, COST>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e == cudaSuccess) C::smem_allowed[dev] = static_cast<int>(sm);
    return e;
}

template <int BAND, bool LB, bool TIGHT, int COST>
cudaError_t launch_band(const SearchArgs& args, int blocks, cudaStream_t s) {
    const size_t sm = search_smem_bytes(args.q.m);
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        const cudaError_t e = allow_smem<BAND, LB, TIGHT, COST>(sm, current_device());
        if (e != cudaSuccess) return e;
    }
    search_kernel<K, BAND, LB, EAPDTW_KJW, TIGHT, COST><<<blocks, search_warps(args.q.m) * 32, sm, s>>>(args);
    return cudaGetLastError();
}
template <int BAND, bool LB, bool TIGHT, int COST>
int occupancy_blocks(int m) {
    using C = LaunchCache<BAND, LB, TIGHT, COST>;
    std::lock_guard<std::mutex> g(g_cache_mu);
    const int dev = current_device();
    if (C::last_m[dev] == m && C::last_blocks[dev] > 0) return C::last_blocks[dev];
    const size_t sm = search_smem_bytes(m);
    allow_smem<BAND, LB, TIGHT, COST>(sm, dev);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<K, BAND, LB, EAPDTW_KJW, TIGHT, COST>,
                                                      search_warps(m) * 32, sm) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
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

cudaError_t EAPDTW_PASTE(launch_search_k, EAPDTW_UNIT_K)(int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s,
                                          bool tight, int cost) {
    if (cost == kCostAbsolute) return lb ? cudaErrorInvalidValue : launch_lb<false, false, kCostAbsolute>(band, args, blocks, s);
    if (lb) return tight ? launch_lb<true, true, 0>(band, args, blocks, s) : launch_lb<true, false, 0>(band, args, blocks, s);
    return launch_lb<false, false, 0>(band, args, blocks, s);
}

int EAPDTW_PASTE(search_blocks_k, EAPDTW_UNIT_K)(int band, bool lb, int m, bool tight, int cost) {
    if (cost == kCostAbsolute) return blocks_lb<false, false, kCostAbsolute>(band, m);
    if (lb) return tight ? blocks_lb<true, true, 0>(band, m) : blocks_lb<true, false, 0>(band, m);
    return blocks_lb<false, false, 0>(band, m);
}

}  // namespace eapdtw
