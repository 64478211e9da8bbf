// Instantiations of the first level with the narrow-block elastic wavefront
// (search_elastic_kernel): with and without the lower bounds, the
// no-lower-bound variant with the absolute cost, each unconstrained or banded.
//
// Each band mode is compiled as its own unit (build.py defines
// EAPDTW_UNIT_EBAND and this file is compiled once per mode, plus once without
// it for the dispatcher).
#include <mutex>

#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {

template <bool LB, int BAND, int COST>
cudaError_t elastic_launch_unit(const SearchArgs& args, int blocks, cudaStream_t s);
template <bool LB, int BAND, int COST>
int elastic_blocks_unit(int m);

#if defined(EAPDTW_UNIT_EBAND)

namespace {
// Per device: the shared-memory size the kernel is allowed and the resident
// blocks for the last query length asked.  Guarded by one mutex: several host
// threads (the one-query API, the no-allocation entry point) may launch at once.
std::mutex g_cache_mu;
template <bool LB, int BAND, int COST>
struct ElCache {
    static int smem_allowed[64];
    static int last_m[64];
    static int last_blocks[64];
};
template <bool LB, int BAND, int COST> int ElCache<LB, BAND, COST>::smem_allowed[64] = {};
template <bool LB, int BAND, int COST> int ElCache<LB, BAND, COST>::last_m[64] = {};
template <bool LB, int BAND, int COST> int ElCache<LB, BAND, COST>::last_blocks[64] = {};

inline int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev & 63;
}

template <bool LB, int BAND, int COST>
cudaError_t allow_smem(size_t sm, int dev) {
    using C = ElCache<LB, BAND, COST>;
    if (static_cast<int>(sm) <= C::smem_allowed[dev]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(search_elastic_kernel<LB, BAND, COST>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e == cudaSuccess) C::smem_allowed[dev] = static_cast<int>(sm);
    return e;
}
}  // namespace

template <bool LB, int BAND, int COST>
cudaError_t elastic_launch_unit(const SearchArgs& args, int blocks, cudaStream_t s) {
    const int m = args.q.m;
    const size_t sm = elastic_smem_bytes(m, LB);
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        const cudaError_t e = allow_smem<LB, BAND, COST>(sm, current_device());
        if (e != cudaSuccess) return e;
    }
    search_elastic_kernel<LB, BAND, COST><<<blocks, elastic_warps(m, LB) * 32, sm, s>>>(args);
    return cudaGetLastError();
}

template <bool LB, int BAND, int COST>
int elastic_blocks_unit(int m) {
    using C = ElCache<LB, BAND, COST>;
    std::lock_guard<std::mutex> g(g_cache_mu);
    const int dev = current_device();
    if (C::last_m[dev] == m && C::last_blocks[dev] > 0) return C::last_blocks[dev];
    const size_t sm = elastic_smem_bytes(m, LB);
    allow_smem<LB, BAND, COST>(sm, dev);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_elastic_kernel<LB, BAND, COST>,
                                                      elastic_warps(m, LB) * 32, sm) != cudaSuccess) {
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

#define EAPDTW_EL_INST(L, C)                                                                                 \
    template cudaError_t elastic_launch_unit<L, EAPDTW_UNIT_EBAND, C>(const SearchArgs&, int, cudaStream_t); \
    template int elastic_blocks_unit<L, EAPDTW_UNIT_EBAND, C>(int);
EAPDTW_EL_INST(true, kCostSquared)
EAPDTW_EL_INST(false, kCostSquared)
EAPDTW_EL_INST(false, kCostAbsolute)
#undef EAPDTW_EL_INST

#else

#define EAPDTW_EL_EXTERN(L, B, C)                                                                     \
    extern template cudaError_t elastic_launch_unit<L, B, C>(const SearchArgs&, int, cudaStream_t); \
    extern template int elastic_blocks_unit<L, B, C>(int);
EAPDTW_EL_EXTERN(true, 0, kCostSquared)
EAPDTW_EL_EXTERN(false, 0, kCostSquared)
EAPDTW_EL_EXTERN(false, 0, kCostAbsolute)
EAPDTW_EL_EXTERN(true, 1, kCostSquared)
EAPDTW_EL_EXTERN(false, 1, kCostSquared)
EAPDTW_EL_EXTERN(false, 1, kCostAbsolute)
#undef EAPDTW_EL_EXTERN

namespace {
template <int BAND>
cudaError_t launch_b(bool lb, const SearchArgs& args, int blocks, cudaStream_t s, int cost) {
    if (cost == kCostAbsolute)
        return lb ? cudaErrorInvalidValue : elastic_launch_unit<false, BAND, kCostAbsolute>(args, blocks, s);
    return lb ? elastic_launch_unit<true, BAND, kCostSquared>(args, blocks, s)
              : elastic_launch_unit<false, BAND, kCostSquared>(args, blocks, s);
}
template <int BAND>
int blocks_b(bool lb, int m, int cost) {
    if (cost == kCostAbsolute) return elastic_blocks_unit<false, BAND, kCostAbsolute>(m);
    return lb ? elastic_blocks_unit<true, BAND, kCostSquared>(m) : elastic_blocks_unit<false, BAND, kCostSquared>(m);
}
}  // namespace

cudaError_t launch_search_elastic(bool lb, int band, const SearchArgs& args, int blocks, cudaStream_t s, int cost) {
    if (elastic_warps(args.q.m, lb) < 1) return cudaErrorInvalidValue;
    return band ? launch_b<1>(lb, args, blocks, s, cost) : launch_b<0>(lb, args, blocks, s, cost);
}

int search_blocks_elastic(bool lb, int band, int m, int cost) {
    return band ? blocks_b<1>(lb, m, cost) : blocks_b<0>(lb, m, cost);
}

#endif

}  // namespace eapdtw
