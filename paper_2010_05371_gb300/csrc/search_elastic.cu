// Instantiations of the unconstrained first level with the narrow-block
// elastic wavefront (search_elastic_kernel): with and without the lower
// bounds, and the no-lower-bound variant with the absolute cost.
#include <mutex>

#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {

namespace {
// Per device: the shared-memory size the kernel is allowed and the resident
// blocks for the last query length asked.  Guarded by one mutex: several host
// threads (the one-query API, the no-allocation entry point) may launch at once.
std::mutex g_cache_mu;
template <bool LB, int COST>
struct ElCache {
    static int smem_allowed[64];
    static int last_m[64];
    static int last_blocks[64];
};
template <bool LB, int COST> int ElCache<LB, COST>::smem_allowed[64] = {};
template <bool LB, int COST> int ElCache<LB, COST>::last_m[64] = {};
template <bool LB, int COST> int ElCache<LB, COST>::last_blocks[64] = {};

inline int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev & 63;
}

template <bool LB, int COST>
cudaError_t allow_smem(size_t sm, int dev) {
    using C = ElCache<LB, COST>;
    if (static_cast<int>(sm) <= C::smem_allowed[dev]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(search_elastic_kernel<LB, COST>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e == cudaSuccess) C::smem_allowed[dev] = static_cast<int>(sm);
    return e;
}

template <bool LB, int COST>
cudaError_t launch_t(const SearchArgs& args, int blocks, cudaStream_t s) {
    const int m = args.q.m;
    const size_t sm = elastic_smem_bytes(m, LB);
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        const cudaError_t e = allow_smem<LB, COST>(sm, current_device());
        if (e != cudaSuccess) return e;
    }
    search_elastic_kernel<LB, COST><<<blocks, elastic_warps(m, LB) * 32, sm, s>>>(args);
    return cudaGetLastError();
}

template <bool LB, int COST>
int blocks_t(int m) {
    using C = ElCache<LB, COST>;
    std::lock_guard<std::mutex> g(g_cache_mu);
    const int dev = current_device();
    if (C::last_m[dev] == m && C::last_blocks[dev] > 0) return C::last_blocks[dev];
    const size_t sm = elastic_smem_bytes(m, LB);
    allow_smem<LB, COST>(sm, dev);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_elastic_kernel<LB, COST>,
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
}  // namespace

cudaError_t launch_search_elastic(bool lb, const SearchArgs& args, int blocks, cudaStream_t s, int cost) {
    if (elastic_warps(args.q.m, lb) < 1) return cudaErrorInvalidValue;
    if (cost == kCostAbsolute) return lb ? cudaErrorInvalidValue : launch_t<false, kCostAbsolute>(args, blocks, s);
    return lb ? launch_t<true, kCostSquared>(args, blocks, s) : launch_t<false, kCostSquared>(args, blocks, s);
}

int search_blocks_elastic(bool lb, int m, int cost) {
    if (cost == kCostAbsolute) return blocks_t<false, kCostAbsolute>(m);
    return lb ? blocks_t<true, kCostSquared>(m) : blocks_t<false, kCostSquared>(m);
}

}  // namespace eapdtw
