// The group levels of the one-query search (dtw_group.cuh: the warps of a
// group share one candidate, warp g owning columns 512 g + 1 .. 512 g + 512 in
// registers, the edge columns passing through shared memory):
//  * the widest re-run level (list mode): candidates whose live region
//    overflowed one warp's window at K = 32 (queries of more than 1024
//    points), and the seed windows of such queries;
//  * a first level (tile mode, LB = true) for banded queries whose band does
//    not fit one warp's window: warp 0 of the group stages a tile of 32
//    windows and runs the lower-bound cascade lane by lane (tile_lanes), then
//    the whole group runs the survivors one after another.
// Groups of group_warps(m) warps; the block's eight warps hold as many groups
// as fit (warps left over stay idle).  The query arrays are staged once per
// block in dynamic shared memory, followed by one tile of points per group.
//
// Each (band mode, lower bounds, cost) triple is compiled as its own unit
// (build.py defines EAPDTW_UNIT_BAND, EAPDTW_UNIT_LB and EAPDTW_UNIT_COST and
// this file is compiled once per triple, plus once without them for the
// dispatcher).
#include "dtw_group.cuh"
#include "kernels.h"
#include "search_kernel.cuh"

namespace eapdtw {

constexpr int kMaxGroups = 4;   // groups per block (one warp each below 513 columns)

__host__ __device__ inline int group_count(int m) {
    const int G = group_warps(m);
    const int n = G <= kGrpMaxWarps ? kWarpsPerBlock / G : 0;
    return n < kMaxGroups ? n : kMaxGroups;
}

__host__ inline size_t group_smem_bytes(int m) {
    return sizeof(float) * (5 * static_cast<size_t>(query_pad(m)) +
                            static_cast<size_t>(group_count(m)) * tile_floats(m));
}

template <int BAND, bool LB, int COST>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, EAPDTW_MINB_GROUP) search_group_kernel(const SearchArgs A) {
    extern __shared__ __align__(16) float smem[];
    __shared__ GroupSync s_gs[kMaxGroups];
    __shared__ unsigned long long s_cnt[10];
    const int m = A.q.m;
    const int mp = query_pad(m);
    float* s_zq = smem;
    float* s_uq = s_zq + mp;
    float* s_lq = s_uq + mp;
    float* s_zqo = s_lq + mp;
    int* s_ord = reinterpret_cast<int*>(s_zqo + mp);
    if (threadIdx.x < 10) s_cnt[threadIdx.x] = 0;
    for (int j = threadIdx.x; j < mp; j += blockDim.x) {
        s_zq[j] = j < m ? A.q.zq[j] : f_nan();
        if (LB) {
            s_uq[j] = A.q.uq_o[j];
            s_lq[j] = A.q.lq_o[j];
            s_zqo[j] = A.q.zq_o[j];
            s_ord[j] = A.q.ord[j];
        }
    }
    __syncthreads();
    const int G = group_warps(m);
    const int ngroups = group_count(m);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int gi = warp / G;
    const int g = warp - gi * G;
    auto count = [&](int c, unsigned long long v) { if (v) atomicAdd(s_cnt + c, v); };
    if (gi < ngroups) {
        GroupSync& gs = s_gs[gi];
        volatile GroupSync& vs = gs;
        float* tile = reinterpret_cast<float*>(s_ord + mp) + gi * tile_floats(m);
        const bool list_mode = A.ovf_in != nullptr;
        int64_t nitems;
        if (list_mode) {
            const int c = *A.ovf_in_count;
            nitems = c < A.ovf_in_cap ? c : A.ovf_in_cap;
        } else {
            const int64_t hi = A.tile_hi > 0 ? A.tile_hi : (A.nw + 31) / 32;
            nitems = hi - A.tile_lo;
        }
        TileCtx C{};
        C.ref = A.ref;
        C.zq = s_zq;
        C.uq = s_uq;
        C.lq = s_lq;
        C.zqo = s_zqo;
        C.ord = s_ord;
        C.m = m;
        C.w = A.w;
        C.use_lb = LB ? A.use_lb : 0;
        C.use_ec = LB ? A.use_lb : 0;
        C.ur = A.ur;
        C.lr = A.lr;
        C.lb_scale = A.lb_scale;
        C.bsf = A.bsf;
        C.nw = A.nw;
        C.dbg = A.dbg;
        if (g == 0 && lane == 0) {
            group_reset(gs);
            vs.abort_flag = 0;
        }
        for (;;) {
            if (g == 0 && lane == 0)
                vs.unit = vs.abort_flag ? nitems : static_cast<long long>(atomicAdd(A.work_counter, 1));
            group_bar(gi, G);
            const int64_t u = vs.unit;   // the same reading on every warp of the group
            if (u >= nitems) break;
            const int64_t i0 = list_mode ? (A.ovf_in[u] & 0xffffffffll) : (A.tile_lo + u) * 32;
            const int nl = list_mode ? 1 : static_cast<int>(A.nw - i0 < 32 ? A.nw - i0 : 32);
            if (g == 0) {
                // warp 0: the tile's points, then statistics, bounds and corner lane by lane
                const int len = nl - 1 + m;
                if ((reinterpret_cast<uintptr_t>(A.ref.R + i0) & 15) == 0 && !list_mode) {
                    const float4* src = reinterpret_cast<const float4*>(A.ref.R + i0);
                    const int nv = len / 4;
                    for (int v = lane; v < nv; v += 32) reinterpret_cast<float4*>(tile)[v] = __ldg(src + v);
                    for (int j = nv * 4 + lane; j < len; j += 32) tile[j] = __ldg(A.ref.R + i0 + j);
                } else {
                    for (int j = lane; j < len; j += 32) tile[j] = __ldg(A.ref.R + i0 + j);
                }
                __syncwarp();
                float a, cw, isd, lb;
                const bool alive = tile_lanes<BAND, LB, 1, COST>(C, tile, list_mode, i0, nl, count, a, cw, isd, lb);
                const unsigned mask = __ballot_sync(kFull, alive);
                vs.sa[lane] = a;
                vs.scw[lane] = cw;
                vs.sisd[lane] = isd;
                vs.slb[lane] = lb;
                if (lane == 0) vs.surv = mask;
            }
            group_bar(gi, G);
            unsigned mask = vs.surv;
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                if (g == 0 && lane == 0) {
                    // one reading of the bound decides for the whole group
                    const float ub = A.bsf.load();
                    const bool skip = LB && C.use_lb && !list_mode && vs.slb[src] > ub * C.lb_scale;
                    if (skip) count(kCntRecheck, 1);
                    vs.cand = skip ? -1 : src;
                    vs.ub = ub;
                }
                group_bar(gi, G);
                const int cand = vs.cand;
                if (cand >= 0) {
                    const int off = list_mode ? 0 : cand;
                    const int64_t iw = i0 + off;
                    const DtwOut o = dtw_group<BAND, COST>(gs, g, tile + off, vs.sa[cand], vs.scw[cand],
                                                           vs.sisd[cand], s_zq, m, m, A.w, A.bsf, vs.ub, A.err, 1);
                    if (lane == 0) count(kCntCells, static_cast<unsigned long long>(o.busy) * kGrpK);
                    if (g == G - 1 && lane == 0 && o.status == 0) {
                        count(kCntSteps, static_cast<unsigned long long>(o.steps));
                        const float ubn = A.bsf.load();
                        if (o.dist <= ubn && o.dist < f_inf()) {
                            A.bsf.insert(o.dist, static_cast<uint32_t>(iw));
                            count(kCntCompleted, 1);
                        } else {
                            count(kCntAbandoned, 1);
                        }
                    }
                }
                group_bar(gi, G);   // every warp is done with the candidate and the group's state
                if (g == 0 && lane == 0) group_reset(gs);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 10 && s_cnt[threadIdx.x]) atomicAdd(A.counters + threadIdx.x, s_cnt[threadIdx.x]);
}

template <int BAND, bool LB, int COST>
cudaError_t launch_group_unit(const SearchArgs& args, int blocks, cudaStream_t s) {
    const size_t sm = group_smem_bytes(args.q.m);
    cudaError_t e = cudaFuncSetAttribute(search_group_kernel<BAND, LB, COST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    search_group_kernel<BAND, LB, COST><<<blocks, kWarpsPerBlock * 32, sm, s>>>(args);
    return cudaGetLastError();
}

template <int BAND, bool LB, int COST>
int blocks_group_unit(int m) {
    const size_t sm = group_smem_bytes(m);
    cudaFuncSetAttribute(search_group_kernel<BAND, LB, COST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sm));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_group_kernel<BAND, LB, COST>,
                                                      kWarpsPerBlock * 32, sm) != cudaSuccess)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * sms;
}

#if defined(EAPDTW_UNIT_BAND) && defined(EAPDTW_UNIT_LB) && defined(EAPDTW_UNIT_COST)

template cudaError_t launch_group_unit<EAPDTW_UNIT_BAND, (EAPDTW_UNIT_LB != 0), EAPDTW_UNIT_COST>(const SearchArgs&,
                                                                                              int, cudaStream_t);
template int blocks_group_unit<EAPDTW_UNIT_BAND, (EAPDTW_UNIT_LB != 0), EAPDTW_UNIT_COST>(int);

#else

#define EAPDTW_GROUP_EXTERN(B, L, C)                                                                \
    extern template cudaError_t launch_group_unit<B, L, C>(const SearchArgs&, int, cudaStream_t); \
    extern template int blocks_group_unit<B, L, C>(int);
EAPDTW_GROUP_EXTERN(0, false, 0)
EAPDTW_GROUP_EXTERN(1, false, 0)
EAPDTW_GROUP_EXTERN(2, false, 0)
EAPDTW_GROUP_EXTERN(0, true, 0)
EAPDTW_GROUP_EXTERN(1, true, 0)
EAPDTW_GROUP_EXTERN(2, true, 0)
EAPDTW_GROUP_EXTERN(0, false, 1)
EAPDTW_GROUP_EXTERN(1, false, 1)
EAPDTW_GROUP_EXTERN(2, false, 1)
#undef EAPDTW_GROUP_EXTERN

namespace {
template <bool LB, int COST>
cudaError_t launch_lc(int band, const SearchArgs& args, int blocks, cudaStream_t s) {
    if (band == 0) return launch_group_unit<0, LB, COST>(args, blocks, s);
    if (band == 1) return launch_group_unit<1, LB, COST>(args, blocks, s);
    return launch_group_unit<2, LB, COST>(args, blocks, s);
}
template <bool LB, int COST>
int blocks_lc(int band, int m) {
    if (band == 0) return blocks_group_unit<0, LB, COST>(m);
    if (band == 1) return blocks_group_unit<1, LB, COST>(m);
    return blocks_group_unit<2, LB, COST>(m);
}
}  // namespace

cudaError_t launch_search_wide(int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s, int cost) {
    if (group_count(args.q.m) < 1) return cudaErrorInvalidValue;
    if (cost == kCostAbsolute) return lb ? cudaErrorInvalidValue : launch_lc<false, kCostAbsolute>(band, args, blocks, s);
    return lb ? launch_lc<true, 0>(band, args, blocks, s) : launch_lc<false, 0>(band, args, blocks, s);
}

int search_blocks_wide(int band, bool lb, int m, int cost) {
    if (cost == kCostAbsolute) return blocks_lc<false, kCostAbsolute>(band, m);
    return lb ? blocks_lc<true, 0>(band, m) : blocks_lc<false, 0>(band, m);
}

#endif

}  // namespace eapdtw
