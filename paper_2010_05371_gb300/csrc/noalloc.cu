// subseq_search_noalloc: the subsequence search for callers that cannot
// allocate memory.  All scratch lives in one fixed device array of this file;
// the kernels are the same ones subseq_search launches.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "eapdtw.h"
#include "kernels.h"
#include "plan.h"
#include "search_kernel.cuh"

using namespace eapdtw;

namespace {

constexpr int64_t kMaxN = EAPDTW_NOALLOC_MAX_N;
constexpr int64_t kMaxChunks = (kMaxN + kChunk - 1) / kChunk;
constexpr int kMaxQ = EAPDTW_MAX_QUERY;
constexpr int kSeedN = 4096;
constexpr int kSeedBest = 32;

// Byte offsets of the sub-arrays inside the scratch array (each 256-aligned).
constexpr int64_t al(int64_t x) { return (x + 255) / 256 * 256; }
constexpr int64_t kOffP1 = 0;
constexpr int64_t kOffP2 = kOffP1 + al(8 * kMaxN);
constexpr int64_t kOffUR = kOffP2 + al(8 * kMaxN);
constexpr int64_t kOffLR = kOffUR + al(4 * kMaxN);
constexpr int64_t kOffOvf0 = kOffLR + al(4 * kMaxN);
constexpr int64_t kOffOvf1 = kOffOvf0 + al(8 * kMaxN);
constexpr int64_t kOffT1 = kOffOvf1 + al(8 * kMaxN);
constexpr int64_t kOffT2 = kOffT1 + al(8 * kMaxChunks);
constexpr int64_t kOffA = kOffT2 + al(8 * kMaxChunks);
constexpr int64_t kOffZq = kOffA + al(4 * kMaxChunks);
constexpr int64_t kOffUq = kOffZq + al(4 * kMaxQ);
constexpr int64_t kOffLq = kOffUq + al(4 * kMaxQ);
constexpr int64_t kOffZqo = kOffLq + al(4 * kMaxQ);
constexpr int64_t kOffOrd = kOffZqo + al(4 * kMaxQ);
constexpr int64_t kOffState = kOffOrd + al(4 * kMaxQ);   // slots | counters | seed counters | ints | ub_seed
constexpr int64_t kOffSeedEd = kOffState + 1024;
constexpr int64_t kOffSeedIdx = kOffSeedEd + al(4 * kSeedN);
constexpr int64_t kOffSeedBest = kOffSeedIdx + al(4 * kSeedN);
constexpr int64_t kUsed = kOffSeedBest + al(8 * 64);
static_assert(kUsed <= EAPDTW_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");

__device__ __align__(256) unsigned char g_scratch[EAPDTW_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
unsigned char* g_addr[64] = {nullptr};  // device address of g_scratch, per device

#define CKN(expr)                     \
    do {                              \
        if ((expr) != cudaSuccess) {  \
            cudaGetLastError();       \
            return EAPDTW_ERR_CUDA;   \
        }                             \
    } while (0)

}  // namespace

extern "C" int32_t subseq_search_noalloc(const float* Q, int64_t lQ, const float* R, int64_t lR,
                                         int64_t w, int32_t k, int64_t* out_idx, double* out_dist,
                                         void* stream) {
    if (!Q || !R || !out_idx || !out_dist || lQ < 1 || lR < lQ || w < 0 || k < 1)
        return EAPDTW_ERR_INVALID_ARG;
    if (lR > kMaxN || lQ > kMaxQ || k > EAPDTW_MAX_K) return EAPDTW_ERR_UNSUPPORTED;
    const int m = static_cast<int>(lQ);
    if (search_warps(m) < 1) return EAPDTW_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return EAPDTW_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        // Set-up on this device (the device is current): the host-side name
        // g_scratch is not a device address, so look the address up once.
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return EAPDTW_ERR_CUDA;
        }
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    unsigned char* base = g_addr[dev];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = lR;
    const int64_t nw = n - m + 1;
    const int wi = static_cast<int>(w < m ? w : m);

    double* P1 = reinterpret_cast<double*>(base + kOffP1);
    double* P2 = reinterpret_cast<double*>(base + kOffP2);
    double* T1 = reinterpret_cast<double*>(base + kOffT1);
    double* T2 = reinterpret_cast<double*>(base + kOffT2);
    float* A = reinterpret_cast<float*>(base + kOffA);
    float* UR = reinterpret_cast<float*>(base + kOffUR);
    float* LR = reinterpret_cast<float*>(base + kOffLR);
    long long* ovf[2] = {reinterpret_cast<long long*>(base + kOffOvf0), reinterpret_cast<long long*>(base + kOffOvf1)};
    float* zq = reinterpret_cast<float*>(base + kOffZq);
    float* uq = reinterpret_cast<float*>(base + kOffUq);
    float* lq = reinterpret_cast<float*>(base + kOffLq);
    float* zqo = reinterpret_cast<float*>(base + kOffZqo);
    int* ord = reinterpret_cast<int*>(base + kOffOrd);
    unsigned char* state = base + kOffState;
    auto* slots = reinterpret_cast<unsigned long long*>(state);
    auto* counters = reinterpret_cast<unsigned long long*>(state + 512);
    auto* seed_counters = reinterpret_cast<unsigned long long*>(state + 640);
    int* ints = reinterpret_cast<int*>(state + 768);
    float* ub_seed = reinterpret_cast<float*>(state + 896);
    float* seed_ed = reinterpret_cast<float*>(base + kOffSeedEd);
    int* seed_idx = reinterpret_cast<int*>(base + kOffSeedIdx);
    long long* seed_best = reinterpret_cast<long long*>(base + kOffSeedBest);
    const int ovf_cap = static_cast<int>(nw);

    // the same levels as subseq_search (plan.h)
    const Plan plan = plan_levels(m, m, wi, 0);
    const int nlev = plan.nlev;

    // the previous call's state is overwritten here: slots, counters, work lists
    CKN(launch_init_state(slots, k, ub_seed, counters, ints, kNumInts, st));
    CKN(cudaMemsetAsync(seed_counters, 0, 128, st));
    CKN(launch_ref_prefix(R, n, P1, P2, T1, T2, A, ints + kBad, st));
    CKN(launch_query_prep(Q, m, wi, zq, uq, lq, zqo, ord, ints + kBad, st));
    CKN(launch_envelope(R, n, wi < m - 1 ? wi : m - 1, UR, LR, st));

    SearchArgs a{};
    a.ref = RefView{R, n, P1, P2, T1, T2, A};
    a.q = QueryView{zq, uq, lq, zqo, ord, m};
    a.ur = UR;
    a.lr = LR;
    a.bsf = BestSoFar{slots, ub_seed, k, 0, 0.0f};
    a.nw = nw;
    a.w = wi;
    a.use_lb = 1;
    a.lb_scale = 1.0001f;
    a.counters = counters;
    a.err = ints + kTimeout;
    if (nw >= 2048) {
        const int ns = static_cast<int>(nw < kSeedN ? nw : kSeedN);
        CKN(launch_seed(a.ref, zq, m, nw, ns, seed_ed, seed_idx, k, ub_seed, seed_best, kSeedBest,
                        ints + kNBest, st));
        SearchArgs sa = a;
        sa.use_lb = 0;
        sa.work_counter = ints + kWorkSeed;
        sa.ovf_in = seed_best;
        sa.ovf_in_count = ints + kNBest;
        sa.ovf_in_cap = kSeedBest;
        sa.ovf_out = nullptr;
        sa.ovf_out_count = ints + kSeedOvf;
        sa.ovf_cap = 0;
        sa.counters = seed_counters;
        const int K = plan.K[nlev - 1], bd = plan.band[nlev - 1];
        if (plan.wide[nlev - 1]) {
            CKN(launch_search_wide(bd, false, sa, search_blocks_wide(bd, false, m) / 4 + 1, st));
        } else {
            CKN(launch_search(K, bd, false, sa, search_blocks(K, bd, false, m) / 4 + 1, st));
        }
    }
    for (int lev = 0; lev < nlev; ++lev) {
        SearchArgs la = a;
        la.work_counter = ints + kWork0 + lev;
        la.ovf_out = ovf[lev & 1];
        la.ovf_out_count = ints + kOvf0 + lev;
        la.ovf_cap = ovf_cap;
        if (lev > 0) {
            la.ovf_in = ovf[(lev - 1) & 1];
            la.ovf_in_count = ints + kOvf0 + lev - 1;
            la.ovf_in_cap = ovf_cap;
        }
        const bool lb = lev == 0;
        if (plan.wide[lev]) {
            CKN(launch_search_wide(plan.band[lev], lb, la, search_blocks_wide(plan.band[lev], lb, m), st));
        } else if (plan.elastic[lev]) {
            CKN(launch_search_elastic(lb, plan.band[lev], la, search_blocks_elastic(lb, plan.band[lev], m), st));
        } else {
            CKN(launch_search(plan.K[lev], plan.band[lev], lb, la, search_blocks(plan.K[lev], plan.band[lev], lb, m), st));
        }
    }
    CKN(launch_finalize(slots, k, out_idx, out_dist, st));
    int hi[kNumInts];
    CKN(cudaMemcpyAsync(hi, ints, sizeof(hi), cudaMemcpyDeviceToHost, st));
    CKN(cudaStreamSynchronize(st));
    if (hi[kBad]) return EAPDTW_ERR_NAN_INPUT;
    if (hi[kTimeout]) return EAPDTW_ERR_TIMEOUT;
    if (hi[kOvf0 + nlev - 1] > 0) return EAPDTW_ERR_UNSUPPORTED;
    return EAPDTW_OK;
}
