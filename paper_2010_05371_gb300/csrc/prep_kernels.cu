// Preparation kernels of the search (sm_103a): window statistics of the
// reference, query normalisation and envelope, reference envelope for
// LB_Keogh EC, the sampled upper-bound seed, and result conversion.
#include <cfloat>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "search_kernel.cuh"
#include "batch.cuh"

namespace eapdtw {

// ---------------------------------------------------------------------------
// Chunk-anchored FP64 prefix sums (one block of 256 threads per 4096-point
// chunk; each thread sums 16 consecutive points sequentially, then a block
// scan of the 256 partial sums).  Also flags non-finite input values.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ref_prefix_kernel(const float* __restrict__ R, int64_t n,
                                                         double* P1, double* P2, double* T1,
                                                         double* T2, float* A, int* bad) {
    constexpr int kPer = kChunk / 256;
    const int64_t c = blockIdx.x;
    const int64_t base = c << kChunkLog;
    const int64_t len = n - base < kChunk ? n - base : kChunk;
    const int tid = threadIdx.x;
    const float anchor = R[base];
    const double a = static_cast<double>(anchor);
    double s1 = 0.0, s2 = 0.0;
    bool finite = true;
    double d[kPer];
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const int64_t j = tid * kPer + e;
        float x = j < len ? R[base + j] : anchor;
        finite &= isfinite(x);
        d[e] = __dsub_rn(static_cast<double>(x), a);
        s1 = __dadd_rn(s1, d[e]);
        s2 = __fma_rn(d[e], d[e], s2);
    }
    if (!finite) atomicOr(bad, 1);
    // block exclusive scan of (s1, s2)
    __shared__ double w1[8], w2[8];
    const int lane = tid & 31, warp = tid >> 5;
    double i1 = s1, i2 = s2;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u1 = __shfl_up_sync(0xffffffffu, i1, o);
        const double u2 = __shfl_up_sync(0xffffffffu, i2, o);
        if (lane >= o) {
            i1 = __dadd_rn(i1, u1);
            i2 = __dadd_rn(i2, u2);
        }
    }
    if (lane == 31) { w1[warp] = i1; w2[warp] = i2; }
    __syncthreads();
    double b1 = 0.0, b2 = 0.0;
    for (int q = 0; q < warp; ++q) {
        b1 = __dadd_rn(b1, w1[q]);
        b2 = __dadd_rn(b2, w2[q]);
    }
    // exclusive prefix of this thread
    double r1 = __dsub_rn(__dadd_rn(b1, i1), s1), r2 = __dsub_rn(__dadd_rn(b2, i2), s2);
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const int64_t j = tid * kPer + e;
        if (j < len) {
            P1[base + j] = r1;
            P2[base + j] = r2;
        }
        r1 = __dadd_rn(r1, d[e]);
        r2 = __fma_rn(d[e], d[e], r2);
    }
    if (tid == 255) {
        // padded points contribute d = 0
        T1[c] = r1;
        T2[c] = r2;
        A[c] = anchor;
    }
}

// ---------------------------------------------------------------------------
// Query preparation (one block of 1024 threads): two-pass FP64 mean and
// population variance, zq = (q - mean) / sd (zeros if sd == 0), the envelope
// U/L of zq over +-w clipped to the query (LB_Keogh EQ), and the order of
// positions by decreasing |zq| (ties by position) used to visit LB terms.
// Arrays are padded to query_pad(m) with neutral terms.
// ---------------------------------------------------------------------------
// Body shared by the one-query kernel and the batch kernel (sm: dynamic
// shared memory of query_prep_smem(m) bytes; all threads of the block call it).
__device__ void query_prep_block(const float* __restrict__ Q, int m, int w, float* zq, float* uq_o,
                                 float* lq_o, float* zq_o, int* ord, int* bad, unsigned char* sm) {
    const int tid = threadIdx.x;
    const int np2 = 1 << (32 - __clz(m - 1 > 0 ? m - 1 : 1));  // next pow2 >= m (>= 2)
    float* s_z = reinterpret_cast<float*>(sm);                // [m]
    float* s_u = s_z + m;                                     // [m]
    float* s_l = s_u + m;                                     // [m]
    unsigned long long* s_key = reinterpret_cast<unsigned long long*>(s_l + m + (m & 1));  // [np2]
    __shared__ double red[32];
    __shared__ int s_bad;
    if (tid == 0) s_bad = 0;
    __syncthreads();

    // block sum: a thread's strided terms in order, a butterfly over the warp
    // (every lane ends with the same value), then the warps' sums in order
    auto block_sum = [&](double v) -> double {
        for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = __dadd_rn(t, red[q]);
        return t;
    };
    double s = 0.0;
    for (int j = tid; j < m; j += blockDim.x) {
        const float x = Q[j];
        if (!isfinite(x)) s_bad = 1;
        s = __dadd_rn(s, static_cast<double>(x));
    }
    const double mean = __ddiv_rn(block_sum(s), static_cast<double>(m));
    double v = 0.0;
    for (int j = tid; j < m; j += blockDim.x) {
        const double dx = __dsub_rn(static_cast<double>(Q[j]), mean);
        v = __fma_rn(dx, dx, v);
    }
    const double var = __ddiv_rn(block_sum(v), static_cast<double>(m));
    const double sd = var > 0.0 ? __dsqrt_rn(var) : 0.0;
    for (int j = tid; j < m; j += blockDim.x) {
        const float z = sd > 0.0 ? __double2float_rn(__ddiv_rn(__dsub_rn(static_cast<double>(Q[j]), mean), sd))
                                 : 0.0f;
        s_z[j] = z;
        zq[j] = z;
    }
    __syncthreads();
    if (tid == 0 && s_bad) atomicOr(bad, 2);
    // envelope over [j - w, j + w] clipped to [0, m)
    const int wc = w < m - 1 ? w : m - 1;
    for (int j = tid; j < m; j += blockDim.x) {
        const int lo = j - wc > 0 ? j - wc : 0;
        const int hi = j + wc < m - 1 ? j + wc : m - 1;
        float u = s_z[lo], l = s_z[lo];
        for (int k = lo + 1; k <= hi; ++k) {
            u = fmaxf(u, s_z[k]);
            l = fminf(l, s_z[k]);
        }
        s_u[j] = u;
        s_l[j] = l;
    }
    // bitonic sort of keys (descending |zq|, then ascending position)
    for (int j = tid; j < np2; j += blockDim.x) {
        unsigned long long key = ~0ull;
        if (j < m) {
            const unsigned mag = __float_as_uint(fabsf(s_z[j]));  // order of |zq|
            key = (static_cast<unsigned long long>(~mag) << 32) | static_cast<unsigned>(j);
        }
        s_key[j] = key;
    }
    __syncthreads();
    for (int size = 2; size <= np2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int j = tid; j < np2; j += blockDim.x) {
                const int p = j ^ stride;
                if (p > j) {
                    const bool up = (j & size) == 0;
                    const unsigned long long x = s_key[j], y = s_key[p];
                    if ((x > y) == up) {
                        s_key[j] = y;
                        s_key[p] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int mp = query_pad(m);
    for (int p = tid; p < mp; p += blockDim.x) {
        if (p < m) {
            const int j = static_cast<int>(s_key[p] & 0xffffffffu);
            ord[p] = j;
            uq_o[p] = s_u[j];
            lq_o[p] = s_l[j];
            zq_o[p] = s_z[j];
        } else {
            ord[p] = 0;
            uq_o[p] = __int_as_float(0x7f800000);
            lq_o[p] = __int_as_float(0xff800000);
            zq_o[p] = __int_as_float(0x7fffffff);
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) query_prep_kernel(const float* __restrict__ Q, int m, int w,
                                                          float* zq, float* uq_o, float* lq_o,
                                                          float* zq_o, int* ord, int* bad) {
    extern __shared__ __align__(16) unsigned char sm[];
    query_prep_block(Q, m, w, zq, uq_o, lq_o, zq_o, ord, bad, sm);
}

size_t query_prep_smem(int m) {
    int np2 = 2;
    while (np2 < m) np2 <<= 1;
    return sizeof(float) * (3 * static_cast<size_t>(m) + (m & 1)) + sizeof(unsigned long long) * np2;
}

// ---------------------------------------------------------------------------
// Reference envelope for LB_Keogh EC: U[t] = max R[t-w .. t+w], L[t] = min,
// clipped to [0, n).  Each block owns kEnvTile outputs; it loads the tile plus
// a +-w halo (padded with -inf / +inf outside the series) into shared memory
// and builds sliding maxima by doubling: after pass p, M[s] = max of the 2^p
// values starting at s.  The window of 2w+1 values is then covered by two
// overlapping runs of length 2^p <= 2w+1.
// ---------------------------------------------------------------------------
constexpr int kEnvTile = 4096;

__global__ void __launch_bounds__(512) envelope_kernel(const float* __restrict__ R, int64_t n, int w,
                                                       float* U, float* L) {
    extern __shared__ __align__(16) float se[];
    const int span = kEnvTile + 2 * w;
    float* smax = se;
    float* smin = se + span;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * kEnvTile;
    const float NEG = __int_as_float(0xff800000), POS = __int_as_float(0x7f800000);
    for (int s = threadIdx.x; s < span; s += blockDim.x) {
        const int64_t g = t0 - w + s;
        const bool in = g >= 0 && g < n;
        const float x = in ? R[g] : 0.0f;
        smax[s] = in ? x : NEG;
        smin[s] = in ? x : POS;
    }
    __syncthreads();
    const int W = 2 * w + 1;
    int len = 1;
    while (2 * len <= W) {
        // M_{2len}[s] = max(M_len[s], M_len[s + len]) for s + 2len <= span
        const int lim = span - 2 * len + 1;
        for (int base = 0; base < lim; base += blockDim.x * 8) {
            float hx[8], lx[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int s = base + e * blockDim.x + threadIdx.x;
                if (s < lim) {
                    hx[e] = fmaxf(smax[s], smax[s + len]);
                    lx[e] = fminf(smin[s], smin[s + len]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int s = base + e * blockDim.x + threadIdx.x;
                if (s < lim) {
                    smax[s] = hx[e];
                    smin[s] = lx[e];
                }
            }
            __syncthreads();
        }
        len *= 2;
    }
    for (int t = threadIdx.x; t < kEnvTile; t += blockDim.x) {
        const int64_t g = t0 + t;
        if (g >= n) break;
        // window [t, t + 2w] in tile coordinates
        const float u = fmaxf(smax[t], smax[t + W - len]);
        const float l = fminf(smin[t], smin[t + W - len]);
        U[g] = u;
        L[g] = l;
    }
}

size_t envelope_smem(int w) { return sizeof(float) * 2 * (kEnvTile + 2 * static_cast<size_t>(w)); }
int envelope_blocks(int64_t n) { return static_cast<int>((n + kEnvTile - 1) / kEnvTile); }

// ---------------------------------------------------------------------------
// Sparse table of running extrema (LB_Keogh EC of the batched search): level
// p holds max / min of R[t .. min(t + 2^p, n)); level p comes from level p-1 as
// the extremum of two runs of 2^(p-1) values.
// ---------------------------------------------------------------------------
__global__ void env_level_kernel(const float* __restrict__ smax, const float* __restrict__ smin, int64_t n,
                                 int64_t half, float* dmax, float* dmin) {
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t u = t + half < n ? t + half : t;
        dmax[t] = fmaxf(smax[t], smax[u]);
        dmin[t] = fminf(smin[t], smin[u]);
    }
}

// ---------------------------------------------------------------------------
// The first-level probe's windows: ns indices spread evenly over [0, nw).
// ---------------------------------------------------------------------------
__global__ void probe_list_kernel(long long* list, int ns, int64_t nw, int* count) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < ns) list[s] = ns > 1 ? (nw - 1) * s / (ns - 1) : 0;
    if (s == 0) *count = ns;
}

// ---------------------------------------------------------------------------
// Search state initialisation.
// ---------------------------------------------------------------------------
__global__ void init_state_kernel(unsigned long long* slots, int k, float* ub_seed,
                                  unsigned long long* counters, int* ints, int nints) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) slots[j] = kEmptyKey;
    for (int j = threadIdx.x; j < kNumCounters; j += blockDim.x) counters[j] = 0;
    for (int j = threadIdx.x; j < nints; j += blockDim.x) ints[j] = 0;
    if (threadIdx.x == 0) *ub_seed = __int_as_float(0x7f800000);
}

// ---------------------------------------------------------------------------
// Upper-bound seed: the z-normalised squared Euclidean distance (the w = 0
// diagonal, an admissible warping path for every w >= 0) of sampled windows,
// one warp per sample.  ED(c) >= DTW_w(c), so the k-th smallest sampled ED
// bounds the k-th smallest DTW from above (the sampled windows are real
// candidates that the search will also visit).
// ---------------------------------------------------------------------------
// Sample gw of nsamples (spread evenly over the nw windows) on one warp.
// cost: kCostSquared sums (z - q)^2; kCostAbsolute sums |z - q| (the diagonal
// path's cost under the absolute cost, so the same argument bounds it).
__device__ __forceinline__ void seed_ed_sample(const RefView& ref, const float* __restrict__ zq, int m,
                                              int64_t nw, int nsamples, int gw, float* ed, int* idx, int cost = 0) {
    const int lane = threadIdx.x & 31;
    const int64_t i = nsamples > 1 ? (nw - 1) * gw / (nsamples - 1) : 0;
    const float* x = ref.R + i;
    double mean, var, m2a;
    window_moments(ref, i, m, mean, var, m2a);
    float a = x[0], cw = 0.0f, isd = 0.0f;
    const float v32 = static_cast<float>(var);
    if (v32 > 0.0f && var > 1e-6 * m2a) {
        isd = __frsqrt_rn(v32);
        cw = static_cast<float>(mean - static_cast<double>(a));
    }
    float s = 0.0f;
    for (int j = lane; j < m; j += 32) {
        const float d = __fsub_rn(znorm1(x[j], a, cw, isd), zq[j]);
        s = (cost == kCostAbsolute) ? __fadd_rn(s, fabsf(d)) : __fmaf_rn(d, d, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        // a window whose statistics need the exact path is left out of the seed
        ed[gw] = (isd > 0.0f) ? s : __int_as_float(0x7f800000);
        idx[gw] = static_cast<int>(i);
    }
}

__global__ void seed_ed_kernel(const RefView ref, const float* __restrict__ zq, int m, int64_t nw,
                               int nsamples, float* ed, int* idx, int cost) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= nsamples) return;
    seed_ed_sample(ref, zq, m, nw, nsamples, gw, ed, idx, cost);
}

// One block: ub_seed = the k-th smallest sampled ED (distinct windows; +inf if
// fewer than k are finite), raised by 0.1% so that FP32 rounding of the ED sum
// cannot place it below the DTW of its own window; also writes the windows of
// the `nbest` smallest samples (for an exact DTW pass that seeds the k-best list).
// Body shared by the one-query and batch kernels (all threads of the block
// call it; best entries are tag | window).
__device__ void seed_select_block(const float* ed, const int* idx, int ns, int k, float* ub_seed,
                                  long long* best, int nbest, int* nbest_out, long long tag) {
    __shared__ float s_v[64];
    __shared__ int s_i[64];
    __shared__ float r_v[32];
    __shared__ int r_i[32];
    const int tid = threadIdx.x;
    const float INF = __int_as_float(0x7f800000);
    const int nr = k > nbest ? k : nbest;   // <= 64
    int taken = 0;
    auto better = [](float v, int j, float bv, int bj) { return v < bv || (v == bv && j < bj); };
    for (int round = 0; round < nr; ++round) {
        float bv = INF;
        int bj = 0x7fffffff;
        for (int j = tid; j < ns; j += blockDim.x) {
            bool used = false;
            for (int q = 0; q < taken; ++q) used |= (s_i[q] == j);
            if (!used && better(ed[j], j, bv, bj)) { bv = ed[j]; bj = j; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (better(ov, oj, bv, bj)) { bv = ov; bj = oj; }
        }
        if ((tid & 31) == 0) { r_v[tid >> 5] = bv; r_i[tid >> 5] = bj; }
        __syncthreads();
        if (tid == 0) {
            float fv = r_v[0];
            int fj = r_i[0];
            for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
                if (better(r_v[q], r_i[q], fv, fj)) { fv = r_v[q]; fj = r_i[q]; }
            s_v[taken] = fv;
            s_i[taken] = fj;
        }
        __syncthreads();
        if (!(s_v[taken] < INF)) break;
        ++taken;
    }
    if (tid == 0) {
        const float kth = taken >= k ? s_v[k - 1] : INF;
        *ub_seed = kth < INF ? kth * 1.001f : INF;
        int nb = 0;
        for (int q = 0; q < taken && q < nbest; ++q) best[nb++] = tag | static_cast<long long>(idx[s_i[q]]);
        *nbest_out = nb;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) seed_select_kernel(const float* ed, const int* idx, int ns, int k,
                                                           float* ub_seed, long long* best, int nbest,
                                                           int* nbest_out) {
    seed_select_block(ed, idx, ns, k, ub_seed, best, nbest, nbest_out, 0);
}

// ---------------------------------------------------------------------------
// Results: slots -> (int64 index, double distance); empty -> (-1, +inf).
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(const unsigned long long* slots, int k, int64_t* out_idx,
                                double* out_dist) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const unsigned long long key = slots[j];
        if (key == kEmptyKey) {
            out_idx[j] = -1;
            out_dist[j] = __longlong_as_double(0x7ff0000000000000ll);
        } else {
            out_idx[j] = static_cast<int64_t>(key & 0xffffffffull);
            out_dist[j] = static_cast<double>(__uint_as_float(static_cast<uint32_t>(key >> 32)));
        }
    }
}

// ---------------------------------------------------------------------------
// Batch versions (fixed grids that loop over the items and query slots named
// in the device tables, so that one captured graph serves every batch).
// ---------------------------------------------------------------------------
__global__ void batch_init_kernel(BatchDev D, int cap_items, unsigned long long* counters, int ncounters,
                                  unsigned long long* work, int nwork, int* rr_counts, int nrr) {
    const int n = *D.nitems;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    // fresh items start from an empty state; the others keep theirs
    for (int64_t j = tid; j < static_cast<int64_t>(n) * kBatchSlots; j += stride) {
        const BatchItem& it = D.items[j / kBatchSlots];
        if (it.fresh) D.slots[static_cast<int64_t>(it.state) * kBatchSlots + j % kBatchSlots] = kEmptyKey;
    }
    for (int64_t j = tid; j < n; j += stride) {
        const BatchItem& it = D.items[j];
        if (it.fresh) {
            D.ub_seed[it.state] = __int_as_float(0x7f800000);
            D.nbest[it.state] = 0;
        }
        D.flags[it.state] = 0;
        D.cost[it.state] = 0;
    }
    for (int64_t j = tid; j < *D.nslots; j += stride) D.qbad[j] = 0;
    if (tid < ncounters) counters[tid] = 0;
    if (tid < nwork) work[tid] = 0;
    if (tid < nrr) rr_counts[tid] = 0;
    (void)cap_items;
}

__global__ void __launch_bounds__(1024) batch_query_prep_kernel(BatchDev D, int mp_cap) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int ns = *D.nslots;
    for (int q = blockIdx.x; q < ns; q += gridDim.x) {
        const QuerySlot S = D.qslots[q];
        const int mp = query_pad(S.m);
        float* base = D.qarena + S.off;
        query_prep_block(S.Q, S.m, S.w, base, base + mp, base + 2 * mp, base + 3 * mp,
                         reinterpret_cast<int*>(base + 4 * mp), D.qbad + q, sm);
    }
    (void)mp_cap;
}

// One warp per sample; sample g belongs to the item whose prefix range holds it.
__global__ void batch_seed_ed_kernel(BatchDev D) {
    const int n = *D.nitems;
    const int64_t total = D.sprefix[n];
    const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t g = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; g < total; g += warps) {
        int lo = 0, hi = n;  // sprefix[lo] <= g < sprefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (D.sprefix[mid] <= g) lo = mid;
            else hi = mid;
        }
        const BatchItem& it = D.items[lo];
        const int s = static_cast<int>(g - D.sprefix[lo]);
        seed_ed_sample(it.ref, it.zq, it.m, it.nw, it.seed_ns, s, D.seed_ed + it.seed_off, D.seed_idx + it.seed_off);
    }
}

__global__ void __launch_bounds__(1024) batch_seed_select_kernel(BatchDev D) {
    const int n = *D.nitems;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const BatchItem& it = D.items[i];
        if (it.seed_ns <= 0) continue;  // uniform over the block
        seed_select_block(D.seed_ed + it.seed_off, D.seed_idx + it.seed_off, it.seed_ns, it.k, D.ub_seed + it.state,
                          D.best + static_cast<int64_t>(it.state) * kBatchSeedBest, kBatchSeedBest,
                          D.nbest + it.state, static_cast<long long>(i) << 32);
    }
}

__global__ void batch_finalize_kernel(BatchDev D) {
    const int n = *D.nitems;
    const int ks = *D.kstride;
    const int64_t total = static_cast<int64_t>(n) * ks;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(g / ks);
        const int j = static_cast<int>(g % ks);
        const BatchItem& it = D.items[i];
        const unsigned long long key = j < it.k ? D.slots[static_cast<int64_t>(it.state) * kBatchSlots + j] : kEmptyKey;
        if (key == kEmptyKey) {
            D.res_idx[g] = -1;
            D.res_dist[g] = __longlong_as_double(0x7ff0000000000000ll);
        } else {
            D.res_idx[g] = static_cast<int64_t>(key & 0xffffffffull);
            D.res_dist[g] = static_cast<double>(__uint_as_float(static_cast<uint32_t>(key >> 32)));
        }
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers (declared in kernels.h).
// ---------------------------------------------------------------------------
cudaError_t launch_ref_prefix(const float* R, int64_t n, double* P1, double* P2, double* T1,
                              double* T2, float* A, int* bad, cudaStream_t s) {
    const int64_t nch = (n + kChunk - 1) / kChunk;
    ref_prefix_kernel<<<static_cast<unsigned>(nch), 256, 0, s>>>(R, n, P1, P2, T1, T2, A, bad);
    return cudaGetLastError();
}

cudaError_t launch_query_prep(const float* Q, int m, int w, float* zq, float* uq_o, float* lq_o,
                              float* zq_o, int* ord, int* bad, cudaStream_t s) {
    const size_t sm = query_prep_smem(m);
    cudaError_t e = cudaFuncSetAttribute(query_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    query_prep_kernel<<<1, 1024, sm, s>>>(Q, m, w, zq, uq_o, lq_o, zq_o, ord, bad);
    return cudaGetLastError();
}

cudaError_t launch_envelope(const float* R, int64_t n, int w, float* U, float* L, cudaStream_t s) {
    const size_t sm = envelope_smem(w);
    cudaError_t e = cudaFuncSetAttribute(envelope_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    envelope_kernel<<<envelope_blocks(n), 512, sm, s>>>(R, n, w, U, L);
    return cudaGetLastError();
}

cudaError_t launch_init_state(unsigned long long* slots, int k, float* ub_seed,
                              unsigned long long* counters, int* ints, int nints, cudaStream_t s) {
    init_state_kernel<<<1, 128, 0, s>>>(slots, k, ub_seed, counters, ints, nints);
    return cudaGetLastError();
}

cudaError_t launch_seed(const RefView& ref, const float* zq, int m, int64_t nw, int nsamples,
                        float* ed, int* idx, int k, float* ub_seed, long long* best, int nbest,
                        int* nbest_out, cudaStream_t s, int cost) {
    const int threads = 256;
    const int blocks = (nsamples * 32 + threads - 1) / threads;
    seed_ed_kernel<<<blocks, threads, 0, s>>>(ref, zq, m, nw, nsamples, ed, idx, cost);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    seed_select_kernel<<<1, 1024, 0, s>>>(ed, idx, nsamples, k, ub_seed, best, nbest, nbest_out);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const unsigned long long* slots, int k, int64_t* out_idx,
                            double* out_dist, cudaStream_t s) {
    finalize_kernel<<<1, 64, 0, s>>>(slots, k, out_idx, out_dist);
    return cudaGetLastError();
}

cudaError_t launch_batch_prep(const BatchDev& D, int cap_items, unsigned long long* counters, int ncounters,
                              unsigned long long* work, int nwork, int* rr_counts, int nrr, int m_cap,
                              cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    batch_init_kernel<<<sms * 4, 256, 0, s>>>(D, cap_items, counters, ncounters, work, nwork, rr_counts, nrr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t sm = query_prep_smem(m_cap);
    batch_query_prep_kernel<<<sms, 1024, sm, s>>>(D, query_pad(m_cap));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_seed_ed_kernel<<<sms * 8, 256, 0, s>>>(D);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_seed_select_kernel<<<sms, 1024, 0, s>>>(D);
    return cudaGetLastError();
}

cudaError_t launch_env_level(const float* smax, const float* smin, int64_t n, int64_t half, float* dmax,
                             float* dmin, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    env_level_kernel<<<sms * 8, 256, 0, s>>>(smax, smin, n, half, dmax, dmin);
    return cudaGetLastError();
}

cudaError_t launch_probe_list(long long* list, int ns, int64_t nw, int* count, cudaStream_t s) {
    probe_list_kernel<<<(ns + 255) / 256, 256, 0, s>>>(list, ns, nw, count);
    return cudaGetLastError();
}

cudaError_t batch_prep_attributes(int m_cap) {
    return cudaFuncSetAttribute(batch_query_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(query_prep_smem(m_cap)));
}

cudaError_t launch_batch_finalize(const BatchDev& D, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    batch_finalize_kernel<<<sms, 256, 0, s>>>(D);
    return cudaGetLastError();
}

}  // namespace eapdtw
