// DTW between whole series without an external upper bound (Section 2.3): the
// matrix of all pairwise distances, and k-nearest-neighbour (1-NN
// classification) search of test series among training series.
//
//  * Pairwise: every pair (a_i, b_j) runs EAPrunedDTW under its own diagonal
//    cost -- the squared Euclidean distance, the cost of one admissible warping
//    path and so an upper bound of the DTW (PrunedDTW's threshold) -- raised by
//    0.1% against FP32 rounding.  The result is the exact DTW; the bound only
//    prunes cells that cannot be on the optimal path.
//  * k-NN: each test series keeps a k-best list; every (test, training) pair
//    runs EAPrunedDTW against the test's current k-th best distance, the
//    tightest bound available, with no lower bounds (the nolb setting of
//    Section 5).
// One warp per pair, through the search's wavefront (dtw_wavefront.cuh) with a
// window of blocks wide enough for the whole series, so no pair overflows.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "common.cuh"
#include "dtw_wavefront.cuh"
#include "eapdtw.h"

namespace eapdtw {

namespace {

constexpr int kPairWarps = 8;

// z-normalise (znorm = 1) or copy each series of length len (one warp per
// series; two-pass FP64 mean and population variance; a constant series
// normalises to zeros).  bad: set when a value is not finite.
__global__ void pairs_prep_kernel(const float* __restrict__ X, int64_t count, int len, int znorm, float* Z,
                                  int* bad) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < count; s += warps) {
        const float* x = X + s * len;
        float* z = Z + s * len;
        double sum = 0.0;
        bool fin = true;
        for (int j = lane; j < len; j += 32) {
            fin &= isfinite(x[j]);
            sum = __dadd_rn(sum, static_cast<double>(x[j]));
        }
        if (__any_sync(kFull, !fin) && lane == 0) atomicOr(bad, 1);
        if (!znorm) {
            for (int j = lane; j < len; j += 32) z[j] = x[j];
            continue;
        }
        for (int o = 16; o > 0; o >>= 1) sum = __dadd_rn(sum, __shfl_xor_sync(kFull, sum, o));
        const double mean = __ddiv_rn(sum, static_cast<double>(len));
        double v = 0.0;
        for (int j = lane; j < len; j += 32) {
            const double d = __dsub_rn(static_cast<double>(x[j]), mean);
            v = __fma_rn(d, d, v);
        }
        for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, o));
        const double var = __ddiv_rn(v, static_cast<double>(len));
        const double sd = var > 0.0 ? __dsqrt_rn(var) : 0.0;
        for (int j = lane; j < len; j += 32)
            z[j] = sd > 0.0 ? __double2float_rn(__ddiv_rn(__dsub_rn(static_cast<double>(x[j]), mean), sd)) : 0.0f;
    }
}

// Squared Euclidean distance of two series (the diagonal path), on one warp.
__device__ __forceinline__ float diagonal_cost(const float* a, const float* b, int len) {
    const int lane = threadIdx.x & 31;
    float s = 0.0f;
    for (int j = lane; j < len; j += 32) {
        const float d = __fsub_rn(a[j], b[j]);
        s = __fmaf_rn(d, d, s);
    }
    for (int o = 16; o > 0; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(kFull, s, o));
    return s;
}

// The window of blocks covers every column: K = 8 up to 256 points, K = 32 up
// to 1024, then two or four windows of K = 32 with the column values streamed.
template <int K, int J>
__device__ __forceinline__ DtwOut pair_dtw(const float* rows, const float* cols, int len, int w, float ub) {
    BestSoFar fixed{nullptr, nullptr, 1, 1, ub};
    return dtw_warp<K, 2, J, (J > 1)>(rows, 0.0f, 0.0f, 1.0f, cols, len, len, w, fixed, ub);
}

template <int K, int J>
__global__ void __launch_bounds__(kPairWarps * 32) pairwise_kernel(const float* __restrict__ A, int64_t na,
                                                                   const float* __restrict__ B, int64_t nb, int len,
                                                                   int w, double* out, unsigned long long* work) {
    const int lane = threadIdx.x & 31;
    const int64_t total = na * nb;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(work, 1ull);
        u = __shfl_sync(kFull, u, 0);
        if (static_cast<int64_t>(u) >= total) break;
        const int64_t i = static_cast<int64_t>(u) / nb, j = static_cast<int64_t>(u) % nb;
        const float* a = A + i * len;
        const float* b = B + j * len;
        const float ed = __shfl_sync(kFull, diagonal_cost(a, b, len), 0);
        // every warping path costs at least the DTW, and the diagonal is one
        float ub = __fmaf_rn(ed, 1.0e-3f, ed);
        DtwOut o = pair_dtw<K, J>(a, b, len, w, ub);
        if (!(o.dist < f_inf())) o = pair_dtw<K, J>(a, b, len, w, f_inf());   // rounding beyond the margin
        if (lane == 0) out[i * nb + j] = static_cast<double>(o.dist);
    }
}

template <int K, int J>
__global__ void __launch_bounds__(kPairWarps * 32) nn_kernel(const float* __restrict__ train, int64_t ntrain,
                                                             const float* __restrict__ test, int64_t ntest, int len,
                                                             int w, int k, unsigned long long* slots,
                                                             const float* no_seed, unsigned long long* work) {
    const int lane = threadIdx.x & 31;
    // units: (training block of 32 series, test series), test fastest, so every
    // test series gets its first candidates early
    const int64_t nblk = (ntrain + 31) / 32;
    const int64_t total = nblk * ntest;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(work, 1ull);
        u = __shfl_sync(kFull, u, 0);
        if (static_cast<int64_t>(u) >= total) break;
        const int64_t t = static_cast<int64_t>(u) % ntest, blk = static_cast<int64_t>(u) / ntest;
        const BestSoFar bsf{slots + t * EAPDTW_MAX_K, no_seed, k, 0, 0.0f};   // no_seed: +inf in global memory
        const float* q = test + t * len;
        const int64_t j0 = blk * 32;
        const int64_t j1 = j0 + 32 < ntrain ? j0 + 32 : ntrain;
        // Lane l first checks the corner of training series j0 + l (rows and
        // columns 1..kCorner) against the test's current k-th best; the warp
        // then runs the survivors.
        bool alive = j0 + lane < j1;
        if (alive && len >= kCorner && w >= kCorner - 1)
            alive = !corner_dead<kCostSquared>(train + (j0 + lane) * len, 0.0f, 0.0f, 1.0f, q, bsf.load());
        unsigned mask = __ballot_sync(kFull, alive);
        while (mask) {
            const int64_t j = j0 + (__ffs(mask) - 1);
            mask &= mask - 1;
            const float ub = __shfl_sync(kFull, bsf.load(), 0);   // one reading for the whole warp
            const DtwOut o = dtw_warp<K, 2, J, (J > 1)>(train + j * len, 0.0f, 0.0f, 1.0f, q, len, len, w, bsf, ub);
            if (lane == 0 && o.dist < f_inf() && o.dist <= ub) bsf.insert(o.dist, static_cast<uint32_t>(j));
        }
    }
}

__global__ void nn_init_kernel(unsigned long long* slots, int64_t n, float* no_seed) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *no_seed = f_inf();
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        slots[i] = kEmptyKey;
}

__global__ void nn_finalize_kernel(const unsigned long long* slots, int64_t ntest, int k, int64_t* idx, double* dist) {
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < ntest * k;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const unsigned long long key = slots[(g / k) * EAPDTW_MAX_K + g % k];
        idx[g] = key == kEmptyKey ? -1 : static_cast<int64_t>(key & 0xffffffffull);
        dist[g] = key == kEmptyKey ? __longlong_as_double(0x7ff0000000000000ll)
                                   : static_cast<double>(__uint_as_float(static_cast<uint32_t>(key >> 32)));
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <typename F>
int blocks_of(F kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPairWarps * 32, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * sm_count();
}

// Scratch of a call (released at its end): normalised copies, counters, slots.
struct PairScratch {
    float* za = nullptr;
    float* zb = nullptr;
    unsigned long long* ints = nullptr;   // [0] work, [1] bad flag
    unsigned long long* slots = nullptr;
    ~PairScratch() {
        if (za) cudaFree(za);
        if (zb) cudaFree(zb);
        if (ints) cudaFree(ints);
        if (slots) cudaFree(slots);
    }
};

int32_t check_len(int64_t len, int64_t w) {
    if (len < 1 || w < 0) return EAPDTW_ERR_INVALID_ARG;
    if (len > EAPDTW_MAX_QUERY) return EAPDTW_ERR_UNSUPPORTED;
    return EAPDTW_OK;
}

int32_t prep(const float* X, int64_t count, int len, int znorm, float** Z, unsigned long long* ints, cudaStream_t st) {
    if (cudaMalloc(reinterpret_cast<void**>(Z), sizeof(float) * static_cast<size_t>(count * len)) != cudaSuccess) {
        cudaGetLastError();
        *Z = nullptr;
        return EAPDTW_ERR_OUT_OF_MEMORY;
    }
    pairs_prep_kernel<<<sm_count() * 4, 256, 0, st>>>(X, count, len, znorm, *Z, reinterpret_cast<int*>(ints + 1));
    return cudaGetLastError() == cudaSuccess ? EAPDTW_OK : EAPDTW_ERR_CUDA;
}

#define CKP(expr)                    \
    do {                             \
        if ((expr) != cudaSuccess) { \
            cudaGetLastError();      \
            return EAPDTW_ERR_CUDA;  \
        }                            \
    } while (0)

}  // namespace

}  // namespace eapdtw

using namespace eapdtw;

extern "C" {

int32_t eapdtw_pairwise(const float* A, int64_t na, const float* B, int64_t nb, int64_t len, int64_t w, int32_t znorm,
                        double* out, void* stream) {
    if (!A || !B || !out || na < 1 || nb < 1) return EAPDTW_ERR_INVALID_ARG;
    int32_t rc = check_len(len, w);
    if (rc != EAPDTW_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int L = static_cast<int>(len);
    const int wi = static_cast<int>(w < len ? w : len);
    PairScratch S;
    if (cudaMalloc(reinterpret_cast<void**>(&S.ints), 64) != cudaSuccess) {
        cudaGetLastError();
        return EAPDTW_ERR_OUT_OF_MEMORY;
    }
    CKP(cudaMemsetAsync(S.ints, 0, 64, st));
    if ((rc = prep(A, na, L, znorm, &S.za, S.ints, st)) != EAPDTW_OK) return rc;
    if ((rc = prep(B, nb, L, znorm, &S.zb, S.ints, st)) != EAPDTW_OK) return rc;
    if (L <= 256) {
        pairwise_kernel<8, 1><<<blocks_of(pairwise_kernel<8, 1>), kPairWarps * 32, 0, st>>>(S.za, na, S.zb, nb, L, wi,
                                                                                            out, S.ints);
    } else if (L <= 1024) {
        pairwise_kernel<32, 1><<<blocks_of(pairwise_kernel<32, 1>), kPairWarps * 32, 0, st>>>(S.za, na, S.zb, nb, L,
                                                                                              wi, out, S.ints);
    } else if (L <= 2048) {
        pairwise_kernel<32, 2><<<blocks_of(pairwise_kernel<32, 2>), kPairWarps * 32, 0, st>>>(S.za, na, S.zb, nb, L,
                                                                                              wi, out, S.ints);
    } else {
        pairwise_kernel<32, 4><<<blocks_of(pairwise_kernel<32, 4>), kPairWarps * 32, 0, st>>>(S.za, na, S.zb, nb, L,
                                                                                              wi, out, S.ints);
    }
    CKP(cudaGetLastError());
    int bad = 0;
    CKP(cudaMemcpyAsync(&bad, S.ints + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKP(cudaStreamSynchronize(st));
    return bad ? EAPDTW_ERR_NAN_INPUT : EAPDTW_OK;
}

int32_t eapdtw_nn(const float* train, int64_t ntrain, const float* test, int64_t ntest, int64_t len, int64_t w,
                  int32_t k, int32_t znorm, int64_t* out_idx, double* out_dist, void* stream) {
    if (!train || !test || !out_idx || !out_dist || ntrain < 1 || ntest < 1 || k < 1) return EAPDTW_ERR_INVALID_ARG;
    if (k > EAPDTW_MAX_K || ntrain >= (int64_t(1) << 32)) return EAPDTW_ERR_UNSUPPORTED;
    int32_t rc = check_len(len, w);
    if (rc != EAPDTW_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int L = static_cast<int>(len);
    const int wi = static_cast<int>(w < len ? w : len);
    PairScratch S;
    if (cudaMalloc(reinterpret_cast<void**>(&S.ints), 64) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&S.slots), sizeof(unsigned long long) * ntest * EAPDTW_MAX_K) !=
            cudaSuccess) {
        cudaGetLastError();
        return EAPDTW_ERR_OUT_OF_MEMORY;
    }
    CKP(cudaMemsetAsync(S.ints, 0, 64, st));
    float* no_seed = reinterpret_cast<float*>(S.ints + 2);
    nn_init_kernel<<<sm_count(), 256, 0, st>>>(S.slots, ntest * EAPDTW_MAX_K, no_seed);
    CKP(cudaGetLastError());
    if ((rc = prep(train, ntrain, L, znorm, &S.za, S.ints, st)) != EAPDTW_OK) return rc;
    if ((rc = prep(test, ntest, L, znorm, &S.zb, S.ints, st)) != EAPDTW_OK) return rc;
    if (L <= 256) {
        nn_kernel<8, 1><<<blocks_of(nn_kernel<8, 1>), kPairWarps * 32, 0, st>>>(S.za, ntrain, S.zb, ntest, L, wi, k,
                                                                                S.slots, no_seed, S.ints);
    } else if (L <= 1024) {
        nn_kernel<32, 1><<<blocks_of(nn_kernel<32, 1>), kPairWarps * 32, 0, st>>>(S.za, ntrain, S.zb, ntest, L, wi, k,
                                                                                  S.slots, no_seed, S.ints);
    } else if (L <= 2048) {
        nn_kernel<32, 2><<<blocks_of(nn_kernel<32, 2>), kPairWarps * 32, 0, st>>>(S.za, ntrain, S.zb, ntest, L, wi, k,
                                                                                  S.slots, no_seed, S.ints);
    } else {
        nn_kernel<32, 4><<<blocks_of(nn_kernel<32, 4>), kPairWarps * 32, 0, st>>>(S.za, ntrain, S.zb, ntest, L, wi, k,
                                                                                  S.slots, no_seed, S.ints);
    }
    CKP(cudaGetLastError());
    nn_finalize_kernel<<<sm_count(), 256, 0, st>>>(S.slots, ntest, k, out_idx, out_dist);
    CKP(cudaGetLastError());
    int bad = 0;
    CKP(cudaMemcpyAsync(&bad, S.ints + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKP(cudaStreamSynchronize(st));
    return bad ? EAPDTW_ERR_NAN_INPUT : EAPDTW_OK;
}

}  // extern "C"
