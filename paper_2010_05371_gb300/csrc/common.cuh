// Shared device-side definitions of the EAPrunedDTW search library (sm_103a).
//
// Method: Herrmann & Webb, "Early Abandoning PrunedDTW and its application to
// similarity search" (arXiv 2010.05371).  Cost (a - b)^2 and the recurrence of
// Eq. 1-5; window |i - j| <= w (Section 2.1); best-so-far / early abandoning
// (Section 2.2); UCR-Suite search loop with z-normalised windows (Section 5).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace eapdtw {

// ---------------------------------------------------------------------------
// Window statistics.  The reference is cut into chunks of kChunk points; each
// chunk has an anchor (its first value) and FP64 prefix sums of (x - anchor)
// and (x - anchor)^2 restarted at the chunk start, so that sums over a window
// are differences of numbers of the window's own magnitude rather than of the
// whole series (plain running sums over 1e7-1e8 points lose digits).
// ---------------------------------------------------------------------------
constexpr int kChunkLog = 12;
constexpr int kChunk = 1 << kChunkLog;

struct RefView {
    const float* R;     // [n] raw series
    int64_t n;
    const double* P1;   // [n]  sum of (x - A[c]) over chunk c before index i
    const double* P2;   // [n]  same for (x - A[c])^2
    const double* T1;   // [nchunks] chunk totals
    const double* T2;
    const float* A;     // [nchunks] chunk anchors
};

// Query staging: z-normalised query and its +-w envelope (LB_Keogh EQ), with
// the lower-bound terms visited in decreasing |zq| order (largest terms first,
// so that early exit triggers sooner).
struct QueryView {
    const float* zq;    // [m]
    const float* uq_o;  // [m] upper envelope, LB order
    const float* lq_o;  // [m] lower envelope, LB order
    const float* zq_o;  // [m] zq, LB order
    const int* ord;     // [m] column index of LB position p
    int m;
};

// Best-so-far list: k slots of packed keys (float bits of the distance << 32 |
// window index), ascending.  Non-negative floats order like their bit
// patterns, so one 64-bit atomicMin orders by (distance, index): a distance tie
// goes to the smaller index.
constexpr unsigned long long kEmptyKey = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ unsigned long long pack_key(float d, uint32_t idx) {
    return (static_cast<unsigned long long>(__float_as_uint(d)) << 32) | idx;
}

__device__ __forceinline__ float key_dist(unsigned long long key) {
    return key == kEmptyKey ? __int_as_float(0x7f800000) : __uint_as_float(static_cast<uint32_t>(key >> 32));
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ float ld_relaxed_f32(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}

struct BestSoFar {
    unsigned long long* slots;  // [k]
    const float* ub_seed;       // upper bound from sampled candidates (+inf if none)
    int k;
    int audit;                  // 1: ub is held at ub_fixed
    float ub_fixed;

    // Current upper bound: the k-th best distance so far, bounded by the seed.
    __device__ __forceinline__ float load() const {
        if (audit) return ub_fixed;
        float u = key_dist(ld_relaxed_u64(slots + (k - 1)));
        float s = ld_relaxed_f32(ub_seed);
        return fminf(u, s);
    }

    // The same reading split in two, so that the loads' latency can pass
    // under other work: issue() reads the k-th key and the seed without using
    // them; finish() turns that reading into the bound load() would return.
    struct Raw {
        unsigned long long key;
        float seed;
    };
    __device__ __forceinline__ Raw issue() const {
        if (audit) return Raw{kEmptyKey, ub_fixed};
        return Raw{ld_relaxed_u64(slots + (k - 1)), ld_relaxed_f32(ub_seed)};
    }
    __device__ __forceinline__ static Raw of(float ub) { return Raw{kEmptyKey, ub}; }
    __device__ __forceinline__ static float finish(Raw r) { return fminf(key_dist(r.key), r.seed); }

    // Insert (d, idx): a chain of atomicMin over the sorted slots.  Each slot
    // keeps the smaller of (its value, the carried key) and the larger one is
    // carried on, so slot s ends as the (s+1)-th smallest key ever inserted,
    // whatever the interleaving of concurrent inserters.
    __device__ __forceinline__ void insert(float d, uint32_t idx) const {
        unsigned long long carry = pack_key(d, idx);
        for (int s = 0; s < k; ++s) {
            unsigned long long old = atomicMin(slots + s, carry);
            if (old == kEmptyKey || old == carry) break;  // empty slot, or already listed
            carry = old > carry ? old : carry;
        }
    }
};

// Counter indices (must match include/eapdtw.h).
enum Counter : int {
    kCntWindows = 0,
    kCntKim = 1,
    kCntEq = 2,
    kCntEc = 3,
    kCntAbandoned = 4,
    kCntCompleted = 5,
    kCntCells = 6,
    kCntRecheck = 7,
    kCntOverflow = 8,
    kCntSteps = 9,
    kNumCounters = 16
};

// Window moments from the chunk-anchored sums: mean, population variance and
// the anchored second moment (the scale of the cancellation error of var).
// Every FP64 operation of the statistics is an explicit round-to-nearest
// intrinsic, so that the operation sequence (and an emulation of it) is fixed
// whatever the compiler's contraction settings.
__device__ __forceinline__ void window_moments(const RefView& ref, int64_t i, int m, double& mean,
                                               double& var, double& m2anch) {
    const int64_t end = i + m;
    int64_t c0 = i >> kChunkLog;
    const double a0 = static_cast<double>(ref.A[c0]);
    double s1 = 0.0, s2 = 0.0;
    int64_t lo = i;
    for (int64_t c = c0; lo < end; ++c) {
        const int64_t cend = ((c + 1) << kChunkLog) < ref.n ? ((c + 1) << kChunkLog) : ref.n;
        const int64_t hi = end < cend ? end : cend;
        const double e1 = (hi == cend) ? ref.T1[c] : ref.P1[hi];
        const double e2 = (hi == cend) ? ref.T2[c] : ref.P2[hi];
        const double p1 = __dsub_rn(e1, ref.P1[lo]);
        const double p2 = __dsub_rn(e2, ref.P2[lo]);
        const double cnt = static_cast<double>(hi - lo);
        const double dl = __dsub_rn(static_cast<double>(ref.A[c]), a0);  // re-anchor to a0
        // sum (x - a0) = p1 + cnt dl;  sum (x - a0)^2 = p2 + dl (2 p1 + cnt dl)
        s1 = __dadd_rn(s1, __fma_rn(cnt, dl, p1));
        s2 = __dadd_rn(s2, __fma_rn(dl, __fma_rn(cnt, dl, __dmul_rn(2.0, p1)), p2));
        lo = hi;
    }
    const double mu1 = __ddiv_rn(s1, static_cast<double>(m));
    mean = __dadd_rn(a0, mu1);
    m2anch = __ddiv_rn(s2, static_cast<double>(m));
    var = __dsub_rn(m2anch, __dmul_rn(mu1, mu1));
}

// Window-anchored z coefficients: z(x) = ((x - a) - cw) * isd with a the
// window's first value, cw = fl32(mean - a), isd = fl32(1 / sd).  The two
// subtractions stay at the window's scale, so z keeps FP32 relative accuracy
// even when |mean| >> sd.  A window with zero variance normalises to zeros
// (isd = 0).  When the variance is small against the anchored second moment
// (cancellation), mean and variance are recomputed two-pass from the window.
__device__ __forceinline__ void window_coeffs(const RefView& ref, int64_t i, int m,
                                              const float* x /* x[0..m) = R[i..i+m) */, float& a,
                                              float& cw, float& isd) {
    double mean, var, m2a;
    window_moments(ref, i, m, mean, var, m2a);
    a = x[0];
    if (!(var > __dmul_rn(1e-6, m2a))) {
        double s = 0.0;
        for (int p = 0; p < m; ++p) s = __dadd_rn(s, static_cast<double>(x[p]));
        mean = __ddiv_rn(s, static_cast<double>(m));
        double v = 0.0;
        for (int p = 0; p < m; ++p) {
            const double d = __dsub_rn(static_cast<double>(x[p]), mean);
            v = __fma_rn(d, d, v);
        }
        var = __ddiv_rn(v, static_cast<double>(m));
    }
    const float var32 = __double2float_rn(var);
    if (var32 > 0.0f) {
        isd = __frsqrt_rn(var32);
        cw = __double2float_rn(__dsub_rn(mean, static_cast<double>(a)));
    } else {
        isd = 0.0f;
        cw = 0.0f;
    }
}

// Optional device self-checks (build with -DEAPDTW_DEVICE_CHECKS): a failed
// check records (code, value) in dbg[0..2] (first failure wins) and the caller
// skips the access it guards.  Off by default.
#ifdef EAPDTW_DEVICE_CHECKS
#define EAPDTW_CHECK(dbg, ok, code, value)                                   \
    ((ok) ? true                                                             \
          : ((dbg) && atomicCAS((dbg), 0, (code)) == 0 ? ((dbg)[1] = (int)(value), false) : false))
#else
#define EAPDTW_CHECK(dbg, ok, code, value) true
#endif

// min(a, b, c) in one instruction (the three-operand min.f32 of sm_100 and
// later).  Like fminf it ignores a NaN operand; the result is exact, so it
// equals fminf(fminf(a, b), c) for every input of the DTW recurrence.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float znorm1(float x, float a, float cw, float isd) {
    return __fmul_rn(__fsub_rn(__fsub_rn(x, a), cw), isd);
}

}  // namespace eapdtw
