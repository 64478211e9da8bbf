// eap_dtw: EAPrunedDTW of one pair of raw series (Algorithm 3 contract) on one
// warp, through the same wavefront as the search (dtw_wavefront.cuh).
#include "dtw_wavefront.cuh"
#include "kernels.h"

namespace eapdtw {

// *out holds NaN until some level succeeds.  A level whose live region
// overflows its window of blocks leaves NaN for the next (wider) level; the
// last level leaves NaN if it overflows too.
template <int K, int BAND, bool WIDE>
__global__ void __launch_bounds__(32) pair_kernel(const float* __restrict__ rows, int nr,
                                                  const float* __restrict__ cols, int nc, int w,
                                                  float ub, double* out) {
    if (!isnan(*out)) return;  // an earlier level finished
    BestSoFar fixed{nullptr, nullptr, 1, 1, ub};
    constexpr int kJ = WIDE ? 4 : dtw_windows(K, BAND);
    const DtwOut o = dtw_warp<K, BAND, kJ, WIDE>(rows, 0.0f, 0.0f, 1.0f, cols, nr, nc, w, fixed, ub);
    if (threadIdx.x == 0 && o.status == 0) {
        *out = (o.dist <= ub) ? static_cast<double>(o.dist)
                              : __longlong_as_double(0x7ff0000000000000ll);
    }
}

template <int K, bool WIDE>
cudaError_t launch_pair_k(int band, const float* rows, int nr, const float* cols, int nc, int w, float ub,
                          double* out, cudaStream_t s) {
    if (band == 0) pair_kernel<K, 0, WIDE><<<1, 32, 0, s>>>(rows, nr, cols, nc, w, ub, out);
    else if (band == 1) pair_kernel<K, 1, WIDE><<<1, 32, 0, s>>>(rows, nr, cols, nc, w, ub, out);
    else pair_kernel<K, 2, WIDE><<<1, 32, 0, s>>>(rows, nr, cols, nc, w, ub, out);
    return cudaGetLastError();
}

// The four-window variant compiles as its own unit (EAPDTW_UNIT_PAIR_WIDE,
// see build.py); the narrow ones and the dispatcher in the other.
#ifdef EAPDTW_UNIT_PAIR_WIDE

template cudaError_t launch_pair_k<32, true>(int, const float*, int, const float*, int, int, float, double*,
                                             cudaStream_t);

#else

extern template cudaError_t launch_pair_k<32, true>(int, const float*, int, const float*, int, int, float,
                                                    double*, cudaStream_t);

cudaError_t launch_pair(int K, int band, bool wide, const float* rows, int nr, const float* cols, int nc,
                        int w, float ub, double* out, cudaStream_t s) {
    if (wide) return launch_pair_k<32, true>(band, rows, nr, cols, nc, w, ub, out, s);
    switch (K) {
        case 4: return launch_pair_k<4, false>(band, rows, nr, cols, nc, w, ub, out, s);
        case 8: return launch_pair_k<8, false>(band, rows, nr, cols, nc, w, ub, out, s);
        case 16: return launch_pair_k<16, false>(band, rows, nr, cols, nc, w, ub, out, s);
        default: return launch_pair_k<32, false>(band, rows, nr, cols, nc, w, ub, out, s);
    }
}

#endif

}  // namespace eapdtw
