// Host-side launchers shared between the CUDA translation units of the library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace eapdtw {

struct SearchArgs;
struct BatchDev;
struct BatchLaunch;

cudaError_t launch_ref_prefix(const float* R, int64_t n, double* P1, double* P2, double* T1,
                              double* T2, float* A, int* bad, cudaStream_t s);
cudaError_t launch_query_prep(const float* Q, int m, int w, float* zq, float* uq_o, float* lq_o,
                              float* zq_o, int* ord, int* bad, cudaStream_t s);
cudaError_t launch_envelope(const float* R, int64_t n, int w, float* U, float* L, cudaStream_t s);
cudaError_t launch_init_state(unsigned long long* slots, int k, float* ub_seed,
                              unsigned long long* counters, int* ints, int nints, cudaStream_t s);
cudaError_t launch_seed(const RefView& ref, const float* zq, int m, int64_t nw, int nsamples,
                        float* ed, int* idx, int k, float* ub_seed, long long* best, int nbest,
                        int* nbest_out, cudaStream_t s, int cost = 0);
cudaError_t launch_finalize(const unsigned long long* slots, int k, int64_t* out_idx,
                            double* out_dist, cudaStream_t s);
// ns window indices spread evenly over [0, nw) into list; *count = ns.
cudaError_t launch_probe_list(long long* list, int ns, int64_t nw, int* count, cudaStream_t s);

// search_kernel<K, BAND, LB> for K in {4, 8, 16, 32}, BAND in {0, 1, 2} and
// LB in {false, true}; one translation unit per K.  search_blocks gives the
// persistent grid (resident blocks per SM x SMs).
// tight: the first-level variant with upper-bound tightening (lb only).
// cost: kCostSquared, or kCostAbsolute (no lower bounds only).
cudaError_t launch_search(int K, int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s,
                          bool tight = false, int cost = 0);
int search_blocks(int K, int band, bool lb, int m, bool tight = false, int cost = 0);
// The widest re-run level (K = 32, columns streamed from shared memory; two
// windows, 2048 columns, for m <= 2048; four windows, 4096 columns, beyond).
// The group levels (search_wide.cu): lb = true runs tiles through the
// lower-bound cascade (a first level), lb = false the list or tiles without it.
cudaError_t launch_search_wide(int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s, int cost = 0);
int search_blocks_wide(int band, bool lb, int m, int cost = 0);

// The first level with the narrow-block elastic wavefront
// (search_elastic_kernel; tile mode only): band 0 unconstrained, 1 banded.
cudaError_t launch_search_elastic(bool lb, int band, const SearchArgs& args, int blocks, cudaStream_t s, int cost = 0);
int search_blocks_elastic(bool lb, int band, int m, int cost = 0);

// eap_dtw single pair: one warp; wide selects the four-window level.
cudaError_t launch_pair(int K, int band, bool wide, const float* rows, int nr, const float* cols, int nc,
                        int w, float ub, double* out, cudaStream_t s);

// Batched search (batch.cuh): preparation (state reset, query slots, seed
// samples and selection) and result conversion; query_prep shared memory is
// sized for queries up to m_cap points (batch_prep_attributes sets it and must
// run outside stream capture).
cudaError_t batch_prep_attributes(int m_cap);
// Level p of the running-extrema table from level p-1 (half = 2^(p-1)).
cudaError_t launch_env_level(const float* smax, const float* smin, int64_t n, int64_t half, float* dmax,
                             float* dmin, cudaStream_t s);
cudaError_t launch_batch_prep(const BatchDev& D, int cap_items, unsigned long long* counters, int ncounters,
                              unsigned long long* work, int nwork, int* rr_counts, int nrr, int m_cap,
                              cudaStream_t s);
cudaError_t launch_batch_finalize(const BatchDev& D, cudaStream_t s);
// batch_kernel for one level (0..3: K = 4 << level, columns in registers;
// 4, 5: K = 32 with two or four windows, columns streamed from shared
// memory); batch_attributes must run outside stream capture.
cudaError_t launch_batch(int level, int band, const BatchLaunch& args, int blocks, cudaStream_t s);
int batch_blocks(int level, int band);
cudaError_t batch_attributes();
// The elastic first level of the batch (batch_elastic.cu): class kElClass0 + ec.
cudaError_t launch_batch_elastic(int ec, const BatchLaunch& args, int blocks, cudaStream_t s);
int batch_blocks_el(int ec);

}  // namespace eapdtw
