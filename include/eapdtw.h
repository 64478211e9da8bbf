/*
 * eapdtw.h - C ABI of the GB300 (sm_103a) EAPrunedDTW subsequence-search library.
 *
 * Method: Herrmann & Webb, "Early Abandoning PrunedDTW and its application to
 * similarity search" (arXiv 2010.05371).  DTW is the recurrence of Eq. 1-5 with
 * the squared Euclidean cost (Section 2); the warping window w is the
 * Sakoe-Chiba band |i - j| <= w (Section 2.1); early abandoning against an
 * upper bound ub follows Algorithm 3 (EAPrunedDTW) and Section 2.2; the search
 * is the UCR-Suite loop of Section 5 (z-normalised sliding windows, LB_Kim and
 * LB_Keogh lower bounds, best-so-far tightening).
 *
 * Conventions shared by every entry point:
 *  - Return value: EAPDTW_OK (0) or a negative EAPDTW_ERR_* code.  No C++
 *    exception crosses this boundary.  eapdtw_strerror() names a code.
 *  - Unless a name ends in _host, array arguments are DEVICE pointers (memory
 *    of the current CUDA device, e.g. allocated by PyTorch), owned by the
 *    caller; the library never frees them and keeps no reference after the
 *    call returns.  _host variants take host pointers and copy.
 *  - Series are float32, contiguous.  Distances are returned as float64
 *    holding the float32 DTW value (a sum of squared costs, no square root).
 *  - stream: a cudaStream_t (NULL = the legacy default stream).  Every call
 *    enqueues its work on that stream; calls documented as "blocking"
 *    additionally wait for it before returning.
 *  - Scratch memory (prefix sums, envelopes, queues) is owned by the library,
 *    cached per device and grown on demand; it is released by
 *    eapdtw_release_scratch() or at process exit.  Calls on one device from
 *    several host threads are serialised internally.
 *  - Window semantics: cell (i, j) exists iff |i - j| <= w.  w >= max(lS,lT)-1
 *    is unconstrained DTW.  w < |lS - lT| admits no warping path: the result
 *    is +inf.
 */
#ifndef EAPDTW_H
#define EAPDTW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EAPDTW_OK 0
#define EAPDTW_ERR_INVALID_ARG -1   /* NULL pointer, length <= 0, w < 0, k < 1, NaN ub, lQ > lR */
#define EAPDTW_ERR_NAN_INPUT -2     /* a NaN or Inf in an input series */
#define EAPDTW_ERR_OUT_OF_MEMORY -3 /* scratch allocation failed */
#define EAPDTW_ERR_CUDA -4          /* a CUDA runtime call failed */
#define EAPDTW_ERR_TIMEOUT -5       /* a device-side wait ran out: the widest level's warps wait on their
                                       neighbours with a bounded number of polls; the results are void */
#define EAPDTW_ERR_UNSUPPORTED -6   /* size beyond what this build supports (see each call) */
#define EAPDTW_ERR_INTERNAL -7      /* a device-side consistency check failed */
#define EAPDTW_ERR_BUSY -8          /* the object is in use (a reference read by the serving loop; a second server) */
#define EAPDTW_ERR_CANCELLED -9     /* the serving request was cancelled */
#define EAPDTW_PENDING 1            /* eapdtw_serve_poll: the request has not finished yet */

/* Upper limits of this build.  The query (shorter series) length is bounded
 * by the query staging buffer in shared memory. */
#define EAPDTW_MAX_QUERY 4096
#define EAPDTW_MAX_K 64

/* Counters of one search (indices into the int64 counter array). */
#define EAPDTW_CNT_WINDOWS 0        /* candidate windows scanned */
#define EAPDTW_CNT_KIM_PRUNED 1     /* skipped by LB_Kim > ub */
#define EAPDTW_CNT_EQ_PRUNED 2      /* skipped by LB_Keogh(EQ) > ub */
#define EAPDTW_CNT_EC_PRUNED 3      /* skipped by LB_Keogh(EC) > ub */
#define EAPDTW_CNT_DTW_ABANDONED 4  /* EAPrunedDTW returned +inf (DTW > ub), whether the
                                       per-lane check of the first 16 rows or the warp
                                       wavefront found the dead row */
#define EAPDTW_CNT_DTW_COMPLETED 5  /* EAPrunedDTW returned a value <= ub */
#define EAPDTW_CNT_CELLS 6          /* DP cells executed by the kernel: K per busy lane-step
                                       of the wavefront, plus 16 x 16 per window given to
                                       the per-lane first-rows check */
#define EAPDTW_CNT_LB_RECHECK 7     /* LB re-tested against a tighter ub before DTW and skipped */
#define EAPDTW_CNT_OVERFLOW 8       /* candidates re-run with a wider tile */
#define EAPDTW_CNT_STEPS 9          /* warp wavefront steps executed */
/* Device time of the phases of the search, in ns, measured with CUDA events on
 * the call's stream: */
#define EAPDTW_CNT_NS_MAIN 10       /* the main search kernel (LB cascade + EAPrunedDTW) */
#define EAPDTW_CNT_NS_WIDER 11      /* re-runs of overflowed windows with wider tiles */
#define EAPDTW_CNT_NS_PREP 12       /* window statistics, query preparation, envelope */
#define EAPDTW_CNT_NS_SEED 13       /* sampled upper-bound seed */
#define EAPDTW_CNT_NS_TOTAL 14      /* whole call, first to last kernel */
#define EAPDTW_CNT_LAUNCHES 15      /* kernels launched by the call */
#define EAPDTW_CNT_PROBE_OVERFLOW 16 /* overflows among the first-level probe's windows (-1: no probe) */
#define EAPDTW_CNT_FIRST_TILE 17    /* DP cells per lane of the first level after the probe */
#define EAPDTW_NCOUNTERS 18

/* eapdtw_strerror: static description of a return code (never NULL). */
const char* eapdtw_strerror(int32_t code);

/* eapdtw_version: library version string (static). */
const char* eapdtw_version(void);

/*
 * eap_dtw - DTW of two raw series with early abandoning (Algorithm 3).
 *
 * Computes DTW_w(S, T) per Eq. 1-5 (cost (a - b)^2, band |i - j| <= w) on the
 * raw values (no z-normalisation).  *out_dist receives the DTW value if it is
 * <= ub, else +inf (Algorithm 3 returns +inf exactly when DTW > ub).
 * ub = +INFINITY gives plain banded DTW.
 *
 *   S, T      device float32 arrays of lS and lT points (lS, lT >= 1).
 *   w         window, w >= 0.
 *   ub        upper bound; not NaN.
 *   out_dist  DEVICE pointer to one double.
 *   stream    cudaStream_t.  Asynchronous: the result is valid once the stream
 *             reaches this point.
 * Errors: INVALID_ARG; UNSUPPORTED if min(lS, lT) > EAPDTW_MAX_PAIR_COLS.
 */
#define EAPDTW_MAX_PAIR_COLS 65536
int32_t eap_dtw(const float* S, int64_t lS, const float* T, int64_t lT, int64_t w, double ub,
                double* out_dist, void* stream);

/* eap_dtw_host - eap_dtw on host arrays; blocking; *out_dist is a host double. */
int32_t eap_dtw_host(const float* S, int64_t lS, const float* T, int64_t lT, int64_t w,
                     double ub, double* out_dist);

/*
 * subseq_search - k nearest subsequences of R to Q under DTW (Section 5).
 *
 * Every window R[i .. i+lQ), i in [0, lR - lQ], and the query Q are
 * z-normalised (population standard deviation; a constant window normalises to
 * zeros); d_i = DTW_w(z(window_i), z(Q)) with the window as rows and the query
 * as columns.  Returns the k smallest (d_i, i), ascending by (d_i, i); a
 * distance tie goes to the smaller i.  Windows may overlap (no exclusion zone).
 * If k > lR - lQ + 1 the extra slots are (-1, +inf).
 *
 * The search runs LB_Kim (first/last points), LB_Keogh EQ (window against the
 * query envelope) and LB_Keogh EC (query against the reference envelope), then
 * EAPrunedDTW against the running k-th best distance; these never change the
 * result, only the work done.
 *
 *   Q         device float32 [lQ], 1 <= lQ <= EAPDTW_MAX_QUERY.
 *   R         device float32 [lR], lR >= lQ, lR < 2^31.
 *   w         window, w >= 0 (w >= lQ - 1 is unconstrained).
 *   k         1 <= k <= EAPDTW_MAX_K.
 *   out_idx   DEVICE int64 [k];  out_dist  DEVICE double [k].
 *   stream    cudaStream_t.  Blocking: returns after the results are written.
 * Errors: INVALID_ARG, NAN_INPUT (NaN/Inf in Q or R), UNSUPPORTED, OUT_OF_MEMORY,
 *         CUDA.
 */
int32_t subseq_search(const float* Q, int64_t lQ, const float* R, int64_t lR, int64_t w,
                      int32_t k, int64_t* out_idx, double* out_dist, void* stream);

#define EAPDTW_COST_SQUARED 0
#define EAPDTW_COST_ABSOLUTE 1

/* Options of subseq_search_ex (zero-initialise, then set fields). */
typedef struct {
    int32_t no_lb;        /* 1: skip LB_Kim / LB_Keogh ("nolb" variant of Section 5) */
    int32_t tile;         /* first level: DP cells per lane per step (4, 8, 16, 32), 512 = a group of
                             warps per candidate (512 columns per warp, lQ <= 4096); 0 = automatic */
    int32_t no_seed;      /* 1: start from ub = +inf instead of a sampled seed */
    int32_t audit;        /* 1: hold ub fixed at ub_fixed for the whole search */
    double ub_fixed;      /* used when audit = 1 */
    int64_t* counters;    /* optional HOST int64[EAPDTW_NCOUNTERS], filled on return */
    int32_t tighten;      /* 1: upper-bound tightening with the LB_Keogh EQ terms (the UCR
                             Suite technique Section 5 keeps): during EAPrunedDTW a cell of
                             row r is dead once its value plus the terms of rows r+1.. exceed
                             ub.  Changes the work done, never the result.  First level of the
                             search, lower bounds on.  Off by default: it saves DTW steps but
                             costs more time than it saves on the measured workloads. */
    int32_t cost;         /* pointwise cost of the DTW recurrence: EAPDTW_COST_SQUARED (0, Eq. 5)
                             or EAPDTW_COST_ABSOLUTE (1, |a - b|: another elastic distance with
                             the same recurrence, Section 6).  The absolute cost requires
                             no_lb = 1 (LB_Kim / LB_Keogh bound the squared cost); its sampled
                             seed sums |z - q| along the diagonal. */
    int32_t reserved[6];
} eapdtw_search_opts;

/* subseq_search_ex - subseq_search with options (opts may be NULL). */
int32_t subseq_search_ex(const float* Q, int64_t lQ, const float* R, int64_t lR, int64_t w,
                         int32_t k, const eapdtw_search_opts* opts, int64_t* out_idx,
                         double* out_dist, void* stream);

/* subseq_search_host - subseq_search on HOST arrays (Q, R, out_idx, out_dist),
 * copying inputs to the device and results back; blocking. */
int32_t subseq_search_host(const float* Q, int64_t lQ, const float* R, int64_t lR, int64_t w,
                           int32_t k, const eapdtw_search_opts* opts, int64_t* out_idx,
                           double* out_dist);

/* eapdtw_release_scratch - free the cached scratch memory of the current device. */
int32_t eapdtw_release_scratch(void);

/*
 * subseq_search_noalloc - subseq_search for callers that cannot allocate memory.
 *
 * The paper has no counterpart: this entry point exists for callers that must
 * not call cudaMalloc, for example code running inside a memory pool or an
 * allocator they do not own, or under a policy that forbids device allocation
 * after start-up.  It computes exactly what subseq_search computes, with the
 * same arguments and results, but it allocates nothing, on the device or the
 * host.  Its scratch memory (window statistics, envelopes, query staging,
 * best-so-far state, work lists) is one fixed array in the library's device
 * memory, EAPDTW_NOALLOC_SCRATCH_BYTES long, which every GPU on which the
 * entry point has been called keeps until the process exits.
 *
 *   Limits: lR <= EAPDTW_NOALLOC_MAX_N, lQ <= EAPDTW_MAX_QUERY,
 *           k <= EAPDTW_MAX_K.  Larger sizes return EAPDTW_ERR_UNSUPPORTED
 *           and launch nothing.
 *   Pointers, stream and blocking behaviour are those of subseq_search.
 *   The first call on a device looks up the array's device address on that
 *   device.  With CUDA's default lazy module loading, that is also when the
 *   array's device memory is committed, so the first call on each device can
 *   fail with EAPDTW_ERR_CUDA for lack of memory.  Make that first call at
 *   start-up, before any phase that must not allocate and before any stream
 *   capture; later calls commit nothing.
 *   All calls share the one array, and each call leaves its contents behind;
 *   the call clears what must start from zero itself.  Calls are serialised
 *   on the host, and each returns only after its work is done; two calls that
 *   overlapped on the GPU (for example from a launch issued around this API)
 *   would race on the array.
 */
#define EAPDTW_NOALLOC_MAX_N (1 << 20)
#define EAPDTW_NOALLOC_SCRATCH_BYTES (40 * (int64_t)EAPDTW_NOALLOC_MAX_N + (1 << 20))
int32_t subseq_search_noalloc(const float* Q, int64_t lQ, const float* R, int64_t lR, int64_t w,
                              int32_t k, int64_t* out_idx, double* out_dist, void* stream);

/*
 * eapdtw_cell_peak - measured throughput ceiling of the DP cell (a measurement
 * utility; the paper has no counterpart).
 *
 * Runs the cell of Eq. 1-5 (d = q - z, v = d * d + min(top, diag, left) in
 * FP32) with nothing else around it, on every SM of the current device, and
 * returns the fastest of three timed launches (CUDA events, after one
 * warm-up) as DP cells per second.  It bounds what any schedule of the same
 * cells can reach, and is the roofline denominator of the search kernels.
 *   mode 0: scalar operations, one row per step (3 issue slots per cell);
 *   mode 1: the subtractions of adjacent columns paired in packed f32x2 adds;
 *   mode 2: two rows per step, anti-diagonal cell pairs in packed f32x2 adds
 *           and fused multiply-adds;
 *   mode 3: mode 2 with two independent blocks per thread.
 *   steps     rows per thread, even, >= 2 (2^18 takes about 50 ms per launch).
 *   *cells_per_s  receives the rate; *ms (optional) the launch time.
 * Blocking; allocates and frees a small result buffer.
 * Errors: INVALID_ARG (bad mode or steps), CUDA.
 */
int32_t eapdtw_cell_peak(int32_t mode, int64_t steps, double* cells_per_s, double* ms);

/* ------------------------------------------------------------------------
 * Contexts and the batched search.
 *
 * Not in the paper, which searches one query in one series at a time
 * (Section 5): a context keeps references resident on one device (their raw
 * values and the chunk-anchored FP64 prefix sums behind the window statistics)
 * and runs many (query, reference) items in one launch sequence.  Each item is
 * exactly a subseq_search(Q, lQ, R, lR, w, k) call and returns the same
 * result (the lower bounds change which windows reach EAPrunedDTW, never the
 * result; LB_Keogh EC is not used in batches).
 * ------------------------------------------------------------------------ */
typedef struct eapdtw_ctx eapdtw_ctx;

/* One item of a batch. */
typedef struct {
    const float* Q;    /* DEVICE pointer to lQ query values (caller-owned; read during the call) */
    int64_t lQ;        /* 1 <= lQ <= min(EAPDTW_MAX_QUERY, length of the reference) */
    int64_t w;         /* warping window, >= 0 (w >= lQ - 1: unconstrained) */
    int32_t ref_id;    /* a reference registered with the context */
    int32_t k;         /* 1 <= k <= kstride of the call */
    int32_t no_lb;     /* 1: skip LB_Kim / LB_Keogh for this item */
    int32_t reserved;  /* set to 0 */
} eapdtw_item;

/* eapdtw_ctx_create - a context on CUDA device `device`.  mem_budget (bytes,
 * 0 = no limit) bounds the device memory the context holds: resident
 * references plus its batch arena; a call that would exceed it returns
 * EAPDTW_ERR_OUT_OF_MEMORY and leaves the context unchanged. */
int32_t eapdtw_ctx_create(int32_t device, int64_t mem_budget, eapdtw_ctx** out);

/* eapdtw_ctx_destroy - wait for the device, free everything the context holds. */
int32_t eapdtw_ctx_destroy(eapdtw_ctx* ctx);

/* eapdtw_ref_register - COPY the device series R[0..lR) into the context and
 * build its window statistics (chunk-anchored FP64 prefix sums, 20 bytes per
 * point in all).  The caller may free R when the call returns (blocking).
 * lR < 2^31.  A NaN or Inf in R returns EAPDTW_ERR_NAN_INPUT and registers
 * nothing.  *ref_id receives the handle. */
int32_t eapdtw_ref_register(eapdtw_ctx* ctx, const float* R, int64_t lR, int32_t* ref_id, void* stream);

/* eapdtw_ref_unregister - wait for the device, then free a reference. */
int32_t eapdtw_ref_unregister(eapdtw_ctx* ctx, int32_t ref_id);

/* eapdtw_ref_info - device address and length of a registered reference's
 * copy (owned by the context; valid until it is unregistered). */
int32_t eapdtw_ref_info(eapdtw_ctx* ctx, int32_t ref_id, const float** R, int64_t* lR);

/* eapdtw_ctx_info - out[0..min(nout, EAPDTW_CTX_NINFO)): bytes held, budget,
 * live references, batch arena bytes, batches run, items run, items that were
 * re-run alone (a re-run list was full), 1 if the launch graph is captured. */
#define EAPDTW_CTX_NINFO 8
int32_t eapdtw_ctx_info(eapdtw_ctx* ctx, int64_t* out, int32_t nout);

/* eapdtw_search_batch - run n items (a HOST array) on the context's device.
 * Item i's k results go to out_idx/out_dist[i*kstride .. i*kstride + k)
 * (DEVICE arrays of n*kstride), ascending by (distance, index) as in
 * subseq_search; slots k..kstride-1 hold (-1, +inf).  Items that share the
 * same (Q pointer, lQ, w) share one query preparation.  counters: optional
 * HOST int64[EAPDTW_NCOUNTERS] with the summed counters 0..9 of the batch and, at
 * EAPDTW_CNT_NS_TOTAL, the device time of its launch sequence (CUDA events on
 * `stream`; items re-run alone after a full re-run list are not included).
 * Blocking.  The launch sequence is captured into a CUDA graph on the first
 * call (and again after the context's arena grows), so the call must not be
 * made while `stream` is being captured.  kstride <= EAPDTW_MAX_K. */
int32_t eapdtw_search_batch(eapdtw_ctx* ctx, const eapdtw_item* items, int32_t n, int32_t kstride,
                            int64_t* out_idx, double* out_dist, int64_t* counters, void* stream);

/* eapdtw_set_first_tile - the autotuner's choice of the first level's DP
 * cells per lane (4, 8, 16, 32; 1 = the narrow-block elastic wavefront, which
 * runs queries of 129 to 2048 points that are unconstrained or have a band of
 * at least 64 and a quarter of lQ, others falling back to the built-in rule;
 * 0 = the built-in rule: the elastic wavefront where it runs for queries of
 * up to 1024 points, else the narrowest one-warp K whose window holds the
 * band or every column) for items with
 * floor(log2 lQ) == log2_m, window ratio floor(10 w / lQ) == ratio_tenths
 * (10 for unconstrained) and band (0 unconstrained, 1 banded).  Any choice
 * gives the same results; only the speed differs. */
int32_t eapdtw_set_first_tile(eapdtw_ctx* ctx, int32_t log2_m, int32_t ratio_tenths, int32_t band, int32_t tile);

/* eapdtw_get_first_tile - the table entry (0 = none, the built-in rule). */
int32_t eapdtw_get_first_tile(eapdtw_ctx* ctx, int32_t log2_m, int32_t ratio_tenths, int32_t band, int32_t* tile);

/* eapdtw_set_tuning - the autotuner's whole choice for a signature (see
 * eapdtw_set_first_tile): the first level's DP cells per lane (4, 8, 16, 32, 1
 * for the elastic wavefront; 0 = the built-in rule) and check_double (1: the warp wavefront checks its
 * borders and the best-so-far bound at twice its built-in interval of 8
 * steps, 16 for the one-window unconstrained levels; 0: the built-in
 * interval).  Both 0 removes the entry.  Any choice gives the same results. */
int32_t eapdtw_set_tuning(eapdtw_ctx* ctx, int32_t log2_m, int32_t ratio_tenths, int32_t band, int32_t tile,
                          int32_t check_double);

/* eapdtw_get_tuning - the table entry (0, 0 = none). */
int32_t eapdtw_get_tuning(eapdtw_ctx* ctx, int32_t log2_m, int32_t ratio_tenths, int32_t band, int32_t* tile,
                          int32_t* check_double);

/* eapdtw_autotune - the autotuner of the first level's DP cells per lane and
 * of the wavefront's check (poll) interval.  For every signature (see
 * eapdtw_set_first_tile) of the n HOST items that has no table entry yet, it
 * times the batched search of one representative item (the one with the
 * longest reference) over a prefix of its reference holding about
 * sample_windows windows, with the built-in K, twice it and half it (where
 * the built-in first level is the elastic wavefront: it, the band's one-warp
 * K and twice that), each at
 * the built-in check interval and at twice it (two runs each, the faster
 * counts, device time of the launch sequence), and enters the fastest pair if
 * it beats the built-in choice by 5% (else the built-in choice).
 * *n_tuned (optional) receives the number of signatures entered.  Blocking;
 * results of later searches are unchanged. */
int32_t eapdtw_autotune(eapdtw_ctx* ctx, const eapdtw_item* items, int32_t n, int64_t sample_windows,
                        void* stream, int32_t* n_tuned);

/* ------------------------------------------------------------------------
 * Whole-series DTW without an external upper bound (Section 2.3: PrunedDTW's
 * setting, where no best-so-far exists).  Series are rows of length len,
 * contiguous, DEVICE arrays; znorm = 1 z-normalises each series first
 * (population deviation; a constant series becomes zeros).  Window as in
 * eap_dtw.  len <= EAPDTW_MAX_QUERY.  Blocking.
 * ------------------------------------------------------------------------ */

/* eapdtw_pairwise - out[i * nb + j] = DTW_w(A_i, B_j) for all pairs (DEVICE,
 * na * nb doubles).  Each pair runs EAPrunedDTW under its own diagonal cost
 * (squared Euclidean distance: the cost of an admissible path, so an upper
 * bound of the DTW, PrunedDTW's threshold), so the values are exact DTW. */
int32_t eapdtw_pairwise(const float* A, int64_t na, const float* B, int64_t nb, int64_t len, int64_t w,
                        int32_t znorm, double* out, void* stream);

/* eapdtw_nn - for each test series, the k nearest training series under DTW_w
 * (1-NN classification for k = 1): out_idx/out_dist[t * k .. t * k + k)
 * (DEVICE), ascending by (distance, index), (-1, +inf) when ntrain < k.  Each
 * pair runs EAPrunedDTW against the test's current k-th best distance, with no
 * lower bounds.  k <= EAPDTW_MAX_K. */
int32_t eapdtw_nn(const float* train, int64_t ntrain, const float* test, int64_t ntest, int64_t len, int64_t w,
                  int32_t k, int32_t znorm, int64_t* out_idx, double* out_dist, void* stream);

/* ------------------------------------------------------------------------
 * Serving loop (continuous batching).
 *
 * Not in the paper: a server thread of the context takes requests from any
 * host thread and runs them in rounds of the batched launch sequence.  Each
 * round processes the next chunk_windows windows of every admitted request,
 * so a request that arrives while others are on the GPU is admitted at the
 * next round boundary (a free state slot and the memory it needs, see below)
 * and its work overlaps with theirs.  The references, their window
 * statistics and each admitted request's state (prepared query, seed bound,
 * k-best list) stay on the device across rounds.  A request's result is
 * exactly subseq_search of its (Q, R, w, k), whatever else runs with it.
 * Admission: up to max_active requests hold a state slot; a request whose
 * LB_Keogh EC needs a running-extrema level of its reference that does not
 * fit the context's memory budget finishes with EAPDTW_ERR_OUT_OF_MEMORY.
 * ------------------------------------------------------------------------ */

/* eapdtw_serve_start - start the server thread (one per context): max_active
 * state slots (1..4096), chunk_windows windows per request per round (>= 32,
 * rounded up to a multiple of 32).  Reserves its arena (tables, re-run lists
 * for max_active * chunk_windows windows, result rows) within the budget. */
int32_t eapdtw_serve_start(eapdtw_ctx* ctx, int32_t max_active, int64_t chunk_windows);

/* eapdtw_serve_stop - stop the server thread after its current round and free
 * its arena; requests not yet polled are dropped.  No thread may be inside
 * eapdtw_serve_poll while it runs. */
int32_t eapdtw_serve_stop(eapdtw_ctx* ctx);

/* eapdtw_serve_submit - queue a request: Q is a HOST array of lQ values
 * (copied before the call returns), searched in reference ref_id with window
 * w for the k best windows (k <= EAPDTW_MAX_K), lower bounds skipped if
 * no_lb.  *req_id receives its handle.  Never blocks on the GPU. */
int32_t eapdtw_serve_submit(eapdtw_ctx* ctx, const float* Q, int64_t lQ, int32_t ref_id, int64_t w, int32_t k,
                            int32_t no_lb, int64_t* req_id);

/* eapdtw_serve_poll - the state of a request, waiting up to timeout_ms
 * milliseconds (0: do not wait) for it to finish.  EAPDTW_PENDING: not done.
 * EAPDTW_OK: out_idx/out_dist (HOST, k entries; either may be NULL) and
 * *latency_ns (submission to completion; may be NULL) are filled and the
 * handle is released.  A negative code (the request failed, or
 * EAPDTW_ERR_CANCELLED) also releases the handle. */
int32_t eapdtw_serve_poll(eapdtw_ctx* ctx, int64_t req_id, int64_t* out_idx, double* out_dist, int64_t* latency_ns,
                          int32_t timeout_ms);

/* eapdtw_serve_cancel - cancel a request: a queued one at once, an admitted
 * one at the next round boundary.  Poll it to release the handle. */
int32_t eapdtw_serve_cancel(eapdtw_ctx* ctx, int64_t req_id);

/* eapdtw_serve_stats - out[0..min(nout, EAPDTW_SERVE_NSTATS)): completed,
 * cancelled, queued, admitted, rounds, windows processed, p50 and p99 latency
 * of the completed requests (ns, -1 if none), requests re-run alone, sticky
 * CUDA error of the loop (0 if none). */
#define EAPDTW_SERVE_NSTATS 10
int32_t eapdtw_serve_stats(eapdtw_ctx* ctx, int64_t* out, int32_t nout);

#ifdef __cplusplus
}
#endif

#endif /* EAPDTW_H */
