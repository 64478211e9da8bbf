// C ABI of the library (declared in include/eapdtw.h): argument checks, scratch
// management and the launch sequence of eap_dtw and subseq_search.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "eapdtw.h"
#include "kernels.h"
#include "plan.h"
#include "search_kernel.cuh"

using namespace eapdtw;

namespace {

constexpr int kSeedSamples = 4096;
constexpr int kSeedBest = 32;
constexpr float kLbScale = 1.0001f;   // prune iff lb > ub * kLbScale (FP32 rounding margin)
// First-level probe: kProbeSamples windows spread evenly over the reference run
// through EAPrunedDTW at the planned K (after the seed pass, under its bound);
// if more than kProbeRate of them overflow the warp's window, the whole first
// level runs one level wider (the live regions are too wide for the planned K,
// and re-running a window costs its partial first run on top of the wider run).
constexpr int kProbeSamples = 2048;
constexpr double kProbeRate = 0.05;

float ub_to_f32_up(double ub) {
    if (std::isinf(ub)) return ub > 0 ? INFINITY : -INFINITY;
    float f = static_cast<float>(ub);
    if (static_cast<double>(f) < ub) f = std::nextafter(f, INFINITY);
    return f;
}

// Device-side scratch of one device, grown on demand.
struct Scratch {
    int device = -1;
    std::mutex mu;
    // reference statistics
    double *P1 = nullptr, *P2 = nullptr, *T1 = nullptr, *T2 = nullptr;
    float* A = nullptr;
    int64_t cap_n = 0;
    float *UR = nullptr, *LR = nullptr;
    int64_t cap_env = 0;
    // query
    float *zq = nullptr, *uq = nullptr, *lq = nullptr, *zqo = nullptr;
    int* ord = nullptr;
    int cap_m = 0;
    // state: slots[64] | counters[16] | seed counters[16] | ints[32] | ub_seed
    unsigned char* state = nullptr;
    unsigned char* host_state = nullptr;  // pinned copy of counters, seed counters, ints
    // seed
    float* seed_ed = nullptr;
    int* seed_idx = nullptr;
    long long* seed_best = nullptr;
    // overflow lists
    long long* ovf[2] = {nullptr, nullptr};
    int cap_ovf = 0;
    // upper-bound tightening rows
    float* cb = nullptr;
    int64_t cap_cb = 0;
    long long* probe_list = nullptr;  // the first-level probe's sampled windows
    // host-pointer entry points
    float *dQ = nullptr, *dR = nullptr;
    int64_t cap_dq = 0, cap_dr = 0;
    int64_t* dIdx = nullptr;
    double* dDist = nullptr;
    // phase timing of the last search (CUDA events on the caller's stream)
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};

    unsigned long long* slots() { return reinterpret_cast<unsigned long long*>(state); }
    unsigned long long* counters() { return reinterpret_cast<unsigned long long*>(state + 512); }
    unsigned long long* seed_counters() { return reinterpret_cast<unsigned long long*>(state + 640); }
    int* ints() { return reinterpret_cast<int*>(state + 768); }
    float* ub_seed() { return reinterpret_cast<float*>(state + 896); }
};

// (Re)allocate p with room for n elements (previous contents are dropped).
template <typename T>
bool alloc(T*& p, int64_t n) {
    if (p) cudaFree(p);
    p = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&p), sizeof(T) * static_cast<size_t>(n)) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return false;
    }
    return true;
}

template <typename T>
void release(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

std::mutex g_mu;
Scratch* g_scratch[64] = {nullptr};

Scratch* scratch_for_current_device(int* dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    *dev_out = dev;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch[dev]) {
        Scratch* s = new (std::nothrow) Scratch();
        if (!s) return nullptr;
        s->device = dev;
        if (cudaMalloc(reinterpret_cast<void**>(&s->state), 1024) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&s->host_state), 1024) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&s->seed_ed), sizeof(float) * kSeedSamples) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&s->seed_idx), sizeof(int) * kSeedSamples) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&s->seed_best), sizeof(long long) * 64) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&s->probe_list), sizeof(long long) * kProbeSamples) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return nullptr;
        }
        for (auto& e : s->ev) {
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                delete s;
                return nullptr;
            }
        }
        g_scratch[dev] = s;
    }
    return g_scratch[dev];
}


#define CK(expr)                                     \
    do {                                             \
        cudaError_t e_ = (expr);                     \
        if (e_ != cudaSuccess) {                     \
            cudaGetLastError();                      \
            return EAPDTW_ERR_CUDA;                  \
        }                                            \
    } while (0)

int32_t search_impl(Scratch& S, const float* Q, int64_t lQ, const float* R, int64_t lR, int64_t w,
                    int32_t k, const eapdtw_search_opts* opts, int64_t* out_idx, double* out_dist,
                    cudaStream_t st) {
    const int m = static_cast<int>(lQ);
    const int64_t n = lR;
    const int64_t nw = n - m + 1;
    const int wi = static_cast<int>(w < m ? w : m);   // w >= m - 1 is unconstrained
    const int cost = opts ? opts->cost : 0;
    if (cost != kCostSquared && cost != kCostAbsolute) return EAPDTW_ERR_INVALID_ARG;
    const bool use_lb = !(opts && opts->no_lb);
    if (cost == kCostAbsolute && use_lb) return EAPDTW_ERR_INVALID_ARG;   // bounds are for the squared cost
    const bool seed = !(opts && opts->no_seed) && nw >= 2048;
    const bool audit = opts && opts->audit;
    if (audit && std::isnan(opts->ub_fixed)) return EAPDTW_ERR_INVALID_ARG;
    if (search_warps(m) < 1) return EAPDTW_ERR_UNSUPPORTED;
    const bool tighten_req = use_lb && opts && opts->tighten;
    // the elastic first level does not implement upper-bound tightening
    const Plan plan = plan_levels(m, m, wi, opts ? opts->tile : 0, !tighten_req);

    // scratch
    if (S.cap_n < n) {
        const int64_t ncap = (n + kChunk - 1) / kChunk;
        S.cap_n = 0;
        if (!alloc(S.P1, n) || !alloc(S.P2, n) || !alloc(S.T1, ncap) || !alloc(S.T2, ncap) ||
            !alloc(S.A, ncap))
            return EAPDTW_ERR_OUT_OF_MEMORY;
        S.cap_n = n;
    }
    if (use_lb && S.cap_env < n) {
        S.cap_env = 0;
        if (!alloc(S.UR, n) || !alloc(S.LR, n)) return EAPDTW_ERR_OUT_OF_MEMORY;
        S.cap_env = n;
    }
    const int mp = query_pad(m);
    if (S.cap_m < mp) {
        S.cap_m = 0;
        if (!alloc(S.zq, mp) || !alloc(S.uq, mp) || !alloc(S.lq, mp) || !alloc(S.zqo, mp) ||
            !alloc(S.ord, mp))
            return EAPDTW_ERR_OUT_OF_MEMORY;
        S.cap_m = mp;
    }
    // a window overflows at most once per level: nw entries always suffice
    const int want_ovf = static_cast<int>(nw);
    // upper-bound tightening scratch: one row of suffix sums per warp of the largest grid
    const bool tighten = use_lb && opts && opts->tighten;
    const int cb_stride = query_pad(m) + 8;
    if (tighten) {
        int64_t warps = 0;
        if (!plan.wide[0]) warps = search_blocks(plan.K[0], plan.band[0], true, m, true) *
                                   static_cast<int64_t>(search_warps(m));
        const int64_t want_cb = warps * cb_stride;
        if (S.cap_cb < want_cb) {
            S.cap_cb = 0;
            if (!alloc(S.cb, want_cb)) return EAPDTW_ERR_OUT_OF_MEMORY;
            S.cap_cb = want_cb;
        }
    }
    if (S.cap_ovf < want_ovf) {
        S.cap_ovf = 0;
        if (!alloc(S.ovf[0], want_ovf) || !alloc(S.ovf[1], want_ovf)) return EAPDTW_ERR_OUT_OF_MEMORY;
        S.cap_ovf = want_ovf;
    }

    int* ints = S.ints();
    int launches = 0;
    CK(cudaEventRecord(S.ev[0], st));
    CK(launch_init_state(S.slots(), k, S.ub_seed(), S.counters(), ints, kNumInts, st));
    CK(cudaMemsetAsync(S.seed_counters(), 0, 128, st));
    CK(launch_ref_prefix(R, n, S.P1, S.P2, S.T1, S.T2, S.A, ints + kBad, st));
    CK(launch_query_prep(Q, m, wi, S.zq, S.uq, S.lq, S.zqo, S.ord, ints + kBad, st));
    launches += 3;
    if (use_lb) {
        CK(launch_envelope(R, n, wi < m - 1 ? wi : m - 1, S.UR, S.LR, st));
        ++launches;
    }
    CK(cudaEventRecord(S.ev[1], st));

    SearchArgs a{};
    a.ref = RefView{R, n, S.P1, S.P2, S.T1, S.T2, S.A};
    a.q = QueryView{S.zq, S.uq, S.lq, S.zqo, S.ord, m};
    a.ur = S.UR;
    a.lr = S.LR;
    a.bsf = BestSoFar{S.slots(), S.ub_seed(), k, audit ? 1 : 0,
                      audit ? ub_to_f32_up(opts->ub_fixed) : 0.0f};
    a.nw = nw;
    a.w = wi;
    a.use_lb = use_lb ? 1 : 0;
    a.lb_scale = kLbScale;
    a.counters = S.counters();
    a.dbg = ints + kDbgSlot;
    a.err = ints + kTimeout;
    a.cb = tighten ? S.cb : nullptr;
    a.cb_stride = cb_stride;

    if (seed && !audit) {
        const int ns = static_cast<int>(nw < kSeedSamples ? nw : kSeedSamples);
        CK(launch_seed(a.ref, S.zq, m, nw, ns, S.seed_ed, S.seed_idx, k, S.ub_seed(), S.seed_best,
                       kSeedBest, ints + kNBest, st, cost));
        SearchArgs sa = a;
        sa.use_lb = 0;
        sa.work_counter = ints + kWorkSeed;
        sa.ovf_in = S.seed_best;
        sa.ovf_in_count = ints + kNBest;
        sa.ovf_in_cap = kSeedBest;
        sa.ovf_out = nullptr;
        sa.ovf_out_count = ints + kSeedOvf;
        sa.ovf_cap = 0;
        sa.counters = S.seed_counters();  // kept apart from the search's own counts
        const int K = plan.K[plan.nlev - 1];
        const int bd = plan.band[plan.nlev - 1];
        if (plan.wide[plan.nlev - 1]) {
            CK(launch_search_wide(bd, false, sa, search_blocks_wide(bd, false, m, cost) / 4 + 1, st, cost));
        } else {
            CK(launch_search(K, bd, false, sa, search_blocks(K, bd, false, m, false, cost) / 4 + 1, st, false, cost));
        }
        launches += 3;
    }
    CK(cudaEventRecord(S.ev[2], st));
    const bool probe = !(opts && opts->tile) && plan.nlev >= 2 && !plan.elastic[0] && !plan.wide[0] && !plan.wide[1] &&
                       nw >= 256 * static_cast<int64_t>(kProbeSamples);
    int64_t probe_ovf = -1;
    int first_tile = plan.K[0];
    for (int lev = 0; lev < plan.nlev; ++lev) {
        SearchArgs la = a;
        la.work_counter = ints + kWork0 + lev;
        la.ovf_out = S.ovf[lev & 1];
        la.ovf_out_count = ints + kOvf0 + lev;
        la.ovf_cap = S.cap_ovf;
        if (lev > 0) {
            la.ovf_in = S.ovf[(lev - 1) & 1];
            la.ovf_in_count = ints + kOvf0 + lev - 1;
            la.ovf_in_cap = S.cap_ovf;
        }
        const bool lb = use_lb && lev == 0;
        if (plan.wide[lev]) {
            CK(launch_search_wide(plan.band[lev], lb, la, search_blocks_wide(plan.band[lev], lb, m, cost), st, cost));
        } else if (plan.elastic[lev]) {
            CK(launch_search_elastic(lb, plan.band[lev], la, search_blocks_elastic(lb, plan.band[lev], m, cost), st, cost));
        } else if (lev == 0 && probe) {
            // the probe (sampled windows, single-window mode, overflows only
            // counted), then the first level at the planned or the next width:
            // both launches are enqueued, and each reads the probe's count on the
            // device and exits at once unless it is the chosen one
            const bool tight = tighten && lb;
            CK(launch_probe_list(S.probe_list, kProbeSamples, nw, ints + kWorkTail, st));
            SearchArgs pa = a;
            pa.use_lb = 0;
            pa.work_counter = ints + kWorkTail + 1;
            pa.ovf_in = S.probe_list;
            pa.ovf_in_count = ints + kWorkTail;
            pa.ovf_in_cap = kProbeSamples;
            pa.ovf_out = nullptr;
            pa.ovf_out_count = ints + kProbeCount;
            pa.ovf_cap = 0;
            pa.counters = S.seed_counters();   // kept apart from the search's own counts
            CK(launch_search(plan.K[0], plan.band[0], false, pa, search_blocks(plan.K[0], plan.band[0], false, m, false, cost),
                             st, false, cost));
            launches += 2;
            const int threshold = static_cast<int>(kProbeRate * kProbeSamples);
            for (int L = 0; L < 2; ++L) {
                SearchArgs lt = la;
                lt.ovf_out = S.ovf[L & 1];
                lt.ovf_out_count = ints + kOvf0 + L;
                lt.gate_count = ints + kProbeCount;
                lt.gate_threshold = threshold;
                lt.gate_wider = L;
                CK(launch_search(plan.K[L], plan.band[L], lb, lt,
                                 search_blocks(plan.K[L], plan.band[L], lb, m, tight, cost), st, tight, cost));
                ++launches;
            }
            probe_ovf = threshold;   // marks that a probe ran (the count is read back below)
        } else {
            const bool tight = tighten && lb;   // first level only
            CK(launch_search(plan.K[lev], plan.band[lev], lb, la,
                             search_blocks(plan.K[lev], plan.band[lev], lb, m, tight, cost), st, tight, cost));
        }
        ++launches;
        if (lev == 0) CK(cudaEventRecord(S.ev[3], st));
    }
    CK(cudaEventRecord(S.ev[4], st));
    CK(launch_finalize(S.slots(), k, out_idx, out_dist, st));
    ++launches;
    CK(cudaEventRecord(S.ev[5], st));
    CK(cudaMemcpyAsync(S.host_state, S.state + 512, 384, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const unsigned long long* hc = reinterpret_cast<const unsigned long long*>(S.host_state);
    const int* hi = reinterpret_cast<const int*>(S.host_state + 256);
    if (opts && opts->counters) {
        for (int c = 0; c < EAPDTW_NCOUNTERS; ++c) opts->counters[c] = static_cast<int64_t>(hc[c]);
        auto ns = [&](int a, int b) -> int64_t {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, S.ev[a], S.ev[b]) != cudaSuccess) {
                cudaGetLastError();
                return -1;
            }
            return static_cast<int64_t>(ms * 1.0e6);
        };
        opts->counters[EAPDTW_CNT_NS_MAIN] = ns(2, 3);
        opts->counters[EAPDTW_CNT_NS_WIDER] = ns(3, 4);
        opts->counters[EAPDTW_CNT_NS_PREP] = ns(0, 1);
        opts->counters[EAPDTW_CNT_NS_SEED] = ns(1, 2);
        opts->counters[EAPDTW_CNT_NS_TOTAL] = ns(0, 5);
        opts->counters[EAPDTW_CNT_LAUNCHES] = launches;
        if (probe_ovf >= 0) {
            probe_ovf = hi[kProbeCount];
            if (probe_ovf > static_cast<int>(kProbeRate * kProbeSamples)) first_tile = plan.K[1];
        }
        opts->counters[EAPDTW_CNT_PROBE_OVERFLOW] = probe_ovf;
        opts->counters[EAPDTW_CNT_FIRST_TILE] = first_tile;
    }
#ifdef EAPDTW_DEVICE_CHECKS
    if (hi[kDbgSlot]) {
        fprintf(stderr, "eapdtw device check failed: code %d value %d\n", hi[kDbgSlot], hi[kDbgSlot + 1]);
        return EAPDTW_ERR_INTERNAL;
    }
#endif
    if (hi[kBad]) return EAPDTW_ERR_NAN_INPUT;
    if (hi[kTimeout]) return EAPDTW_ERR_TIMEOUT;
    for (int lev = 0; lev + 1 < plan.nlev; ++lev)
        if (hi[kOvf0 + lev] > S.cap_ovf) return EAPDTW_ERR_INTERNAL;
    if (hi[kOvf0 + plan.nlev - 1] > 0) return EAPDTW_ERR_UNSUPPORTED;
    return EAPDTW_OK;
}

int32_t check_search_args(const float* Q, int64_t lQ, const float* R, int64_t lR, int64_t w,
                          int32_t k, const void* out_idx, const void* out_dist) {
    if (!Q || !R || !out_idx || !out_dist) return EAPDTW_ERR_INVALID_ARG;
    if (lQ < 1 || lR < lQ || w < 0 || k < 1) return EAPDTW_ERR_INVALID_ARG;
    if (lQ > EAPDTW_MAX_QUERY || k > EAPDTW_MAX_K || lR >= (int64_t(1) << 31))
        return EAPDTW_ERR_UNSUPPORTED;
    return EAPDTW_OK;
}

}  // namespace

extern "C" {

const char* eapdtw_strerror(int32_t code) {
    switch (code) {
        case EAPDTW_OK: return "ok";
        case EAPDTW_ERR_INVALID_ARG: return "invalid argument";
        case EAPDTW_ERR_NAN_INPUT: return "NaN or Inf in an input series";
        case EAPDTW_ERR_OUT_OF_MEMORY: return "out of device memory";
        case EAPDTW_ERR_CUDA: return "CUDA runtime error";
        case EAPDTW_ERR_TIMEOUT: return "a device-side wait ran out";
        case EAPDTW_ERR_UNSUPPORTED: return "size not supported by this build";
        case EAPDTW_ERR_INTERNAL: return "internal consistency check failed";
        case EAPDTW_ERR_BUSY: return "in use";
        case EAPDTW_ERR_CANCELLED: return "request cancelled";
        case EAPDTW_PENDING: return "pending";
        default: return "unknown error code";
    }
}

const char* eapdtw_version(void) { return "eapdtw-gb300 0.1 (sm_103a)"; }

int32_t eap_dtw(const float* S, int64_t lS, const float* T, int64_t lT, int64_t w, double ub,
                double* out_dist, void* stream) {
    if (!S || !T || !out_dist || lS < 1 || lT < 1 || w < 0 || std::isnan(ub))
        return EAPDTW_ERR_INVALID_ARG;
    const bool t_rows = lT > lS;  // rows = longer series; ties: rows = S
    const float* rows = t_rows ? T : S;
    const float* cols = t_rows ? S : T;
    const int64_t nr = t_rows ? lT : lS;
    const int64_t nc = t_rows ? lS : lT;
    if (nc > EAPDTW_MAX_PAIR_COLS || nr >= (int64_t(1) << 30)) return EAPDTW_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemsetAsync(out_dist, 0xff, sizeof(double), st));  // NaN until a level succeeds
    if (w < nr - nc) {
        // no admissible warping path
        const double inf = INFINITY;
        CK(cudaMemcpyAsync(out_dist, &inf, sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return EAPDTW_OK;
    }
    const int64_t lmax = nr;
    const int wi = static_cast<int>(w < lmax ? w : lmax);
    const Plan plan = plan_levels(nr, nc, wi, 0, false);   // the pair kernel's levels
    const float ubf = ub_to_f32_up(ub);
    for (int lev = 0; lev < plan.nlev; ++lev)
        CK(launch_pair(plan.K[lev], plan.band[lev], plan.wide[lev], rows, static_cast<int>(nr), cols,
                       static_cast<int>(nc), wi, ubf, out_dist, st));
    return EAPDTW_OK;
}

int32_t eap_dtw_host(const float* S, int64_t lS, const float* T, int64_t lT, int64_t w, double ub,
                     double* out_dist) {
    if (!S || !T || !out_dist || lS < 1 || lT < 1 || w < 0 || std::isnan(ub))
        return EAPDTW_ERR_INVALID_ARG;
    float *dS = nullptr, *dT = nullptr;
    double* dOut = nullptr;
    int32_t rc = EAPDTW_OK;
    if (cudaMalloc(reinterpret_cast<void**>(&dS), sizeof(float) * lS) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&dT), sizeof(float) * lT) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&dOut), sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        rc = EAPDTW_ERR_OUT_OF_MEMORY;
    }
    if (rc == EAPDTW_OK &&
        (cudaMemcpy(dS, S, sizeof(float) * lS, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(dT, T, sizeof(float) * lT, cudaMemcpyHostToDevice) != cudaSuccess))
        rc = EAPDTW_ERR_CUDA;
    if (rc == EAPDTW_OK) rc = eap_dtw(dS, lS, dT, lT, w, ub, dOut, nullptr);
    if (rc == EAPDTW_OK &&
        cudaMemcpy(out_dist, dOut, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = EAPDTW_ERR_CUDA;
    if (rc == EAPDTW_OK && std::isnan(*out_dist)) rc = EAPDTW_ERR_UNSUPPORTED;
    cudaFree(dS);
    cudaFree(dT);
    cudaFree(dOut);
    cudaGetLastError();
    return rc;
}

int32_t subseq_search_ex(const float* Q, int64_t lQ, const float* R, int64_t lR, int64_t w,
                         int32_t k, const eapdtw_search_opts* opts, int64_t* out_idx,
                         double* out_dist, void* stream) {
    int32_t rc = check_search_args(Q, lQ, R, lR, w, k, out_idx, out_dist);
    if (rc != EAPDTW_OK) return rc;
    int dev = 0;
    Scratch* S = scratch_for_current_device(&dev);
    if (!S) return EAPDTW_ERR_OUT_OF_MEMORY;
    std::lock_guard<std::mutex> g(S->mu);
    try {
        return search_impl(*S, Q, lQ, R, lR, w, k, opts, out_idx, out_dist,
                           static_cast<cudaStream_t>(stream));
    } catch (...) {
        return EAPDTW_ERR_INTERNAL;
    }
}

int32_t subseq_search(const float* Q, int64_t lQ, const float* R, int64_t lR, int64_t w,
                      int32_t k, int64_t* out_idx, double* out_dist, void* stream) {
    return subseq_search_ex(Q, lQ, R, lR, w, k, nullptr, out_idx, out_dist, stream);
}

int32_t subseq_search_host(const float* Q, int64_t lQ, const float* R, int64_t lR, int64_t w,
                           int32_t k, const eapdtw_search_opts* opts, int64_t* out_idx,
                           double* out_dist) {
    int32_t rc = check_search_args(Q, lQ, R, lR, w, k, out_idx, out_dist);
    if (rc != EAPDTW_OK) return rc;
    int dev = 0;
    Scratch* S = scratch_for_current_device(&dev);
    if (!S) return EAPDTW_ERR_OUT_OF_MEMORY;
    std::lock_guard<std::mutex> g(S->mu);
    if (S->cap_dq < lQ) {
        S->cap_dq = 0;
        if (!alloc(S->dQ, lQ)) return EAPDTW_ERR_OUT_OF_MEMORY;
        S->cap_dq = lQ;
    }
    if (S->cap_dr < lR) {
        S->cap_dr = 0;
        if (!alloc(S->dR, lR)) return EAPDTW_ERR_OUT_OF_MEMORY;
        S->cap_dr = lR;
    }
    if (!S->dIdx) {
        if (cudaMalloc(reinterpret_cast<void**>(&S->dIdx), sizeof(int64_t) * EAPDTW_MAX_K) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&S->dDist), sizeof(double) * EAPDTW_MAX_K) != cudaSuccess) {
            cudaGetLastError();
            return EAPDTW_ERR_OUT_OF_MEMORY;
        }
    }
    cudaStream_t st = nullptr;
    CK(cudaMemcpyAsync(S->dQ, Q, sizeof(float) * lQ, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->dR, R, sizeof(float) * lR, cudaMemcpyHostToDevice, st));
    try {
        rc = search_impl(*S, S->dQ, lQ, S->dR, lR, w, k, opts, S->dIdx, S->dDist, st);
    } catch (...) {
        rc = EAPDTW_ERR_INTERNAL;
    }
    if (rc != EAPDTW_OK) return rc;
    CK(cudaMemcpyAsync(out_idx, S->dIdx, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(out_dist, S->dDist, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return EAPDTW_OK;
}

int32_t eapdtw_release_scratch(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EAPDTW_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    Scratch* S = (dev >= 0 && dev < 64) ? g_scratch[dev] : nullptr;
    if (!S) return EAPDTW_OK;
    {
        std::lock_guard<std::mutex> g2(S->mu);
        release(S->P1); release(S->P2); release(S->T1); release(S->T2); release(S->A);
        release(S->UR); release(S->LR);
        release(S->zq); release(S->uq); release(S->lq); release(S->zqo); release(S->ord);
        release(S->ovf[0]); release(S->ovf[1]); release(S->cb);
        release(S->dQ); release(S->dR); release(S->dIdx); release(S->dDist);
        release(S->state); release(S->seed_ed); release(S->seed_idx); release(S->seed_best); release(S->probe_list);
        if (S->host_state) cudaFreeHost(S->host_state);
        S->host_state = nullptr;

    }
    delete S;
    g_scratch[dev] = nullptr;
    return EAPDTW_OK;
}

}  // extern "C"

namespace eapdtw {

cudaError_t launch_search_k4(int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s, bool tight, int cost);
cudaError_t launch_search_k8(int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s, bool tight, int cost);
cudaError_t launch_search_k16(int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s, bool tight,
                              int cost);
cudaError_t launch_search_k32(int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s, bool tight,
                              int cost);
int search_blocks_k4(int band, bool lb, int m, bool tight, int cost);
int search_blocks_k8(int band, bool lb, int m, bool tight, int cost);
int search_blocks_k16(int band, bool lb, int m, bool tight, int cost);
int search_blocks_k32(int band, bool lb, int m, bool tight, int cost);

cudaError_t launch_search(int K, int band, bool lb, const SearchArgs& args, int blocks, cudaStream_t s, bool tight,
                          int cost) {
    switch (K) {
        case 4: return launch_search_k4(band, lb, args, blocks, s, tight, cost);
        case 8: return launch_search_k8(band, lb, args, blocks, s, tight, cost);
        case 16: return launch_search_k16(band, lb, args, blocks, s, tight, cost);
        default: return launch_search_k32(band, lb, args, blocks, s, tight, cost);
    }
}

int search_blocks(int K, int band, bool lb, int m, bool tight, int cost) {
    switch (K) {
        case 4: return search_blocks_k4(band, lb, m, tight, cost);
        case 8: return search_blocks_k8(band, lb, m, tight, cost);
        case 16: return search_blocks_k16(band, lb, m, tight, cost);
        default: return search_blocks_k32(band, lb, m, tight, cost);
    }
}

}  // namespace eapdtw
