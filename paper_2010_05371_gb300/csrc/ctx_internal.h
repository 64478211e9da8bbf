// Host-side state of a context (include/eapdtw.h), shared by the batched
// search (ctx.cu) and the serving loop (serve.cu).
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "batch.cuh"
#include "eapdtw.h"

namespace eapdtw {

constexpr int kEnvLevels = 13;   // running extrema over 2^p points, p = 0..12 (radius <= 4095)
constexpr float kBatchLbScale = 1.0001f;   // prune iff lb > ub * scale (as subseq_search)
constexpr int kNumWork = kBatchLevels * 3 + kSeedClasses + kElClasses;
constexpr int kElWork0 = kBatchLevels * 3 + kSeedClasses;   // work counters of the elastic classes

struct RefEntry {
    bool live = false;
    float* R = nullptr;
    int64_t n = 0;
    double *P1 = nullptr, *P2 = nullptr, *T1 = nullptr, *T2 = nullptr;
    float* A = nullptr;
    int64_t bytes = 0;
    int users = 0;   // serving requests that still read it
    // sparse table of running maxima / minima for LB_Keogh EC, built on
    // demand; level 0 is R itself
    float* emax[kEnvLevels] = {nullptr};
    float* emin[kEnvLevels] = {nullptr};
    int env_levels = 1;
};

// Byte offsets of the work tables (the same layout in the pinned host staging
// buffer and on the device).
struct Layout {
    int64_t hdr = 0, classes = 0, items = 0, citems = 0, cprefix = 0, sprefix = 0, qslots = 0, total = 0;
    void make(int cap_items, int cap_slots);
};

// Device buffers, tables and the captured launch sequence of one stream of
// batches (the batch API owns one, the serving loop another).
struct Arena {
    int cap_items = 0, cap_slots = 0, cap_states = 0;
    int64_t cap_qf = 0, cap_samples = 0;
    int rr_cap = 0;
    int64_t rr_cap_max = 1 << 25;   // entries per re-run list (a fuller list marks items for a re-run)
    int64_t bytes = 0;
    Layout lay;
    unsigned char* tables = nullptr;     // device
    unsigned char* htables = nullptr;    // pinned host staging
    float* qarena = nullptr;
    int* qbad = nullptr;
    unsigned long long* slots = nullptr;
    float* ub_seed = nullptr;
    int* nbest = nullptr;
    long long* best = nullptr;
    int* flags = nullptr;
    unsigned long long* cost = nullptr;  // [cap_states] GPU cycles per state of the last launch sequence
    float* seed_ed = nullptr;
    int* seed_idx = nullptr;
    int64_t* res_idx = nullptr;
    double* res_dist = nullptr;
    long long* rr = nullptr;             // [kRerunBuffers][3][rr_cap]
    unsigned char* small = nullptr;      // rr counts [16] | work [32] | counters [16] | seed counters [16]
    unsigned char* hbuf = nullptr;       // pinned: flags [cap_states] | query flags [cap_slots] | counters | cost [cap_states]
    int64_t* hres_idx = nullptr;         // pinned result rows (serving)
    double* hres_dist = nullptr;
    cudaStream_t cap_stream = nullptr;   // stream the launch sequence is captured on
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    int* rr_counts() { return reinterpret_cast<int*>(small); }
    unsigned long long* work() { return reinterpret_cast<unsigned long long*>(small + 64); }
    unsigned long long* counters() { return reinterpret_cast<unsigned long long*>(small + 320); }
    unsigned long long* seed_counters() { return reinterpret_cast<unsigned long long*>(small + 448); }
    int* hflags() { return reinterpret_cast<int*>(hbuf); }
    int* hqbad() { return hflags() + cap_states; }
    unsigned long long* hcounters() {
        return reinterpret_cast<unsigned long long*>(hbuf + al8(sizeof(int) * (static_cast<int64_t>(cap_states) + cap_slots)));
    }
    unsigned long long* hcost() { return hcounters() + 2 * kNumCounters; }
    static int64_t al8(int64_t x) { return (x + 7) / 8 * 8; }
};

struct Server;

}  // namespace eapdtw

struct eapdtw_ctx {
    int device = 0;
    int64_t budget = 0;        // bytes (0: no limit of the context's own)
    int64_t used = 0;          // bytes held: references, tables and arenas
    std::mutex mu;             // guards everything below except the server's own state
    std::vector<eapdtw::RefEntry> refs;
    eapdtw::Arena batch;
    // per (log2 m, window ratio in tenths, band mode), set by the autotuner: the
    // first level's K (0: the built-in rule) and the check-interval choice
    // (1: twice the wavefront's built-in interval)
    std::map<std::tuple<int, int, int>, std::pair<int, int>> tuned;
    int64_t batches = 0, items_run = 0, items_rerun = 0;
    eapdtw::Server* server = nullptr;
};

namespace eapdtw {

// Runs a scope with the context's device current, then restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

// One (query, reference) item of a launch sequence, as planned on the host.
struct PlannedItem {
    BatchItem b;      // device descriptor (query pointers filled by the caller)
    int cls = 0;      // tile class (first level x band mode)
    int scls = -1;    // seed class (-1: no seed pass)
    int64_t tiles = 0;
};

// Planning helpers (the caller holds ctx->mu).
std::tuple<int, int, int> signature(int m, int w);
int first_level(const eapdtw_ctx* c, int m, int w);
int check_choice(const eapdtw_ctx* c, int m, int w);   // 1: twice the built-in check interval
int band_mode(int level, int w, bool unconstrained);
int env_level(int radius);
int32_t ensure_env(eapdtw_ctx* c, RefEntry& r, int p, cudaStream_t st);
// Fill everything of `item` but the query pointers, state and window range.
void plan_item(const eapdtw_ctx* c, const RefEntry& r, int64_t n_used, int m, int w, int k, bool no_lb,
               PlannedItem& out);

// Arena management (the caller holds ctx->mu).
int32_t arena_reserve(eapdtw_ctx* c, Arena& a, int items, int qslots, int states, int64_t qf, int64_t samples,
                      int64_t rr_want);
void arena_free(eapdtw_ctx* c, Arena& a);

// Upload the tables of one launch sequence and replay it on `st` (the graph is
// captured on first use).  Tables: the planned items (their seed sample
// offsets are assigned here) and the query slots to prepare.  kstride: row
// length of the results.  Enqueues the copies of the item flags, query flags
// and counters to the arena's pinned buffer; the caller synchronises.
int32_t arena_run(Arena& a, std::vector<PlannedItem>& items, const std::vector<QuerySlot>& qslots, int kstride,
                  cudaStream_t st, bool time_it);

}  // namespace eapdtw
