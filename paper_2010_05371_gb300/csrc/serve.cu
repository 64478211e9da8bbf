// Serving loop of a context (declared in include/eapdtw.h): requests arrive
// from any host thread; a server thread admits them into resident state slots
// and runs rounds of the batched launch sequence (batch.cuh).  Each round
// takes the next windows of every admitted request, so requests that arrive
// while others are on the GPU join at the next round and their work overlaps
// with the others'; a request's k-best list, seed bound and prepared query
// stay on the device from its first round to its last.
//
// How many windows a request gets in a round: the batch kernel measures, per
// request, the SM cycles its warps spent, so each request has an estimate of
// its cost per window after its first round (which takes chunk windows).  A
// round's budget is what chunk windows of every admitted request would cost;
// it goes to the requests in order of their estimated remaining cost
// (shortest remaining first), each at least a floor of windows so that none
// starves, and at most kMaxChunks chunks.  So a cheap request is not held for
// the whole mix: it finishes in a few rounds while the expensive ones go on.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "batch.cuh"
#include "ctx_internal.h"
#include "eapdtw.h"
#include "kernels.h"

namespace eapdtw {

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    std::vector<float> q;   // host copy of the query
    int m = 0, w = 0, k = 0, ref = 0;
    bool no_lb = false;
    int state = -1;         // slot while admitted
    int64_t nw = 0, next = 0;
    bool started = false;
    bool cancel = false;
    bool lost = false;
    double cpw = -1.0;      // estimated SM cycles per window (< 0: not measured yet)
    int32_t status = EAPDTW_PENDING;
    Clock::time_point t_submit, t_admit, t_done;
    int64_t idx[EAPDTW_MAX_K];
    double dist[EAPDTW_MAX_K];
};

}  // namespace

struct Server {
    eapdtw_ctx* c = nullptr;
    std::thread th;
    std::mutex mu;                 // guards the queues, the requests and the statistics
    std::condition_variable cv;    // wakes the server thread
    std::condition_variable done;  // wakes waiters
    bool stop = false;
    int max_active = 0;
    int64_t chunk = 0;
    std::deque<Request*> pending;
    std::vector<Request*> slot;    // [max_active]
    std::unordered_map<int64_t, Request*> reqs;
    int64_t next_id = 1;
    Arena A;
    cudaStream_t st = nullptr;
    float* dq = nullptr;           // raw queries, EAPDTW_MAX_QUERY floats per slot
    int32_t error = EAPDTW_OK;     // a CUDA failure of the loop (sticky)
    // statistics
    int64_t rounds = 0, completed = 0, cancelled = 0, windows = 0, reruns = 0;
    std::vector<int64_t> lat_ns;   // latencies of completed requests

    void loop();
    int32_t round(std::vector<Request*>& act);
};

namespace {

int32_t finish_lost(Server* S, Request* r) {
    // a re-run entry did not fit its list: search the request again alone
    const RefEntry& ref = S->c->refs[r->ref];
    int64_t* di = nullptr;
    double* dd = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&di), sizeof(int64_t) * r->k) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&dd), sizeof(double) * r->k) != cudaSuccess) {
        cudaGetLastError();
        if (di) cudaFree(di);
        return EAPDTW_ERR_OUT_OF_MEMORY;
    }
    eapdtw_search_opts o{};
    o.no_lb = r->no_lb ? 1 : 0;
    int32_t rc = subseq_search_ex(S->dq + static_cast<int64_t>(r->state) * EAPDTW_MAX_QUERY, r->m, ref.R, ref.n, r->w,
                                  r->k, &o, di, dd, S->st);
    if (rc == EAPDTW_OK &&
        (cudaMemcpy(r->idx, di, sizeof(int64_t) * r->k, cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(r->dist, dd, sizeof(double) * r->k, cudaMemcpyDeviceToHost) != cudaSuccess)) {
        cudaGetLastError();
        rc = EAPDTW_ERR_CUDA;
    }
    cudaFree(di);
    cudaFree(dd);
    return rc;
}

}  // namespace

// Windows each admitted request gets in a round (see the file's header).
constexpr int64_t kMaxChunks = 8;
std::vector<int64_t> allocate_windows(const std::vector<Request*>& act, int64_t chunk) {
    std::vector<int64_t> nwin(act.size(), 0);
    const int64_t floor_w = std::max<int64_t>(32, chunk / 16);
    double budget = 0.0;
    std::vector<size_t> known;
    for (size_t i = 0; i < act.size(); ++i) {
        const Request* r = act[i];
        const int64_t rem = r->nw - r->next;
        if (r->cpw < 0.0) {
            nwin[i] = std::min<int64_t>(chunk, rem);   // first round: measure
        } else {
            budget += static_cast<double>(std::min<int64_t>(chunk, rem)) * r->cpw;
            known.push_back(i);
        }
    }
    std::sort(known.begin(), known.end(), [&](size_t a, size_t b) {
        const double ca = static_cast<double>(act[a]->nw - act[a]->next) * act[a]->cpw;
        const double cb = static_cast<double>(act[b]->nw - act[b]->next) * act[b]->cpw;
        return ca < cb || (ca == cb && act[a]->id < act[b]->id);
    });
    // every known request first gets its floor, then the rest of the budget in order
    for (size_t i : known) {
        const Request* r = act[i];
        nwin[i] = std::min<int64_t>(floor_w, r->nw - r->next);
        budget -= static_cast<double>(nwin[i]) * r->cpw;
    }
    for (size_t i : known) {
        const Request* r = act[i];
        const int64_t rem = r->nw - r->next - nwin[i];
        if (rem <= 0 || budget <= 0.0) continue;
        const double afford = r->cpw > 0.0 ? budget / r->cpw : static_cast<double>(rem);
        int64_t extra = std::min<int64_t>(rem, static_cast<int64_t>(std::min(afford, 1e18)));
        extra = std::min<int64_t>(extra, kMaxChunks * chunk - nwin[i]);
        if (extra < rem) extra = extra / 32 * 32;   // whole tiles, or the whole tail
        if (extra <= 0) continue;
        nwin[i] += extra;
        budget -= static_cast<double>(extra) * r->cpw;
    }
    return nwin;
}

// One round over the admitted requests `act` (the server thread; S->mu not held).
int32_t Server::round(std::vector<Request*>& act) {
    std::vector<PlannedItem> P(act.size());
    const std::vector<int64_t> alloc = allocate_windows(act, chunk);
    std::vector<QuerySlot> qs;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (size_t i = 0; i < act.size(); ++i) {
            Request* r = act[i];
            const RefEntry& ref = c->refs[r->ref];
            plan_item(c, ref, ref.n, r->m, r->w, r->k, r->no_lb, P[i]);
            BatchItem& b = P[i].b;
            b.state = r->state;
            b.fresh = r->started ? 0 : 1;
            b.win0 = r->next;
            b.nwin = alloc[i];
            if (r->started) b.seed_ns = 0;   // seeds run in the first round only
            P[i].tiles = (b.nwin + 31) / 32;
            const int64_t off = static_cast<int64_t>(r->state) * 5 * query_pad(EAPDTW_MAX_QUERY);
            const int mp = query_pad(r->m);
            const float* base = A.qarena + off;
            b.zq = base;
            b.uq = base + mp;
            b.lq = base + 2 * mp;
            b.zqo = base + 3 * mp;
            b.ord = reinterpret_cast<const int*>(base + 4 * mp);
            if (!r->started) {
                QuerySlot q{};
                q.Q = dq + static_cast<int64_t>(r->state) * EAPDTW_MAX_QUERY;
                q.m = r->m;
                q.w = r->w;
                q.off = static_cast<int>(off);
                qs.push_back(q);
            }
        }
    }
    for (Request* r : act) {
        if (r->started) continue;
        if (cudaMemcpyAsync(dq + static_cast<int64_t>(r->state) * EAPDTW_MAX_QUERY, r->q.data(), sizeof(float) * r->m,
                            cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            return EAPDTW_ERR_CUDA;
        }
    }
    int32_t rc = arena_run(A, P, qs, EAPDTW_MAX_K, st, false);
    if (rc != EAPDTW_OK) return rc;
    const size_t rows = act.size() * EAPDTW_MAX_K;
    if (cudaMemcpyAsync(A.hres_idx, A.res_idx, sizeof(int64_t) * rows, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(A.hres_dist, A.res_dist, sizeof(double) * rows, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return EAPDTW_ERR_CUDA;
    }
    const int* hf = A.hflags();
    const int* hqb = A.hqbad();
    int qi = 0;
    std::vector<Request*> lost;
    std::vector<char> bad(act.size(), 0);
    std::vector<char> tmo(act.size(), 0);
    {
        std::lock_guard<std::mutex> lk(mu);
        ++rounds;
        for (size_t i = 0; i < act.size(); ++i) {
            Request* r = act[i];
            if (!r->started && hqb[qi++]) {
                bad[i] = 1;   // the status is set below, with the slot released
                r->next = r->nw;
            }
            r->started = true;
            if (hf[r->state] & kFlagTimeout) {   // a device-side wait ran out: the request fails
                tmo[i] = 1;
                r->next = r->nw;
            }
            r->lost |= (hf[r->state] & kFlagLost) != 0;
            windows += P[i].b.nwin;
            // cost per window: this round's measurement, smoothed over rounds
            // (the first round also prepared the query and ran the seeds)
            if (P[i].b.nwin > 0) {
                const double c = static_cast<double>(A.hcost()[r->state]) / static_cast<double>(P[i].b.nwin);
                r->cpw = r->cpw < 0.0 ? c : 0.5 * (r->cpw + c);
            }
            if (r->status == EAPDTW_PENDING) r->next += P[i].b.nwin;
            if (r->next >= r->nw) {
                std::memcpy(r->idx, A.hres_idx + i * EAPDTW_MAX_K, sizeof(int64_t) * r->k);
                std::memcpy(r->dist, A.hres_dist + i * EAPDTW_MAX_K, sizeof(double) * r->k);
                if (r->lost && !bad[i] && !tmo[i]) lost.push_back(r);
            }
        }
    }
    std::vector<int32_t> lost_rc(lost.size(), EAPDTW_OK);
    for (size_t j = 0; j < lost.size(); ++j) lost_rc[j] = finish_lost(this, lost[j]);
    {
        std::lock_guard<std::mutex> lk(mu);
        reruns += static_cast<int64_t>(lost.size());
        for (size_t i = 0; i < act.size(); ++i) {
            Request* r = act[i];
            if (r->next < r->nw) continue;
            int32_t rs = bad[i] ? EAPDTW_ERR_NAN_INPUT : (tmo[i] ? EAPDTW_ERR_TIMEOUT : EAPDTW_OK);
            for (size_t j = 0; j < lost.size(); ++j)
                if (lost[j] == r && lost_rc[j] != EAPDTW_OK) rs = lost_rc[j];
            r->t_done = Clock::now();
            if (rs == EAPDTW_OK) {
                ++completed;
                lat_ns.push_back(std::chrono::duration_cast<std::chrono::nanoseconds>(r->t_done - r->t_submit).count());
            }
            r->status = rs;   // from here on a poller may take (and free) the request
            slot[r->state] = nullptr;
            r->state = -1;
            {
                std::lock_guard<std::mutex> lk2(c->mu);
                --c->refs[r->ref].users;
            }
        }
    }
    done.notify_all();
    return EAPDTW_OK;
}

void Server::loop() {
    cudaSetDevice(c->device);
    for (;;) {
        std::vector<Request*> act;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] {
                if (stop) return true;
                if (!pending.empty()) return true;
                for (Request* r : slot)
                    if (r) return true;
                return false;
            });
            if (stop) break;
            // cancelled requests leave at the round boundary
            for (int s = 0; s < max_active; ++s) {
                Request* r = slot[s];
                if (r && r->cancel) {
                    r->status = EAPDTW_ERR_CANCELLED;
                    ++cancelled;
                    slot[s] = nullptr;
                    r->state = -1;
                    std::lock_guard<std::mutex> lk2(c->mu);
                    --c->refs[r->ref].users;
                }
            }
            // admission: a free state slot, and the memory the request needs
            // (the reference's envelope table up to its radius)
            while (!pending.empty()) {
                int s = 0;
                while (s < max_active && slot[s]) ++s;
                if (s == max_active) break;
                Request* r = pending.front();
                pending.pop_front();
                if (r->cancel) {
                    r->status = EAPDTW_ERR_CANCELLED;
                    ++cancelled;
                    continue;
                }
                int32_t e = EAPDTW_OK;
                {
                    std::lock_guard<std::mutex> lk2(c->mu);
                    RefEntry& ref = c->refs[r->ref];
                    if (!r->no_lb) e = ensure_env(c, ref, env_level(std::min(r->w, r->m - 1)), st);
                    if (e == EAPDTW_OK) ++ref.users;
                }
                if (e != EAPDTW_OK) {
                    r->status = e;
                    continue;
                }
                r->state = s;
                r->t_admit = Clock::now();
                slot[s] = r;
            }
            for (Request* r : slot)
                if (r) act.push_back(r);
        }
        done.notify_all();
        if (act.empty()) continue;
        const int32_t e = round(act);
        if (e != EAPDTW_OK) {
            std::lock_guard<std::mutex> lk(mu);
            error = e;
            for (Request* r : act) {
                if (r->status == EAPDTW_PENDING) r->status = e;
                if (r->state >= 0) slot[r->state] = nullptr;
                r->state = -1;
                std::lock_guard<std::mutex> lk2(c->mu);
                --c->refs[r->ref].users;
            }
            done.notify_all();
        }
    }
}

int32_t server_shutdown(eapdtw_ctx* c) {
    Server* S = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        S = c->server;
        c->server = nullptr;
    }
    if (!S) return EAPDTW_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    {
        std::lock_guard<std::mutex> lk(c->mu);
        DeviceGuard g(c->device);
        cudaStreamSynchronize(S->st);
        for (Request* r : S->slot)
            if (r) --c->refs[r->ref].users;
        arena_free(c, S->A);
        if (S->A.cap_stream) cudaStreamDestroy(S->A.cap_stream);
        if (S->dq) {
            cudaFree(S->dq);
            c->used -= sizeof(float) * static_cast<int64_t>(S->max_active) * EAPDTW_MAX_QUERY;
        }
        if (S->st) cudaStreamDestroy(S->st);
    }
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
    return EAPDTW_OK;
}

}  // namespace eapdtw

using namespace eapdtw;

extern "C" {

int32_t eapdtw_serve_start(eapdtw_ctx* c, int32_t max_active, int64_t chunk_windows) {
    if (!c || max_active < 1 || max_active > 4096 || chunk_windows < 32) return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->server) return EAPDTW_ERR_BUSY;
    DeviceGuard g(c->device);
    if (!g.ok) return EAPDTW_ERR_CUDA;
    Server* S = new (std::nothrow) Server;
    if (!S) return EAPDTW_ERR_OUT_OF_MEMORY;
    S->c = c;
    S->max_active = max_active;
    S->chunk = (chunk_windows + 31) / 32 * 32;
    S->slot.assign(max_active, nullptr);
    S->A.rr_cap_max = c->batch.rr_cap_max;
    const int64_t dq_bytes = sizeof(float) * static_cast<int64_t>(max_active) * EAPDTW_MAX_QUERY;
    auto fail = [&](int32_t rc) {
        arena_free(c, S->A);
        if (S->dq) {
            cudaFree(S->dq);
            c->used -= dq_bytes;
        }
        if (S->st) cudaStreamDestroy(S->st);
        delete S;
        return rc;
    };
    if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(EAPDTW_ERR_CUDA);
    }
    if (cudaMalloc(reinterpret_cast<void**>(&S->dq), dq_bytes) != cudaSuccess) {
        cudaGetLastError();
        S->dq = nullptr;
        return fail(EAPDTW_ERR_OUT_OF_MEMORY);
    }
    c->used += dq_bytes;
    // the arena for max_active items in max_active states, each round's
    // re-run lists sized for every admitted request's chunk (a round may give
    // one request up to kMaxChunks chunks; a list that fills up marks its
    // items for a search alone, so the results never depend on the sizing)
    const int64_t qf = static_cast<int64_t>(max_active) * 5 * query_pad(EAPDTW_MAX_QUERY);
    const int64_t samples = static_cast<int64_t>(max_active) * kBatchSeedSamples;
    const int64_t rr = static_cast<int64_t>(max_active) * (S->chunk + kBatchSeedBest);
    int32_t rc = arena_reserve(c, S->A, max_active, max_active, max_active, qf, samples, rr);
    if (rc == EAPDTW_OK && c->budget > 0 && c->used > c->budget) rc = EAPDTW_ERR_OUT_OF_MEMORY;
    if (rc != EAPDTW_OK) return fail(rc);
    try {
        S->th = std::thread([S] { S->loop(); });
    } catch (...) {
        return fail(EAPDTW_ERR_INTERNAL);
    }
    c->server = S;
    return EAPDTW_OK;
}

int32_t eapdtw_serve_stop(eapdtw_ctx* c) {
    if (!c) return EAPDTW_ERR_INVALID_ARG;
    return server_shutdown(c);
}

int32_t eapdtw_serve_submit(eapdtw_ctx* c, const float* Q, int64_t lQ, int32_t ref_id, int64_t w, int32_t k,
                            int32_t no_lb, int64_t* req_id) {
    if (!c || !Q || lQ < 1 || w < 0 || k < 1 || !req_id) return EAPDTW_ERR_INVALID_ARG;
    if (lQ > EAPDTW_MAX_QUERY || k > EAPDTW_MAX_K) return EAPDTW_ERR_UNSUPPORTED;
    Server* S = nullptr;
    int64_t n = 0;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        S = c->server;
        if (!S) return EAPDTW_ERR_INVALID_ARG;
        if (ref_id < 0 || ref_id >= static_cast<int32_t>(c->refs.size()) || !c->refs[ref_id].live)
            return EAPDTW_ERR_INVALID_ARG;
        n = c->refs[ref_id].n;
    }
    if (lQ > n) return EAPDTW_ERR_INVALID_ARG;
    Request* r = new (std::nothrow) Request;
    if (!r) return EAPDTW_ERR_OUT_OF_MEMORY;
    r->q.assign(Q, Q + lQ);
    r->m = static_cast<int>(lQ);
    r->w = static_cast<int>(w < lQ ? w : lQ);
    r->k = k;
    r->ref = ref_id;
    r->no_lb = no_lb != 0;
    r->nw = n - lQ + 1;
    for (int j = 0; j < EAPDTW_MAX_K; ++j) {
        r->idx[j] = -1;
        r->dist[j] = INFINITY;
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return EAPDTW_ERR_INVALID_ARG;
        }
        r->id = S->next_id++;
        S->reqs[r->id] = r;
        S->pending.push_back(r);
    }
    S->cv.notify_all();
    *req_id = r->id;
    return EAPDTW_OK;
}

int32_t eapdtw_serve_poll(eapdtw_ctx* c, int64_t req_id, int64_t* out_idx, double* out_dist, int64_t* latency_ns,
                          int32_t timeout_ms) {
    if (!c) return EAPDTW_ERR_INVALID_ARG;
    Server* S = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        S = c->server;
    }
    if (!S) return EAPDTW_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto f = S->reqs.find(req_id);
    if (f == S->reqs.end()) return EAPDTW_ERR_INVALID_ARG;
    Request* r = f->second;
    if (timeout_ms > 0) {
        S->done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->status != EAPDTW_PENDING; });
    }
    if (r->status == EAPDTW_PENDING) return EAPDTW_PENDING;
    const int32_t st = r->status;
    if (st == EAPDTW_OK) {
        if (out_idx) std::memcpy(out_idx, r->idx, sizeof(int64_t) * r->k);
        if (out_dist) std::memcpy(out_dist, r->dist, sizeof(double) * r->k);
        if (latency_ns)
            *latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(r->t_done - r->t_submit).count();
    }
    S->reqs.erase(f);
    delete r;
    return st;
}

int32_t eapdtw_serve_cancel(eapdtw_ctx* c, int64_t req_id) {
    if (!c) return EAPDTW_ERR_INVALID_ARG;
    Server* S = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        S = c->server;
    }
    if (!S) return EAPDTW_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto f = S->reqs.find(req_id);
        if (f == S->reqs.end()) return EAPDTW_ERR_INVALID_ARG;
        f->second->cancel = true;
        // a request still waiting for admission leaves at once
        auto it = std::find(S->pending.begin(), S->pending.end(), f->second);
        if (it != S->pending.end()) {
            S->pending.erase(it);
            f->second->status = EAPDTW_ERR_CANCELLED;
            ++S->cancelled;
        }
    }
    S->cv.notify_all();
    S->done.notify_all();
    return EAPDTW_OK;
}

int32_t eapdtw_serve_stats(eapdtw_ctx* c, int64_t* out, int32_t nout) {
    if (!c || !out || nout < 1) return EAPDTW_ERR_INVALID_ARG;
    Server* S = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        S = c->server;
    }
    if (!S) return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t active = 0;
    for (Request* r : S->slot) active += r ? 1 : 0;
    std::vector<int64_t> l = S->lat_ns;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) -> int64_t {
        if (l.empty()) return -1;
        const size_t i = static_cast<size_t>(p * static_cast<double>(l.size() - 1) + 0.5);
        return l[std::min(i, l.size() - 1)];
    };
    const int64_t v[EAPDTW_SERVE_NSTATS] = {S->completed, S->cancelled, static_cast<int64_t>(S->pending.size()),
                                           active, S->rounds, S->windows, pct(0.5), pct(0.99), S->reruns,
                                           S->error};
    for (int i = 0; i < nout && i < EAPDTW_SERVE_NSTATS; ++i) out[i] = v[i];
    return EAPDTW_OK;
}

}  // extern "C"
