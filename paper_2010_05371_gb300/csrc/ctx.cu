// Contexts, resident references and the batched search (declared in
// include/eapdtw.h): many (query, reference) items run as one fixed sequence
// of persistent launches (batch.cuh), captured once into a CUDA graph and
// replayed for every batch with new device-side work tables.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "batch.cuh"
#include "ctx_internal.h"
#include "eapdtw.h"
#include "kernels.h"
#include "plan.h"

namespace eapdtw {

int32_t server_shutdown(eapdtw_ctx* c);  // serve.cu

namespace {

int64_t al256(int64_t x) { return (x + 255) / 256 * 256; }

#define CKC(expr)                    \
    do {                             \
        if ((expr) != cudaSuccess) { \
            cudaGetLastError();      \
            return EAPDTW_ERR_CUDA;  \
        }                            \
    } while (0)

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

template <typename T>
bool dalloc(T*& p, int64_t count, int64_t& bytes) {
    p = nullptr;
    const size_t b = sizeof(T) * static_cast<size_t>(count > 0 ? count : 1);
    if (cudaMalloc(reinterpret_cast<void**>(&p), b) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return false;
    }
    bytes += static_cast<int64_t>(b);
    return true;
}

void free_ref(RefEntry& r) {
    for (int p = 1; p < kEnvLevels; ++p) {
        dfree(r.emax[p]);
        dfree(r.emin[p]);
    }
    dfree(r.R); dfree(r.P1); dfree(r.P2); dfree(r.T1); dfree(r.T2); dfree(r.A);
    r = RefEntry{};
}

int64_t grow(int64_t want, int64_t have) {
    if (want <= have) return have;
    int64_t c = 64;
    while (c < want) c *= 2;
    return c;
}

void drop_graph(Arena& a) {
    if (a.exec) cudaGraphExecDestroy(a.exec);
    if (a.graph) cudaGraphDestroy(a.graph);
    a.exec = nullptr;
    a.graph = nullptr;
}

BatchDev dev_view(Arena& a) {
    BatchDev D{};
    const Layout& L = a.lay;
    D.nitems = reinterpret_cast<const int*>(a.tables + L.hdr);
    D.nslots = D.nitems + 1;
    D.kstride = D.nitems + 2;
    D.classes = reinterpret_cast<const BatchClass*>(a.tables + L.classes);
    D.items = reinterpret_cast<const BatchItem*>(a.tables + L.items);
    D.citems = reinterpret_cast<const int*>(a.tables + L.citems);
    D.cprefix = reinterpret_cast<const int64_t*>(a.tables + L.cprefix);
    D.sprefix = reinterpret_cast<const int64_t*>(a.tables + L.sprefix);
    D.qslots = reinterpret_cast<const QuerySlot*>(a.tables + L.qslots);
    D.qarena = a.qarena;
    D.qbad = a.qbad;
    D.slots = a.slots;
    D.ub_seed = a.ub_seed;
    D.nbest = a.nbest;
    D.best = a.best;
    D.flags = a.flags;
    D.cost = a.cost;
    D.seed_ed = a.seed_ed;
    D.seed_idx = a.seed_idx;
    D.res_idx = a.res_idx;
    D.res_dist = a.res_dist;
    return D;
}

cudaError_t batch_attrs_once() {
    static std::once_flag once[64];
    static cudaError_t err[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        err[dev] = batch_prep_attributes(EAPDTW_MAX_QUERY);
        if (err[dev] == cudaSuccess) err[dev] = batch_attributes();
    });
    return err[dev];
}

// The launch sequence of one batch; every count it needs is read on the device.
cudaError_t enqueue_sequence(Arena& a, cudaStream_t s) {
    const BatchDev D = dev_view(a);
    int* rrc = a.rr_counts();
    cudaError_t e = launch_batch_prep(D, a.cap_items, a.counters(), 2 * kNumCounters, a.work(), kNumWork, rrc,
                                      3 * kRerunBuffers, EAPDTW_MAX_QUERY, s);
    if (e != cudaSuccess) return e;
    // seed passes at each query's widest level, where no live region overflows
    for (int sc = 0; sc < kSeedClasses; ++sc) {
        BatchLaunch L{};
        L.D = D;
        L.level = 3 + sc / 3;
        L.band = sc % 3;
        L.cls = -1;
        L.scls = kBatchClasses + sc;
        L.rr_in = nullptr;
        L.rr_in_count = rrc;
        L.rr = a.rr;
        L.rr_count = rrc;
        L.rr_cap = 0;
        L.work = a.work() + kBatchLevels * 3 + sc;
        L.counters = a.seed_counters();
        L.lb_scale = kBatchLbScale;
        e = launch_batch(L.level, L.band, L, batch_blocks(L.level, L.band), s);
        if (e != cudaSuccess) return e;
    }
    // The re-run lists of levels 1, 2 and 3 (buffers 1, 2, 0) start empty: the
    // elastic first level and levels 0..2 fill them.  Levels 4 and 5 reuse
    // buffers 1 and 2 once levels 1 and 2 have read them.
    e = cudaMemsetAsync(rrc, 0, sizeof(int) * 3 * kRerunBuffers, s);
    if (e != cudaSuccess) return e;
    for (int ec = 0; ec < kElClasses; ++ec) {
        BatchLaunch L{};
        L.D = D;
        L.level = kElLevel;
        L.band = ec & 1;
        L.cls = kElClass0 + ec;
        L.scls = -1;
        L.rr_in = nullptr;
        L.rr_in_count = rrc;
        L.rr = a.rr;
        L.rr_count = rrc;
        L.rr_cap = a.rr_cap;
        L.work = a.work() + kElWork0 + ec;
        L.counters = a.counters();
        L.lb_scale = kBatchLbScale;
        e = launch_batch_elastic(ec, L, batch_blocks_el(ec), s);
        if (e != cudaSuccess) return e;
    }
    for (int level = 0; level < kBatchLevels; ++level) {
        if (level == 3) {   // the lists of levels 4 and 5
            e = cudaMemsetAsync(rrc + 3 * (4 % kRerunBuffers), 0, sizeof(int) * 3, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(rrc + 3 * (5 % kRerunBuffers), 0, sizeof(int) * 3, s);
            if (e != cudaSuccess) return e;
        }
        const int bin = level % kRerunBuffers;
        for (int band = 0; band < 3; ++band) {
            BatchLaunch L{};
            L.D = D;
            L.level = level;
            L.band = band;
            L.cls = level < 4 ? level * 3 + band : -1;
            L.scls = -1;
            L.rr_in = level > 0 ? a.rr + static_cast<int64_t>(3 * bin + band) * a.rr_cap : nullptr;
            L.rr_in_count = rrc + 3 * bin + band;
            L.rr = a.rr;
            L.rr_count = rrc;
            L.rr_cap = a.rr_cap;
            L.work = a.work() + level * 3 + band;
            L.counters = a.counters();
            L.lb_scale = kBatchLbScale;
            e = launch_batch(level, band, L, batch_blocks(level, band), s);
            if (e != cudaSuccess) return e;
        }
    }
    return launch_batch_finalize(D, s);
}

int32_t ensure_graph(Arena& a) {
    if (a.exec) return EAPDTW_OK;
    if (batch_attrs_once() != cudaSuccess) { cudaGetLastError(); return EAPDTW_ERR_CUDA; }
    // occupancy queries before the capture (they are not stream work)
    for (int level = 0; level < kBatchLevels; ++level)
        for (int band = 0; band < 3; ++band) batch_blocks(level, band);
    for (int ec = 0; ec < kElClasses; ++ec) batch_blocks_el(ec);
    if (!a.cap_stream && cudaStreamCreateWithFlags(&a.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return EAPDTW_ERR_CUDA;
    }
    if (cudaStreamBeginCapture(a.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return EAPDTW_ERR_CUDA;
    }
    const cudaError_t e = enqueue_sequence(a, a.cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(a.cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return EAPDTW_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&a.exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        a.exec = nullptr;
        return EAPDTW_ERR_CUDA;
    }
    a.graph = g;
    return EAPDTW_OK;
}

}  // namespace

void Layout::make(int cap_items, int cap_slots) {
    hdr = 0;
    classes = 256;
    items = al256(classes + sizeof(BatchClass) * kAllClasses);
    citems = al256(items + sizeof(BatchItem) * static_cast<int64_t>(cap_items));
    cprefix = al256(citems + sizeof(int) * 2 * static_cast<int64_t>(cap_items));
    sprefix = al256(cprefix + sizeof(int64_t) * static_cast<int64_t>(cap_items + kBatchClasses));
    qslots = al256(sprefix + sizeof(int64_t) * static_cast<int64_t>(cap_items + 1));
    total = al256(qslots + sizeof(QuerySlot) * static_cast<int64_t>(cap_slots));
}

DeviceGuard::DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        prev = -1;
        return;
    }
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
    if (!ok) cudaGetLastError();
}

DeviceGuard::~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
}

// Level of the table for envelope radius r: the largest p with 2^p <= 2r + 1.
int env_level(int r) {
    int p = 0;
    while ((2 << p) <= 2 * r + 1) ++p;
    return p;
}

// Build the reference's running-extrema table up to level p (blocking).
int32_t ensure_env(eapdtw_ctx* c, RefEntry& r, int p, cudaStream_t st) {
    if (p < r.env_levels) return EAPDTW_OK;
    for (int q = r.env_levels; q <= p; ++q) {
        int64_t bytes = 0;
        if (!dalloc(r.emax[q], r.n, bytes) || !dalloc(r.emin[q], r.n, bytes) ||
            (c->budget > 0 && c->used + bytes > c->budget)) {
            dfree(r.emax[q]);
            dfree(r.emin[q]);
            return EAPDTW_ERR_OUT_OF_MEMORY;
        }
        if (launch_env_level(r.emax[q - 1], r.emin[q - 1], r.n, int64_t(1) << (q - 1), r.emax[q], r.emin[q], st) !=
            cudaSuccess) {
            cudaGetLastError();
            dfree(r.emax[q]);
            dfree(r.emin[q]);
            return EAPDTW_ERR_CUDA;
        }
        c->used += bytes;
        r.bytes += bytes;
        r.env_levels = q + 1;
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? EAPDTW_OK : EAPDTW_ERR_CUDA;
}

// Signature of an item for the first-level table.
std::tuple<int, int, int> signature(int m, int w) {
    const bool unc = w >= m - 1;
    int lg = 0;
    while ((2 << lg) <= m) ++lg;
    const int tenth = unc ? 10 : std::min(9, static_cast<int>(10.0 * w / m));
    return std::make_tuple(lg, tenth, unc ? 0 : 1);
}

// One-warp level (block width 4 << level) of a (query length, window) pair:
// the narrowest K whose window of 32 blocks covers the band with margin or
// every column, 8 (or 4 for short queries) when unconstrained.
int rule_level(int m, int w) {
    const bool unconstrained = w >= m - 1;
    int K = 32;
    if (!unconstrained) {
        for (int k = 4; k <= 32; k *= 2)
            if ((2 * w + k) / (k + 1) + 3 <= 32 || 32 * k >= m) { K = k; break; }
    } else {
        K = 8;
        for (int k = 4; k <= 8; k *= 2)
            if (32 * k >= m) { K = k; break; }
    }
    int level = 0;
    while ((4 << level) < K) ++level;
    return level;
}

// Whether the elastic wavefront can be the first level: queries of 129 to
// kElMaxM points, unconstrained or with a band as wide as the one-query
// search's plan asks (plan.h).
bool elastic_ok(int m, int w) {
    if (m <= 128 || m > kElMaxM) return false;
    return w >= m - 1 || (w >= kElBandMinW && 4 * w >= kElBandMinQuarters * m);
}

// First level of a pair: the autotuner's choice (tile 1: the elastic
// wavefront; 4..32: that one-warp level), else the elastic wavefront where it
// can run for queries of up to 1024 points, else rule_level.  Longer queries
// start on one warp: measured on the batched mix, their wide bands come with
// wide live regions (long ECG-like queries against random walks), most
// candidates are handed over, and the elastic pass made those items 3-6%
// slower (the autotuner may still choose it).
int first_level(const eapdtw_ctx* c, int m, int w) {
    auto it = c->tuned.find(signature(m, w));
    if (it != c->tuned.end() && it->second.first) {
        const int K = it->second.first;
        if (K == kTileElastic) return elastic_ok(m, w) ? kElLevel : rule_level(m, w);
        int level = 0;
        while ((4 << level) < K) ++level;
        return level;
    }
    return (m <= 1024 && elastic_ok(m, w)) ? kElLevel : rule_level(m, w);
}
int check_choice(const eapdtw_ctx* c, int m, int w) {
    auto it = c->tuned.find(signature(m, w));
    return it != c->tuned.end() ? it->second.second : 0;
}

int band_mode(int level, int w, bool unconstrained) {
    const int K = batch_level_K(level);
    return unconstrained ? 0 : (K <= 2 * w + 2 ? 1 : 2);
}

void plan_item(const eapdtw_ctx* c, const RefEntry& r, int64_t n_used, int m, int w, int k, bool no_lb,
               PlannedItem& out) {
    BatchItem& b = out.b;
    b = BatchItem{};
    const bool unc = w >= m - 1;
    b.ref = RefView{r.R, n_used, r.P1, r.P2, r.T1, r.T2, r.A};
    b.nw = n_used - m + 1;
    b.win0 = 0;
    b.nwin = b.nw;
    b.m = m;
    b.w = w;
    b.k = k;
    b.use_lb = no_lb ? 0 : 1;
    b.seed_ns = b.nw >= 2048 ? static_cast<int>(std::min<int64_t>(b.nw, kBatchSeedSamples)) : 0;
    b.level0 = first_level(c, m, w);
    b.check2 = check_choice(c, m, w);
    const int last = batch_last_level(m);
    for (int lv = 0; lv < kBatchLevels; ++lv) {
        const int nx = lv < 3 ? lv + 1 : (lv == 3 && last > 3 ? last : -1);
        b.next_level[lv] = nx;
        b.next_band[lv] = nx >= 0 ? band_mode(nx, w, unc) : -1;
    }
    // the elastic level hands its overflows to K = 16 (unconstrained: its
    // windows hold 384 columns) or to the band's one-warp level
    const int enx = unc ? 2 : rule_level(m, w);
    b.next_level[kElLevel] = enx;
    b.next_band[kElLevel] = band_mode(enx, w, unc);
    const int er = std::min(w, m - 1);
    const int ep = env_level(er);
    b.ec_w = er;
    b.ec_d = er - (1 << ep) + 1;
    b.eu = no_lb ? nullptr : r.emax[ep];
    b.el = no_lb ? nullptr : r.emin[ep];
    b.fresh = 1;
    out.cls = b.level0 == kElLevel ? kElClass0 + 2 * (m > 1024 ? 1 : 0) + (unc ? 0 : 1)
                                   : b.level0 * 3 + band_mode(b.level0, w, unc);
    out.scls = kBatchClasses + 3 * (last - 3) + band_mode(last, w, unc);
    out.tiles = (b.nwin + 31) / 32;
}

void arena_free(eapdtw_ctx* c, Arena& a) {
    drop_graph(a);
    dfree(a.tables); dfree(a.qarena); dfree(a.qbad); dfree(a.slots); dfree(a.ub_seed);
    dfree(a.nbest); dfree(a.best); dfree(a.flags); dfree(a.cost); dfree(a.seed_ed); dfree(a.seed_idx);
    dfree(a.res_idx); dfree(a.res_dist); dfree(a.rr); dfree(a.small);
    if (a.htables) cudaFreeHost(a.htables);
    if (a.hbuf) cudaFreeHost(a.hbuf);
    if (a.hres_idx) cudaFreeHost(a.hres_idx);
    if (a.hres_dist) cudaFreeHost(a.hres_dist);
    a.htables = nullptr;
    a.hbuf = nullptr;
    a.hres_idx = nullptr;
    a.hres_dist = nullptr;
    c->used -= a.bytes;
    a.bytes = 0;
    a.cap_items = a.cap_slots = a.cap_states = 0;
    a.cap_qf = a.cap_samples = 0;
    a.rr_cap = 0;
}

int32_t arena_reserve(eapdtw_ctx* c, Arena& a, int items, int qslots, int states, int64_t qf, int64_t samples,
                      int64_t rr_want) {
    const int64_t ci = grow(items, a.cap_items), cs = grow(qslots, a.cap_slots), ct = grow(states, a.cap_states);
    const int64_t cq = grow(qf, a.cap_qf), cm = grow(samples, a.cap_samples);
    const int64_t cr = std::max<int64_t>(std::min<int64_t>(grow(rr_want, a.rr_cap), a.rr_cap_max), 1);
    if (ci == a.cap_items && cs == a.cap_slots && ct == a.cap_states && cq == a.cap_qf && cm == a.cap_samples &&
        cr <= a.rr_cap && a.tables)
        return EAPDTW_OK;
    arena_free(c, a);
    Layout lay;
    lay.make(static_cast<int>(ci), static_cast<int>(cs));
    int64_t bytes = 0;
    const int64_t rows = ci * EAPDTW_MAX_K;
    const bool ok = dalloc(a.tables, lay.total, bytes) && dalloc(a.qarena, cq, bytes) && dalloc(a.qbad, cs, bytes) &&
                    dalloc(a.slots, ct * kBatchSlots, bytes) && dalloc(a.ub_seed, ct, bytes) &&
                    dalloc(a.nbest, ct, bytes) && dalloc(a.best, ct * kBatchSeedBest, bytes) &&
                    dalloc(a.flags, ct, bytes) && dalloc(a.cost, ct, bytes) && dalloc(a.seed_ed, cm, bytes) &&
                    dalloc(a.seed_idx, cm, bytes) &&
                    dalloc(a.res_idx, rows, bytes) && dalloc(a.res_dist, rows, bytes) &&
                    dalloc(a.rr, 3 * kRerunBuffers * cr, bytes) && dalloc(a.small, 1024, bytes);
    a.bytes = bytes;
    c->used += bytes;
    if (!ok || (c->budget > 0 && c->used > c->budget)) {
        arena_free(c, a);
        return EAPDTW_ERR_OUT_OF_MEMORY;
    }
    const size_t hb = Arena::al8(sizeof(int) * (ct + cs)) + sizeof(unsigned long long) * (2 * kNumCounters + ct);
    if (cudaHostAlloc(reinterpret_cast<void**>(&a.htables), lay.total, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&a.hbuf), hb, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&a.hres_idx), sizeof(int64_t) * rows, cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&a.hres_dist), sizeof(double) * rows, cudaHostAllocDefault) !=
            cudaSuccess) {
        cudaGetLastError();
        arena_free(c, a);
        return EAPDTW_ERR_OUT_OF_MEMORY;
    }
    a.lay = lay;
    a.cap_items = static_cast<int>(ci);
    a.cap_slots = static_cast<int>(cs);
    a.cap_states = static_cast<int>(ct);
    a.cap_qf = cq;
    a.cap_samples = cm;
    a.rr_cap = static_cast<int>(cr);
    return EAPDTW_OK;
}

int32_t arena_run(Arena& a, std::vector<PlannedItem>& items, const std::vector<QuerySlot>& qslots, int kstride,
                  cudaStream_t st, bool time_it) {
    const int n = static_cast<int>(items.size());
    const int nslots = static_cast<int>(qslots.size());
    const Layout& L = a.lay;
    unsigned char* H = a.htables;
    int* hdr = reinterpret_cast<int*>(H + L.hdr);
    hdr[0] = n;
    hdr[1] = nslots;
    hdr[2] = kstride;
    BatchClass* cls = reinterpret_cast<BatchClass*>(H + L.classes);
    BatchItem* hit = reinterpret_cast<BatchItem*>(H + L.items);
    int* citems = reinterpret_cast<int*>(H + L.citems);
    int64_t* cprefix = reinterpret_cast<int64_t*>(H + L.cprefix);
    int64_t* sprefix = reinterpret_cast<int64_t*>(H + L.sprefix);
    QuerySlot* hq = reinterpret_cast<QuerySlot*>(H + L.qslots);
    if (nslots) std::memcpy(hq, qslots.data(), sizeof(QuerySlot) * nslots);
    int cnt[kAllClasses] = {0};
    for (const PlannedItem& p : items) {
        ++cnt[p.cls];
        if (p.scls >= 0 && p.b.seed_ns > 0) ++cnt[p.scls];
    }
    int off = 0;
    for (int k = 0; k < kAllClasses; ++k) {
        cls[k].item_off = off;
        cls[k].nitems = 0;
        off += cnt[k];
    }
    sprefix[0] = 0;
    for (int i = 0; i < n; ++i) {
        PlannedItem& p = items[i];
        p.b.seed_off = sprefix[i];
        hit[i] = p.b;
        sprefix[i + 1] = sprefix[i] + p.b.seed_ns;
        BatchClass& k = cls[p.cls];
        citems[k.item_off + k.nitems++] = i;
        if (p.scls >= 0 && p.b.seed_ns > 0) {
            BatchClass& sk = cls[p.scls];
            citems[sk.item_off + sk.nitems++] = i;
        }
    }
    for (int k = 0; k < kBatchClasses; ++k) {
        int64_t* pre = cprefix + cls[k].item_off + k;
        pre[0] = 0;
        for (int j = 0; j < cls[k].nitems; ++j) pre[j + 1] = pre[j] + items[citems[cls[k].item_off + j]].tiles;
    }
    auto up = [&](int64_t o, int64_t bytes) {
        return cudaMemcpyAsync(a.tables + o, H + o, static_cast<size_t>(bytes), cudaMemcpyHostToDevice, st);
    };
    CKC(up(L.hdr, 64));
    CKC(up(L.classes, sizeof(BatchClass) * kAllClasses));
    CKC(up(L.items, sizeof(BatchItem) * static_cast<int64_t>(n)));
    CKC(up(L.citems, sizeof(int) * static_cast<int64_t>(off)));
    CKC(up(L.cprefix, sizeof(int64_t) * static_cast<int64_t>(n + kBatchClasses)));
    CKC(up(L.sprefix, sizeof(int64_t) * static_cast<int64_t>(n + 1)));
    if (nslots) CKC(up(L.qslots, sizeof(QuerySlot) * static_cast<int64_t>(nslots)));
    const int32_t rc = ensure_graph(a);
    if (rc != EAPDTW_OK) return rc;
    if (time_it) {
        if (!a.ev0 && (cudaEventCreate(&a.ev0) != cudaSuccess || cudaEventCreate(&a.ev1) != cudaSuccess)) {
            cudaGetLastError();
            return EAPDTW_ERR_CUDA;
        }
        CKC(cudaEventRecord(a.ev0, st));
    }
    CKC(cudaGraphLaunch(a.exec, st));
    if (time_it) CKC(cudaEventRecord(a.ev1, st));
    CKC(cudaMemcpyAsync(a.hflags(), a.flags, sizeof(int) * a.cap_states, cudaMemcpyDeviceToHost, st));
    if (nslots) CKC(cudaMemcpyAsync(a.hqbad(), a.qbad, sizeof(int) * nslots, cudaMemcpyDeviceToHost, st));
    CKC(cudaMemcpyAsync(a.hcounters(), a.counters(), sizeof(unsigned long long) * 2 * kNumCounters,
                        cudaMemcpyDeviceToHost, st));
    CKC(cudaMemcpyAsync(a.hcost(), a.cost, sizeof(unsigned long long) * a.cap_states, cudaMemcpyDeviceToHost, st));
    return EAPDTW_OK;
}

namespace {

// The batched search with the context locked and its device current.
// ref_len (optional): item i searches only the first ref_len[i] points of its
// reference (a multiple of the statistics chunk, or the whole reference).
// graph_ms (optional): device time of the launch sequence.
int32_t run_batch(eapdtw_ctx* c, const eapdtw_item* items, int32_t n, int32_t kstride, int64_t* out_idx,
                  double* out_dist, int64_t* counters, void* stream, const int64_t* ref_len, float* graph_ms) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<PlannedItem> P(n);
    std::vector<int64_t> nused(n);
    std::map<std::tuple<const float*, int, int>, int> slot_of;
    std::vector<QuerySlot> slots;
    std::vector<int> slot_idx(n);
    int64_t qf = 0, samples = 0, sum_nw = 0;
    for (int i = 0; i < n; ++i) {
        const eapdtw_item& it = items[i];
        if (!it.Q || it.lQ < 1 || it.w < 0 || it.k < 1 || it.k > kstride) return EAPDTW_ERR_INVALID_ARG;
        if (it.ref_id < 0 || it.ref_id >= static_cast<int32_t>(c->refs.size()) || !c->refs[it.ref_id].live)
            return EAPDTW_ERR_INVALID_ARG;
        const RefEntry& r = c->refs[it.ref_id];
        const int64_t rn = ref_len ? std::min(ref_len[i], r.n) : r.n;
        if (it.lQ > rn) return EAPDTW_ERR_INVALID_ARG;
        if (it.lQ > EAPDTW_MAX_QUERY) return EAPDTW_ERR_UNSUPPORTED;
        nused[i] = rn;
        const int m = static_cast<int>(it.lQ);
        const int w = static_cast<int>(it.w < m ? it.w : m);
        const auto key = std::make_tuple(it.Q, m, w);
        auto f = slot_of.find(key);
        if (f == slot_of.end()) {
            QuerySlot q{};
            q.Q = it.Q;
            q.m = m;
            q.w = w;
            q.off = static_cast<int>(qf);
            qf += 5 * static_cast<int64_t>(query_pad(m));
            if (qf >= (int64_t(1) << 31)) return EAPDTW_ERR_UNSUPPORTED;
            slot_idx[i] = static_cast<int>(slots.size());
            slot_of.emplace(key, slot_idx[i]);
            slots.push_back(q);
        } else {
            slot_idx[i] = f->second;
        }
    }
    // running-extrema levels the items' LB_Keogh EC needs
    for (int i = 0; i < n; ++i) {
        if (items[i].no_lb) continue;
        const int m = static_cast<int>(items[i].lQ);
        const int w = static_cast<int>(items[i].w < m ? items[i].w : m);
        const int32_t e = ensure_env(c, c->refs[items[i].ref_id], env_level(std::min(w, m - 1)), st);
        if (e != EAPDTW_OK) return e;
    }
    for (int i = 0; i < n; ++i) {
        const eapdtw_item& it = items[i];
        const int m = static_cast<int>(it.lQ);
        const int w = static_cast<int>(it.w < m ? it.w : m);
        plan_item(c, c->refs[it.ref_id], nused[i], m, w, it.k, it.no_lb != 0, P[i]);
        P[i].b.state = i;
        samples += P[i].b.seed_ns;
        sum_nw += P[i].b.nw;
    }
    const int nslots = static_cast<int>(slots.size());
    int32_t rc = arena_reserve(c, c->batch, n, nslots, n, qf, samples, sum_nw + static_cast<int64_t>(kBatchSeedBest) * n);
    if (rc != EAPDTW_OK) return rc;
    Arena& a = c->batch;
    for (int i = 0; i < n; ++i) {
        const int mp = query_pad(P[i].b.m);
        const float* base = a.qarena + slots[slot_idx[i]].off;
        P[i].b.zq = base;
        P[i].b.uq = base + mp;
        P[i].b.lq = base + 2 * mp;
        P[i].b.zqo = base + 3 * mp;
        P[i].b.ord = reinterpret_cast<const int*>(base + 4 * mp);
    }
    rc = arena_run(a, P, slots, kstride, st, graph_ms != nullptr);
    if (rc != EAPDTW_OK) return rc;
    const size_t rows = static_cast<size_t>(n) * kstride;
    CKC(cudaMemcpyAsync(out_idx, a.res_idx, sizeof(int64_t) * rows, cudaMemcpyDeviceToDevice, st));
    CKC(cudaMemcpyAsync(out_dist, a.res_dist, sizeof(double) * rows, cudaMemcpyDeviceToDevice, st));
    CKC(cudaStreamSynchronize(st));
    ++c->batches;
    c->items_run += n;
    const int* hf = a.hflags();
    const int* hqb = a.hqbad();
    const unsigned long long* hc = a.hcounters();
    for (int q = 0; q < nslots; ++q)
        if (hqb[q]) return EAPDTW_ERR_NAN_INPUT;
    if (graph_ms) CKC(cudaEventElapsedTime(graph_ms, a.ev0, a.ev1));
    if (counters) {
        for (int j = 0; j < EAPDTW_NCOUNTERS; ++j) counters[j] = j < 10 ? static_cast<int64_t>(hc[j]) : 0;
    }
    for (int i = 0; i < n; ++i)
        if (hf[i] & kFlagTimeout) return EAPDTW_ERR_TIMEOUT;
    // items that lost a re-run entry (a list was full): run them alone
    for (int i = 0; i < n; ++i) {
        if (!(hf[i] & kFlagLost)) continue;
        const eapdtw_item& it = items[i];
        const RefEntry& r = c->refs[it.ref_id];
        eapdtw_search_opts o{};
        o.no_lb = it.no_lb;
        rc = subseq_search_ex(it.Q, it.lQ, r.R, nused[i], it.w, it.k, &o, out_idx + static_cast<int64_t>(i) * kstride,
                              out_dist + static_cast<int64_t>(i) * kstride, stream);
        if (rc != EAPDTW_OK) return rc;
        ++c->items_rerun;
    }
    return EAPDTW_OK;
}

}  // namespace

cudaError_t launch_batch_k4(int band, const BatchLaunch& args, int blocks, cudaStream_t s);
cudaError_t launch_batch_k8(int band, const BatchLaunch& args, int blocks, cudaStream_t s);
cudaError_t launch_batch_k16(int band, const BatchLaunch& args, int blocks, cudaStream_t s);
cudaError_t launch_batch_k32(int band, const BatchLaunch& args, int blocks, cudaStream_t s);
cudaError_t launch_batch_wide(int level, int band, const BatchLaunch& args, int blocks, cudaStream_t s);
int batch_blocks_k4(int band);
int batch_blocks_k8(int band);
int batch_blocks_k16(int band);
int batch_blocks_k32(int band);
int batch_blocks_wide(int level, int band);
cudaError_t batch_attributes_k4();
cudaError_t batch_attributes_k8();
cudaError_t batch_attributes_k16();
cudaError_t batch_attributes_k32();
cudaError_t batch_attributes_wide();
int batch_blocks_elastic(int e);
cudaError_t batch_attributes_elastic();

cudaError_t launch_batch(int level, int band, const BatchLaunch& args, int blocks, cudaStream_t s) {
    switch (level) {
        case 0: return launch_batch_k4(band, args, blocks, s);
        case 1: return launch_batch_k8(band, args, blocks, s);
        case 2: return launch_batch_k16(band, args, blocks, s);
        case 3: return launch_batch_k32(band, args, blocks, s);
        default: return launch_batch_wide(level, band, args, blocks, s);
    }
}

int batch_blocks(int level, int band) {
    // cached per (device, level, band): the occupancy query is not free
    static std::mutex mu;
    static int cache[64][kBatchLevels][3] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    int& v = cache[dev & 63][level][band];
    if (v == 0) {
        switch (level) {
            case 0: v = batch_blocks_k4(band); break;
            case 1: v = batch_blocks_k8(band); break;
            case 2: v = batch_blocks_k16(band); break;
            case 3: v = batch_blocks_k32(band); break;
            default: v = batch_blocks_wide(level, band); break;
        }
    }
    return v;
}

cudaError_t batch_attributes() {
    cudaError_t e = batch_attributes_k4();
    if (e == cudaSuccess) e = batch_attributes_k8();
    if (e == cudaSuccess) e = batch_attributes_k16();
    if (e == cudaSuccess) e = batch_attributes_k32();
    if (e == cudaSuccess) e = batch_attributes_wide();
    if (e == cudaSuccess) e = batch_attributes_elastic();
    return e;
}

int batch_blocks_el(int ec) {
    static std::mutex mu;
    static int cache[64][kElClasses] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    int& v = cache[dev & 63][ec];
    if (v == 0) v = batch_blocks_elastic(ec);
    return v;
}

}  // namespace eapdtw

using namespace eapdtw;

extern "C" {

int32_t eapdtw_ctx_create(int32_t device, int64_t mem_budget, eapdtw_ctx** out) {
    if (!out || mem_budget < 0) return EAPDTW_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return EAPDTW_ERR_CUDA; }
    if (device < 0 || device >= ndev) return EAPDTW_ERR_INVALID_ARG;
    eapdtw_ctx* c = new (std::nothrow) eapdtw_ctx;
    if (!c) return EAPDTW_ERR_OUT_OF_MEMORY;
    c->device = device;
    c->budget = mem_budget;
    if (const char* e = std::getenv("EAPDTW_RERUN_LIST_CAP")) {
        const long long v = std::atoll(e);
        if (v >= 1) c->batch.rr_cap_max = v;
    }
    *out = c;
    return EAPDTW_OK;
}

int32_t eapdtw_ctx_destroy(eapdtw_ctx* c) {
    if (!c) return EAPDTW_ERR_INVALID_ARG;
    server_shutdown(c);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        DeviceGuard g(c->device);
        cudaDeviceSynchronize();
        arena_free(c, c->batch);
        if (c->batch.ev0) cudaEventDestroy(c->batch.ev0);
        if (c->batch.ev1) cudaEventDestroy(c->batch.ev1);
        if (c->batch.cap_stream) cudaStreamDestroy(c->batch.cap_stream);
        for (RefEntry& r : c->refs) free_ref(r);
        c->refs.clear();
    }
    delete c;
    return EAPDTW_OK;
}

int32_t eapdtw_ref_register(eapdtw_ctx* c, const float* R, int64_t lR, int32_t* ref_id, void* stream) {
    if (!c || !R || !ref_id || lR < 1) return EAPDTW_ERR_INVALID_ARG;
    if (lR >= (int64_t(1) << 31)) return EAPDTW_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    if (!g.ok) return EAPDTW_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nch = (lR + kChunk - 1) / kChunk;
    RefEntry r;
    r.n = lR;
    int64_t bytes = 0;
    const bool ok = dalloc(r.R, lR, bytes) && dalloc(r.P1, lR, bytes) && dalloc(r.P2, lR, bytes) &&
                    dalloc(r.T1, nch, bytes) && dalloc(r.T2, nch, bytes) && dalloc(r.A, nch, bytes);
    int* bad = nullptr;
    int64_t bb = 0;
    auto undo = [&](int32_t rc) {
        free_ref(r);
        dfree(bad);
        return rc;
    };
    if (!ok || (c->budget > 0 && c->used + bytes > c->budget)) return undo(EAPDTW_ERR_OUT_OF_MEMORY);
    if (!dalloc(bad, 1, bb)) return undo(EAPDTW_ERR_OUT_OF_MEMORY);
    int hbad = 0;
    if (cudaMemcpyAsync(r.R, R, sizeof(float) * lR, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(bad, 0, sizeof(int), st) != cudaSuccess ||
        launch_ref_prefix(r.R, lR, r.P1, r.P2, r.T1, r.T2, r.A, bad, st) != cudaSuccess ||
        cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return undo(EAPDTW_ERR_CUDA);
    }
    dfree(bad);
    if (hbad) return undo(EAPDTW_ERR_NAN_INPUT);
    r.live = true;
    r.bytes = bytes;
    r.emax[0] = r.R;
    r.emin[0] = r.R;
    c->used += bytes;
    int id = -1;
    for (size_t i = 0; i < c->refs.size(); ++i)
        if (!c->refs[i].live) { id = static_cast<int>(i); break; }
    if (id < 0) {
        id = static_cast<int>(c->refs.size());
        c->refs.push_back(r);
    } else {
        c->refs[id] = r;
    }
    *ref_id = id;
    return EAPDTW_OK;
}

int32_t eapdtw_ref_unregister(eapdtw_ctx* c, int32_t ref_id) {
    if (!c) return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (ref_id < 0 || ref_id >= static_cast<int32_t>(c->refs.size()) || !c->refs[ref_id].live)
        return EAPDTW_ERR_INVALID_ARG;
    if (c->refs[ref_id].users > 0) return EAPDTW_ERR_BUSY;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();  // no batch may still read it
    RefEntry& r = c->refs[ref_id];
    c->used -= r.bytes;
    free_ref(r);
    return EAPDTW_OK;
}

int32_t eapdtw_ref_info(eapdtw_ctx* c, int32_t ref_id, const float** R, int64_t* lR) {
    if (!c) return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (ref_id < 0 || ref_id >= static_cast<int32_t>(c->refs.size()) || !c->refs[ref_id].live)
        return EAPDTW_ERR_INVALID_ARG;
    if (R) *R = c->refs[ref_id].R;
    if (lR) *lR = c->refs[ref_id].n;
    return EAPDTW_OK;
}

int32_t eapdtw_ctx_info(eapdtw_ctx* c, int64_t* out, int32_t nout) {
    if (!c || !out || nout < 1) return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    int64_t live = 0;
    for (const RefEntry& r : c->refs) live += r.live ? 1 : 0;
    const int64_t v[EAPDTW_CTX_NINFO] = {c->used, c->budget, live, c->batch.bytes, c->batches, c->items_run,
                                        c->items_rerun, c->batch.exec ? 1 : 0};
    for (int i = 0; i < nout && i < EAPDTW_CTX_NINFO; ++i) out[i] = v[i];
    return EAPDTW_OK;
}

int32_t eapdtw_set_first_tile(eapdtw_ctx* c, int32_t log2_m, int32_t ratio_tenths, int32_t band, int32_t tile) {
    if (!c || log2_m < 0 || log2_m > 12 || ratio_tenths < 0 || ratio_tenths > 10 || band < 0 || band > 1)
        return EAPDTW_ERR_INVALID_ARG;
    if (tile != 0 && tile != kTileElastic && tile != 4 && tile != 8 && tile != 16 && tile != 32)
        return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    const auto key = std::make_tuple(static_cast<int>(log2_m), static_cast<int>(ratio_tenths), static_cast<int>(band));
    auto f = c->tuned.find(key);
    const int chk = f == c->tuned.end() ? 0 : f->second.second;
    if (tile == 0 && chk == 0) c->tuned.erase(key);
    else c->tuned[key] = std::make_pair(static_cast<int>(tile), chk);
    return EAPDTW_OK;
}

int32_t eapdtw_get_first_tile(eapdtw_ctx* c, int32_t log2_m, int32_t ratio_tenths, int32_t band, int32_t* tile) {
    if (!c || !tile) return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    auto f = c->tuned.find(std::make_tuple(static_cast<int>(log2_m), static_cast<int>(ratio_tenths), static_cast<int>(band)));
    *tile = f == c->tuned.end() ? 0 : f->second.first;
    return EAPDTW_OK;
}

int32_t eapdtw_set_tuning(eapdtw_ctx* c, int32_t log2_m, int32_t ratio_tenths, int32_t band, int32_t tile,
                          int32_t check_double) {
    if (!c || log2_m < 0 || log2_m > 12 || ratio_tenths < 0 || ratio_tenths > 10 || band < 0 || band > 1)
        return EAPDTW_ERR_INVALID_ARG;
    if ((tile != 0 && tile != kTileElastic && tile != 4 && tile != 8 && tile != 16 && tile != 32) || check_double < 0 ||
        check_double > 1)
        return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    const auto key = std::make_tuple(static_cast<int>(log2_m), static_cast<int>(ratio_tenths), static_cast<int>(band));
    if (tile == 0 && check_double == 0) c->tuned.erase(key);
    else c->tuned[key] = std::make_pair(static_cast<int>(tile), static_cast<int>(check_double));
    return EAPDTW_OK;
}

int32_t eapdtw_get_tuning(eapdtw_ctx* c, int32_t log2_m, int32_t ratio_tenths, int32_t band, int32_t* tile,
                          int32_t* check_double) {
    if (!c || !tile || !check_double) return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    auto f = c->tuned.find(std::make_tuple(static_cast<int>(log2_m), static_cast<int>(ratio_tenths), static_cast<int>(band)));
    *tile = f == c->tuned.end() ? 0 : f->second.first;
    *check_double = f == c->tuned.end() ? 0 : f->second.second;
    return EAPDTW_OK;
}

int32_t eapdtw_search_batch(eapdtw_ctx* c, const eapdtw_item* items, int32_t n, int32_t kstride,
                            int64_t* out_idx, double* out_dist, int64_t* counters, void* stream) {
    if (!c || !items || n < 1 || !out_idx || !out_dist || kstride < 1) return EAPDTW_ERR_INVALID_ARG;
    if (kstride > EAPDTW_MAX_K) return EAPDTW_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    if (!g.ok) return EAPDTW_ERR_CUDA;
    if (!counters) return run_batch(c, items, n, kstride, out_idx, out_dist, nullptr, stream, nullptr, nullptr);
    // with counters, the launch sequence is timed with CUDA events on the call's stream
    float ms = 0.0f;
    const int32_t rc = run_batch(c, items, n, kstride, out_idx, out_dist, counters, stream, nullptr, &ms);
    if (rc == EAPDTW_OK) counters[EAPDTW_CNT_NS_TOTAL] = static_cast<int64_t>(static_cast<double>(ms) * 1.0e6);
    return rc;
}

constexpr float kTuneMargin = 0.05f;   // a tuned choice must beat the built-in one by 5% on the sample

int32_t eapdtw_autotune(eapdtw_ctx* c, const eapdtw_item* items, int32_t n, int64_t sample_windows, void* stream,
                        int32_t* n_tuned) {
    if (!c || !items || n < 1 || sample_windows < 1) return EAPDTW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    if (!g.ok) return EAPDTW_ERR_CUDA;
    // one representative per signature not tuned yet: the item with the longest reference
    std::map<std::tuple<int, int, int>, int> rep;
    for (int i = 0; i < n; ++i) {
        const eapdtw_item& it = items[i];
        if (!it.Q || it.lQ < 1 || it.lQ > EAPDTW_MAX_QUERY || it.w < 0 || it.k < 1 || it.k > EAPDTW_MAX_K)
            return EAPDTW_ERR_INVALID_ARG;
        if (it.ref_id < 0 || it.ref_id >= static_cast<int32_t>(c->refs.size()) || !c->refs[it.ref_id].live)
            return EAPDTW_ERR_INVALID_ARG;
        const int m = static_cast<int>(it.lQ);
        const int w = static_cast<int>(it.w < m ? it.w : m);
        const auto key = signature(m, w);
        if (c->tuned.count(key)) continue;
        auto f = rep.find(key);
        if (f == rep.end() || c->refs[items[f->second].ref_id].n < c->refs[it.ref_id].n) rep[key] = i;
    }
    int64_t* d_idx = nullptr;
    double* d_dist = nullptr;
    int64_t bytes = 0;
    if (!dalloc(d_idx, EAPDTW_MAX_K, bytes) || !dalloc(d_dist, EAPDTW_MAX_K, bytes)) {
        dfree(d_idx);
        return EAPDTW_ERR_OUT_OF_MEMORY;
    }
    int32_t rc = EAPDTW_OK;
    int tuned = 0;
    for (const auto& kv : rep) {
        eapdtw_item it = items[kv.second];
        const RefEntry& r = c->refs[it.ref_id];
        // a prefix of whole statistics chunks holding about sample_windows windows
        int64_t len = (sample_windows + it.lQ - 1 + kChunk - 1) / kChunk * kChunk;
        if (len >= r.n) len = r.n;
        const int m = static_cast<int>(it.lQ);
        const int w = static_cast<int>(it.w < m ? it.w : m);
        c->tuned.erase(kv.first);
        // candidates: the built-in first level and its neighbours (the
        // elastic level, where it can run, against the band's one-warp K and
        // twice that)
        const int lv0 = first_level(c, m, w);
        int cand[3];
        if (lv0 == kElLevel) {
            const int kr = 4 << rule_level(m, w);
            cand[0] = kTileElastic;
            cand[1] = kr;
            cand[2] = kr * 2;
        } else {
            const int base = 4 << lv0;
            cand[0] = base;
            cand[1] = base * 2;
            cand[2] = base / 2;
        }
        // the built-in choice (the first candidate at the built-in interval)
        // stays unless another one is faster by kTuneMargin on the sample: a
        // sample's small differences did not carry over to whole references
        float best_ms = INFINITY, builtin_ms = INFINITY;
        std::pair<int, int> best(cand[0], 0);
        for (int chk = 0; chk < 2 && rc == EAPDTW_OK; ++chk) {
            for (int K : cand) {
                if (K != kTileElastic && (K < 4 || K > 32)) continue;
                c->tuned[kv.first] = std::make_pair(K, chk);
                float ms = 0.0f, ms2 = 0.0f;
                rc = run_batch(c, &it, 1, it.k, d_idx, d_dist, nullptr, stream, &len, &ms);   // warm-up
                if (rc == EAPDTW_OK) rc = run_batch(c, &it, 1, it.k, d_idx, d_dist, nullptr, stream, &len, &ms2);
                if (rc != EAPDTW_OK) break;
                ms = std::min(ms, ms2);
                if (K == cand[0] && chk == 0) builtin_ms = ms;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = std::make_pair(K, chk);
                }
            }
        }
        if (!(best_ms < builtin_ms * (1.0f - kTuneMargin))) best = std::make_pair(cand[0], 0);
        if (rc != EAPDTW_OK) {
            c->tuned.erase(kv.first);
            break;
        }
        c->tuned[kv.first] = best;
        ++tuned;
    }
    dfree(d_idx);
    dfree(d_dist);
    if (n_tuned) *n_tuned = tuned;
    return rc;
}

}  // extern "C"
