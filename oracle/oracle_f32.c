/*
 * FP32-emulating oracle mode of the subsequence search (test infrastructure
 * only: loaded by the tests, the smoke check and the benchmark's CPU leg,
 * never by the product path; it shares no code with the CUDA sources).
 *
 * The FP64 oracle (oracle.c) fixes WHAT the search computes.  This file fixes
 * HOW the GPU search rounds it: it repeats, operation by operation and in the
 * same order, the FP64 and FP32 arithmetic of the GPU search, so that the
 * search's integer outcomes -- which windows LB_Kim, LB_Keogh EQ and LB_Keogh
 * EC prune under a fixed upper bound, which EAPrunedDTW runs complete and
 * which are abandoned (Section 2.2, Algorithm 3), the nearest-neighbour
 * indices -- and its FP32 distances can be compared bit for bit.  The
 * arithmetic it reproduces:
 *
 *  - Window statistics: the reference is cut into chunks of 4096 points; in
 *    each chunk the FP64 sums of (x - a) and (x - a)^2, a = the chunk's first
 *    value, are prefix-summed in the order of a 256-thread block scan: each
 *    thread sums 16 consecutive points, the 32 threads of a warp combine by an
 *    inclusive Hillis-Steele scan, the warps' totals are added in order.
 *    Squares are accumulated with fused multiply-adds.  A window's moments
 *    combine the sums of at most two chunks re-anchored to its first chunk.
 *  - z-normalisation z(x) = ((x - a) - cw) * isd in FP32, a = the window's
 *    first value, cw = fl32(mean - a), isd = the correctly rounded FP32
 *    reciprocal square root of fl32(var); a two-pass FP64 fallback when the
 *    variance is below 1e-6 of the anchored second moment.
 *  - The query: FP64 mean and variance summed by 1024 threads (strided terms,
 *    a butterfly inside each warp, the 32 warp sums in order), two-pass.
 *  - Lower bounds in FP32 with fused multiply-adds, terms in decreasing |zq|
 *    order; a window is pruned when a bound exceeds fl32(ub * 1.0001).
 *  - The DTW recurrence of Eq. 1-5 in FP32: cell = fma(d, d, min(top, diag,
 *    left)), d = z - q.
 *
 * Compiled with -ffp-contract=off: every FP operation below is exactly the one
 * written (fma() and fmaf() where a fused operation is meant).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O7_CHUNK_LOG 12
#define O7_CHUNK (1 << O7_CHUNK_LOG)
#define O7_THREADS 256
#define O7_PER (O7_CHUNK / O7_THREADS)
#define O7_QTHREADS 1024

/* ------------------------------------------------------------------------
 * Correctly rounded reciprocal square root of a positive finite float.
 * The candidate comes from FP64; its two neighbours are tested against the
 * exact midpoints: r = v^(-1/2) lies below mid iff mid^2 * v > 1, decided on
 * integers (mid has at most 26 significant bits, v 24).
 * ------------------------------------------------------------------------ */
static void split(double x, uint64_t* mant, int* ex) {
    /* x = mant * 2^ex with mant odd (x > 0) */
    int e;
    double f = frexp(x, &e);
    uint64_t M = (uint64_t)ldexp(f, 53);
    e -= 53;
    while ((M & 1) == 0) {
        M >>= 1;
        ++e;
    }
    *mant = M;
    *ex = e;
}

/* 1 if mid^2 * v > 1, exactly */
static int mid_sq_v_above_one(double mid, float v) {
    uint64_t Mm, Mv;
    int em, ev;
    split(mid, &Mm, &em);
    split((double)v, &Mv, &ev);
    unsigned __int128 P = (unsigned __int128)Mm * Mm * Mv;  /* < 2^(26+26+24) */
    int E = 2 * em + ev;                                    /* mid^2 v = P * 2^E */
    if (E >= 0) return P >= 1;
    if (-E >= 127) return 0;
    unsigned __int128 one = (unsigned __int128)1 << (-E);
    return P > one;
}

float o7_rsqrt_rn(float v) {
    float y = (float)(1.0 / sqrt((double)v));
    /* y is within one ulp of the correctly rounded result: move while the
       neighbour is closer to r = v^(-1/2) */
    for (int it = 0; it < 4; ++it) {
        float up = nextafterf(y, INFINITY), dn = nextafterf(y, 0.0f);
        double mid_up = ((double)y + (double)up) * 0.5;
        double mid_dn = ((double)y + (double)dn) * 0.5;
        if (!mid_sq_v_above_one(mid_up, v)) {
            /* r >= mid_up: up is at least as close */
            y = up;
        } else if (mid_sq_v_above_one(mid_dn, v)) {
            /* r < mid_dn: dn is closer */
            y = dn;
        } else {
            break;
        }
    }
    return y;
}

/* ------------------------------------------------------------------------
 * Chunk-anchored prefix sums (see the header for the order).  P1[j], P2[j]:
 * sums over the points of j's chunk before j; T1[c], T2[c]: chunk totals;
 * A[c]: the anchor.
 * ------------------------------------------------------------------------ */
void o7_ref_prefix(const float* R, int64_t n, double* P1, double* P2, double* T1, double* T2, float* A) {
    const int64_t nch = (n + O7_CHUNK - 1) / O7_CHUNK;
    double d[O7_CHUNK];
    double s1[O7_THREADS], s2[O7_THREADS], i1[O7_THREADS], i2[O7_THREADS], p1[O7_THREADS], p2[O7_THREADS];
    double w1[O7_THREADS / 32], w2[O7_THREADS / 32];
    for (int64_t c = 0; c < nch; ++c) {
        const int64_t base = c << O7_CHUNK_LOG;
        const int64_t len = n - base < O7_CHUNK ? n - base : O7_CHUNK;
        const float anchor = R[base];
        const double a = (double)anchor;
        for (int j = 0; j < O7_CHUNK; ++j) d[j] = (double)(j < len ? R[base + j] : anchor) - a;
        for (int t = 0; t < O7_THREADS; ++t) {
            double u = 0.0, q = 0.0;
            for (int e = 0; e < O7_PER; ++e) {
                u = u + d[t * O7_PER + e];
                q = fma(d[t * O7_PER + e], d[t * O7_PER + e], q);
            }
            s1[t] = u;
            s2[t] = q;
            i1[t] = u;
            i2[t] = q;
        }
        /* inclusive scan inside each warp: at stride o lane l adds lane l-o's previous value */
        for (int o = 1; o < 32; o <<= 1) {
            memcpy(p1, i1, sizeof(i1));
            memcpy(p2, i2, sizeof(i2));
            for (int t = 0; t < O7_THREADS; ++t) {
                if ((t & 31) >= o) {
                    i1[t] = p1[t] + p1[t - o];
                    i2[t] = p2[t] + p2[t - o];
                }
            }
        }
        for (int wp = 0; wp < O7_THREADS / 32; ++wp) {
            w1[wp] = i1[wp * 32 + 31];
            w2[wp] = i2[wp * 32 + 31];
        }
        for (int t = 0; t < O7_THREADS; ++t) {
            double b1 = 0.0, b2 = 0.0;
            for (int q = 0; q < t / 32; ++q) {
                b1 = b1 + w1[q];
                b2 = b2 + w2[q];
            }
            double r1 = (b1 + i1[t]) - s1[t], r2 = (b2 + i2[t]) - s2[t];
            for (int e = 0; e < O7_PER; ++e) {
                const int64_t j = (int64_t)t * O7_PER + e;
                if (j < len) {
                    P1[base + j] = r1;
                    P2[base + j] = r2;
                }
                r1 = r1 + d[j];
                r2 = fma(d[j], d[j], r2);
            }
            if (t == O7_THREADS - 1) {
                T1[c] = r1;
                T2[c] = r2;
                A[c] = anchor;
            }
        }
    }
}

/* z coefficients of window [i, i + m) (see the header). */
void o7_window_coeffs(const float* R, int64_t n, const double* P1, const double* P2, const double* T1,
                      const double* T2, const float* A, int64_t i, int64_t m, float* a_out, float* cw_out,
                      float* isd_out) {
    const int64_t end = i + m;
    const int64_t c0 = i >> O7_CHUNK_LOG;
    const double a0 = (double)A[c0];
    double s1 = 0.0, s2 = 0.0;
    int64_t lo = i;
    for (int64_t c = c0; lo < end; ++c) {
        const int64_t cend = ((c + 1) << O7_CHUNK_LOG) < n ? ((c + 1) << O7_CHUNK_LOG) : n;
        const int64_t hi = end < cend ? end : cend;
        const double e1 = (hi == cend) ? T1[c] : P1[hi];
        const double e2 = (hi == cend) ? T2[c] : P2[hi];
        const double p1 = e1 - P1[lo];
        const double p2 = e2 - P2[lo];
        const double cnt = (double)(hi - lo);
        const double dl = (double)A[c] - a0;
        s1 = s1 + fma(cnt, dl, p1);
        s2 = s2 + fma(dl, fma(cnt, dl, 2.0 * p1), p2);
        lo = hi;
    }
    const double mu1 = s1 / (double)m;
    double mean = a0 + mu1;
    const double m2a = s2 / (double)m;
    double var = m2a - mu1 * mu1;
    const float a = R[i];
    if (!(var > 1e-6 * m2a)) {
        double s = 0.0;
        for (int64_t p = 0; p < m; ++p) s = s + (double)R[i + p];
        mean = s / (double)m;
        double v = 0.0;
        for (int64_t p = 0; p < m; ++p) {
            const double dd = (double)R[i + p] - mean;
            v = fma(dd, dd, v);
        }
        var = v / (double)m;
    }
    const float var32 = (float)var;
    *a_out = a;
    if (var32 > 0.0f) {
        *isd_out = o7_rsqrt_rn(var32);
        *cw_out = (float)(mean - (double)a);
    } else {
        *isd_out = 0.0f;
        *cw_out = 0.0f;
    }
}

static inline float znorm1(float x, float a, float cw, float isd) { return ((x - a) - cw) * isd; }

/* ------------------------------------------------------------------------
 * Query preparation: zq[m], the envelope of zq over +-min(w, m-1) clipped to
 * the query, and the order of positions by decreasing |zq| (ties: position)
 * with the envelope and zq in that order.
 * ------------------------------------------------------------------------ */
static double block_sum(const double* part /* [O7_QTHREADS] */) {
    double red[O7_QTHREADS / 32];
    double v[32], nv[32];
    for (int wp = 0; wp < O7_QTHREADS / 32; ++wp) {
        for (int l = 0; l < 32; ++l) v[l] = part[wp * 32 + l];
        for (int o = 16; o > 0; o >>= 1) {
            for (int l = 0; l < 32; ++l) nv[l] = v[l] + v[l ^ o];
            memcpy(v, nv, sizeof(v));
        }
        red[wp] = v[0];
    }
    double t = 0.0;
    for (int q = 0; q < O7_QTHREADS / 32; ++q) t = t + red[q];
    return t;
}

typedef struct {
    uint32_t mag;
    int32_t j;
} o7_key;

static int key_cmp(const void* x, const void* y) {
    const o7_key* p = (const o7_key*)x;
    const o7_key* q = (const o7_key*)y;
    if (p->mag != q->mag) return p->mag > q->mag ? -1 : 1;  /* decreasing |zq| */
    return p->j < q->j ? -1 : (p->j > q->j);
}

void o7_query_prep(const float* Q, int64_t m, int64_t w, float* zq, float* uq_o, float* lq_o, float* zq_o,
                   int32_t* ord) {
    double* part = (double*)calloc(O7_QTHREADS, sizeof(double));
    float* U = (float*)malloc(sizeof(float) * m);
    float* L = (float*)malloc(sizeof(float) * m);
    o7_key* keys = (o7_key*)malloc(sizeof(o7_key) * m);
    for (int t = 0; t < O7_QTHREADS; ++t) {
        double s = 0.0;
        for (int64_t j = t; j < m; j += O7_QTHREADS) s = s + (double)Q[j];
        part[t] = s;
    }
    const double mean = block_sum(part) / (double)m;
    for (int t = 0; t < O7_QTHREADS; ++t) {
        double v = 0.0;
        for (int64_t j = t; j < m; j += O7_QTHREADS) {
            const double dx = (double)Q[j] - mean;
            v = fma(dx, dx, v);
        }
        part[t] = v;
    }
    const double var = block_sum(part) / (double)m;
    const double sd = var > 0.0 ? sqrt(var) : 0.0;
    for (int64_t j = 0; j < m; ++j) zq[j] = sd > 0.0 ? (float)(((double)Q[j] - mean) / sd) : 0.0f;
    const int64_t wc = w < m - 1 ? w : m - 1;
    for (int64_t j = 0; j < m; ++j) {
        const int64_t lo = j - wc > 0 ? j - wc : 0;
        const int64_t hi = j + wc < m - 1 ? j + wc : m - 1;
        float u = zq[lo], l = zq[lo];
        for (int64_t k = lo + 1; k <= hi; ++k) {
            u = fmaxf(u, zq[k]);
            l = fminf(l, zq[k]);
        }
        U[j] = u;
        L[j] = l;
    }
    for (int64_t j = 0; j < m; ++j) {
        const float az = fabsf(zq[j]);
        uint32_t bits;
        memcpy(&bits, &az, sizeof(bits));
        keys[j].mag = bits;
        keys[j].j = (int32_t)j;
    }
    qsort(keys, (size_t)m, sizeof(o7_key), key_cmp);
    for (int64_t p = 0; p < m; ++p) {
        const int32_t j = keys[p].j;
        ord[p] = j;
        uq_o[p] = U[j];
        lq_o[p] = L[j];
        zq_o[p] = zq[j];
    }
    free(part);
    free(U);
    free(L);
    free(keys);
}

/* DTW of Eq. 1-5 in FP32 with the band |r - c| <= w: rows z_r, columns q_c. */
float o7_dtw_f32(const float* z, const float* q, int64_t m, int64_t w) {
    float* prev = (float*)malloc(sizeof(float) * (m + 1));
    float* curr = (float*)malloc(sizeof(float) * (m + 1));
    for (int64_t c = 0; c <= m; ++c) prev[c] = INFINITY;
    prev[0] = 0.0f;
    for (int64_t r = 1; r <= m; ++r) {
        curr[0] = INFINITY;
        for (int64_t c = 1; c <= m; ++c) {
            const int64_t dd = r - c;
            if (dd > w || -dd > w) {
                curr[c] = INFINITY;
                continue;
            }
            const float d = z[r - 1] - q[c - 1];
            curr[c] = fmaf(d, d, fminf(fminf(prev[c], prev[c - 1]), curr[c - 1]));
        }
        float* t = prev;
        prev = curr;
        curr = t;
    }
    const float out = prev[m];
    free(prev);
    free(curr);
    return out;
}

typedef struct {
    int k, n;
    float d[64];
    int64_t i[64];
} o7_topk;

static void topk_put(o7_topk* t, float d, int64_t i) {
    /* keep the k smallest (d, i) */
    int pos = t->n;
    while (pos > 0 && (t->d[pos - 1] > d || (t->d[pos - 1] == d && t->i[pos - 1] > i))) --pos;
    if (pos >= t->k) return;
    const int last = t->n < t->k ? t->n : t->k - 1;
    for (int s = last; s > pos; --s) {
        t->d[s] = t->d[s - 1];
        t->i[s] = t->i[s - 1];
    }
    t->d[pos] = d;
    t->i[pos] = i;
    if (t->n < t->k) ++t->n;
}

/* ------------------------------------------------------------------------
 * The search in FP32 emulation.  Q[m], R[n] are the FP32 inputs; w the
 * window; k <= 64.
 *   exact (audit = 0): the k smallest (dist, index) over every window's FP32
 *     DTW (no bound, no pruning): the result the GPU must return.
 *   audit (audit = 1): the cascade under the fixed bound ub: a window is
 *     pruned by the first lower bound above fl32(ub * 1.0001) (use_lb = 0:
 *     none), else its DTW completes if <= ub and is abandoned otherwise.
 *     counters: windows, LB_Kim, LB_Keogh EQ, LB_Keogh EC prunes, abandoned,
 *     completed; the k-best list is over the completed windows.
 *   why (optional, nw entries): each window's outcome, 1 LB_Kim, 2 LB_Keogh
 *     EQ, 3 LB_Keogh EC (pruned), 4 abandoned, 5 completed (audit), or 5
 *     (exact mode: every window's DTW is computed).
 * Returns 0, or -1 on invalid arguments.
 * ------------------------------------------------------------------------ */
int o7_search(const float* Q, int64_t m, const float* R, int64_t n, int64_t w, int k, int audit, float ub,
              int use_lb, int64_t* counters, int64_t* idx, double* dist, int8_t* why) {
    if (!Q || !R || m < 1 || n < m || w < 0 || k < 1 || k > 64) return -1;
    const int64_t nch = (n + O7_CHUNK - 1) / O7_CHUNK;
    const int64_t nw = n - m + 1;
    double* P1 = (double*)malloc(sizeof(double) * n);
    double* P2 = (double*)malloc(sizeof(double) * n);
    double* T1 = (double*)malloc(sizeof(double) * nch);
    double* T2 = (double*)malloc(sizeof(double) * nch);
    float* A = (float*)malloc(sizeof(float) * nch);
    float* zq = (float*)malloc(sizeof(float) * m);
    float* uq = (float*)malloc(sizeof(float) * m);
    float* lq = (float*)malloc(sizeof(float) * m);
    float* zqo = (float*)malloc(sizeof(float) * m);
    int32_t* ord = (int32_t*)malloc(sizeof(int32_t) * m);
    float* z = (float*)malloc(sizeof(float) * m);
    float* U = (float*)malloc(sizeof(float) * n);
    float* L = (float*)malloc(sizeof(float) * n);
    const int64_t wi = w < m ? w : m;
    o7_ref_prefix(R, n, P1, P2, T1, T2, A);
    o7_query_prep(Q, m, wi, zq, uq, lq, zqo, ord);
    /* raw envelope of R over +-min(w, m-1), clipped to the series */
    const int64_t re = wi < m - 1 ? wi : m - 1;
    for (int64_t t = 0; t < n; ++t) {
        const int64_t lo = t - re > 0 ? t - re : 0;
        const int64_t hi = t + re < n - 1 ? t + re : n - 1;
        float u = R[lo], l = R[lo];
        for (int64_t s = lo + 1; s <= hi; ++s) {
            u = fmaxf(u, R[s]);
            l = fminf(l, R[s]);
        }
        U[t] = u;
        L[t] = l;
    }
    const float ub_lb = ub * 1.0001f;
    int64_t cnt[6] = {0, 0, 0, 0, 0, 0};
    o7_topk top;
    memset(&top, 0, sizeof(top));
    top.k = k;
    for (int64_t i = 0; i < nw; ++i) {
        float a, cw, isd;
        o7_window_coeffs(R, n, P1, P2, T1, T2, A, i, m, &a, &cw, &isd);
        ++cnt[0];
        if (audit && use_lb) {
            const float d0 = znorm1(R[i], a, cw, isd) - zq[0];
            float kim = d0 * d0;
            if (m > 1) {
                const float dl = znorm1(R[i + m - 1], a, cw, isd) - zq[m - 1];
                kim = fmaf(dl, dl, kim);
            }
            if (kim > ub_lb) {
                ++cnt[1];
                if (why) why[i] = 1;
                continue;
            }
            float s = 0.0f;
            for (int64_t p = 0; p < m; ++p) {
                const float zz = znorm1(R[i + ord[p]], a, cw, isd);
                const float e = fmaxf(fmaxf(zz - uq[p], lq[p] - zz), 0.0f);
                s = fmaf(e, e, s);
            }
            if (s > ub_lb) {
                ++cnt[2];
                if (why) why[i] = 2;
                continue;
            }
            float s2 = 0.0f;
            for (int64_t p = 0; p < m; ++p) {
                const float uu = znorm1(U[i + ord[p]], a, cw, isd);
                const float ll = znorm1(L[i + ord[p]], a, cw, isd);
                const float e = fmaxf(fmaxf(zqo[p] - uu, ll - zqo[p]), 0.0f);
                s2 = fmaf(e, e, s2);
            }
            if (s2 > ub_lb) {
                ++cnt[3];
                if (why) why[i] = 3;
                continue;
            }
        }
        for (int64_t r = 0; r < m; ++r) z[r] = znorm1(R[i + r], a, cw, isd);
        const float d = o7_dtw_f32(z, zq, m, wi);
        if (why) why[i] = (audit && !(d <= ub)) ? 4 : 5;
        if (audit) {
            if (d <= ub) {
                ++cnt[5];
                topk_put(&top, d, i);
            } else {
                ++cnt[4];
            }
        } else {
            topk_put(&top, d, i);
        }
    }
    for (int s = 0; s < k; ++s) {
        if (s < top.n) {
            idx[s] = top.i[s];
            dist[s] = (double)top.d[s];
        } else {
            idx[s] = -1;
            dist[s] = INFINITY;
        }
    }
    if (counters)
        for (int c = 0; c < 6; ++c) counters[c] = cnt[c];
    free(P1); free(P2); free(T1); free(T2); free(A);
    free(zq); free(uq); free(lq); free(zqo); free(ord); free(z); free(U); free(L);
    return 0;
}
