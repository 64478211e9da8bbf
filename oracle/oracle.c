/*
 * Oracle for subsequence nearest-neighbour search under DTW with EAPrunedDTW
 * (Herrmann & Webb, "Early Abandoning PrunedDTW and its application to
 * similarity search", arXiv 2010.05371).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, sequential CPU
 * restatement of what the method computes, in FP64.  It exists to check the
 * CUDA library against the paper.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never
 * does, and it shares no code, header or table with the CUDA sources.
 *
 * Conventions (1-based indices follow the paper's notation):
 *   - cost(a, b) = (a - b)^2, the squared Euclidean cost (Section 2).
 *   - The warping window w is a Sakoe-Chiba band: cell (i, j) exists iff
 *     |i - j| <= w (Section 2.1).  Cells outside the band are +inf.
 *     w >= max(lS, lT) - 1 is unconstrained DTW; w < |lS - lT| admits no
 *     warping path and every DTW routine returns +inf.
 *   - "li" (rows) is the longer series, "co" (columns) the shorter one; on a
 *     tie li = S, the first argument (Algorithms 1-3 leave ties open).
 *   - Every routine returns NaN for invalid arguments (NULL, length <= 0,
 *     w < 0).
 *
 * Readings where the paper is silent or wrong are marked READING below.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF HUGE_VAL

static inline double cost(double a, double b) {
    double d = a - b;
    return d * d;
}

static inline double min2(double a, double b) { return a < b ? a : b; }
static inline double min3(double a, double b, double c) { return min2(min2(a, b), c); }

static int bad_args(const double* S, int64_t lS, const double* T, int64_t lT, int64_t w) {
    return S == NULL || T == NULL || lS <= 0 || lT <= 0 || w < 0;
}

static int64_t abs64(int64_t x) { return x < 0 ? -x : x; }

/* ------------------------------------------------------------------------ */
/* O1: the DTW recurrence of Eq. 1-5 over the full (lS+1) x (lT+1) matrix.   */
/* Rows are S, columns are T, exactly as Eq. 5 indexes them.  If M is not    */
/* NULL it receives the whole matrix, row-major, border row/column included. */
/* ------------------------------------------------------------------------ */
double orc_dtw_matrix(const double* S, int64_t lS, const double* T, int64_t lT,
                      int64_t w, double* M) {
    if (bad_args(S, lS, T, lT, w)) return NAN;
    int64_t cols = lT + 1;
    double* D = M ? M : (double*)malloc(sizeof(double) * (size_t)((lS + 1) * cols));
    if (!D) return NAN;
    /* Eq. 2-4: (0,0) = 0, (i,0) = (0,j) = +inf. */
    for (int64_t j = 0; j <= lT; ++j) D[j] = ORC_INF;
    for (int64_t i = 1; i <= lS; ++i) D[i * cols] = ORC_INF;
    D[0] = 0.0;
    /* Eq. 5, restricted to the band |i - j| <= w (Section 2.1). */
    for (int64_t i = 1; i <= lS; ++i) {
        for (int64_t j = 1; j <= lT; ++j) {
            if (abs64(i - j) > w) {
                D[i * cols + j] = ORC_INF;
                continue;
            }
            double top = D[(i - 1) * cols + j];
            double left = D[i * cols + j - 1];
            double diag = D[(i - 1) * cols + j - 1];
            D[i * cols + j] = cost(S[i - 1], T[j - 1]) + min3(top, left, diag);
        }
    }
    double r = D[lS * cols + lT];
    if (!M) free(D);
    return r;
}

/* Pick rows (li = longer) and columns (co = shorter); ties go to li = S. */
static void orient(const double* S, int64_t lS, const double* T, int64_t lT,
                   const double** li, int64_t* l_li, const double** co, int64_t* l_co) {
    if (lT > lS) {
        *li = T; *l_li = lT; *co = S; *l_co = lS;
    } else {
        *li = S; *l_li = lS; *co = T; *l_co = lT;
    }
}

/* ------------------------------------------------------------------------ */
/* O2: Algorithm 1, the O(n)-space DTW with two rows of length l_co + 1.     */
/* The window is applied by giving out-of-band cells the value +inf.         */
/* ------------------------------------------------------------------------ */
double orc_dtw_tworow(const double* S, int64_t lS, const double* T, int64_t lT, int64_t w) {
    if (bad_args(S, lS, T, lT, w)) return NAN;
    if (w < abs64(lS - lT)) return ORC_INF;
    const double *li, *co;
    int64_t l_li, l_co;
    orient(S, lS, T, lT, &li, &l_li, &co, &l_co);
    double* prev = (double*)malloc(sizeof(double) * (size_t)(l_co + 1));
    double* curr = (double*)malloc(sizeof(double) * (size_t)(l_co + 1));
    for (int64_t j = 0; j <= l_co; ++j) prev[j] = curr[j] = ORC_INF;
    curr[0] = 0.0;
    for (int64_t i = 1; i <= l_li; ++i) {
        double* t = prev; prev = curr; curr = t;
        curr[0] = ORC_INF;
        for (int64_t j = 1; j <= l_co; ++j) {
            if (abs64(i - j) > w) {
                curr[j] = ORC_INF;
                continue;
            }
            double c = cost(li[i - 1], co[j - 1]);
            curr[j] = c + min3(curr[j - 1], prev[j], prev[j - 1]);
        }
    }
    double r = curr[l_co];
    free(prev);
    free(curr);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, pruning from the left, as in Section 3 (no window).  Used    */
/* only to pin the worked example of Section 3.  *abandon_row receives the   */
/* 1-based row whose discard points covered the whole line, or 0.            */
/* ------------------------------------------------------------------------ */
double orc_dtw_prune_left(const double* S, int64_t lS, const double* T, int64_t lT,
                          double ub, int64_t* abandon_row) {
    if (bad_args(S, lS, T, lT, 0) || isnan(ub)) return NAN;
    const double *li, *co;
    int64_t l_li, l_co;
    orient(S, lS, T, lT, &li, &l_li, &co, &l_co);
    double* prev = (double*)malloc(sizeof(double) * (size_t)(l_co + 1));
    double* curr = (double*)malloc(sizeof(double) * (size_t)(l_co + 1));
    for (int64_t j = 0; j <= l_co; ++j) prev[j] = curr[j] = ORC_INF;
    curr[0] = 0.0;
    int64_t next_start = 1;
    double result = ORC_INF;
    if (abandon_row) *abandon_row = 0;
    for (int64_t i = 1; i <= l_li; ++i) {
        double* t = prev; prev = curr; curr = t;
        int64_t j = next_start;
        curr[j - 1] = ORC_INF;
        /* Stage 1: successive discard points; the left neighbour is > ub. */
        while (j == next_start && j <= l_co) {
            double c = cost(li[i - 1], co[j - 1]);
            curr[j] = c + min2(prev[j], prev[j - 1]);
            if (curr[j] > ub) next_start = next_start + 1;
            j = j + 1;
        }
        if (j > l_co) {
            if (next_start > l_co) {  /* the whole line is discard points */
                if (abandon_row) *abandon_row = i;
                goto done;
            }
        }
        /* Stage 2: plain DTW to the end of the line. */
        while (j <= l_co) {
            double c = cost(li[i - 1], co[j - 1]);
            curr[j] = c + min3(curr[j - 1], prev[j], prev[j - 1]);
            j = j + 1;
        }
    }
    result = curr[l_co];
done:
    free(prev);
    free(curr);
    return result;
}

/* ------------------------------------------------------------------------ */
/* O3: Algorithm 3, EAPrunedDTW, with two adaptations.                       */
/*                                                                          */
/* READING (stage 4): the printed stage-4 loop adds the cost c left over     */
/* from stage 3 to every cell; the cell (i, j) needs cost(li(i), co(j)), so  */
/* c is recomputed for each j.  With the printed form the result differs     */
/* from Eq. 1-5 on random inputs; with the recomputation it never does.      */
/*                                                                          */
/* READING (window): Section 2.1 leaves the window out of the algorithms.    */
/* For row i the band is [lo_i, hi_i] = [max(1, i - w), min(l_co, i + w)].   */
/* Before the left border of row i is set, next_start is raised to lo_i      */
/* (cells left of the band are +inf, i.e. discard points); the stage-3 test  */
/* and the stage-4 bound use hi_i in place of l_co.  The final test keeps    */
/* l_co.  The right side needs no change: prev_pruning_point <= i + w.       */
/*                                                                          */
/* Returns DTW if DTW <= ub, else +inf.  trace (optional) receives the cell  */
/* count, the row of early abandoning, and per-row next_start/pruning_point. */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t cells;          /* cells whose value was computed */
    int64_t rows;           /* rows entered */
    int64_t abandon_row;    /* 1-based row where +inf was returned, 0 if none */
    int64_t* next_start;    /* optional [l_li]: next_start at the end of row i */
    int64_t* pruning_point; /* optional [l_li]: pruning_point at the end of row i */
} orc_eap_trace;

double orc_eapruned_dtw(const double* S, int64_t lS, const double* T, int64_t lT,
                        int64_t w, double ub, orc_eap_trace* tr) {
    if (bad_args(S, lS, T, lT, w) || isnan(ub)) return NAN;
    if (tr) { tr->cells = 0; tr->rows = 0; tr->abandon_row = 0; }
    if (w < abs64(lS - lT)) return ORC_INF;
    const double *li, *co;
    int64_t l_li, l_co;
    orient(S, lS, T, lT, &li, &l_li, &co, &l_co);
    double* prev = (double*)malloc(sizeof(double) * (size_t)(l_co + 1));
    double* curr = (double*)malloc(sizeof(double) * (size_t)(l_co + 1));
    for (int64_t j = 0; j <= l_co; ++j) prev[j] = curr[j] = ORC_INF;
    curr[0] = 0.0;
    int64_t next_start = 1;
    int64_t prev_pruning_point = 1;
    int64_t pruning_point = 0;
    int64_t cells = 0;
    double result = ORC_INF;
    int64_t i;
    for (i = 1; i <= l_li; ++i) {
        double* t = prev; prev = curr; curr = t;
        int64_t lo = i - w > 1 ? i - w : 1;
        int64_t hi = i + w < l_co ? i + w : l_co;
        if (next_start < lo) next_start = lo;
        int64_t j = next_start;
        curr[j - 1] = ORC_INF;
        if (tr) tr->rows = i;
        /* Stage 1: discard points; the left neighbour is > ub. */
        while (j == next_start && j < prev_pruning_point) {
            double c = cost(li[i - 1], co[j - 1]);
            curr[j] = c + min2(prev[j], prev[j - 1]);
            ++cells;
            if (curr[j] <= ub) pruning_point = j + 1;
            else next_start = next_start + 1;
            j = j + 1;
        }
        /* Stage 2: full three-neighbour cells up to the previous pruning point. */
        while (j < prev_pruning_point) {
            double c = cost(li[i - 1], co[j - 1]);
            curr[j] = c + min3(curr[j - 1], prev[j], prev[j - 1]);
            ++cells;
            if (curr[j] <= ub) pruning_point = j + 1;
            j = j + 1;
        }
        /* Stage 3: the column of the previous pruning point (top is > ub). */
        if (j <= hi) {
            double c = cost(li[i - 1], co[j - 1]);
            ++cells;
            if (j == next_start) {
                /* Border collision: only the diagonal is left. */
                curr[j] = c + prev[j - 1];
                if (curr[j] <= ub) pruning_point = j + 1;
                else goto abandon;
            } else {
                curr[j] = c + min2(curr[j - 1], prev[j - 1]);
                if (curr[j] <= ub) pruning_point = j + 1;
            }
            j = j + 1;
        } else if (j == next_start) {
            goto abandon;  /* discard points cover the whole line */
        }
        /* Stage 4: past the previous pruning point only the left neighbour. */
        while (j == pruning_point && j <= hi) {
            double c = cost(li[i - 1], co[j - 1]);  /* READING: recomputed */
            curr[j] = c + curr[j - 1];
            ++cells;
            if (curr[j] <= ub) pruning_point = j + 1;
            j = j + 1;
        }
        prev_pruning_point = pruning_point;
        if (tr && tr->next_start) tr->next_start[i - 1] = next_start;
        if (tr && tr->pruning_point) tr->pruning_point[i - 1] = pruning_point;
    }
    if (prev_pruning_point > l_co) result = curr[l_co];
    else if (tr) tr->abandon_row = l_li;
    goto out;
abandon:
    if (tr) {
        tr->abandon_row = i;
        if (tr->next_start) tr->next_start[i - 1] = next_start;
        if (tr->pruning_point) tr->pruning_point[i - 1] = pruning_point;
    }
out:
    if (tr) tr->cells = cells;
    free(prev);
    free(curr);
    return result;
}

/* ------------------------------------------------------------------------ */
/* z-normalisation.  The paper inherits it from the UCR Suite without        */
/* stating it.  READING: population standard deviation, two-pass FP64:      */
/* mu = sum(x)/m, var = sum((x - mu)^2)/m; a window with var == 0 (a        */
/* constant window) normalises to all zeros.                                */
/* ------------------------------------------------------------------------ */
void orc_znorm(const double* x, int64_t m, double* z) {
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += x[i];
    double mu = s / (double)m;
    double v = 0.0;
    for (int64_t i = 0; i < m; ++i) v += (x[i] - mu) * (x[i] - mu);
    v /= (double)m;
    if (!(v > 0.0)) {
        for (int64_t i = 0; i < m; ++i) z[i] = 0.0;
        return;
    }
    double sd = sqrt(v);
    for (int64_t i = 0; i < m; ++i) z[i] = (x[i] - mu) / sd;
}

/* Mean and population standard deviation of x[0..m), two-pass FP64. */
void orc_mean_std(const double* x, int64_t m, double* mu_out, double* sd_out) {
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += x[i];
    double mu = s / (double)m;
    double v = 0.0;
    for (int64_t i = 0; i < m; ++i) v += (x[i] - mu) * (x[i] - mu);
    v /= (double)m;
    *mu_out = mu;
    *sd_out = v > 0.0 ? sqrt(v) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Lower bounds (Section 2.2 names LB_Kim and LB_Keogh without formulas).    */
/* ------------------------------------------------------------------------ */

/* Envelope over +-w: U[i] = max x[k], L[i] = min x[k], |k - i| <= w, k in   */
/* [0, n).  Written as the definition (O(n w)).                              */
void orc_envelope(const double* x, int64_t n, int64_t w, double* U, double* L) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t a = i - w < 0 ? 0 : i - w;
        int64_t b = i + w > n - 1 ? n - 1 : i + w;
        double u = x[a], l = x[a];
        for (int64_t k = a + 1; k <= b; ++k) {
            if (x[k] > u) u = x[k];
            if (x[k] < l) l = x[k];
        }
        U[i] = u;
        L[i] = l;
    }
}

/* READING (LB_Kim): the first-last form.  Every warping path contains       */
/* (1, 1) and (lS, lT) (Section 2), so the two end costs bound DTW for any   */
/* window.  For m == 1 the two cells coincide and one term is used.          */
double orc_lb_kim_fl(const double* zc, const double* zq, int64_t m) {
    if (m == 1) return cost(zc[0], zq[0]);
    return cost(zc[0], zq[0]) + cost(zc[m - 1], zq[m - 1]);
}

/* LB_Keogh of x against the envelope [L, U]: sum of squared distances from  */
/* x[i] to the interval [L[i], U[i]].  A point's path cells all lie inside   */
/* its +-w neighbourhood, so any envelope covering that neighbourhood gives  */
/* a lower bound of DTW.                                                     */
double orc_lb_keogh(const double* x, const double* U, const double* L, int64_t m) {
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        if (x[i] > U[i]) s += cost(x[i], U[i]);
        else if (x[i] < L[i]) s += cost(x[i], L[i]);
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* k-best list, ascending by (dist, index).  READING: ties in distance go to */
/* the smaller window start, as a left-to-right scan that replaces only on   */
/* a strict improvement would keep.                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t k, n;
    double* d;
    int64_t* idx;
} topk_t;

static int topk_less(double d1, int64_t i1, double d2, int64_t i2) {
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

static void topk_insert(topk_t* t, double d, int64_t i) {
    if (t->n == t->k && !topk_less(d, i, t->d[t->n - 1], t->idx[t->n - 1])) return;
    int32_t p = t->n < t->k ? t->n : t->k - 1;
    while (p > 0 && topk_less(d, i, t->d[p - 1], t->idx[p - 1])) {
        t->d[p] = t->d[p - 1];
        t->idx[p] = t->idx[p - 1];
        --p;
    }
    t->d[p] = d;
    t->idx[p] = i;
    if (t->n < t->k) t->n++;
}

/* Current upper bound: the k-th best distance, +inf until k are known. */
static double topk_ub(const topk_t* t) { return t->n < t->k ? ORC_INF : t->d[t->k - 1]; }

static void topk_out(const topk_t* t, int64_t* idx, double* dist) {
    for (int32_t p = 0; p < t->k; ++p) {
        idx[p] = p < t->n ? t->idx[p] : -1;
        dist[p] = p < t->n ? t->d[p] : ORC_INF;
    }
}

/* ------------------------------------------------------------------------ */
/* O5: brute-force subsequence search.  For every window start i in          */
/* [0, n - m]: z-normalise R[i..i+m), d_i = DTW_w(z_i, zQ) by Algorithm 1    */
/* (rows = candidate, columns = query); return the k smallest (d_i, i).      */
/* Slots beyond the number of windows are (-1, +inf).  Returns 0, or -1 on   */
/* invalid arguments.                                                        */
/* ------------------------------------------------------------------------ */
int orc_search_brute(const double* Q, int64_t m, const double* R, int64_t n, int64_t w,
                     int32_t k, int64_t* idx, double* dist) {
    if (!Q || !R || !idx || !dist || m <= 0 || n < m || w < 0 || k < 1) return -1;
    double* zq = (double*)malloc(sizeof(double) * (size_t)m);
    double* zc = (double*)malloc(sizeof(double) * (size_t)m);
    topk_t t = {k, 0, (double*)malloc(sizeof(double) * (size_t)k),
                (int64_t*)malloc(sizeof(int64_t) * (size_t)k)};
    orc_znorm(Q, m, zq);
    for (int64_t i = 0; i + m <= n; ++i) {
        orc_znorm(R + i, m, zc);
        topk_insert(&t, orc_dtw_tworow(zc, m, zq, m, w), i);
    }
    topk_out(&t, idx, dist);
    free(zq); free(zc); free(t.d); free(t.idx);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* O6: cascade search, the UCR-Suite loop with EAPrunedDTW (Section 5):      */
/* per window, z-normalise, then LB_Kim > ub, LB_Keogh EQ > ub, LB_Keogh EC  */
/* > ub each skip the window; otherwise EAPrunedDTW(z_c, zQ, w, ub), and a   */
/* value <= ub enters the k-best list, whose k-th value is the new ub.       */
/*                                                                          */
/*  - EQ: the candidate against the query's envelope over +-w, clipped to    */
/*    the query.  EC: the query against the envelope of the raw reference    */
/*    over +-min(w, m-1) (not clipped to the window), normalised with the    */
/*    window's mean and deviation; a constant window normalises to zeros.    */
/*  - use_lb = 0 skips all three bounds ("nolb", Section 5).                 */
/*  - ub_fixed: NaN for the running k-th best; a number fixes ub for the     */
/*    whole scan (audit mode: pruning counts no longer depend on order).     */
/*  - nthreads > 1 splits the windows into contiguous ranges; the threads    */
/*    share one k-best list under a mutex.  The result does not depend on    */
/*    the split: pruning is strict (> ub), and every window of the final     */
/*    k-best list has d <= every ub seen.                                    */
/* counters (optional, int64[7]): windows, pruned by Kim, by EQ, by EC, DTW  */
/* abandoned, DTW completed, cells computed.                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *zq, *uq, *lq, *R, *ur, *lr;
    int64_t m, n, w, i0, i1;
    int use_lb;
    double ub_fixed;
    topk_t* t;
    pthread_mutex_t* mu;
    double* ub_shared;
    int64_t cnt[7];
} casc_job;

static double load_ub(casc_job* j) {
    if (!isnan(j->ub_fixed)) return j->ub_fixed;
    double v;
    __atomic_load(j->ub_shared, &v, __ATOMIC_RELAXED);
    return v;
}

static void* casc_worker(void* arg) {
    casc_job* J = (casc_job*)arg;
    int64_t m = J->m;
    double* zc = (double*)malloc(sizeof(double) * (size_t)m);
    double* uc = (double*)malloc(sizeof(double) * (size_t)m);
    double* lc = (double*)malloc(sizeof(double) * (size_t)m);
    for (int64_t i = J->i0; i < J->i1; ++i) {
        J->cnt[0]++;
        double mu, sd;
        orc_mean_std(J->R + i, m, &mu, &sd);
        for (int64_t p = 0; p < m; ++p) zc[p] = sd > 0.0 ? (J->R[i + p] - mu) / sd : 0.0;
        double ub = load_ub(J);
        if (J->use_lb) {
            if (orc_lb_kim_fl(zc, J->zq, m) > ub) { J->cnt[1]++; continue; }
            if (orc_lb_keogh(zc, J->uq, J->lq, m) > ub) { J->cnt[2]++; continue; }
            for (int64_t p = 0; p < m; ++p) {
                uc[p] = sd > 0.0 ? (J->ur[i + p] - mu) / sd : 0.0;
                lc[p] = sd > 0.0 ? (J->lr[i + p] - mu) / sd : 0.0;
            }
            if (orc_lb_keogh(J->zq, uc, lc, m) > ub) { J->cnt[3]++; continue; }
        }
        orc_eap_trace tr;
        memset(&tr, 0, sizeof tr);
        double d = orc_eapruned_dtw(zc, m, J->zq, m, J->w, ub, &tr);
        J->cnt[6] += tr.cells;
        if (d > ub || isinf(d)) {
            J->cnt[4]++;
            continue;
        }
        J->cnt[5]++;
        pthread_mutex_lock(J->mu);
        topk_insert(J->t, d, i);
        if (isnan(J->ub_fixed)) {
            double v = topk_ub(J->t);
            __atomic_store(J->ub_shared, &v, __ATOMIC_RELAXED);
        }
        pthread_mutex_unlock(J->mu);
    }
    free(zc); free(uc); free(lc);
    return NULL;
}

int orc_search_cascade(const double* Q, int64_t m, const double* R, int64_t n, int64_t w,
                       int32_t k, int use_lb, double ub_fixed, int nthreads,
                       int64_t* idx, double* dist, int64_t* counters) {
    if (!Q || !R || !idx || !dist || m <= 0 || n < m || w < 0 || k < 1) return -1;
    if (nthreads < 1) nthreads = 1;
    int64_t nw = n - m + 1;
    if (nthreads > nw) nthreads = (int)nw;
    double* zq = (double*)malloc(sizeof(double) * (size_t)m);
    double* uq = (double*)malloc(sizeof(double) * (size_t)m);
    double* lq = (double*)malloc(sizeof(double) * (size_t)m);
    double* ur = NULL;
    double* lr = NULL;
    orc_znorm(Q, m, zq);
    orc_envelope(zq, m, w, uq, lq);
    if (use_lb) {
        /* READING: the EC envelope radius is min(w, m - 1).  A window point is
         * only ever aligned with points of the same window, which lie within
         * m - 1 of it; any radius >= that gives a valid (superset) envelope,
         * and m - 1 is the tightest such radius for w >= m - 1. */
        ur = (double*)malloc(sizeof(double) * (size_t)n);
        lr = (double*)malloc(sizeof(double) * (size_t)n);
        orc_envelope(R, n, w < m - 1 ? w : m - 1, ur, lr);
    }
    topk_t t = {k, 0, (double*)malloc(sizeof(double) * (size_t)k),
                (int64_t*)malloc(sizeof(int64_t) * (size_t)k)};
    pthread_mutex_t mu;
    pthread_mutex_init(&mu, NULL);
    double ub_shared = ORC_INF;
    casc_job* jobs = (casc_job*)calloc((size_t)nthreads, sizeof(casc_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int p = 0; p < nthreads; ++p) {
        casc_job* J = &jobs[p];
        J->zq = zq; J->uq = uq; J->lq = lq; J->R = R; J->ur = ur; J->lr = lr;
        J->m = m; J->n = n; J->w = w;
        J->i0 = nw * p / nthreads;
        J->i1 = nw * (p + 1) / nthreads;
        J->use_lb = use_lb; J->ub_fixed = ub_fixed;
        J->t = &t; J->mu = &mu; J->ub_shared = &ub_shared;
    }
    if (nthreads == 1) {
        casc_worker(&jobs[0]);
    } else {
        for (int p = 0; p < nthreads; ++p) pthread_create(&th[p], NULL, casc_worker, &jobs[p]);
        for (int p = 0; p < nthreads; ++p) pthread_join(th[p], NULL);
    }
    if (counters) {
        for (int c = 0; c < 7; ++c) {
            counters[c] = 0;
            for (int p = 0; p < nthreads; ++p) counters[c] += jobs[p].cnt[c];
        }
    }
    topk_out(&t, idx, dist);
    pthread_mutex_destroy(&mu);
    free(jobs); free(th);
    free(zq); free(uq); free(lq); free(ur); free(lr);
    free(t.d); free(t.idx);
    return 0;
}

/* Per-window mean/deviation of every window of R (two-pass FP64), for tests  */
/* of the window statistics.                                                 */
void orc_window_stats(const double* R, int64_t n, int64_t m, double* mu, double* sd) {
    for (int64_t i = 0; i + m <= n; ++i) orc_mean_std(R + i, m, &mu[i], &sd[i]);
}

/* ------------------------------------------------------------------------ */
/* Other pointwise costs (Section 6: elastic distances that share DTW's      */
/* recurrence).  cost_mode 0: (a - b)^2 (Eq. 5); 1: |a - b|.  The recurrence */
/* of Eq. 1-4 is unchanged: D(i, j) = cost(i, j) + min(D(i-1, j-1),          */
/* D(i-1, j), D(i, j-1)), D(0, 0) = 0, borders +inf, band |i - j| <= w.      */
/* ------------------------------------------------------------------------ */
static inline double cost_of(double a, double b, int cost_mode) {
    const double d = a - b;
    return cost_mode == 1 ? fabs(d) : d * d;
}

/* Full (lS+1) x (lT+1) DTW matrix with the given cost; returns D(lS, lT),  */
/* NaN on invalid arguments.                                                 */
double orc_dtw_cost(const double* S, int64_t lS, const double* T, int64_t lT, int64_t w, int cost_mode) {
    if (bad_args(S, lS, T, lT, w) || (cost_mode != 0 && cost_mode != 1)) return NAN;
    if (w < abs64(lS - lT)) return ORC_INF;
    const int64_t W = lT + 1;
    double* D = (double*)malloc(sizeof(double) * (size_t)((lS + 1) * W));
    for (int64_t i = 0; i <= lS; ++i)
        for (int64_t j = 0; j <= lT; ++j) D[i * W + j] = ORC_INF;
    D[0] = 0.0;
    for (int64_t i = 1; i <= lS; ++i) {
        for (int64_t j = 1; j <= lT; ++j) {
            if (abs64(i - j) > w) continue;
            D[i * W + j] = cost_of(S[i - 1], T[j - 1], cost_mode) +
                           min3(D[(i - 1) * W + j - 1], D[(i - 1) * W + j], D[i * W + j - 1]);
        }
    }
    const double out = D[lS * W + lT];
    free(D);
    return out;
}

/* Brute-force subsequence search with the given cost: z-normalise Q and     */
/* every window R[i..i+m), d_i = orc_dtw_cost(z_i, zQ, w); the k smallest.   */
int orc_search_brute_cost(const double* Q, int64_t m, const double* R, int64_t n, int64_t w, int32_t k,
                          int cost_mode, int64_t* idx, double* dist) {
    if (!Q || !R || !idx || !dist || m <= 0 || n < m || w < 0 || k < 1 || (cost_mode != 0 && cost_mode != 1))
        return -1;
    double* zq = (double*)malloc(sizeof(double) * (size_t)m);
    double* zc = (double*)malloc(sizeof(double) * (size_t)m);
    topk_t t = {k, 0, (double*)malloc(sizeof(double) * (size_t)k),
                (int64_t*)malloc(sizeof(int64_t) * (size_t)k)};
    orc_znorm(Q, m, zq);
    for (int64_t i = 0; i + m <= n; ++i) {
        orc_znorm(R + i, m, zc);
        topk_insert(&t, orc_dtw_cost(zc, m, zq, m, w, cost_mode), i);
    }
    topk_out(&t, idx, dist);
    free(zq); free(zc); free(t.d); free(t.idx);
    return 0;
}
