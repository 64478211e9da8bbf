/*
 * Exercises every function of the oracles (oracle/oracle.c, oracle/oracle_f32.c)
 * on seeded random inputs, including edge sizes, for a build with AddressSanitizer
 * and UndefinedBehaviorSanitizer (tests/test_oracle_sanitize.py compiles and runs
 * it; any report fails the test).  The values are not checked here: the other
 * oracle tests pin them.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

typedef struct {
    int64_t cells, rows, abandon_row;
    int64_t* next_start;
    int64_t* pruning_point;
} orc_eap_trace;

double orc_dtw_matrix(const double*, int64_t, const double*, int64_t, int64_t, double*);
double orc_dtw_tworow(const double*, int64_t, const double*, int64_t, int64_t);
double orc_dtw_prune_left(const double*, int64_t, const double*, int64_t, double, int64_t*);
double orc_eapruned_dtw(const double*, int64_t, const double*, int64_t, int64_t, double, orc_eap_trace*);
void orc_znorm(const double*, int64_t, double*);
void orc_mean_std(const double*, int64_t, double*, double*);
void orc_envelope(const double*, int64_t, int64_t, double*, double*);
double orc_lb_kim_fl(const double*, const double*, int64_t);
double orc_lb_keogh(const double*, const double*, const double*, int64_t);
int orc_search_brute(const double*, int64_t, const double*, int64_t, int64_t, int32_t, int64_t*, double*);
int orc_search_cascade(const double*, int64_t, const double*, int64_t, int64_t, int32_t, int, double, int,
                       int64_t*, double*, int64_t*);
void orc_window_stats(const double*, int64_t, int64_t, double*, double*);
double orc_dtw_cost(const double*, int64_t, const double*, int64_t, int64_t, int);
int orc_search_brute_cost(const double*, int64_t, const double*, int64_t, int64_t, int32_t, int, int64_t*, double*);
float o7_rsqrt_rn(float);
int o7_search(const float*, int64_t, const float*, int64_t, int64_t, int, int, float, int, int64_t*, int64_t*,
              double*, int8_t*);

static uint64_t st = 88172645463325252ull;
static double rnd(void) {
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    return (double)(st >> 11) / 9007199254740992.0 - 0.5;
}

int main(void) {
    enum { N = 9000 };
    double* R = malloc(sizeof(double) * N);
    float* Rf = malloc(sizeof(float) * N);
    double acc = 0.0;
    for (int i = 0; i < N; ++i) {
        acc += rnd();
        R[i] = acc;
        Rf[i] = (float)acc;
    }
    const int64_t sizes[][3] = {{1, 1, 0}, {1, 5, 2}, {7, 3, 1}, {20, 20, 0}, {33, 40, 45}, {64, 64, 64}};
    for (int c = 0; c < 6; ++c) {
        const int64_t a = sizes[c][0], b = sizes[c][1], w = sizes[c][2];
        double* M = malloc(sizeof(double) * (a + 1) * (b + 1));
        int64_t ns[64], pp[64], ab = 0;
        orc_eap_trace tr = {0, 0, 0, ns, pp};
        orc_dtw_matrix(R, a, R + 100, b, w, M);
        orc_dtw_tworow(R, a, R + 100, b, w);
        orc_dtw_prune_left(R, a, R + 100, b, 5.0, &ab);
        orc_eapruned_dtw(R, a, R + 100, b, w, 3.0, &tr);
        orc_dtw_cost(R, a, R + 100, b, w, 1);
        free(M);
    }
    double z[300], U[300], L[300], mu, sd;
    orc_znorm(R, 300, z);
    orc_mean_std(R, 300, &mu, &sd);
    orc_envelope(z, 300, 7, U, L);
    orc_lb_kim_fl(z, z, 300);
    orc_lb_keogh(z, U, L, 300);
    double* mus = malloc(sizeof(double) * N);
    double* sds = malloc(sizeof(double) * N);
    orc_window_stats(R, N, 50, mus, sds);
    int64_t idx[5], cnt[7], c6[6];
    double dist[5];
    orc_search_brute(R + 10, 40, R, 2000, 5, 3, idx, dist);
    orc_search_cascade(R + 10, 40, R, N, 5, 3, 1, NAN, 4, idx, dist, cnt);
    orc_search_cascade(R + 10, 40, R, N, 40, 1, 0, 9.0, 2, idx, dist, cnt);
    orc_search_brute_cost(R + 10, 40, R, 2000, 5, 2, 1, idx, dist);
    for (int i = 1; i < 2000; ++i) o7_rsqrt_rn((float)(i * 0.37));
    int8_t* why = (int8_t*)malloc((size_t)N);
    o7_search(Rf + 10, 64, Rf, N, 6, 3, 0, 0.0f, 1, c6, idx, dist, NULL);
    o7_search(Rf + 10, 64, Rf, N, 6, 3, 1, 30.0f, 1, c6, idx, dist, why);
    o7_search(Rf + 10, 5000, Rf, 5001, 5000, 1, 1, 1e9f, 0, c6, idx, dist, why);
    free(why);
    free(R); free(Rf); free(mus); free(sds);
    printf("ok\n");
    return 0;
}
