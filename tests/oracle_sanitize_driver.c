/* Built by tests/test_sanitizers.py together with oracle/umi_oracle.c under
 * AddressSanitizer and UndefinedBehaviorSanitizer: every oracle entry point
 * on edge cases (empty and one-sample curves, windows longer than the curve,
 * all-missing curves, missing runs, ties, the largest window, the MAD scale,
 * gap splitting, sampled positions, a threaded batch with empty curves).
 * Every buffer is allocated at its exact size, so any read or write past an
 * end is reported.  Exit status 0 means every call returned as expected. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int umi_oracle_window_length(double cadence_days, double window_days);
int umi_oracle_detrend_mode(const float *x, int64_t n, int32_t W, double alpha, double c,
                            int iters, int min_valid, int scale_mode, double *trend, double *detr,
                            double *median, int32_t *nvalid, int32_t *nplus, double *scale);
int umi_oracle_detrend_positions(const float *x, int64_t n, int32_t W, double alpha, double c,
                                 int iters, int min_valid, const int64_t *positions,
                                 int64_t count, double *trend, double *detr, double *median,
                                 int32_t *nvalid, int32_t *nplus, double *scale);
int umi_oracle_detrend_segmented(const float *x, int64_t n, int32_t W, double alpha, double c,
                                 int iters, int min_valid, int64_t gap_min, int64_t min_seg,
                                 double *trend, double *detr);
int umi_oracle_detrend_batch(const float *x, const int64_t *offsets, const int32_t *W, int32_t B,
                             double alpha, double c, int iters, int min_valid, double *trend,
                             double *detr, int nthreads);

static uint64_t rng_state = 0x9e3779b97f4a7c15ull;
static double uniform(void)
{
    /* splitmix64 */
    uint64_t z = (rng_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

static float *curve(int64_t n, double nan_frac, int run, int ties)
{
    float *x = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        double v = 1.0 + 1e-3 * (uniform() - 0.5);
        if (ties) v = 1.0 + 1e-3 * floor(uniform() * 4.0);
        x[i] = (float)v;
        if (uniform() < nan_frac) x[i] = NAN;
    }
    if (run > 0 && n > 0) {
        int64_t s = (int64_t)(uniform() * (double)n);
        for (int64_t i = s; i < n && i < s + run; ++i) x[i] = NAN;
    }
    return x;
}

static int run_one(int64_t n, int32_t W, int mode, double nan_frac, int run, int ties)
{
    float *x = curve(n, nan_frac, run, ties);
    size_t m = (size_t)(n > 0 ? n : 1);
    double *t = (double *)malloc(sizeof(double) * m), *d = (double *)malloc(sizeof(double) * m);
    double *md = (double *)malloc(sizeof(double) * m), *sc = (double *)malloc(sizeof(double) * m);
    int32_t *nv = (int32_t *)malloc(sizeof(int32_t) * m), *np = (int32_t *)malloc(sizeof(int32_t) * m);
    int rc = umi_oracle_detrend_mode(x, n, W, 2.0, 5.0, 5, -1, mode, t, d, md, nv, np, sc);
    int bad = rc != 0;
    for (int64_t i = 0; i < n && !bad; ++i) {
        if (nv[i] < 0 || nv[i] > W || np[i] < 0 || np[i] > nv[i]) bad = 1;
        if (!isnan(t[i]) && !isfinite(t[i])) bad = 1;
    }
    /* Sampled positions, including both ends. */
    if (n > 0 && !bad) {
        int64_t pos[3] = {0, n / 2, n - 1};
        double pt[3], pd[3], pm[3], ps[3];
        int32_t pn[3], pp[3];
        rc = umi_oracle_detrend_positions(x, n, W, 2.0, 5.0, 5, -1, pos, 3, pt, pd, pm, pn, pp, ps);
        if (rc != 0) bad = 1;
        for (int k = 0; k < 3 && !bad; ++k)
            if (pn[k] != nv[pos[k]]) bad = 1;
    }
    /* Gap splitting with default and explicit parameters. */
    if (!bad) {
        if (umi_oracle_detrend_segmented(x, n, W, 2.0, 5.0, 5, -1, 0, -1, t, d) < 0) bad = 1;
        if (umi_oracle_detrend_segmented(x, n, W, 2.0, 5.0, 5, 0, 3, 0, t, d) < 0) bad = 1;
    }
    free(x);
    free(t);
    free(d);
    free(md);
    free(sc);
    free(nv);
    free(np);
    return bad;
}

int main(void)
{
    int fails = 0;
    if (umi_oracle_window_length(2.0 / 1440.0, 0.5) != 361) ++fails;
    static const int64_t ns[] = {0, 1, 2, 3, 24, 25, 26, 100, 700};
    static const int32_t Ws[] = {1, 3, 25, 61, 361};
    for (size_t a = 0; a < sizeof(ns) / sizeof(ns[0]); ++a)
        for (size_t b = 0; b < sizeof(Ws) / sizeof(Ws[0]); ++b)
            for (int mode = 0; mode < 2; ++mode) {
                fails += run_one(ns[a], Ws[b], mode, 0.0, 0, 0);
                fails += run_one(ns[a], Ws[b], mode, 0.05, Ws[b], 0);
                fails += run_one(ns[a], Ws[b], mode, 1.0, 0, 0); /* all missing */
                fails += run_one(ns[a], Ws[b], mode, 0.0, 0, 1); /* ties */
            }
    fails += run_one(5000, 4095, 0, 0.01, 300, 0); /* the largest window */
    fails += run_one(5000, 4095, 1, 0.0, 0, 1);
    /* Invalid arguments are refused without touching the buffers. */
    if (umi_oracle_detrend_mode(NULL, 10, 4, 2.0, 5.0, 5, -1, 0, NULL, NULL, NULL, NULL, NULL,
                                NULL) != -1)
        ++fails;
    /* A threaded batch with empty curves and mixed windows. */
    {
        enum { B = 9 };
        const int64_t lens[B] = {0, 5, 0, 1, 800, 0, 3, 300, 2};
        const int32_t W[B] = {3, 361, 25, 1, 61, 7, 2161, 25, 5};
        int64_t off[B + 1];
        off[0] = 0;
        for (int b = 0; b < B; ++b) off[b + 1] = off[b] + lens[b];
        float *x = curve(off[B], 0.02, 20, 0);
        double *t = (double *)malloc(sizeof(double) * (size_t)off[B]);
        double *d = (double *)malloc(sizeof(double) * (size_t)off[B]);
        if (umi_oracle_detrend_batch(x, off, W, B, 2.0, 5.0, 5, -1, t, d, 4) != 0) ++fails;
        free(x);
        free(t);
        free(d);
    }
    printf("oracle sanitizer driver: %d failures\n", fails);
    return fails == 0 ? 0 : 1;
}
