/*
 * umi_oracle.c -- FP64 CPU oracle for the UMI sliding-window robust trend.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library, and the product path never
 * calls it.
 *
 * Every floating-point step runs in IEEE double.  Input samples are FP32 and
 * are promoted to double exactly.  The steps follow the paper's Section 2
 * ("Algorithm") in its order:
 *
 *   window        Section 2 opening paragraph: a W-sample window per position,
 *                 W = round(0.5 d / cadence) | 1.
 *   Phase 1       Section 2.1: the exact sample median (here: sort the valid
 *                 samples with the C library qsort and take one order
 *                 statistic).
 *   Phase 2       Section 2.2, Eq. 1: sigma_up = sqrt(mean over x_i > median of
 *                 (x_i - median)^2), s = 0.6745 * sigma_up.
 *   Phase 3       Section 2.3, Eqs. 2-4: u = (x - mu) / (c s); u_eff = alpha u
 *                 for u < 0, else u; w = (1 - u_eff^2)^2 for |u_eff| < 1, else
 *                 0; mu <- sum(w x) / sum(w); a fixed number of iterations
 *                 (5 in the paper, no convergence test).
 *   output        detrended flux = flux / trend.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - the window is centred, h = (W-1)/2 samples each side, and truncated at
 *     the ends of the curve (never shifted or padded);
 *   - a sample is missing when it is not finite; missing samples are dropped
 *     from the window (the window still spans W index slots);
 *   - a position whose own sample is missing, or whose window holds fewer than
 *     min_valid valid samples (default floor(W/3), read from the W/3 minimum
 *     segment rule of Section 4, Kepler Long-Cadence), yields NaN;
 *   - for an even count n the median is the lower median, rank floor((n-1)/2)
 *     (0-based), a single order statistic;
 *   - "above the median" is strict (x > median), as Eq. 1 is written;
 *   - when no sample lies above the median, or s == 0, the trend is the median;
 *   - when sum(w) == 0 in an iteration, mu keeps its value;
 *   - u == 0 takes the u >= 0 branch of Eq. 2, and |u_eff| < 1 is strict (Eq. 3);
 *   - s is computed once (Phase 2) and held fixed through the iterations;
 *   - the constant 0.6745 is used as printed in Section 2.2.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_SCALE_FACTOR 0.6745 /* Section 2.2, as printed */

/* ---- Section 2 opening paragraph: W = round(0.5 / dt) | 1 ---------------- */
int umi_oracle_window_length(double cadence_days, double window_days)
{
    if (!(cadence_days > 0.0) || !(window_days > 0.0) || !isfinite(cadence_days) ||
        !isfinite(window_days))
        return -1;
    double ratio = window_days / cadence_days;
    if (!(ratio < 1.0e9))
        return -1;
    long w = lround(ratio); /* nearest, halves away from zero */
    return (int)(w | 1L);
}

/* ---- Section 2.3, Eqs. 2 and 3: the asymmetric bisquare weight of u ------- */
double umi_oracle_weight(double u, double alpha)
{
    double u_eff = (u < 0.0) ? alpha * u : u; /* Eq. 2 */
    if (fabs(u_eff) < 1.0) {                  /* Eq. 3 */
        double t = 1.0 - u_eff * u_eff;
        return t * t;
    }
    return 0.0;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Scale estimators: Eq. 1 (the method) and the MAD it is compared with. */
enum { ORACLE_SCALE_UPPER_RMS = 0, ORACLE_SCALE_MAD = 1 };

/*
 * One window, given as the multiset of its valid samples v[0..n) (all finite).
 * The array is sorted in place.  Writes the median (Phase 1), the count of
 * samples strictly above it, the scale s and the location after `iters`
 * iterations of Phase 3.  scale_mode 0 is the upper-RMS scale of Eq. 1
 * (Section 2.2); scale_mode 1 is the standard MAD the paper compares it with
 * (Sections 1 and 2.2, and the ablation of Section 3.1): the median of
 * |v - m|, taken as the same lower-median order statistic, without a factor
 * (the MAD is the convention 0.6745 * sigma_up is matched to).
 * Returns 0, or -1 when n < 1.
 */
int umi_oracle_window_estimate_mode(double *v, int n, double alpha, double c, int iters,
                                    int scale_mode, double *median_out, int *nplus_out,
                                    double *scale_out, double *mu_out)
{
    if (n < 1)
        return -1;
    /* Phase 1 (Section 2.1): exact order statistic of rank floor((n-1)/2). */
    qsort(v, (size_t)n, sizeof(double), cmp_double);
    double m = v[(n - 1) / 2];

    /* Phase 2 (Section 2.2, Eq. 1): upper RMS about the median. */
    int nplus = 0;
    double s2 = 0.0;
    for (int i = 0; i < n; ++i) {
        if (v[i] > m) {
            double d = v[i] - m;
            s2 += d * d;
            ++nplus;
        }
    }
    double s = 0.0;
    if (scale_mode == ORACLE_SCALE_MAD) {
        double *dev = (double *)malloc(sizeof(double) * (size_t)n);
        if (!dev)
            return -1;
        for (int i = 0; i < n; ++i)
            dev[i] = fabs(v[i] - m);
        qsort(dev, (size_t)n, sizeof(double), cmp_double);
        s = dev[(n - 1) / 2];
        free(dev);
    } else if (nplus > 0) {
        s = ORACLE_SCALE_FACTOR * sqrt(s2 / (double)nplus);
    }

    /* Phase 3 (Section 2.3, Eqs. 2-4): fixed number of reweighting steps.
     * With the upper-RMS scale n_plus = 0 means s = 0; both give the median. */
    double mu = m;
    if (s > 0.0) {
        double cs = c * s;
        for (int it = 0; it < iters; ++it) {
            double sw = 0.0, swx = 0.0;
            for (int i = 0; i < n; ++i) {
                double u = (v[i] - mu) / cs;
                double w = umi_oracle_weight(u, alpha);
                sw += w;
                swx += w * v[i];
            }
            if (sw > 0.0)
                mu = swx / sw; /* Eq. 4 */
        }
    }
    if (median_out)
        *median_out = m;
    if (nplus_out)
        *nplus_out = nplus;
    if (scale_out)
        *scale_out = s;
    if (mu_out)
        *mu_out = mu;
    return 0;
}

int umi_oracle_window_estimate(double *v, int n, double alpha, double c, int iters,
                               double *median_out, int *nplus_out, double *scale_out,
                               double *mu_out)
{
    return umi_oracle_window_estimate_mode(v, n, alpha, c, iters, ORACLE_SCALE_UPPER_RMS,
                                           median_out, nplus_out, scale_out, mu_out);
}

/* Everything the oracle reports for one output position. */
typedef struct {
    double trend, detr, median, scale;
    int32_t nvalid, nplus;
} position_result;

/*
 * One output position j of a curve x[0..n).  `scratch` holds at least W
 * doubles.  Fields:
 *   trend, detr   NaN when x[j] is missing, the window is empty, or it holds
 *                 fewer than min_valid valid samples;
 *   median        the window median whenever the window holds a valid sample
 *                 (NaN otherwise), also at positions whose output is NaN;
 *   nvalid        number of valid samples in the window;
 *   nplus         samples strictly above the median (0 for an empty window);
 *   scale         s of Phase 2 where the trend is produced, else NaN.
 */
static position_result oracle_position(const float *x, int64_t n, int32_t W, double alpha,
                                       double c, int iters, int min_valid, int scale_mode,
                                       int64_t j, double *scratch)
{
    int64_t h = (W - 1) / 2;
    int64_t lo = j - h < 0 ? 0 : j - h;
    int64_t hi = j + h > n - 1 ? n - 1 : j + h;
    int cnt = 0;
    for (int64_t i = lo; i <= hi; ++i) {
        double xi = (double)x[i];
        if (isfinite(xi))
            scratch[cnt++] = xi;
    }
    double m = NAN, s = NAN, mu = NAN;
    int np = 0;
    if (cnt >= 1)
        umi_oracle_window_estimate_mode(scratch, cnt, alpha, c, iters, scale_mode, &m, &np, &s,
                                        &mu);
    int produce = cnt >= 1 && cnt >= min_valid && isfinite((double)x[j]);
    position_result r;
    r.trend = produce ? mu : NAN;
    r.detr = produce ? (double)x[j] / mu : NAN;
    r.median = m;
    r.nvalid = cnt;
    r.nplus = np;
    r.scale = produce ? s : NAN;
    return r;
}

static int resolve_min_valid(int32_t W, int min_valid)
{
    return min_valid < 0 ? W / 3 : min_valid;
}

static int bad_args(int64_t n, int32_t W, double alpha, double c, int iters)
{
    return n < 0 || W < 1 || (W % 2) == 0 || iters < 0 || !(alpha > 0.0) || !(c > 0.0) ||
           !isfinite(alpha) || !isfinite(c);
}

/*
 * Whole curve.  Output arrays have n entries; any may be NULL.  Returns 0, or
 * -1 on an invalid argument (W not odd or < 1, n < 0, iters < 0, alpha or c
 * not a positive finite number).
 */
int umi_oracle_detrend_mode(const float *x, int64_t n, int32_t W, double alpha, double c,
                            int iters, int min_valid, int scale_mode, double *trend, double *detr,
                            double *median, int32_t *nvalid, int32_t *nplus, double *scale)
{
    if (bad_args(n, W, alpha, c, iters) || scale_mode < 0 || scale_mode > 1)
        return -1;
    if (n == 0)
        return 0;
    double *scratch = (double *)malloc(sizeof(double) * (size_t)W);
    if (!scratch)
        return -1;
    int mv = resolve_min_valid(W, min_valid);
    for (int64_t j = 0; j < n; ++j) {
        position_result r = oracle_position(x, n, W, alpha, c, iters, mv, scale_mode, j, scratch);
        if (trend) trend[j] = r.trend;
        if (detr) detr[j] = r.detr;
        if (median) median[j] = r.median;
        if (nvalid) nvalid[j] = r.nvalid;
        if (nplus) nplus[j] = r.nplus;
        if (scale) scale[j] = r.scale;
    }
    free(scratch);
    return 0;
}

int umi_oracle_detrend(const float *x, int64_t n, int32_t W, double alpha, double c, int iters,
                       int min_valid, double *trend, double *detr, double *median,
                       int32_t *nvalid, int32_t *nplus, double *scale)
{
    return umi_oracle_detrend_mode(x, n, W, alpha, c, iters, min_valid, ORACLE_SCALE_UPPER_RMS,
                                   trend, detr, median, nvalid, nplus, scale);
}

/*
 * Selected positions of one curve (for sampled checks on curves too long to
 * evaluate in full).  Output arrays are indexed like `positions`.
 */
int umi_oracle_detrend_positions(const float *x, int64_t n, int32_t W, double alpha, double c,
                                 int iters, int min_valid, const int64_t *positions,
                                 int64_t count, double *trend, double *detr, double *median,
                                 int32_t *nvalid, int32_t *nplus, double *scale)
{
    if (bad_args(n, W, alpha, c, iters) || count < 0)
        return -1;
    for (int64_t q = 0; q < count; ++q)
        if (positions[q] < 0 || positions[q] >= n)
            return -1;
    double *scratch = (double *)malloc(sizeof(double) * (size_t)W);
    if (!scratch)
        return -1;
    int mv = resolve_min_valid(W, min_valid);
    for (int64_t q = 0; q < count; ++q) {
        position_result r =
            oracle_position(x, n, W, alpha, c, iters, mv, ORACLE_SCALE_UPPER_RMS, positions[q], scratch);
        if (trend) trend[q] = r.trend;
        if (detr) detr[q] = r.detr;
        if (median) median[q] = r.median;
        if (nvalid) nvalid[q] = r.nvalid;
        if (nplus) nplus[q] = r.nplus;
        if (scale) scale[q] = r.scale;
    }
    free(scratch);
    return 0;
}

/*
 * Gap handling before the detrend (the pipeline step the paper lists before
 * detrending in Table 3's caption; the W/3 minimum segment length of
 * Section 4, Kepler Long-Cadence).  Reading: a curve splits into segments at
 * every run of at least `gap_min` consecutive missing samples (default W);
 * leading and trailing missing runs belong to no segment.  A segment holding
 * fewer than `min_seg` valid samples (default floor(W/3)) is dropped.  Each
 * kept segment is detrended on its own, so windows are truncated at segment
 * ends exactly as at curve ends.  Positions outside kept segments get NaN.
 * Returns the number of kept segments, or -1 on invalid arguments.
 */
int umi_oracle_detrend_segmented(const float *x, int64_t n, int32_t W, double alpha, double c,
                                 int iters, int min_valid, int64_t gap_min, int64_t min_seg,
                                 double *trend, double *detr)
{
    if (bad_args(n, W, alpha, c, iters))
        return -1;
    if (gap_min <= 0)
        gap_min = W;
    if (min_seg < 0)
        min_seg = W / 3;
    for (int64_t j = 0; j < n; ++j) {
        trend[j] = NAN;
        detr[j] = NAN;
    }
    int kept = 0;
    int64_t j = 0;
    while (j < n) {
        /* Skip missing samples to the next segment start. */
        while (j < n && !isfinite((double)x[j]))
            ++j;
        if (j >= n)
            break;
        int64_t start = j, last_valid = j, valid = 0;
        int64_t run = 0; /* current run of missing samples */
        while (j < n) {
            if (isfinite((double)x[j])) {
                run = 0;
                last_valid = j;
                ++valid;
            } else if (++run >= gap_min) {
                break;
            }
            ++j;
        }
        int64_t len = last_valid + 1 - start;
        if (valid >= 1 && valid >= min_seg) {
            if (umi_oracle_detrend(x + start, len, W, alpha, c, iters, min_valid, trend + start,
                                   detr + start, NULL, NULL, NULL, NULL) != 0)
                return -1;
            ++kept;
        }
        j = last_valid + 1;
    }
    return kept;
}

/* ---- many curves in CSR layout, one curve per task, over pthreads -------- */
typedef struct {
    const float *x;
    const int64_t *offsets;
    const int32_t *W;
    int32_t B;
    double alpha, c;
    int iters, min_valid;
    double *trend, *detr;
    int next; /* next curve to take, updated atomically */
    int failed;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *job = (batch_job *)arg;
    for (;;) {
        int b = __atomic_fetch_add(&job->next, 1, __ATOMIC_RELAXED);
        if (b >= job->B)
            break;
        int64_t o = job->offsets[b], len = job->offsets[b + 1] - o;
        if (umi_oracle_detrend(job->x + o, len, job->W[b], job->alpha, job->c, job->iters,
                               job->min_valid, job->trend + o, job->detr + o, NULL, NULL, NULL,
                               NULL) != 0)
            __atomic_store_n(&job->failed, 1, __ATOMIC_RELAXED);
    }
    return NULL;
}

int umi_oracle_detrend_batch(const float *x, const int64_t *offsets, const int32_t *W, int32_t B,
                             double alpha, double c, int iters, int min_valid, double *trend,
                             double *detr, int nthreads)
{
    if (B < 0 || nthreads < 1)
        return -1;
    for (int32_t b = 0; b < B; ++b)
        if (offsets[b + 1] < offsets[b])
            return -1;
    batch_job job = {x, offsets, W, B, alpha, c, iters, min_valid, trend, detr, 0, 0};
    if (nthreads > 256)
        nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, batch_worker, &job) != 0)
            break;
        ++started;
    }
    if (started == 0)
        batch_worker(&job);
    for (int t = 0; t < started; ++t)
        pthread_join(th[t], NULL);
    return job.failed ? -1 : 0;
}
