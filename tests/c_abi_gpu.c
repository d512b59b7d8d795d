/* Built by tests/test_abi.py (GPU part): a plain C99 program that uses the
 * library through include/umi.h alone -- no Python, no torch -- with device
 * memory from the CUDA runtime.  It runs the batched, host-buffer,
 * single-curve and server entry points on a small uneven batch and checks
 * every trend against the C oracle (linked from oracle/umi_oracle.c, test
 * infrastructure): NaN at the same positions, relative error <= 1e-5.
 * Exit status 0 and "c gpu ok" on success. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "umi.h"

int umi_oracle_detrend(const float *x, int64_t n, int32_t W, double alpha, double c, int iters,
                       int min_valid, double *trend, double *detr, double *median,
                       int32_t *nvalid, int32_t *nplus, double *scale);

enum { B = 7 };
static const int64_t kLen[B] = {1, 500, 3000, 20000, 777, 12000, 0};
static const int32_t kW[B] = {3, 25, 361, 361, 2161, 25, 7};

static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Flux-like test curve: 1 + slow sine + uniform noise, a missing run. */
static void make_curve(float *x, int64_t n, int b)
{
    for (int64_t i = 0; i < n; ++i) {
        const double u = (double)(mix64((uint64_t)(b * 1000003 + i) + 0x9e3779b97f4a7c15ull) >> 11) * 0x1.0p-53;
        x[i] = (float)(1.0 + 2e-3 * sin(0.001 * (double)i + b) + 1e-3 * (u - 0.5));
    }
    for (int64_t i = n / 3; i < n / 3 + n / 20; ++i) x[i] = NAN;
}

static int check(const char *what, const float *got, const float *x, int64_t n, int32_t W)
{
    double *ref = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (umi_oracle_detrend(x, n, W, 2.0, 5.0, 5, -1, ref, NULL, NULL, NULL, NULL, NULL) != 0) {
        free(ref);
        return 1;
    }
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (isnan(ref[i]) != isnan(got[i])) bad = 1;
        else if (!isnan(ref[i]) && fabs((double)got[i] - ref[i]) > 1e-5 * fabs(ref[i])) bad = 1;
        if (bad) {
            fprintf(stderr, "%s: W=%d position %lld: %.9g vs %.9g\n", what, (int)W, (long long)i,
                    (double)got[i], ref[i]);
            break;
        }
    }
    free(ref);
    return bad;
}

#define CUDA_OK(call)                                                               \
    do {                                                                            \
        if ((call) != cudaSuccess) {                                                \
            fprintf(stderr, "CUDA call failed: %s\n", #call);                     \
            return 10;                                                              \
        }                                                                           \
    } while (0)
#define UMI_OK_OR(call)                                                             \
    do {                                                                            \
        if ((call) != UMI_OK) {                                                     \
            fprintf(stderr, "%s failed: %s\n", #call, umi_last_error());            \
            return 11;                                                              \
        }                                                                           \
    } while (0)

int main(void)
{
    int64_t off[B + 1];
    off[0] = 0;
    for (int b = 0; b < B; ++b) off[b + 1] = off[b] + kLen[b];
    const int64_t total = off[B];
    float *x = (float *)malloc(sizeof(float) * (size_t)total);
    float *t_h = (float *)malloc(sizeof(float) * (size_t)total);
    float *t_h2 = (float *)malloc(sizeof(float) * (size_t)total);
    float *d_h2 = (float *)malloc(sizeof(float) * (size_t)total);
    for (int b = 0; b < B; ++b) make_curve(x + off[b], kLen[b], b);

    /* Batched on device buffers. */
    float *x_d = NULL, *t_d = NULL, *d_d = NULL;
    CUDA_OK(cudaMalloc((void **)&x_d, sizeof(float) * (size_t)total));
    CUDA_OK(cudaMalloc((void **)&t_d, sizeof(float) * (size_t)total));
    CUDA_OK(cudaMalloc((void **)&d_d, sizeof(float) * (size_t)total));
    CUDA_OK(cudaMemcpy(x_d, x, sizeof(float) * (size_t)total, cudaMemcpyHostToDevice));
    UMI_OK_OR(umi_detrend_batched(x_d, off, kW, B, NULL, t_d, d_d, NULL));
    CUDA_OK(cudaDeviceSynchronize());
    CUDA_OK(cudaMemcpy(t_h, t_d, sizeof(float) * (size_t)total, cudaMemcpyDeviceToHost));
    int fails = 0;
    for (int b = 0; b < B; ++b) fails += check("batched", t_h + off[b], x + off[b], kLen[b], kW[b]);

    /* The same batch from host buffers: identical to the device-buffer call. */
    UMI_OK_OR(umi_detrend_batched_host(x, off, kW, B, NULL, t_h2, d_h2, NULL));
    if (memcmp(t_h, t_h2, sizeof(float) * (size_t)total) != 0) {
        fprintf(stderr, "host-buffer call differs from the device-buffer call\n");
        ++fails;
    }

    /* One curve at a time. */
    for (int b = 0; b < B; ++b) {
        if (kLen[b] == 0) continue;
        UMI_OK_OR(umi_detrend(x_d + off[b], kLen[b], kW[b], NULL, t_d + off[b], d_d + off[b], NULL));
    }
    CUDA_OK(cudaDeviceSynchronize());
    CUDA_OK(cudaMemcpy(t_h, t_d, sizeof(float) * (size_t)total, cudaMemcpyDeviceToHost));
    for (int b = 0; b < B; ++b) fails += check("single", t_h + off[b], x + off[b], kLen[b], kW[b]);

    /* The server, host inputs. */
    umi_server_config cfg;
    umi_server_default_config(&cfg);
    cfg.mem_budget_bytes = 64ull << 20;
    umi_server *srv = NULL;
    UMI_OK_OR(umi_server_create(&cfg, &srv));
    uint64_t ticket[B];
    for (int b = 0; b < B; ++b) {
        ticket[b] = 0;
        if (kLen[b] == 0) continue;
        UMI_OK_OR(umi_server_submit(srv, x + off[b], 0, kLen[b], kW[b], NULL, &ticket[b]));
    }
    for (int b = 0; b < B; ++b) {
        if (kLen[b] == 0) continue;
        UMI_OK_OR(umi_server_wait(srv, ticket[b], 60.0));
        UMI_OK_OR(umi_server_copy_out(srv, ticket[b], t_h + off[b], NULL));
        UMI_OK_OR(umi_server_release(srv, ticket[b]));
        fails += check("server", t_h + off[b], x + off[b], kLen[b], kW[b]);
    }
    umi_server_destroy(srv);

    cudaFree(x_d);
    cudaFree(t_d);
    cudaFree(d_d);
    free(x);
    free(t_h);
    free(t_h2);
    free(d_h2);
    if (fails) {
        fprintf(stderr, "%d checks failed\n", fails);
        return 1;
    }
    printf("c gpu ok: %d curves, %lld samples, %lld kernels\n", B, (long long)total,
           umi_kernel_launch_count());
    return 0;
}
