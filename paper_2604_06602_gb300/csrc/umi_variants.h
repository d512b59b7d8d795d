// umi_variants.h -- table of compiled kernel variants (lanes per window G,
// register slots per lane R).  Each variant serves windows with W <= G*R.
#pragma once

#include <cuda_runtime.h>

#include "umi_kernel.cuh"

namespace umi {

typedef cudaError_t (*LaunchFn)(const LaunchArgs &args, int grid, int threads, size_t smem,
                                cudaStream_t stream);

struct Variant {
    int G;
    int R;
    LaunchFn launch;       // trend / detr only
    LaunchFn launch_diag;  // with the diagnostic outputs
    const void *kernel;    // for occupancy queries and attributes
    const void *kernel_diag;
};

// All compiled variants, ordered by slot capacity G*R (ascending).
const Variant *variant_table(int *count);

}  // namespace umi

// Defines the launchers of one (G, R) variant in the including translation unit.
#define UMI_DEFINE_VARIANT(G_, R_)                                                            \
    namespace umi {                                                                           \
    cudaError_t launch_v##G_##_##R_(const LaunchArgs &a, int grid, int threads, size_t smem, \
                                    cudaStream_t st)                                         \
    {                                                                                         \
        umi_tile_kernel<G_, R_, false><<<grid, threads, smem, st>>>(a);                       \
        return cudaGetLastError();                                                            \
    }                                                                                         \
    cudaError_t launch_d##G_##_##R_(const LaunchArgs &a, int grid, int threads, size_t smem, \
                                    cudaStream_t st)                                         \
    {                                                                                         \
        umi_tile_kernel<G_, R_, true><<<grid, threads, smem, st>>>(a);                        \
        return cudaGetLastError();                                                            \
    }                                                                                         \
    const void *kernel_v##G_##_##R_() { return (const void *)umi_tile_kernel<G_, R_, false>; } \
    const void *kernel_d##G_##_##R_() { return (const void *)umi_tile_kernel<G_, R_, true>; }  \
    }

#define UMI_DECLARE_VARIANT(G_, R_)                                                           \
    namespace umi {                                                                           \
    cudaError_t launch_v##G_##_##R_(const LaunchArgs &, int, int, size_t, cudaStream_t);     \
    cudaError_t launch_d##G_##_##R_(const LaunchArgs &, int, int, size_t, cudaStream_t);     \
    const void *kernel_v##G_##_##R_();                                                        \
    const void *kernel_d##G_##_##R_();                                                        \
    }

// The variant list: (G, R).  Capacities 8 .. 4096 slots.
#define UMI_VARIANT_LIST(X) \
    X(1, 8)                 \
    X(1, 16)                \
    X(1, 32)                \
    X(2, 32)                \
    X(4, 32)                \
    X(8, 24)                \
    X(8, 46)                \
    X(16, 48)               \
    X(32, 48)               \
    X(32, 68)               \
    X(32, 128)
