// umi_variants.h -- table of compiled kernel variants: lanes per window G,
// register slots per lane R, and MINB, the CTAs of 256 threads per SM the
// register allocation aims for.  Each variant serves windows with W <= G*R.
#pragma once

#include <cuda_runtime.h>

#include "umi_kernel.cuh"

namespace umi {

typedef cudaError_t (*LaunchFn)(const LaunchArgs &args, int grid, int threads, size_t smem,
                                cudaStream_t stream);

struct Variant {
    int G;
    int R;
    int minb;
    LaunchFn launch;       // trend / detr only
    LaunchFn launch_diag;  // with the diagnostic outputs
    const void *kernel;    // for occupancy queries and attributes
    const void *kernel_diag;
};

// All compiled variants, ordered by slot capacity G*R (ascending).
const Variant *variant_table(int *count);

}  // namespace umi

// Defines the launchers of one (G, R, MINB) variant in the including translation unit.
#define UMI_VNAME(p, G_, R_, M_) p##G_##_##R_##_##M_
#define UMI_DEFINE_VARIANT(G_, R_, M_)                                                        \
    namespace umi {                                                                           \
    cudaError_t UMI_VNAME(launch_v, G_, R_, M_)(const LaunchArgs &a, int grid, int threads,  \
                                                size_t smem, cudaStream_t st)                \
    {                                                                                         \
        umi_tile_kernel<G_, R_, M_, false><<<grid, threads, smem, st>>>(a);                   \
        return cudaGetLastError();                                                            \
    }                                                                                         \
    cudaError_t UMI_VNAME(launch_d, G_, R_, M_)(const LaunchArgs &a, int grid, int threads,  \
                                                size_t smem, cudaStream_t st)                \
    {                                                                                         \
        umi_tile_kernel<G_, R_, M_, true><<<grid, threads, smem, st>>>(a);                    \
        return cudaGetLastError();                                                            \
    }                                                                                         \
    const void *UMI_VNAME(kernel_v, G_, R_, M_)()                                             \
    {                                                                                         \
        return (const void *)umi_tile_kernel<G_, R_, M_, false>;                              \
    }                                                                                         \
    const void *UMI_VNAME(kernel_d, G_, R_, M_)()                                             \
    {                                                                                         \
        return (const void *)umi_tile_kernel<G_, R_, M_, true>;                               \
    }                                                                                         \
    }

#define UMI_DECLARE_VARIANT(G_, R_, M_)                                                       \
    namespace umi {                                                                           \
    cudaError_t UMI_VNAME(launch_v, G_, R_, M_)(const LaunchArgs &, int, int, size_t,        \
                                                cudaStream_t);                               \
    cudaError_t UMI_VNAME(launch_d, G_, R_, M_)(const LaunchArgs &, int, int, size_t,        \
                                                cudaStream_t);                               \
    const void *UMI_VNAME(kernel_v, G_, R_, M_)();                                            \
    const void *UMI_VNAME(kernel_d, G_, R_, M_)();                                            \
    }

// The variant list: (G, R, MINB), ordered by slot capacity G*R; for equal
// capacity the first entry is the default and the autotuner may pick others.
#define UMI_VARIANT_LIST(X) \
    X(1, 8, 4)              \
    X(1, 16, 4)             \
    X(1, 26, 4)             \
    X(1, 32, 3)             \
    X(2, 32, 3)             \
    X(4, 32, 3)             \
    X(8, 24, 3)             \
    X(8, 46, 2)             \
    X(8, 46, 3)             \
    X(16, 24, 4)            \
    X(32, 12, 4)            \
    X(16, 48, 2)            \
    X(32, 48, 2)            \
    X(32, 68, 2)            \
    X(32, 128, 1)
