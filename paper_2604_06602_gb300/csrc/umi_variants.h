// umi_variants.h -- table of compiled kernel variants: lanes per window G,
// register slots per lane R, and MINB, the CTAs of 256 threads per SM the
// register allocation aims for.  Each variant serves windows with W <= G*R.
#pragma once

#include <cuda_runtime.h>

#include "umi_kernel.cuh"

namespace umi {

typedef cudaError_t (*LaunchFn)(const LaunchArgs &args, int grid, int threads, size_t smem,
                                cudaStream_t stream);

// Kernel flavours: index = kFlagDiag | kFlagMad bits.
constexpr int kFlavours = 4;

struct Variant {
    int G;
    int R;
    int minb;
    LaunchFn launch[kFlavours];
    const void *kernel[kFlavours];  // for occupancy queries and attributes
};

// All compiled variants, ordered by slot capacity G*R (ascending).
const Variant *variant_table(int *count);

}  // namespace umi

// Defines the launchers of one (G, R, MINB) variant in the including translation unit.
#define UMI_VNAME(p, G_, R_, M_) p##G_##_##R_##_##M_
#define UMI_DEFINE_VARIANT(G_, R_, M_)                                                        \
    namespace umi {                                                                           \
    template <int F>                                                                          \
    static cudaError_t UMI_VNAME(launch_, G_, R_, M_)(const LaunchArgs &a, int grid,          \
                                                      int threads, size_t smem,               \
                                                      cudaStream_t st)                        \
    {                                                                                         \
        umi_tile_kernel<G_, R_, M_, F><<<grid, threads, smem, st>>>(a);                       \
        return cudaGetLastError();                                                            \
    }                                                                                         \
    void UMI_VNAME(fill_, G_, R_, M_)(Variant * v)                                            \
    {                                                                                         \
        v->G = G_;                                                                            \
        v->R = R_;                                                                            \
        v->minb = M_;                                                                         \
        v->launch[0] = UMI_VNAME(launch_, G_, R_, M_)<0>;                                     \
        v->launch[1] = UMI_VNAME(launch_, G_, R_, M_)<1>;                                     \
        v->launch[2] = UMI_VNAME(launch_, G_, R_, M_)<2>;                                     \
        v->launch[3] = UMI_VNAME(launch_, G_, R_, M_)<3>;                                     \
        v->kernel[0] = (const void *)umi_tile_kernel<G_, R_, M_, 0>;                          \
        v->kernel[1] = (const void *)umi_tile_kernel<G_, R_, M_, 1>;                          \
        v->kernel[2] = (const void *)umi_tile_kernel<G_, R_, M_, 2>;                          \
        v->kernel[3] = (const void *)umi_tile_kernel<G_, R_, M_, 3>;                          \
    }                                                                                         \
    }

#define UMI_DECLARE_VARIANT(G_, R_, M_)                   \
    namespace umi {                                       \
    void UMI_VNAME(fill_, G_, R_, M_)(Variant * v);       \
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
