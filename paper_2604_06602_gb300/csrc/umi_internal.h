// umi_internal.h -- shared host-side pieces of libumi (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <map>
#include <utility>
#include <vector>

#include "umi.h"
#include "umi_kernel.cuh"
#include "umi_variants.h"

namespace umi {

// Records a message for umi_last_error() and returns the status.
umi_status fail(umi_status st, const std::string &msg);
umi_status fail_cuda(cudaError_t err, const char *what);
void clear_error();

struct DeviceInfo {
    int device = -1;
    int sms = 0;
    size_t smem_optin = 0;
    std::string name;
};
const DeviceInfo &device_info(int device);
int current_device();

// Planning regimes: a band that fills the GPU at the shortest chain of its
// throughput variant, and one that does not (see make_plan).
enum : int { kRegimeThroughput = 0, kRegimeLatency = 1 };

// A launch plan for one window band.
struct Plan {
    int variant = -1;
    int G = 0, R = 0;
    int chain = 0;    // positions per group
    int threads = 0;  // per CTA
    int regime = 0;   // kRegimeThroughput or kRegimeLatency
    int64_t tuned_at = 0;  // band size a tuned plan was measured at (0: unknown)
    // Positions per work item (one warp's tile).
    int tile() const { return (32 / G) * chain; }
    size_t smem_bytes() const
    {
        return sizeof(float) * (size_t)(threads / 32) *
               (size_t)(tile() + G * R - 1 + (stages_outputs(G) ? tile() : 0));
    }
};

// Longest window a kernel variant covers.
constexpr int kMaxWindow = 4095;

// ---- planner (umi_plan.cu) ----
bool legal_chain(int G, int chain);
// Smallest legal chain of at least `target` positions; the shortest legal
// chain; the longest chain the rule uses.
int chain_at_least(int G, int64_t target);
int shortest_chain(int G);
int chain_cap(int G);
// Regime of a band of `positions` windows of length W (positions <= 0: throughput).
int plan_regime(int W, int64_t positions);
// Plan for a band of `positions` windows of length W (positions <= 0: a band
// large enough for the longest chain): the tuned plan for (W, regime) if any,
// else the measured rule; the chain shrinks for small bands.
umi_status make_plan(int W, int64_t positions, Plan *plan);
// The plans umi_autotune times for a band of `positions` windows of length W.
std::vector<Plan> autotune_candidates(int W, int64_t positions);
// Records a tuned plan for (W, p.regime).
void store_tuned(int W, const Plan &p);
// Bumped by every change of the tuned-plan table (part of the graph-cache key).
uint64_t tune_epoch();
void plan_out(const Plan &p, umi_plan *out);
umi_status check_params(const umi_params *p, umi_params *out);
int resolve_min_valid(int W, int min_valid);
// `flavour` = kFlagDiag | kFlagMad bits (the kernel build to use).
umi_status prepare_kernel(const Plan &plan, int flavour);
// Persistent grid size for a plan on the current device.
int persistent_grid(const Plan &plan, int flavour);

// Windows per (window length, scale mode) band.  A call that runs its
// curves in several pieces (pipelined chunks, gap segments) plans every piece
// from the sizes of the whole call's bands, so that it runs the same kernel
// variants as one batched launch over the same curves.
using BandSizes = std::map<std::pair<int, int>, int64_t>;

// One batched launch over an explicit curve table (used by the CSR entry
// point and by the server).  `curves` are host descriptors with device data
// pointers; device scratch is taken with cudaMallocAsync on `stream`.
// `launches` (may be null) receives the number of kernels launched;
// `plan_sizes` (may be null: the table's own bands) sizes the plans.
umi_status launch_curve_table(const std::vector<Curve> &curves, cudaStream_t stream,
                              int *launches, const BandSizes *plan_sizes = nullptr);

// One curve in one launch without work-queue tables (the kernel numbers the
// curve's tiles itself): nothing is copied to the device first.
// `plan_positions` is the size of the band the curve is planned with.
umi_status launch_single_curve(const Curve &c, int64_t plan_positions, const Diag *diag,
                               cudaStream_t stream, int *launches);

// Adds to the process-wide count of kernels launched by libumi.
void count_launches(int n);

// A named NVTX range over a scope, for profilers (NVTX 3 is header-only and
// costs a branch when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Raises the release threshold of the current device's default memory pool
// (once per device), so cudaMallocAsync scratch is reused across calls.
void keep_pool_memory();

// Gap-split detrend (umi_segments.cu).
umi_status detrend_segmented(const float *flux, const int64_t *offsets, const int32_t *W, int32_t B,
                             const umi_params *params, const umi_segment_params *seg, float *trend,
                             float *detr, int64_t *segments_out, cudaStream_t stream);

// Work-item list and per-variant launch layout for a curve table.
struct BatchLayout {
    struct Band {
        Plan plan;
        int flavour = 0;  // kFlagMad when the band's curves use the MAD scale
        int32_t first_item = 0;
        int32_t n_items = 0;
    };
    std::vector<Band> bands;
    std::vector<Item> items;
    int32_t n_curves = 0;  // entries of the curve table the items index
};
umi_status build_layout(const std::vector<Curve> &curves, BatchLayout *layout,
                        const BandSizes *plan_sizes = nullptr);

// A batch planned for caller-owned buffers: `dev_bytes` of device scratch and
// `host_bytes` of (preferably pinned) host staging for the tables.
struct PreparedBatch {
    BatchLayout layout;
    size_t curve_off = 0, item_off = 0, counter_off = 0;
    size_t dev_bytes = 0, host_bytes = 0;
};
umi_status prepare_batch(const std::vector<Curve> &curves, PreparedBatch *pb);
// Stages the tables in `host`, copies them to `dev` on `stream`, clears the
// counters and launches the bands.  The host buffer must stay untouched until
// the copy has run (stream order).
umi_status enqueue_prepared(const std::vector<Curve> &curves, const PreparedBatch &pb, char *dev,
                            char *host, cudaStream_t stream, int *launches);

}  // namespace umi
