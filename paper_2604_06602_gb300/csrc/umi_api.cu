// umi_api.cu -- the C ABI of libumi: validation, launches, the batched work
// queue, the CUDA-graph cache and the autotuner's timing runs (the planner
// and the tuned-plan table are umi_plan.cu).
//
// The estimator is Section 2 of the paper (window rule; Phase 1 median;
// Phase 2 upper-RMS scale, Eq. 1; Phase 3 asymmetric bisquare, Eqs. 2-4);
// the device code is umi_kernel.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "umi_internal.h"

namespace umi {

// ---------------------------------------------------------------- errors --
static thread_local std::string t_error;

umi_status fail(umi_status st, const std::string &msg)
{
    t_error = msg;
    return st;
}

umi_status fail_cuda(cudaError_t err, const char *what)
{
    t_error = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
    return err == cudaErrorMemoryAllocation ? UMI_ERR_OOM : UMI_ERR_CUDA;
}

void clear_error() { t_error.clear(); }

#define UMI_CUDA(call, what)                         \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return fail_cuda(e_, what); \
    } while (0)

// ----------------------------------------------------------- device info --
static std::mutex g_dev_mu;

int current_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return -1;
    return d;
}

const DeviceInfo &device_info(int device)
{
    static std::map<int, DeviceInfo> cache;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = cache.find(device);
    if (it != cache.end()) return it->second;
    DeviceInfo di;
    di.device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) {
        di.sms = prop.multiProcessorCount;
        di.smem_optin = prop.sharedMemPerBlockOptin;
        di.name = prop.name;
    }
    return cache.emplace(device, di).first->second;
}

int resolve_min_valid(int W, int min_valid) { return min_valid < 0 ? W / 3 : min_valid; }

umi_status check_params(const umi_params *p, umi_params *out)
{
    umi_params q;
    umi_default_params(&q);
    if (p) q = *p;
    if (!(q.alpha > 0.f) || !std::isfinite(q.alpha))
        return fail(UMI_ERR_INVALID_ARG, "alpha must be a positive finite number");
    if (!(q.c > 0.f) || !std::isfinite(q.c))
        return fail(UMI_ERR_INVALID_ARG, "c must be a positive finite number");
    if (q.iters < 0 || q.iters > 1000) return fail(UMI_ERR_INVALID_ARG, "iters must be in [0, 1000]");
    if (q.min_valid < -1) return fail(UMI_ERR_INVALID_ARG, "min_valid must be >= -1");
    if (q.scale_mode != UMI_SCALE_UPPER_RMS && q.scale_mode != UMI_SCALE_MAD)
        return fail(UMI_ERR_INVALID_ARG, "scale_mode must be UMI_SCALE_UPPER_RMS or UMI_SCALE_MAD");
    *out = q;
    return UMI_OK;
}

static std::mutex g_attr_mu;

// ---------------------------------------------------------- checked build --
// Builds compiled with UMI_CHECKED give every launch a device flag word (one
// per device, allocated by prepare_kernel, which runs before any launch or
// graph capture); the kernel sets a bit for each failed index check and skips
// the access.  Normal builds pass no word and compile no checks.
#ifdef UMI_CHECKED
static std::mutex g_check_mu;
static std::map<int, uint32_t *> g_check_words;

static uint32_t *check_word()
{
    std::lock_guard<std::mutex> lk(g_check_mu);
    auto it = g_check_words.find(current_device());
    return it == g_check_words.end() ? nullptr : it->second;
}

static umi_status ensure_check_word()
{
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_check_mu);
    if (g_check_words.count(dev)) return UMI_OK;
    uint32_t *w = nullptr;
    UMI_CUDA(cudaMalloc((void **)&w, sizeof(uint32_t)), "cudaMalloc (check flags)");
    UMI_CUDA(cudaMemset(w, 0, sizeof(uint32_t)), "cudaMemset (check flags)");
    g_check_words[dev] = w;
    return UMI_OK;
}
#else
static uint32_t *check_word() { return nullptr; }
static umi_status ensure_check_word() { return UMI_OK; }
#endif

umi_status prepare_kernel(const Plan &plan, int flavour)
{
    int n = 0;
    const Variant *t = variant_table(&n);
    if (plan.variant < 0 || plan.variant >= n) return fail(UMI_ERR_INVALID_ARG, "bad plan");
    {
        const umi_status cst = ensure_check_word();
        if (cst != UMI_OK) return cst;
    }
    const size_t smem = plan.smem_bytes();
    const DeviceInfo &di = device_info(current_device());
    if (smem > di.smem_optin)
        return fail(UMI_ERR_INVALID_ARG, "tile needs more shared memory than the device allows");
    if (smem > 48 * 1024) {
        std::lock_guard<std::mutex> lk(g_attr_mu);
        const void *k = t[plan.variant].kernel[flavour];
        UMI_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                 "cudaFuncSetAttribute");
    }
    return UMI_OK;
}

int persistent_grid(const Plan &plan, int flavour)
{
    int n = 0;
    const Variant *t = variant_table(&n);
    const void *k = t[plan.variant].kernel[flavour];
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, plan.threads, plan.smem_bytes()) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int sms = std::max(1, device_info(current_device()).sms);
    return sms * per_sm;
}

static Curve make_curve(const float *flux, float *trend, float *detr, int64_t n, int W,
                        const umi_params &p)
{
    Curve c;
    c.flux = flux;
    c.trend = trend;
    c.detr = detr;
    c.n = n;
    c.W = W;
    c.min_valid = resolve_min_valid(W, p.min_valid);
    c.alpha = p.alpha;
    c.c = p.c;
    c.iters = p.iters;
    c.scale_mode = p.scale_mode;
    return c;
}

// -------------------------------------------------------- single curve --
umi_status launch_single_curve(const Curve &c, int64_t plan_positions, const Diag *diag,
                               cudaStream_t stream, int *launches)
{
    if (launches) *launches = 0;
    if (c.n <= 0) return UMI_OK;
    Plan plan;
    umi_status st = make_plan(c.W, plan_positions, &plan);
    if (st != UMI_OK) return st;
    const int flavour = (diag ? kFlagDiag : 0) | (c.scale_mode == UMI_SCALE_MAD ? kFlagMad : 0);
    st = prepare_kernel(plan, flavour);
    if (st != UMI_OK) return st;
    const int64_t T = plan.tile();
    const int64_t items = (c.n + T - 1) / T;
    if (items > INT32_MAX) return fail(UMI_ERR_INVALID_ARG, "curve too long");
    LaunchArgs a;
    memset(&a, 0, sizeof(a));
    a.curves = nullptr;
    a.single = c;
    a.items = nullptr;
    a.n_items = (int32_t)items;
    a.chain = plan.chain;
    a.queue = nullptr;
    if (diag) a.diag = *diag;
    a.n_curves = 0;
    a.check = check_word();
    int nv = 0;
    const Variant *t = variant_table(&nv);
    LaunchFn fn = t[plan.variant].launch[flavour];
    const int warps = plan.threads / 32;
    const int64_t grid = (items + warps - 1) / warps;
    cudaError_t e = fn(a, (int)grid, plan.threads, plan.smem_bytes(), stream);
    if (e != cudaSuccess) return fail_cuda(e, "kernel launch");
    if (launches) *launches = 1;
    return UMI_OK;
}

static umi_status detrend_single(const float *flux, int64_t n, int32_t W, const umi_params *params,
                                 float *trend, float *detr, const Diag *diag, cudaStream_t stream)
{
    NvtxRange nvtx("umi detrend");
    clear_error();
    umi_params p;
    umi_status st = check_params(params, &p);
    if (st != UMI_OK) return st;
    if (n < 0) return fail(UMI_ERR_INVALID_ARG, "n must be >= 0");
    if (W < 1 || (W % 2) == 0 || W > kMaxWindow)
        return fail(UMI_ERR_INVALID_ARG, "W must be odd and in [1, " + std::to_string(kMaxWindow) + "]");
    if (n == 0) return UMI_OK;
    if (!flux || !trend || !detr) return fail(UMI_ERR_INVALID_ARG, "null buffer");
    return launch_single_curve(make_curve(flux, trend, detr, n, W, p), n, diag, stream, nullptr);
}

// ------------------------------------------------------------- batches --
umi_status build_layout(const std::vector<Curve> &curves, BatchLayout *layout,
                        const BandSizes *plan_sizes)
{
    int nvar = 0;
    variant_table(&nvar);
    // One band per distinct plan (variant, chain, threads), in descending
    // slot capacity so that the heaviest tiles start first.
    // Positions per (window length, scale mode) size each band's plan
    // (make_plan): a small band gets a latency plan and shorter chains so that
    // its work still spreads over the whole GPU.
    BandSizes band_positions;
    for (const Curve &c : curves)
        band_positions[std::make_pair(c.W, c.scale_mode)] += c.n;
    if (plan_sizes)
        for (auto &kv : band_positions) {
            auto it = plan_sizes->find(kv.first);
            if (it != plan_sizes->end()) kv.second = std::max(kv.second, it->second);
        }
    std::map<std::tuple<int, int, int, int, int>, std::vector<int>> by_plan;
    std::vector<Plan> plans;
    for (size_t b = 0; b < curves.size(); ++b) {
        Plan p;
        umi_status st =
            make_plan(curves[b].W, band_positions[std::make_pair(curves[b].W, curves[b].scale_mode)], &p);
        if (st != UMI_OK) return st;
        const int flavour = curves[b].scale_mode == UMI_SCALE_MAD ? kFlagMad : 0;
        by_plan[std::make_tuple(-p.G * p.R, p.variant, p.chain, p.threads, flavour)].push_back((int)b);
        plans.push_back(p);
    }
    layout->bands.clear();
    layout->items.clear();
    layout->n_curves = (int32_t)curves.size();
    for (auto &kv : by_plan) {
        BatchLayout::Band band;
        band.plan = plans[kv.second.front()];
        band.flavour = std::get<4>(kv.first);
        band.first_item = (int32_t)layout->items.size();
        const int64_t T = band.plan.tile();
        // Longest curves first: their tiles are interleaved with others by the
        // queue anyway, but this keeps the tail short.
        std::vector<int> order = kv.second;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return curves[a].n > curves[b].n; });
        for (int b : order) {
            const int64_t tiles = (curves[b].n + T - 1) / T;
            for (int64_t k = 0; k < tiles; ++k) {
                if (layout->items.size() >= (size_t)INT32_MAX)
                    return fail(UMI_ERR_INVALID_ARG, "too many work items");
                layout->items.push_back(Item{(int32_t)b, (int32_t)k});
            }
        }
        band.n_items = (int32_t)layout->items.size() - band.first_item;
        if (band.n_items > 0) layout->bands.push_back(band);
    }
    return UMI_OK;
}

// Device scratch for one batch: [curve table][items][one counter per band].
struct Scratch {
    size_t curve_off = 0, item_off = 0, counter_off = 0, bytes = 0;
};

static Scratch scratch_layout(size_t n_curves, size_t n_items, size_t n_bands)
{
    Scratch s;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    s.curve_off = 0;
    s.item_off = up(n_curves * sizeof(Curve));
    s.counter_off = s.item_off + up(n_items * sizeof(Item));
    s.bytes = s.counter_off + up(std::max<size_t>(1, n_bands) * sizeof(int32_t));
    return s;
}

static umi_status enqueue_bands(const BatchLayout &lay, char *dev, const Scratch &sc,
                                cudaStream_t stream, int *launches)
{
    int nv = 0;
    const Variant *t = variant_table(&nv);
    UMI_CUDA(cudaMemsetAsync(dev + sc.counter_off, 0, lay.bands.size() * sizeof(int32_t), stream),
             "cudaMemsetAsync");
    int count = 0;
    for (size_t k = 0; k < lay.bands.size(); ++k) {
        const BatchLayout::Band &band = lay.bands[k];
        LaunchArgs a;
        memset(&a, 0, sizeof(a));
        a.curves = reinterpret_cast<const Curve *>(dev + sc.curve_off);
        a.items = reinterpret_cast<const Item *>(dev + sc.item_off) + band.first_item;
        a.n_items = band.n_items;
        a.chain = band.plan.chain;
        a.queue = reinterpret_cast<int32_t *>(dev + sc.counter_off) + k;
        a.n_curves = lay.n_curves;
        a.check = check_word();
        const int warps = band.plan.threads / 32;
        const int grid =
            std::min((band.n_items + warps - 1) / warps, persistent_grid(band.plan, band.flavour));
        cudaError_t e = t[band.plan.variant].launch[band.flavour](a, grid, band.plan.threads,
                                                                  band.plan.smem_bytes(), stream);
        if (e != cudaSuccess) return fail_cuda(e, "kernel launch");
        ++count;
    }
    if (launches) *launches = count;
    return UMI_OK;
}

umi_status prepare_batch(const std::vector<Curve> &curves, PreparedBatch *pb)
{
    umi_status st = build_layout(curves, &pb->layout);
    if (st != UMI_OK) return st;
    for (const auto &band : pb->layout.bands) {
        st = prepare_kernel(band.plan, band.flavour);
        if (st != UMI_OK) return st;
    }
    const Scratch sc = scratch_layout(curves.size(), pb->layout.items.size(), pb->layout.bands.size());
    pb->curve_off = sc.curve_off;
    pb->item_off = sc.item_off;
    pb->counter_off = sc.counter_off;
    pb->dev_bytes = sc.bytes;
    pb->host_bytes = sc.counter_off;
    return UMI_OK;
}

umi_status enqueue_prepared(const std::vector<Curve> &curves, const PreparedBatch &pb, char *dev,
                            char *host, cudaStream_t stream, int *launches)
{
    if (launches) *launches = 0;
    if (pb.layout.items.empty()) return UMI_OK;
    memcpy(host + pb.curve_off, curves.data(), curves.size() * sizeof(Curve));
    memcpy(host + pb.item_off, pb.layout.items.data(), pb.layout.items.size() * sizeof(Item));
    UMI_CUDA(cudaMemcpyAsync(dev, host, pb.host_bytes, cudaMemcpyHostToDevice, stream), "cudaMemcpyAsync");
    Scratch sc;
    sc.curve_off = pb.curve_off;
    sc.item_off = pb.item_off;
    sc.counter_off = pb.counter_off;
    sc.bytes = pb.dev_bytes;
    return enqueue_bands(pb.layout, dev, sc, stream, launches);
}

// Pinned host staging for work-queue tables: a ring of a few buffers per
// host thread.  A copy from pageable memory would make CUDA wait for all
// earlier work on the stream first; from pinned memory it is enqueued
// asynchronously.  Each buffer carries an event recorded after its copy, and
// is reused only once that event has completed (normally long since).
namespace {
struct PinnedSlot {
    char *p = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
};
constexpr int kPinnedSlots = 4;
thread_local PinnedSlot t_pinned[kPinnedSlots];  // intentionally never freed
thread_local int t_pinned_next = 0;
}  // namespace

static umi_status acquire_pinned(size_t bytes, int *slot, char **out)
{
    const int k = t_pinned_next;
    t_pinned_next = (k + 1) % kPinnedSlots;
    PinnedSlot &ps = t_pinned[k];
    if (ps.pending) {
        UMI_CUDA(cudaEventSynchronize(ps.ev), "cudaEventSynchronize (staging)");
        ps.pending = false;
    }
    if (!ps.ev) UMI_CUDA(cudaEventCreateWithFlags(&ps.ev, cudaEventDisableTiming), "cudaEventCreate");
    if (ps.cap < bytes) {
        if (ps.p) cudaFreeHost(ps.p);
        ps.p = nullptr;
        ps.cap = 0;
        const size_t cap = std::max<size_t>(bytes, 64 << 10);
        UMI_CUDA(cudaMallocHost((void **)&ps.p, cap), "cudaMallocHost (staging)");
        ps.cap = cap;
    }
    *slot = k;
    *out = ps.p;
    return UMI_OK;
}

static void release_pinned(int slot, cudaStream_t stream)
{
    PinnedSlot &ps = t_pinned[slot];
    if (cudaEventRecord(ps.ev, stream) == cudaSuccess) {
        ps.pending = true;
    } else {
        // The event belongs to another device than this stream: fall back to
        // waiting for the copy here, which keeps the buffer safe to reuse.
        cudaGetLastError();
        cudaStreamSynchronize(stream);
    }
}

// The entry points take their device scratch with cudaMallocAsync from the
// device's default memory pool.  Its release threshold is raised once per
// device, so that freed blocks stay in the pool for the next call instead of
// being unmapped at every synchronisation (with the default threshold of 0 the
// host entry point's 216 MB buffer for 1000 curves of 18,000 samples was
// mapped again on every call).  The pool then keeps up to the largest scratch
// a call has taken.
void keep_pool_memory()
{
    static std::mutex mu;
    static std::vector<int> done;
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done.push_back(dev);
}

// Side streams and events of the pipelined host entry point, per host thread
// and device, created on first use and kept (never freed).
namespace {
struct HostPipe {
    cudaStream_t s_in = nullptr, s_out = nullptr, s_c2 = nullptr;
    std::vector<cudaEvent_t> events;
};
thread_local std::map<int, HostPipe> t_pipes;  // intentionally never freed
}  // namespace

static cudaError_t host_pipe(int dev, HostPipe **out)
{
    HostPipe &hp = t_pipes[dev];
    cudaError_t e = cudaSuccess;
    if (!hp.s_in) e = cudaStreamCreateWithFlags(&hp.s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !hp.s_out) e = cudaStreamCreateWithFlags(&hp.s_out, cudaStreamNonBlocking);
    if (e == cudaSuccess && !hp.s_c2) e = cudaStreamCreateWithFlags(&hp.s_c2, cudaStreamNonBlocking);
    *out = &hp;
    return e;
}

umi_status launch_curve_table(const std::vector<Curve> &curves, cudaStream_t stream, int *launches,
                              const BandSizes *plan_sizes)
{
    if (launches) *launches = 0;
    if (curves.empty()) return UMI_OK;
    if (curves.size() == 1) {
        // One curve needs no work-queue tables: nothing is copied to the
        // device before the kernel.  The plan is the one-curve band's.
        int64_t P = curves[0].n;
        if (plan_sizes) {
            auto it = plan_sizes->find(std::make_pair(curves[0].W, curves[0].scale_mode));
            if (it != plan_sizes->end()) P = std::max(P, it->second);
        }
        return launch_single_curve(curves[0], P, nullptr, stream, launches);
    }
    BatchLayout lay;
    umi_status st = build_layout(curves, &lay, plan_sizes);
    if (st != UMI_OK) return st;
    if (lay.items.empty()) return UMI_OK;
    for (const auto &band : lay.bands) {
        st = prepare_kernel(band.plan, band.flavour);
        if (st != UMI_OK) return st;
    }
    const Scratch sc = scratch_layout(curves.size(), lay.items.size(), lay.bands.size());
    keep_pool_memory();
    // Host staging in one pinned block so a single asynchronous copy moves the tables.
    int slot = 0;
    char *host = nullptr;
    st = acquire_pinned(sc.counter_off, &slot, &host);
    if (st != UMI_OK) return st;
    memcpy(host + sc.curve_off, curves.data(), curves.size() * sizeof(Curve));
    memcpy(host + sc.item_off, lay.items.data(), lay.items.size() * sizeof(Item));
    void *dev = nullptr;
    UMI_CUDA(cudaMallocAsync(&dev, sc.bytes, stream), "cudaMallocAsync");
    cudaError_t e = cudaMemcpyAsync(dev, host, sc.counter_off, cudaMemcpyHostToDevice, stream);
    release_pinned(slot, stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(dev, stream);
        return fail_cuda(e, "cudaMemcpyAsync");
    }
    st = enqueue_bands(lay, (char *)dev, sc, stream, launches);
    cudaError_t ef = cudaFreeAsync(dev, stream);
    if (st != UMI_OK) return st;
    if (ef != cudaSuccess) return fail_cuda(ef, "cudaFreeAsync");
    return UMI_OK;
}

// ---------------------------------------------------- CUDA-graph cache --
// Equal-shaped batches (same buffers, offsets, windows and parameters)
// replay a captured graph whose work-queue tables live in persistent device
// memory, so the steady state costs one graph launch and no host planning.
struct GraphEntry {
    uint64_t key = 0;
    std::vector<int64_t> offsets;
    std::vector<int32_t> W;
    const float *flux = nullptr;
    float *trend = nullptr, *detr = nullptr;
    umi_params params{};
    int device = -1;
    uint64_t tune_epoch = 0;
    void *dev = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

static std::mutex g_graph_mu;
static std::list<GraphEntry> g_graphs;  // most recent first
static std::atomic<int> g_graph_enabled{1};
static const size_t kMaxGraphs = 8;

static uint64_t fnv1a(const void *data, size_t n, uint64_t h)
{
    const unsigned char *p = (const unsigned char *)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

static void destroy_entry(GraphEntry &g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.dev) cudaFree(g.dev);  // synchronises with prior work using it
    g.exec = nullptr;
    g.dev = nullptr;
}

static umi_status build_graph(const std::vector<Curve> &curves, GraphEntry *g)
{
    NvtxRange nvtx("umi graph capture");
    BatchLayout lay;
    umi_status st = build_layout(curves, &lay);
    if (st != UMI_OK) return st;
    for (const auto &band : lay.bands) {
        st = prepare_kernel(band.plan, band.flavour);
        if (st != UMI_OK) return st;
    }
    // Batches of two or more curves only (one curve launches directly).
    const Scratch sc = scratch_layout(curves.size(), lay.items.size(), lay.bands.size());
    {
        std::vector<char> host(sc.counter_off);
        memcpy(host.data() + sc.curve_off, curves.data(), curves.size() * sizeof(Curve));
        if (!lay.items.empty())
            memcpy(host.data() + sc.item_off, lay.items.data(), lay.items.size() * sizeof(Item));
        UMI_CUDA(cudaMalloc(&g->dev, sc.bytes), "cudaMalloc (graph tables)");
        UMI_CUDA(cudaMemcpy(g->dev, host.data(), sc.counter_off, cudaMemcpyHostToDevice), "cudaMemcpy");
    }
    cudaStream_t cs;
    UMI_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail_cuda(e, "cudaStreamBeginCapture");
    }
    umi_status est = enqueue_bands(lay, (char *)g->dev, sc, cs, &g->launches);
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (est != UMI_OK) {
        if (graph) cudaGraphDestroy(graph);
        return est;
    }
    if (e != cudaSuccess) return fail_cuda(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGraphInstantiate");
    return UMI_OK;
}

static std::atomic<long long> g_kernel_launches{0};

void count_launches(int n) { g_kernel_launches += n; }

static umi_status batched_impl(const float *flux, const int64_t *offsets, const int32_t *W,
                               int32_t B, const umi_params *params, float *trend, float *detr,
                               cudaStream_t stream, bool allow_graph,
                               const BandSizes *plan_sizes = nullptr)
{
    NvtxRange nvtx("umi detrend batched");
    clear_error();
    umi_params p;
    umi_status st = check_params(params, &p);
    if (st != UMI_OK) return st;
    if (B < 0) return fail(UMI_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return UMI_OK;
    if (!offsets || !W) return fail(UMI_ERR_INVALID_ARG, "null offsets or W");
    if (offsets[0] != 0) return fail(UMI_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int32_t b = 0; b < B; ++b) {
        if (offsets[b + 1] < offsets[b]) return fail(UMI_ERR_INVALID_ARG, "offsets must be non-decreasing");
        if (W[b] < 1 || (W[b] % 2) == 0 || W[b] > kMaxWindow)
            return fail(UMI_ERR_INVALID_ARG, "W[" + std::to_string(b) + "] must be odd and in [1, " +
                                                 std::to_string(kMaxWindow) + "]");
    }
    if (offsets[B] == 0) return UMI_OK;
    if (!flux || !trend || !detr) return fail(UMI_ERR_INVALID_ARG, "null buffer");
    std::vector<Curve> curves;
    curves.reserve(B);
    for (int32_t b = 0; b < B; ++b) {
        const int64_t o = offsets[b], n = offsets[b + 1] - offsets[b];
        if (n == 0) continue;
        curves.push_back(make_curve(flux + o, trend + o, detr + o, n, W[b], p));
    }
    // One curve launches directly: it needs no device tables, and a graph
    // holding its one kernel costs about 1 us more on the GPU than a launch.
    if (!allow_graph || plan_sizes || !g_graph_enabled.load() || curves.size() == 1) {
        int launches = 0;
        st = launch_curve_table(curves, stream, &launches, plan_sizes);
        g_kernel_launches += launches;
        return st;
    }
    const int dev = current_device();
    const uint64_t epoch = tune_epoch();
    uint64_t key = 1469598103934665603ull;
    key = fnv1a(&epoch, sizeof(epoch), key);
    key = fnv1a(offsets, sizeof(int64_t) * (B + 1), key);
    key = fnv1a(W, sizeof(int32_t) * B, key);
    key = fnv1a(&p, sizeof(p), key);
    key = fnv1a(&flux, sizeof(flux), key);
    key = fnv1a(&trend, sizeof(trend), key);
    key = fnv1a(&detr, sizeof(detr), key);
    key = fnv1a(&dev, sizeof(dev), key);
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
        GraphEntry &g = *it;
        if (g.key != key || g.device != dev || g.tune_epoch != epoch || g.flux != flux ||
            g.trend != trend || g.detr != detr ||
            (int32_t)g.W.size() != B || memcmp(&g.params, &p, sizeof(p)) != 0 ||
            memcmp(g.offsets.data(), offsets, sizeof(int64_t) * (B + 1)) != 0 ||
            memcmp(g.W.data(), W, sizeof(int32_t) * B) != 0)
            continue;
        UMI_CUDA(cudaGraphLaunch(g.exec, stream), "cudaGraphLaunch");
        g_kernel_launches += g.launches;
        g_graphs.splice(g_graphs.begin(), g_graphs, it);
        return UMI_OK;
    }
    GraphEntry g;
    g.key = key;
    g.offsets.assign(offsets, offsets + B + 1);
    g.W.assign(W, W + B);
    g.flux = flux;
    g.trend = trend;
    g.detr = detr;
    g.params = p;
    g.device = dev;
    g.tune_epoch = epoch;
    st = build_graph(curves, &g);
    if (st != UMI_OK) {
        destroy_entry(g);
        return st;
    }
    cudaError_t e = cudaGraphLaunch(g.exec, stream);
    if (e != cudaSuccess) {
        destroy_entry(g);
        return fail_cuda(e, "cudaGraphLaunch");
    }
    g_kernel_launches += g.launches;
    g_graphs.push_front(std::move(g));
    while (g_graphs.size() > kMaxGraphs) {
        destroy_entry(g_graphs.back());
        g_graphs.pop_back();
    }
    return UMI_OK;
}

// ------------------------------------------------------------ autotuner --
__global__ void fill_noise_kernel(float *x, int64_t n, uint64_t seed)
{
    // Flux-like samples 1 + N(0, 1e-3) from a counter-based hash (SplitMix64)
    // and Box-Muller; only used to time kernels.
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9e3779b97f4a7c15ull * (uint64_t)(i + 1);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        const float u1 = ((z >> 40) + 1) * (1.0f / 16777217.0f);
        const float u2 = ((z & 0xffffffu)) * (1.0f / 16777216.0f);
        x[i] = 1.0f + 1e-3f * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    }
}

// Times one plan on consecutive curves of the given lengths (one band, one
// launch per run), the way a batch of such curves runs.
static umi_status time_plan(const Plan &plan, const float *flux, float *trend, float *detr,
                            const std::vector<int64_t> &lengths, int W, cudaStream_t stream, double *ms)
{
    umi_params p;
    umi_default_params(&p);
    std::vector<Curve> curves;
    int64_t o = 0;
    for (int64_t n : lengths) {
        curves.push_back(make_curve(flux + o, trend + o, detr + o, n, W, p));
        o += n;
    }
    BatchLayout lay;
    lay.n_curves = (int32_t)curves.size();
    lay.bands.resize(1);
    lay.bands[0].plan = plan;
    lay.bands[0].first_item = 0;
    const int64_t T = plan.tile();
    for (size_t c = 0; c < lengths.size(); ++c) {
        const int64_t tiles = (lengths[c] + T - 1) / T;
        for (int64_t k = 0; k < tiles; ++k) lay.items.push_back(Item{(int32_t)c, (int32_t)k});
    }
    lay.bands[0].n_items = (int32_t)lay.items.size();
    umi_status st = prepare_kernel(plan, 0);
    if (st != UMI_OK) return st;
    const Scratch sc = scratch_layout(curves.size(), lay.items.size(), 1);
    std::vector<char> host(sc.counter_off);
    memcpy(host.data() + sc.curve_off, curves.data(), curves.size() * sizeof(Curve));
    memcpy(host.data() + sc.item_off, lay.items.data(), lay.items.size() * sizeof(Item));
    void *dev = nullptr;
    UMI_CUDA(cudaMalloc(&dev, sc.bytes), "cudaMalloc");
    UMI_CUDA(cudaMemcpy(dev, host.data(), sc.counter_off, cudaMemcpyHostToDevice), "cudaMemcpy");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // Every launch is timed alone (events around it, the host waiting for
    // it), as one call runs.  The first run warms up and the second sizes
    // the timed runs: a plan that takes microseconds (one curve) is near the
    // event timer's resolution, so a run repeats it for about a millisecond
    // and counts the mean; the best of three timed runs is the plan's time.
    double best = 1e30;
    int reps_per_run = 1;
    for (int run = 0; run < 5 && st == UMI_OK; ++run) {
        double sum = 0.0;
        for (int r = 0; r < reps_per_run && st == UMI_OK; ++r) {
            cudaEventRecord(e0, stream);
            st = enqueue_bands(lay, (char *)dev, sc, stream, nullptr);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(UMI_ERR_CUDA, "autotune run failed");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            sum += t;
        }
        const double mean = sum / reps_per_run;
        if (run == 1) reps_per_run = (int)std::min(64.0, std::max(1.0, std::floor(1.0 / std::max(mean, 1e-3))));
        if (run >= 2) best = std::min(best, mean);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dev);
    *ms = best;
    return st;
}

// ------------------------------------------------ allocation-free batch --
// The work-queue tables of umi_detrend_batched_noalloc live in this fixed
// array instead of stream-ordered allocations.  Host code must not pass the
// array's name to a kernel (on the host it names a shadow variable); it looks
// up the device address once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[UMI_NOALLOC_SCRATCH_BYTES];

// The tables reach the array inside kernel parameters: a launch copies its
// parameters by value when it is enqueued, so the host's table buffer may be
// freed at once and the call never waits for the stream (a cudaMemcpyAsync
// from pageable memory may wait for all earlier work on the stream), and no
// pinned staging buffer has to be allocated.  One chunk is just under the
// 32,764-byte parameter limit of sm_70 and later GPUs.
constexpr uint32_t kTableChunkWords = 8000;

struct TableChunk {
    uint32_t off_words;  // destination, in 4-byte words from the array's start
    uint32_t n_words;    // words of `w` to copy, <= kTableChunkWords
    uint32_t w[kTableChunkWords];
};

__global__ void noalloc_write_tables(uint32_t *dst, const TableChunk c)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < c.n_words; i += gridDim.x * blockDim.x)
        dst[c.off_words + i] = c.w[i];
}

static std::mutex g_noalloc_mu;
static std::map<int, void *> g_noalloc_addr;  // device ordinal -> address of the array

static umi_status noalloc_scratch_address(void **out)
{
    const int dev = current_device();
    if (dev < 0) return fail(UMI_ERR_CUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) {
        *out = it->second;
        return UMI_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress (no-alloc scratch)");
    g_noalloc_addr[dev] = p;
    *out = p;
    return UMI_OK;
}

static umi_status noalloc_batched(const float *flux, const int64_t *offsets, const int32_t *W,
                                  int32_t B, const umi_params *params, float *trend, float *detr,
                                  cudaStream_t stream)
{
    NvtxRange nvtx("umi detrend batched noalloc");
    clear_error();
    umi_params p;
    umi_status st = check_params(params, &p);
    if (st != UMI_OK) return st;
    if (B < 0) return fail(UMI_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return UMI_OK;
    if (!offsets || !W) return fail(UMI_ERR_INVALID_ARG, "null offsets or W");
    if (offsets[0] != 0) return fail(UMI_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int32_t b = 0; b < B; ++b) {
        if (offsets[b + 1] < offsets[b]) return fail(UMI_ERR_INVALID_ARG, "offsets must be non-decreasing");
        if (W[b] < 1 || (W[b] % 2) == 0 || W[b] > kMaxWindow)
            return fail(UMI_ERR_INVALID_ARG, "W[" + std::to_string(b) + "] must be odd and in [1, " +
                                                 std::to_string(kMaxWindow) + "]");
    }
    if (offsets[B] == 0) return UMI_OK;
    if (!flux || !trend || !detr) return fail(UMI_ERR_INVALID_ARG, "null buffer");
    std::vector<Curve> curves;
    curves.reserve(B);
    for (int32_t b = 0; b < B; ++b) {
        const int64_t o = offsets[b], n = offsets[b + 1] - offsets[b];
        if (n == 0) continue;
        curves.push_back(make_curve(flux + o, trend + o, detr + o, n, W[b], p));
    }
    BatchLayout lay;
    st = build_layout(curves, &lay);
    if (st != UMI_OK) return st;
    if (lay.items.empty()) return UMI_OK;
    const Scratch sc = scratch_layout(curves.size(), lay.items.size(), lay.bands.size());
    if (sc.bytes > UMI_NOALLOC_SCRATCH_BYTES)
        return fail(UMI_ERR_INVALID_ARG,
                    "batch needs " + std::to_string(sc.bytes) + " bytes of work-queue tables, above the " +
                        std::to_string((size_t)UMI_NOALLOC_SCRATCH_BYTES) +
                        "-byte no-alloc scratch; split the batch");
    for (const auto &band : lay.bands) {
        st = prepare_kernel(band.plan, band.flavour);
        if (st != UMI_OK) return st;
    }
    void *dev = nullptr;
    st = noalloc_scratch_address(&dev);
    if (st != UMI_OK) return st;
    // Host image of the tables (the scratch layout's offsets are multiples of
    // 256 bytes, so it is a whole number of words).
    std::vector<uint32_t> host(sc.counter_off / sizeof(uint32_t));
    memcpy((char *)host.data() + sc.curve_off, curves.data(), curves.size() * sizeof(Curve));
    memcpy((char *)host.data() + sc.item_off, lay.items.data(), lay.items.size() * sizeof(Item));
    // Stream-ordered after any earlier call's kernels on this stream.
    std::unique_ptr<TableChunk> chunk(new TableChunk);
    int writers = 0;
    for (size_t w0 = 0; w0 < host.size(); w0 += kTableChunkWords) {
        const uint32_t nw = (uint32_t)std::min<size_t>(kTableChunkWords, host.size() - w0);
        chunk->off_words = (uint32_t)w0;
        chunk->n_words = nw;
        memcpy(chunk->w, host.data() + w0, nw * sizeof(uint32_t));
        // The argument array points at the heap chunk, so the 32 KB parameter
        // is copied into the launch from there (no stack copy on the host).
        uint32_t *dst = (uint32_t *)dev;
        void *args[] = {&dst, chunk.get()};
        cudaError_t e = cudaLaunchKernel((const void *)noalloc_write_tables, dim3((nw + 255) / 256), dim3(256),
                                         args, 0, stream);
        if (e != cudaSuccess) return fail_cuda(e, "no-alloc table write");
        ++writers;
    }
    int launches = 0;
    st = enqueue_bands(lay, (char *)dev, sc, stream, &launches);  // clears the counters first
    g_kernel_launches += writers + launches;
    return st;
}

}  // namespace umi

using namespace umi;

// ================================================================== C ABI ==
extern "C" {

void umi_default_params(umi_params *p)
{
    if (!p) return;
    p->alpha = 2.0f;
    p->c = 5.0f;
    p->iters = 5;
    p->min_valid = -1;
    p->scale_mode = UMI_SCALE_UPPER_RMS;
}

int32_t umi_window_length(double cadence_days, double window_days)
{
    if (!(cadence_days > 0.0) || !(window_days > 0.0) || !std::isfinite(cadence_days) ||
        !std::isfinite(window_days))
        return -1;
    const double ratio = window_days / cadence_days;
    if (!(ratio <= 1e9)) return -1;
    const long long w = std::llround(ratio);
    return (int32_t)(w | 1LL);
}

int32_t umi_max_window(void) { return kMaxWindow; }

const char *umi_last_error(void) { return t_error.c_str(); }

const char *umi_version(void) { return "umi-gb300 0.1.0 (sm_103a)"; }

umi_status umi_detrend(const float *flux_d, int64_t n, int32_t W, const umi_params *params,
                       float *trend_d, float *detr_d, void *stream)
{
    umi_status st = detrend_single(flux_d, n, W, params, trend_d, detr_d, nullptr,
                                   (cudaStream_t)stream);
    if (st == UMI_OK && n > 0) g_kernel_launches += 1;
    return st;
}

umi_status umi_detrend_diag(const float *flux_d, int64_t n, int32_t W, const umi_params *params,
                            float *trend_d, float *detr_d, float *median_d, int32_t *nvalid_d,
                            int32_t *nplus_d, float *scale_d, void *stream)
{
    Diag d{median_d, nvalid_d, nplus_d, scale_d};
    umi_status st = detrend_single(flux_d, n, W, params, trend_d, detr_d, &d, (cudaStream_t)stream);
    if (st == UMI_OK && n > 0) g_kernel_launches += 1;
    return st;
}

umi_status umi_detrend_batched(const float *flux_d, const int64_t *offsets_h, const int32_t *W_h,
                               int32_t B, const umi_params *params, float *trend_d, float *detr_d,
                               void *stream)
{
    return batched_impl(flux_d, offsets_h, W_h, B, params, trend_d, detr_d, (cudaStream_t)stream,
                        true);
}

umi_status umi_detrend_batched_noalloc(const float *flux_d, const int64_t *offsets_h,
                                       const int32_t *W_h, int32_t B, const umi_params *params,
                                       float *trend_d, float *detr_d, void *stream)
{
    return noalloc_batched(flux_d, offsets_h, W_h, B, params, trend_d, detr_d, (cudaStream_t)stream);
}

umi_status umi_detrend_batched_host(const float *flux_h, const int64_t *offsets_h,
                                    const int32_t *W_h, int32_t B, const umi_params *params,
                                    float *trend_h, float *detr_h, void *stream)
{
    NvtxRange nvtx("umi detrend batched host");
    clear_error();
    if (B < 0 || (B > 0 && (!offsets_h || !W_h))) return fail(UMI_ERR_INVALID_ARG, "bad batch");
    if (B == 0) return UMI_OK;
    umi_params p;
    umi_status st = check_params(params, &p);
    if (st != UMI_OK) return st;
    if (offsets_h[0] != 0) return fail(UMI_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int32_t b = 0; b < B; ++b) {
        if (offsets_h[b + 1] < offsets_h[b]) return fail(UMI_ERR_INVALID_ARG, "offsets must be non-decreasing");
        if (W_h[b] < 1 || (W_h[b] % 2) == 0 || W_h[b] > kMaxWindow)
            return fail(UMI_ERR_INVALID_ARG, "W[" + std::to_string(b) + "] must be odd and in [1, " +
                                                 std::to_string(kMaxWindow) + "]");
    }
    const int64_t total = offsets_h[B];
    if (total == 0) return UMI_OK;
    if (!flux_h || !trend_h || !detr_h) return fail(UMI_ERR_INVALID_ARG, "null buffer");

    // Pipeline over chunks of curves: the copy-in of chunk c+1 and the
    // copy-out of chunk c-1 overlap the detrend of chunk c (copy engines and
    // SMs work at once; pinned host buffers make the copies asynchronous).
    const int64_t kChunkSamples = 1 << 20;
    const int K = (int)std::max<int64_t>(1, std::min<int64_t>({16, B, total / kChunkSamples}));
    std::vector<int32_t> cut(1, 0);
    for (int c = 1; c < K; ++c) {
        const int64_t target = total * c / K;
        int32_t b = (int32_t)(std::upper_bound(offsets_h, offsets_h + B + 1, target) - offsets_h) - 1;
        b = std::max(b, cut.back() + 1);
        if (b < B) cut.push_back(b);
    }
    cut.push_back(B);

    // Chunks alternate between the caller's stream and a second compute
    // stream, so the next chunk's persistent kernel fills SMs while the
    // previous one drains.  The side streams and the events belong to the
    // calling thread (HostPipe) and are reused by its next call: every use
    // of them has completed when a call returns.
    cudaStream_t s = (cudaStream_t)stream;
    HostPipe *hp = nullptr;
    cudaError_t e = host_pipe(current_device(), &hp);
    if (e != cudaSuccess) return fail_cuda(e, "batched host pipeline streams");
    cudaStream_t s_in = hp->s_in, s_out = hp->s_out, s_c2 = hp->s_c2;
    size_t n_ev = 0;
    auto new_event = [&](cudaEvent_t *out) {
        if (n_ev == hp->events.size()) {
            cudaEvent_t x = nullptr;
            cudaError_t ce = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
            if (ce != cudaSuccess) return ce;
            hp->events.push_back(x);
        }
        *out = hp->events[n_ev++];
        return cudaSuccess;
    };
    const size_t bytes = sizeof(float) * (size_t)total;
    float *dev = nullptr;
    keep_pool_memory();
    e = cudaMallocAsync((void **)&dev, 3 * bytes, s);
    cudaEvent_t ev_alloc = nullptr;
    if (e == cudaSuccess) e = new_event(&ev_alloc);
    if (e == cudaSuccess) e = cudaEventRecord(ev_alloc, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ev_alloc, 0);
    if (e != cudaSuccess) {
        if (dev) cudaFreeAsync(dev, s);
        cudaStreamSynchronize(s);
        return fail_cuda(e, "batched host pipeline setup");
    }
    float *dflux = dev, *dtrend = dev + total, *ddetr = dev + 2 * total;
    // Every chunk is planned from the whole call's bands.
    BandSizes sizes;
    for (int32_t b = 0; b < B; ++b)
        sizes[std::make_pair((int)W_h[b], p.scale_mode)] += offsets_h[b + 1] - offsets_h[b];
    std::vector<int64_t> off_c;
    for (size_t c = 0; c + 1 < cut.size() && st == UMI_OK; ++c) {
        const int32_t b0 = cut[c], b1 = cut[c + 1];
        const int64_t o = offsets_h[b0], n = offsets_h[b1] - o;
        cudaEvent_t ev_in = nullptr, ev_done = nullptr;
        e = new_event(&ev_in);
        if (e == cudaSuccess) e = new_event(&ev_done);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(dflux + o, flux_h + o, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, s_in);
        cudaStream_t cs = (c % 2 == 0) ? s : s_c2;
        if (e == cudaSuccess) e = cudaEventRecord(ev_in, s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in, 0);
        if (e != cudaSuccess) {
            st = fail_cuda(e, "cudaMemcpyAsync H2D");
            break;
        }
        off_c.assign(offsets_h + b0, offsets_h + b1 + 1);
        for (auto &x : off_c) x -= o;
        st = batched_impl(dflux + o, off_c.data(), W_h + b0, b1 - b0, &p, dtrend + o, ddetr + o, cs, false,
                          &sizes);
        if (st != UMI_OK) break;
        e = cudaEventRecord(ev_done, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev_done, 0);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(trend_h + o, dtrend + o, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s_out);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(detr_h + o, ddetr + o, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s_out);
        if (e != cudaSuccess) st = fail_cuda(e, "cudaMemcpyAsync D2H");
    }
    // The caller's stream waits for every copy and the second compute
    // stream, then frees the buffers.
    cudaEvent_t ev_out = nullptr, ev_c2 = nullptr;
    if (new_event(&ev_out) == cudaSuccess && new_event(&ev_c2) == cudaSuccess) {
        cudaEventRecord(ev_out, s_out);
        cudaEventRecord(ev_c2, s_c2);
        cudaStreamWaitEvent(s, ev_out, 0);
        cudaStreamWaitEvent(s, ev_c2, 0);
    } else {
        cudaStreamSynchronize(s_out);
        cudaStreamSynchronize(s_c2);
    }
    cudaStreamSynchronize(s_in);
    cudaFreeAsync(dev, s);
    e = cudaStreamSynchronize(s);
    if (st == UMI_OK && e != cudaSuccess) st = fail_cuda(e, "cudaStreamSynchronize");
    return st;
}

// `flux` holds the curves back to back, or is null for synthetic flux-like
// noise.
static umi_status autotune_impl(int32_t W, const float *flux, const std::vector<int64_t> &lengths,
                                void *stream, umi_plan *best_out, double *best_ms)
{
    if (W < 1 || (W % 2) == 0 || W > kMaxWindow) return fail(UMI_ERR_INVALID_ARG, "bad W");
    int64_t positions = 0;
    for (int64_t n : lengths) {
        if (n < 1 || n > ((int64_t)1 << 31) - positions) return fail(UMI_ERR_INVALID_ARG, "bad positions");
        positions += n;
    }
    if (positions < 1) return fail(UMI_ERR_INVALID_ARG, "bad positions");
    cudaStream_t s = (cudaStream_t)stream;
    float *buf = nullptr;
    UMI_CUDA(cudaMalloc((void **)&buf, (flux ? 2 : 3) * sizeof(float) * (size_t)positions), "cudaMalloc");
    float *out = flux ? buf : buf + positions;  // trend, then detr
    if (!flux) {
        fill_noise_kernel<<<1024, 256, 0, s>>>(buf, positions, 0x5eedull + (uint64_t)W);
        flux = buf;
    }
    std::vector<std::pair<double, Plan>> timed;
    umi_status st = UMI_OK;
    for (const Plan &p : autotune_candidates(W, positions)) {
        if (p.smem_bytes() > device_info(current_device()).smem_optin) continue;
        double ms = 0;
        st = time_plan(p, flux, out, out + positions, lengths, W, s, &ms);
        if (st != UMI_OK) break;
        timed.emplace_back(ms, p);
    }
    // Near-ties are timed again: the (at most six) choices within 3 % of the
    // fastest run three more rounds, interleaved, and each keeps the best of
    // all its runs, so that a difference below the run-to-run noise does not
    // decide alone.
    using Timed = std::pair<double, Plan>;
    std::stable_sort(timed.begin(), timed.end(),
                     [](const Timed &a, const Timed &b) { return a.first < b.first; });
    size_t close = 0;
    while (st == UMI_OK && close < timed.size() && close < 6 &&
           timed[close].first <= 1.03 * timed[0].first)
        ++close;
    for (int round = 0; round < 3 && st == UMI_OK && close > 1; ++round)
        for (size_t i = 0; i < close && st == UMI_OK; ++i) {
            double ms = 0;
            st = time_plan(timed[i].second, flux, out, out + positions, lengths, W, s, &ms);
            timed[i].first = std::min(timed[i].first, ms);
        }
    cudaFree(buf);
    if (st != UMI_OK) return st;
    if (timed.empty()) return fail(UMI_ERR_INVALID_ARG, "no eligible variant");
    size_t b = 0;
    for (size_t i = 1; i < close; ++i)
        if (timed[i].first < timed[b].first) b = i;
    const Plan best = timed[b].second;
    const double bms = timed[b].first;
    if (best.variant < 0) return fail(UMI_ERR_INVALID_ARG, "no eligible variant");
    store_tuned(W, best);
    if (best_out) plan_out(best, best_out);
    if (best_ms) *best_ms = bms;
    return UMI_OK;
}

umi_status umi_autotune(int32_t W, int64_t positions, void *stream, umi_plan *best_out,
                        double *best_ms)
{
    NvtxRange nvtx("umi autotune");
    clear_error();
    return autotune_impl(W, nullptr, std::vector<int64_t>{positions}, stream, best_out, best_ms);
}

umi_status umi_autotune_batch(int32_t W, const float *flux_d, const int64_t *curve_len_h, int32_t n_curves,
                              void *stream, umi_plan *best_out, double *best_ms)
{
    NvtxRange nvtx("umi autotune batch");
    clear_error();
    if (!curve_len_h || n_curves < 1) return fail(UMI_ERR_INVALID_ARG, "bad curve lengths");
    return autotune_impl(W, flux_d, std::vector<int64_t>(curve_len_h, curve_len_h + n_curves), stream,
                         best_out, best_ms);
}

void umi_set_graph_cache(int enabled)
{
    g_graph_enabled.store(enabled ? 1 : 0);
    if (!enabled) {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        for (auto &g : g_graphs) destroy_entry(g);
        g_graphs.clear();
    }
}

// Number of kernels this library has launched in the process (for reports).
long long umi_kernel_launch_count(void) { return g_kernel_launches.load(); }

int32_t umi_checked_build(void)
{
#ifdef UMI_CHECKED
    return 1;
#else
    return 0;
#endif
}

umi_status umi_check_flags(uint32_t *flags, int32_t clear)
{
    clear_error();
    if (!flags) return fail(UMI_ERR_INVALID_ARG, "null flags");
    *flags = 0;
#ifdef UMI_CHECKED
    UMI_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    uint32_t *w = check_word();
    if (!w) return UMI_OK;  // nothing has launched on this device yet
    UMI_CUDA(cudaMemcpy(flags, w, sizeof(uint32_t), cudaMemcpyDeviceToHost), "cudaMemcpy (check flags)");
    if (clear) UMI_CUDA(cudaMemset(w, 0, sizeof(uint32_t)), "cudaMemset (check flags)");
    return UMI_OK;
#else
    (void)clear;
    return fail(UMI_ERR_INVALID_ARG, "library built without UMI_CHECKED: no index checks ran");
#endif
}

}  // extern "C"
