/*
 * umi.h -- C ABI of libumi, the GB300 (sm_103a) implementation of UMI, the
 * sliding-window asymmetric robust trend of arXiv 2604.06602 ("UMI: A
 * GPU-Accelerated Asymmetric Robust Estimator for Photometric Detrending").
 *
 * What every detrend entry point computes (Section 2 of the paper):
 *   for each sample position j of a light curve x[0..n):
 *     window   the W samples x[j-h .. j+h], h = (W-1)/2, truncated at the ends
 *              of the curve; non-finite samples are missing and are dropped;
 *     Phase 1  m = exact median of the valid window samples (Section 2.1);
 *              for an even count the lower median, rank floor((n_valid-1)/2);
 *     Phase 2  s = 0.6745 * sqrt(mean over x > m of (x - m)^2)  (Eq. 1), or
 *              the MAD median |x - m| when params->scale_mode is UMI_SCALE_MAD;
 *     Phase 3  mu = m, then `iters` times: u = (x - mu)/(c s),
 *              u_eff = alpha u if u < 0 else u (Eq. 2),
 *              w = (1 - u_eff^2)^2 if |u_eff| < 1 else 0 (Eq. 3),
 *              mu <- sum(w x)/sum(w) (Eq. 4; mu kept if sum(w) == 0);
 *     output   trend[j] = mu, detr[j] = x[j] / mu.
 *   If no sample lies above m, or s == 0, the trend is m.  Positions whose
 *   own sample is missing, or whose window holds fewer than min_valid valid
 *   samples, get NaN in both outputs.
 *
 * Arithmetic: FP32 on the GPU.  Medians and the set of above-median samples
 * are exact (they are comparisons of the FP32 inputs); the trend agrees with
 * an FP64 evaluation of the same definition to about 1e-6 relative for
 * flux-like data.  Finite input samples must satisfy |x| < 2^60; larger
 * magnitudes overflow the FP32 sums of Eq. 1 and give unspecified results.
 *
 * Conventions for every call below:
 *   - `_d` pointers are CUDA device pointers (any allocator), `_h` pointers
 *     are host pointers.  All buffers stay owned by the caller.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *     is enqueued on it; the call returns without waiting for the GPU unless
 *     the entry point says otherwise.  Results are valid once the stream has
 *     reached the end of the enqueued work.
 *   - Arguments are validated on the host before anything is enqueued; an
 *     invalid argument returns UMI_ERR_INVALID_ARG and enqueues nothing.
 *     Errors are returned, never raised by abort().  umi_last_error() gives a
 *     message for the calling thread's most recent failure.
 *   - Calls are thread-safe.  Calls on different streams may overlap, except
 *     umi_detrend_batched_noalloc: all its calls share one device array, so
 *     they must be ordered on one stream (or otherwise serialised).
 *   - umi_detrend_batched, umi_detrend_batched_host and umi_detrend_segmented
 *     keep their own CUDA-graph cache and stage their work tables through
 *     reused pinned host buffers; do not capture them into a graph of your
 *     own (a captured table copy would not see the buffer's later contents).
 */
#ifndef UMI_H
#define UMI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    UMI_OK = 0,
    UMI_ERR_INVALID_ARG = 1,    /* an argument failed validation; nothing enqueued */
    UMI_ERR_CUDA = 2,           /* a CUDA runtime call failed (see umi_last_error) */
    UMI_ERR_OOM = 3,            /* device or host allocation failed */
    UMI_ERR_BUSY = 4,           /* server: the request can never fit the budget / slots */
    UMI_ERR_NOT_READY = 5,      /* server: the result is not finished yet */
    UMI_ERR_TIMEOUT = 6,        /* a bounded host-side wait ran out */
    UMI_ERR_UNKNOWN_TICKET = 7, /* server: no such ticket (never issued or released) */
    UMI_ERR_FAILED = 8          /* server: the request's batch failed; others unaffected */
} umi_status;

/* Estimator parameters (Section 2.3; presets in Section 4, Table 4). */
typedef struct {
    float alpha;       /* asymmetry of Eq. 2, > 0; 2.0 default (TESS), 3.0 Kepler,
                          1.0 symmetric biweight, 10.0 with c = 2.5 aggressive */
    float c;           /* tuning constant of the standardised residual, > 0; 5.0 */
    int32_t iters;     /* fixed number of Phase 3 iterations, >= 0; 5 */
    int32_t min_valid; /* minimum valid samples per window for an output; -1 means
                          floor(W/3) (the W/3 rule of Section 4, Kepler Long-Cadence);
                          0 disables the check */
    int32_t scale_mode; /* UMI_SCALE_UPPER_RMS (0, the method: Eq. 1) or UMI_SCALE_MAD
                           (1: s = median |x - m| over the window, the standard MAD the
                           paper compares against in Sections 1, 2.2 and 3.1; alpha = 1
                           with the MAD is the usual symmetric biweight).  The MAD mode
                           runs one more exact selection per window and is several times
                           slower. */
} umi_params;

#define UMI_SCALE_UPPER_RMS 0
#define UMI_SCALE_MAD 1

/* Fill `p` with alpha 2, c 5, iters 5, min_valid -1, upper-RMS scale.  NULL
 * is ignored. */
void umi_default_params(umi_params *p);

/*
 * Window length in samples for a cadence and a window span, both in days:
 * W = round(window_days / cadence_days) | 1 (Section 2 opening paragraph;
 * the bracket printed there is read as round-to-nearest, so that a cadence
 * recovered from time stamps with rounding error still gives 361 for
 * TESS 2-min data).  Returns W >= 1, or -1 for a non-positive or non-finite
 * argument or a ratio above 1e9.  Host only; never touches the GPU.
 */
int32_t umi_window_length(double cadence_days, double window_days);

/*
 * One light curve (Section 2; one launch).
 *   flux_d   [n] FP32 samples on the device; non-finite = missing
 *   n        number of samples, >= 0 (n == 0 returns UMI_OK and enqueues nothing)
 *   W        window length, odd, 1 <= W <= umi_max_window()
 *   params   NULL means umi_default_params()
 *   trend_d, detr_d  [n] FP32 outputs on the device (may not alias flux_d)
 * Allocates no device memory.  Asynchronous on `stream`.
 */
umi_status umi_detrend(const float *flux_d, int64_t n, int32_t W, const umi_params *params,
                       float *trend_d, float *detr_d, void *stream);

/*
 * Many light curves of any lengths and window lengths in one persistent
 * launch per window band (Section 2.6 runs one thread per (star, position);
 * here CTAs pull (curve, tile) work items from a device queue).
 *   flux_d     CSR samples on the device: curve b is flux_d[offsets_h[b] ..
 *              offsets_h[b+1]); outputs use the same layout
 *   offsets_h  [B+1] host array, offsets_h[0] == 0, non-decreasing
 *   W_h        [B] host array of odd window lengths, one per curve
 *   B          number of curves, >= 0
 *   params     shared by all curves; NULL means defaults
 * Device scratch (the work queue, a few bytes per tile) comes from the
 * stream-ordered allocator (cudaMallocAsync) on `stream` and is released on
 * the same stream.  Asynchronous on `stream`.  Equal-shaped batches of two or
 * more curves replay a cached CUDA graph (see umi_set_graph_cache); a batch
 * with one non-empty curve is one direct launch and needs no scratch.
 */
umi_status umi_detrend_batched(const float *flux_d, const int64_t *offsets_h, const int32_t *W_h,
                               int32_t B, const umi_params *params, float *trend_d,
                               float *detr_d, void *stream);

/*
 * umi_detrend_batched on HOST buffers: copies flux_h to the device, runs the
 * batched path and copies trend_h / detr_h back, and waits for all of it
 * before returning.  Batches of more than a couple of million samples are
 * split into up to 16 chunks of whole curves, pipelined over `stream`, a second
 * compute stream and two copy streams so that copies overlap the detrend;
 * every chunk is planned from the whole batch's bands, so the result does not
 * depend on the chunking.  The three side streams and the pipeline's events
 * belong to the calling host thread: they are created on its first call (per
 * device) and kept for its later calls.  Device buffers come from
 * cudaMallocAsync on `stream` and are freed before return.  Pinned host
 * memory makes the copies asynchronous DMA; pageable memory works but
 * serialises them.
 *
 * Memory pool: the entry points that take cudaMallocAsync scratch raise the
 * release threshold of the device's default memory pool to its maximum (once
 * per device), so that freed scratch stays mapped for the next call; the pool
 * then holds up to the largest scratch one call has taken.  A caller can trim
 * it with cudaMemPoolTrimTo.
 */
umi_status umi_detrend_batched_host(const float *flux_h, const int64_t *offsets_h,
                                    const int32_t *W_h, int32_t B, const umi_params *params,
                                    float *trend_h, float *detr_h, void *stream);

/* Capacity of the fixed device array behind umi_detrend_batched_noalloc. */
#define UMI_NOALLOC_SCRATCH_BYTES (4u * 1024u * 1024u)

/*
 * umi_detrend_batched for callers that cannot allocate device memory.  The
 * paper has no counterpart to this entry point; it exists for the library's
 * users.  Some callers cannot call cudaMalloc or cudaMallocAsync at the point
 * where they detrend: a host application whose device memory is already
 * reserved in full by another framework's caching allocator, a real-time
 * pipeline that forbids allocation after start-up (cudaMalloc and cudaFree
 * may synchronise the device and block for an unbounded time), or a
 * deployment where the stream-ordered memory pool is disabled.  This call
 * runs the same batched work-queue kernel, but its work-queue tables (curve
 * descriptors, tile items, counters) live in one file-scope device array of
 * UMI_NOALLOC_SCRATCH_BYTES (4 MiB) that every GPU loading libumi holds until
 * the process exits.  The caller still passes the input and output buffers.
 *   - It calls no cudaMalloc, cudaMallocAsync, cudaFree or other device
 *     allocator (nor cudaMallocHost), and does not use the CUDA-graph cache.
 *   - The tables reach the array inside the parameters of small copy kernels
 *     (one per 32,000 bytes of tables), enqueued on `stream` before the
 *     detrend; a launch copies its parameters when it is enqueued, so the
 *     call does not wait for earlier work on `stream` and returns at once.
 *   - A batch whose tables need more than UMI_NOALLOC_SCRATCH_BYTES returns
 *     UMI_ERR_INVALID_ARG with the size in umi_last_error(); 56 bytes per
 *     curve plus 8 bytes per tile, and a tile covers 288 to 544 positions at
 *     W = 361 depending on the plan (roughly 7,500 to 12,000 curves of
 *     18,000 samples); split larger batches.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the one array, which keeps the last call's tables;
 *     each call rewrites the tables and clears its counters on `stream`
 *     before its kernels run.  Calls whose work overlaps on the GPU (for
 *     example on two streams at once) race on the array: order them on one
 *     stream or serialise them.
 * Arguments, validation and results are those of umi_detrend_batched.
 */
umi_status umi_detrend_batched_noalloc(const float *flux_d, const int64_t *offsets_h,
                                       const int32_t *W_h, int32_t B, const umi_params *params,
                                       float *trend_d, float *detr_d, void *stream);

/*
 * Diagnostic form of umi_detrend, for parity checks.  Besides trend and
 * detr it writes, per position:
 *   median_d  the window median (also where the output is NaN), NaN for an
 *             empty window
 *   nvalid_d  valid samples in the window
 *   nplus_d   samples strictly above the median (the support of Eq. 1)
 *   scale_d   s of Eq. 1 (times 0.6745) where the trend is produced, else NaN
 * Any of the four may be NULL.  Same ownership and ordering as umi_detrend.
 */
umi_status umi_detrend_diag(const float *flux_d, int64_t n, int32_t W, const umi_params *params,
                            float *trend_d, float *detr_d, float *median_d, int32_t *nvalid_d,
                            int32_t *nplus_d, float *scale_d, void *stream);

/*
 * Gap handling before the detrend (the pipeline step the paper lists before
 * detrending, Table 3's caption; the W/3 minimum segment length of Section
 * 4, Kepler Long-Cadence).  Each curve splits at every run of at least
 * `gap_min` consecutive missing samples; leading and trailing missing runs
 * belong to no segment; segments holding fewer than `min_seg` valid samples
 * are dropped.  Kept segments are detrended as curves of their own, so no
 * window reaches across a split; every other position gets NaN.
 */
typedef struct {
    int64_t gap_min; /* missing-run length that splits a curve; <= 0 means W */
    int64_t min_seg; /* minimum valid samples of a kept segment; < 0 means floor(W/3) */
} umi_segment_params;

void umi_default_segment_params(umi_segment_params *sp);

/*
 * umi_detrend_batched with gap handling.  Same buffers and layout; `seg`
 * NULL means the defaults; `segments_out` (may be NULL) receives the number
 * of kept segments.  The segment scan needs the validity of every sample on
 * the host: the call enqueues a bit-packing kernel, copies 1 bit per sample
 * back and synchronises `stream` before it enqueues the batched launch (the
 * detrend itself stays asynchronous).  Scratch comes from cudaMallocAsync.
 */
umi_status umi_detrend_segmented(const float *flux_d, const int64_t *offsets_h, const int32_t *W_h,
                                 int32_t B, const umi_params *params, const umi_segment_params *seg,
                                 float *trend_d, float *detr_d, int64_t *segments_out, void *stream);

/* Largest supported window length (odd). */
int32_t umi_max_window(void);

/*
 * Kernel plan chosen for a window length and a band size (`positions` =
 * windows of that length in one launch; <= 0 means a band large enough for
 * the longest chain), for inspection and tuning.  `lanes` = lanes per window
 * (1-32), `slots` = register slots per lane, `chain` = consecutive positions
 * per lane group, `threads` = threads per CTA, `latency` = 1 when the band is
 * too small to fill the GPU at the shortest chain of the throughput variant
 * (then a 32-lane variant is used where one covers W within 2W, so that
 * every window can start its own chain).
 *
 * Every call plans each band from its own size, so the same curve can run on
 * different variants alone and inside a large batch.  Variants differ only in
 * how the FP32 sums of Eqs. 1 and 4 are split over lanes: the median and the
 * above-median set are the same, and the trends differ only by the rounding
 * of those sums (well inside 1e-5 relative).  Calls whose bands plan to the
 * same variant give bit-identical results.
 */
typedef struct {
    int32_t lanes;
    int32_t slots;
    int32_t chain;
    int32_t threads;
    int32_t variant; /* index into the compiled variant table */
    int32_t latency; /* 1: latency regime, 0: throughput regime */
} umi_plan;

umi_status umi_get_plan(int32_t W, int64_t positions, umi_plan *plan);

/*
 * Autotuner.  Times every eligible (lanes, slots, chain, threads) choice for
 * window length W on a synthetic flux-like curve of `positions` samples on
 * `stream` (blocking; every launch is timed alone, as one call runs, and
 * each choice's time is the best of three timed runs, a run repeating a
 * short plan for about a millisecond and counting the mean; the choices
 * within 3 % of the fastest get three more rounds; `best_ms` is the chosen
 * plan's time), and records the fastest for
 * W in the regime of that band size (see umi_plan: latency or throughput);
 * later bands of W in the same regime use it (a band smaller than
 * `positions` gets the planner's own chain for its size times the ratio the
 * tuner preferred at `positions`, if that is shorter).  umi_save_tuning /
 * umi_load_tuning persist the table as text lines
 * "gpu|W|regime|G|R|MINB|chain|threads|positions" (regime
 * "latency" or "throughput"; a line without the regime field is a throughput
 * plan; without `positions`, smaller bands get the planner's own chain when
 * it is shorter) keyed by GPU name (MINB: the register budget of the
 * variant, in CTAs of 256 threads per SM).
 * Lines for other GPUs are skipped; a malformed line fails the load and
 * leaves the table unchanged.
 */
umi_status umi_autotune(int32_t W, int64_t positions, void *stream, umi_plan *best,
                        double *best_ms);

/* Autotuner on a batch: as umi_autotune, with every choice timed on a batch
 * of `n_curves` curves of window W whose lengths are curve_len_h[0..n_curves)
 * (host array, read during the call; one band of their total positions,
 * which sets the regime and the size the plan is tuned at), so the tile
 * rounding at each curve's end, the work queue's tail and the data's own
 * gaps and outliers count as they do in such a batch.  flux_d: the curves'
 * samples back to back on the device (read only, and only by the calls'
 * launches on `stream`), or NULL for synthetic flux-like noise.  A single
 * long curve of noise shows none of these: for many short curves of uneven
 * length a shorter chain can be faster than the one such a curve of the
 * same total length prefers.  Every length >= 1 and their sum <= 2^31, else
 * UMI_ERR_INVALID_ARG. */
umi_status umi_autotune_batch(int32_t W, const float *flux_d, const int64_t *curve_len_h,
                              int32_t n_curves, void *stream, umi_plan *best, double *best_ms);
umi_status umi_save_tuning(const char *path);
umi_status umi_load_tuning(const char *path);
void umi_clear_tuning(void);

/* Enable (1) or disable (0) the CUDA-graph cache of umi_detrend_batched. */
void umi_set_graph_cache(int enabled);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of detrend requests under a device-memory
 * budget.  A scheduler thread admits queued requests while their resident
 * bytes (trend + detr, plus a copy of the flux for host inputs: 8 or 12 bytes
 * per sample, plus alignment) fit the budget and a slot is free, gathers the
 * admitted requests into batched launches (one window length per batch, or
 * arrival order) on `n_streams` streams so that batches overlap on the GPU, and
 * marks each request done when its batch's completion event fires.  Results
 * stay on the device until released.
 * ------------------------------------------------------------------------ */
typedef struct umi_server umi_server;

typedef struct {
    uint64_t mem_budget_bytes; /* resident request memory (default 40 GiB) */
    int32_t max_slots;         /* resident requests at most (default 65536) */
    int32_t n_streams;         /* batches in flight at most (default 4) */
    int32_t max_batch_curves;  /* curves per launch at most (default 1024) */
    int32_t device;            /* CUDA device ordinal (default 0) */
    double max_wait_s;         /* longest a request waits to be batched while a
                                  stream is idle (default 0: launch at once) */
    int32_t busy_poll;         /* 1 (default): the scheduler thread spins, polling
                                  for new requests and for finished batches with
                                  cudaEventQuery (lowest latency, one host core
                                  busy); 0: it sleeps on a condition variable and
                                  learns of finished batches from host callbacks */
    int32_t batch_by_window;   /* 1 (default): a batch holds requests of one window
                                  length (the oldest admitted request's), so short
                                  windows never wait for a long band of the same
                                  batch and the window classes run on separate
                                  streams; 0: batches take admitted requests in
                                  arrival order whatever their window length */
    int32_t priority_window;   /* with batch_by_window and n_streams >= 2:
                                  batches of windows at least this long run on
                                  the low-priority half of the streams and shorter
                                  ones on the high-priority half, so short windows
                                  pass queued long ones on the GPU (default 1025,
                                  which separates 20-s-cadence windows; 0: all
                                  streams have the same priority) */
} umi_server_config;

typedef struct {
    uint64_t submitted, admitted, completed, failed, rejected, released;
    uint64_t batches_launched;
    uint64_t resident_bytes, peak_resident_bytes;
    uint64_t queued_requests;
    double mean_batch_curves;
    double launch_host_s; /* scheduler time spent enqueuing batches (host seconds) */
} umi_server_stats;

void umi_server_default_config(umi_server_config *cfg);

/* Creates the server and its arena (one cudaMalloc of mem_budget_bytes). */
umi_status umi_server_create(const umi_server_config *cfg, umi_server **out);

/*
 * Queue one curve.  `flux` is a host pointer (is_device_ptr == 0) or a device
 * pointer (1).  Host data are copied into a staging buffer before this call
 * returns (the caller may reuse its buffer at once) and into server memory at
 * launch.  Device data are read in place by the kernel: the caller keeps the
 * buffer valid and unchanged until the ticket is done.  Returns UMI_ERR_BUSY
 * if the request can never fit the budget, UMI_ERR_INVALID_ARG for bad
 * W/n/params.  `ticket` receives a non-zero id.
 */
umi_status umi_server_submit(umi_server *s, const float *flux, int is_device_ptr, int64_t n,
                             int32_t W, const umi_params *params, uint64_t *ticket);

/*
 * Non-blocking.  UMI_OK when done: *trend_d / *detr_d (device pointers into
 * server memory, valid until umi_server_release) and *latency_s (submit to
 * completion) are filled (any may be NULL).  UMI_ERR_NOT_READY while queued
 * or running, UMI_ERR_FAILED if its batch failed.
 */
umi_status umi_server_poll(umi_server *s, uint64_t ticket, const float **trend_d,
                           const float **detr_d, double *latency_s);

/*
 * Timeline of a finished request, in seconds after its submit (host clock):
 * admitted (memory reserved), launched (its batch handed to the GPU) and
 * done (the batch's completion seen by the scheduler; equals *latency_s of
 * umi_server_poll).  Any pointer may be NULL.  UMI_ERR_NOT_READY before the
 * request is done; UMI_ERR_FAILED / UMI_ERR_UNKNOWN_TICKET as for poll.
 */
umi_status umi_server_timeline(umi_server *s, uint64_t ticket, double *admit_s, double *launch_s,
                               double *done_s);

/* Blocks until the ticket is done or failed, or timeout_s passes. */
umi_status umi_server_wait(umi_server *s, uint64_t ticket, double timeout_s);

/* Copies a finished result to host buffers of n floats (either may be NULL).
 * UMI_ERR_NOT_READY / UMI_ERR_FAILED / UMI_ERR_UNKNOWN_TICKET as for poll.
 * The copy runs after the server lock is dropped, so the ticket must not be
 * released by another thread while it runs. */
umi_status umi_server_copy_out(umi_server *s, uint64_t ticket, float *trend_h, float *detr_h);

/* Frees the ticket's device memory; the pointers from poll become invalid.
 * Queued, admitted, done and failed tickets can be released (a queued or
 * admitted one is withdrawn); UMI_ERR_NOT_READY while its batch runs. */
umi_status umi_server_release(umi_server *s, uint64_t ticket);

umi_status umi_server_get_stats(umi_server *s, umi_server_stats *out);

/*
 * Host-side fault injection for tests (no GPU fault is ever involved):
 * kind 1 makes the next `count` batches fail before launch (their requests
 * end UMI_ERR_FAILED), kind 2 makes the next `count` admissions fail as if
 * the arena allocation had failed.  Other requests are unaffected.
 */
umi_status umi_server_inject_fault(umi_server *s, int kind, int count);

/* Waits for in-flight batches, then frees everything. */
void umi_server_destroy(umi_server *s);

/* Message for the calling thread's last failed call ("" if none). */
const char *umi_last_error(void);

/* Library version string. */
const char *umi_version(void);

/* Number of kernels libumi has launched in this process (all entry points;
 * a graph replay counts the kernels it contains).  For launch accounting. */
long long umi_kernel_launch_count(void);

/*
 * Checked builds.  The library can be built with UMI_CHECKED
 * (`python -m paper_2604_06602_gb300.build --checked`, giving
 * libumi_checked.so): every kernel then checks its shared-memory tile reads,
 * its work items and its shared-memory size, records each failed check as a
 * bit in a per-device flag word, and skips the access instead of performing
 * it.  Bits: 1 = tile slices exceed the launch's dynamic shared memory,
 * 2 = a tile read outside the warp's slice, 4 = a work item naming a curve
 * outside the table, 8 = a work item whose tile starts past its curve's end.
 * A checked build allocates one 4-byte flag word per device on first use
 * (so umi_detrend_batched_noalloc allocates once there).  The paper has no
 * counterpart; this stands in for a memory checker on GPUs where none runs.
 *
 * umi_checked_build: 1 in a checked build, 0 otherwise.
 * umi_check_flags: synchronises the current device, stores its flag word in
 * *flags and clears it when `clear` is nonzero.  In a normal build it returns
 * UMI_ERR_INVALID_ARG (no checks ran, so there is nothing to report).
 */
int32_t umi_checked_build(void);
umi_status umi_check_flags(uint32_t *flags, int32_t clear);

#ifdef __cplusplus
}
#endif

#endif /* UMI_H */
