// umi_server.cu -- continuous-batching detrend server.
//
// Requests (one light curve each) are queued by umi_server_submit.  A
// scheduler thread
//   1. admits queued requests in arrival order while their resident memory
//      (trend + detr, plus flux for host inputs, each rounded up to 256 bytes)
//      fits the arena and
//      a slot is free; memory is handed out by a first-fit allocator over one
//      cudaMalloc of the budget;
//   2. gathers the admitted requests into one batch per idle stream (up to
//      max_batch_curves; by default only requests of the oldest admitted
//      request's window length, so a batch of short windows never waits for
//      a long band launched before it on the same stream; or in arrival
//      order), enqueues their host-input copies (device inputs are
//      read in place) and one batched launch
//      (the persistent work-queue kernel of umi_api.cu) on that stream, then a
//      completion marker (an event the scheduler polls, or a host callback),
//      so up to n_streams batches run on the GPU at once while new requests
//      keep arriving;
//   3. marks requests done when their batch's marker has fired.
// Results stay in the arena until umi_server_release.  A batch that fails to
// launch fails only its own requests; the server keeps serving.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "umi_host.h"
#include "umi_internal.h"

namespace umi {

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}


enum class ReqState { Queued, Admitted, Running, Done, Failed };

struct Request {
    uint64_t ticket = 0;
    int64_t n = 0;
    int32_t W = 0;
    umi_params params{};
    std::vector<float> host_copy;   // input staged at submit (host pointers)
    const float *dev_src = nullptr;  // input left on the device by the caller
    size_t off = 0, bytes = 0;       // arena range
    float *flux = nullptr, *trend = nullptr, *detr = nullptr;
    bool admitted_mem = false;       // owns its arena range
    ReqState state = ReqState::Queued;
    double t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;  // host clock, seconds
};

struct Batch {
    umi_server *srv = nullptr;
    int stream = 0;
    std::vector<uint64_t> tickets;
    std::atomic<bool> done{false};
    double t_done = 0;
};

}  // namespace umi

using namespace umi;

struct StreamBuffers {
    char *dev = nullptr;   // work-queue tables of this stream's batch
    size_t dev_bytes = 0;
    char *host = nullptr;  // pinned staging for the tables
    size_t host_bytes = 0;
};

struct umi_server {
    umi_server_config cfg{};
    char *arena = nullptr;
    std::unique_ptr<ArenaAllocator> alloc;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done_events;  // busy-poll mode: one per stream
    std::vector<StreamBuffers> bufs;  // one per stream; a stream runs one batch at a time
    std::vector<std::shared_ptr<Batch>> inflight;  // one slot per stream
    std::mutex mu;
    std::condition_variable cv_sched;
    std::condition_variable cv_done;
    std::deque<uint64_t> pending;
    std::vector<uint64_t> admitted;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    size_t resident_slots = 0;
    bool stop = false;
    std::thread worker;
    umi_server_stats stats{};
    double batch_curves_sum = 0;
    int inject_launch_failures = 0;
    int inject_alloc_failures = 0;
    std::atomic<uint64_t> change_seq{0};  // bumped by submit / release (busy-poll wake-up)
};

namespace umi {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
// Device-resident inputs are read in place, so they need no arena copy.
static size_t request_bytes(int64_t n, bool device_input)
{
    return (device_input ? 2 : 3) * align256(sizeof(float) * (size_t)n);
}

static void CUDART_CB batch_done_cb(void *arg)
{
    // Once `done` is visible the scheduler may reap and free the batch, so it
    // is set under the lock and the batch is not touched afterwards (the
    // server outlives the callback: destroy synchronizes every stream).
    Batch *b = static_cast<Batch *>(arg);
    umi_server *s = b->srv;
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        b->t_done = t;
        b->done.store(true);
    }
    s->cv_sched.notify_one();
}

// Called with the lock held.
static void admit_locked(umi_server *s)
{
    while (!s->pending.empty()) {
        const uint64_t t = s->pending.front();
        auto it = s->reqs.find(t);
        if (it == s->reqs.end()) {  // released while queued
            s->pending.pop_front();
            continue;
        }
        Request &r = *it->second;
        if (s->resident_slots >= (size_t)s->cfg.max_slots) break;
        size_t off = 0;
        if (s->inject_alloc_failures > 0) {
            --s->inject_alloc_failures;
            r.state = ReqState::Failed;
            r.t_done = now_s();
            r.host_copy.clear();
            r.host_copy.shrink_to_fit();
            s->stats.failed++;
            s->pending.pop_front();
            s->cv_done.notify_all();
            continue;
        }
        if (!s->alloc->alloc(r.bytes, &off)) break;  // head-of-line waits for memory
        r.off = off;
        const size_t one = align256(sizeof(float) * (size_t)r.n);
        char *base = s->arena + off;
        if (r.dev_src) {
            r.flux = nullptr;
            r.trend = reinterpret_cast<float *>(base);
            r.detr = reinterpret_cast<float *>(base + one);
        } else {
            r.flux = reinterpret_cast<float *>(base);
            r.trend = reinterpret_cast<float *>(base + one);
            r.detr = reinterpret_cast<float *>(base + 2 * one);
        }
        r.admitted_mem = true;
        r.state = ReqState::Admitted;
        r.t_admit = now_s();
        s->resident_slots++;
        s->stats.admitted++;
        s->stats.resident_bytes = s->alloc->used();
        s->stats.peak_resident_bytes = std::max<uint64_t>(s->stats.peak_resident_bytes, s->alloc->used());
        s->admitted.push_back(t);
        s->pending.pop_front();
    }
    s->stats.queued_requests = s->pending.size();
}

// Marks finished batches; called with the lock held.
static void reap_locked(umi_server *s)
{
    for (size_t k = 0; k < s->inflight.size(); ++k) {
        auto &b = s->inflight[k];
        if (!b) continue;
        if (s->cfg.busy_poll && !b->done.load()) {
            const cudaError_t q = cudaEventQuery(s->done_events[k]);
            if (q == cudaSuccess) {
                b->t_done = now_s();
                b->done.store(true);
            } else if (q != cudaErrorNotReady) {
                cudaGetLastError();
            }
        }
        if (!b->done.load()) continue;
        for (uint64_t t : b->tickets) {
            auto it = s->reqs.find(t);
            if (it == s->reqs.end()) continue;
            it->second->state = ReqState::Done;
            it->second->t_done = b->t_done;
            s->stats.completed++;
        }
        b.reset();
        s->cv_done.notify_all();
    }
}

static void fail_requests_locked(umi_server *s, const std::vector<uint64_t> &tickets)
{
    for (uint64_t t : tickets) {
        auto it = s->reqs.find(t);
        if (it == s->reqs.end()) continue;
        it->second->state = ReqState::Failed;
        it->second->t_done = now_s();
        s->stats.failed++;
    }
    s->cv_done.notify_all();
}

// Launches one batch on stream k; called with the lock held, drops it while
// enqueuing device work.
static void launch_batch_locked(umi_server *s, int k, int32_t W0, std::unique_lock<std::mutex> &lk)
{
    NvtxRange nvtx("umi server batch launch");
    std::vector<uint64_t> tickets;
    take_batch(&s->admitted, [s](uint64_t t) { return s->reqs[t]->W; }, W0, (size_t)s->cfg.max_batch_curves,
               s->cfg.batch_by_window != 0, &tickets);
    const size_t take = tickets.size();
    struct Job {
        float *flux, *trend, *detr;
        const float *src_dev;
        std::vector<float> src_host;
        int64_t n;
        int32_t W;
        umi_params p;
    };
    std::vector<Job> jobs;
    jobs.reserve(take);
    const double t_launch = now_s();
    for (uint64_t t : tickets) {
        Request &r = *s->reqs[t];
        r.state = ReqState::Running;
        r.t_launch = t_launch;
        Job j{r.flux, r.trend, r.detr, r.dev_src, std::move(r.host_copy), r.n, r.W, r.params};
        r.host_copy = std::vector<float>();
        jobs.push_back(std::move(j));
    }
    auto batch = std::make_shared<Batch>();
    batch->srv = s;
    batch->stream = k;
    batch->tickets = tickets;
    s->inflight[k] = batch;
    const bool inject = s->inject_launch_failures > 0;
    if (inject) --s->inject_launch_failures;
    lk.unlock();
    const double t_enq0 = now_s();

    cudaStream_t st = s->streams[k];
    bool ok = !inject;
    std::vector<Curve> curves;
    curves.reserve(jobs.size());
    for (auto &j : jobs) {
        if (!ok) break;
        if (!j.src_dev) {
            const cudaError_t e = cudaMemcpyAsync(j.flux, j.src_host.data(), sizeof(float) * j.n,
                                                  cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) ok = false;
        }
        Curve c;
        c.flux = j.src_dev ? j.src_dev : j.flux;
        c.trend = j.trend;
        c.detr = j.detr;
        c.n = j.n;
        c.W = j.W;
        c.min_valid = resolve_min_valid(j.W, j.p.min_valid);
        c.alpha = j.p.alpha;
        c.c = j.p.c;
        c.iters = j.p.iters;
        c.scale_mode = j.p.scale_mode;
        curves.push_back(c);
    }
    int launches = 0;
    if (curves.size() == 1) {
        // A batch of one request needs no work-queue tables (the common case
        // at low load): its kernel follows the input copy directly.
        if (ok && launch_single_curve(curves[0], curves[0].n, nullptr, st, &launches) != UMI_OK) ok = false;
    } else {
        PreparedBatch pb;
        if (ok && prepare_batch(curves, &pb) != UMI_OK) ok = false;
        StreamBuffers &sb = s->bufs[k];
        // This stream's previous batch has completed (it is idle), so its
        // buffers may be regrown or rewritten.
        if (ok && pb.dev_bytes > sb.dev_bytes) {
            if (sb.dev) cudaFree(sb.dev);
            sb.dev = nullptr;
            sb.dev_bytes = 0;
            if (cudaMalloc((void **)&sb.dev, 2 * pb.dev_bytes) == cudaSuccess) sb.dev_bytes = 2 * pb.dev_bytes;
            else ok = false;
        }
        if (ok && pb.host_bytes > sb.host_bytes) {
            if (sb.host) cudaFreeHost(sb.host);
            sb.host = nullptr;
            sb.host_bytes = 0;
            if (cudaMallocHost((void **)&sb.host, 2 * pb.host_bytes) == cudaSuccess) sb.host_bytes = 2 * pb.host_bytes;
            else ok = false;
        }
        if (ok && enqueue_prepared(curves, pb, sb.dev, sb.host, st, &launches) != UMI_OK) ok = false;
    }
    if (ok) {
        const cudaError_t e = s->cfg.busy_poll ? cudaEventRecord(s->done_events[k], st)
                                               : cudaLaunchHostFunc(st, batch_done_cb, batch.get());
        if (e != cudaSuccess) ok = false;
    }
    const double t_enq = now_s() - t_enq0;
    count_launches(launches);

    lk.lock();
    s->stats.launch_host_s += t_enq;
    s->stats.batches_launched++;
    s->batch_curves_sum += (double)take;
    s->stats.mean_batch_curves = s->batch_curves_sum / (double)s->stats.batches_launched;
    if (!ok) {
        // Nothing of this batch is relied upon: wait for any copies already
        // enqueued, then fail its requests only.
        lk.unlock();
        cudaStreamSynchronize(st);
        cudaGetLastError();
        lk.lock();
        s->inflight[k].reset();
        fail_requests_locked(s, tickets);
    }
}

static void scheduler_main(umi_server *s)
{
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        reap_locked(s);
        admit_locked(s);
        bool hold = false;
        if (s->cfg.max_wait_s > 0.0 && !s->admitted.empty() && s->pending.empty() &&
            s->admitted.size() < (size_t)s->cfg.max_batch_curves) {
            // Hold a small batch back a little so that it can grow.
            const double age = now_s() - s->reqs[s->admitted.front()]->t_submit;
            if (age < s->cfg.max_wait_s) {
                if (!s->cfg.busy_poll) {
                    s->cv_sched.wait_for(lk, std::chrono::duration<double>(s->cfg.max_wait_s - age));
                    continue;
                }
                hold = true;
            }
        }
        bool launched = false;
        while (!hold && !s->admitted.empty() && !s->stop) {
            // The window length to batch and an idle stream for it
            // (choose_batch: oldest first; long windows on the low-priority
            // half of the streams when priority_window is set).
            const BatchChoice ch = choose_batch(
                s->admitted, [s](uint64_t t) { return s->reqs[t]->W; },
                [s](int k) { return !s->inflight[k]; }, (int)s->streams.size(), s->cfg.priority_window);
            if (ch.stream < 0) break;
            launch_batch_locked(s, ch.stream, ch.W, lk);
            launched = true;
        }
        if (launched) continue;
        if (s->cfg.busy_poll) {
            // Spin without the lock until a request arrives or is released, a
            // batch in flight finishes, or 200 us pass.  Only this thread
            // touches `inflight` and the events, so they are read unlocked.
            const uint64_t seen = s->change_seq.load();
            std::vector<int> busy;
            for (size_t k = 0; k < s->inflight.size(); ++k)
                if (s->inflight[k]) busy.push_back((int)k);
            const bool holding = hold;
            lk.unlock();
            const double t_spin = now_s();
            for (;;) {
                if (s->stop || s->change_seq.load() != seen) break;
                bool finished = false;
                for (int k : busy)
                    if (cudaEventQuery(s->done_events[k]) != cudaErrorNotReady) finished = true;
                if (finished || holding || now_s() - t_spin > 200e-6) break;
                std::this_thread::yield();
            }
            lk.lock();
        } else {
            s->cv_sched.wait_for(lk, std::chrono::microseconds(500));
        }
    }
}

}  // namespace umi

extern "C" {

void umi_server_default_config(umi_server_config *cfg)
{
    if (!cfg) return;
    cfg->mem_budget_bytes = 40ull << 30;
    cfg->max_slots = 65536;
    cfg->n_streams = 4;
    cfg->max_batch_curves = 1024;
    cfg->device = 0;
    cfg->max_wait_s = 0.0;
    cfg->busy_poll = 1;
    cfg->batch_by_window = 1;
    cfg->priority_window = 1025;
}

umi_status umi_server_create(const umi_server_config *cfg_in, umi_server **out)
{
    clear_error();
    if (!out) return fail(UMI_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    umi_server_config cfg;
    umi_server_default_config(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.mem_budget_bytes < 4096 || cfg.max_slots < 1 || cfg.n_streams < 1 || cfg.n_streams > 64 ||
        cfg.max_batch_curves < 1 || cfg.device < 0 || !(cfg.max_wait_s >= 0.0) ||
        (cfg.batch_by_window != 0 && cfg.batch_by_window != 1) || cfg.priority_window < 0)
        return fail(UMI_ERR_INVALID_ARG, "bad server config");
    // Priorities need window-homogeneous batches and streams to split.
    if (!cfg.batch_by_window || cfg.n_streams < 2) cfg.priority_window = 0;
    cudaError_t e = cudaSetDevice(cfg.device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    std::unique_ptr<umi_server> s(new umi_server());
    s->cfg = cfg;
    e = cudaMalloc((void **)&s->arena, cfg.mem_budget_bytes);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMalloc (server arena)");
    s->alloc.reset(new ArenaAllocator(cfg.mem_budget_bytes));
    s->streams.resize(cfg.n_streams);
    s->done_events.resize(cfg.n_streams);
    s->bufs.resize(cfg.n_streams);
    s->inflight.resize(cfg.n_streams);
    int least = 0, greatest = 0;
    if (cfg.priority_window > 0 && cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    for (int k = 0; k < cfg.n_streams; ++k) {
        // With priority_window, streams [0, n/2) take short windows at the
        // greatest priority and the rest long windows at the least.
        const int prio = cfg.priority_window > 0 ? (k < cfg.n_streams / 2 ? greatest : least) : 0;
        e = cudaStreamCreateWithPriority(&s->streams[k], cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->done_events[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (auto &x : s->streams)
                if (x) cudaStreamDestroy(x);
            for (auto &x : s->done_events)
                if (x) cudaEventDestroy(x);
            cudaFree(s->arena);
            return fail_cuda(e, "cudaStreamCreate");
        }
    }
    umi_server *raw = s.release();
    raw->worker = std::thread(scheduler_main, raw);
    *out = raw;
    return UMI_OK;
}

umi_status umi_server_submit(umi_server *s, const float *flux, int is_device_ptr, int64_t n,
                             int32_t W, const umi_params *params, uint64_t *ticket)
{
    clear_error();
    if (!s || !ticket) return fail(UMI_ERR_INVALID_ARG, "null server or ticket");
    *ticket = 0;
    umi_params p;
    umi_status st = check_params(params, &p);
    if (st != UMI_OK) return st;
    if (n < 1) return fail(UMI_ERR_INVALID_ARG, "n must be >= 1");
    if (!flux) return fail(UMI_ERR_INVALID_ARG, "null flux");
    Plan plan;
    st = make_plan(W, -1, &plan);
    if (st != UMI_OK) return st;
    const size_t bytes = request_bytes(n, is_device_ptr != 0);
    if (bytes > s->cfg.mem_budget_bytes) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.rejected++;
        return fail(UMI_ERR_BUSY, "request larger than the server memory budget");
    }
    std::unique_ptr<Request> r(new Request());
    r->n = n;
    r->W = W;
    r->params = p;
    r->bytes = bytes;
    if (is_device_ptr) r->dev_src = flux;
    else r->host_copy.assign(flux, flux + n);
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->pending.push_back(r->ticket);
        s->reqs.emplace(r->ticket, std::move(r));
        s->stats.submitted++;
        s->stats.queued_requests = s->pending.size();
    }
    s->change_seq.fetch_add(1);
    s->cv_sched.notify_one();
    return UMI_OK;
}

umi_status umi_server_poll(umi_server *s, uint64_t ticket, const float **trend_d, const float **detr_d,
                           double *latency_s)
{
    clear_error();
    if (!s) return fail(UMI_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(UMI_ERR_UNKNOWN_TICKET, "unknown ticket");
    const Request &r = *it->second;
    if (r.state == ReqState::Failed) return fail(UMI_ERR_FAILED, "request failed");
    if (r.state != ReqState::Done) return UMI_ERR_NOT_READY;
    if (trend_d) *trend_d = r.trend;
    if (detr_d) *detr_d = r.detr;
    if (latency_s) *latency_s = r.t_done - r.t_submit;
    return UMI_OK;
}

umi_status umi_server_timeline(umi_server *s, uint64_t ticket, double *admit_s, double *launch_s,
                               double *done_s)
{
    clear_error();
    if (!s) return fail(UMI_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(UMI_ERR_UNKNOWN_TICKET, "unknown ticket");
    const Request &r = *it->second;
    if (r.state == ReqState::Failed) return fail(UMI_ERR_FAILED, "request failed");
    if (r.state != ReqState::Done) return UMI_ERR_NOT_READY;
    if (admit_s) *admit_s = r.t_admit - r.t_submit;
    if (launch_s) *launch_s = r.t_launch - r.t_submit;
    if (done_s) *done_s = r.t_done - r.t_submit;
    return UMI_OK;
}

umi_status umi_server_wait(umi_server *s, uint64_t ticket, double timeout_s)
{
    clear_error();
    if (!s) return fail(UMI_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(std::max(0.0, timeout_s)));
    for (;;) {
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(UMI_ERR_UNKNOWN_TICKET, "unknown ticket");
        if (it->second->state == ReqState::Done) return UMI_OK;
        if (it->second->state == ReqState::Failed) return fail(UMI_ERR_FAILED, "request failed");
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto jt = s->reqs.find(ticket);
            if (jt != s->reqs.end() && jt->second->state == ReqState::Done) return UMI_OK;
            return fail(UMI_ERR_TIMEOUT, "wait timed out");
        }
    }
}

umi_status umi_server_copy_out(umi_server *s, uint64_t ticket, float *trend_h, float *detr_h)
{
    clear_error();
    if (!s) return fail(UMI_ERR_INVALID_ARG, "null server");
    const float *tr = nullptr, *de = nullptr;
    int64_t n = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(UMI_ERR_UNKNOWN_TICKET, "unknown ticket");
        const Request &r = *it->second;
        if (r.state == ReqState::Failed) return fail(UMI_ERR_FAILED, "request failed");
        if (r.state != ReqState::Done) return UMI_ERR_NOT_READY;
        tr = r.trend;
        de = r.detr;
        n = r.n;
    }
    if (trend_h) {
        cudaError_t e = cudaMemcpy(trend_h, tr, sizeof(float) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpy D2H");
    }
    if (detr_h) {
        cudaError_t e = cudaMemcpy(detr_h, de, sizeof(float) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpy D2H");
    }
    return UMI_OK;
}

umi_status umi_server_release(umi_server *s, uint64_t ticket)
{
    clear_error();
    if (!s) return fail(UMI_ERR_INVALID_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(UMI_ERR_UNKNOWN_TICKET, "unknown ticket");
        Request &r = *it->second;
        if (r.state == ReqState::Running) return fail(UMI_ERR_NOT_READY, "request still running");
        if (r.state == ReqState::Admitted) {
            s->admitted.erase(std::remove(s->admitted.begin(), s->admitted.end(), ticket),
                              s->admitted.end());
        }
        if (r.admitted_mem) {  // admitted at some point: owns arena memory
            s->alloc->release(r.off, r.bytes);
            s->resident_slots--;
            s->stats.resident_bytes = s->alloc->used();
        }
        // Queued requests are dropped from `pending` lazily by admit_locked.
        s->reqs.erase(it);
        s->stats.released++;
    }
    s->change_seq.fetch_add(1);
    s->cv_sched.notify_one();
    return UMI_OK;
}

umi_status umi_server_get_stats(umi_server *s, umi_server_stats *out)
{
    clear_error();
    if (!s || !out) return fail(UMI_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->resident_bytes = s->alloc->used();
    out->queued_requests = s->pending.size();
    return UMI_OK;
}

umi_status umi_server_inject_fault(umi_server *s, int kind, int count)
{
    clear_error();
    if (!s || count < 0) return fail(UMI_ERR_INVALID_ARG, "bad fault injection");
    std::lock_guard<std::mutex> lk(s->mu);
    if (kind == 1) s->inject_launch_failures = count;
    else if (kind == 2) s->inject_alloc_failures = count;
    else return fail(UMI_ERR_INVALID_ARG, "unknown fault kind");
    return UMI_OK;
}

void umi_server_destroy(umi_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto &b : s->bufs) {
        if (b.dev) cudaFree(b.dev);
        if (b.host) cudaFreeHost(b.host);
    }
    for (auto &x : s->done_events) cudaEventDestroy(x);
    s->inflight.clear();
    if (s->arena) cudaFree(s->arena);
    delete s;
}

}  // extern "C"
