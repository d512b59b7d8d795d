// Built by tests/test_sanitizers.py with AddressSanitizer and
// UndefinedBehaviorSanitizer: the library's host-only pieces
// (paper_2604_06602_gb300/csrc/umi_host.h) against brute-force models.
//   * ArenaAllocator: random allocation and release sequences against a
//     shadow list of live ranges (inside the capacity, disjoint, `used`
//     exact, everything coalesced back into one range at the end).
//   * find_segments over the 1-bit validity mask: random validity patterns
//     and parameters against a per-sample scan of a bool array.
//   * The server's batching policy (choose_batch / take_batch) driven by a
//     mock launcher: a discrete-event run of the serving loop -- arrivals,
//     first-come-first-served admission into an ArenaAllocator under a slot
//     limit, batch launches on streams, completions after random run times --
//     checked at every decision against the policy's rules, and for liveness.
// Exit status 0 and "host ok" on success.
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <deque>
#include <random>
#include <vector>

#include "umi_host.h"

using umi::ArenaAllocator;

static int check_arena(std::mt19937_64 &rng)
{
    const size_t cap = 1 << 20;
    ArenaAllocator a(cap);
    struct Live { size_t off, bytes; };
    std::vector<Live> live;
    for (int step = 0; step < 20000; ++step) {
        const bool do_alloc = live.empty() || (rng() % 3 != 0);
        if (do_alloc) {
            const size_t bytes = 1 + rng() % 20000;
            size_t off = 0;
            size_t used = 0;
            for (auto &l : live) used += l.bytes;
            if (a.alloc(bytes, &off)) {
                if (off + bytes > cap) return 1;
                for (auto &l : live)
                    if (off < l.off + l.bytes && l.off < off + bytes) return 2;
                live.push_back({off, bytes});
            } else if (used + bytes <= cap / 4) {
                return 3;  // plenty of room left, yet refused: fragmentation this bad is a bug
            }
        } else {
            const size_t k = rng() % live.size();
            a.release(live[k].off, live[k].bytes);
            live.erase(live.begin() + (long)k);
        }
        size_t used = 0;
        for (auto &l : live) used += l.bytes;
        if (a.used() != used) return 4;
    }
    for (auto &l : live) a.release(l.off, l.bytes);
    size_t off = 7;
    if (a.used() != 0 || !a.alloc(cap, &off) || off != 0) return 5;  // fully coalesced
    return 0;
}

// Brute force: segments of valid[o, o+n) split at runs of >= gap_min missing
// samples, leading/trailing runs dropped, kept when they hold >= max(1, min_seg)
// valid samples.
static std::vector<umi::Segment> brute(const std::vector<bool> &valid, int64_t o, int64_t n,
                                       int64_t gap_min, int64_t min_seg)
{
    std::vector<umi::Segment> out;
    int64_t i = o, end = o + n;
    while (i < end && !valid[i]) ++i;
    while (i < end) {
        const int64_t start = i;
        int64_t last = i, run = 0, j = i;
        for (; j < end; ++j) {
            if (valid[j]) {
                last = j;
                run = 0;
            } else if (++run >= gap_min) {
                break;
            }
        }
        int64_t cnt = 0;
        for (int64_t k = start; k <= last; ++k) cnt += valid[k] ? 1 : 0;
        if (cnt >= 1 && cnt >= min_seg) out.push_back({start - o, last + 1 - start});
        i = last + 1;
        while (i < end && !valid[i]) ++i;
    }
    return out;
}

static int check_segments(std::mt19937_64 &rng)
{
    for (int trial = 0; trial < 3000; ++trial) {
        const int64_t total = 1 + (int64_t)(rng() % 700);
        std::vector<bool> valid((size_t)total);
        const double p_gap = (rng() % 5) * 0.1;
        for (int64_t i = 0; i < total; ++i) valid[(size_t)i] = (rng() % 1000) >= p_gap * 1000;
        for (int r = 0; r < 3; ++r) {  // runs of missing samples
            const int64_t s = (int64_t)(rng() % (uint64_t)total);
            const int64_t len = (int64_t)(rng() % 80);
            for (int64_t i = s; i < total && i < s + len; ++i) valid[(size_t)i] = false;
        }
        std::vector<unsigned> words((size_t)((total + 31) / 32), 0u);
        for (int64_t i = 0; i < total; ++i)
            if (valid[(size_t)i]) words[(size_t)(i >> 5)] |= 1u << (i & 31);
        umi::Bits bits{words.data()};
        const int64_t o = (int64_t)(rng() % (uint64_t)total);
        const int64_t n = (int64_t)(rng() % (uint64_t)(total - o + 1));
        const int64_t gap_min = 1 + (int64_t)(rng() % 40);
        const int64_t min_seg = (int64_t)(rng() % 30);
        std::vector<umi::Segment> got;
        umi::find_segments(bits, o, n, gap_min, min_seg, &got);
        const std::vector<umi::Segment> ref = brute(valid, o, n, gap_min, min_seg);
        if (got.size() != ref.size()) return 10;
        for (size_t k = 0; k < got.size(); ++k)
            if (got[k].start != ref[k].start || got[k].len != ref[k].len) return 11;
        // Counting agrees with the bools on random ranges.
        const int64_t a = (int64_t)(rng() % (uint64_t)total);
        const int64_t b = a + (int64_t)(rng() % (uint64_t)(total - a + 1));
        int64_t c = 0;
        for (int64_t i = a; i < b; ++i) c += valid[(size_t)i] ? 1 : 0;
        if (bits.count(a, b) != c) return 12;
    }
    return 0;
}

// One serving configuration; the server normalises priority_window the same
// way (off without by-window batching or with fewer than two streams).
struct SimConfig {
    int n_streams;
    int priority_window;
    bool by_window;
    size_t cap;        // max_batch_curves
    size_t max_slots;
    size_t arena;      // bytes
};

struct SimReq {
    int32_t W;
    size_t bytes;
    double t_arrive;
    size_t off = 0;
    int launched = 0, done = 0;
};

static int simulate(std::mt19937_64 &rng, SimConfig cfg, int n_req, double mean_gap)
{
    if (!cfg.by_window || cfg.n_streams < 2) cfg.priority_window = 0;
    static const int32_t kWs[] = {25, 181, 361, 721, 1025, 2161, 3601};
    std::vector<SimReq> req;
    double t = 0;
    for (int i = 0; i < n_req; ++i) {
        t += std::exponential_distribution<double>(1.0 / mean_gap)(rng);
        SimReq r;
        r.W = kWs[rng() % 7];
        r.bytes = 256 * (1 + rng() % 64);
        r.t_arrive = t;
        req.push_back(r);
    }
    const int n = cfg.n_streams, pw = cfg.priority_window;
    auto window = [&](uint64_t k) { return req[(size_t)k].W; };
    ArenaAllocator arena(cfg.arena);
    std::deque<uint64_t> pending;
    std::vector<uint64_t> admitted;
    size_t slots = 0;
    std::vector<std::vector<uint64_t>> inflight((size_t)n);
    std::vector<double> finish((size_t)n, 0.0);
    std::vector<int32_t> last_launch_of_W(4096, -1);  // per window: last ticket launched
    size_t next_arrival = 0;
    double now = 0;
    int launches = 0;
    for (int guard = 0; guard < 100 * n_req + 1000; ++guard) {
        // Completions release their arena ranges and slots.
        for (int k = 0; k < n; ++k) {
            if (inflight[(size_t)k].empty() || finish[(size_t)k] > now) continue;
            for (uint64_t q : inflight[(size_t)k]) {
                SimReq &r = req[(size_t)q];
                r.done++;
                arena.release(r.off, r.bytes);
                slots--;
            }
            inflight[(size_t)k].clear();
        }
        while (next_arrival < req.size() && req[next_arrival].t_arrive <= now) pending.push_back(next_arrival++);
        // Admission: first come, first served; the head waits for a slot or room.
        while (!pending.empty() && slots < cfg.max_slots) {
            SimReq &r = req[(size_t)pending.front()];
            if (!arena.alloc(r.bytes, &r.off)) break;
            slots++;
            admitted.push_back(pending.front());
            pending.pop_front();
        }
        // Launch while the policy finds a batch and an idle stream.
        for (;;) {
            auto idle = [&](int k) { return inflight[(size_t)k].empty(); };
            const umi::BatchChoice ch = umi::choose_batch(admitted, window, idle, n, pw);
            if (ch.stream < 0) {
                if (admitted.empty()) break;
                // Nothing launched: no stream the rules allow is idle.
                const int32_t W0 = window(admitted.front());
                bool any_short = false;
                for (uint64_t q : admitted) any_short |= pw > 0 && window(q) < pw;
                for (int k = 0; k < n; ++k) {
                    const bool allowed = pw <= 0 || k >= n / 2 || W0 < pw || any_short;
                    if (allowed && idle(k)) return 20;
                }
                break;
            }
            const int k = ch.stream;
            if (k >= n || !idle(k)) return 21;
            // Oldest first: the front's window, unless it is long, every
            // low-priority stream is busy, and the oldest short request goes.
            const int32_t W0 = window(admitted.front());
            if (ch.W != W0) {
                if (pw <= 0 || W0 < pw) return 22;
                for (int j = n / 2; j < n; ++j)
                    if (idle(j)) return 23;
                for (uint64_t q : admitted) {
                    if (window(q) < pw) {
                        if (window(q) != ch.W) return 24;
                        break;
                    }
                }
            }
            // Stream classes, and the lowest idle stream of the class.
            if (pw > 0) {
                if (ch.W >= pw && k < n / 2) return 25;
                if (ch.W < pw && k >= n / 2)
                    for (int j = 0; j < n / 2; ++j)
                        if (idle(j)) return 26;
                const int lo = (ch.W >= pw || k >= n / 2) ? n / 2 : 0;
                for (int j = lo; j < k; ++j)
                    if (idle(j)) return 27;
            } else {
                for (int j = 0; j < k; ++j)
                    if (idle(j)) return 27;
            }
            const std::vector<uint64_t> before = admitted;
            std::vector<uint64_t> batch;
            umi::take_batch(&admitted, window, ch.W, cfg.cap, cfg.by_window, &batch);
            if (batch.empty() || batch.size() > cfg.cap) return 28;
            // The batch plus what stays is the queue before, order kept.
            std::vector<uint64_t> expect_batch, expect_rest;
            for (uint64_t q : before) {
                const bool take = cfg.by_window ? (window(q) == ch.W && expect_batch.size() < cfg.cap)
                                                : expect_batch.size() < cfg.cap;
                (take ? expect_batch : expect_rest).push_back(q);
            }
            if (batch != expect_batch || admitted != expect_rest) return 29;
            for (uint64_t q : batch) {
                SimReq &r = req[(size_t)q];
                if (cfg.by_window && r.W != ch.W) return 30;
                // Within one window length, launches follow arrival order.
                if (last_launch_of_W[(size_t)r.W] > (int32_t)q) return 31;
                last_launch_of_W[(size_t)r.W] = (int32_t)q;
                r.launched++;
            }
            inflight[(size_t)k] = batch;
            // Long windows run longer; a batch costs a little per request.
            finish[(size_t)k] = now + 0.05 * (double)ch.W / 361.0 + 0.02 * (double)batch.size() +
                                std::uniform_real_distribution<double>(0.0, 0.5)(rng);
            launches++;
        }
        // Advance to the next arrival or completion.
        double next = 1e300;
        if (next_arrival < req.size()) next = req[next_arrival].t_arrive;
        for (int k = 0; k < n; ++k)
            if (!inflight[(size_t)k].empty()) next = std::min(next, finish[(size_t)k]);
        if (next == 1e300) break;
        now = std::max(now, next);
    }
    // Liveness: every request ran once and finished; the arena is empty again.
    for (const SimReq &r : req)
        if (r.launched != 1 || r.done != 1) return 32;
    if (!pending.empty() || !admitted.empty() || slots != 0 || arena.used() != 0) return 33;
    if (launches < 1) return 34;
    return 0;
}

static int check_scheduler(std::mt19937_64 &rng)
{
    for (int trial = 0; trial < 400; ++trial) {
        static const int kStreams[] = {1, 2, 3, 4, 8};
        static const int kPw[] = {0, 1025, 362, 4000};
        SimConfig cfg;
        cfg.n_streams = kStreams[rng() % 5];
        cfg.priority_window = kPw[rng() % 4];
        cfg.by_window = (rng() % 4) != 0;
        cfg.cap = 1 + rng() % 16;
        cfg.max_slots = 1 + rng() % 64;
        cfg.arena = 256 * 64 * (1 + rng() % 40);  // at least one request of the largest size fits
        static const double kGap[] = {0.01, 0.1, 1.0};  // from overload to light load
        const int rc = simulate(rng, cfg, 50 + (int)(rng() % 300), kGap[rng() % 3]);
        if (rc) {
            std::printf("scheduler: n_streams=%d priority_window=%d by_window=%d cap=%zu slots=%zu arena=%zu\n",
                        cfg.n_streams, cfg.priority_window, (int)cfg.by_window, cfg.cap, cfg.max_slots, cfg.arena);
            return rc;
        }
    }
    return 0;
}

int main()
{
    std::mt19937_64 rng(20260406);
    int rc = check_arena(rng);
    if (rc) {
        std::printf("arena check failed: %d\n", rc);
        return rc;
    }
    rc = check_segments(rng);
    if (rc) {
        std::printf("segment check failed: %d\n", rc);
        return rc;
    }
    rc = check_scheduler(rng);
    if (rc) {
        std::printf("scheduler check failed: %d\n", rc);
        return rc;
    }
    std::printf("host ok\n");
    return 0;
}
