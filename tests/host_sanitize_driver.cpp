// Built by tests/test_sanitizers.py with AddressSanitizer and
// UndefinedBehaviorSanitizer: the library's host-only pieces
// (paper_2604_06602_gb300/csrc/umi_host.h) against brute-force models.
//   * ArenaAllocator: random allocation and release sequences against a
//     shadow list of live ranges (inside the capacity, disjoint, `used`
//     exact, everything coalesced back into one range at the end).
//   * find_segments over the 1-bit validity mask: random validity patterns
//     and parameters against a per-sample scan of a bool array.
// Exit status 0 and "host ok" on success.
#include <cstdio>
#include <cstdlib>
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
    std::printf("host ok\n");
    return 0;
}
