// umi_host.h -- host-only pieces of the library, kept free of CUDA headers so
// that they can be built and checked on their own (tests build them with
// AddressSanitizer and UndefinedBehaviorSanitizer):
//   * the server's first-fit arena allocator (umi_server.cu);
//   * the gap scan of the segmented entry point (umi_segments.cu), which
//     reads a 1-bit-per-sample validity mask;
//   * the server's batching policy: which window length and stream the next
//     batch takes, and which admitted requests go into it.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>
#include <vector>

namespace umi {

// First-fit allocator over [0, capacity) with coalescing of free ranges.
class ArenaAllocator {
  public:
    explicit ArenaAllocator(size_t capacity) : cap_(capacity) { free_[0] = capacity; }
    bool alloc(size_t bytes, size_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
        used_ -= bytes;
    }
    size_t used() const { return used_; }
    size_t capacity() const { return cap_; }

  private:
    size_t cap_;
    size_t used_ = 0;
    std::map<size_t, size_t> free_;  // offset -> length
};

// Reader over the 32-bit-word validity mask: word-at-a-time run scans.
struct Bits {
    const unsigned *w;
    // First index in [i, end) whose bit equals `want`, or end.
    int64_t find(int64_t i, int64_t end, bool want) const
    {
        while (i < end) {
            unsigned word = w[i >> 5];
            if (!want) word = ~word;
            word &= ~0u << (i & 31);  // ignore bits below i
            if (word) {
                const int64_t j = (i & ~(int64_t)31) + __builtin_ctz(word);
                return j < end ? j : end;
            }
            i = (i & ~(int64_t)31) + 32;
        }
        return end;
    }
    // Valid samples in [a, b).
    int64_t count(int64_t a, int64_t b) const
    {
        int64_t c = 0;
        while (a < b) {
            const int64_t word_end = std::min<int64_t>((a & ~(int64_t)31) + 32, b);
            unsigned word = w[a >> 5] >> (a & 31);
            const int nb = (int)(word_end - a);
            if (nb < 32) word &= (1u << nb) - 1u;
            c += __builtin_popcount(word);
            a = word_end;
        }
        return c;
    }
};

struct Segment {
    int64_t start, len;
};

// Kept segments of the curve occupying [o, o + n) of the flat array.
inline void find_segments(const Bits &bits, int64_t o, int64_t n, int64_t gap_min, int64_t min_seg,
                          std::vector<Segment> *out)
{
    const int64_t end = o + n;
    int64_t j = bits.find(o, end, true);  // first valid sample
    while (j < end) {
        const int64_t start = j;
        int64_t cur = j;  // last valid sample known to be in this segment
        int64_t last, next;
        for (;;) {
            const int64_t g = bits.find(cur + 1, end, false);  // next missing sample
            if (g >= end) {                                      // valid up to the end
                last = end - 1;
                next = end;
                break;
            }
            const int64_t v = bits.find(g, end, true);  // first valid after the run
            if (v >= end || v - g >= gap_min) {          // trailing run, or a split
                last = g - 1;
                next = v;
                break;
            }
            cur = v;  // a short run of missing samples stays inside the segment
        }
        const int64_t valid = bits.count(start, last + 1);
        if (valid >= 1 && valid >= min_seg) out->push_back(Segment{start - o, last + 1 - start});
        j = next;
    }
}

// ---- serving policy ---------------------------------------------------------
// The admitted queue holds tickets in arrival order; window(t) is a ticket's
// window length W and idle(k) tells whether stream k has no batch in flight.

struct BatchChoice {
    int stream = -1;  // -1: nothing is launched now
    int32_t W = -1;   // the window length the batch takes
};

// The oldest admitted request names the window length, and any idle stream
// takes it.  With priority_window > 0 the streams split in halves: windows
// with W >= priority_window run only on the low-priority half [n/2, n); when
// none of those is idle, the oldest request with a shorter window goes
// instead.  Short windows take the high-priority half [0, n/2) first and the
// other half when all of it is busy.
template <class WindowOf, class IdleFn>
inline BatchChoice choose_batch(const std::vector<uint64_t> &admitted, WindowOf window, IdleFn idle,
                                int n_streams, int priority_window)
{
    BatchChoice c;
    if (admitted.empty()) return c;
    auto first_idle = [&](int a, int b) {
        for (int k = a; k < b; ++k)
            if (idle(k)) return k;
        return -1;
    };
    const int pw = priority_window;
    int32_t W0 = window(admitted.front());
    int k = -1;
    if (pw <= 0) {
        k = first_idle(0, n_streams);
    } else if (W0 >= pw) {
        k = first_idle(n_streams / 2, n_streams);
        if (k < 0) {
            W0 = -1;
            for (uint64_t t : admitted)
                if (window(t) < pw) {
                    W0 = window(t);
                    break;
                }
        }
    }
    if (pw > 0 && W0 >= 0 && W0 < pw) {
        k = first_idle(0, n_streams / 2);
        if (k < 0) k = first_idle(n_streams / 2, n_streams);
    }
    if (k < 0 || W0 < 0) return c;
    c.stream = k;
    c.W = W0;
    return c;
}

// Moves the next batch out of `admitted` into `tickets`.  By window: up to
// `cap` requests of window length W, in arrival order, while the others keep
// theirs.  Otherwise the first `cap` requests, whatever their windows.
template <class WindowOf>
inline void take_batch(std::vector<uint64_t> *admitted, WindowOf window, int32_t W, size_t cap, bool by_window,
                       std::vector<uint64_t> *tickets)
{
    tickets->clear();
    if (by_window) {
        std::vector<uint64_t> rest;
        rest.reserve(admitted->size());
        for (uint64_t t : *admitted) {
            if (tickets->size() < cap && window(t) == W) tickets->push_back(t);
            else rest.push_back(t);
        }
        admitted->swap(rest);
    } else {
        const size_t n = std::min(admitted->size(), cap);
        tickets->assign(admitted->begin(), admitted->begin() + (long)n);
        admitted->erase(admitted->begin(), admitted->begin() + (long)n);
    }
}

}  // namespace umi
