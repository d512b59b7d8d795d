// umi_plan.cu -- the kernel planner and the tuned-plan table.
//
// A band is the set of windows of one length W (and scale mode) in a call.
// Its plan picks the kernel variant (G lanes per window, R slots per lane,
// register budget), the chain of positions each group walks, and the CTA
// size, by a rule fitted to measured plans on GB300; umi_autotune (timing
// runs in umi_api.cu) replaces the rule for a (W, regime) pair, and the table
// it fills can be saved to and loaded from a text file.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "umi_internal.h"

namespace umi {

bool legal_chain(int G, int chain)
{
    // The 32/G groups of a warp start `chain` positions apart in the tile, so
    // one slot row's loads read words g * chain + lane (g < 32/G, lane < G).
    // A chain of G * (odd number) positions keeps the groups on disjoint
    // banks; a chain of at most G makes the groups' words one contiguous run
    // of at most 32 (overlapping windows read the same words), so no two
    // distinct words share a bank either.
    if (chain < 1) return false;
    if (G >= 32 || chain <= G) return true;
    return chain % G == 0 && ((chain / G) & 1) == 1;
}

// Smallest legal chain of at least `target` positions.
int chain_at_least(int G, int64_t target)
{
    target = std::min<int64_t>(std::max<int64_t>(target, 1), 1 << 20);
    if (G >= 32) return (int)target;
    int64_t odd = (target + G - 1) / G;
    if ((odd & 1) == 0) ++odd;
    return (int)(G * odd);
}

int shortest_chain(int G) { return G >= 32 ? 1 : G; }
// Longest chain the planner uses: about 136 positions for groups of 8 or more
// lanes, about 33 for narrower groups (whose tile is already 32 windows wide).
int chain_cap(int G) { return chain_at_least(G, G >= 8 ? 136 : 33); }
static int default_threads(int G) { return G <= 2 ? 128 : 256; }

// Planning constants, measured on GB300 over window lengths 25 to 2161 and
// bands of 1e4 to 3e6 positions:
//  * the chain is sized so that about kWarpsPerSm warps per SM get a tile
//    (kWarpsPerSmNarrow for one- and two-lane groups in the latency regime);
//  * a band is in the latency regime when, even at the shortest chain of its
//    throughput variant, it has fewer than kLatencyItemsPerSm tiles per SM;
//  * below kRegisterRichBelow positions the variant with the larger register
//    budget wins (the tighter budget pays only once many warps share an SM);
//  * below kSmallCtaBelow positions 128-thread CTAs spread a band more evenly.
static const int kWarpsPerSm = 16;
static const int kWarpsPerSmNarrow = 8;
static const int kLatencyItemsPerSm = 32;
static const int64_t kRegisterRichBelow = 500000;
static const int64_t kSmallCtaBelow = 300000;

// Tuned plans, keyed by (window length, regime) (filled by umi_autotune /
// umi_load_tuning).  Every change bumps g_tune_epoch, which is part of the
// CUDA-graph cache key, so a cached graph never replays a plan that is no
// longer current.
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, Plan> g_tuned;
static std::atomic<uint64_t> g_tune_epoch{0};

static int smallest_capacity(int W)
{
    int n = 0;
    const Variant *t = variant_table(&n);
    int best = 1 << 30;
    for (int v = 0; v < n; ++v)
        if (t[v].G * t[v].R >= W) best = std::min(best, t[v].G * t[v].R);
    return best;
}

// Capacity S covers W and wastes at most a third of it (the smallest covering
// capacity always qualifies).
static bool tight_fit(const Variant &v, int W, int smallest)
{
    const int S = v.G * v.R;
    return S >= W && (S == smallest || 3 * S <= 4 * W);
}

// Variant for bands that fill the GPU: the smallest covering capacity; below
// kRegisterRichBelow positions, the tight fit with the largest register budget
// (lowest MINB), then the smallest capacity.
static int throughput_variant(int W, int64_t positions)
{
    int n = 0;
    const Variant *t = variant_table(&n);
    const int smallest = smallest_capacity(W);
    const bool rich = positions > 0 && positions < kRegisterRichBelow;
    int best = -1;
    for (int v = 0; v < n; ++v) {
        if (!tight_fit(t[v], W, smallest)) continue;
        if (best < 0) {
            best = v;
            continue;
        }
        const Variant &a = t[v], &b = t[best];
        const int Sa = a.G * a.R, Sb = b.G * b.R;
        if (rich ? (a.minb < b.minb || (a.minb == b.minb && Sa < Sb)) : Sa < Sb) best = v;
    }
    return best;
}

// Variant for bands too small to fill the GPU.  A group narrower than a warp
// needs a chain of at least G positions, so its tile is at least 32 windows
// and the band yields at most positions/32 tiles; a 32-lane group can run a
// chain of 1.  So when a 32-lane variant covers W within 2W (or is the
// smallest covering capacity), it is used -- a tight fit first, then the
// largest register budget, then the smallest capacity; otherwise the
// throughput variant stays.
static int latency_variant(int W, int64_t positions)
{
    int n = 0;
    const Variant *t = variant_table(&n);
    const int smallest = smallest_capacity(W);
    int best = -1;
    for (int v = 0; v < n; ++v) {
        const int S = t[v].G * t[v].R;
        if (t[v].G != 32 || S < W || (S != smallest && S > 2 * W)) continue;
        if (best < 0) {
            best = v;
            continue;
        }
        const Variant &a = t[v], &b = t[best];
        const bool ta = tight_fit(a, W, smallest), tb = tight_fit(b, W, smallest);
        if (ta != tb) {
            if (ta) best = v;
            continue;
        }
        if (a.minb != b.minb) {
            if (a.minb < b.minb) best = v;
            continue;
        }
        if (S < b.G * b.R) best = v;
    }
    return best >= 0 ? best : throughput_variant(W, positions);
}

int plan_regime(int W, int64_t positions)
{
    if (positions <= 0) return kRegimeThroughput;
    const int v = throughput_variant(W, positions);
    if (v < 0) return kRegimeThroughput;
    int n = 0;
    const Variant *t = variant_table(&n);
    const int G = t[v].G;
    const int64_t tile = (int64_t)(32 / G) * shortest_chain(G);
    const int64_t items = (positions + tile - 1) / tile;
    const int sms = std::max(1, device_info(current_device()).sms);
    return items < (int64_t)kLatencyItemsPerSm * sms ? kRegimeLatency : kRegimeThroughput;
}

// Chain for `positions` windows of a band in `regime`: about kWarpsPerSm
// warps per SM get a tile -- kWarpsPerSmNarrow for groups of one or two lanes
// in the latency regime, whose chain-start selects (a lane scans its whole
// window once per bit) cost more than the longer chains they save.
static int chain_for(int G, int64_t positions, int regime)
{
    const int sms = std::max(1, device_info(current_device()).sms);
    const int target = (regime == kRegimeLatency && G <= 2) ? kWarpsPerSmNarrow : kWarpsPerSm;
    const int64_t warps = (int64_t)sms * target;
    const int64_t per_warp = (positions + warps - 1) / warps;  // windows per warp tile
    return chain_at_least(G, (per_warp * G + 31) / 32);       // 32/G groups share a tile
}

umi_status make_plan(int W, int64_t positions, Plan *plan)
{
    if (W < 1 || W > kMaxWindow || (W % 2) == 0)
        return fail(UMI_ERR_INVALID_ARG, "W must be odd and in [1, " + std::to_string(kMaxWindow) + "]");
    int n = 0;
    const Variant *t = variant_table(&n);
    const int regime = plan_regime(W, positions);
    Plan p;
    bool tuned = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(std::make_pair(W, regime));
        if (it != g_tuned.end()) {
            p = it->second;
            tuned = true;
        }
    }
    if (!tuned) {
        const int v = regime == kRegimeLatency ? latency_variant(W, positions) : throughput_variant(W, positions);
        if (v < 0) return fail(UMI_ERR_INVALID_ARG, "no kernel variant for W=" + std::to_string(W));
        p.variant = v;
        p.G = t[v].G;
        p.R = t[v].R;
        p.threads = (positions > 0 && positions < kSmallCtaBelow) ? 128 : default_threads(p.G);
        p.chain = chain_cap(p.G);
    }
    // A band smaller than the chain was sized for gets a shorter chain, so
    // that its tiles still reach every SM: the rule's chain, or for a plan
    // tuned at a known band size the rule's chain times the ratio the tuner
    // preferred at that size (the tuned chain itself at the tuned size).
    if (positions > 0) {
        const int rule = std::min(chain_cap(p.G), chain_for(p.G, positions, regime));
        if (p.tuned_at <= 0) {
            p.chain = std::min(p.chain, rule);
        } else if (positions < p.tuned_at) {
            const int64_t at = std::min(chain_cap(p.G), chain_for(p.G, p.tuned_at, regime));
            p.chain = std::min(p.chain, chain_at_least(p.G, ((int64_t)rule * p.chain + at - 1) / at));
        }
    }
    p.regime = regime;
    *plan = p;
    return UMI_OK;
}

// The candidates umi_autotune times for a band: the variants that waste at
// most a third of W (the smallest covering capacity always qualifies) -- in
// the latency regime also the 32-lane variants within 2W --, two CTA sizes,
// and chains of about 8 to 136 positions plus a third, half, once, twice and
// three times the chain the rule gives for this band; in the latency regime
// groups narrower than a warp also try chains shorter than G (1, 2, 4, 6),
// which give a warp several windows in flight at once.
std::vector<Plan> autotune_candidates(int W, int64_t positions)
{
    const int regime = plan_regime(W, positions);
    int nv = 0;
    const Variant *t = variant_table(&nv);
    const int smallest = smallest_capacity(W);
    std::vector<Plan> out;
    for (int v = 0; v < nv; ++v) {
        const int S = t[v].G * t[v].R;
        const bool wide = regime == kRegimeLatency && t[v].G == 32 && S >= W && S <= 2 * W;
        if (!tight_fit(t[v], W, smallest) && !wide) continue;
        const int G = t[v].G;
        const int base = chain_for(G, positions, regime);
        std::vector<int> chains;
        for (int64_t target : {(int64_t)8, (int64_t)24, (int64_t)40, (int64_t)72, (int64_t)136,
                               (int64_t)base / 3, (int64_t)base / 2, (int64_t)base, 2 * (int64_t)base,
                               3 * (int64_t)base}) {
            const int c = chain_at_least(G, std::max<int64_t>(target, shortest_chain(G)));
            if (c <= chain_cap(G) + 2 * G && legal_chain(G, c) &&
                std::find(chains.begin(), chains.end(), c) == chains.end())
                chains.push_back(c);
        }
        if (regime == kRegimeLatency && G < 32)
            for (int c : {1, 2, 4, 6})
                if (c < G && std::find(chains.begin(), chains.end(), c) == chains.end()) chains.push_back(c);
        for (int threads : {128, 256}) {
            for (int c : chains) {
                Plan p;
                p.variant = v;
                p.G = G;
                p.R = t[v].R;
                p.threads = threads;
                p.chain = c;
                p.regime = regime;
                p.tuned_at = positions;
                out.push_back(p);
            }
        }
    }
    return out;
}

void store_tuned(int W, const Plan &p)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::make_pair(W, p.regime)] = p;
    ++g_tune_epoch;
}

uint64_t tune_epoch() { return g_tune_epoch.load(); }

void plan_out(const Plan &p, umi_plan *out)
{
    out->lanes = p.G;
    out->slots = p.R;
    out->chain = p.chain;
    out->threads = p.threads;
    out->variant = p.variant;
    out->latency = p.regime == kRegimeLatency ? 1 : 0;
}

}  // namespace umi

using namespace umi;

extern "C" {

umi_status umi_get_plan(int32_t W, int64_t positions, umi_plan *out)
{
    clear_error();
    if (!out) return fail(UMI_ERR_INVALID_ARG, "null plan");
    Plan p;
    umi_status st = make_plan(W, positions, &p);
    if (st != UMI_OK) return st;
    plan_out(p, out);
    return UMI_OK;
}

static const char *regime_name(int r) { return r == kRegimeLatency ? "latency" : "throughput"; }

umi_status umi_save_tuning(const char *path)
{
    clear_error();
    if (!path) return fail(UMI_ERR_INVALID_ARG, "null path");
    std::ofstream f(path);
    if (!f) return fail(UMI_ERR_INVALID_ARG, std::string("cannot write ") + path);
    const std::string gpu = device_info(current_device()).name;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    int nv = 0;
    const Variant *t = variant_table(&nv);
    f << "# umi tuning table: gpu|W|regime|G|R|MINB|chain|threads|positions\n";
    for (auto &kv : g_tuned)
        f << gpu << "|" << kv.first.first << "|" << regime_name(kv.first.second) << "|" << kv.second.G
          << "|" << kv.second.R << "|" << t[kv.second.variant].minb << "|" << kv.second.chain << "|"
          << kv.second.threads << "|" << kv.second.tuned_at << "\n";
    return UMI_OK;
}

umi_status umi_load_tuning(const char *path)
{
    clear_error();
    if (!path) return fail(UMI_ERR_INVALID_ARG, "null path");
    std::ifstream f(path);
    if (!f) return fail(UMI_ERR_INVALID_ARG, std::string("cannot read ") + path);
    const std::string gpu = device_info(current_device()).name;
    int nv = 0;
    const Variant *t = variant_table(&nv);
    std::string line;
    std::map<std::pair<int, int>, Plan> loaded;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::vector<std::string> parts;
        std::stringstream ss(line);
        std::string tok;
        while (std::getline(ss, tok, '|')) parts.push_back(tok);
        // Lines without a regime field are throughput plans; the band size
        // the plan was tuned at is optional (0: unknown).
        if (parts.size() == 7) parts.insert(parts.begin() + 2, "throughput");
        if (parts.size() == 8) parts.push_back("0");
        if (parts.size() != 9) return fail(UMI_ERR_INVALID_ARG, "bad tuning line: " + line);
        if (parts[0] != gpu) continue;
        int regime = -1;
        if (parts[2] == "throughput") regime = kRegimeThroughput;
        if (parts[2] == "latency") regime = kRegimeLatency;
        Plan p;
        const int W = std::atoi(parts[1].c_str());
        p.G = std::atoi(parts[3].c_str());
        p.R = std::atoi(parts[4].c_str());
        const int minb = std::atoi(parts[5].c_str());
        p.chain = std::atoi(parts[6].c_str());
        p.threads = std::atoi(parts[7].c_str());
        p.regime = regime;
        p.tuned_at = std::atoll(parts[8].c_str());
        for (int v = 0; v < nv; ++v)
            if (t[v].G == p.G && t[v].R == p.R && t[v].minb == minb) p.variant = v;
        if (regime < 0 || p.variant < 0 || W < 1 || (W % 2) == 0 || W > kMaxWindow || p.G * p.R < W ||
            !legal_chain(p.G, p.chain) || p.chain > (1 << 20) || p.threads < p.G || p.threads > 256 ||
            p.threads % 32 || p.tuned_at < 0)
            return fail(UMI_ERR_INVALID_ARG, "bad tuning line: " + line);
        loaded[std::make_pair(W, regime)] = p;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : loaded) g_tuned[kv.first] = kv.second;
    ++g_tune_epoch;
    return UMI_OK;
}

void umi_clear_tuning(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
    ++g_tune_epoch;
}

}  // extern "C"
