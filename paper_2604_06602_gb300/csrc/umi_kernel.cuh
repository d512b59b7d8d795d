// umi_kernel.cuh -- sm_103a kernel for the UMI sliding-window robust trend.
//
// Method (paper Section 2): per output position, over the W-sample window
// with missing samples dropped: Phase 1 exact median (Section 2.1), Phase 2
// upper-RMS scale s = 0.6745 sqrt(mean_{x > m} (x - m)^2) (Eq. 1), Phase 3
// `iters` asymmetric bisquare reweighting steps (Eqs. 2-4), trend = mu,
// detrended flux = x / mu.
//
// GPU design (not the paper's one-thread-per-window kernel, Section 2.6):
//  * A warp owns a tile of T consecutive positions of one curve and stages the
//    T + S - 1 samples its windows touch into its slice of shared memory once,
//    with 4-byte cp.async copies; missing samples (non-finite, or outside the
//    curve) become kGap.
//  * A "group" of G lanes (G = 1..32, a power of two) evaluates one window at a
//    time, each lane holding R window slots in registers (S = G*R >= W slots;
//    slots past W hold kGap).  The 32/G groups of a warp run in lock step on
//    neighbouring chains; every block that shuffles is entered warp-uniformly.
//  * Each group walks a chain of P consecutive positions.  At the chain start
//    (or after an empty window) the median comes from an exact binary search
//    over order-preserving integer keys.  Afterwards the group keeps the
//    counts L = #{x < m}, E = #{x == m}, G+ = #{x > m} of the current window
//    and updates them in O(1) per step from the sample that leaves and the one
//    that enters.  One step moves the median's rank by at most one, so the new
//    median is m itself, the largest sample below m, or the smallest above m;
//    the last two take one pass over the registers.  Every median is the exact
//    order statistic of rank floor((n_valid - 1)/2).
//  * Eq. 1 is one pass over the registers, G+ comes from the counts.
//  * Phase 3 keeps y = x - m in registers, in pairs for the packed FP32x2
//    instructions, and runs the fixed number of steps on mu = m + delta: per
//    slot u_eff^2 = t (t + rho |t|) with t = sigma (y - delta) (for
//    1/4 <= alpha <= 4; otherwise u_eff = min(y kp - delta kp, y kn - delta
//    kn) with kp = 1/(c s), kn = alpha/(c s): Eq. 2 without a branch either
//    way), z = sat(1 - u_eff^2), w = z^2 (Eq. 3), and delta = sum(w y)/sum(w)
//    (Eq. 4 about m).  A kGap slot has u_eff^2 >= 1 (or it overflows, or is
//    NaN), so sat() makes its weight exactly 0 without a mask.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace umi {

// Missing-sample marker inside the tile.  Finite, below every admissible
// sample (|x| < 2^60), and so far below that its standardised residual never
// reaches the bisquare support.
constexpr float kGap = -0x1p100f;
constexpr float kGapLimit = -0x1p99f;  // x > kGapLimit  <=>  a real sample
constexpr float kScaleFactor = 0.6745f;  // Section 2.2, as printed

struct Curve {
    const float *flux;
    float *trend;
    float *detr;
    int64_t n;
    int32_t W;
    int32_t min_valid;  // resolved, >= 0
    float alpha;
    float c;
    int32_t iters;
    int32_t scale_mode;  // 0: upper-RMS scale (Eq. 1); 1: MAD
};

struct Diag {
    float *median;
    int32_t *nvalid;
    int32_t *nplus;
    float *scale;
};

struct Item {
    int32_t curve;  // index into the curve table
    int32_t tile;   // tile index within the curve; first position = tile * T
};

struct LaunchArgs {
    const Curve *curves;  // device curve table, or nullptr to use `single`
    Curve single;
    const Item *items;    // device item list, or nullptr: item i = {0, i}
    int32_t n_items;
    int32_t chain;        // P: consecutive positions per group
    int32_t *queue;       // persistent work counter, or nullptr: one item per CTA
    Diag diag;
    int32_t n_curves;     // entries of `curves` (checked builds test item indices)
    uint32_t *check;      // checked builds: flag word of failed index checks
};

// Index checks of the checked build (compiled with UMI_CHECKED).  A failed
// check sets its bit in LaunchArgs::check and the access is skipped (a read
// gives kGap, a write is dropped), so a bad index is reported, never
// performed.  Normal builds compile none of it.
enum : uint32_t {
    kCheckSmemSize = 1u << 0,    // the warps' tile slices exceed the launch's dynamic smem
    kCheckTileRead = 1u << 1,    // window, slide or centre read outside the warp's tile
    kCheckCurveIndex = 1u << 2,  // work item names a curve outside the table
    kCheckItemTile = 1u << 3,    // work item's tile starts past its curve's end
};

// Read-only view of a warp's tile: a bare pointer in normal builds, a
// bounds-checked reader in checked builds.
struct TileRef {
    const float *p;
#ifdef UMI_CHECKED
    int len;
    uint32_t *check;
    __device__ __forceinline__ float operator[](int i) const
    {
        if (i < 0 || i >= len) {
            if (check) atomicOr(check, kCheckTileRead);
            return kGap;
        }
        return p[i];
    }
#else
    __device__ __forceinline__ float operator[](int i) const { return p[i]; }
#endif
};

// ---- group-wide reductions over G aligned lanes --------------------------
template <int G>
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ int group_sum_int(int v)
{
    if constexpr (G == 32) {
        return (int)__reduce_add_sync(0xffffffffu, (unsigned)v);
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
}

template <int G>
__device__ __forceinline__ float group_max(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int G>
__device__ __forceinline__ unsigned group_umin(unsigned v)
{
    if constexpr (G == 32) {
        return __reduce_min_sync(0xffffffffu, v);
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
}

template <int G>
__device__ __forceinline__ unsigned group_umax(unsigned v)
{
    if constexpr (G == 32) {
        return __reduce_max_sync(0xffffffffu, v);
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
}

// d = clamp(a*b + c, 0, 1), NaN -> 0, as one saturating FMA.
__device__ __forceinline__ float fma_sat(float a, float b, float c)
{
    float d;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// 1.0f when a >= b, else 0.0f (one compare, result as a float).
__device__ __forceinline__ float ge_flag(float a, float b)
{
    float d;
    asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// 1.0f when a <= b, else 0.0f (also 0.0f when either is NaN).
__device__ __forceinline__ float le_flag(float a, float b)
{
    float d;
    asm("set.le.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// 1.0f when a == b, else 0.0f.
__device__ __forceinline__ float eq_flag(float a, float b)
{
    float d;
    asm("set.eq.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// 4-byte asynchronous copy from global to shared memory (cp.async): the copy
// is issued without waiting for it, so a lane's staging loads are all in
// flight at once; cp_async_wait_all waits for the calling thread's copies.
__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Order-preserving map from non-NaN floats to unsigned keys (-0 sorts just
// below +0; the counts that follow compare floats, where they are equal).
__device__ __forceinline__ unsigned float_key(float f)
{
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_float(unsigned k)
{
    unsigned b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

// Load the window of tile position q into registers: slot s = glane + G*i
// holds tile[q + s] for s < W, kGap past W.  Slots are stored in pairs
// (i = 2k, 2k+1 in x[k].x, x[k].y) for the packed FP32x2 arithmetic.
// `tail_only` (uniform) says that G*(R-2) <= W, so only the last register pair
// can hold slots past W; the general path re-derives each row's limit from an
// opaque register so the compiler does not keep R loop-invariant predicates
// alive across the chain.
template <int G, int R>
__device__ __forceinline__ void load_window(float2 (&x)[R / 2], const TileRef tile, int q, int glane,
                                            int W, bool tail_only)
{
    const int base = q + glane;
    if (tail_only) {
#pragma unroll
        for (int k = 0; k < R / 2 - 1; ++k) {
            x[k].x = tile[base + G * (2 * k)];
            x[k].y = tile[base + G * (2 * k + 1)];
        }
        const float a = tile[base + G * (R - 2)];
        const float b = tile[base + G * (R - 1)];
        x[R / 2 - 1].x = (glane + G * (R - 2) < W) ? a : kGap;
        x[R / 2 - 1].y = (glane + G * (R - 1) < W) ? b : kGap;
    } else {
        int lim = W - glane;  // slot row i is valid for this lane iff G*i < lim
        asm volatile("" : "+r"(lim));
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const float a = tile[base + G * (2 * k)];
            const float b = tile[base + G * (2 * k + 1)];
            x[k].x = (G * (2 * k) < lim) ? a : kGap;
            x[k].y = (G * (2 * k + 1) < lim) ? b : kGap;
        }
    }
}

// Per-group median state carried along a chain.
struct MedianState {
    float m;   // current median (valid when `have`)
    int L;     // valid samples < m
    int E;     // samples == m
    int Gp;    // samples > m
    int nv;    // valid samples in the window
    bool have;
};

// Kernel flags: diagnostic outputs, MAD scale instead of Eq. 1.
enum : int { kFlagDiag = 1, kFlagMad = 2 };

// Narrow groups (G <= 4 lanes per window) stage their trend values in the
// warp's shared-memory slice and write trend and detrended flux at the end of
// the tile, coalesced: their 32/G groups walk chains a whole chain apart, so a
// direct store from every group would touch 32/G separate DRAM sectors with
// 4 bytes each.  The slice then holds T more floats after the staged samples.
__host__ __device__ constexpr bool stages_outputs(int G) { return G <= 4; }

template <int G, int R, int FLAGS>
__device__ __forceinline__ void process_chain(const Curve &cv, const Diag &dg, const TileRef tile,
                                              float *out, int64_t t0, int q0, int P, int glane)
{
    constexpr int S = G * R;
    const int W = cv.W;
    const int h = (W - 1) >> 1;
    const float alpha = cv.alpha;
    const float cst = cv.c;
    // Sign select of Eq. 2 through |t| (Phase 3): rho = (1 - alpha^2)/(1 +
    // alpha^2) and sigma = sqrt((1 + alpha^2)/2)/(c s).  The branch on the
    // small side is t (1 - |rho|), a difference, so rho's rounding (at most 3
    // units of roundoff) grows by (a^2 - 1)/2 there, a = max(alpha, 1/alpha).
    // This form serves 1/4 <= alpha <= 4, where u_eff^2 stays within
    // 4 + 1.5 (a^2 - 1) units of its value for the window's sigma (1.6e-6
    // relative at a = 4); every other alpha takes the min of two scaled
    // residuals.  With r = 1/sqrt(msq) (Phase 2), sigma = r k1 in that form,
    // and in the other kp = r k1, kn = alpha kp (k1 negated when alpha < 1).
    const bool abs_form = alpha >= 0.25f && alpha <= 4.f;
    const float rho = fmaf(-alpha, alpha, 1.f) / fmaf(alpha, alpha, 1.f);
    const float k1 = (abs_form ? sqrtf(0.5f * fmaf(alpha, alpha, 1.f)) : (alpha >= 1.f ? 1.f : -1.f)) /
                     (kScaleFactor * cst);
    const int iters = cv.iters;
    const bool tail_only = G * (R - 2) <= W;  // rows 0..R-3 hold only slots < W
    static_assert(R % 2 == 0, "slots are processed in pairs");
    float2 x[R / 2];
    MedianState st;
    st.m = 0.f;
    st.L = st.E = st.Gp = 0;
    st.nv = 0;
    st.have = false;

#pragma unroll 1
    for (int t = 0; t < P; ++t) {
        const int q = q0 + t;
        const int64_t p = t0 + q;

        // ---- slide: one sample leaves, one enters --------------------------
        if (t > 0) {
            const float out = tile[q - 1];
            const float in = tile[q + W - 1];
            const bool ov = out > kGapLimit;
            const bool iv = in > kGapLimit;
            st.nv += (int)iv - (int)ov;
            if (st.have) {
                if (ov) {
                    if (out < st.m) --st.L;
                    else if (out == st.m) --st.E;
                    else --st.Gp;
                }
                if (iv) {
                    if (in < st.m) ++st.L;
                    else if (in == st.m) ++st.E;
                    else ++st.Gp;
                }
            }
        }

        load_window<G, R>(x, tile, q, glane, W, tail_only);

        if (t == 0) {
            int c = 0;
#pragma unroll
            for (int k = 0; k < R / 2; ++k)
                c += ((x[k].x > kGapLimit) ? 1 : 0) + ((x[k].y > kGapLimit) ? 1 : 0);
            st.nv = group_sum_int<G>(c);
        }
        if (st.nv == 0) st.have = false;
        const int k = (st.nv - 1) >> 1;  // rank of the lower median among valid samples
        const bool need_full = (st.nv >= 1) && !st.have;
        // 0 = median unchanged, +1 = moves to the largest sample below m,
        // -1 = moves to the smallest sample above m.
        int move = 0;
        if (st.have) {
            if (k < st.L) move = 1;
            else if (k >= st.L + st.E) move = -1;
        }

        // ---- exact selection by key bisection (chain start / restart) -------
        if (__any_sync(0xffffffffu, need_full)) {
            // Binary search over the integer keys for the key of rank
            // `target` among the S slots (slots past W and missing samples
            // hold kGap, whose key sorts below every sample's), over the
            // window just loaded into registers: the smallest key v with
            // more than `target` slots at or below it, which is always a
            // sample's key.  It bisects the interval [min, max] of the valid
            // samples' keys, so it takes ceil(log2(max - min + 1)) passes (a
            // window of flux around 1.0, whose keys differ from bit 23 on
            // because 1.0 starts a binade, spans only about 2^17 keys).
            // With few slots per lane the keys are computed once into
            // registers; otherwise each pass compares the slots' floats with
            // the midpoint's float, which needs no key array: between two
            // finite keys every key is a finite float, and key order is
            // float order except that -0 sorts below +0, which can only
            // change the sign of a zero median, never its value or the counts
            // that follow.
            constexpr bool kRegKeys = R <= 12;
            unsigned key[kRegKeys ? R : 1];
            unsigned lo = 0xffffffffu, hi = 0u;
#pragma unroll
            for (int k2 = 0; k2 < R / 2; ++k2) {
                const unsigned ka = float_key(x[k2].x), kb = float_key(x[k2].y);
                if constexpr (kRegKeys) {
                    key[2 * k2] = ka;
                    key[2 * k2 + 1] = kb;
                }
                if (x[k2].x > kGapLimit) {
                    lo = min(lo, ka);
                    hi = max(hi, ka);
                }
                if (x[k2].y > kGapLimit) {
                    lo = min(lo, kb);
                    hi = max(hi, kb);
                }
            }
            lo = group_umin<G>(lo);
            hi = group_umax<G>(hi);
            const int target = (S - st.nv) + k;  // rank among all S slots
#pragma unroll 1
            while (__any_sync(0xffffffffu, need_full && lo < hi)) {
                const unsigned mid = lo + ((hi - lo) >> 1);
                int c = 0;
                if constexpr (kRegKeys) {
#pragma unroll
                    for (int i = 0; i < R; ++i) c += (key[i] <= mid) ? 1 : 0;
                } else {
                    const float midf = key_float(mid);
                    if constexpr (R >= 32) {
                        // 0/1 float flags summed with FADD2 (exact: at most R < 2^24),
                        // so half of a long pass runs on the FMA pipe.
                        // Two accumulators (even and odd pairs) halve the
                        // dependent chain; the count is exact in any order.
                        float2 cf0 = make_float2(0.f, 0.f), cf1 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k2 = 0; k2 < R / 2; ++k2) {
                            const float2 fl = make_float2(le_flag(x[k2].x, midf), le_flag(x[k2].y, midf));
                            if (k2 & 1) cf1 = __fadd2_rn(cf1, fl);
                            else cf0 = __fadd2_rn(cf0, fl);
                        }
                        c = (int)((cf0.x + cf0.y) + (cf1.x + cf1.y));
                    } else {
#pragma unroll
                        for (int k2 = 0; k2 < R / 2; ++k2)
                            c += ((x[k2].x <= midf) ? 1 : 0) + ((x[k2].y <= midf) ? 1 : 0);
                    }
                }
                c = group_sum_int<G>(c);
                if (c > target) hi = mid;
                else lo = mid + 1;
            }
            const float mf = key_float(lo);
            int cl = 0, ce = 0;
#pragma unroll
            for (int k = 0; k < R / 2; ++k) {
                cl += ((x[k].x < mf) ? 1 : 0) + ((x[k].y < mf) ? 1 : 0);
                ce += ((x[k].x == mf) ? 1 : 0) + ((x[k].y == mf) ? 1 : 0);
            }
            cl = group_sum_int<G>(cl);
            ce = group_sum_int<G>(ce);
            if (need_full) {
                st.m = mf;
                st.L = cl - (S - st.nv);
                st.E = ce;
                st.Gp = st.nv - st.L - st.E;
                st.have = true;
            }
        }

        // ---- one-rank move of the median -----------------------------------
        if (__any_sync(0xffffffffu, move != 0)) {
            // The two passes are built so that half their work runs on the
            // FMA pipe, which is otherwise idle here: a 0/1 float flag marks
            // slots at or above sm, one FFMA2 pushes them 2^127 down (slots
            // below keep their exact value), and ties are counted as float
            // sums of 0/1 flags (exact: at most S < 2^24).
            const float sg = (move < 0) ? -1.f : 1.f;
            const float2 sg2 = make_float2(sg, sg);
            const float sm = sg * st.m;
            const float2 push = make_float2(-0x1p127f, -0x1p127f);
            // Even and odd pairs keep separate maxima and tie counts (exact in
            // any order), which halves the dependent chains of both scans.
            float best0 = -INFINITY, best1 = -INFINITY;
#pragma unroll
            for (int k = 0; k < R / 2; ++k) {
                const float2 y = __fmul2_rn(x[k], sg2);
                const float2 f = make_float2(ge_flag(y.x, sm), ge_flag(y.y, sm));
                const float2 yb = __ffma2_rn(f, push, y);
                if (k & 1) best1 = fmaxf(best1, fmaxf(yb.x, yb.y));
                else best0 = fmaxf(best0, fmaxf(yb.x, yb.y));
            }
            float best = group_max<G>(fmaxf(best0, best1));
            const float cand = sg * best;
            float2 ef0 = make_float2(0.f, 0.f), ef1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < R / 2; ++k) {
                const float2 fl = make_float2(eq_flag(x[k].x, cand), eq_flag(x[k].y, cand));
                if (k & 1) ef1 = __fadd2_rn(ef1, fl);
                else ef0 = __fadd2_rn(ef0, fl);
            }
            const int e = group_sum_int<G>((int)((ef0.x + ef0.y) + (ef1.x + ef1.y)));
            if (move > 0) {
                st.Gp += st.E;
                st.L -= e;
                st.E = e;
                st.m = cand;
            } else if (move < 0) {
                st.L += st.E;
                st.Gp -= e;
                st.E = e;
                st.m = cand;
            }
        }

        // ---- Phases 2 and 3 -------------------------------------------------
        const float centre = tile[q + h];
        const bool produce = (p < cv.n) && (st.nv >= 1) && (st.nv >= cv.min_valid) &&
                             (centre > kGapLimit);
        float mu = st.m;
        float s = 0.f;
        if (__any_sync(0xffffffffu, produce)) {
            const float m = st.m;
            const float2 negm = make_float2(-m, -m);
            float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < R / 2; ++k) {
                x[k] = __fadd2_rn(x[k], negm);  // y = x - m, exact sign
                const float2 yp = make_float2(fmaxf(x[k].x, 0.f), fmaxf(x[k].y, 0.f));
                s2 = __ffma2_rn(yp, yp, s2);
            }
            const float s2sum = group_sum<G>(s2.x + s2.y);
            // msq = S2 / n+ and s = 0.6745 sqrt(msq) (Eq. 1).  The iterations
            // take 1/(c s) as rsqrt(msq) / (0.6745 c): a fast quotient and an
            // approximate reciprocal square root, 2 ulp each, far below what
            // the trend resolves, in place of an IEEE quotient, root and
            // reciprocal.  A subnormal mean square takes the IEEE root.
            const float msq = (st.Gp > 0) ? __fdividef(s2sum, (float)st.Gp) : 0.f;
            s = kScaleFactor * sqrtf(msq);  // for the diagnostic output
            if constexpr ((FLAGS & kFlagMad) != 0) {
                // MAD = the order statistic of rank floor((nv-1)/2) of |y| over
                // the valid slots, by bisection on the bit patterns of
                // non-negative floats (their order as unsigned integers).
                // Gap slots have |y| near 2^100 and sort above every candidate.
                float hi = 0.f;
#pragma unroll
                for (int k = 0; k < R / 2; ++k) {
                    const float a = fabsf(x[k].x), b = fabsf(x[k].y);
                    hi = fmaxf(hi, a < 0x1p98f ? a : 0.f);
                    hi = fmaxf(hi, b < 0x1p98f ? b : 0.f);
                }
                hi = group_max<G>(hi);
                const unsigned hk = __float_as_uint(hi);
                const int nbits = hk ? 32 - __clz((int)hk) : 0;
                const int nb = (int)__reduce_max_sync(0xffffffffu, (unsigned)(produce ? nbits : 0));
                const int target = (st.nv - 1) >> 1;
                unsigned res = 0u;
#pragma unroll 1
                for (int b = nb - 1; b >= 0; --b) {
                    const float cand = __uint_as_float(res | (1u << b));
                    int c = 0;
#pragma unroll
                    for (int k = 0; k < R / 2; ++k)
                        c += ((fabsf(x[k].x) < cand) ? 1 : 0) + ((fabsf(x[k].y) < cand) ? 1 : 0);
                    c = group_sum_int<G>(c);
                    if (c <= target) res |= (1u << b);
                }
                s = __uint_as_float(res);
            }
            const bool iterate = produce && ((FLAGS & kFlagMad) != 0 ? (s > 0.f) : (msq > 0.f));
            if (__any_sync(0xffffffffu, iterate)) {
                // Eq. 2 needs only u_eff^2 = k^2 (y - delta)^2 with k = kp =
                // 1/(c s) above the trend and k = kn = alpha/(c s) below it.
                // Eq. 4 in centred form: delta_new = sum(w y)/sum(w), since
                // mu = m + delta.
                float r;  // 0.6745 / s
                if constexpr ((FLAGS & kFlagMad) != 0) r = kScaleFactor / s;
                else r = (msq >= 0x1p-126f) ? rsqrtf(msq) : 1.f / sqrtf(msq);
                float delta = 0.f;
                if (abs_form) {
                    // t = sigma (y - delta), sigma^2 = (kp^2 + kn^2)/2:
                    // t (t + rho |t|) = kp^2 u^2 for u >= 0, kn^2 u^2 for u < 0,
                    // so one FMA with |t| as an operand does the sign select.
                    const float sg = r * k1;
                    const float2 sg2 = make_float2(sg, sg);
                    const float2 rho2 = make_float2(rho, rho);
#pragma unroll 1
                    for (int it = 0; it < iters; ++it) {
                        const float2 c0 = make_float2(-delta * sg, -delta * sg);
                        float2 swt = make_float2(0.f, 0.f), swyt = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < R / 2; ++k) {
                            const float2 ts = __ffma2_rn(x[k], sg2, c0);
                            // t + rho |t| per slot: one FFMA2 with |t| as its
                            // operand, or two scalar FMAs (the same value
                            // either way); the scalar pair schedules better
                            // in the 8-lane variants (0.25 % on 1000 TESS
                            // curves), the packed form in the others (3.3 % on
                            // the 32-lane W = 2161 batch).
                            float2 v;
                            if constexpr (G != 8) {
                                v = __ffma2_rn(rho2, make_float2(fabsf(ts.x), fabsf(ts.y)), ts);
                            } else {
                                v = make_float2(fmaf(rho, fabsf(ts.x), ts.x), fmaf(rho, fabsf(ts.y), ts.y));
                            }
                            const float2 z = make_float2(fma_sat(-ts.x, v.x, 1.f), fma_sat(-ts.y, v.y, 1.f));
                            if constexpr (G == 1) {
                                // sum z^2 and sum z (z y): the same three
                                // packed instructions, scheduled 1.6 % faster
                                // in the one-lane variants (the W = 25 band)
                                // and 1 % slower in the others.
                                const float2 zy = __fmul2_rn(z, x[k]);
                                swt = __ffma2_rn(z, z, swt);
                                swyt = __ffma2_rn(z, zy, swyt);
                            } else {
                                const float2 w = __fmul2_rn(z, z);
                                swt = __fadd2_rn(swt, w);
                                swyt = __ffma2_rn(w, x[k], swyt);
                            }
                        }
                        const float sws = group_sum<G>(swt.x + swt.y);
                        const float swys = group_sum<G>(swyt.x + swyt.y);
                        // sws <= S, so the fast quotient (2 ulp) is safe here;
                        // its error is far below the FP32 rounding of the sums.
                        if (sws > 0.f) delta = __fdividef(swys, sws);
                    }
                } else {
                    // u_eff = min(y kp - delta kp, y kn - delta kn) when
                    // alpha >= 1 (max when alpha < 1; negating both keeps one
                    // code path).
                    const float kp = r * k1;
                    const float kn = alpha * kp;
                    const float2 kp2 = make_float2(kp, kp);
                    const float2 kn2 = make_float2(kn, kn);
#pragma unroll 1
                    for (int it = 0; it < iters; ++it) {
                        const float2 c1 = make_float2(-delta * kp, -delta * kp);
                        const float2 c2 = make_float2(-delta * kn, -delta * kn);
                        float2 swt = make_float2(0.f, 0.f), swyt = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < R / 2; ++k) {
                            const float2 p1 = __ffma2_rn(x[k], kp2, c1);
                            const float2 p2 = __ffma2_rn(x[k], kn2, c2);
                            const float qa = fminf(p1.x, p2.x);
                            const float qb = fminf(p1.y, p2.y);
                            const float2 z = make_float2(fma_sat(-qa, qa, 1.f), fma_sat(-qb, qb, 1.f));
                            const float2 w = __fmul2_rn(z, z);
                            swt = __fadd2_rn(swt, w);
                            swyt = __ffma2_rn(w, x[k], swyt);
                        }
                        const float sws = group_sum<G>(swt.x + swt.y);
                        const float swys = group_sum<G>(swyt.x + swyt.y);
                        if (sws > 0.f) delta = __fdividef(swys, sws);
                    }
                }
                if (iterate) mu = m + delta;
            }
        }

        if (glane == 0 && p < cv.n) {
            const float nanv = __int_as_float(0x7fc00000);
            if constexpr (stages_outputs(G)) {
                out[q] = produce ? mu : nanv;  // written out by the tile's flush
            } else {
                cv.trend[p] = produce ? mu : nanv;
                cv.detr[p] = produce ? __fdiv_rn(centre, mu) : nanv;
            }
            if constexpr ((FLAGS & kFlagDiag) != 0) {
                if (dg.median) dg.median[p] = (st.nv >= 1) ? st.m : nanv;
                if (dg.nvalid) dg.nvalid[p] = st.nv;
                if (dg.nplus) dg.nplus[p] = (st.nv >= 1) ? st.Gp : 0;
                if (dg.scale) dg.scale[p] = produce ? s : nanv;
            }
        }
    }
}

// Work items belong to warps: each warp stages its own tile of T = (32/G)*P
// positions (plus the S-1 halo samples) in its slice of shared memory, so no
// CTA-wide barrier is ever needed.  Without a queue, warp w of CTA b takes
// item b*warps + w; with a queue, each warp pulls items until none is left.
// Dynamic shared memory: warps * (T + S - 1) floats, plus warps * T for the
// staged trend when stages_outputs(G).  MINB (CTAs of 256
// threads per SM) sets the register budget the compiler aims for.  FLAGS
// selects the diagnostic outputs and the MAD scale; every curve of one launch
// must have the scale mode the kernel was built for.
template <int G, int R, int MINB, int FLAGS>
__global__ void __launch_bounds__(256, MINB) umi_tile_kernel(LaunchArgs a)
{
    extern __shared__ float smem[];
    constexpr int S = G * R;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int n_warps = blockDim.x >> 5;
    const int glane = lane & (G - 1);
    const int group = lane / G;
    const int P = a.chain;
    const int T = (32 / G) * P;
    const int tile_len = T + S - 1;
    const int slice_len = tile_len + (stages_outputs(G) ? T : 0);
    float *tile = smem + (size_t)warp * slice_len;
    float *out = tile + tile_len;  // staged trend of the tile's positions (narrow groups)
#ifdef UMI_CHECKED
    {
        unsigned dsm;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
        if ((uint64_t)n_warps * (uint64_t)slice_len * sizeof(float) > dsm) {
            if (threadIdx.x == 0 && a.check) atomicOr(a.check, kCheckSmemSize);
            return;
        }
    }
    const TileRef tref{tile, tile_len, a.check};
#else
    const TileRef tref{tile};
#endif

    int item = blockIdx.x * n_warps + warp;
    for (;;) {
        if (a.queue) {
            int v = 0;
            if (lane == 0) v = atomicAdd(a.queue, 1);
            item = __shfl_sync(0xffffffffu, v, 0);
        }
        if (item >= a.n_items) break;
        const Item wi = a.items ? a.items[item] : Item{0, item};
#ifdef UMI_CHECKED
        if (a.curves && (wi.curve < 0 || wi.curve >= a.n_curves)) {
            if (lane == 0 && a.check) atomicOr(a.check, kCheckCurveIndex);
            if (!a.queue) break;
            continue;
        }
#endif
        const Curve cv = a.curves ? a.curves[wi.curve] : a.single;
        const int64_t t0 = (int64_t)wi.tile * T;
        const int h = (cv.W - 1) >> 1;
#ifdef UMI_CHECKED
        if (wi.tile < 0 || t0 >= (cv.n > 0 ? cv.n : 1)) {
            if (lane == 0 && a.check) atomicOr(a.check, kCheckItemTile);
            if (!a.queue) break;
            continue;
        }
#endif

        // Stage with asynchronous 4-byte copies (no alignment beyond the
        // float's), then turn the non-finite samples each lane copied into
        // the gap marker; slots outside the curve get it directly.
        for (int k = lane; k < tile_len; k += 32) {
            const int64_t idx = t0 - h + k;
            if (idx >= 0 && idx < cv.n) cp_async4(tile + k, cv.flux + idx);
            else tile[k] = kGap;
        }
        cp_async_wait_all();
        for (int k = lane; k < tile_len; k += 32)
            if (!isfinite(tile[k])) tile[k] = kGap;
        __syncwarp();
        process_chain<G, R, FLAGS>(cv, a.diag, tref, out, t0, group * P, P, glane);
        __syncwarp();  // every lane is done with the tile before it is restaged
        if constexpr (stages_outputs(G)) {
            // Flush: position k of the tile has its sample at tile[k + h];
            // a NaN trend (no estimate) gives a NaN quotient too.
            const float nanv = __int_as_float(0x7fc00000);
            const int kend = (int)min((int64_t)T, cv.n - t0);
            for (int k = lane; k < kend; k += 32) {
                const float mu = out[k];
                cv.trend[t0 + k] = mu;
                cv.detr[t0 + k] = (mu == mu) ? __fdiv_rn(tref[k + h], mu) : nanv;
            }
            __syncwarp();  // the flush reads the tile: done before it is restaged
        }
        if (!a.queue) break;
    }
}

}  // namespace umi
