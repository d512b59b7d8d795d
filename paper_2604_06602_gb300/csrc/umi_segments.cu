// umi_segments.cu -- gap handling before the detrend.
//
// The paper lists gap handling as the pipeline step before detrending
// (Table 3's caption) and scales the minimum segment length to W/3
// (Section 4, Kepler Long-Cadence).  Reading used here: a curve splits at
// every run of at least `gap_min` consecutive missing samples (default W);
// leading and trailing missing runs belong to no segment; a segment with
// fewer than `min_seg` valid samples (default floor(W/3)) is dropped.  Each
// kept segment is detrended as a curve of its own, so no window reaches
// across a split, and positions outside kept segments get NaN.
//
// Device side: one ballot kernel packs the validity of every sample into a
// bitmask (1 bit per sample).  Host side: the bitmask comes back and runs of
// missing samples are found a 32-bit word at a time; the kept segments form
// the curve table of one batched launch (umi_api.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "umi_host.h"
#include "umi_internal.h"

namespace umi {

// bits[w] bit b = flux[32 w + b] is finite (bits past `total` are 0).
__global__ void validity_bits_kernel(const float *__restrict__ flux, int64_t total,
                                     unsigned *__restrict__ bits)
{
    const int64_t words = (total + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; w < words;
         w += ((int64_t)gridDim.x * blockDim.x) / 32) {
        const int64_t i = w * 32 + lane;
        const bool ok = i < total && isfinite(flux[i]);
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) bits[w] = b;
    }
}


umi_status detrend_segmented(const float *flux, const int64_t *offsets, const int32_t *W, int32_t B,
                             const umi_params *params, const umi_segment_params *seg, float *trend,
                             float *detr, int64_t *segments_out, cudaStream_t stream)
{
    NvtxRange nvtx("umi detrend segmented");
    clear_error();
    if (segments_out) *segments_out = 0;
    umi_params p;
    umi_status st = check_params(params, &p);
    if (st != UMI_OK) return st;
    umi_segment_params sp;
    umi_default_segment_params(&sp);
    if (seg) sp = *seg;
    if (B < 0) return fail(UMI_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return UMI_OK;
    if (!offsets || !W) return fail(UMI_ERR_INVALID_ARG, "null offsets or W");
    if (offsets[0] != 0) return fail(UMI_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int32_t b = 0; b < B; ++b) {
        if (offsets[b + 1] < offsets[b]) return fail(UMI_ERR_INVALID_ARG, "offsets must be non-decreasing");
        if (W[b] < 1 || (W[b] % 2) == 0 || W[b] > umi_max_window())
            return fail(UMI_ERR_INVALID_ARG, "W[" + std::to_string(b) + "] must be odd and in range");
    }
    const int64_t total = offsets[B];
    if (total == 0) return UMI_OK;
    if (!flux || !trend || !detr) return fail(UMI_ERR_INVALID_ARG, "null buffer");

    const int64_t words = (total + 31) / 32;
    unsigned *dbits = nullptr;
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync((void **)&dbits, sizeof(unsigned) * (size_t)words, stream);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMallocAsync (validity bits)");
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((words * 32 + threads - 1) / threads, 1 << 16);
    validity_bits_kernel<<<(int)blocks, threads, 0, stream>>>(flux, total, dbits);
    std::vector<unsigned> hbits((size_t)words);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hbits.data(), dbits, sizeof(unsigned) * (size_t)words,
                            cudaMemcpyDeviceToHost, stream);
    cudaFreeAsync(dbits, stream);
    // NaN everywhere first; kept segments are overwritten by the batch below.
    if (e == cudaSuccess) e = cudaMemsetAsync(trend, 0xff, sizeof(float) * (size_t)total, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(detr, 0xff, sizeof(float) * (size_t)total, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail_cuda(e, "segment scan");

    Bits bits{hbits.data()};
    // Segments are planned from the whole curves' bands, as the plain batched
    // call would plan them.
    BandSizes sizes;
    for (int32_t b = 0; b < B; ++b)
        sizes[std::make_pair((int)W[b], p.scale_mode)] += offsets[b + 1] - offsets[b];
    std::vector<Curve> curves;
    std::vector<Segment> segs;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t o = offsets[b], n = offsets[b + 1] - offsets[b];
        if (n == 0) continue;
        const int64_t gap_min = sp.gap_min > 0 ? sp.gap_min : W[b];
        const int64_t min_seg = sp.min_seg >= 0 ? sp.min_seg : W[b] / 3;
        segs.clear();
        find_segments(bits, o, n, gap_min, min_seg, &segs);
        for (const Segment &sg : segs) {
            Curve c;
            c.flux = flux + o + sg.start;
            c.trend = trend + o + sg.start;
            c.detr = detr + o + sg.start;
            c.n = sg.len;
            c.W = W[b];
            c.min_valid = resolve_min_valid(W[b], p.min_valid);
            c.alpha = p.alpha;
            c.c = p.c;
            c.iters = p.iters;
            c.scale_mode = p.scale_mode;
            curves.push_back(c);
        }
    }
    if (segments_out) *segments_out = (int64_t)curves.size();
    int launches = 0;
    st = launch_curve_table(curves, stream, &launches, &sizes);
    count_launches(launches + 1);
    return st;
}

}  // namespace umi

extern "C" {

void umi_default_segment_params(umi_segment_params *sp)
{
    if (!sp) return;
    sp->gap_min = 0;
    sp->min_seg = -1;
}

umi_status umi_detrend_segmented(const float *flux_d, const int64_t *offsets_h, const int32_t *W_h,
                                 int32_t B, const umi_params *params, const umi_segment_params *seg,
                                 float *trend_d, float *detr_d, int64_t *segments_out, void *stream)
{
    return umi::detrend_segmented(flux_d, offsets_h, W_h, B, params, seg, trend_d, detr_d,
                                  segments_out, (cudaStream_t)stream);
}

}  // extern "C"
