// One integration of host-resident voltages through the whole cycle of the
// paper's Fig. 1 (FFT-correlator, reduced X-engine, calibration), streamed
// channel chunk by channel chunk: the host->device copy of chunk i+1 (on the
// context's copy stream) overlaps the correlator and X-engine kernels of
// chunk i (on the caller's stream); calibration runs on groups of chunks as
// their V^reduced complete, so that each launch still fills the GPU.
// Host code only: every step is one of the library's own kernels.
#include <algorithm>

#include "gc_sel.h"

namespace {

size_t esz_of(int vfmt) { return vfmt == GC_C64 ? 8 : (vfmt == GC_C32H ? 4 : 1); }

gc_status ensure_streaming(gc_ctx *ctx, size_t stage_bytes) {
    cudaError_t e;
    if (!ctx->copy_stream) {
        e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaStreamCreate(copy)");
        for (int b = 0; b < 2; ++b) {
            if ((e = cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&ctx->ev_free[b], cudaEventDisableTiming)) != cudaSuccess)
                return gc_cuda_fail(ctx, e, "cudaEventCreate");
        }
        e = cudaEventCreateWithFlags(&ctx->ev_entry, cudaEventDisableTiming);
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaEventCreate");
    }
    if (stage_bytes > ctx->stage_bytes) {
        // the old buffers may still be read by queued kernels
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaDeviceSynchronize before staging growth");
        for (int b = 0; b < 2; ++b) {
            if (ctx->stage[b]) cudaFree(ctx->stage[b]);
            ctx->stage[b] = nullptr;
        }
        ctx->stage_bytes = 0;
        for (int b = 0; b < 2; ++b) {
            e = cudaMalloc(&ctx->stage[b], stage_bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return gc_cuda_fail(ctx, e, "cudaMalloc(staging)");
            }
        }
        ctx->stage_bytes = stage_bytes;
    }
    return GC_OK;
}

}  // namespace

extern "C" gc_status gc_integrate_host(gc_ctx *ctx, const void *h_volt, int vfmt, int L, int C, int T,
                                       const gc_sel *sel, const float *gains_in, float *vunique, void *vreduced,
                                       void *autos, const gc_calopts *opts, float *gains_out, float *vmodel,
                                       gc_calstats *stats, int chunk, void *stream) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    if (!h_volt || !sel || !gains_in || !vunique || !vreduced || !gains_out || !vmodel || !stats)
        return gc_fail(ctx, GC_EINVAL, "gc_integrate_host: null argument");
    if (vfmt != GC_C64 && vfmt != GC_I4C && vfmt != GC_C32H)
        return gc_fail(ctx, GC_EINVAL, "gc_integrate_host: unknown voltage format");
    if (L != sel->L || C < 1 || T < sel->T || chunk < 0)
        return gc_fail(ctx, GC_EINVAL, "gc_integrate_host: sizes do not match the selection");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    const int N = L * L, W = 2 * L - 1;
    const size_t per_ch = (size_t)T * N * esz_of(vfmt);
    // default chunk: eight chunks, at least 16 channels each
    if (chunk == 0) chunk = std::min(C, std::max(16, (C + 7) / 8));
    chunk = std::min(chunk, C);
    gc_status st = ensure_streaming(ctx, (size_t)chunk * per_ch);
    if (st != GC_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // calibration groups: whole chunks, about two resident CTAs per SM's worth
    const int cal_group = std::max(1, (2 * ctx->sm_count + chunk - 1) / chunk);
    // the staging buffers may still be read by work queued earlier on `stream`
    if ((e = cudaEventRecord(ctx->ev_entry, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_entry, 0)) != cudaSuccess)
        return gc_cuda_fail(ctx, e, "order the copy stream");
    const size_t vr_pair_bytes = 8;   // float2 sums or int2 exact sums per pair
    const size_t au_bytes = 4;
    const int n_chunks = (C + chunk - 1) / chunk;
    int cal_from = 0;
    const char *h = static_cast<const char *>(h_volt);
    for (int i = 0; i < n_chunks; ++i) {
        const int b = i & 1;
        const int c0 = i * chunk, cc = std::min(chunk, C - c0);
        if (i >= 2 && (e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[b], 0)) != cudaSuccess)
            return gc_cuda_fail(ctx, e, "wait for a free staging buffer");
        e = cudaMemcpyAsync(ctx->stage[b], h + (size_t)c0 * per_ch, (size_t)cc * per_ch, cudaMemcpyHostToDevice,
                            ctx->copy_stream);
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaMemcpyAsync(voltages)");
        if ((e = cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, ctx->ev_copied[b], 0)) != cudaSuccess)
            return gc_cuda_fail(ctx, e, "order the chunk copy");
        st = gc_correlate(ctx, ctx->stage[b], vfmt, L, cc, T, gains_in + (size_t)c0 * N * 2,
                          vunique + (size_t)c0 * W * W * 2, stream);
        if (st != GC_OK) return st;
        st = gc_reduce(ctx, ctx->stage[b], vfmt, L, cc, T, sel,
                       static_cast<char *>(vreduced) + (size_t)c0 * sel->P * vr_pair_bytes,
                       autos ? static_cast<char *>(autos) + (size_t)c0 * N * au_bytes : nullptr, stream);
        if (st != GC_OK) return st;
        if ((e = cudaEventRecord(ctx->ev_free[b], s)) != cudaSuccess)
            return gc_cuda_fail(ctx, e, "record staging release");
        if ((i + 1) % cal_group == 0 || i + 1 == n_chunks) {
            const int c1 = c0 + cc, n = c1 - cal_from;
            const int cfmt = vfmt == GC_I4C ? GC_I4C : GC_C64;   // X-engine output format
            st = gc_calibrate(ctx, static_cast<const char *>(vreduced) + (size_t)cal_from * sel->P * vr_pair_bytes,
                              cfmt, sel, n,
                              autos ? static_cast<const char *>(autos) + (size_t)cal_from * N * au_bytes : nullptr,
                              opts, gains_out + (size_t)cal_from * N * 2, vmodel + (size_t)cal_from * sel->n_ubl * 2,
                              stats + cal_from, stream);
            if (st != GC_OK) return st;
            cal_from = c1;
        }
    }
    return GC_OK;
}
