// One integration of host-resident voltages through the whole cycle of the
// paper's Fig. 1 (FFT-correlator, reduced X-engine, calibration), streamed
// channel chunk by channel chunk: the host->device copy of chunk i+1 (on the
// context's copy stream) overlaps the correlator and X-engine kernels of
// chunk i (on the caller's stream); with three staging buffers a copy can
// run two chunks ahead, so a host link about as fast as the kernels still
// stays hidden.  The first chunk is a quarter of the
// others, so that little copy time is exposed before the first kernel; the
// calibration is one launch over all channels at the end (the kernels share
// one stream, so splitting it would only leave partial waves of CTAs).
// Gains in host memory are copied on the copy stream too, ahead of the
// first chunk, into one of two device buffers used by alternate calls, so
// that no voltage copy ever waits behind a copy queued on the caller's
// stream or behind the previous call's last kernels.  Host code only:
// every step is one of the library's own kernels.
#include <algorithm>
#include <vector>

#include "gc_sel.h"

namespace {

size_t esz_of(int vfmt) { return vfmt == GC_C64 ? 8 : (vfmt == GC_C32H ? 4 : 1); }

gc_status ensure_streaming(gc_ctx *ctx, size_t stage_bytes) {
    cudaError_t e;
    if (!ctx->copy_stream) {
        e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaStreamCreate(copy)");
        for (int b = 0; b < GC_NSTAGE; ++b) {
            if ((e = cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&ctx->ev_free[b], cudaEventDisableTiming)) != cudaSuccess)
                return gc_cuda_fail(ctx, e, "cudaEventCreate");
        }
        if ((e = cudaEventCreateWithFlags(&ctx->ev_gains_copied, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ctx->ev_gains_free[0], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ctx->ev_gains_free[1], cudaEventDisableTiming)) != cudaSuccess)
            return gc_cuda_fail(ctx, e, "cudaEventCreate");
    }
    if (stage_bytes > ctx->stage_bytes) {
        // the old buffers may still be read by queued kernels
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaDeviceSynchronize before staging growth");
        for (int b = 0; b < GC_NSTAGE; ++b) {
            if (ctx->stage[b]) cudaFree(ctx->stage[b]);
            ctx->stage[b] = nullptr;
        }
        ctx->stage_bytes = 0;
        for (int b = 0; b < GC_NSTAGE; ++b) {
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

// Whether p is host memory (page-locked or pageable) rather than device memory.
bool is_host_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;   // not known to the runtime: ordinary pageable memory
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
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
    const size_t vr_pair_bytes = 8;   // float2 sums or int2 exact sums per pair
    const size_t au_bytes = 4;
    // chunk boundaries: a short first chunk, then full ones
    std::vector<int> bounds{0};
    if (chunk < C) bounds.push_back(std::max(1, chunk / 4));
    while (bounds.back() < C) bounds.push_back(std::min(C, bounds.back() + chunk));
    const int n_chunks = (int)bounds.size() - 1;
    const char *h = static_cast<const char *>(h_volt);
    // host-resident gains: copied on the copy stream ahead of the first
    // chunk, into one of two context buffers (alternate calls), so that the
    // copy waits only for the correlator kernels of the call before the
    // previous one -- never for this call's predecessor, whose last chunks
    // may still be running; the correlator waits for the copy
    const float *gains_d = gains_in;
    int gslot = -1;
    if (is_host_pointer(gains_in)) {
        const size_t gb = (size_t)C * N * 2 * sizeof(float);
        if (gb > ctx->gains_bytes) {
            if ((e = cudaDeviceSynchronize()) != cudaSuccess) return gc_cuda_fail(ctx, e, "synchronize before growth");
            for (int b = 0; b < 2; ++b) {
                if (ctx->gains_dev[b]) cudaFree(ctx->gains_dev[b]);
                ctx->gains_dev[b] = nullptr;
            }
            ctx->gains_bytes = 0;
            for (int b = 0; b < 2; ++b)
                if ((e = cudaMalloc(&ctx->gains_dev[b], gb)) != cudaSuccess) {
                    cudaGetLastError();
                    return gc_cuda_fail(ctx, e, "cudaMalloc(gains)");
                }
            ctx->gains_bytes = gb;
        }
        gslot = ctx->gains_slot;
        ctx->gains_slot ^= 1;
        if ((e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_gains_free[gslot], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ctx->gains_dev[gslot], gains_in, gb, cudaMemcpyHostToDevice, ctx->copy_stream)) !=
                cudaSuccess ||
            (e = cudaEventRecord(ctx->ev_gains_copied, ctx->copy_stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, ctx->ev_gains_copied, 0)) != cudaSuccess)
            return gc_cuda_fail(ctx, e, "copy the gains");
        gains_d = static_cast<const float *>(ctx->gains_dev[gslot]);
    }
    for (int i = 0; i < n_chunks; ++i) {
        const int b = i % GC_NSTAGE;
        const int c0 = bounds[i], cc = bounds[i + 1] - c0;
        // a staging buffer is refilled once the last kernel that read it --
        // of this call, or of the previous call for the first two chunks --
        // is done, so the next integration's first copies overlap this one's
        // calibration (an event never recorded makes the wait a no-op)
        if ((e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[b], 0)) != cudaSuccess)
            return gc_cuda_fail(ctx, e, "wait for a free staging buffer");
        const int rec = gc_prof_begin(ctx, ctx->copy_stream, "h2d_chunk");
        e = cudaMemcpyAsync(ctx->stage[b], h + (size_t)c0 * per_ch, (size_t)cc * per_ch, cudaMemcpyHostToDevice,
                            ctx->copy_stream);
        gc_prof_end(ctx, ctx->copy_stream, rec);
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaMemcpyAsync(voltages)");
        if ((e = cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, ctx->ev_copied[b], 0)) != cudaSuccess)
            return gc_cuda_fail(ctx, e, "order the chunk copy");
        st = gc_correlate(ctx, ctx->stage[b], vfmt, L, cc, T, gains_d + (size_t)c0 * N * 2,
                          vunique + (size_t)c0 * W * W * 2, stream);
        if (st != GC_OK) return st;
        st = gc_reduce(ctx, ctx->stage[b], vfmt, L, cc, T, sel,
                       static_cast<char *>(vreduced) + (size_t)c0 * sel->P * vr_pair_bytes,
                       autos ? static_cast<char *>(autos) + (size_t)c0 * N * au_bytes : nullptr, stream);
        if (st != GC_OK) return st;
        if ((e = cudaEventRecord(ctx->ev_free[b], s)) != cudaSuccess)
            return gc_cuda_fail(ctx, e, "record staging release");
    }
    if (gslot >= 0 && (e = cudaEventRecord(ctx->ev_gains_free[gslot], s)) != cudaSuccess)
        return gc_cuda_fail(ctx, e, "record gains release");
    const int cfmt = vfmt == GC_I4C ? GC_I4C : GC_C64;   // X-engine output format
    return gc_calibrate(ctx, vreduced, cfmt, sel, C, autos, opts, gains_out, vmodel, stats, stream);
}
