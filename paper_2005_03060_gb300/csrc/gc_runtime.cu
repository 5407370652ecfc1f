// Context, errors, workspace and tensor-map encoding for the gridcorr C ABI.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "gc_internal.h"

gc_status gc_fail(gc_ctx *ctx, gc_status st, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

gc_status gc_cuda_fail(gc_ctx *ctx, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return gc_fail(ctx, GC_ENOMEM, m);
    return gc_fail(ctx, GC_ECUDA, m);
}

bool gc_aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

gc_status gc_scratch_reserve(gc_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->scratch_bytes) return GC_OK;
    // the old buffer may still be read by kernels queued on any stream
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaDeviceSynchronize before workspace growth");
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    size_t want = bytes + bytes / 8;   // grow with a margin
    e = cudaMalloc(&ctx->scratch, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return gc_cuda_fail(ctx, e, "cudaMalloc(workspace)");
    }
    ctx->scratch_bytes = want;
    return GC_OK;
}

gc_status gc_encode_tiled(gc_ctx *ctx, CUtensorMap *map, CUtensorMapDataType dt, int rank, void *base,
                          const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box) {
    using Fn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                            const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                            CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                            CUtensorMapFloatOOBfill);
    if (!ctx->encode_tiled) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return gc_fail(ctx, GC_ECUDA, "cuTensorMapEncodeTiled entry point not available");
        ctx->encode_tiled = fn;
    }
    cuuint64_t gdim[5], gstr[4];
    cuuint32_t bdim[5], estr[5];
    for (int i = 0; i < rank; ++i) {
        gdim[i] = dims[i];
        bdim[i] = box[i];
        estr[i] = 1;
        if (i + 1 < rank) gstr[i] = strides_bytes[i];
    }
    CUresult r = reinterpret_cast<Fn>(ctx->encode_tiled)(
        map, dt, (cuuint32_t)rank, base, gdim, gstr, bdim, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[128];
        snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
        return gc_fail(ctx, GC_ECUDA, buf);
    }
    return GC_OK;
}

static cudaEvent_t pool_get(gc_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

int gc_prof_begin(gc_ctx *ctx, cudaStream_t s, const char *name) {
    if (!ctx->profile) return -1;
    gc_prof_rec r{name, pool_get(ctx), pool_get(ctx)};
    if (!r.start || !r.stop) return -1;
    cudaEventRecord(r.start, s);
    ctx->prof.push_back(r);
    return (int)ctx->prof.size() - 1;
}

void gc_prof_end(gc_ctx *ctx, cudaStream_t s, int rec) {
    if (rec < 0 || rec >= (int)ctx->prof.size()) return;
    cudaEventRecord(ctx->prof[rec].stop, s);
}

static void prof_clear(gc_ctx *ctx) {
    for (auto &r : ctx->prof) {
        ctx->event_pool.push_back(r.start);
        ctx->event_pool.push_back(r.stop);
    }
    ctx->prof.clear();
}

extern "C" {

gc_status gc_create(gc_ctx **out, int device) {
    if (!out) return GC_EINVAL;
    *out = nullptr;
    gc_ctx *ctx = new (std::nothrow) gc_ctx();
    if (!ctx) return GC_ENOMEM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->status_dev, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(ctx->status_dev, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->status_dev) cudaFree(ctx->status_dev);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? GC_ENOMEM : GC_ECUDA;
    }
    *out = ctx;
    return GC_OK;
}

void gc_destroy(gc_ctx *ctx) {
    if (!ctx) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    prof_clear(ctx);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    for (int b = 0; b < GC_NSTAGE; ++b) {
        if (ctx->stage[b]) cudaFree(ctx->stage[b]);
        if (ctx->ev_copied[b]) cudaEventDestroy(ctx->ev_copied[b]);
        if (ctx->ev_free[b]) cudaEventDestroy(ctx->ev_free[b]);
    }
    for (int b = 0; b < 2; ++b) {
        if (ctx->gains_dev[b]) cudaFree(ctx->gains_dev[b]);
        if (ctx->ev_gains_free[b]) cudaEventDestroy(ctx->ev_gains_free[b]);
    }
    if (ctx->ev_gains_copied) cudaEventDestroy(ctx->ev_gains_copied);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->status_dev) cudaFree(ctx->status_dev);
    cudaSetDevice(prev);
    delete ctx;
}

const char *gc_last_error(const gc_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

gc_status gc_device_status(gc_ctx *ctx, void *stream) {
    if (!ctx) return GC_EINVAL;
    unsigned int h = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(&h, ctx->status_dev, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status_dev, 0, sizeof h, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "gc_device_status");
    if (h & (GC_DEV_TIMEOUT_FFT | GC_DEV_TIMEOUT_XENG | GC_DEV_TIMEOUT_CAL)) {
        char buf[96];
        snprintf(buf, sizeof buf, "device-side bounded wait ran out (flags 0x%x)", h);
        return gc_fail(ctx, GC_ETIMEOUT, buf);
    }
    if (h & GC_DEV_BADINDEX) return gc_fail(ctx, GC_EINVAL, "device saw an out-of-range index");
    if (h & GC_DEV_BADINPUT)
        return gc_fail(ctx, GC_EINVAL, "a gain was zero or not finite, or the voltages gave non-finite sums");
    return GC_OK;
}

gc_status gc_profile_enable(gc_ctx *ctx, int enable) {
    if (!ctx) return GC_EINVAL;
    ctx->profile = enable != 0;
    if (!ctx->profile) prof_clear(ctx);
    return GC_OK;
}

int gc_profile_read(gc_ctx *ctx, char *names, double *total_ms, int *launches, int max_kinds) {
    if (!ctx || max_kinds < 0) return -1;
    std::vector<std::string> kinds;
    std::vector<double> ms;
    std::vector<int> cnt;
    for (auto &r : ctx->prof) {
        if (cudaEventSynchronize(r.stop) != cudaSuccess) continue;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess) continue;
        size_t k = 0;
        while (k < kinds.size() && kinds[k] != r.name) ++k;
        if (k == kinds.size()) {
            kinds.push_back(r.name);
            ms.push_back(0.0);
            cnt.push_back(0);
        }
        ms[k] += t;
        cnt[k] += 1;
    }
    prof_clear(ctx);
    const int n = (int)kinds.size();
    for (int k = 0; k < n && k < max_kinds; ++k) {
        if (names) {
            strncpy(names + 64 * k, kinds[k].c_str(), 63);
            names[64 * k + 63] = 0;
        }
        if (total_ms) total_ms[k] = ms[k];
        if (launches) launches[k] = cnt[k];
    }
    return n;
}

static int tune_index(const char *name) {
    if (!name) return -1;
    static const char *names[GC_TUNE_N] = {"fft.chunk_len", "xeng.tsplit", "cal.ctas_per_sm", "cal.order",
                                                 "cal.operator", "xeng.path",
                                                 "xeng.tc_shape", "fft.shape", "fft.path"};
    for (int k = 0; k < GC_TUNE_N; ++k)
        if (strcmp(name, names[k]) == 0) return k;
    return -1;
}

gc_status gc_set_tuning(gc_ctx *ctx, const char *name, int value) {
    const int k = tune_index(name);
    if (!ctx || k < 0 || value < 0) return GC_EINVAL;
    ctx->tune[k] = value;
    return GC_OK;
}

gc_status gc_get_tuning(const gc_ctx *ctx, const char *name, int *value) {
    const int k = tune_index(name);
    if (!ctx || k < 0 || !value) return GC_EINVAL;
    *value = ctx->tune[k];
    return GC_OK;
}

int gc_fft_size(int L) {
    if (L < 1 || L > 128) return 0;
    int M = 1;
    while (M < 2 * L - 1) M <<= 1;
    return M < 2 ? 2 : M;
}

}  // extern "C"
