// Arithmetic-throughput probes for the roofline denominators of the
// FP32-issue-bound FFT-correlator and the FP64 normal equations (not part
// of the paper's method).  Each thread runs independent FMA chains; the
// result is folded into one word so the work cannot be removed.
#include <cstdio>

#include "gc_internal.h"

namespace {

template <class R>
__global__ void __launch_bounds__(256) fma_probe(int iters, R seed, R *sink) {
    R a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + (R)(threadIdx.x + k);
    const R m = (R)0.999999, c = (R)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == (R)-1.2345) *sink = s;   // practically never true
}

}  // namespace

extern "C" gc_status gc_peak_probe(gc_ctx *ctx, int kind, double *tflops) {
    if (!ctx || !tflops || (kind != 0 && kind != 1)) return GC_EINVAL;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    gc_status st = gc_scratch_reserve(ctx, 64);
    if (st != GC_OK) return st;
    const int blocks = ctx->sm_count * 8;
    const int iters = kind == 0 ? (1 << 16) : (1 << 12);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // first launch warms up
        cudaEventRecord(a);
        if (kind == 0) fma_probe<float><<<blocks, 256>>>(iters, 1.0f, static_cast<float *>(ctx->scratch));
        else fma_probe<double><<<blocks, 256>>>(iters, 1.0, static_cast<double *>(ctx->scratch));
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
    }
    e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "fma probe");
    const double flops = 2.0 * 8.0 * (double)iters * blocks * 256.0;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return GC_OK;
}
