// Arithmetic-throughput probes for the roofline denominators of the
// FP32-issue-bound FFT-correlator, the FP64 normal equations and the integer
// (dp4a) X-engine (not part of the paper's method).  Each thread runs
// independent chains; the result is folded into one word so the work cannot
// be removed.
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

__global__ void __launch_bounds__(256) dp4a_probe(int iters, int seed, int *sink) {
    int a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed * (int)(threadIdx.x + k);
    const int b = seed ^ 0x01020304, c = seed ^ 0x7f7f7f7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = __dp4a(a[k] ^ b, c, a[k]);
    }
    int s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 0x12345678) *sink = s;   // practically never true
}

}  // namespace

extern "C" gc_status gc_peak_probe(gc_ctx *ctx, int kind, double *tflops) {
    if (!ctx || !tflops || kind < 0 || kind > 2) return GC_EINVAL;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    gc_status st = gc_scratch_reserve(ctx, 64);
    if (st != GC_OK) return st;
    const int blocks = ctx->sm_count * 8;
    const int iters = kind == 1 ? (1 << 12) : (1 << 16);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // first launch warms up
        cudaEventRecord(a);
        if (kind == 0) fma_probe<float><<<blocks, 256>>>(iters, 1.0f, static_cast<float *>(ctx->scratch));
        else if (kind == 1) fma_probe<double><<<blocks, 256>>>(iters, 1.0, static_cast<double *>(ctx->scratch));
        else dp4a_probe<<<blocks, 256>>>(iters, 3, static_cast<int *>(ctx->scratch));
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
    }
    e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "fma probe");
    // FMA = 2 flops; dp4a = four 8-bit products and four additions = 8 ops
    const double flops = (kind == 2 ? 8.0 : 2.0) * 8.0 * (double)iters * blocks * 256.0;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return GC_OK;
}
