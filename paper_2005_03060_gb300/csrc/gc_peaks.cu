// Arithmetic-throughput probes for the roofline denominators of the
// FP32-issue-bound FFT-correlator, the FP64 normal equations, the integer
// (dp4a) X-engine, the legacy warp-level int8 MMA and the tensor-core (FP8
// MMA) X-engine (not part of the
// paper's method).  Each SIMT thread runs independent chains; the result is
// folded into one word so the work cannot be removed.  The tensor probe issues
// back-to-back dense MMAs (M = 128, N = 256, K = 32, e4m3 x e4m3 -> FP32) on
// operands resident in shared memory, one CTA per SM.
#include <cstdio>

#include "gc_tcgen05.h"

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

// Warp-level integer MMA (m16n8k32, s8 x s8 -> s32): the legacy tensor path,
// eight independent accumulator chains per warp.
__global__ void __launch_bounds__(256) mma_s8_probe(int iters, int seed, int *sink) {
    int acc[8][4];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[k][q] = 0;
    const uint32_t a0 = (uint32_t)seed * threadIdx.x, a1 = a0 ^ 0x11u, a2 = a0 ^ 0x2222u, a3 = a0 ^ 0x33333u;
    const uint32_t b0 = (uint32_t)seed ^ threadIdx.x, b1 = b0 * 7u;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+r"(acc[k][0]), "+r"(acc[k][1]), "+r"(acc[k][2]), "+r"(acc[k][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    int s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) s += acc[k][q];
    if (s == 0x12345) *sink = s;   // practically never true
}

constexpr int kTcProbeN = 256;

__global__ void __launch_bounds__(128, 1) tc_f8_probe(int iters, unsigned int *sink, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    // e4m3 1.0 everywhere: A (128 rows) then B (256 rows), 32 bytes of K each,
    // K-major core matrices (8 rows x 16 bytes) at 128 / 256 byte strides
    for (int i = tid; i < (128 + kTcProbeN) * 32 / 4; i += 128) reinterpret_cast<uint32_t *>(sm)[i] = 0x38383838u;
    if (warp == 0) gc_tmem_alloc(&slot, 512);
    if (tid == 0) {
        gc_mbar_init(&bar, 1);
        gc_fence_mbar_init();
    }
    gc_fence_proxy_async();
    gc_tc_fence_before();
    __syncthreads();
    gc_tc_fence_after();
    const uint32_t tmem = slot;
    if (tid == 0) {
        const uint64_t a = gc_tc_sdesc(gc_smem_addr(sm), 128, 256);
        const uint64_t b = gc_tc_sdesc(gc_smem_addr(sm + 128 * 32), 128, 256);
        const uint32_t id = gc_tc_idesc(128, kTcProbeN, false, false);
        for (int i = 0; i < iters; ++i) gc_tc_mma_f8(tmem + (i & 1) * 256, a, b, id, i > 1 ? 1u : 0u);
        gc_tc_commit(&bar);
    }
    const bool ok = gc_mbar_wait(&bar, 0, GC_WAIT_LIMIT_NS);
    gc_tc_fence_after();
    if (!ok) {
        if (tid == 0) atomicOr(status, GC_DEV_TIMEOUT_XENG);
    } else {
        uint32_t r[32];
        gc_tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), r);
        if (r[0] == 0x12345678u) *sink = r[1];   // practically never true
    }
    gc_tc_fence_before();
    __syncthreads();
    if (warp == 0) gc_tmem_dealloc(tmem, 512);
}

}  // namespace

extern "C" gc_status gc_peak_probe(gc_ctx *ctx, int kind, double *tflops) {
    if (!ctx || !tflops || kind < 0 || kind > 4) return GC_EINVAL;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    gc_status st = gc_scratch_reserve(ctx, 64);
    if (st != GC_OK) return st;
    const int blocks = kind == 3 ? ctx->sm_count : ctx->sm_count * 8;
    const int iters = kind == 1 ? (1 << 12) : (kind >= 3 ? (1 << 14) : (1 << 16));
    const int tc_smem = (128 + kTcProbeN) * 32;
    if (kind == 3) {
        e = cudaFuncSetAttribute(tc_f8_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem);
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaFuncSetAttribute(tc_f8_probe)");
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // first launch warms up
        cudaEventRecord(a);
        if (kind == 0) fma_probe<float><<<blocks, 256>>>(iters, 1.0f, static_cast<float *>(ctx->scratch));
        else if (kind == 1) fma_probe<double><<<blocks, 256>>>(iters, 1.0, static_cast<double *>(ctx->scratch));
        else if (kind == 2) dp4a_probe<<<blocks, 256>>>(iters, 3, static_cast<int *>(ctx->scratch));
        else if (kind == 3) tc_f8_probe<<<blocks, 128, tc_smem>>>(iters, static_cast<unsigned int *>(ctx->scratch), ctx->status_dev);
        else mma_s8_probe<<<blocks, 256>>>(iters, 3, static_cast<int *>(ctx->scratch));
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
    }
    e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "fma probe");
    // FMA = 2 flops; dp4a = four 8-bit products and four additions = 8 ops;
    // one MMA = 2 M N K flops (m16n8k32 per warp: 8192 ops)
    double flops;
    if (kind == 3) flops = 2.0 * 128 * kTcProbeN * 32 * (double)iters * blocks;
    else if (kind == 4) flops = 2.0 * 16 * 8 * 32 * 8.0 * (double)iters * blocks * (256 / 32);
    else flops = (kind == 2 ? 8.0 : 2.0) * 8.0 * (double)iters * blocks * 256.0;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return GC_OK;
}
