// 4+4-bit quantiser of the voltage stream (precision variant of the voltage
// path; the paper itself works with unquantised voltages).
//
// Per channel: rms = sqrt(sum(re^2 + im^2) / (2 T N)) accumulated in FP64,
// scale = (float)(3 / rms) so that each component has an RMS of 3 levels,
// q = clip(round_half_away(x * scale), -7, 7) with the product rounded to
// float, byte = (q_re << 4) | (q_im & 15).  The FP64 sum is formed in a
// fixed order (block partials, then a sequential sum), so a channel's scale
// does not depend on the launch.
#include <algorithm>

#include "gc_internal.h"

namespace {

constexpr int kQThreads = 256;

__global__ void __launch_bounds__(kQThreads)
quant_sumsq(const float4 *__restrict__ v, size_t n4_per_ch, int nblk, double *__restrict__ part) {
    const int c = blockIdx.y, b = blockIdx.x;
    const float4 *src = v + (size_t)c * n4_per_ch;
    const size_t per = (n4_per_ch + nblk - 1) / nblk;
    const size_t lo = (size_t)b * per, hi = min(n4_per_ch, lo + per);
    double s = 0.0;
    for (size_t i = lo + threadIdx.x; i < hi; i += kQThreads) {
        const float4 q = src[i];
        s += (double)q.x * q.x + (double)q.y * q.y + (double)q.z * q.z + (double)q.w * q.w;
    }
    __shared__ double red[kQThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kQThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)c * nblk + b] = red[0];
}

__global__ void quant_scale(const double *__restrict__ part, int nblk, int C, double n_components,
                            float *__restrict__ scale) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)c * nblk + b];
    const double rms = sqrt(s / n_components);
    scale[c] = rms > 0.0 ? (float)(3.0 / rms) : 0.0f;
}

__device__ __forceinline__ int q4(float x) {
    const float a = fabsf(x);
    float f = floorf(a);
    if (a - f >= 0.5f) f += 1.0f;
    int q = (int)f;
    q = q > 7 ? 7 : q;
    return x < 0.0f ? -q : q;
}

__global__ void __launch_bounds__(kQThreads)
quant_apply(const float4 *__restrict__ v, size_t n2_per_ch, int C, const float *__restrict__ scale,
            uint16_t *__restrict__ out) {
    // each thread packs two antenna-samples (one float4) into two bytes
    const size_t total = n2_per_ch * C;
    for (size_t i = blockIdx.x * (size_t)kQThreads + threadIdx.x; i < total; i += (size_t)gridDim.x * kQThreads) {
        const int c = (int)(i / n2_per_ch);
        const float s = scale[c];
        const float4 q = v[i];
        const int r0 = q4(__fmul_rn(q.x, s)), i0 = q4(__fmul_rn(q.y, s));
        const int r1 = q4(__fmul_rn(q.z, s)), i1 = q4(__fmul_rn(q.w, s));
        const unsigned b0 = ((unsigned)(r0 & 15) << 4) | (unsigned)(i0 & 15);
        const unsigned b1 = ((unsigned)(r1 & 15) << 4) | (unsigned)(i1 & 15);
        out[i] = (uint16_t)(b0 | (b1 << 8));
    }
}

}  // namespace

extern "C" gc_status gc_quantize(gc_ctx *ctx, const float *volt, int C, int T, int N, uint8_t *out, float *scales,
                                 void *stream) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    if (!volt || !out) return gc_fail(ctx, GC_EINVAL, "gc_quantize: null buffer");
    if (C < 1 || T < 1 || N < 1 || ((size_t)T * N) % 2 != 0)
        return gc_fail(ctx, GC_EINVAL, "gc_quantize: need C, T, N >= 1 and T*N even");
    if (!gc_aligned(volt, 16) || !gc_aligned(out, 2) || (scales && !gc_aligned(scales, 4)))
        return gc_fail(ctx, GC_EINVAL, "gc_quantize: misaligned buffer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    const size_t n2 = (size_t)T * N / 2;        // float4 (two complex) per channel
    const int nblk = (int)std::max<size_t>(1, std::min<size_t>(64, n2 / 4096));
    const size_t need = (size_t)C * nblk * sizeof(double) + (size_t)C * sizeof(float) + 256;
    gc_status st = gc_scratch_reserve(ctx, need);
    if (st != GC_OK) return st;
    double *part = static_cast<double *>(ctx->scratch);
    float *sc = scales ? scales
                       : reinterpret_cast<float *>(static_cast<char *>(ctx->scratch) +
                                                   (((size_t)C * nblk * sizeof(double) + 255) / 256) * 256);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float4 *v4 = reinterpret_cast<const float4 *>(volt);
    int rec = gc_prof_begin(ctx, s, "quant_sumsq");
    quant_sumsq<<<dim3(nblk, C), kQThreads, 0, s>>>(v4, n2, nblk, part);
    gc_prof_end(ctx, s, rec);
    quant_scale<<<(C + 127) / 128, 128, 0, s>>>(part, nblk, C, 2.0 * (double)T * N, sc);
    const size_t total = n2 * C;
    const int grid = (int)std::min<size_t>((total + kQThreads - 1) / kQThreads, (size_t)ctx->sm_count * 16);
    rec = gc_prof_begin(ctx, s, "quant_apply");
    quant_apply<<<grid, kQThreads, 0, s>>>(v4, n2, C, sc, reinterpret_cast<uint16_t *>(out));
    gc_prof_end(ctx, s, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch quantiser");
    return GC_OK;
}
