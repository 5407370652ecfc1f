// chi^2 of the redundant model against V^reduced (numerator of Eq. redchi,
// per channel) and its adjoint.
//
//   chi2_c = sum_p w_p |r_p|^2,   r_p = V_p - g_i conj(g_j) V_alpha(p),
//   V_p = S_p / t_p (X-engine sums over the pair's window).
// Gradients in the d/dRe + i d/dIm convention (what torch stores in .grad
// for a real loss of complex leaves), scaled by the incoming dL/dchi2_c:
//   dchi2/dg_k     = -2 [ sum_{p: i_p = k} w r g_j conj(V) + sum_{p: j_p = k} w conj(r) g_i V ]
//   dchi2/dV_alpha = -2 sum_{p in alpha} w r conj(g_i) g_j
// The backward pass recomputes the residuals from (g, V) -- nothing but the
// inputs is kept between forward and backward -- or, in the checkpointed
// form, reads the residuals the forward pass stored.  FP32 products, FP64
// sums.
#include <algorithm>

#include "gc_sel.h"

namespace {

constexpr int kKThreads = 256;

struct Chi2Params {
    const void *vred;
    int vfmt, C, L, N, P, n_ubl;
    const int32_t *types, *type_ptr, *pair_i, *pair_j, *pair_type, *win_t0, *win_t1;
    const float2 *g, *V;
    const float *w;          // [C][P] or null
    double *chi2;            // [C]
    const double *gout;      // [C] dL/dchi2 (backward)
    float2 *dg, *dV;         // [C][N], [C][n_ubl]
    float2 *resid_out;       // [C][P] residuals stored by the forward pass, or null
    const float2 *resid_in;  // [C][P] residuals the backward pass reads, or null (recompute)
    const int32_t *pair_of2; // partly occupied lattice: pair index of (r_j + d_k, r_j) by [k][j], or null
};

__device__ __forceinline__ float2 obs(const Chi2Params &p, int c, int q) {
    const int k = p.pair_type[q];
    const float inv = 1.0f / (float)(p.win_t1[k] - p.win_t0[k]);
    if (p.vfmt == GC_C64) {
        const float2 v = reinterpret_cast<const float2 *>(p.vred)[(size_t)c * p.P + q];
        return make_float2(v.x * inv, v.y * inv);
    }
    const int2 v = reinterpret_cast<const int2 *>(p.vred)[(size_t)c * p.P + q];
    return make_float2((float)v.x * inv, (float)v.y * inv);
}

// residual of pair q of channel c
__device__ __forceinline__ float2 resid(const Chi2Params &p, int c, int q, int i, int j, int k) {
    const float2 gi = p.g[(size_t)c * p.N + i], gj = p.g[(size_t)c * p.N + j];
    const float2 V = p.V[(size_t)c * p.n_ubl + k];
    const float ex = gi.x * gj.x + gi.y * gj.y, ey = gi.y * gj.x - gi.x * gj.y;
    const float2 o = obs(p, c, q);
    return make_float2(o.x - (ex * V.x - ey * V.y), o.y - (ex * V.y + ey * V.x));
}

// residual for the backward pass: stored, or recomputed from (g, V)
__device__ __forceinline__ float2 resid_b(const Chi2Params &p, int c, int q, int i, int j, int k) {
    if (p.resid_in) return p.resid_in[(size_t)c * p.P + q];
    return resid(p, c, q, i, j, k);
}

__device__ __forceinline__ int pidx(const Chi2Params &p, int k, int xj, int yj) {
    const int dx = p.types[2 * k], dy = p.types[2 * k + 1], L = p.L;
    const int xi = xj + dx, yi = yj + dy;
    if (xj < 0 || xj >= L || yj < 0 || yj >= L || xi < 0 || xi >= L || yi < 0 || yi >= L) return -1;
    if (p.pair_of2) return p.pair_of2[(size_t)k * p.N + yj * L + xj];
    return p.type_ptr[k] + (yj - max(0, -dy)) * (L - abs(dx)) + (xj - max(0, -dx));
}

__global__ void __launch_bounds__(kKThreads) chi2_fwd(const Chi2Params p) {
    __shared__ double red[kKThreads / 32];
    for (int c = blockIdx.x; c < p.C; c += gridDim.x) {
        double s = 0.0;
        for (int q = threadIdx.x; q < p.P; q += blockDim.x) {
            const float2 r = resid(p, c, q, p.pair_i[q], p.pair_j[q], p.pair_type[q]);
            if (p.resid_out) p.resid_out[(size_t)c * p.P + q] = r;
            const float wq = p.w ? p.w[(size_t)c * p.P + q] : 1.0f;
            s += (double)wq * ((double)r.x * r.x + (double)r.y * r.y);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int u = 0; u < kKThreads / 32; ++u) t += red[u];
            p.chi2[c] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kKThreads) chi2_bwd(const Chi2Params p) {
    const int L = p.L;
    for (int c = blockIdx.x; c < p.C; c += gridDim.x) {
        const double go = p.gout ? p.gout[c] : 1.0;
        // gains: gather over each antenna's pairs
        for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
            const int xi = i % L, yi = i / L;
            double ax = 0.0, ay = 0.0;
            for (int k = 0; k < p.n_ubl; ++k) {
                const float2 V = p.V[(size_t)c * p.n_ubl + k];
                const int dx = p.types[2 * k], dy = p.types[2 * k + 1];
                int q = pidx(p, k, xi - dx, yi - dy);
                if (q >= 0) {   // i = i_p: w r g_j conj(V)
                    const int j = (yi - dy) * L + (xi - dx);
                    const float2 r = resid_b(p, c, q, i, j, k);
                    const float2 gj = p.g[(size_t)c * p.N + j];
                    const float wq = p.w ? p.w[(size_t)c * p.P + q] : 1.0f;
                    const float tx = gj.x * V.x + gj.y * V.y, ty = gj.y * V.x - gj.x * V.y;   // g_j conj(V)
                    ax += (double)wq * (r.x * tx - r.y * ty);
                    ay += (double)wq * (r.x * ty + r.y * tx);
                }
                q = pidx(p, k, xi, yi);
                if (q >= 0) {   // i = j_p: w conj(r) g_i' V
                    const int ip = (yi + dy) * L + (xi + dx);
                    const float2 r = resid_b(p, c, q, ip, i, k);
                    const float2 gp = p.g[(size_t)c * p.N + ip];
                    const float wq = p.w ? p.w[(size_t)c * p.P + q] : 1.0f;
                    const float tx = gp.x * V.x - gp.y * V.y, ty = gp.x * V.y + gp.y * V.x;   // g_i' V
                    ax += (double)wq * (r.x * tx + r.y * ty);
                    ay += (double)wq * (r.x * ty - r.y * tx);
                }
            }
            p.dg[(size_t)c * p.N + i] = make_float2((float)(-2.0 * go * ax), (float)(-2.0 * go * ay));
        }
        // model visibilities: one warp per type
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int k = wp; k < p.n_ubl; k += nw) {
            double sx = 0.0, sy = 0.0;
            for (int q = p.type_ptr[k] + lane; q < p.type_ptr[k + 1]; q += 32) {
                const int i = p.pair_i[q], j = p.pair_j[q];
                const float2 r = resid_b(p, c, q, i, j, k);
                const float2 gi = p.g[(size_t)c * p.N + i], gj = p.g[(size_t)c * p.N + j];
                const float tx = gi.x * gj.x + gi.y * gj.y, ty = gi.x * gj.y - gi.y * gj.x;   // conj(g_i) g_j
                const float wq = p.w ? p.w[(size_t)c * p.P + q] : 1.0f;
                sx += (double)wq * (r.x * tx - r.y * ty);
                sy += (double)wq * (r.x * ty + r.y * tx);
            }
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane == 0)
                p.dV[(size_t)c * p.n_ubl + k] = make_float2((float)(-2.0 * go * sx), (float)(-2.0 * go * sy));
        }
        __syncthreads();
    }
}

gc_status chi2_setup(gc_ctx *ctx, const void *vred, int vfmt, const gc_sel *csel, int C, const float *gains,
                     const float *vmodel, const float *weights, Chi2Params &p) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    gc_sel *sel = const_cast<gc_sel *>(csel);
    if (!vred || !sel || !gains || !vmodel || C < 1) return gc_fail(ctx, GC_EINVAL, "gc_chi2: null argument");
    if (vfmt != GC_C64 && vfmt != GC_I4C) return gc_fail(ctx, GC_EINVAL, "gc_chi2: unknown format");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    gc_status st = gc_sel_upload(ctx, sel);
    if (st != GC_OK) return st;
    p.vred = vred;
    p.vfmt = vfmt;
    p.C = C;
    p.L = sel->L;
    p.N = sel->L * sel->L;
    p.P = sel->P;
    p.n_ubl = sel->n_ubl;
    p.types = sel->d_types;
    p.type_ptr = sel->d_type_ptr;
    p.pair_i = sel->d_pair_i;
    p.pair_j = sel->d_pair_j;
    p.pair_type = sel->d_pair_type;
    p.win_t0 = sel->d_win_t0;
    p.win_t1 = sel->d_win_t1;
    p.g = reinterpret_cast<const float2 *>(gains);
    p.V = reinterpret_cast<const float2 *>(vmodel);
    p.w = weights;
    p.chi2 = nullptr;
    p.gout = nullptr;
    p.dg = p.dV = nullptr;
    p.resid_out = nullptr;
    p.resid_in = nullptr;
    p.pair_of2 = nullptr;
    if (sel->masked) {
        if (!sel->d_nbr) return gc_fail(ctx, GC_EUNSUPPORTED, "gc_chi2: masked selection without pair table");
        p.pair_of2 = sel->d_nbr + (size_t)sel->n_ubl * p.N;
    }
    return GC_OK;
}

}  // namespace

extern "C" gc_status gc_chi2(gc_ctx *ctx, const void *vreduced, int vfmt, const gc_sel *sel, int C,
                             const float *gains, const float *vmodel, const float *weights, double *chi2,
                             void *stream) {
    Chi2Params p;
    gc_status st = chi2_setup(ctx, vreduced, vfmt, sel, C, gains, vmodel, weights, p);
    if (st != GC_OK) return st;
    if (!chi2) return gc_fail(ctx, GC_EINVAL, "gc_chi2: null output");
    p.chi2 = chi2;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = std::min(C, ctx->sm_count * 8);
    int rec = gc_prof_begin(ctx, s, "chi2_fwd");
    chi2_fwd<<<grid, kKThreads, 0, s>>>(p);
    gc_prof_end(ctx, s, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch chi2_fwd");
    return GC_OK;
}

extern "C" gc_status gc_chi2_backward(gc_ctx *ctx, const void *vreduced, int vfmt, const gc_sel *sel, int C,
                                      const float *gains, const float *vmodel, const float *weights,
                                      const double *grad_out, float *grad_gains, float *grad_vmodel,
                                      void *stream) {
    Chi2Params p;
    gc_status st = chi2_setup(ctx, vreduced, vfmt, sel, C, gains, vmodel, weights, p);
    if (st != GC_OK) return st;
    if (!grad_gains || !grad_vmodel) return gc_fail(ctx, GC_EINVAL, "gc_chi2_backward: null output");
    p.gout = grad_out;
    p.dg = reinterpret_cast<float2 *>(grad_gains);
    p.dV = reinterpret_cast<float2 *>(grad_vmodel);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = std::min(C, ctx->sm_count * 8);
    int rec = gc_prof_begin(ctx, s, "chi2_bwd");
    chi2_bwd<<<grid, kKThreads, 0, s>>>(p);
    gc_prof_end(ctx, s, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch chi2_bwd");
    return GC_OK;
}

extern "C" gc_status gc_chi2_ckpt(gc_ctx *ctx, const void *vreduced, int vfmt, const gc_sel *sel, int C,
                                  const float *gains, const float *vmodel, const float *weights, double *chi2,
                                  float *residuals, void *stream) {
    Chi2Params p;
    gc_status st = chi2_setup(ctx, vreduced, vfmt, sel, C, gains, vmodel, weights, p);
    if (st != GC_OK) return st;
    if (!chi2 || !residuals || !gc_aligned(residuals, 8))
        return gc_fail(ctx, GC_EINVAL, "gc_chi2_ckpt: null or misaligned output");
    p.chi2 = chi2;
    p.resid_out = reinterpret_cast<float2 *>(residuals);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = std::min(C, ctx->sm_count * 8);
    int rec = gc_prof_begin(ctx, s, "chi2_fwd");
    chi2_fwd<<<grid, kKThreads, 0, s>>>(p);
    gc_prof_end(ctx, s, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch chi2_fwd");
    return GC_OK;
}

extern "C" gc_status gc_chi2_backward_ckpt(gc_ctx *ctx, const float *residuals, const gc_sel *sel, int C,
                                           const float *gains, const float *vmodel, const float *weights,
                                           const double *grad_out, float *grad_gains, float *grad_vmodel,
                                           void *stream) {
    Chi2Params p;
    // the stored residuals stand in for V^reduced, which the backward pass no longer reads
    gc_status st = chi2_setup(ctx, residuals, GC_C64, sel, C, gains, vmodel, weights, p);
    if (st != GC_OK) return st;
    if (!grad_gains || !grad_vmodel || !gc_aligned(residuals, 8))
        return gc_fail(ctx, GC_EINVAL, "gc_chi2_backward_ckpt: null output or misaligned residuals");
    p.gout = grad_out;
    p.dg = reinterpret_cast<float2 *>(grad_gains);
    p.dV = reinterpret_cast<float2 *>(grad_vmodel);
    p.resid_in = reinterpret_cast<const float2 *>(residuals);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = std::min(C, ctx->sm_count * 8);
    int rec = gc_prof_begin(ctx, s, "chi2_bwd");
    chi2_bwd<<<grid, kKThreads, 0, s>>>(p);
    gc_prof_end(ctx, s, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch chi2_bwd");
    return GC_OK;
}
