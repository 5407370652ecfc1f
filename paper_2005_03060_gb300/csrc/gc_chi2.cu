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
// form, reads the residuals the forward pass stored.  FP32 products; sums of
// a few terms (one antenna's pairs, a run of 32 pairs) in FP32, every longer
// sum in FP64.
//
// Selections of at most 16 types on a full grid take the stencil form: the
// thread owning antenna m finds its pairs by grid arithmetic (pair index
// from the type's row-major enumeration), so no pair lists are read; the
// forward pass and the adjoint visit each pair once (m as first member); the
// adjoint passes the second member's term through a shared slot, keeps each
// thread's model-visibility terms per type in shared memory until one
// fixed-order reduction at the end of the CTA, and hands the terms of
// antennas below its range to a small second kernel.
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
        float sf = 0.f;
        int run = 0;
        for (int q = threadIdx.x; q < p.P; q += blockDim.x) {
            const float2 r = resid(p, c, q, p.pair_i[q], p.pair_j[q], p.pair_type[q]);
            if (p.resid_out) p.resid_out[(size_t)c * p.P + q] = r;
            const float wq = p.w ? p.w[(size_t)c * p.P + q] : 1.0f;
            sf = fmaf(wq, fmaf(r.x, r.x, r.y * r.y), sf);
            if (++run == 32) {   // runs of 32 pairs in FP32, the rest in FP64
                s += (double)sf;
                sf = 0.f;
                run = 0;
            }
        }
        s += (double)sf;
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


// ----------------------------------------------------------------- stencil form
constexpr int kStTypes = 16;

// Per-type constants: the observation index of a pair is
// a1 + y (L - |dx|) + x with (x, y) its first member, and a2 + y (L - |dx|) + x
// with (x, y) its second member (the builders enumerate a type's pairs
// row-major over the overlap of the grid with its shift).
struct StTypes {
    int dx[kStTypes], dy[kStTypes], off[kStTypes], rowlen[kStTypes], a1[kStTypes], a2[kStTypes];
    float inv[kStTypes];
};

__device__ __forceinline__ void load_types(const Chi2Params &p, StTypes &t) {
    if (threadIdx.x < p.n_ubl) {
        const int k = threadIdx.x;
        const int dx = p.types[2 * k], dy = p.types[2 * k + 1];
        const int rl = p.L - abs(dx);
        const int a2 = p.type_ptr[k] - max(0, -dy) * rl - max(0, -dx);
        t.dx[k] = dx;
        t.dy[k] = dy;
        t.off[k] = dy * p.L + dx;
        t.rowlen[k] = rl;
        t.a2[k] = a2;
        t.a1[k] = a2 - dy * rl - dx;
        t.inv[k] = 1.0f / (float)(p.win_t1[k] - p.win_t0[k]);
    }
}

// residual of the pair with observation index idx (channel offset included)
// from its gains and model (the same arithmetic as resid(), so stored and
// recomputed residuals agree)
template <int VF>
__device__ __forceinline__ float2 st_resid(const void *vred, size_t idx, float inv, float2 gi, float2 gj, float2 V) {
    float2 o;
    if (VF == GC_C64) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(vred) + idx);
        o = make_float2(v.x * inv, v.y * inv);
    } else {
        const int2 v = __ldg(reinterpret_cast<const int2 *>(vred) + idx);
        o = make_float2((float)v.x * inv, (float)v.y * inv);
    }
    const float ex = gi.x * gj.x + gi.y * gj.y, ey = gi.y * gj.x - gi.x * gj.y;
    return make_float2(o.x - (ex * V.x - ey * V.y), o.y - (ex * V.y + ey * V.x));
}

// The stencil kernels split each channel's antennas into ranges of
// kStJ x kKThreads antennas, one CTA each; a thread holds kStJ antennas (grid
// coordinates packed as x | y << 16, computed once) and the type loop is
// outermost.  Inside a type step nothing branches: a pair that falls off the
// grid reads observation 0 and gain 0 of its channel (valid addresses) and
// its terms are selected away, so the loads of all kStJ antennas issue
// together.  Each CTA writes FP64 partial sums that chi2_st_reduce adds in a
// fixed order, so the results do not depend on scheduling.
constexpr int kStJ = 8;
constexpr int kDvPitch = kKThreads + 8;   // conflict-free column reads of the dV partials
struct StSplit {
    int parts;         // antenna ranges per channel
    double *partial;   // fwd: [C][parts]; bwd: [C][parts][n_ubl][2]
    int halo;          // bwd: largest pair offset dy L + dx over the types
    float2 *hbuf;      // bwd: [C][parts][halo] second-member terms of the antennas below each range
};

// FL: bit 0 weights, bit 1 residuals stored (fwd) / read (bwd)
template <int VF, int FL>
__global__ void __launch_bounds__(kKThreads) chi2_fwd_st(const Chi2Params p, const StSplit sp) {
    __shared__ StTypes t;
    __shared__ float2 sV[kStTypes];
    __shared__ double red[kKThreads / 32];
    load_types(p, t);
    const int L = p.L, nu = p.n_ubl;
    const int c = blockIdx.x / sp.parts, part = blockIdx.x % sp.parts;
    const int m0 = part * kStJ * kKThreads;
    if (threadIdx.x < nu) sV[threadIdx.x] = p.V[(size_t)c * nu + threadIdx.x];
    __syncthreads();
    const float2 *g = p.g + (size_t)c * p.N;
    const size_t cP = (size_t)c * p.P;
    float2 gm[kStJ];
    int xy[kStJ];
#pragma unroll
    for (int j = 0; j < kStJ; ++j) {
        const int m = m0 + threadIdx.x + j * kKThreads;
        const bool in = m < p.N;
        xy[j] = in ? (m % L) | ((m / L) << 16) : -1;
        gm[j] = in ? g[m] : make_float2(0.f, 0.f);
    }
    double s = 0.0;
    for (int k = 0; k < nu; ++k) {
        const int dx = t.dx[k], dy = t.dy[k], off = t.off[k], rl = t.rowlen[k], a1 = t.a1[k];
        const float inv = t.inv[k];
        const float2 V = sV[k];
        float sf = 0.f;   // kStJ terms of one type in FP32
#pragma unroll
        for (int j = 0; j < kStJ; ++j) {
            const int m = m0 + threadIdx.x + j * kKThreads;
            const int x = xy[j] & 0xffff, y = xy[j] >> 16;
            const bool v = xy[j] >= 0 && (unsigned)(x - dx) < (unsigned)L && (unsigned)(y - dy) < (unsigned)L;
            const int q = v ? a1 + y * rl + x : 0;
            const float2 r = st_resid<VF>(p.vred, cP + q, inv, gm[j], g[v ? m - off : 0], V);
            if ((FL & 2) && v) p.resid_out[cP + q] = r;
            float e = fmaf(r.x, r.x, r.y * r.y);
            if (FL & 1) e *= p.w[cP + q];
            sf += v ? e : 0.f;
        }
        s += (double)sf;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tt = 0.0;
        for (int u = 0; u < kKThreads / 32; ++u) tt += red[u];
        sp.partial[blockIdx.x] = tt;
    }
}

// The adjoint visits each pair once, from its first member m: the pair's
// residual feeds dg_m (registers), dV_k (registers, then shared memory) and
// the second member's term w conj(r) g_m V, which goes to a shared slot of
// antenna m - d.  For one type the map m -> m - d is one-to-one, so a slot
// takes at most one term per type and a barrier between types orders them;
// slots below the range (antennas of the previous range, at most `halo`
// of them) go to the workspace and chi2_st_halo adds them afterwards.
template <int VF, int FL>
__global__ void __launch_bounds__(kKThreads, (FL & 2) ? 3 : 2) chi2_bwd_st(const Chi2Params p, const StSplit sp) {
    __shared__ StTypes t;
    __shared__ float2 sV[kStTypes];
    __shared__ float sdv[2 * kStTypes * kDvPitch];   // per-thread dV terms of every type
    __shared__ float2 sspare[kKThreads];              // zero terms of pairs off the grid
    extern __shared__ float2 sacc[];                  // [halo + range] second-member terms
    load_types(p, t);
    const int L = p.L, nu = p.n_ubl, H = sp.halo;
    constexpr int R = kStJ * kKThreads;
    const int c = blockIdx.x / sp.parts, part = blockIdx.x % sp.parts;
    const int m0 = part * R;
    if (threadIdx.x < nu) sV[threadIdx.x] = p.V[(size_t)c * nu + threadIdx.x];
    for (int i = threadIdx.x; i < H + R; i += kKThreads) sacc[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const double go = p.gout ? p.gout[c] : 1.0;
    const float2 *g = p.g + (size_t)c * p.N;
    const size_t cP = (size_t)c * p.P;
    float2 gm[kStJ], acc[kStJ];   // each antenna's gain and its first-member terms (at most 16)
    int xy[kStJ];
#pragma unroll
    for (int j = 0; j < kStJ; ++j) {
        const int m = m0 + threadIdx.x + j * kKThreads;
        const bool in = m < p.N;
        xy[j] = in ? (m % L) | ((m / L) << 16) : -1;
        gm[j] = in ? g[m] : make_float2(0.f, 0.f);
        acc[j] = make_float2(0.f, 0.f);
    }
    for (int k = 0; k < nu; ++k) {
        const int dx = t.dx[k], dy = t.dy[k], off = t.off[k], rl = t.rowlen[k], a1 = t.a1[k];
        const float inv = t.inv[k];
        const float2 V = sV[k];
        float vx = 0.f, vy = 0.f;   // this thread's part of dV_k (kStJ terms)
        // all of the type step's loads first (kStJ partner gains and
        // observations in flight together), then the arithmetic
        float2 gjv[kStJ], obv[kStJ];
        float wv[kStJ];
        unsigned vm = 0u;
#pragma unroll
        for (int j = 0; j < kStJ; ++j) {
            const int m = m0 + threadIdx.x + j * kKThreads;
            const int x = xy[j] & 0xffff, y = xy[j] >> 16;
            const bool v1 = xy[j] >= 0 && (unsigned)(x - dx) < (unsigned)L && (unsigned)(y - dy) < (unsigned)L;
            vm |= v1 ? 1u << j : 0u;
            const int q1 = v1 ? a1 + y * rl + x : 0;
            gjv[j] = __ldg(g + (v1 ? m - off : 0));
            if (FL & 2) {
                obv[j] = __ldg(p.resid_in + cP + q1);
            } else if (VF == GC_C64) {
                const float2 o = __ldg(reinterpret_cast<const float2 *>(p.vred) + cP + q1);
                obv[j] = make_float2(o.x * inv, o.y * inv);
            } else {
                const int2 o = __ldg(reinterpret_cast<const int2 *>(p.vred) + cP + q1);
                obv[j] = make_float2((float)o.x * inv, (float)o.y * inv);
            }
            wv[j] = (FL & 1) ? __ldg(p.w + cP + q1) : 1.f;
        }
#pragma unroll
        for (int j = 0; j < kStJ; ++j) {
            const int m = m0 + threadIdx.x + j * kKThreads;
            const bool v1 = (vm >> j) & 1u;
            const float2 gj = gjv[j];
            float2 r1 = obv[j];
            if (!(FL & 2)) {   // the residual from (g, V), as st_resid computes it
                const float ex = gm[j].x * gj.x + gm[j].y * gj.y, ey = gm[j].y * gj.x - gm[j].x * gj.y;
                r1 = make_float2(r1.x - (ex * V.x - ey * V.y), r1.y - (ex * V.y + ey * V.x));
            }
            const float w1 = wv[j];
            const float rx = v1 ? w1 * r1.x : 0.f, ry = v1 ? w1 * r1.y : 0.f;
            // first member m: w r g_j conj(V) to dg_m
            const float tx = gj.x * V.x + gj.y * V.y, ty = gj.y * V.x - gj.x * V.y;
            acc[j].x = fmaf(rx, tx, fmaf(-ry, ty, acc[j].x));
            acc[j].y = fmaf(rx, ty, fmaf(ry, tx, acc[j].y));
            // w r conj(g_m) g_j to dV_k
            const float ux = gm[j].x * gj.x + gm[j].y * gj.y, uy = gm[j].x * gj.y - gm[j].y * gj.x;
            vx = fmaf(rx, ux, fmaf(-ry, uy, vx));
            vy = fmaf(rx, uy, fmaf(ry, ux, vy));
            // second member m - d: w conj(r) g_m V (a pair off the grid
            // adds its zero term to this thread's own spare slot)
            {
                const float px = gm[j].x * V.x - gm[j].y * V.y, py = gm[j].x * V.y + gm[j].y * V.x;
                float2 &slot = v1 ? sacc[m - off - m0 + H] : sspare[threadIdx.x];
                slot.x += fmaf(rx, px, ry * py);
                slot.y += fmaf(rx, py, -ry * px);
            }
        }
        sdv[(2 * k) * kDvPitch + threadIdx.x] = vx;
        sdv[(2 * k + 1) * kDvPitch + threadIdx.x] = vy;
        __syncthreads();   // a slot takes one term per type
    }
    const float sc = (float)(-2.0 * go);
#pragma unroll
    for (int j = 0; j < kStJ; ++j) {
        const int m = m0 + threadIdx.x + j * kKThreads;
        if (xy[j] >= 0) {
            const float2 s2 = sacc[m - m0 + H];
            p.dg[(size_t)c * p.N + m] = make_float2(sc * (acc[j].x + s2.x), sc * (acc[j].y + s2.y));
        }
    }
    for (int i = threadIdx.x; i < H; i += kKThreads) sp.hbuf[(size_t)blockIdx.x * H + i] = sacc[i];
    // dV partials of the CTA: 8 threads per (type, component), each adding
    // 32 threads' terms, then the 8 in FP64 in a fixed shuffle order
    const int combo = threadIdx.x >> 3, sub = threadIdx.x & 7;
    float fsum = 0.f;   // 32 threads' terms in FP32, the 8 partial sums in FP64
    if (combo < 2 * nu)
#pragma unroll 8
        for (int u = 0; u < kKThreads / 8; ++u) fsum += sdv[combo * kDvPitch + u * 8 + sub];
    double dsum = (double)fsum;
    dsum += __shfl_xor_sync(0xffffffffu, dsum, 1);
    dsum += __shfl_xor_sync(0xffffffffu, dsum, 2);
    dsum += __shfl_xor_sync(0xffffffffu, dsum, 4);
    if (sub == 0 && combo < 2 * nu) sp.partial[((size_t)blockIdx.x * nu + (combo >> 1)) * 2 + (combo & 1)] = dsum;
}

// Second-member terms that range `part` computed for the last `halo`
// antennas of range part - 1, added to their gradients (one thread each).
__global__ void chi2_st_halo(const Chi2Params p, const StSplit sp) {
    const int H = sp.halo;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long per = (long)(sp.parts - 1) * H;
    if (per <= 0 || idx >= (long)p.C * per) return;
    const int c = (int)(idx / per), rem = (int)(idx % per);
    const int part = 1 + rem / H, i = rem % H;
    const int m = part * kStJ * kKThreads - H + i;
    if (m < 0 || m >= p.N) return;
    const float sc = (float)(-2.0 * (p.gout ? p.gout[c] : 1.0));
    const float2 h = sp.hbuf[((size_t)c * sp.parts + part) * H + i];
    float2 &d = p.dg[(size_t)c * p.N + m];
    d = make_float2(d.x + sc * h.x, d.y + sc * h.y);
}

// chi^2 (fwd) or dV (bwd) from the ranges' partial sums, in range order
__global__ void chi2_st_reduce(const Chi2Params p, const StSplit sp, int bwd) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (!bwd) {
        if (idx >= p.C) return;
        double s = 0.0;
        for (int u = 0; u < sp.parts; ++u) s += sp.partial[(size_t)idx * sp.parts + u];
        p.chi2[idx] = s;
        return;
    }
    if (idx >= p.C * p.n_ubl) return;
    const int c = idx / p.n_ubl, k = idx % p.n_ubl;
    double sx = 0.0, sy = 0.0;
    for (int u = 0; u < sp.parts; ++u) {
        const size_t b = (((size_t)c * sp.parts + u) * p.n_ubl + k) * 2;
        sx += sp.partial[b];
        sy += sp.partial[b + 1];
    }
    const double go = p.gout ? p.gout[c] : 1.0;
    p.dV[(size_t)c * p.n_ubl + k] = make_float2((float)(-2.0 * go * sx), (float)(-2.0 * go * sy));
}

bool use_stencil(const gc_sel *sel) { return !sel->masked && sel->n_ubl <= kStTypes; }

// largest pair offset dy L + dx of the selection's types (all positive: the
// types are taken in the half-plane dy > 0 or dy = 0, dx > 0)
int st_halo(const gc_sel *sel) {
    int h = 0;
    for (int k = 0; k < sel->n_ubl; ++k) h = std::max(h, sel->types[2 * k + 1] * sel->L + sel->types[2 * k]);
    return h;
}

// kStJ x kKThreads antennas per CTA
gc_status st_launch(gc_ctx *ctx, const Chi2Params &p, bool bwd, int halo, cudaStream_t s) {
    StSplit sp;
    sp.parts = (p.N + kStJ * kKThreads - 1) / (kStJ * kKThreads);
    sp.halo = bwd ? halo : 0;
    const size_t n = (size_t)p.C * sp.parts * (bwd ? 2 * p.n_ubl : 1);
    const size_t part_bytes = (n * sizeof(double) + 255) / 256 * 256;
    const size_t hb_bytes = (size_t)p.C * sp.parts * sp.halo * sizeof(float2);
    gc_status st = gc_scratch_reserve(ctx, part_bytes + hb_bytes);
    if (st != GC_OK) return st;
    sp.partial = static_cast<double *>(ctx->scratch);
    sp.hbuf = reinterpret_cast<float2 *>(static_cast<char *>(ctx->scratch) + part_bytes);
    const unsigned grid = (unsigned)(p.C * sp.parts);
    const int dsm = bwd ? (sp.halo + kStJ * kKThreads) * (int)sizeof(float2) : 0;
    const int fl = (p.w ? 1 : 0) | ((bwd ? p.resid_in != nullptr : p.resid_out != nullptr) ? 2 : 0);
    const bool c64 = p.vfmt == GC_C64;
#define GC_ST_CASE(F)                                                                    \
    case F:                                                                              \
        if (bwd) {                                                                       \
            auto kb = c64 ? chi2_bwd_st<GC_C64, F> : chi2_bwd_st<GC_I4C, F>;             \
            cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm);   \
            kb<<<grid, kKThreads, dsm, s>>>(p, sp);                                      \
        } else {                                                                         \
            if (c64) chi2_fwd_st<GC_C64, F><<<grid, kKThreads, 0, s>>>(p, sp);           \
            else chi2_fwd_st<GC_I4C, F><<<grid, kKThreads, 0, s>>>(p, sp);               \
        }                                                                                \
        break;
    switch (fl) {
        GC_ST_CASE(0)
        GC_ST_CASE(1)
        GC_ST_CASE(2)
        GC_ST_CASE(3)
    }
#undef GC_ST_CASE
    const int nr = bwd ? p.C * p.n_ubl : p.C;
    chi2_st_reduce<<<(nr + 255) / 256, 256, 0, s>>>(p, sp, bwd ? 1 : 0);
    if (bwd && sp.parts > 1 && sp.halo > 0) {
        const long nh = (long)p.C * (sp.parts - 1) * sp.halo;
        chi2_st_halo<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(p, sp);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, bwd ? "launch chi2_bwd" : "launch chi2_fwd");
    return GC_OK;
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
    if (use_stencil(sel)) {
        st = st_launch(ctx, p, false, 0, s);
        if (st != GC_OK) return st;
    } else {
        chi2_fwd<<<grid, kKThreads, 0, s>>>(p);
    }
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
    if (use_stencil(sel) && st_halo(sel) <= kStJ * kKThreads) {
        st = st_launch(ctx, p, true, st_halo(sel), s);
        if (st != GC_OK) return st;
    } else {
        chi2_bwd<<<grid, kKThreads, 0, s>>>(p);
    }
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
    if (use_stencil(sel)) {
        st = st_launch(ctx, p, false, 0, s);
        if (st != GC_OK) return st;
    } else {
        chi2_fwd<<<grid, kKThreads, 0, s>>>(p);
    }
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
    if (use_stencil(sel) && st_halo(sel) <= kStJ * kKThreads) {
        st = st_launch(ctx, p, true, st_halo(sel), s);
        if (st != GC_OK) return st;
    } else {
        chi2_bwd<<<grid, kKThreads, 0, s>>>(p);
    }
    gc_prof_end(ctx, s, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch chi2_bwd");
    return GC_OK;
}
