// Per-channel redundant-baseline calibration (paper Sec. 2, Eq. redcal;
// lincal / omnical, Sec. 2 and Sec. 3; degeneracies, Sec. 5.2; chi^2_r and
// DoF, Eq. redchi / Eq. dof).
//
// One CTA calibrates one channel at a time (grid-stride over channels) with
// its state and linear-algebra workspace in global memory (L2 resident).
//
// lincal (Gauss-Newton): unknowns x = [Re g_0, Im g_0, Re g_1, ... ; Re V_0,
// Im V_0, ...].  With antennas in row-major order every selected pair couples
// antennas at most D = max |dy L + dx| apart, so the gain block of J^T J is a
// band of half-width bw = 2D + 1; the model visibilities form a dense border.
//   * assembly by gather: the thread owning antenna i walks its pairs (as
//     i_p and as j_p) and writes its own band rows, border columns and
//     right-hand side -- deterministic, no atomics;
//   * banded Cholesky, one barrier per column (the scaling of column k is
//     folded into the update pass of column k+1), with the forward solve of
//     the right-hand side and of the border riding along;
//   * Schur complement onto the model visibilities, a small dense Cholesky,
//     then the banded back substitution;
//   * the four exact degeneracy directions (amplitude, phase, two slopes)
//     are projected out of the step, a vanishing Levenberg term keeps the
//     factorisation definite, and a halving line search guards chi^2.
// Template on the real type: double (FP64 normal equations) or float.
//
// omnical: damped simultaneous least-squares fixed point (FP32), gain update
// by gather over each antenna's pairs, model-visibility update one warp per
// baseline-type.
#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gc_sel.h"

namespace {

constexpr int kCThreads = 512;
constexpr int kCgThreads = 512;   // matrix-free kernels, pair-scatter operator
constexpr int kCgStThreads = 256; // matrix-free kernels, stencil operator (128 registers a thread)
constexpr int kStencilTypes = 16; // baseline-types the stencil operator holds in registers
// shared arena cap: two CTAs per SM.  Arrays whose hot vectors need more keep
// them in global memory (L2) at two CTAs per SM -- measured faster than one
// CTA per SM with a larger arena (the solver is latency-bound).
constexpr size_t kCgSmemMax = 100u * 1024u;
constexpr int kMaxUbl = 64;   // lincal border limit (2 * 64 reals)

struct CalParams {
    const void *vred;            // c64 [C][P] float2 | i4c [C][P] int2
    int vfmt;
    const void *autos;           // c64 float | i4c int [C][N], or null
    int C, L, N, P, n_ubl;
    const int32_t *types, *type_ptr, *pair_i, *pair_j, *pair_type, *win_t0, *win_t1;
    const int32_t *nbr;          // [2][n_ubl][N] neighbour table or null
    int ax, ay;                  // indices of types (1,0) and (0,1)
    int stencil;                 // matrix-free operator by per-antenna gather (<= kStencilTypes types)
    int st_halo;                 // largest |dx| or |dy| of a type (stencil operator)
    // partly occupied lattice (null / L*L otherwise): occupancy [N], the
    // breadth-first start-point tree over the axis types, antennas
    const int32_t *mask, *tree_ant, *tree_pair, *tree_sign;
    int n_occ;
    int t_autos;                 // samples summed in autos
    float2 *gains;               // [C][N] (in: warm start when warm != 0)
    float2 *vmodel;              // [C][n_ubl]
    gc_calstats *stats;          // [C]
    int solver, max_iter, warm;
    double tol, damping, mu_rel;
    int bw;                      // band half-width (reals)
    char *work;
    size_t work_per_cta;
    unsigned int *counter;   // next channel to take (matrix-free kernels; zeroed before the launch)
    unsigned int *status;
    unsigned long long deadline_ns;   // per-channel time budget
    int red32;                   // matrix-free solver: every reduction in FP32 (the plain-FP32 form)
};

__device__ __forceinline__ float2 vobs(const CalParams &p, int c, int pidx) {
    const int k = p.pair_type[pidx];
    const float inv = 1.0f / (float)(p.win_t1[k] - p.win_t0[k]);
    if (p.vfmt == GC_C64) {
        const float2 v = reinterpret_cast<const float2 *>(p.vred)[(size_t)c * p.P + pidx];
        return make_float2(v.x * inv, v.y * inv);
    }
    const int2 v = reinterpret_cast<const int2 *>(p.vred)[(size_t)c * p.P + pidx];
    return make_float2((float)v.x * inv, (float)v.y * inv);
}

__device__ __forceinline__ float auto_of(const CalParams &p, int c, int i) {
    if (!p.autos) return 1.0f;
    if (p.vfmt == GC_C64) return reinterpret_cast<const float *>(p.autos)[(size_t)c * p.N + i];
    return (float)reinterpret_cast<const int *>(p.autos)[(size_t)c * p.N + i];
}

// index of the pair (r_j + d_k, r_j) in the selection, or -1
__device__ __forceinline__ int pair_index(const CalParams &p, int k, int xj, int yj) {
    const int dx = p.types[2 * k], dy = p.types[2 * k + 1];
    const int L = p.L;
    const int xi = xj + dx, yi = yj + dy;
    if (xj < 0 || xj >= L || yj < 0 || yj >= L || xi < 0 || xi >= L || yi < 0 || yi >= L) return -1;
    const int xlo = max(0, -dx), ylo = max(0, -dy);
    return p.type_ptr[k] + (yj - ylo) * (L - abs(dx)) + (xj - xlo);
}

template <class R>
struct C2 {
    R x, y;
};
template <class R>
__device__ __forceinline__ C2<R> cm(C2<R> a, C2<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class R>
__device__ __forceinline__ C2<R> cj(C2<R> a) {
    return {a.x, -a.y};
}

// ----------------------------------------------------------------- block reductions
template <class R, int NV>
__device__ void block_sum(R (&v)[NV], R *red /* smem [32][NV] */) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[w * NV + q] = v[q];
    __syncthreads();
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        R s = 0;
        for (int u = 0; u < nw; ++u) s += red[u * NV + q];
        v[q] = s;
    }
    __syncthreads();
}

// ----------------------------------------------------------------- start point
// Spanning-tree phases over the (1,0) and (0,1) types (arg V_(1,0) = arg V_(0,1)
// = 0 fixes the slopes), unit amplitudes, V_alpha = group mean of V_p / (g_i g_j^*).
template <class R>
__device__ void start_point(const CalParams &p, int c, R *xg, R *xv, R *red, R *phi /* N reals of scratch */) {
    const int L = p.L, N = p.N;
    if (p.tree_ant) {
        // partly occupied lattice: walk the breadth-first tree, phi_i - phi_j
        // = arg V_p along each linking pair p = (i, j); empty points get 0
        for (int i = threadIdx.x; i < N; i += blockDim.x) phi[i] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int h = 1; h < p.n_occ; ++h) {
                const int a = p.tree_ant[h], q = p.tree_pair[h];
                const float2 v = vobs(p, c, q);
                const R arg = (R)atan2f(v.y, v.x);
                phi[a] = p.tree_sign[h] > 0 ? phi[p.pair_j[q]] + arg : phi[p.pair_i[q]] - arg;
            }
        }
    } else {
        if (threadIdx.x == 0) {
            phi[0] = 0;
            for (int x = 1; x < L; ++x) {
                const float2 v = vobs(p, c, pair_index(p, p.ax, x - 1, 0));
                phi[x] = phi[x - 1] + (R)atan2f(v.y, v.x);
            }
        }
        __syncthreads();
        for (int x = threadIdx.x; x < L; x += blockDim.x) {
            R acc = phi[x];
            for (int y = 1; y < L; ++y) {
                const float2 v = vobs(p, c, pair_index(p, p.ay, x, y - 1));
                acc += (R)atan2f(v.y, v.x);
                phi[y * L + x] = acc;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        R s, co;
        if (sizeof(R) == 8) {
            double sd, cd;
            sincos((double)phi[i], &sd, &cd);
            s = (R)sd;
            co = (R)cd;
        } else {
            float sf, cf;
            sincosf((float)phi[i], &sf, &cf);
            s = (R)sf;
            co = (R)cf;
        }
        const bool occ = !p.mask || p.mask[i];   // empty points hold g = 0
        xg[2 * i] = occ ? co : (R)0;
        xg[2 * i + 1] = occ ? s : (R)0;
    }
    __syncthreads();
    // V_alpha: one warp per type
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = w; k < p.n_ubl; k += nw) {
        R sx = 0, sy = 0;
        for (int q = p.type_ptr[k] + lane; q < p.type_ptr[k + 1]; q += 32) {
            const int i = p.pair_i[q], j = p.pair_j[q];
            const float2 v = vobs(p, c, q);
            C2<R> gi{xg[2 * i], xg[2 * i + 1]}, gj{xg[2 * j], xg[2 * j + 1]};
            C2<R> e = cm(cj(gi), gj);   // 1 / (g_i g_j^*) for unit gains
            C2<R> t = cm(C2<R>{(R)v.x, (R)v.y}, e);
            sx += t.x;
            sy += t.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) {
            const R n = (R)(p.type_ptr[k + 1] - p.type_ptr[k]);
            xv[2 * k] = sx / n;
            xv[2 * k + 1] = sy / n;
        }
    }
    __syncthreads();
}

// chi^2 = sum_p |V_p - g_i g_j^* V_alpha|^2 over all pairs (one visit each)
template <class R>
__device__ R chi2_of(const CalParams &p, int c, const R *xg, const R *xv, R *red) {
    R s[1] = {0};
    for (int q = threadIdx.x; q < p.P; q += blockDim.x) {
        const int i = p.pair_i[q], j = p.pair_j[q], k = p.pair_type[q];
        const float2 v = vobs(p, c, q);
        C2<R> m = cm(cm(C2<R>{xg[2 * i], xg[2 * i + 1]}, cj(C2<R>{xg[2 * j], xg[2 * j + 1]})),
                     C2<R>{xv[2 * k], xv[2 * k + 1]});
        const R rx = (R)v.x - m.x, ry = (R)v.y - m.y;
        s[0] += rx * rx + ry * ry;
    }
    block_sum<R, 1>(s, red);
    return s[0];
}

// ----------------------------------------------------------------- lincal
template <class R>
struct GnWork {
    R *xg, *xv, *band, *border, *rhs, *S, *xs, *tg, *tv, *delta, *trial;
    int n, m, bw;
};

template <class R>
__device__ GnWork<R> gn_layout(const CalParams &p, char *base) {
    GnWork<R> w;
    w.n = 2 * p.N;
    w.m = 2 * p.n_ubl;
    w.bw = p.bw;
    R *q = reinterpret_cast<R *>(base);
    auto take = [&](size_t cnt) {
        R *r = q;
        q += (cnt + 31) & ~size_t(31);
        return r;
    };
    w.xg = take(w.n);
    w.xv = take(w.m + p.N);          // + N scratch for the start point
    w.band = take((size_t)w.n * (w.bw + 1));
    w.border = take((size_t)w.m * w.n);
    w.rhs = take(w.n + w.m);
    w.S = take((size_t)w.m * w.m);
    w.xs = take(w.n + w.m);
    w.tg = take((size_t)4 * w.n);
    w.tv = take((size_t)4 * w.m);
    w.delta = take(w.n + w.m);
    w.trial = take(w.n + w.m);
    return w;
}

template <class R>
size_t gn_bytes(int N, int n_ubl, int bw) {
    auto r = [](size_t c) { return (c + 31) & ~size_t(31); };
    const size_t n = 2 * (size_t)N, m = 2 * (size_t)n_ubl;
    return sizeof(R) * (r(n) + r(m + N) + r(n * (bw + 1)) + r(m * n) + r(n + m) + r(m * m) + r(n + m) +
                        r(4 * n) + r(4 * m) + r(n + m) + r(n + m));
}

// Jacobian blocks of one pair: dm/d(Re,Im g_i) = (a, i a), a = conj(g_j) V;
// dm/d(Re,Im g_j) = (b, -i b), b = g_i V; dm/d(Re,Im V) = (e, i e), e = g_i conj(g_j).
// As real 2x2 blocks acting on (Re x, Im x): columns are (Re z, Im z) and (Re(iz), Im(iz)).
template <class R>
struct Jb {
    R c0x, c0y, c1x, c1y;   // column 0 = (c0x, c0y), column 1 = (c1x, c1y)
};
template <class R>
__device__ __forceinline__ Jb<R> jb_plus(C2<R> z) {   // (z, i z)
    return {z.x, z.y, -z.y, z.x};
}
template <class R>
__device__ __forceinline__ Jb<R> jb_minus(C2<R> z) {  // (z, -i z)
    return {z.x, z.y, z.y, -z.x};
}
// A^T B for 2x2 real blocks given by columns
template <class R>
__device__ __forceinline__ void atb(const Jb<R> &a, const Jb<R> &b, R (&o)[2][2]) {
    o[0][0] = a.c0x * b.c0x + a.c0y * b.c0y;
    o[0][1] = a.c0x * b.c1x + a.c0y * b.c1y;
    o[1][0] = a.c1x * b.c0x + a.c1y * b.c0y;
    o[1][1] = a.c1x * b.c1x + a.c1y * b.c1y;
}

// Assemble the banded normal equations; returns chi^2 and the largest diagonal.
template <class R>
__device__ void gn_assemble(const CalParams &p, int c, GnWork<R> &w, R *red, R &chi2, R &dmax) {
    const int L = p.L, N = p.N, nu = p.n_ubl, bw = w.bw, n = w.n;
    // zero border and rhs
    for (size_t i = threadIdx.x; i < (size_t)w.m * n; i += blockDim.x) w.border[i] = 0;
    for (int i = threadIdx.x; i < n + w.m; i += blockDim.x) w.rhs[i] = 0;
    __syncthreads();
    R loc_dmax = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        R *row0 = w.band + (size_t)(2 * i) * (bw + 1);
        R *row1 = row0 + (bw + 1);
        for (int o = 0; o <= bw; ++o) {
            row0[o] = 0;
            row1[o] = 0;
        }
        const int xi = i % L, yi = i / L;
        const C2<R> gi{w.xg[2 * i], w.xg[2 * i + 1]};
        R d00 = 0, d10 = 0, d11 = 0, b0 = 0, b1 = 0;
        for (int k = 0; k < nu; ++k) {
            const C2<R> V{w.xv[2 * k], w.xv[2 * k + 1]};
            const int dx = p.types[2 * k], dy = p.types[2 * k + 1];
            // role A: pair (i, j = i - d), i is i_p
            {
                const int q = pair_index(p, k, xi - dx, yi - dy);
                if (q >= 0) {
                    const int j = (yi - dy) * L + (xi - dx);
                    const C2<R> gj{w.xg[2 * j], w.xg[2 * j + 1]};
                    const C2<R> a = cm(cj(gj), V), b = cm(gi, V), e = cm(gi, cj(gj));
                    const float2 v = vobs(p, c, q);
                    const C2<R> mm = cm(e, V);
                    const R rx = (R)v.x - mm.x, ry = (R)v.y - mm.y;
                    const Jb<R> Ji = jb_plus(a), Jj = jb_minus(b), Jv = jb_plus(e);
                    R o[2][2];
                    atb(Ji, Ji, o);
                    d00 += o[0][0];
                    d10 += o[1][0];
                    d11 += o[1][1];
                    // off-diagonal block rows (2i, 2i+1) x cols (2j, 2j+1), j < i
                    atb(Ji, Jj, o);
                    const int off = 2 * i - 2 * j;   // band offset of (2i, 2j)
                    row0[off] += o[0][0];
                    row0[off - 1] += o[0][1];
                    row1[off + 1] += o[1][0];
                    row1[off] += o[1][1];
                    // border (V_k rows) x (g_i cols)
                    atb(Jv, Ji, o);
                    w.border[(size_t)(2 * k) * n + 2 * i] += o[0][0];
                    w.border[(size_t)(2 * k) * n + 2 * i + 1] += o[0][1];
                    w.border[(size_t)(2 * k + 1) * n + 2 * i] += o[1][0];
                    w.border[(size_t)(2 * k + 1) * n + 2 * i + 1] += o[1][1];
                    b0 += Ji.c0x * rx + Ji.c0y * ry;
                    b1 += Ji.c1x * rx + Ji.c1y * ry;
                }
            }
            // role B: pair (i' = i + d, i), i is j_p
            {
                const int q = pair_index(p, k, xi, yi);
                if (q >= 0) {
                    const int ip = (yi + dy) * L + (xi + dx);
                    const C2<R> gp{w.xg[2 * ip], w.xg[2 * ip + 1]};
                    const C2<R> b = cm(gp, V), e = cm(gp, cj(gi));
                    const float2 v = vobs(p, c, q);
                    const C2<R> mm = cm(e, V);
                    const R rx = (R)v.x - mm.x, ry = (R)v.y - mm.y;
                    const Jb<R> Jj = jb_minus(b), Jv = jb_plus(e);
                    R o[2][2];
                    atb(Jj, Jj, o);
                    d00 += o[0][0];
                    d10 += o[1][0];
                    d11 += o[1][1];
                    atb(Jv, Jj, o);
                    w.border[(size_t)(2 * k) * n + 2 * i] += o[0][0];
                    w.border[(size_t)(2 * k) * n + 2 * i + 1] += o[0][1];
                    w.border[(size_t)(2 * k + 1) * n + 2 * i] += o[1][0];
                    w.border[(size_t)(2 * k + 1) * n + 2 * i + 1] += o[1][1];
                    b0 += Jj.c0x * rx + Jj.c0y * ry;
                    b1 += Jj.c1x * rx + Jj.c1y * ry;
                }
            }
        }
        row0[0] = d00;
        row1[1] = d10;
        row1[0] = d11;
        w.rhs[2 * i] = b0;
        w.rhs[2 * i + 1] = b1;
        loc_dmax = fmax(loc_dmax, fmax(d00, d11));
    }
    // model-visibility block (2x2 per type), its rhs and chi^2: one warp per type
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    R csum = 0;
    for (int k = wp; k < nu; k += nw) {
        const C2<R> V{w.xv[2 * k], w.xv[2 * k + 1]};
        R s00 = 0, s11 = 0, s10 = 0, r0 = 0, r1 = 0, cc = 0;
        for (int q = p.type_ptr[k] + lane; q < p.type_ptr[k + 1]; q += 32) {
            const int i = p.pair_i[q], j = p.pair_j[q];
            const C2<R> e = cm(C2<R>{w.xg[2 * i], w.xg[2 * i + 1]}, cj(C2<R>{w.xg[2 * j], w.xg[2 * j + 1]}));
            const float2 v = vobs(p, c, q);
            const C2<R> mm = cm(e, V);
            const R rx = (R)v.x - mm.x, ry = (R)v.y - mm.y;
            const R e2 = e.x * e.x + e.y * e.y;
            s00 += e2;
            s11 += e2;
            r0 += e.x * rx + e.y * ry;
            r1 += -e.y * rx + e.x * ry;
            cc += rx * rx + ry * ry;
        }
        for (int o = 16; o > 0; o >>= 1) {
            s00 += __shfl_xor_sync(0xffffffffu, s00, o);
            s11 += __shfl_xor_sync(0xffffffffu, s11, o);
            r0 += __shfl_xor_sync(0xffffffffu, r0, o);
            r1 += __shfl_xor_sync(0xffffffffu, r1, o);
            cc += __shfl_xor_sync(0xffffffffu, cc, o);
        }
        (void)s10;
        if (lane == 0) {
            // S holds A_VV here (diagonal 2x2 blocks: Jv^T Jv = |e|^2 I)
            w.S[(size_t)(2 * k) * w.m + 2 * k] = s00;
            w.S[(size_t)(2 * k + 1) * w.m + 2 * k + 1] = s11;
            w.S[(size_t)(2 * k + 1) * w.m + 2 * k] = 0;
            w.S[(size_t)(2 * k) * w.m + 2 * k + 1] = 0;
            w.rhs[n + 2 * k] = r0;
            w.rhs[n + 2 * k + 1] = r1;
        }
        csum += lane == 0 ? cc : (R)0;
    }
    // zero the off-diagonal blocks of A_VV (types do not share a model visibility)
    for (int idx = threadIdx.x; idx < w.m * w.m; idx += blockDim.x) {
        const int a = idx / w.m, b = idx % w.m;
        if ((a >> 1) != (b >> 1)) w.S[idx] = 0;
    }
    R v2[2] = {csum, loc_dmax};
    // chi^2 sum; max via a separate reduction
    R s1[1] = {csum};
    block_sum<R, 1>(s1, red);
    chi2 = s1[0];
    // block max of diagonals
    for (int o = 16; o > 0; o >>= 1) loc_dmax = fmax(loc_dmax, __shfl_xor_sync(0xffffffffu, loc_dmax, o));
    if (lane == 0) red[wp] = loc_dmax;
    __syncthreads();
    R mx = 0;
    for (int u = 0; u < nw; ++u) mx = fmax(mx, red[u]);
    dmax = mx;
    __syncthreads();
    (void)v2;
}

// In-place banded Cholesky of the gain block with the forward solve of the
// m border rows and the gain rhs riding along.  The diagonal keeps the
// unscaled pivot B_kk (L_kk = sqrt(B_kk)); off-diagonal entries become L.
// Column k is scaled during the pass of column k+1 (disjoint entries), so
// each column costs one barrier.  Returns false if a pivot is not positive.
template <class R>
__device__ bool gn_factor_forward(GnWork<R> &w, R mu, R *s_flag) {
    const int n = w.n, bw = w.bw, m = w.m;
    R *B = w.band;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    auto at = [&](int r, int o) -> R & { return B[(size_t)r * (bw + 1) + o]; };
    for (int r = threadIdx.x; r < n; r += blockDim.x) at(r, 0) += mu;
    __syncthreads();
    for (int k = 0; k <= n; ++k) {
        if (k > 0) {
            // finish column k-1: l_ik = B_ik / sqrt(B_kk), z_k = rhs_k / sqrt(B_kk)
            const int kk = k - 1;
            const R inv = (R)1 / sqrt(at(kk, 0));
            const int wk = min(bw, n - 1 - kk);
            for (int t = threadIdx.x; t < wk + m + 1; t += blockDim.x) {
                if (t < wk) at(kk + 1 + t, t + 1) *= inv;
                else if (t < wk + m) w.border[(size_t)(t - wk) * n + kk] *= inv;
                else w.rhs[kk] *= inv;
            }
        }
        if (k == n) break;
        const R bkk = at(k, 0);
        if (!(bkk > (R)0)) {
            if (threadIdx.x == 0) s_flag[0] = 1;
            return false;   // uniform: every thread read the same pivot
        }
        const R invb = (R)1 / bkk;
        const int wk = min(bw, n - 1 - k);
        // trailing update, one warp per row: B_ij -= B_ik B_jk / B_kk
        for (int ti = wp; ti < wk; ti += nw) {
            const int i = k + 1 + ti;
            const R bik = at(i, ti + 1) * invb;
            for (int tj = lane; tj <= ti; tj += 32) {
                const int j = k + 1 + tj;
                at(i, ti - tj) -= bik * at(j, tj + 1);
            }
        }
        // forward elimination of the border rows and the gain rhs
        for (int t = threadIdx.x; t < (m + 1) * wk; t += blockDim.x) {
            const int q = t / wk, ti = t - q * wk;
            const int i = k + 1 + ti;
            const R lik = at(i, ti + 1) * invb;
            if (q < m) w.border[(size_t)q * n + i] -= lik * w.border[(size_t)q * n + k];
            else w.rhs[i] -= lik * w.rhs[k];
        }
        __syncthreads();
    }
    __syncthreads();
    return true;
}

// Dense m x m Cholesky + solve by one warp (m <= 128); S is overwritten.
template <class R>
__device__ bool small_chol_solve(R *S, R *b, int m) {
    bool ok = true;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int k = 0; k < m; ++k) {
            R d = S[(size_t)k * m + k];
            if (!(d > (R)0)) ok = false;
            d = sqrt(d > (R)0 ? d : (R)1);
            __syncwarp();
            for (int i = k + 1 + lane; i < m; i += 32) S[(size_t)i * m + k] /= d;
            if (lane == 0) S[(size_t)k * m + k] = d;
            __syncwarp();
            for (int i = k + 1 + lane; i < m; i += 32)
                for (int j = k + 1; j <= i; ++j) S[(size_t)i * m + j] -= S[(size_t)i * m + k] * S[(size_t)j * m + k];
            __syncwarp();
        }
        if (lane == 0) {
            for (int i = 0; i < m; ++i) {
                R s = b[i];
                for (int j = 0; j < i; ++j) s -= S[(size_t)i * m + j] * b[j];
                b[i] = s / S[(size_t)i * m + i];
            }
            for (int i = m - 1; i >= 0; --i) {
                R s = b[i];
                for (int j = i + 1; j < m; ++j) s -= S[(size_t)j * m + i] * b[j];
                b[i] = s / S[(size_t)i * m + i];
            }
        }
    }
    return ok;
}

template <class R>
__device__ void gn_solve(GnWork<R> &w, R mu_rel, R *red) {
    const int n = w.n, m = w.m, bw = w.bw;
    // Schur complement S = A_VV - Z Z^T, rhs_V -= Z z  (Z = forward-solved border)
    const int npairs = m * (m + 1) / 2;
    for (int t = threadIdx.x; t < npairs + m; t += blockDim.x) {
        if (t < npairs) {
            int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
            while ((a + 1) * (a + 2) / 2 <= t) ++a;
            while (a * (a + 1) / 2 > t) --a;
            const int b = t - a * (a + 1) / 2;
            R s = 0;
            const R *za = w.border + (size_t)a * n, *zb = w.border + (size_t)b * n;
            for (int i = 0; i < n; ++i) s += za[i] * zb[i];
            w.S[(size_t)a * m + b] -= s;
            if (a != b) w.S[(size_t)b * m + a] = w.S[(size_t)a * m + b];
        } else {
            const int a = t - npairs;
            R s = 0;
            const R *za = w.border + (size_t)a * n;
            for (int i = 0; i < n; ++i) s += za[i] * w.rhs[i];
            w.rhs[n + a] -= s;
        }
    }
    __syncthreads();
    // Levenberg term on the Schur block (its near-null directions are the
    // amplitude and slope degeneracies)
    if (threadIdx.x == 0) {
        R mx = 0;
        for (int a = 0; a < m; ++a) mx = fmax(mx, w.S[(size_t)a * m + a]);
        for (int a = 0; a < m; ++a) w.S[(size_t)a * m + a] += mu_rel * mx;
    }
    __syncthreads();
    small_chol_solve<R>(w.S, w.rhs + n, m);
    __syncthreads();
    // rhs_g = z - Z^T x_V, then back substitution with L^T
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        R s = w.rhs[i];
        for (int a = 0; a < m; ++a) s -= w.border[(size_t)a * n + i] * w.rhs[n + a];
        w.rhs[i] = s;
    }
    __syncthreads();
    R *B = w.band;
    for (int k = n - 1; k >= 0; --k) {
        const R xk = w.rhs[k] / sqrt(B[(size_t)k * (bw + 1)]);
        for (int t = threadIdx.x; t < bw; t += blockDim.x) {
            const int j = k - 1 - t;
            if (j >= 0) w.rhs[j] -= B[(size_t)k * (bw + 1) + (k - j)] * xk;
        }
        if (threadIdx.x == 0) w.xs[k] = xk;
        __syncthreads();
    }
    for (int a = threadIdx.x; a < m; a += blockDim.x) w.xs[n + a] = w.rhs[n + a];
    __syncthreads();
    (void)red;
}

// Project the four degeneracy directions out of delta (Sec. 5.2).
// Solve G c = r for the 4 degeneracy coefficients from the packed lower
// triangle of the Gram matrix (acc[0..9]) and the right-hand side acc[10..13]
// (Cholesky; c = 0 when a direction vanishes).
template <class R>
__device__ void solve_gram4(const R (&acc)[14], R (&cvec)[4]) {
    R G[4][4], r[4];
    {
        int q = 0;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b <= a; ++b) {
                G[a][b] = acc[q];
                G[b][a] = acc[q];
                ++q;
            }
        for (int a = 0; a < 4; ++a) r[a] = acc[10 + a];
        // Cholesky with a guard
        R Lm[4][4] = {};
        bool ok = true;
        for (int a = 0; a < 4 && ok; ++a) {
            R s = G[a][a];
            for (int b = 0; b < a; ++b) s -= Lm[a][b] * Lm[a][b];
            if (!(s > (R)1e-30)) {
                ok = false;
                break;
            }
            Lm[a][a] = sqrt(s);
            for (int i = a + 1; i < 4; ++i) {
                R t = G[i][a];
                for (int b = 0; b < a; ++b) t -= Lm[i][b] * Lm[a][b];
                Lm[i][a] = t / Lm[a][a];
            }
        }
        if (ok) {
            R y[4];
            for (int a = 0; a < 4; ++a) {
                R s = r[a];
                for (int b = 0; b < a; ++b) s -= Lm[a][b] * y[b];
                y[a] = s / Lm[a][a];
            }
            for (int a = 3; a >= 0; --a) {
                R s = y[a];
                for (int b = a + 1; b < 4; ++b) s -= Lm[b][a] * cvec[b];
                cvec[a] = s / Lm[a][a];
            }
        } else {
            for (int a = 0; a < 4; ++a) cvec[a] = 0;
        }
    }
}

template <class R>
__device__ void gn_project(const CalParams &p, GnWork<R> &w, R *red) {
    const int n = w.n, m = w.m, L = p.L;
    // tangent vectors at the current point
    for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
        const R gx = w.xg[2 * i], gy = w.xg[2 * i + 1];
        const R xx = (R)(i % L), yy = (R)(i / L);
        R *t = w.tg;
        t[0 * n + 2 * i] = gx;          t[0 * n + 2 * i + 1] = gy;          // amplitude: g
        t[1 * n + 2 * i] = -gy;         t[1 * n + 2 * i + 1] = gx;          // phase: i g
        t[2 * n + 2 * i] = -xx * gy;    t[2 * n + 2 * i + 1] = xx * gx;     // x slope: i x g
        t[3 * n + 2 * i] = -yy * gy;    t[3 * n + 2 * i + 1] = yy * gx;     // y slope: i y g
    }
    for (int k = threadIdx.x; k < p.n_ubl; k += blockDim.x) {
        const R vx = w.xv[2 * k], vy = w.xv[2 * k + 1];
        const R dx = (R)p.types[2 * k], dy = (R)p.types[2 * k + 1];
        R *t = w.tv;
        t[0 * m + 2 * k] = -2 * vx;     t[0 * m + 2 * k + 1] = -2 * vy;     // amplitude: -2 V
        t[1 * m + 2 * k] = 0;           t[1 * m + 2 * k + 1] = 0;
        t[2 * m + 2 * k] = dx * vy;     t[2 * m + 2 * k + 1] = -dx * vx;    // -i dx V
        t[3 * m + 2 * k] = dy * vy;     t[3 * m + 2 * k + 1] = -dy * vx;
    }
    __syncthreads();
    R acc[14];
#pragma unroll
    for (int q = 0; q < 14; ++q) acc[q] = 0;
    for (int i = threadIdx.x; i < n + m; i += blockDim.x) {
        R t[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) t[a] = i < n ? w.tg[a * n + i] : w.tv[a * m + (i - n)];
        const R d = w.xs[i];
        int q = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) acc[q++] += t[a] * t[b];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[10 + a] += t[a] * d;
    }
    block_sum<R, 14>(acc, red);
    R cvec[4];
    solve_gram4<R>(acc, cvec);
    for (int i = threadIdx.x; i < n + m; i += blockDim.x) {
        R d = w.xs[i];
#pragma unroll
        for (int a = 0; a < 4; ++a) d -= cvec[a] * (i < n ? w.tg[a * n + i] : w.tv[a * m + (i - n)]);
        w.delta[i] = d;
    }
    __syncthreads();
}

// Degeneracy convention of the output: mean ln|g| = 0, arg V_(1,0) =
// arg V_(0,1) = 0, arg g_0 = 0.  Works on float2 gains in place.
__device__ void output_convention(const CalParams &p, float2 *g, float2 *V, double *red) {
    // per antenna in FP32 (the gains are FP32 values), summed in FP64
    double s[1] = {0.0};
    for (int i = threadIdx.x; i < p.N; i += blockDim.x)
        if (!p.mask || p.mask[i]) s[0] += (double)logf(hypotf(g[i].x, g[i].y));
    block_sum<double, 1>(s, red);
    const double sc = exp(s[0] / p.n_occ);
    const double kx = atan2((double)V[p.ax].y, (double)V[p.ax].x);
    const double ky = atan2((double)V[p.ay].y, (double)V[p.ay].x);
    __syncthreads();
    for (int k = threadIdx.x; k < p.n_ubl; k += blockDim.x) {
        const double ph = -(kx * p.types[2 * k] + ky * p.types[2 * k + 1]);
        double sn, cs;
        sincos(ph, &sn, &cs);
        const double vx = V[k].x * sc * sc, vy = V[k].y * sc * sc;
        V[k] = make_float2((float)(vx * cs - vy * sn), (float)(vx * sn + vy * cs));
    }
    // phase of the first antenna after the slope change (antenna 0 of a full
    // grid, at x = y = 0; the first occupied point of a partly occupied one)
    const int r0 = p.tree_ant ? p.tree_ant[0] : 0;
    const double psi = atan2((double)g[r0].y, (double)g[r0].x) + kx * (r0 % p.L) + ky * (r0 / p.L);
    __syncthreads();
    // the ramp phase in FP64, reduced to [-pi, pi] there, then rotated in FP32
    constexpr double kTwoPi = 6.283185307179586, kInvTwoPi = 0.15915494309189535;
    const float isc = (float)(1.0 / sc);
    for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
        const double ph = kx * (i % p.L) + ky * (i / p.L) - psi;
        float sn, cs;
        sincosf((float)(ph - kTwoPi * rint(ph * kInvTwoPi)), &sn, &cs);
        const float gx = g[i].x * isc, gy = g[i].y * isc;
        g[i] = make_float2(gx * cs - gy * sn, gx * sn + gy * cs);
    }
    __syncthreads();
}

template <class R>
__device__ void finish_channel(const CalParams &p, int c, const R *xg, const R *xv, int iters, int st,
                               double *red, int inner = 0) {
    float2 *g = p.gains + (size_t)c * p.N;
    float2 *V = p.vmodel + (size_t)c * p.n_ubl;
    for (int i = threadIdx.x; i < p.N; i += blockDim.x) g[i] = make_float2((float)xg[2 * i], (float)xg[2 * i + 1]);
    for (int k = threadIdx.x; k < p.n_ubl; k += blockDim.x) V[k] = make_float2((float)xv[2 * k], (float)xv[2 * k + 1]);
    __syncthreads();
    output_convention(p, g, V, red);
    // chi^2 and chi^2_r (Eq. redchi, Eq. dof) at the output point: the
    // model products in the solver's precision (FP32 for the FP32 solvers,
    // FP64 for the FP64 one), the sums in FP64; the noise weight
    // 1 / sigma_p^2 = t_p (t_a / a_i) (t_a / a_j) in FP32 (no FP64 division)
    double acc[2] = {0.0, 0.0};
    const float ta = (float)p.t_autos;
    for (int q = threadIdx.x; q < p.P; q += blockDim.x) {
        const int i = p.pair_i[q], j = p.pair_j[q], k = p.pair_type[q];
        const float2 v = vobs(p, c, q);
        double r2;
        if constexpr (sizeof(R) == sizeof(float)) {
            const float2 gi = g[i], gj = g[j], Vk = V[k];
            const float ex = gi.x * gj.x + gi.y * gj.y, ey = gi.y * gj.x - gi.x * gj.y;   // g_i conj(g_j)
            const float mx = ex * Vk.x - ey * Vk.y, my = ex * Vk.y + ey * Vk.x;
            const float rx = v.x - mx, ry = v.y - my;
            r2 = (double)rx * rx + (double)ry * ry;
        } else {
            const double gx = g[i].x, gy = g[i].y, hx = g[j].x, hy = -g[j].y;
            const double ex = gx * hx - gy * hy, ey = gx * hy + gy * hx;
            const double mx = ex * V[k].x - ey * V[k].y, my = ex * V[k].y + ey * V[k].x;
            const double rx = v.x - mx, ry = v.y - my;
            r2 = rx * rx + ry * ry;
        }
        acc[0] += r2;
        const float wp = (float)(p.win_t1[k] - p.win_t0[k]) * (ta / auto_of(p, c, i)) * (ta / auto_of(p, c, j));
        acc[1] += r2 * (double)wp;
    }
    block_sum<double, 2>(acc, red);
    if (threadIdx.x == 0) {
        gc_calstats s;
        s.chi2 = acc[0];
        s.dof = p.P - p.n_occ - p.n_ubl + 2;
        s.chi2r = p.autos && s.dof > 0 ? acc[1] / s.dof : -1.0;
        s.iters = iters;
        // observations or solution not finite: the channel has no result
        s.status = isfinite(acc[0]) ? st : GC_EINVAL;
        s.inner = inner;
        p.stats[c] = s;
    }
    __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(kCThreads) lincal_kernel(const CalParams p) {
    __shared__ R red[32 * 14];
    __shared__ double redd[64];
    __shared__ R s_flag[1];
    GnWork<R> w = gn_layout<R>(p, p.work + (size_t)blockIdx.x * p.work_per_cta);
    for (int c = blockIdx.x; c < p.C; c += gridDim.x) {
        const uint64_t t_start = gc_globaltimer();
        if (p.warm) {
            for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
                const float2 g = p.gains[(size_t)c * p.N + i];
                w.xg[2 * i] = g.x;
                w.xg[2 * i + 1] = g.y;
            }
            for (int k = threadIdx.x; k < p.n_ubl; k += blockDim.x) {
                const float2 v = p.vmodel[(size_t)c * p.n_ubl + k];
                w.xv[2 * k] = v.x;
                w.xv[2 * k + 1] = v.y;
            }
            __syncthreads();
        } else {
            start_point<R>(p, c, w.xg, w.xv, red, w.xv + 2 * p.n_ubl);
        }
        int st = GC_ENOCONV, it = 0;
        for (it = 1; it <= p.max_iter; ++it) {
            R chi2, dmax;
            gn_assemble<R>(p, c, w, red, chi2, dmax);
            const R mu = (R)p.mu_rel * dmax;
            if (!gn_factor_forward<R>(w, mu, s_flag)) {
                st = GC_EDEGEN;
                break;
            }
            gn_solve<R>(w, (R)p.mu_rel, red);
            gn_project<R>(p, w, red);
            // norms for the convergence test
            R nr[2] = {0, 0};
            for (int i = threadIdx.x; i < w.n + w.m; i += blockDim.x) {
                const R x = i < w.n ? w.xg[i] : w.xv[i - w.n];
                nr[0] += x * x;
                nr[1] += w.delta[i] * w.delta[i];
            }
            block_sum<R, 2>(nr, red);
            // halving line search on chi^2
            R step = 1;
            for (int ls = 0; ls < 8; ++ls) {
                for (int i = threadIdx.x; i < w.n + w.m; i += blockDim.x)
                    w.trial[i] = (i < w.n ? w.xg[i] : w.xv[i - w.n]) + step * w.delta[i];
                __syncthreads();
                const R c2 = chi2_of<R>(p, c, w.trial, w.trial + w.n, red);
                if (c2 <= chi2 * (R)(1 + 1e-12) + (R)1e-30 || ls == 7) break;
                step *= (R)0.5;
            }
            for (int i = threadIdx.x; i < w.n + w.m; i += blockDim.x) {
                if (i < w.n) w.xg[i] = w.trial[i];
                else w.xv[i - w.n] = w.trial[i];
            }
            __syncthreads();
            if (step * sqrt(nr[1]) <= (R)p.tol * sqrt(nr[0])) {
                st = GC_OK;
                break;
            }
            if (gc_globaltimer() - t_start > p.deadline_ns) {
                st = GC_ETIMEOUT;
                if (threadIdx.x == 0) atomicOr(p.status, GC_DEV_TIMEOUT_CAL);
                break;
            }
        }
        finish_channel<R>(p, c, w.xg, w.xv, min(it, p.max_iter), st, redd);
    }
}

// ----------------------------------------------------------------- lincal, matrix-free (mixed precision)
// Gauss-Newton with the step from preconditioned conjugate gradients on
// (J^T J + mu I) delta = J^T r, never forming J^T J.  Two operator forms: the
// gather over the grid in relative coordinates (rel_op_pass and
// cg_solve_channel_rel, for selections of <= kStencilTypes types) and the
// pair-list scatter below (cg_pass and cg_solve_channel, any selection).
// The scatter form is one pass over the pairs: each pair evaluates its entry of J v,
//   u_p = a_p v_gi + b_p conj(v_gj) + e_p v_V,  a = conj(g_j) V, b = g_i V, e = g_i conj(g_j),
// and scatters J^T u -- conj(a) u to g_i, b conj(u) to g_j (shared-memory
// atomics) and conj(e) u to V (warp-reduced when a warp's pairs share a type,
// which the type-major pair order makes the common case).  The diagonal
// blocks of J^T J are |a|^2 I and |e|^2 I, the Jacobi preconditioner.  FP32
// products, FP64 reductions; the randomly accessed vectors (state, search
// direction, operator output, diagonals) live in shared memory when they fit.
struct CgWork {
    float *xg, *xv;          // state 2N; 2 n_ubl (+ N scratch for the start point)
    float *pp, *acc;         // search direction and operator output (n + m)
    float *dg, *dv;          // Jacobi diagonals (N, n_ubl)
    float *b, *x, *r, *z, *trial, *tg;   // streaming vectors (global); tg: 4 (n + m)
    // two-level preconditioner: patch-aggregation coarse space (see cg_coarse_setup)
    float *Ca, *Cp;          // coarse amplitude / phase operators, then their inverses (nc x nc)
    float *rc, *yc;          // coarse residual / solution (2 nc; shared memory)
    float *cscr;             // shared-memory scratch for one nc x nc system (or null)
    // relative-coordinate solver (stencil operator): |g_i|^2 then |V_k|^2, the
    // diagonal of J^T J in those coordinates, and the coarse index per element
    float *G, *D;
    unsigned short *cid;
    int coarse_gather;       // every type offset within one patch side: gather assembly
    int n, m;
    int B, npx, ncp, nc, cv; // patch side, patches per row, patches, coarse size, V in coarse space
};

constexpr int kMaxCoarse = 160;

__host__ __device__ inline void cg_coarse_dims(int L, int n_ubl, int &B, int &npx, int &ncp, int &nc, int &cv) {
    B = L >= 16 ? L / 8 : (L >= 4 ? 2 : 1);
    npx = (L + B - 1) / B;
    ncp = npx * npx;
    cv = n_ubl <= 64 ? 1 : 0;
    nc = ncp + (cv ? n_ubl : 0);
    if (nc > kMaxCoarse) {   // keep the coarse system small
        cv = 0;
        nc = ncp;
    }
}

// Vectors read at random per pair (xg 2N, xv 2 n_ubl, pp and acc nm each, dv
// n_ubl) and, when `with_dg`, the gain diagonal dg (N).
__host__ __device__ inline size_t cg_hot_floats(int N, int n_ubl, bool with_dg) {
    return 6 * (size_t)N + 7 * (size_t)n_ubl + (with_dg ? (size_t)N : 0) + 64;
}

// Shared-memory vectors of the relative-coordinate solver: the search
// direction q (gathered by the operator), G = |g|^2 / |V|^2 (gathered), the
// Jacobi diagonal D and the coarse index of every element.
__host__ __device__ inline size_t cg_sten_floats(int N, int n_ubl) {
    const size_t ne = (size_t)N + n_ubl;
    return 2 * ne + 2 * ne + (ne + 1) / 2 + 64;   // q, G, D, coarse index (16 bit)
}

// hot_mode 2: hot vectors and dg in shared memory; 1: hot vectors in shared
// memory, dg in global; 0: everything in global (L2-resident) memory;
// 3 (stencil operator): xg, xv and pp in shared memory, the rest in global.
__device__ CgWork cg_layout(const CalParams &p, char *base, float *smem_arena, int smem_floats, int hot_mode,
                            bool use_coarse_smem) {
    CgWork w;
    w.n = 2 * p.N;
    w.m = 2 * p.n_ubl;
    const size_t nm = w.n + w.m;
    float *g = reinterpret_cast<float *>(base);
    auto takeg = [&](size_t cnt) {
        float *r = g;
        g += (cnt + 63) & ~size_t(63);
        return r;
    };
    float *ghot = takeg(cg_hot_floats(p.N, p.n_ubl, true));
    float *h = hot_mode == 1 || hot_mode == 2 ? smem_arena : ghot;
    float *hot_end = hot_mode == 3 ? smem_arena + cg_sten_floats(p.N, p.n_ubl)
                                   : h + cg_hot_floats(p.N, p.n_ubl, hot_mode != 1);
    w.xg = h;
    h += 2 * p.N;
    w.xv = h;
    h += 2 * p.n_ubl;
    w.pp = h;
    h += nm;
    w.acc = h;
    h += nm;
    w.dv = h;
    h += p.n_ubl;
    w.dg = hot_mode == 1 ? ghot : h;
    // relative-coordinate vectors: in the arena (mode 3) or in global memory
    {
        float *rb = hot_mode == 3 ? smem_arena : takeg(cg_sten_floats(p.N, p.n_ubl));
        const int ne = p.N + p.n_ubl;
        if (hot_mode == 3) w.pp = rb;   // q replaces the search direction
        w.G = rb + 2 * ne;
        w.D = w.G + ne;
        w.cid = reinterpret_cast<unsigned short *>(w.D + ne);
    }
    w.b = takeg(nm);
    w.x = takeg(nm);
    w.r = takeg(nm);
    w.z = takeg(nm);
    w.trial = takeg(nm);
    w.tg = takeg(4 * nm);
    cg_coarse_dims(p.L, p.n_ubl, w.B, w.npx, w.ncp, w.nc, w.cv);
    if (use_coarse_smem) {
        w.Ca = hot_end;
        w.Cp = hot_end + (size_t)w.nc * w.nc;
    } else {
        w.Ca = takeg((size_t)w.nc * w.nc);
        w.Cp = takeg((size_t)w.nc * w.nc);
    }
    w.coarse_gather = 1;
    for (int k = 0; k < p.n_ubl; ++k)
        if (abs(p.types[2 * k]) > w.B || abs(p.types[2 * k + 1]) > w.B) w.coarse_gather = 0;
    w.cscr = nullptr;
    if (!use_coarse_smem && smem_floats > 0) {   // room for one system beside the hot vectors?
        float *sc = hot_mode == 0 ? smem_arena : hot_end;
        if (sc + (size_t)w.nc * w.nc <= smem_arena + smem_floats) w.cscr = sc;
    }
    return w;
}

__host__ __device__ inline size_t cg_coarse_floats(int L, int n_ubl) {
    int B, npx, ncp, nc, cv;
    cg_coarse_dims(L, n_ubl, B, npx, ncp, nc, cv);
    return 2 * (size_t)nc * nc;
}

size_t cg_bytes(int N, int n_ubl, int /*P*/) {
    auto r = [](size_t c) { return (c + 63) & ~size_t(63); };
    const size_t nm = 2 * (size_t)N + 2 * (size_t)n_ubl;
    int B, npx, ncp, nc, cv;
    const int L = (int)lround(sqrt((double)N));
    cg_coarse_dims(L, n_ubl, B, npx, ncp, nc, cv);
    const size_t c2 = (size_t)nc * nc;
    return sizeof(float) * (r(cg_hot_floats(N, n_ubl, true)) + 5 * r(nm) + r(4 * nm) + 2 * r(c2) +
                            r(cg_sten_floats(N, n_ubl)));
}

// Shared arena for one array: hot vectors with dg and the coarse operators if
// they fit the cap, else the hot vectors alone, else nothing (0: global).
// The split mode (hot vectors in shared memory, dg in global) is kept in the
// kernel but not chosen: on the 4096-antenna array it measured slower than
// the all-global layout, whose fire-and-forget L2 reductions do not stall
// the issuing warps the way contended shared-memory atomics do.
// With the stencil operator the arena holds only the gathered vectors (and
// the coarse operators when they fit beside them).
size_t cg_arena_bytes(int N, int n_ubl, int L, size_t cap, bool stencil) {
    const size_t h2 = (stencil ? cg_sten_floats(N, n_ubl) : cg_hot_floats(N, n_ubl, true)) * sizeof(float);
    const size_t cf = cg_coarse_floats(L, n_ubl) * sizeof(float);
    const size_t c1 = cf / 2;   // one system: the inversion's shared-memory scratch
    if (h2 + cf <= cap) return h2 + cf;
    if (h2 + c1 <= cap) return h2 + c1;
    if (h2 <= cap) return h2;
    return c1 <= cap ? c1 : 0;
}

// the kernel side of the same choice, from the arena size it was given
__device__ __forceinline__ void cg_modes(const CalParams &p, int smem_floats, int &hot_mode, bool &coarse_smem) {
    const size_t cf = cg_coarse_floats(p.L, p.n_ubl), sf = (size_t)smem_floats;
    if (p.stencil) {
        const size_t hs = cg_sten_floats(p.N, p.n_ubl);
        hot_mode = hs <= sf ? 3 : 0;
        coarse_smem = hot_mode != 0 && hs + cf <= sf;
        return;
    }
    const size_t h2 = cg_hot_floats(p.N, p.n_ubl, true), h1 = cg_hot_floats(p.N, p.n_ubl, false);
    hot_mode = h2 <= sf ? 2 : (h1 <= sf ? 1 : 0);
    coarse_smem = hot_mode != 0 && (hot_mode == 2 ? h2 : h1) + cf <= sf;
}

// One pass over the pairs.  resid: u = r (the residual), acc = J^T r, dg/dv
// = diagonals, returns chi^2.  Otherwise u = J pp and acc = J^T u.
// Each warp walks a contiguous chunk of the (type-major) pair list, so the
// model-visibility terms accumulate in registers and are flushed with one
// warp reduction per type boundary.
// kPipe: hot vectors in global memory -- pipeline the pair loads (a separate
// instantiation: the pipeline's registers would slow the shared-memory form)
template <bool kPipe>
__device__ double cg_pass(const CalParams &p, int c, const CgWork &w, bool resid, double *red) {
    const int nm = w.n + w.m;
    if (resid) {   // the operator passes find acc already zeroed by the caller
        for (int i = threadIdx.x; i < nm; i += blockDim.x) w.acc[i] = 0.f;
        for (int i = threadIdx.x; i < p.N; i += blockDim.x) w.dg[i] = 0.f;
        for (int k = threadIdx.x; k < p.n_ubl; k += blockDim.x) w.dv[k] = 0.f;
        __syncthreads();
    }
    float chi = 0.f;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int chunk = ((p.P + nw - 1) / nw + 31) & ~31;
    const int q_lo = wp * chunk, q_hi = min(p.P, q_lo + chunk);
    int k_cur = q_lo < q_hi ? p.pair_type[q_lo] : 0;
    float vx = 0.f, vy = 0.f, vd = 0.f;
    auto flush = [&](int k) {
        float a = vx, b = vy, d = vd;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (lane == 0) {
            atomicAdd(&w.acc[w.n + 2 * k], a);
            atomicAdd(&w.acc[w.n + 2 * k + 1], b);
            if (resid) atomicAdd(&w.dv[k], d);
        }
        vx = vy = vd = 0.f;
    };
    // software pipeline over 32-pair batches: the index loads run two
    // batches ahead and the gathers one batch ahead of the arithmetic and the
    // reductions, so each warp keeps three batches of L2 traffic in flight
    struct Idx {
        int i, j, k, q;
    };
    struct Dat {
        int i, j, k, q;
        float gix, giy, gjx, gjy, Vx, Vy, a0, a1, a2, a3, a4, a5;
    };
    auto fetch_idx = [&](int q) {
        Idx r{-1, -1, 0, q};
        if (q < q_hi) {
            r.i = p.pair_i[q];
            r.j = p.pair_j[q];
            r.k = p.pair_type[q];
        }
        return r;
    };
    auto fetch_dat = [&](const Idx &x) {
        Dat d;
        d.i = x.i;
        d.j = x.j;
        d.k = x.k;
        d.q = x.q;
        if (x.i >= 0) {
            d.gix = w.xg[2 * x.i];
            d.giy = w.xg[2 * x.i + 1];
            d.gjx = w.xg[2 * x.j];
            d.gjy = w.xg[2 * x.j + 1];
            d.Vx = w.xv[2 * x.k];
            d.Vy = w.xv[2 * x.k + 1];
            if (resid) {
                const float2 o = vobs(p, c, x.q);
                d.a0 = o.x;
                d.a1 = o.y;
            } else {
                d.a0 = w.pp[2 * x.i];
                d.a1 = w.pp[2 * x.i + 1];
                d.a2 = w.pp[2 * x.j];
                d.a3 = w.pp[2 * x.j + 1];
                d.a4 = w.pp[w.n + 2 * x.k];
                d.a5 = w.pp[w.n + 2 * x.k + 1];
            }
        }
        return d;
    };
    auto process = [&](const Dat &d) {
        const bool valid = d.i >= 0;
        const int k = valid ? d.k : k_cur;
        float ux = 0.f, uy = 0.f, ex = 0.f, ey = 0.f;
        if (valid) {
            const int i = d.i, j = d.j;
            const float gix = d.gix, giy = d.giy, gjx = d.gjx, gjy = d.gjy, Vx = d.Vx, Vy = d.Vy;
            ex = gix * gjx + giy * gjy;
            ey = giy * gjx - gix * gjy;                                        // g_i conj(g_j)
            const float ax = gjx * Vx + gjy * Vy, ay = gjx * Vy - gjy * Vx;    // conj(g_j) V
            const float bx = gix * Vx - giy * Vy, by = gix * Vy + giy * Vx;    // g_i V
            if (resid) {
                ux = d.a0 - (ex * Vx - ey * Vy);
                uy = d.a1 - (ex * Vy + ey * Vx);
                chi = fmaf(ux, ux, fmaf(uy, uy, chi));
                atomicAdd(&w.dg[i], ax * ax + ay * ay);
                atomicAdd(&w.dg[j], bx * bx + by * by);
            } else {
                const float vix = d.a0, viy = d.a1, vjx = d.a2, vjy = -d.a3, vvx = d.a4, vvy = d.a5;
                ux = ax * vix - ay * viy + bx * vjx - by * vjy + ex * vvx - ey * vvy;
                uy = ax * viy + ay * vix + bx * vjy + by * vjx + ex * vvy + ey * vvx;
            }
            // conj(a) u -> g_i ; b conj(u) -> g_j
            atomicAdd(&w.acc[2 * i], ax * ux + ay * uy);
            atomicAdd(&w.acc[2 * i + 1], ax * uy - ay * ux);
            atomicAdd(&w.acc[2 * j], bx * ux + by * uy);
            atomicAdd(&w.acc[2 * j + 1], by * ux - bx * uy);
        }
        // conj(e) u -> V_k (and |e|^2 -> dv_k)
        const float tx = ex * ux + ey * uy, ty = ex * uy - ey * ux, td = resid ? ex * ex + ey * ey : 0.f;
        if (__all_sync(0xffffffffu, k == k_cur)) {
            vx += tx;
            vy += ty;
            vd += td;
        } else {
            flush(k_cur);
            if (valid) {
                atomicAdd(&w.acc[w.n + 2 * k], tx);
                atomicAdd(&w.acc[w.n + 2 * k + 1], ty);
                if (resid) atomicAdd(&w.dv[k], td);
            }
            k_cur = __shfl_sync(0xffffffffu, k, 31);
        }
    };
    if (q_lo < q_hi) {
        if constexpr (kPipe) {
            Idx nxt = fetch_idx(q_lo + 32 + lane);
            Dat cur = fetch_dat(fetch_idx(q_lo + lane));
            for (int q0 = q_lo; q0 < q_hi; q0 += 32) {
                const Dat d2 = fetch_dat(nxt);   // gathers of the next batch
                nxt = fetch_idx(q0 + 64 + lane); // indices two batches ahead
                process(cur);
                cur = d2;
            }
        } else {   // shared-memory hot vectors: short latencies, no pipeline
            for (int q0 = q_lo; q0 < q_hi; q0 += 32) process(fetch_dat(fetch_idx(q0 + lane)));
        }
    }
    if (q_lo < q_hi) flush(k_cur);
    double s[1] = {(double)chi};
    if (resid) block_sum<double, 1>(s, red);
    else __syncthreads();
    return s[0];
}

// Relative coordinates.  With the step written as dg_i = g_i q_i and
// dV_k = V_k w_k, the linearised model of pair p = (i, j) of type k is
//   dM_p = m_p (q_i + conj(q_j) + w_k),   m_p = g_i conj(g_j) V_k,
// so in (q, w) the Gauss-Newton matrix is a weighted graph operator with the
// real weights W_p = |m_p|^2 = |g_i|^2 |g_j|^2 |V_k|^2:
//   (A q)_i = sum_{p: i first} W_p s_p + sum_{p: i second} W_p conj(s_p),
//   (A q)_k = sum_{p in k} W_p s_p,     s_p = q_i + conj(q_j) + w_k,
// the right-hand side is sum conj(m_p) r_p (first) + m_p conj(r_p) (second),
// and the Levenberg term mu I becomes mu |g_i|^2 / mu |V_k|^2.  This is the
// same system as the (g, V) form under the diagonal change of variables, so
// preconditioned CG takes the same steps (the Jacobi and patch-level coarse
// spaces map onto themselves), but an operator evaluation costs a handful
// of adds and multiplies instead of three complex products.
//
// The thread owning antenna m evaluates its pairs as first member (m, m - d_k)
// and as second member (m + d_k, m), found by grid arithmetic (every
// selection takes baseline-types whole, in pair_index order), and sums its
// own row in registers: every pair is visited by both antennas and nothing
// is scattered, so there are no atomics and the result does not depend on
// the schedule.  The model-visibility rows are summed per type over the
// first-member visits in registers and reduced across the warp, then in
// shared memory across the CTA.
// Antenna order of the stencil passes: index t < n_in walks the interior
// (antennas at least st_halo from every edge, whose pairs of every type are
// all on the grid) in row order; t >= n_in walks the border ring: the h top
// rows, the h bottom rows, then the 2h edge columns of each middle row.
// Without an interior (L <= 2h) t is the grid index itself.
struct RelOrder {
    int L, h, Wi, n_in;
    __device__ explicit RelOrder(const CalParams &p) : L(p.L), h(p.st_halo) {
        Wi = L > 2 * h ? L - 2 * h : 0;
        n_in = Wi * Wi;
    }
    __device__ __forceinline__ int antenna(int t) const {
        if (t < n_in) {
            const int yy = t / Wi;
            return (yy + h) * L + (t - yy * Wi) + h;
        }
        if (n_in == 0) return t;
        const int u = t - n_in, hl = h * L;
        if (u < 2 * hl) return u < hl ? u : (L - h) * L + (u - hl);
        const int v = u - 2 * hl, row = h + v / (2 * h), ci = v - (row - h) * 2 * h;
        return row * L + (ci < h ? ci : L - 2 * h + ci);
    }
};

// The end of a residual pass: |V_k|^2, dv_k, the chi^2 block sum and the
// largest gain diagonal, from the thread's chi^2 part and running maximum
// (acc, G and D of the antennas and the type sums are written by then).
__device__ double rel_resid_finish(const CalParams &p, const CgWork &w, const float *xv, double *red, float *dmax,
                                   float chi, float dm) {
    const int nu = p.n_ubl, N = p.N;
    for (int k = threadIdx.x; k < nu; k += blockDim.x) {
        const float Uk = xv[2 * k] * xv[2 * k] + xv[2 * k + 1] * xv[2 * k + 1];
        w.G[N + k] = Uk;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nu; k += blockDim.x) w.dv[k] = w.G[N + k] > 0.f ? w.D[N + k] / w.G[N + k] : 0.f;
    for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    double s[1] = {(double)chi};
    if (p.red32) {   // the plain-FP32 form: the chi^2 sum in FP32 as well
        float sf[1] = {(float)chi};
        block_sum<float, 1>(sf, reinterpret_cast<float *>(red));
        s[0] = (double)sf[0];
    } else {
        block_sum<double, 1>(s, red);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)dm;
    __syncthreads();
    double mx = 0.0;
    for (int u = 0; u < (int)(blockDim.x >> 5); ++u) mx = fmax(mx, red[u]);
    __syncthreads();
    *dmax = (float)mx;
    return s[0];
}

template <int VF>
__device__ __forceinline__ float2 rel_obs(const CalParams &p, int c, int q, float inv) {
    if (VF == GC_C64) {
        const float2 v = reinterpret_cast<const float2 *>(p.vred)[(size_t)c * p.P + q];
        return make_float2(v.x * inv, v.y * inv);
    }
    const int2 v = reinterpret_cast<const int2 *>(p.vred)[(size_t)c * p.P + q];
    return make_float2((float)v.x * inv, (float)v.y * inv);
}

// Residual pass at the current (g, V): chi^2 (returned), the right-hand side
// in relative coordinates (acc), G, the diagonal D of A and, for the coarse
// operators, dv_k = D_k / |V_k|^2.  Also returns, in *dmax, the largest
// (g, V)-form gain diagonal D_i / G_i that scales the Levenberg term.
// Antenna m visits its pairs as first member (m, m - d_k), at pair index
// b_k + y W_k + x - (d_y W_k + d_x), and as second member (m + d_k, m), at
// b_k + y W_k + x (W_k = L - |d_x|, b_k the type's first pair less its
// start offset), in the order of RelOrder; each type's constants come from
// two shared-memory records.  Interior antennas skip the on-grid tests; on
// the ring a pair off the grid reads element 0 and is selected away.
template <int VF>
__device__ __forceinline__ float2 rel_obs(const void *vc, int q, float inv) {
    if (VF == GC_C64) {
        const float2 v = reinterpret_cast<const float2 *>(vc)[q];
        return make_float2(v.x * inv, v.y * inv);
    }
    const int2 v = reinterpret_cast<const int2 *>(vc)[q];
    return make_float2((float)v.x * inv, (float)v.y * inv);
}

template <int VF>
__device__ double rel_resid_pass_t(const CalParams &p, int c, const CgWork &w, bool staged, double *red, float *dmax) {
    constexpr int KT = kStencilTypes;
    __shared__ float s_tsum[(kCgStThreads / 32) * 3 * KT];
    __shared__ int4 s_ra[KT];     // per type: offset d_k, d_y W_k + d_x, b_k, W_k
    __shared__ float4 s_rb[KT];   // per type: 1 / window, V_k
    const int L = p.L, nu = p.n_ubl, N = p.N, bd = blockDim.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = bd >> 5;
    // the gains are gathered from a copy in the q area (free between CG
    // solves); a staged point (a line-search trial) is there already,
    // followed by its model visibilities
    float2 *xg = reinterpret_cast<float2 *>(w.pp);
    const float *xv = staged ? w.pp + 2 * N : w.xv;
    if (!staged)
        for (int m = threadIdx.x; m < N; m += bd) xg[m] = reinterpret_cast<const float2 *>(w.xg)[m];
    if (threadIdx.x < nu) {
        const int k = threadIdx.x;
        const int dx = __ldg(p.types + 2 * k), dy = __ldg(p.types + 2 * k + 1), W = L - abs(dx);
        s_ra[k] = make_int4(dy * L + dx, dy * W + dx, __ldg(p.type_ptr + k) - max(0, -dy) * W - max(0, -dx), W);
        s_rb[k] = make_float4(1.0f / (float)(__ldg(p.win_t1 + k) - __ldg(p.win_t0 + k)), xv[2 * k], xv[2 * k + 1], 0.f);
    }
    __syncthreads();
    const void *vc = VF == GC_C64 ? (const void *)(reinterpret_cast<const float2 *>(p.vred) + (size_t)c * p.P)
                                  : (const void *)(reinterpret_cast<const int2 *>(p.vred) + (size_t)c * p.P);
    float tvx[KT], tvy[KT], tvd[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) tvx[k] = tvy[k] = tvd[k] = 0.f;
    float chi = 0.f, dm = 0.f;
    const RelOrder ord(p);
    for (int t = threadIdx.x; t < N; t += bd) {
        const int m = ord.antenna(t), x = m % L, y = m / L;
        const float2 gm = xg[m];
        float sx = 0.f, sy = 0.f, sd = 0.f;
        // one copy of the type loop per path (kIn: interior, no tests)
        auto types_loop = [&](auto kIn) {
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                if (k >= nu) break;
                const int4 ra = s_ra[k];
                const float4 rb = s_rb[k];
                bool v1 = true, v2 = true;
                if (!decltype(kIn)::value) {
                    const int dx = __ldg(p.types + 2 * k), dy = __ldg(p.types + 2 * k + 1);
                    v1 = (unsigned)(x - dx) < (unsigned)L && (unsigned)(y - dy) < (unsigned)L;
                    v2 = (unsigned)(x + dx) < (unsigned)L && (unsigned)(y + dy) < (unsigned)L;
                }
                const int i2 = ra.z + y * ra.w + x;
                const float2 gj = xg[v1 ? m - ra.x : 0], gi = xg[v2 ? m + ra.x : 0];
                const float2 o1 = rel_obs<VF>(vc, v1 ? i2 - ra.y : 0, rb.x);
                const float2 o2 = rel_obs<VF>(vc, v2 ? i2 : 0, rb.x);
                {   // m first: pair (m, j = m - d_k)
                    const float ex = gm.x * gj.x + gm.y * gj.y, ey = gm.y * gj.x - gm.x * gj.y;   // g_m conj(g_j)
                    const float mx = ex * rb.y - ey * rb.z, my = ex * rb.z + ey * rb.y;         // model m_p
                    const float rx = o1.x - mx, ry = o1.y - my;
                    const float Wp = v1 ? mx * mx + my * my : 0.f;
                    const float hx = v1 ? mx * rx + my * ry : 0.f, hy = v1 ? mx * ry - my * rx : 0.f;   // conj(m) r
                    chi = v1 ? fmaf(rx, rx, fmaf(ry, ry, chi)) : chi;
                    sd += Wp;
                    tvd[k] += Wp;
                    sx += hx;
                    sy += hy;
                    tvx[k] += hx;
                    tvy[k] += hy;
                }
                {   // m second: pair (i = m + d_k, m)
                    const float ex = gi.x * gm.x + gi.y * gm.y, ey = gi.y * gm.x - gi.x * gm.y;   // g_i conj(g_m)
                    const float mx = ex * rb.y - ey * rb.z, my = ex * rb.z + ey * rb.y;
                    const float rx = o2.x - mx, ry = o2.y - my;
                    sd += v2 ? mx * mx + my * my : 0.f;
                    sx += v2 ? mx * rx + my * ry : 0.f;   // m conj(r)
                    sy += v2 ? my * rx - mx * ry : 0.f;
                }
            }
        };
        if (t < ord.n_in) types_loop(std::true_type());
        else types_loop(std::false_type());
        const float Gm = gm.x * gm.x + gm.y * gm.y;
        w.acc[2 * m] = sx;
        w.acc[2 * m + 1] = sy;
        w.G[m] = Gm;
        w.D[m] = sd;
        dm = fmaxf(dm, Gm > 0.f ? sd / Gm : 0.f);
    }
    // per-type rows: warp trees, then one thread per type sums over the warps
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        if (k >= nu) break;
        for (int o = 16; o > 0; o >>= 1) {
            tvx[k] += __shfl_xor_sync(0xffffffffu, tvx[k], o);
            tvy[k] += __shfl_xor_sync(0xffffffffu, tvy[k], o);
            tvd[k] += __shfl_xor_sync(0xffffffffu, tvd[k], o);
        }
        if (lane == 0) {
            s_tsum[(wp * 3 + 0) * KT + k] = tvx[k];
            s_tsum[(wp * 3 + 1) * KT + k] = tvy[k];
            s_tsum[(wp * 3 + 2) * KT + k] = tvd[k];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * nu; t += bd) {
        const int comp = t / nu, k = t - comp * nu;
        float a = 0.f;
        for (int u = 0; u < nw; ++u) a += s_tsum[(u * 3 + comp) * KT + k];
        if (comp < 2) w.acc[2 * (N + k) + comp] = a;
        else w.D[N + k] = a;
    }
    return rel_resid_finish(p, w, xv, red, dmax, chi, dm);
}

__device__ double rel_resid_pass(const CalParams &p, int c, const CgWork &w, bool staged, double *red, float *dmax) {
    return p.vfmt == GC_C64 ? rel_resid_pass_t<GC_C64>(p, c, w, staged, red, dmax)
                            : rel_resid_pass_t<GC_I4C>(p, c, w, staged, red, dmax);
}


// acc = A q (relative coordinates, no Levenberg term): the search direction
// q is w.pp, G and q are gathered (shared memory when the arena holds them).
// Returns this thread's part of q.(A q + mu G q), the CG curvature; acc and
// the partial sums are complete after the caller's next block reduction.
__device__ float rel_op_pass(const CalParams &p, const CgWork &w, float mu) {
    constexpr int KT = kStencilTypes;
    __shared__ float s_tsum[(kCgStThreads / 32) * 2 * KT];
    __shared__ float4 s_ty[KT];   // per type: offset d_k (as int bits), w_k, G_k
    const int L = p.L, nu = p.n_ubl, N = p.N;
    const float2 *q = reinterpret_cast<const float2 *>(w.pp);
    const float *G = w.G;
    if (threadIdx.x < nu) {
        const int k = threadIdx.x;
        const float2 wk = q[N + k];
        s_ty[k] = make_float4(__int_as_float(__ldg(p.types + 2 * k + 1) * L + __ldg(p.types + 2 * k)), wk.x, wk.y,
                              G[N + k]);
    }
    __syncthreads();
    float tvx[KT], tvy[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) tvx[k] = tvy[k] = 0.f;
    float curv = 0.f;
    // Antennas at least st_halo from every edge (index t < n_in, in row
    // order) have both pairs of every type on the grid and take the path
    // without tests; the rest of the grid (the border ring, t >= n_in)
    // tests each pair.
    const RelOrder ord(p);
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const int m = ord.antenna(t);
        const float2 qm = q[m];
        const float Gm = G[m];
        float sx = 0.f, sy = 0.f;
        if (t < ord.n_in) {
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                if (k >= nu) break;
                const float4 ty = s_ty[k];
                const int off = __float_as_int(ty.x);
                const float2 qj = q[m - off], qi = q[m + off];
                const float GU = Gm * ty.w;
                const float W1 = GU * G[m - off], W2 = GU * G[m + off];
                // m first: s = q_m + conj(q_j) + w_k
                const float ax = qm.x + ty.y + qj.x, ay = qm.y + ty.z - qj.y;
                sx = fmaf(W1, ax, sx);
                sy = fmaf(W1, ay, sy);
                tvx[k] = fmaf(W1, ax, tvx[k]);
                tvy[k] = fmaf(W1, ay, tvy[k]);
                // m second: conj(s) = conj(q_i) + q_m + conj(w_k)
                sx = fmaf(W2, qi.x + qm.x + ty.y, sx);
                sy = fmaf(W2, qm.y - qi.y - ty.z, sy);
            }
        } else {
            const int x = m % L, y = m / L;
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                if (k >= nu) break;
                const int dx = __ldg(p.types + 2 * k), dy = __ldg(p.types + 2 * k + 1);
                const float4 ty = s_ty[k];
                const int off = __float_as_int(ty.x);
                // without branches: a pair off the grid reads antenna m itself
                // and gets weight 0 (fmaf(0, a, s) = s, so the sums are those
                // of the pairs that exist)
                const bool v1 = (unsigned)(x - dx) < (unsigned)L && (unsigned)(y - dy) < (unsigned)L;
                const bool v2 = (unsigned)(x + dx) < (unsigned)L && (unsigned)(y + dy) < (unsigned)L;
                const int j = v1 ? m - off : m, i = v2 ? m + off : m;
                const float2 qj = q[j], qi = q[i];
                const float GU = Gm * ty.w;
                const float W1 = v1 ? GU * G[j] : 0.f, W2 = v2 ? GU * G[i] : 0.f;
                const float ax = qm.x + ty.y + qj.x, ay = qm.y + ty.z - qj.y;
                sx = fmaf(W1, ax, sx);
                sy = fmaf(W1, ay, sy);
                tvx[k] = fmaf(W1, ax, tvx[k]);
                tvy[k] = fmaf(W1, ay, tvy[k]);
                sx = fmaf(W2, qi.x + qm.x + ty.y, sx);
                sy = fmaf(W2, qm.y - qi.y - ty.z, sy);
            }
        }
        w.acc[2 * m] = sx;
        w.acc[2 * m + 1] = sy;
        const float mg = mu * Gm;
        curv = fmaf(qm.x, sx + mg * qm.x, fmaf(qm.y, sy + mg * qm.y, curv));
    }
    // per-type rows: warp trees, then one thread per type sums over the warps
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        if (k >= nu) break;
        for (int o = 16; o > 0; o >>= 1) {
            tvx[k] += __shfl_xor_sync(0xffffffffu, tvx[k], o);
            tvy[k] += __shfl_xor_sync(0xffffffffu, tvy[k], o);
        }
        if (lane == 0) {
            s_tsum[(wp * 2 + 0) * KT + k] = tvx[k];
            s_tsum[(wp * 2 + 1) * KT + k] = tvy[k];
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nu; k += blockDim.x) {
        float ax = 0.f, ay = 0.f;
        for (int u = 0; u < nw; ++u) {
            ax += s_tsum[(u * 2 + 0) * KT + k];
            ay += s_tsum[(u * 2 + 1) * KT + k];
        }
        w.acc[2 * (N + k)] = ax;
        w.acc[2 * (N + k) + 1] = ay;
        const float2 wk = q[N + k];
        const float mg = mu * G[N + k];
        curv = fmaf(wk.x, ax + mg * wk.x, fmaf(wk.y, ay + mg * wk.y, curv));
    }
    return curv;
}

// chi^2 at a trial point (g, V) (global memory), each pair once: the thread
// owning antenna m takes the pairs (m, m - d_k).
__device__ float rel_chi2(const CalParams &p, int c, const float *tg, const float *tv, float *red) {
    constexpr int KT = kStencilTypes;
    const int L = p.L, nu = p.n_ubl;
    const float2 *g = reinterpret_cast<const float2 *>(tg);
    const float2 *vobs2 = reinterpret_cast<const float2 *>(p.vred) + (size_t)c * p.P;
    const int2 *vobsi = reinterpret_cast<const int2 *>(p.vred) + (size_t)c * p.P;
    float s[1] = {0.f};
    for (int m = threadIdx.x; m < p.N; m += blockDim.x) {
        const int x = m % L, y = m / L;
        const float2 gm = g[m];
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            if (k >= nu) break;
            const int dx = __ldg(p.types + 2 * k), dy = __ldg(p.types + 2 * k + 1);
            const int xj = x - dx, yj = y - dy;
            if (xj < 0 || xj >= L || yj < 0 || yj >= L) continue;
            const float inv = 1.0f / (float)(__ldg(p.win_t1 + k) - __ldg(p.win_t0 + k));
            const int q = __ldg(p.type_ptr + k) + (yj - max(0, -dy)) * (L - abs(dx)) + (xj - max(0, -dx));
            float ox, oy;
            if (p.vfmt == GC_C64) {
                const float2 v = vobs2[q];
                ox = v.x * inv;
                oy = v.y * inv;
            } else {
                const int2 v = vobsi[q];
                ox = (float)v.x * inv;
                oy = (float)v.y * inv;
            }
            const float2 gj = g[m - (dy * L + dx)];
            const float Vx = tv[2 * k], Vy = tv[2 * k + 1];
            const float ex = gm.x * gj.x + gm.y * gj.y, ey = gm.y * gj.x - gm.x * gj.y;
            const float rx = ox - (ex * Vx - ey * Vy), ry = oy - (ex * Vy + ey * Vx);
            s[0] = fmaf(rx, rx, fmaf(ry, ry, s[0]));
        }
    }
    block_sum<float, 1>(s, red);
    return s[0];
}

// Two-level preconditioner.  The coarse space scales each patch of B x B
// antennas by one complex factor and (when there are few types) each model
// visibility by another: dg_i = g_i c_P(i), dV_k = V_k c_k.  For a pair, J
// applied to it gives u_p = m_p (c_Pi + conj(c_Pj) + c_k) with m_p the model,
// so the coarse normal matrix splits into a real "amplitude" system
// (Re c: c_Pi + c_Pj + c_k) and a real "phase" system (Im c: c_Pi - c_Pj + c_k),
// each with entries sum |m_p|^2 -- the patch-level form of Eq. logcal.  The
// coarse operators are inverted (Gauss-Jordan in FP32, with a diagonal shift
// of 1e-5 of the largest diagonal entry) at the first Gauss-Newton iteration
// -- the first two for the pair-list form -- and reused after it; applied in
// FP32: M^-1 = D^-1 + R A_c^-1 R^T.
__device__ __forceinline__ int patch_of(const CgWork &w, int i, int L) {
    return ((i / L) / w.B) * w.npx + (i % L) / w.B;
}

// Single-barrier block sum (FP32 warp trees, fixed-order cross-warp sum):
// buf holds two [32][NV] slots used alternately, so no trailing barrier is
// needed before the next reduction.
constexpr int kFastSumMax = 3;   // values per fast_sum; buf holds 2 x 32 x kFastSumMax floats
template <int NV>
__device__ __forceinline__ void fast_sum(float (&v)[NV], float *buf, int &parity) {
    static_assert(NV <= kFastSumMax, "fast_sum slot size");
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    float *b = buf + parity * 32 * kFastSumMax;   // fixed slots: sums of any size alternate safely
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) b[wp * NV + q] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        float t = 0.f;
        for (int u = 0; u < nw; ++u) t += b[u * NV + q];
        v[q] = t;
    }
    parity ^= 1;
}

// Scatter assembly over the pair list (shared or global atomics), for any
// selection; the upper triangle is accumulated and mirrored.
__device__ void coarse_assemble_scatter(const CalParams &p, const CgWork &w, float mu) {
    const int nc = w.nc, L = p.L;
    for (int t = threadIdx.x; t < nc * nc; t += blockDim.x) {
        w.Ca[t] = 0.f;
        w.Cp[t] = 0.f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < p.P; q += blockDim.x) {
        const int i = p.pair_i[q], j = p.pair_j[q], k = p.pair_type[q];
        const float gix = w.xg[2 * i], giy = w.xg[2 * i + 1], gjx = w.xg[2 * j], gjy = w.xg[2 * j + 1];
        const float Vx = w.xv[2 * k], Vy = w.xv[2 * k + 1];
        const float ex = gix * gjx + giy * gjy, ey = giy * gjx - gix * gjy;
        const float wq = (ex * ex + ey * ey) * (Vx * Vx + Vy * Vy);   // |m_p|^2
        const int a = patch_of(w, i, L), b = patch_of(w, j, L);
        // upper triangle only (row <= col); symmetrised below
        if (a == b) {
            atomicAdd(&w.Ca[a * nc + a], 4.f * wq);
        } else {
            const int lo = min(a, b), hi = max(a, b);
            atomicAdd(&w.Ca[a * nc + a], wq);
            atomicAdd(&w.Ca[b * nc + b], wq);
            atomicAdd(&w.Ca[lo * nc + hi], wq);
            atomicAdd(&w.Cp[a * nc + a], wq);
            atomicAdd(&w.Cp[b * nc + b], wq);
            atomicAdd(&w.Cp[lo * nc + hi], -wq);
        }
        if (w.cv) {
            const int kc = w.ncp + k;   // > every patch index
            if (a == b) {
                atomicAdd(&w.Ca[a * nc + kc], 2.f * wq);
            } else {
                atomicAdd(&w.Ca[a * nc + kc], wq);
                atomicAdd(&w.Ca[b * nc + kc], wq);
                atomicAdd(&w.Cp[a * nc + kc], wq);
                atomicAdd(&w.Cp[b * nc + kc], -wq);
            }
        }
    }
    __syncthreads();
    // Levenberg term mu R^T R: patch P gets mu sum |g_i|^2; the type diagonal
    // is sum_p |m_p|^2 = |V_k|^2 dv_k (+ mu |V_k|^2)
    for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
        const int a = patch_of(w, i, L);
        const float g2 = w.xg[2 * i] * w.xg[2 * i] + w.xg[2 * i + 1] * w.xg[2 * i + 1];
        atomicAdd(&w.Ca[a * nc + a], mu * g2);
        atomicAdd(&w.Cp[a * nc + a], mu * g2);
    }
    if (w.cv)
        for (int k = threadIdx.x; k < p.n_ubl; k += blockDim.x) {
            const int kc = w.ncp + k;
            const float v2 = w.xv[2 * k] * w.xv[2 * k] + w.xv[2 * k + 1] * w.xv[2 * k + 1];
            w.Ca[kc * nc + kc] = v2 * (w.dv[k] + mu);
            w.Cp[kc * nc + kc] = v2 * (w.dv[k] + mu);
        }
    __syncthreads();
    for (int t = threadIdx.x; t < nc * nc; t += blockDim.x) {   // lower from upper
        const int r = t / nc, cc = t % nc;
        if (r > cc) {
            w.Ca[t] = w.Ca[cc * nc + r];
            w.Cp[t] = w.Cp[cc * nc + r];
        }
    }
    __syncthreads();
}

// Gather assembly: one warp per patch a walks the patch's antennas and, for
// every type, the antenna's pair as first and as second member (the same
// grid arithmetic as rel_op_pass, weights from G), summing row a of both coarse
// operators in registers: the patch itself, its eight neighbour patches
// (pairs never reach further when every type offset is within one patch
// side) and the model-visibility columns.  A pair inside the patch is met
// twice and adds half its weight at each visit.  Rows are written whole
// (no atomics, no mirroring); the type rows take their patch columns from
// the same sums and a diagonal of |V_k|^2 (dv_k + mu).
__device__ void coarse_assemble_gather(const CalParams &p, const CgWork &w, float mu) {
    constexpr int KT = kStencilTypes;
    const int nc = w.nc, L = p.L, B = w.B, npx = w.npx, ncp = w.ncp, nu = p.n_ubl;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float *G = w.G;   // |g_i|^2, then |V_k|^2 (relative-coordinate residual pass)
    for (int a = wp; a < ncp; a += nw) {
        const int ax = a % npx, ay = a / npx;
        float sa[9], sp[9], ta[KT], tp[KT];
#pragma unroll
        for (int q = 0; q < 9; ++q) sa[q] = sp[q] = 0.f;
#pragma unroll
        for (int k = 0; k < KT; ++k) ta[k] = tp[k] = 0.f;
        const int x0 = ax * B, y0 = ay * B;
        const int bw = min(B, L - x0), bh = min(B, L - y0);
        for (int t = lane; t < bw * bh; t += 32) {
            const int x = x0 + t % bw, y = y0 + t / bw, m = y * L + x;
            const float gm2 = G[m];
            sa[4] += mu * gm2;
            sp[4] += mu * gm2;
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                if (k >= nu) break;
                const int dx = __ldg(p.types + 2 * k), dy = __ldg(p.types + 2 * k + 1);
                const float v2 = G[p.N + k];
#pragma unroll
                for (int role = 0; role < 2; ++role) {
                    const int xo = role == 0 ? x - dx : x + dx, yo = role == 0 ? y - dy : y + dy;
                    if (xo < 0 || xo >= L || yo < 0 || yo >= L) continue;
                    const float wq = gm2 * G[yo * L + xo] * v2;   // |m_p|^2
                    const int px = xo / B - ax, py = yo / B - ay;              // in -1..1
                    if (px == 0 && py == 0) {
                        sa[4] += 2.f * wq;
                        ta[k] += wq;
                    } else {
                        const int slot = (py + 1) * 3 + (px + 1);
                        sa[4] += wq;
                        sp[4] += wq;
#pragma unroll
                        for (int q = 0; q < 9; ++q)
                            if (q == slot) {
                                sa[q] += wq;
                                sp[q] -= wq;
                            }
                        ta[k] += wq;
                        tp[k] += role == 0 ? wq : -wq;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q)
            for (int o = 16; o > 0; o >>= 1) {
                sa[q] += __shfl_xor_sync(0xffffffffu, sa[q], o);
                sp[q] += __shfl_xor_sync(0xffffffffu, sp[q], o);
            }
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            if (k >= nu) break;
            for (int o = 16; o > 0; o >>= 1) {
                ta[k] += __shfl_xor_sync(0xffffffffu, ta[k], o);
                tp[k] += __shfl_xor_sync(0xffffffffu, tp[k], o);
            }
        }
        // row a (every lane holds every sum)
        for (int cc = lane; cc < nc; cc += 32) {
            float va = 0.f, vp = 0.f;
            if (cc < ncp) {
                const int px = cc % npx - ax, py = cc / npx - ay;
                if (px >= -1 && px <= 1 && py >= -1 && py <= 1) {
                    const int slot = (py + 1) * 3 + (px + 1);
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        if (q == slot) {
                            va = sa[q];
                            vp = sp[q];
                        }
                }
            } else {
                const int k = cc - ncp;
#pragma unroll
                for (int q = 0; q < KT; ++q)
                    if (q == k) {
                        va = ta[q];
                        vp = tp[q];
                    }
            }
            w.Ca[a * nc + cc] = va;
            w.Cp[a * nc + cc] = vp;
        }
        // column a of the type rows
        if (w.cv)
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                if (k >= nu) break;
                if (lane == k) {
                    w.Ca[(ncp + k) * nc + a] = ta[k];
                    w.Cp[(ncp + k) * nc + a] = tp[k];
                }
            }
    }
    if (w.cv)
        for (int t = threadIdx.x; t < nu * nu; t += blockDim.x) {
            const int k = t / nu, k2 = t - k * nu, r = ncp + k, cc = ncp + k2;
            float d = 0.f;
            if (k == k2) d = (w.xv[2 * k] * w.xv[2 * k] + w.xv[2 * k + 1] * w.xv[2 * k + 1]) * (w.dv[k] + mu);
            w.Ca[r * nc + cc] = d;
            w.Cp[r * nc + cc] = d;
        }
    __syncthreads();
}

// Block-wide max / sum of one float (all threads get the result).
__device__ __forceinline__ float block_allreduce(float v, bool is_max, float *buf /* [32] */) {
    for (int o = 16; o > 0; o >>= 1) {
        const float t = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmaxf(v, t) : v + t;
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) buf[wp] = v;
    __syncthreads();
    float r = buf[0];
    for (int u = 1; u < nw; ++u) r = is_max ? fmaxf(r, buf[u]) : r + buf[u];
    return r;
}

// Invert one coarse system in place with the whole CTA: diagonal floor,
// Gauss-Jordan without pivoting (SPD), two barriers per pivot, then the
// projection P A^-1 P that removes the exact coarse null direction n
// (amplitude: patches 1, types -2; phase: patches 1, types 0).
__device__ void coarse_invert(float *A, int nc, int ncp, bool amp, bool cv, float *u /* nc */, float *buf) {
    const int tid = threadIdx.x, nt = blockDim.x, nn = nc * nc;
    float mx = 0.f;
    for (int r = tid; r < nc; r += nt) mx = fmaxf(mx, A[r * nc + r]);
    mx = block_allreduce(mx, true, buf);
    for (int r = tid; r < nc; r += nt) A[r * nc + r] += 1e-5f * mx;
    __syncthreads();
    const int dr = nt / nc, dc = nt - dr * nc;
    for (int k = 0; k < nc; ++k) {
        const float iv = 1.f / A[k * nc + k];
        int r = tid / nc, c = tid - r * nc;
        for (int e = tid; e < nn; e += nt) {
            if (r != k && c != k) A[e] -= A[r * nc + k] * A[k * nc + c] * iv;
            c += dc;
            r += dr;
            if (c >= nc) {
                c -= nc;
                ++r;
            }
        }
        __syncthreads();
        for (int q = tid; q < nc; q += nt)
            if (q != k) {
                A[q * nc + k] *= -iv;
                A[k * nc + q] *= iv;
            }
        if (tid == 0) A[k * nc + k] = iv;
        __syncthreads();
    }
    if (amp && !cv) return;
    auto nv = [&](int t) -> float { return t < ncp ? 1.f : (amp ? -2.f : 0.f); };
    float cl = 0.f, sl = 0.f;
    for (int r = tid; r < nc; r += nt) {
        float acc = 0.f;
        for (int t = 0; t < nc; ++t) acc = fmaf(A[r * nc + t], nv(t), acc);
        u[r] = acc;
        cl += nv(r) * acc;
        sl += nv(r) * nv(r);
    }
    const float cs = block_allreduce(cl, false, buf);
    const float ss = block_allreduce(sl, false, buf);   // its barriers also publish u
    const float is = 1.f / ss;
    int r = tid / nc, c = tid - r * nc;
    for (int e = tid; e < nn; e += nt) {
        A[e] += -u[r] * nv(c) * is - nv(r) * u[c] * is + nv(r) * nv(c) * cs * is * is;
        c += dc;
        r += dr;
        if (c >= nc) {
            c -= nc;
            ++r;
        }
    }
    __syncthreads();
}

// Build and invert the coarse operators (the first Gauss-Newton iteration of the
// relative-coordinate solver, the first two of the pair-list solver).
__device__ void cg_coarse_setup(const CalParams &p, const CgWork &w, float mu) {
    __shared__ float s_buf[32];
    if (p.stencil && w.coarse_gather) coarse_assemble_gather(p, w, mu);
    else coarse_assemble_scatter(p, w, mu);
    const int nn = w.nc * w.nc;
    for (int m = 0; m < 2; ++m) {
        float *A = m ? w.Cp : w.Ca;
        float *W = w.cscr ? w.cscr : A;   // invert in shared memory when there is room
        if (W != A) {
            for (int e = threadIdx.x; e < nn; e += blockDim.x) W[e] = A[e];
            __syncthreads();
        }
        coarse_invert(W, w.nc, w.ncp, m == 0, w.cv != 0, w.yc, s_buf);
        if (W != A) {
            for (int e = threadIdx.x; e < nn; e += blockDim.x) A[e] = W[e];
            __syncthreads();
        }
    }
}

// One channel of matrix-free Gauss-Newton (used by the per-selection and the
// batched kernels).  All threads of the CTA call it.  The CG iteration takes
// four barriers (six with the coarse correction).
template <bool kPipe>
__device__ void cg_solve_channel(const CalParams &p, int c, CgWork &w, double cg_tol, int cg_max, double *red,
                                 float *redf) {
    const int nm = w.n + w.m, ne = p.N + p.n_ubl, L = p.L, nc = w.nc;
    GnWork<float> gw;   // view for the shared projection helper
    gw.xg = w.xg;
    gw.xv = w.xv;
    gw.tg = w.tg;
    gw.tv = w.tg + 4 * w.n;
    gw.xs = w.x;
    gw.delta = w.z;
    gw.n = w.n;
    gw.m = w.m;
    __shared__ float sbuf[2 * 32 * kFastSumMax];
    int par = 0;
    const bool coarse = nc > 0;
    const uint64_t t_start = gc_globaltimer();
    if (p.warm) {
        for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
            const float2 g = (!p.mask || p.mask[i]) ? p.gains[(size_t)c * p.N + i] : make_float2(0.f, 0.f);
            w.xg[2 * i] = g.x;
            w.xg[2 * i + 1] = g.y;
        }
        for (int k = threadIdx.x; k < p.n_ubl; k += blockDim.x) {
            const float2 v = p.vmodel[(size_t)c * p.n_ubl + k];
            w.xv[2 * k] = v.x;
            w.xv[2 * k + 1] = v.y;
        }
        __syncthreads();
    } else {
        start_point<float>(p, c, w.xg, w.xv, redf, w.z);
    }
    // complex element e: antenna e < N, else model visibility e - N
    auto base_of = [&](int e) { return e < p.N ? 2 * e : w.n + 2 * (e - p.N); };
    auto dinv = [&](int e, float mu) { return e < p.N ? 1.f / (w.dg[e] + mu) : 1.f / (w.dv[e - p.N] + mu); };
    auto cidx_of = [&](int e) { return e < p.N ? patch_of(w, e, L) : (w.cv ? w.ncp + (e - p.N) : -1); };
    // z = D^-1 r (+ R y after the coarse solve); restriction rc += conj(s) r
    auto precondition = [&](float mu) {
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            const int b = base_of(e);
            const float rx = w.r[b], ry = w.r[b + 1], iv = dinv(e, mu);
            w.z[b] = rx * iv;
            w.z[b + 1] = ry * iv;
            if (coarse) {
                const int ci = cidx_of(e);
                if (ci >= 0) {
                    const float sx = e < p.N ? w.xg[b] : w.xv[b - w.n];
                    const float sy = e < p.N ? w.xg[b + 1] : w.xv[b - w.n + 1];
                    atomicAdd(&w.rc[ci], sx * rx + sy * ry);
                    atomicAdd(&w.rc[nc + ci], sx * ry - sy * rx);
                }
            }
        }
        if (!coarse) return;
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * nc; t += blockDim.x) {
            const int m = t / nc, row = t - m * nc;
            const float *A = m ? w.Cp : w.Ca;
            const float *rr = w.rc + m * nc;
            float acc = 0.f;
            for (int cc = 0; cc < nc; ++cc) acc = fmaf(A[row * nc + cc], rr[cc], acc);
            w.yc[t] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            const int ci = cidx_of(e);
            if (ci < 0) continue;
            const int b = base_of(e);
            const float sx = e < p.N ? w.xg[b] : w.xv[b - w.n];
            const float sy = e < p.N ? w.xg[b + 1] : w.xv[b - w.n + 1];
            const float ya = w.yc[ci], yp = w.yc[nc + ci];
            w.z[b] += sx * ya - sy * yp;
            w.z[b + 1] += sx * yp + sy * ya;
        }
        for (int t = threadIdx.x; t < 2 * nc; t += blockDim.x) w.rc[t] = 0.f;   // for the next use
    };
    for (int t = threadIdx.x; t < 2 * kMaxCoarse; t += blockDim.x) w.rc[t] = 0.f;
    int st = GC_ENOCONV, it, inner = 0;
    double grad0 = 0.0;
    for (it = 1; it <= p.max_iter; ++it) {
        // residual, right-hand side J^T r and the Jacobi diagonals
        const double chi2 = cg_pass<kPipe>(p, c, w, true, red);
        double dm = 0.0;
        for (int i = threadIdx.x; i < p.N; i += blockDim.x) dm = fmax(dm, (double)w.dg[i]);
        for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dm;
        __syncthreads();
        double dmax = 0.0;
        for (int u = 0; u < (int)(blockDim.x >> 5); ++u) dmax = fmax(dmax, red[u]);
        __syncthreads();
        const float mu = (float)(p.mu_rel * dmax);
        if (coarse && it <= 2) cg_coarse_setup(p, w, mu);   // later iterations reuse it
        // PCG from x = 0
        for (int i = threadIdx.x; i < nm; i += blockDim.x) {
            w.b[i] = w.acc[i];
            w.x[i] = 0.f;
            w.r[i] = w.acc[i];
        }
        __syncthreads();
        precondition(mu);
        // vector loops walk complex elements so that each thread owns both
        // halves of what it precondition()s -- no barrier between them
        float v2[2] = {0.f, 0.f};
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            const int b = base_of(e);
            for (int h = 0; h < 2; ++h) {
                const float ri = w.r[b + h], zi = w.z[b + h];
                w.pp[b + h] = zi;
                w.acc[b + h] = 0.f;
                v2[0] = fmaf(ri, zi, v2[0]);
                v2[1] = fmaf(ri, ri, v2[1]);
            }
        }
        fast_sum<2>(v2, sbuf, par);
        float rz = v2[0];
        const float bnorm2 = v2[1];
        // inexact Newton: each linear solve stops at a relative residual
        // eta = min(0.05, (|grad| / |grad_0|)^(1/4)) (floor cg_tol).  Gauss-
        // Newton on a problem with noise in the data converges linearly, so
        // tighter solves buy little: on the 4096-antenna workload this
        // forcing takes 76 CG steps a channel over 9.0 Gauss-Newton
        // iterations where (|grad| / |grad_0|)^(1/2) capped at 0.1 took 159
        // over 9.3, for the same solution to within FP32 rounding.
        if (it == 1) grad0 = bnorm2;
        const float eta =
            (float)fmin(0.05, fmax(cg_tol, sqrt(sqrt(sqrt((double)bnorm2 / fmax(grad0, 1e-300))))));
        for (int k = 0; k < cg_max && bnorm2 > 0.f; ++k) {
            ++inner;
            cg_pass<kPipe>(p, c, w, false, red);          // acc = J^T J pp (acc was zeroed)
            float v1[1] = {0.f};
            for (int i = threadIdx.x; i < nm; i += blockDim.x) v1[0] = fmaf(w.pp[i], w.acc[i] + mu * w.pp[i], v1[0]);
            fast_sum<1>(v1, sbuf, par);
            if (!(v1[0] > 0.f)) break;
            const float alpha = rz / v1[0];
            for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                const int b = base_of(e);
                for (int h = 0; h < 2; ++h) {
                    const float pi_ = w.pp[b + h];
                    w.x[b + h] += alpha * pi_;
                    w.r[b + h] -= alpha * (w.acc[b + h] + mu * pi_);
                }
            }
            precondition(mu);
            float v3[2] = {0.f, 0.f};
            for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                const int b = base_of(e);
                for (int h = 0; h < 2; ++h) {
                    const float ri = w.r[b + h];
                    v3[0] = fmaf(ri, w.z[b + h], v3[0]);
                    v3[1] = fmaf(ri, ri, v3[1]);
                }
            }
            fast_sum<2>(v3, sbuf, par);
            if (v3[1] <= eta * eta * bnorm2) break;
            const float beta = v3[0] / rz;
            rz = v3[0];
            for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                const int b = base_of(e);
                for (int h = 0; h < 2; ++h) {
                    w.pp[b + h] = w.z[b + h] + beta * w.pp[b + h];
                    w.acc[b + h] = 0.f;
                }
            }
            __syncthreads();
        }
        __syncthreads();
        // project out the degeneracies (delta lands in w.z), line search, update
        gn_project<float>(p, gw, redf);
        double nr[2] = {0.0, 0.0};
        for (int i = threadIdx.x; i < nm; i += blockDim.x) {
            const float x = i < w.n ? w.xg[i] : w.xv[i - w.n];
            nr[0] += (double)x * x;
            nr[1] += (double)w.z[i] * w.z[i];
        }
        block_sum<double, 2>(nr, red);
        float step = 1.f;
        for (int ls = 0; ls < 8; ++ls) {
            for (int i = threadIdx.x; i < nm; i += blockDim.x)
                w.trial[i] = (i < w.n ? w.xg[i] : w.xv[i - w.n]) + step * w.z[i];
            __syncthreads();
            const float c2 = chi2_of<float>(p, c, w.trial, w.trial + w.n, redf);
            if ((double)c2 <= chi2 * (1.0 + 1e-6) + 1e-30 || ls == 7) break;
            step *= 0.5f;
        }
        for (int i = threadIdx.x; i < nm; i += blockDim.x) {
            if (i < w.n) w.xg[i] = w.trial[i];
            else w.xv[i - w.n] = w.trial[i];
        }
        __syncthreads();
        if ((double)step * sqrt(nr[1]) <= p.tol * sqrt(nr[0])) {
            st = GC_OK;
            break;
        }
        if (gc_globaltimer() - t_start > p.deadline_ns) {
            st = GC_ETIMEOUT;
            if (threadIdx.x == 0) atomicOr(p.status, GC_DEV_TIMEOUT_CAL);
            break;
        }
    }
    finish_channel<float>(p, c, w.xg, w.xv, min(it, p.max_iter), st, red, inner);
}

// One channel of matrix-free Gauss-Newton in relative coordinates (the
// stencil operator; see rel_op_pass).  Same outer iteration, forcing terms,
// preconditioner, projection, line search and stopping rule as
// cg_solve_channel; the CG vectors hold (q, w) and the search direction q
// lives in shared memory beside G, D and the coarse indices.  Convergence
// tests use the (g, V)-form norms, |r|^2 / G per element.
__device__ void cg_solve_channel_rel(const CalParams &p, int c, CgWork &w, double cg_tol, int cg_max, double *red,
                                     float *redf) {
    const int ne = p.N + p.n_ubl, L = p.L, nc = w.nc, N = p.N;
    __shared__ float sbuf[2 * 32 * kFastSumMax];
    int par = 0;
    const bool coarse = nc > 0;
    const uint64_t t_start = gc_globaltimer();
    if (p.warm) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const float2 g = p.gains[(size_t)c * N + i];
            w.xg[2 * i] = g.x;
            w.xg[2 * i + 1] = g.y;
        }
        for (int k = threadIdx.x; k < p.n_ubl; k += blockDim.x) {
            const float2 v = p.vmodel[(size_t)c * p.n_ubl + k];
            w.xv[2 * k] = v.x;
            w.xv[2 * k + 1] = v.y;
        }
        __syncthreads();
    } else {
        start_point<float>(p, c, w.xg, w.xv, redf, w.z);
    }
    // coarse index of every element (0xffff: none)
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        int ci = -1;
        if (coarse) ci = e < N ? patch_of(w, e, L) : (w.cv ? w.ncp + (e - N) : -1);
        w.cid[e] = ci < 0 ? (unsigned short)0xffff : (unsigned short)ci;
    }
    float2 *q = reinterpret_cast<float2 *>(w.pp);
    float2 *acc = reinterpret_cast<float2 *>(w.acc);
    float2 *xs = reinterpret_cast<float2 *>(w.x);
    float2 *rs = reinterpret_cast<float2 *>(w.r);
    float2 *zs = reinterpret_cast<float2 *>(w.z);
    float2 *bs = reinterpret_cast<float2 *>(w.b);
    // Preconditioner M^-1 r = (D + mu G)^-1 r + R A_c^-1 R^T r, split so that
    // each CG step streams the global vectors three times: jacobi() applies
    // the diagonal, restricts r to the coarse space (rc) and returns the
    // partial dots r.z_j and |r|^2 (in (g, V)-form norm); coarse() solves
    // y = A_c^-1 rc and returns y.rc (= r.R y), so r.z = r.z_j + y.rc without
    // another pass; the prolongation z = z_j + R y rides on the q update.
    // (called by every lane of a warp, e >= ne with r = 0: the restriction
    // sums each run of equal coarse index across the warp -- consecutive
    // antennas share a patch -- and the run's first lane adds it once; when
    // B divides both L and 32 every patch row is an aligned run of B lanes)
    const bool aligned_runs = coarse && w.B > 0 && L % w.B == 0 && 32 % w.B == 0;
    auto jacobi = [&](int e, float2 r, float mu, float &rzj, float &rr) {
        int ci = -1;
        if (e < ne) {
            // the preconditioner's diagonal and the norm's weights by the
            // fast reciprocal (within 2 ulp; a preconditioner only has to be
            // the same operator at every step, which this is)
            const float iv = __fdividef(1.f, w.D[e] + mu * w.G[e]);
            const float2 z = make_float2(r.x * iv, r.y * iv);
            zs[e] = z;
            rzj = fmaf(r.x, z.x, fmaf(r.y, z.y, rzj));
            rr += __fdividef(r.x * r.x + r.y * r.y, w.G[e]);
            const unsigned cu = w.cid[e];
            ci = cu == 0xffffu ? -1 : (int)cu;
        }
        if (!coarse) return;
        const int lane = threadIdx.x & 31;
        float qx = r.x, qy = r.y;
        if (aligned_runs && e - lane + 32 <= N) {
            // a warp of antennas whose patch rows are aligned runs of B
            // lanes: a butterfly within each run, its first lane adds it
            for (int o = 1; o < w.B; o <<= 1) {
                qx += __shfl_xor_sync(0xffffffffu, qx, o);
                qy += __shfl_xor_sync(0xffffffffu, qy, o);
            }
            if ((lane & (w.B - 1)) == 0 && ci >= 0) {
                atomicAdd(&w.rc[ci], qx);
                atomicAdd(&w.rc[nc + ci], qy);
            }
            return;
        }
        const int kprev = __shfl_up_sync(0xffffffffu, ci, 1);
        const bool head = lane == 0 || kprev != ci;
        {
            const int run = __popc(__ballot_sync(0xffffffffu, head) & (0xffffffffu >> (31 - lane)));
            for (int o = 1; o < 32; o <<= 1) {
                const float tx = __shfl_down_sync(0xffffffffu, qx, o);
                const float ty = __shfl_down_sync(0xffffffffu, qy, o);
                const int tr = __shfl_down_sync(0xffffffffu, run, o);
                if (lane + o < 32 && tr == run) {
                    qx += tx;
                    qy += ty;
                }
            }
        }
        if (head && ci >= 0) {
            atomicAdd(&w.rc[ci], qx);
            atomicAdd(&w.rc[nc + ci], qy);
        }
    };
    auto coarse_solve = [&]() {   // after a barrier that completes rc
        float ry = 0.f;
        if (!coarse) return ry;
        for (int t2 = threadIdx.x; t2 < 2 * nc; t2 += blockDim.x) {
            const int m = t2 / nc, row = t2 - m * nc;
            const float *arow = (m ? w.Cp : w.Ca) + (size_t)row * nc;
            const float *rr = w.rc + m * nc;
            // four partial sums, so that the row's loads (global memory when
            // the coarse operators do not fit beside the vectors) overlap
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            int cc = 0;
#pragma unroll 4
            for (; cc + 4 <= nc; cc += 4) {
                a0 = fmaf(arow[cc], rr[cc], a0);
                a1 = fmaf(arow[cc + 1], rr[cc + 1], a1);
                a2 = fmaf(arow[cc + 2], rr[cc + 2], a2);
                a3 = fmaf(arow[cc + 3], rr[cc + 3], a3);
            }
            for (; cc < nc; ++cc) a0 = fmaf(arow[cc], rr[cc], a0);
            const float a = (a0 + a1) + (a2 + a3);
            w.yc[t2] = a;
            ry = fmaf(a, w.rc[t2], ry);
        }
        return ry;
    };
    // q = z_j + R y + beta q (q is not read when first: the arena may hold
    // anything, NaN patterns included, before the first update); rc is
    // cleared for the next restriction
    auto update_q = [&](float beta, bool first) {
        constexpr int U = 4;   // elements whose z loads are in flight together
        for (int e0 = threadIdx.x; e0 < ne; e0 += U * blockDim.x) {
            float2 zu[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * blockDim.x;
                zu[u] = e < ne ? zs[e] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= ne) break;
            float2 z = zu[u];
            if (coarse) {
                const unsigned ci = w.cid[e];
                if (ci != 0xffffu) {
                    z.x += w.yc[ci];
                    z.y += w.yc[nc + ci];
                }
            }
            if (first) {
                q[e] = z;
            } else {
                const float2 pq = q[e];
                q[e] = make_float2(z.x + beta * pq.x, z.y + beta * pq.y);
            }
            }
        }
        for (int t2 = threadIdx.x; t2 < 2 * nc; t2 += blockDim.x) w.rc[t2] = 0.f;
        __syncthreads();
    };
    for (int t2 = threadIdx.x; t2 < 2 * kMaxCoarse; t2 += blockDim.x) w.rc[t2] = 0.f;
    int st = GC_ENOCONV, it = 1, inner = 0;
    double grad0 = 0.0, chi2 = 0.0;
    double nr[2] = {0.0, 0.0};   // |x|^2 and |step|^2 of the last projected step
    bool staged = false;         // the q area holds the last iteration's full step
    float2 *stage = q;
    for (;;) {
        // residual, right-hand side, G, D and the Levenberg scale, at the
        // current point or at the staged full step of the last iteration.
        // A halving line search on chi^2 follows every step: the full step
        // is tried with this (whole) pass, so that when it is taken (nearly
        // always) the pass is also the next iteration's; shorter steps are
        // tried with chi^2 alone.  (One call site keeps one copy of the
        // pass in the instruction stream.)
        float dmax = 0.f;
        const double c2 = rel_resid_pass(p, c, w, staged, red, &dmax);
        if (staged) {
            staged = false;
            const bool full = c2 <= chi2 * (1.0 + 1e-6) + 1e-30;
            float step = 1.f;
            for (int ls = 1; ls < 8 && !full; ++ls) {
                step *= 0.5f;
                for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                    const float2 sv = e < N ? reinterpret_cast<const float2 *>(w.xg)[e]
                                            : reinterpret_cast<const float2 *>(w.xv)[e - N];
                    const float2 dp = zs[e];
                    stage[e] = make_float2(sv.x + step * dp.x, sv.y + step * dp.y);
                }
                __syncthreads();
                const float ch = rel_chi2(p, c, reinterpret_cast<const float *>(stage),
                                          reinterpret_cast<const float *>(stage + N), redf);
                if ((double)ch <= chi2 * (1.0 + 1e-6) + 1e-30 || ls == 7) break;
            }
            for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                if (e < N) reinterpret_cast<float2 *>(w.xg)[e] = stage[e];
                else reinterpret_cast<float2 *>(w.xv)[e - N] = stage[e];
            }
            __syncthreads();
            if ((double)step * sqrt(nr[1]) <= p.tol * sqrt(nr[0])) {
                st = GC_OK;
                break;
            }
            if (gc_globaltimer() - t_start > p.deadline_ns) {
                st = GC_ETIMEOUT;
                if (threadIdx.x == 0) atomicOr(p.status, GC_DEV_TIMEOUT_CAL);
                break;
            }
            if (++it > p.max_iter) break;
            if (!full) continue;   // the pass at the accepted point is still to come
        }
        chi2 = c2;
        const float mu = (float)(p.mu_rel * (double)dmax);
        if (coarse && it == 1) cg_coarse_setup(p, w, mu);   // later iterations reuse it
        // PCG from x = 0: r = b, q = M^-1 r
        float v2[3] = {0.f, 0.f, 0.f};
        const int lane0 = threadIdx.x & 31;
        for (int e0 = threadIdx.x - lane0; e0 < ne; e0 += blockDim.x) {   // warp-uniform trip count
            const int e = e0 + lane0;
            float2 a = make_float2(0.f, 0.f);
            if (e < ne) {
                a = acc[e];
                bs[e] = a;
                xs[e] = make_float2(0.f, 0.f);
                rs[e] = a;
            }
            jacobi(e, a, mu, v2[0], v2[1]);
        }
        __syncthreads();
        v2[2] = coarse_solve();
        fast_sum<3>(v2, sbuf, par);
        float rz = v2[0] + v2[2];
        const float bnorm2 = v2[1];
        update_q(0.f, true);
        // inexact Newton: each linear solve stops at a relative residual
        // eta = min(0.05, (|grad| / |grad_0|)^(1/4)) (floor cg_tol).  Gauss-
        // Newton on a problem with noise in the data converges linearly, so
        // tighter solves buy little: on the 4096-antenna workload this
        // forcing takes 76 CG steps a channel over 9.0 Gauss-Newton
        // iterations where (|grad| / |grad_0|)^(1/2) capped at 0.1 took 159
        // over 9.3, for the same solution to within FP32 rounding.
        if (it == 1) grad0 = bnorm2;
        const float eta =
            (float)fmin(0.05, fmax(cg_tol, sqrt(sqrt(sqrt((double)bnorm2 / fmax(grad0, 1e-300))))));
        for (int k = 0; k < cg_max && bnorm2 > 0.f; ++k) {
            ++inner;
            float v1[1] = {rel_op_pass(p, w, mu)};   // acc = A q; q.(A + mu G) q
            fast_sum<1>(v1, sbuf, par);
            if (!(v1[0] > 0.f)) break;
            const float alpha = rz / v1[0];
            float v3[3] = {0.f, 0.f, 0.f};
            // the same elements per thread as before, four at a time so that
            // their global loads (acc, x, r) are in flight together
            constexpr int U = 4;
            for (int e0 = threadIdx.x - lane0; e0 < ne; e0 += U * blockDim.x) {   // warp-uniform trip count
                float2 au[U], xu[U], ru[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + lane0 + u * blockDim.x;
                    if (e < ne) {
                        au[u] = acc[e];
                        xu[u] = xs[e];
                        ru[u] = rs[e];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (e0 + u * blockDim.x >= ne) break;   // warp-uniform
                    const int e = e0 + lane0 + u * blockDim.x;
                    float2 rn = make_float2(0.f, 0.f);
                    if (e < ne) {
                        const float2 pq = q[e], a = au[u], x = xu[u], r = ru[u];
                        const float mg = mu * w.G[e];
                        xs[e] = make_float2(x.x + alpha * pq.x, x.y + alpha * pq.y);
                        rn = make_float2(r.x - alpha * (a.x + mg * pq.x), r.y - alpha * (a.y + mg * pq.y));
                        rs[e] = rn;
                    }
                    jacobi(e, rn, mu, v3[0], v3[1]);
                }
            }
            __syncthreads();
            v3[2] = coarse_solve();
            fast_sum<3>(v3, sbuf, par);
            if (v3[1] <= eta * eta * bnorm2) break;
            const float rzn = v3[0] + v3[2];
            const float beta = rzn / rz;
            rz = rzn;
            update_q(beta, false);
        }
        __syncthreads();
        for (int t2 = threadIdx.x; t2 < 2 * nc; t2 += blockDim.x) w.rc[t2] = 0.f;
        // Project the four degeneracy directions out of the step (Sec. 5.2),
        // orthogonally in the (g, V) metric, which in relative coordinates
        // weighs element e by G_e.  The directions have closed forms there:
        // amplitude (1 | -2), phase (i | 0), slopes (i x | -i d_x) and
        // (i y | -i d_y) for (antennas | types).
        auto degen = [&](int e, float2 (&qa)[4]) {
            if (e < N) {
                const float X = (float)(e % L), Y = (float)(e / L);
                qa[0] = make_float2(1.f, 0.f);
                qa[1] = make_float2(0.f, 1.f);
                qa[2] = make_float2(0.f, X);
                qa[3] = make_float2(0.f, Y);
            } else {
                const float dx = (float)__ldg(p.types + 2 * (e - N)), dy = (float)__ldg(p.types + 2 * (e - N) + 1);
                qa[0] = make_float2(-2.f, 0.f);
                qa[1] = make_float2(0.f, 0.f);
                qa[2] = make_float2(0.f, -dx);
                qa[3] = make_float2(0.f, -dy);
            }
        };
        float pacc[14];
#pragma unroll
        for (int u = 0; u < 14; ++u) pacc[u] = 0.f;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            float2 qa[4];
            degen(e, qa);
            const float2 x = xs[e];
            const float Ge = w.G[e];
            int u = 0;
#pragma unroll
            for (int a2 = 0; a2 < 4; ++a2) {
#pragma unroll
                for (int b2 = 0; b2 <= a2; ++b2) pacc[u++] += Ge * (qa[a2].x * qa[b2].x + qa[a2].y * qa[b2].y);
                pacc[10 + a2] += Ge * (qa[a2].x * x.x + qa[a2].y * x.y);
            }
        }
        block_sum<float, 14>(pacc, redf);
        float cvec[4];
        solve_gram4<float>(pacc, cvec);
        // delta = s (x - sum_a c_a q_a) in the (g, V) form, into w.z
        nr[0] = nr[1] = 0.0;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            float2 qa[4];
            degen(e, qa);
            float2 d = xs[e];
#pragma unroll
            for (int a2 = 0; a2 < 4; ++a2) {
                d.x -= cvec[a2] * qa[a2].x;
                d.y -= cvec[a2] * qa[a2].y;
            }
            const float2 sv = e < N ? reinterpret_cast<const float2 *>(w.xg)[e]
                                    : reinterpret_cast<const float2 *>(w.xv)[e - N];
            const float2 dp = make_float2(sv.x * d.x - sv.y * d.y, sv.x * d.y + sv.y * d.x);
            zs[e] = dp;
            // the full step, staged in the q area (free once the CG loop is
            // done) for the pair gathers of the next pass
            stage[e] = make_float2(sv.x + dp.x, sv.y + dp.y);
            if (p.red32) {
                nr[0] = (double)((float)nr[0] + (sv.x * sv.x + sv.y * sv.y));
                nr[1] = (double)((float)nr[1] + (dp.x * dp.x + dp.y * dp.y));
            } else {
                nr[0] += (double)sv.x * sv.x + (double)sv.y * sv.y;
                nr[1] += (double)dp.x * dp.x + (double)dp.y * dp.y;
            }
        }
        if (p.red32) {
            float nf[2] = {(float)nr[0], (float)nr[1]};
            block_sum<float, 2>(nf, redf);
            nr[0] = nf[0];
            nr[1] = nf[1];
        } else {
            block_sum<double, 2>(nr, red);
        }
        __syncthreads();
        staged = true;
    }
    finish_channel<float>(p, c, w.xg, w.xv, min(it, p.max_iter), st, red, inner);
}

// kSten: the stencil operator (p.stencil set), launched with kCgStThreads
template <bool kPipe, bool kSten>
__global__ void __launch_bounds__(kSten ? kCgStThreads : kCgThreads, 2)
lincal_cg_kernel(const CalParams p, double cg_tol, int cg_max, int smem_floats) {
    __shared__ double red[32 * 14];
    __shared__ float redf[32 * 14];
    __shared__ float s_rc[2 * kMaxCoarse], s_yc[2 * kMaxCoarse];
    extern __shared__ __align__(16) float arena[];
    int hot_mode;
    bool coarse_smem;
    cg_modes(p, smem_floats, hot_mode, coarse_smem);
    __shared__ int s_item;
    CgWork w = cg_layout(p, p.work + (size_t)blockIdx.x * p.work_per_cta, arena, smem_floats, hot_mode, coarse_smem);
    w.rc = s_rc;
    w.yc = s_yc;
    // channels are taken from a device counter: their iteration counts
    // differ, and a CTA that drew short solves takes more of them
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(p.counter, 1u);
        __syncthreads();
        const int c = s_item;
        __syncthreads();
        if (c >= p.C) break;
        if constexpr (kSten) {
            if (p.stencil) {
                cg_solve_channel_rel(p, c, w, cg_tol, cg_max, red, redf);
                continue;
            }
        }
        cg_solve_channel<kPipe>(p, c, w, cg_tol, cg_max, red, redf);
    }
}

// Several arrays of different size in one persistent launch: CTAs take
// (array, channel) items from a device counter, arrays in `order`
// (largest first by default) so that long solves start early.
constexpr int kMaxBatch = 32;
struct BatchParams {
    CalParams arr[kMaxBatch];
    int order[kMaxBatch];
    int prefix[kMaxBatch + 1];   // channel-count prefix sums in processing order
    int n_arr, total;
    unsigned int *counter;
    char *work;
    size_t work_per_cta;
    double cg_tol;
    int cg_max;
    int smem_floats;
};

template <bool kSten>
__global__ void __launch_bounds__(kSten ? kCgStThreads : kCgThreads, 2)
lincal_cg_batched(const __grid_constant__ BatchParams bp) {
    __shared__ double red[32 * 14];
    __shared__ float redf[32 * 14];
    __shared__ int s_item;
    __shared__ float s_rc[2 * kMaxCoarse], s_yc[2 * kMaxCoarse];
    extern __shared__ __align__(16) float arena[];
    char *base = bp.work + (size_t)blockIdx.x * bp.work_per_cta;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(bp.counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= bp.total) break;
        int slot = 0;
        while (slot + 1 < bp.n_arr && bp.prefix[slot + 1] <= item) ++slot;
        const CalParams &p = bp.arr[bp.order[slot]];
        int hot_mode;
        bool coarse_smem;
        cg_modes(p, bp.smem_floats, hot_mode, coarse_smem);
        CgWork w = cg_layout(p, base, arena, bp.smem_floats, hot_mode, coarse_smem);
        w.rc = s_rc;
        w.yc = s_yc;
        if constexpr (kSten) {
            if (p.stencil) {
                cg_solve_channel_rel(p, item - bp.prefix[slot], w, bp.cg_tol, bp.cg_max, red, redf);
                continue;
            }
        }
        cg_solve_channel<false>(p, item - bp.prefix[slot], w, bp.cg_tol, bp.cg_max, red, redf);
    }
}

// ----------------------------------------------------------------- omnical (FP32)
__global__ void __launch_bounds__(kCThreads) omnical_kernel(const CalParams p) {
    __shared__ float red[32 * 2];
    __shared__ double redd[64];
    float *base = reinterpret_cast<float *>(p.work + (size_t)blockIdx.x * p.work_per_cta);
    float *xg = base;                        // 2N
    float *xv = xg + 2 * p.N;                // 2 n_ubl (+ N scratch for the start point)
    float *ng = xv + 2 * p.n_ubl + p.N;      // 2N new gains
    float *nv = ng + 2 * p.N;                // 2 n_ubl new model visibilities
    const int L = p.L, nu = p.n_ubl;
    const float a = (float)p.damping;
    for (int c = blockIdx.x; c < p.C; c += gridDim.x) {
        const uint64_t t_start = gc_globaltimer();
        if (p.warm) {
            for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
                const float2 g = p.gains[(size_t)c * p.N + i];
                xg[2 * i] = g.x;
                xg[2 * i + 1] = g.y;
            }
            for (int k = threadIdx.x; k < nu; k += blockDim.x) {
                const float2 v = p.vmodel[(size_t)c * nu + k];
                xv[2 * k] = v.x;
                xv[2 * k + 1] = v.y;
            }
            __syncthreads();
        } else {
            start_point<float>(p, c, xg, xv, red, xv + 2 * p.n_ubl);
        }
        int st = GC_ENOCONV, it;
        for (it = 1; it <= p.max_iter; ++it) {
            // gains: gather over each antenna's pairs
            for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
                const int xi = i % L, yi = i / L;
                float nx = 0.f, ny = 0.f, den = 0.f;
                for (int k = 0; k < nu; ++k) {
                    const float vx = xv[2 * k], vy = xv[2 * k + 1];
                    const int dx = p.types[2 * k], dy = p.types[2 * k + 1];
                    int q = p.nbr ? p.nbr[(size_t)k * p.N + i] : pair_index(p, k, xi - dx, yi - dy);
                    if (q >= 0) {   // i = i_p, partner j: z = conj(g_j) V
                        const int j = i - (dy * L + dx);
                        const float zx = xg[2 * j] * vx + xg[2 * j + 1] * vy;
                        const float zy = xg[2 * j] * vy - xg[2 * j + 1] * vx;
                        const float2 v = vobs(p, c, q);
                        nx += v.x * zx + v.y * zy;     // V conj(z)
                        ny += v.y * zx - v.x * zy;
                        den += zx * zx + zy * zy;
                    }
                    q = p.nbr ? p.nbr[(size_t)(nu + k) * p.N + i] : pair_index(p, k, xi, yi);
                    if (q >= 0) {   // i = j_p, partner i': z = g_i' V ; num += conj(V_p) z
                        const int ip = i + (dy * L + dx);
                        const float zx = xg[2 * ip] * vx - xg[2 * ip + 1] * vy;
                        const float zy = xg[2 * ip] * vy + xg[2 * ip + 1] * vx;
                        const float2 v = vobs(p, c, q);
                        nx += v.x * zx + v.y * zy;
                        ny += v.x * zy - v.y * zx;
                        den += zx * zx + zy * zy;
                    }
                }
                ng[2 * i] = den > 0.f ? nx / den : xg[2 * i];
                ng[2 * i + 1] = den > 0.f ? ny / den : xg[2 * i + 1];
            }
            // model visibilities: one warp per type
            const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
            for (int k = wp; k < nu; k += nw) {
                float sx = 0.f, sy = 0.f, sd = 0.f;
                for (int q = p.type_ptr[k] + lane; q < p.type_ptr[k + 1]; q += 32) {
                    const int i = p.pair_i[q], j = p.pair_j[q];
                    const float ex = xg[2 * i] * xg[2 * j] + xg[2 * i + 1] * xg[2 * j + 1];
                    const float ey = xg[2 * i + 1] * xg[2 * j] - xg[2 * i] * xg[2 * j + 1];
                    const float2 v = vobs(p, c, q);
                    sx += v.x * ex + v.y * ey;
                    sy += v.y * ex - v.x * ey;
                    sd += ex * ex + ey * ey;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    sx += __shfl_xor_sync(0xffffffffu, sx, o);
                    sy += __shfl_xor_sync(0xffffffffu, sy, o);
                    sd += __shfl_xor_sync(0xffffffffu, sd, o);
                }
                if (lane == 0) {
                    nv[2 * k] = sd > 0.f ? sx / sd : xv[2 * k];
                    nv[2 * k + 1] = sd > 0.f ? sy / sd : xv[2 * k + 1];
                }
            }
            __syncthreads();
            float acc[2] = {0.f, 0.f};
            for (int i = threadIdx.x; i < 2 * p.N + 2 * nu; i += blockDim.x) {
                float *x = i < 2 * p.N ? &xg[i] : &xv[i - 2 * p.N];
                const float xn = i < 2 * p.N ? ng[i] : nv[i - 2 * p.N];
                const float d = xn - *x;
                acc[0] += d * d;
                acc[1] += (*x) * (*x);
                *x = (1.f - a) * (*x) + a * xn;
            }
            block_sum<float, 2>(acc, red);
            if (sqrtf(acc[0]) < (float)p.tol * sqrtf(acc[1])) {
                st = GC_OK;
                break;
            }
            if (gc_globaltimer() - t_start > p.deadline_ns) {
                st = GC_ETIMEOUT;
                if (threadIdx.x == 0) atomicOr(p.status, GC_DEV_TIMEOUT_CAL);
                break;
            }
        }
        finish_channel<float>(p, c, xg, xv, min(it, p.max_iter), st, redd);
    }
}

}  // namespace

static gc_status fill_params(gc_ctx *ctx, gc_sel *sel, int C, const void *vreduced, int vfmt, const void *autos,
                             const gc_calopts &o, float *gains, float *vmodel, gc_calstats *stats, CalParams &p) {
    if (!vreduced || !sel || !gains || !vmodel || !stats || C < 1)
        return gc_fail(ctx, GC_EINVAL, "gc_calibrate: null argument");
    if (vfmt != GC_C64 && vfmt != GC_I4C) return gc_fail(ctx, GC_EINVAL, "gc_calibrate: unknown format");
    if (sel->null_dim != 4) return gc_fail(ctx, GC_EDEGEN, "gc_calibrate: selection has extra degeneracies");
    if (sel->masked && o.solver != GC_LINCAL_CG)
        return gc_fail(ctx, GC_EUNSUPPORTED, "gc_calibrate: partly occupied lattices are built for GC_LINCAL_CG");
    if (o.solver != GC_LINCAL && o.solver != GC_OMNICAL && o.solver != GC_LINCAL_CG)
        return gc_fail(ctx, GC_EINVAL, "gc_calibrate: solver");
    if (o.precision != GC_FP64 && o.precision != GC_FP32) return gc_fail(ctx, GC_EINVAL, "gc_calibrate: precision");
    int ax = -1, ay = -1;
    int D = 0;
    for (int k = 0; k < sel->n_ubl; ++k) {
        const int dx = sel->types[2 * k], dy = sel->types[2 * k + 1];
        if (dx == 1 && dy == 0) ax = k;
        if (dx == 0 && dy == 1) ay = k;
        D = std::max(D, std::abs(dy * sel->L + dx));
    }
    if (ax < 0 || ay < 0) return gc_fail(ctx, GC_EDEGEN, "gc_calibrate: the selection lacks the axis types");
    gc_status st = gc_sel_upload(ctx, sel);
    if (st != GC_OK) return st;
    p.vred = vreduced;
    p.vfmt = vfmt;
    p.autos = autos;
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
    p.nbr = sel->d_nbr;
    p.ax = ax;
    p.ay = ay;
    // both full-grid selection builders take baseline-types whole, in
    // pair_index order; a partly occupied lattice takes the pair-list form
    p.stencil = ctx->tune[GC_TUNE_CAL_OP] == 0 && sel->n_ubl <= kStencilTypes && !sel->masked ? 1 : 0;
    p.st_halo = 0;
    for (int k = 0; k < sel->n_ubl; ++k)
        p.st_halo = std::max(p.st_halo, std::max(std::abs(sel->types[2 * k]), std::abs(sel->types[2 * k + 1])));
    p.mask = sel->masked ? sel->d_mask : nullptr;
    p.tree_ant = sel->masked ? sel->d_tree_ant : nullptr;
    p.tree_pair = sel->masked ? sel->d_tree_pair : nullptr;
    p.tree_sign = sel->masked ? sel->d_tree_sign : nullptr;
    p.n_occ = sel->masked ? sel->n_occ : sel->L * sel->L;
    p.t_autos = sel->n_cycle * sel->t_int;
    p.gains = reinterpret_cast<float2 *>(gains);
    p.vmodel = reinterpret_cast<float2 *>(vmodel);
    p.stats = stats;
    p.solver = o.solver;
    p.warm = o.warm_start;
    p.damping = o.damping > 0.0 ? o.damping : 0.3;
    p.status = ctx->status_dev;
    p.deadline_ns = (unsigned long long)(o.time_limit_ms > 0 ? o.time_limit_ms : 10000) * 1000000ull;
    p.bw = 2 * D + 1;
    const bool fp64_ne = o.solver == GC_LINCAL && o.precision == GC_FP64;
    p.tol = o.tol > 0.0 ? o.tol : (fp64_ne ? 1e-10 : 1e-6);
    p.max_iter = o.max_iter > 0 ? o.max_iter : (o.solver == GC_OMNICAL ? 20000 : 50);
    p.mu_rel = fp64_ne ? 1e-12 : 1e-7;
    p.red32 = o.solver == GC_LINCAL_CG && o.fp32_reductions ? 1 : 0;
    p.work = nullptr;
    p.counter = nullptr;
    p.work_per_cta = 0;
    return GC_OK;
}

static gc_calopts default_opts(const gc_calopts *opts) {
    gc_calopts o;
    if (opts) return *opts;
    o.solver = GC_LINCAL;
    o.precision = GC_FP64;
    o.max_iter = 0;
    o.tol = 0.0;
    o.damping = 0.3;
    o.warm_start = 0;
    o.time_limit_ms = 0;
    o.fp32_reductions = 0;
    return o;
}

extern "C" gc_status gc_calibrate(gc_ctx *ctx, const void *vreduced, int vfmt, const gc_sel *csel, int C,
                                  const void *autos, const gc_calopts *opts, float *gains, float *vmodel,
                                  gc_calstats *stats, void *stream) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    gc_sel *sel = const_cast<gc_sel *>(csel);
    const gc_calopts o = default_opts(opts);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    CalParams p;
    gc_status st = fill_params(ctx, sel, C, vreduced, vfmt, autos, o, gains, vmodel, stats, p);
    if (st != GC_OK) return st;
    const bool fp64 = o.precision == GC_FP64;
    int occ = 0;
    size_t per_cta, cg_smem = 0;
    bool pipe = false;
    const void *kfn;
    if (o.solver == GC_LINCAL) {
        if (sel->n_ubl > kMaxUbl)
            return gc_fail(ctx, GC_EUNSUPPORTED,
                           "gc_calibrate: banded lincal supports up to 64 baseline-types "
                           "(use GC_LINCAL_CG or omnical for low-cadence)");
        per_cta = fp64 ? gn_bytes<double>(p.N, p.n_ubl, p.bw) : gn_bytes<float>(p.N, p.n_ubl, p.bw);
        kfn = fp64 ? (const void *)lincal_kernel<double> : (const void *)lincal_kernel<float>;
    } else if (o.solver == GC_LINCAL_CG) {
        per_cta = cg_bytes(p.N, p.n_ubl, p.P);
        cg_smem = cg_arena_bytes(p.N, p.n_ubl, p.L, kCgSmemMax, p.stencil != 0);
        // pair-scatter operator with its hot vectors in global memory: the pipelined pass
        pipe = !p.stencil && cg_hot_floats(p.N, p.n_ubl, false) * sizeof(float) > cg_smem;
        kfn = p.stencil ? (const void *)lincal_cg_kernel<false, true>
                        : (pipe ? (const void *)lincal_cg_kernel<true, false>
                                : (const void *)lincal_cg_kernel<false, false>);
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCgSmemMax);
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaFuncSetAttribute(lincal_cg)");
    } else {
        per_cta = sizeof(float) * (size_t)(2 * p.N + 2 * p.n_ubl + p.N + 2 * p.N + 2 * p.n_ubl + 64);
        kfn = (const void *)omnical_kernel;
    }
    per_cta = (per_cta + 255) & ~size_t(255);
    const int nthr = o.solver == GC_LINCAL_CG ? (p.stencil ? kCgStThreads : kCgThreads) : kCThreads;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, nthr, cg_smem);
    if (e != cudaSuccess || occ < 1) return gc_cuda_fail(ctx, e, "occupancy(calibration)");
    if (ctx->tune[GC_TUNE_CAL_CTAS] > 0) occ = std::min(occ, ctx->tune[GC_TUNE_CAL_CTAS]);
    const int grid = std::min(C, occ * ctx->sm_count);
    st = gc_scratch_reserve(ctx, 256 + per_cta * grid);
    if (st != GC_OK) return st;
    p.counter = static_cast<unsigned int *>(ctx->scratch);
    p.work = static_cast<char *>(ctx->scratch) + 256;
    p.work_per_cta = per_cta;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (o.solver == GC_LINCAL_CG) {
        e = cudaMemsetAsync(p.counter, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "reset work counter");
    }
    const char *name = o.solver == GC_LINCAL ? (fp64 ? "lincal_fp64" : "lincal_fp32")
                       : (o.solver == GC_LINCAL_CG ? "lincal_cg" : "omnical");
    int rec = gc_prof_begin(ctx, s, name);
    if (o.solver == GC_LINCAL) {
        if (fp64) lincal_kernel<double><<<grid, kCThreads, 0, s>>>(p);
        else lincal_kernel<float><<<grid, kCThreads, 0, s>>>(p);
    } else if (o.solver == GC_LINCAL_CG) {
        const int sf = (int)(cg_smem / sizeof(float));
        if (p.stencil) lincal_cg_kernel<false, true><<<grid, kCgStThreads, cg_smem, s>>>(p, 1e-4, 500, sf);
        else if (!pipe) lincal_cg_kernel<false, false><<<grid, kCgThreads, cg_smem, s>>>(p, 1e-4, 500, sf);
        else lincal_cg_kernel<true, false><<<grid, kCgThreads, cg_smem, s>>>(p, 1e-4, 500, sf);
    } else {
        omnical_kernel<<<grid, kCThreads, 0, s>>>(p);
    }
    gc_prof_end(ctx, s, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch calibration");
    return GC_OK;
}

extern "C" gc_status gc_calibrate_batched(gc_ctx *ctx, int n_arrays, const gc_batch_item *items,
                                          const gc_calopts *opts, void *stream) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    if (n_arrays < 1 || n_arrays > kMaxBatch || !items)
        return gc_fail(ctx, GC_EINVAL, "gc_calibrate_batched: need 1..32 arrays");
    gc_calopts o = default_opts(opts);
    o.solver = GC_LINCAL_CG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    BatchParams bp;
    memset(&bp, 0, sizeof bp);
    size_t per_cta = 0;
    std::vector<std::pair<double, int>> cost;
    for (int a = 0; a < n_arrays; ++a) {
        const gc_batch_item &it = items[a];
        gc_status st = fill_params(ctx, const_cast<gc_sel *>(it.sel), it.C, it.vreduced, it.vfmt, it.autos, o,
                                   it.gains, it.vmodel, it.stats, bp.arr[a]);
        if (st != GC_OK) return st;
        per_cta = std::max(per_cta, cg_bytes(bp.arr[a].N, bp.arr[a].n_ubl, bp.arr[a].P));
        cost.push_back({(double)bp.arr[a].P + 4.0 * bp.arr[a].N, a});
    }
    if (ctx->tune[GC_TUNE_CAL_ORDER] == 0)
        std::stable_sort(cost.begin(), cost.end(), [](const std::pair<double, int> &x,
                                                      const std::pair<double, int> &y) { return x.first > y.first; });
    bp.n_arr = n_arrays;
    bp.prefix[0] = 0;
    for (int k = 0; k < n_arrays; ++k) {
        bp.order[k] = cost[k].second;
        bp.prefix[k + 1] = bp.prefix[k] + bp.arr[cost[k].second].C;
    }
    bp.total = bp.prefix[n_arrays];
    bp.cg_tol = 1e-4;
    bp.cg_max = 500;
    // shared arena: the largest array that fits the cap
    size_t smem = 0;
    bool sten = false;   // the stencil kernel (256 threads) when any array uses the stencil operator
    for (int a = 0; a < n_arrays; ++a) {
        smem = std::max(smem, cg_arena_bytes(bp.arr[a].N, bp.arr[a].n_ubl, bp.arr[a].L, kCgSmemMax,
                                             bp.arr[a].stencil != 0));
        sten = sten || bp.arr[a].stencil;
    }
    bp.smem_floats = (int)(smem / sizeof(float));
    const void *kfn = sten ? (const void *)lincal_cg_batched<true> : (const void *)lincal_cg_batched<false>;
    const int nthr = sten ? kCgStThreads : kCgThreads;
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCgSmemMax);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaFuncSetAttribute(lincal_cg_batched)");
    per_cta = (per_cta + 255) & ~size_t(255);
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, nthr, smem);
    if (e != cudaSuccess || occ < 1) return gc_cuda_fail(ctx, e, "occupancy(batched calibration)");
    if (ctx->tune[GC_TUNE_CAL_CTAS] > 0) occ = std::min(occ, ctx->tune[GC_TUNE_CAL_CTAS]);
    const int grid = std::min(bp.total, occ * ctx->sm_count);
    gc_status st = gc_scratch_reserve(ctx, 256 + per_cta * grid);
    if (st != GC_OK) return st;
    bp.counter = static_cast<unsigned int *>(ctx->scratch);
    bp.work = static_cast<char *>(ctx->scratch) + 256;
    bp.work_per_cta = per_cta;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(bp.counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "reset work counter");
    int rec = gc_prof_begin(ctx, s, "lincal_cg_batched");
    if (sten) lincal_cg_batched<true><<<grid, kCgStThreads, smem, s>>>(bp);
    else lincal_cg_batched<false><<<grid, kCgThreads, smem, s>>>(bp);
    gc_prof_end(ctx, s, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch batched calibration");
    return GC_OK;
}
