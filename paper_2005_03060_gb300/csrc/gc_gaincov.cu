// Predicted calibration variances (paper Eq. gaincov / Eq. noisecov with
// uniform unit noise; Sec. 5.2 degeneracies left out): for every unknown u
// of the linearised redundant system -- antenna gains and model
// visibilities -- the diagonal entry of the pseudo-inverse of the normal
// matrix of Eq. logcal,
//   amplitude: [(A^T A)^+]_uu,  rows e_i + e_j + e_alpha,
//   phase:     [(B^T B)^+]_uu,  rows e_i - e_j + e_alpha.
// Both systems are solved at once in complex form: with s_p = q_i +
// conj(q_j) + w_k the real part of s_p is the amplitude row and the
// imaginary part the phase row, so the operator q -> sum_p (s_p, conj(s_p),
// s_p) on (i, j, k) is A^T A on the real parts and B^T B on the imaginary
// parts (the relative-coordinate Gauss-Newton operator with unit weights).
//
// One CTA per unknown: Jacobi-preconditioned CG on the right-hand side
// (1 + i) e_u projected off the exact null space (amplitude: 1 on antennas,
// -2 on types; phase: offset (1, 0), slopes (x, -d_x) and (y, -d_y)), then
// the solution projected the same way (the pseudo-inverse's minimum-norm
// solution); var_amp[u] = Re x_u, var_phase[u] = Im x_u.  Points of a
// partly occupied lattice hold no antenna and get 0; an unknown whose solve
// does not reach the tolerance within max_iter gets NaN.  FP64 throughout
// (these normal matrices are too ill-conditioned for FP32 CG to reach the
// tolerance on large arrays); the operator scatters over the pair list with
// global atomics, so any selection works.  An analysis tool: its cost grows
// as (unknowns) x (CG iterations) x (pairs).
#include <algorithm>

#include "gc_sel.h"

namespace {

constexpr int kVThreads = 256;

struct CovParams {
    int N, L, n_ubl, P;
    const int32_t *pair_i, *pair_j, *pair_type, *types, *mask;
    float *var_amp, *var_phase;   // [N + n_ubl]
    double *work;                 // per CTA: 5 vectors of 2 (N + n_ubl) doubles + D (N + n_ubl)
    size_t work_per_cta;          // doubles
    int max_iter;
    float tol;
    int n_occ;
};

__device__ __forceinline__ double block_sum_d(double v, double *buf) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) buf[wp] = v;
    __syncthreads();
    double s = 0.0;
    for (int u = 0; u < nw; ++u) s += buf[u];
    return s;
}

// Null-space directions at unknown u (antenna u < N, type u - N):
// amplitude n_a; phase n_1, n_x, n_y (zero at empty lattice points).
struct NullVec {
    float a, p1, px, py;
};
__device__ __forceinline__ NullVec null_at(const CovParams &p, int u) {
    if (u < p.N) {
        if (p.mask && !p.mask[u]) return {0.f, 0.f, 0.f, 0.f};
        return {1.f, 1.f, (float)(u % p.L), (float)(u / p.L)};
    }
    const int k = u - p.N;
    return {-2.f, 0.f, -(float)p.types[2 * k], -(float)p.types[2 * k + 1]};
}

// Remove the null-space components of v (complex [ne]): amplitude from the
// real parts, the three phase directions (via their 3 x 3 Gram matrix) from
// the imaginary parts.  gram: inverse phase Gram (9) and |n_a|^2 (1), shared.
__device__ void project_null(const CovParams &p, double2 *v, const double *gram, double *buf) {
    const int ne = p.N + p.n_ubl;
    double ca = 0.0, c1 = 0.0, cx = 0.0, cy = 0.0;
    for (int u = threadIdx.x; u < ne; u += blockDim.x) {
        const NullVec n = null_at(p, u);
        ca += (double)n.a * v[u].x;
        c1 += (double)n.p1 * v[u].y;
        cx += (double)n.px * v[u].y;
        cy += (double)n.py * v[u].y;
    }
    ca = block_sum_d(ca, buf);
    c1 = block_sum_d(c1, buf);
    cx = block_sum_d(cx, buf);
    cy = block_sum_d(cy, buf);
    const double sa = ca / gram[9];
    const double s1 = gram[0] * c1 + gram[1] * cx + gram[2] * cy;
    const double sx = gram[3] * c1 + gram[4] * cx + gram[5] * cy;
    const double sy = gram[6] * c1 + gram[7] * cx + gram[8] * cy;
    for (int u = threadIdx.x; u < ne; u += blockDim.x) {
        const NullVec n = null_at(p, u);
        v[u].x -= sa * n.a;
        v[u].y -= s1 * n.p1 + sx * n.px + sy * n.py;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kVThreads) gaincov_kernel(const CovParams p) {
    __shared__ double buf[32];
    __shared__ double gram[10];
    const int ne = p.N + p.n_ubl;
    double *base = p.work + (size_t)blockIdx.x * p.work_per_cta;
    double2 *x = reinterpret_cast<double2 *>(base);
    double2 *r = x + ne;
    double2 *z = r + ne;
    double2 *q = z + ne;
    double2 *acc = q + ne;
    double *D = reinterpret_cast<double *>(acc + ne);
    // Jacobi diagonal (pair counts: the same for both systems) and the
    // phase Gram matrix of the null directions, once per CTA
    for (int u = threadIdx.x; u < ne; u += blockDim.x) D[u] = 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < p.P; e += blockDim.x) {
        atomicAdd(&D[p.pair_i[e]], 1.0);
        atomicAdd(&D[p.pair_j[e]], 1.0);
        atomicAdd(&D[p.N + p.pair_type[e]], 1.0);
    }
    __syncthreads();
    {
        double g[7] = {0, 0, 0, 0, 0, 0, 0};   // n1.n1 n1.nx n1.ny nx.nx nx.ny ny.ny na.na
        for (int u = threadIdx.x; u < ne; u += blockDim.x) {
            const NullVec n = null_at(p, u);
            g[0] += n.p1 * n.p1;
            g[1] += n.p1 * n.px;
            g[2] += n.p1 * n.py;
            g[3] += n.px * n.px;
            g[4] += n.px * n.py;
            g[5] += n.py * n.py;
            g[6] += n.a * n.a;
        }
        for (int k = 0; k < 7; ++k) g[k] = block_sum_d(g[k], buf);
        if (threadIdx.x == 0) {
            // inverse of the symmetric 3 x 3 [[g0 g1 g2][g1 g3 g4][g2 g4 g5]]
            const double a = g[0], b = g[1], c = g[2], d = g[3], e = g[4], f = g[5];
            const double A = d * f - e * e, B = -(b * f - c * e), Cc = b * e - c * d;
            const double det = a * A + b * B + c * Cc;
            const double id = det != 0.0 ? 1.0 / det : 0.0;
            gram[0] = A * id;
            gram[1] = B * id;
            gram[2] = Cc * id;
            gram[3] = B * id;
            gram[4] = (a * f - c * c) * id;
            gram[5] = -(a * e - b * c) * id;
            gram[6] = Cc * id;
            gram[7] = -(a * e - c * b) * id;
            gram[8] = (a * d - b * b) * id;
            gram[9] = g[6];
        }
        __syncthreads();
    }
    for (int u0 = blockIdx.x; u0 < ne; u0 += gridDim.x) {
        if (u0 < p.N && p.mask && !p.mask[u0]) {
            if (threadIdx.x == 0) {
                p.var_amp[u0] = 0.f;
                p.var_phase[u0] = 0.f;
            }
            continue;
        }
        // b = P (1 + i) e_u, held in r; x = 0
        for (int u = threadIdx.x; u < ne; u += blockDim.x) {
            x[u] = make_double2(0.0, 0.0);
            r[u] = u == u0 ? make_double2(1.0, 1.0) : make_double2(0.0, 0.0);
        }
        __syncthreads();
        project_null(p, r, gram, buf);
        double bb = 0.0, rz = 0.0;
        for (int u = threadIdx.x; u < ne; u += blockDim.x) {
            const double iv = D[u] > 0.0 ? 1.0 / D[u] : 0.0;
            const double2 rr = r[u];
            z[u] = make_double2(rr.x * iv, rr.y * iv);
            q[u] = z[u];
            bb += rr.x * rr.x + rr.y * rr.y;
            rz += rr.x * z[u].x + rr.y * z[u].y;
        }
        bb = block_sum_d(bb, buf);
        rz = block_sum_d(rz, buf);
        bool conv = !(rz > 0.0);
        for (int it = 0; it < p.max_iter && !conv; ++it) {
            // acc = (A^T A (+) B^T B) q by a scatter over the pairs
            for (int u = threadIdx.x; u < ne; u += blockDim.x) acc[u] = make_double2(0.0, 0.0);
            __syncthreads();
            for (int e = threadIdx.x; e < p.P; e += blockDim.x) {
                const int i = p.pair_i[e], j = p.pair_j[e], k = p.N + p.pair_type[e];
                const double2 qi = q[i], qj = q[j], qk = q[k];
                const double sx = qi.x + qj.x + qk.x, sy = qi.y - qj.y + qk.y;
                atomicAdd(&acc[i].x, sx);
                atomicAdd(&acc[i].y, sy);
                atomicAdd(&acc[j].x, sx);
                atomicAdd(&acc[j].y, -sy);
                atomicAdd(&acc[k].x, sx);
                atomicAdd(&acc[k].y, sy);
            }
            __syncthreads();
            double qa = 0.0;
            for (int u = threadIdx.x; u < ne; u += blockDim.x) qa += q[u].x * acc[u].x + q[u].y * acc[u].y;
            qa = block_sum_d(qa, buf);
            if (!(qa > 0.0)) break;
            const double alpha = rz / qa;
            double rn = 0.0, rzn = 0.0;
            for (int u = threadIdx.x; u < ne; u += blockDim.x) {
                x[u].x += alpha * q[u].x;
                x[u].y += alpha * q[u].y;
                r[u].x -= alpha * acc[u].x;
                r[u].y -= alpha * acc[u].y;
                const double iv = D[u] > 0.0 ? 1.0 / D[u] : 0.0;
                z[u] = make_double2(r[u].x * iv, r[u].y * iv);
                rn += r[u].x * r[u].x + r[u].y * r[u].y;
                rzn += r[u].x * z[u].x + r[u].y * z[u].y;
            }
            rn = block_sum_d(rn, buf);
            rzn = block_sum_d(rzn, buf);
            if (rn <= (double)p.tol * p.tol * bb) {
                conv = true;
                break;
            }
            const double beta = rzn / rz;
            rz = rzn;
            for (int u = threadIdx.x; u < ne; u += blockDim.x) {
                q[u].x = z[u].x + beta * q[u].x;
                q[u].y = z[u].y + beta * q[u].y;
            }
            __syncthreads();
        }
        project_null(p, x, gram, buf);
        if (threadIdx.x == 0) {
            p.var_amp[u0] = conv ? (float)x[u0].x : __int_as_float(0x7fc00000);
            p.var_phase[u0] = conv ? (float)x[u0].y : __int_as_float(0x7fc00000);
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" gc_status gc_gain_variance(gc_ctx *ctx, const gc_sel *csel, float *var_amp, float *var_phase,
                                      void *stream) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    gc_sel *sel = const_cast<gc_sel *>(csel);
    if (!sel || !var_amp || !var_phase) return gc_fail(ctx, GC_EINVAL, "gc_gain_variance: null argument");
    if (sel->null_dim != 4) return gc_fail(ctx, GC_EDEGEN, "gc_gain_variance: selection has extra degeneracies");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    gc_status st = gc_sel_upload(ctx, sel);
    if (st != GC_OK) return st;
    CovParams p;
    p.L = sel->L;
    p.N = sel->L * sel->L;
    p.n_ubl = sel->n_ubl;
    p.P = sel->P;
    p.pair_i = sel->d_pair_i;
    p.pair_j = sel->d_pair_j;
    p.pair_type = sel->d_pair_type;
    p.types = sel->d_types;
    p.mask = sel->masked ? sel->d_mask : nullptr;
    p.n_occ = sel->masked ? sel->n_occ : p.N;
    p.var_amp = var_amp;
    p.var_phase = var_phase;
    p.max_iter = 4000;
    p.tol = 1e-8f;
    const int ne = p.N + p.n_ubl;
    p.work_per_cta = ((size_t)11 * ne + 63) & ~size_t(63);
    const int grid = std::min(ne, 4 * ctx->sm_count);
    st = gc_scratch_reserve(ctx, sizeof(double) * p.work_per_cta * grid);
    if (st != GC_OK) return st;
    p.work = static_cast<double *>(ctx->scratch);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rec = gc_prof_begin(ctx, s, "gaincov");
    gaincov_kernel<<<grid, kVThreads, 0, s>>>(p);
    gc_prof_end(ctx, s, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch gaincov");
    return GC_OK;
}
