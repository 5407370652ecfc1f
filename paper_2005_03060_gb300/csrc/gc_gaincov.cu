// Predicted calibration variances and covariances (paper Eq. gaincov /
// Eq. noisecov with uniform unit noise; Sec. 5.2 degeneracies left out) and
// the variance of calibrated redundant visibilities (Sec. 6.2).
//
// For every unknown u of the linearised redundant system -- antenna gains
// and model visibilities -- a column of the pseudo-inverse of the normal
// matrices of Eq. logcal,
//   amplitude: (A^T A)^+ e_u,  rows e_i + e_j + e_alpha,
//   phase:     (B^T B)^+ e_u,  rows e_i - e_j + e_alpha.
// Both systems are solved at once in complex form: with s_p = q_i +
// conj(q_j) + w_k the real part of s_p is the amplitude row and the
// imaginary part the phase row, so the operator q -> sum_p (s_p, conj(s_p),
// s_p) on (i, j, k) is A^T A on the real parts and B^T B on the imaginary
// parts (the relative-coordinate Gauss-Newton operator with unit weights).
//
// One CTA per column: Jacobi-preconditioned CG on the right-hand side
// projected off the exact null space (amplitude: 1 on antennas, -2 on
// types; phase: offset (1, 0), slopes (x, -d_x) and (y, -d_y)), then the
// solution projected the same way (the pseudo-inverse's minimum-norm
// solution).  Three outputs:
//   mode 0  the diagonal entry x_u (gc_gain_variance);
//   mode 1  the whole column, a row of the symmetric pseudo-inverse
//           (covariance rows and matrices, Figs. 7-8);
//   mode 2  the antenna covariance after the degeneracies are fixed against
//           the true gains by least squares over the antennas (the paper's
//           simulations, Sec. 3): P C P with P the projector off the
//           antenna-space directions (amplitude 1; phase 1, x, y); its row
//           r is P [(A^T A)^+ (P e_r)] on the antennas, one solve per row.
// Points of a partly occupied lattice hold no antenna and get 0; a solve that
// does not reach the tolerance within max_iter gives NaN.  FP64 throughout
// (these normal matrices are too ill-conditioned for FP32 CG to reach the
// tolerance on large arrays); the operator scatters over the pair list with
// global atomics, so any selection works.  An analysis tool: its cost grows
// as (columns) x (CG iterations) x (pairs).
//
// The visibility variance takes the mode-2 rows of every antenna (the N x N
// covariance C_a, C_p in the workspace) and, one CTA per lag alpha of the
// full array, forms the per-pair sum of Sec. 6.2 (before Eq. visvar) and the
// full linearised variance of the redundant average (every pair with every
// other of the same lag): see gc_visibility_variance in the header.
#include <algorithm>

#include "gc_sel.h"

namespace {

constexpr int kVThreads = 256;

struct CovParams {
    int N, L, n_ubl, P;
    const int32_t *pair_i, *pair_j, *pair_type, *types, *mask;
    int mode;                     // 0 diagonal, 1 pseudo-inverse rows, 2 rows fixed against the truth
    int n_items;                  // mode 0: unknowns; modes 1, 2: rows
    const int32_t *rows;          // modes 1, 2: [n_items] unknowns (NULL: 0 .. n_items - 1)
    float *out_a, *out_p;         // mode 0: [N + n_ubl]; modes 1, 2: [n_items][row_len]
    int row_len;                  // mode 1: N + n_ubl; mode 2: N
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

__device__ __forceinline__ bool occupied(const CovParams &p, int u) {
    return !p.mask || p.mask[u] != 0;
}

// Null-space directions at unknown u (antenna u < N, type u - N):
// amplitude n_a; phase n_1, n_x, n_y (zero at empty lattice points).
struct NullVec {
    float a, p1, px, py;
};
__device__ __forceinline__ NullVec null_at(const CovParams &p, int u) {
    if (u < p.N) {
        if (!occupied(p, u)) return {0.f, 0.f, 0.f, 0.f};
        return {1.f, 1.f, (float)(u % p.L), (float)(u / p.L)};
    }
    const int k = u - p.N;
    return {-2.f, 0.f, -(float)p.types[2 * k], -(float)p.types[2 * k + 1]};
}

// Inverse of the symmetric 3 x 3 [[g0 g1 g2][g1 g3 g4][g2 g4 g5]] (row-major
// into out[9]; zero when singular).
__device__ void inv3_sym(const double *g, double *out) {
    const double a = g[0], b = g[1], c = g[2], d = g[3], e = g[4], f = g[5];
    const double A = d * f - e * e, B = -(b * f - c * e), Cc = b * e - c * d;
    const double det = a * A + b * B + c * Cc;
    const double id = det != 0.0 ? 1.0 / det : 0.0;
    out[0] = A * id;
    out[1] = B * id;
    out[2] = Cc * id;
    out[3] = B * id;
    out[4] = (a * f - c * c) * id;
    out[5] = -(a * e - b * c) * id;
    out[6] = Cc * id;
    out[7] = -(a * e - c * b) * id;
    out[8] = (a * d - b * b) * id;
}

// Remove the null-space components of v (complex [ne]): amplitude from the
// real parts, the three phase directions (via their 3 x 3 Gram matrix) from
// the imaginary parts.  gram: inverse phase Gram (9) and |n_a|^2 (1), shared.
// antennas_only: the same with the directions restricted to the antennas
// (the least-squares fit of the degeneracies over the antennas); the types'
// entries are left alone.
__device__ void project_null(const CovParams &p, double2 *v, const double *gram, double *buf,
                             bool antennas_only = false) {
    const int ne = antennas_only ? p.N : p.N + p.n_ubl;
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

// Gram data of the null directions over the first ne unknowns: inverse phase
// Gram into gram[0..8], |n_a|^2 into gram[9] (shared).
__device__ void null_gram(const CovParams &p, int ne, double *gram, double *buf) {
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
        inv3_sym(g, gram);
        gram[9] = g[6];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kVThreads) gaincov_kernel(const CovParams p) {
    __shared__ double buf[32];
    __shared__ double gram[10];
    __shared__ double agram[10];
    const int ne = p.N + p.n_ubl;
    double *base = p.work + (size_t)blockIdx.x * p.work_per_cta;
    double2 *x = reinterpret_cast<double2 *>(base);
    double2 *r = x + ne;
    double2 *z = r + ne;
    double2 *q = z + ne;
    double2 *acc = q + ne;
    double *D = reinterpret_cast<double *>(acc + ne);
    // Jacobi diagonal (pair counts: the same for both systems) and the
    // Gram data of the null directions, once per CTA
    for (int u = threadIdx.x; u < ne; u += blockDim.x) D[u] = 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < p.P; e += blockDim.x) {
        atomicAdd(&D[p.pair_i[e]], 1.0);
        atomicAdd(&D[p.pair_j[e]], 1.0);
        atomicAdd(&D[p.N + p.pair_type[e]], 1.0);
    }
    __syncthreads();
    null_gram(p, ne, gram, buf);
    if (p.mode == 2) null_gram(p, p.N, agram, buf);
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        const int u0 = p.mode == 0 ? item : (p.rows ? p.rows[item] : item);
        if (u0 < p.N && !occupied(p, u0)) {
            if (p.mode == 0) {
                if (threadIdx.x == 0) {
                    p.out_a[u0] = 0.f;
                    p.out_p[u0] = 0.f;
                }
            } else {
                for (int u = threadIdx.x; u < p.row_len; u += blockDim.x) {
                    p.out_a[(size_t)item * p.row_len + u] = 0.f;
                    p.out_p[(size_t)item * p.row_len + u] = 0.f;
                }
            }
            continue;
        }
        // b = (1 + i) e_u (mode 2: projected off the antenna-space
        // directions), held in r; x = 0
        for (int u = threadIdx.x; u < ne; u += blockDim.x) {
            x[u] = make_double2(0.0, 0.0);
            r[u] = u == u0 ? make_double2(1.0, 1.0) : make_double2(0.0, 0.0);
        }
        __syncthreads();
        if (p.mode == 2) project_null(p, r, agram, buf, true);
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
        if (p.mode == 2) project_null(p, x, agram, buf, true);
        const float nan = __int_as_float(0x7fc00000);
        if (p.mode == 0) {
            if (threadIdx.x == 0) {
                p.out_a[u0] = conv ? (float)x[u0].x : nan;
                p.out_p[u0] = conv ? (float)x[u0].y : nan;
            }
        } else {
            float *oa = p.out_a + (size_t)item * p.row_len, *op = p.out_p + (size_t)item * p.row_len;
            for (int u = threadIdx.x; u < p.row_len; u += blockDim.x) {
                const bool hole = u < p.N && !occupied(p, u);
                oa[u] = !conv ? nan : hole ? 0.f : (float)x[u].x;
                op[u] = !conv ? nan : hole ? 0.f : (float)x[u].y;
            }
        }
        __syncthreads();
    }
}

// One CTA per lag (dx, dy) of the full (2L-1)^2 plane: the per-pair sum and
// the full linearised variance of the redundant average of the pairs
// (i, j = i + d), both points occupied, from the fixed antenna covariance
// C_a, C_p ([N][N] float, the mode-2 rows of every antenna).
struct LagParams {
    int N, L;
    const int32_t *mask;
    const float *Ca, *Cp;
    double snr_inv2, h;           // SNR_full^-2; sigma_cal^2 / 2
    double *var_pair, *var_exact;
    int32_t *n_pairs;
};

__device__ __forceinline__ bool lag_partner(const LagParams &p, int k, int dx, int dy, int sgn, int *out) {
    const int x = k % p.L + sgn * dx, y = k / p.L + sgn * dy;
    if (x < 0 || x >= p.L || y < 0 || y >= p.L) return false;
    const int j = y * p.L + x;
    if (p.mask && !p.mask[j]) return false;
    *out = j;
    return true;
}

// u_k = [k + d in the array] + [k - d in the array], w_k = the difference
// (k occupied): the pair-count vectors of the lag's amplitude and phase sums
__device__ __forceinline__ void lag_weights(const LagParams &p, int k, int dx, int dy, float *u, float *w) {
    int j;
    const bool occ = !p.mask || p.mask[k];
    const float a = occ && lag_partner(p, k, dx, dy, 1, &j) ? 1.f : 0.f;
    const float b = occ && lag_partner(p, k, dx, dy, -1, &j) ? 1.f : 0.f;
    *u = a + b;
    *w = a - b;
}

__global__ void __launch_bounds__(kVThreads) visvar_lag_kernel(const LagParams p) {
    __shared__ double buf[32];
    const int n = 2 * p.L - 1;
    const int lag = blockIdx.x;
    const int dx = lag % n - (p.L - 1), dy = lag / n - (p.L - 1);
    // per-pair terms
    double pair_sum = 0.0, cnt = 0.0;
    if (dx != 0 || dy != 0) {
        for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
            int j;
            if ((p.mask && !p.mask[i]) || !lag_partner(p, i, dx, dy, 1, &j)) continue;
            const size_t ii = (size_t)i * p.N + i, jj = (size_t)j * p.N + j, ij = (size_t)i * p.N + j;
            pair_sum += p.snr_inv2 + p.h * ((double)p.Ca[ii] + p.Cp[ii] + p.Ca[jj] + p.Cp[jj]) +
                        2.0 * p.h * ((double)p.Ca[ij] - p.Cp[ij]);
            cnt += 1.0;
        }
    }
    pair_sum = block_sum_d(pair_sum, buf);
    cnt = block_sum_d(cnt, buf);
    // quadratic forms u^T C_a u + w^T C_p w: one warp per row k
    double quad = 0.0;
    if (cnt > 0.0) {
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int k = wp; k < p.N; k += nw) {
            float uk, wk;
            lag_weights(p, k, dx, dy, &uk, &wk);
            if (uk == 0.f && wk == 0.f) continue;
            double ra = 0.0, rp = 0.0;
            for (int k2 = lane; k2 < p.N; k2 += 32) {
                float u2, w2;
                lag_weights(p, k2, dx, dy, &u2, &w2);
                ra += (double)p.Ca[(size_t)k * p.N + k2] * u2;
                rp += (double)p.Cp[(size_t)k * p.N + k2] * w2;
            }
            quad += uk * ra + wk * rp;
        }
    }
    quad = block_sum_d(quad, buf);
    if (threadIdx.x == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        const double na = cnt;
        if (p.n_pairs) p.n_pairs[lag] = (int32_t)na;
        p.var_pair[lag] = na > 0.0 ? pair_sum / (na * na) : nan;
        if (p.var_exact) p.var_exact[lag] = na > 0.0 ? (na * p.snr_inv2 + p.h * quad) / (na * na) : nan;
    }
}

gc_status cov_setup(gc_ctx *ctx, gc_sel *sel, CovParams *p) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    gc_status st = gc_sel_upload(ctx, sel);
    if (st != GC_OK) return st;
    p->L = sel->L;
    p->N = sel->L * sel->L;
    p->n_ubl = sel->n_ubl;
    p->P = sel->P;
    p->pair_i = sel->d_pair_i;
    p->pair_j = sel->d_pair_j;
    p->pair_type = sel->d_pair_type;
    p->types = sel->d_types;
    p->mask = sel->masked ? sel->d_mask : nullptr;
    p->n_occ = sel->masked ? sel->n_occ : p->N;
    p->max_iter = 4000;
    p->tol = 1e-8f;
    p->rows = nullptr;
    p->work_per_cta = ((size_t)11 * (p->N + p->n_ubl) + 63) & ~size_t(63);
    return GC_OK;
}

int cov_grid(const gc_ctx *ctx, int n_items) { return std::max(1, std::min(n_items, 4 * ctx->sm_count)); }

}  // namespace

extern "C" gc_status gc_gain_variance(gc_ctx *ctx, const gc_sel *csel, float *var_amp, float *var_phase,
                                      void *stream) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    gc_sel *sel = const_cast<gc_sel *>(csel);
    if (!sel || !var_amp || !var_phase) return gc_fail(ctx, GC_EINVAL, "gc_gain_variance: null argument");
    if (sel->null_dim != 4) return gc_fail(ctx, GC_EDEGEN, "gc_gain_variance: selection has extra degeneracies");
    CovParams p;
    gc_status st = cov_setup(ctx, sel, &p);
    if (st != GC_OK) return st;
    p.mode = 0;
    p.n_items = p.N + p.n_ubl;
    p.out_a = var_amp;
    p.out_p = var_phase;
    p.row_len = 0;
    const int grid = cov_grid(ctx, p.n_items);
    st = gc_scratch_reserve(ctx, sizeof(double) * p.work_per_cta * grid);
    if (st != GC_OK) return st;
    p.work = static_cast<double *>(ctx->scratch);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rec = gc_prof_begin(ctx, s, "gaincov");
    gaincov_kernel<<<grid, kVThreads, 0, s>>>(p);
    gc_prof_end(ctx, s, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch gaincov");
    return GC_OK;
}

extern "C" gc_status gc_gain_covariance(gc_ctx *ctx, const gc_sel *csel, int fixed, int n_rows,
                                        const int32_t *rows, float *cov_amp, float *cov_phase, void *stream) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    gc_sel *sel = const_cast<gc_sel *>(csel);
    if (!sel || !rows || !cov_amp || !cov_phase || n_rows < 0 || (fixed != 0 && fixed != 1))
        return gc_fail(ctx, GC_EINVAL, "gc_gain_covariance: bad argument");
    if (sel->null_dim != 4) return gc_fail(ctx, GC_EDEGEN, "gc_gain_covariance: selection has extra degeneracies");
    const int N = sel->L * sel->L, lim = fixed ? N : N + sel->n_ubl;
    for (int k = 0; k < n_rows; ++k)
        if (rows[k] < 0 || rows[k] >= lim) return gc_fail(ctx, GC_EINVAL, "gc_gain_covariance: row out of range");
    if (n_rows == 0) return GC_OK;
    CovParams p;
    gc_status st = cov_setup(ctx, sel, &p);
    if (st != GC_OK) return st;
    p.mode = fixed ? 2 : 1;
    p.n_items = n_rows;
    p.out_a = cov_amp;
    p.out_p = cov_phase;
    p.row_len = lim;
    const int grid = cov_grid(ctx, n_rows);
    const size_t work_bytes = sizeof(double) * p.work_per_cta * grid;
    st = gc_scratch_reserve(ctx, work_bytes + sizeof(int32_t) * (size_t)n_rows);
    if (st != GC_OK) return st;
    p.work = static_cast<double *>(ctx->scratch);
    int32_t *d_rows = reinterpret_cast<int32_t *>(static_cast<char *>(ctx->scratch) + work_bytes);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the row list is small and read by the kernel once per row: a
    // synchronous copy keeps the caller's host array free on return
    cudaError_t e = cudaMemcpyAsync(d_rows, rows, sizeof(int32_t) * (size_t)n_rows, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "gc_gain_covariance: row list copy");
    p.rows = d_rows;
    int rec = gc_prof_begin(ctx, s, "gaincov_rows");
    gaincov_kernel<<<grid, kVThreads, 0, s>>>(p);
    gc_prof_end(ctx, s, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch gaincov rows");
    return GC_OK;
}

extern "C" gc_status gc_visibility_variance(gc_ctx *ctx, const gc_sel *csel, double snr_full_inv2,
                                            double sigma_cal2, double *var_pair, double *var_exact,
                                            int32_t *n_pairs, void *stream) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    gc_sel *sel = const_cast<gc_sel *>(csel);
    if (!sel || !var_pair || !(snr_full_inv2 >= 0.0) || !(sigma_cal2 >= 0.0))
        return gc_fail(ctx, GC_EINVAL, "gc_visibility_variance: bad argument");
    if (sel->null_dim != 4)
        return gc_fail(ctx, GC_EDEGEN, "gc_visibility_variance: selection has extra degeneracies");
    CovParams p;
    gc_status st = cov_setup(ctx, sel, &p);
    if (st != GC_OK) return st;
    const int N = p.N;
    p.mode = 2;
    p.n_items = N;
    p.row_len = N;
    const int grid = cov_grid(ctx, N);
    const size_t work_bytes = sizeof(double) * p.work_per_cta * grid;
    const size_t cov_bytes = sizeof(float) * (size_t)N * N;
    st = gc_scratch_reserve(ctx, work_bytes + 2 * cov_bytes);
    if (st != GC_OK) return st;
    char *base = static_cast<char *>(ctx->scratch);
    p.work = reinterpret_cast<double *>(base);
    p.out_a = reinterpret_cast<float *>(base + work_bytes);
    p.out_p = reinterpret_cast<float *>(base + work_bytes + cov_bytes);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rec = gc_prof_begin(ctx, s, "gaincov_rows");
    gaincov_kernel<<<grid, kVThreads, 0, s>>>(p);
    gc_prof_end(ctx, s, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch gaincov rows");
    LagParams lp;
    lp.N = N;
    lp.L = sel->L;
    lp.mask = p.mask;
    lp.Ca = p.out_a;
    lp.Cp = p.out_p;
    lp.snr_inv2 = snr_full_inv2;
    lp.h = 0.5 * sigma_cal2;
    lp.var_pair = var_pair;
    lp.var_exact = var_exact;
    lp.n_pairs = n_pairs;
    const int n = 2 * sel->L - 1;
    rec = gc_prof_begin(ctx, s, "visvar_lag");
    visvar_lag_kernel<<<n * n, kVThreads, 0, s>>>(lp);
    gc_prof_end(ctx, s, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch visvar_lag");
    return GC_OK;
}
