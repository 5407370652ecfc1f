// FFT-correlator: calibrate voltages, zero-padded 2-D spatial FFT per time
// sample, |X(k)|^2 integrated over time, inverse FFT to the unique-baseline
// visibilities (paper Fig. 1b yellow box, Sec. 1 convolution theorem,
// Eq. modelvis).
//
// Kernel 1 (fftcorr_accumulate) streams voltages through shared memory with
// TMA and keeps the power spectrum of one time chunk in registers.  One
// work item = (channel c, k_x residue class q mod R, time chunk).  Per time
// sample:
//   row pass    : for every grid row y < L and residue s, fold the row with
//                 the twiddles of k = q + R s and run an F1-point FFT in
//                 registers -> X1[y][k_x] for k_x = k + R S1 m;
//   column pass : for every owned k_x and residue s2 of k_y, fold the column
//                 and run an F2-point FFT -> X(k_y, k_x); P += |X|^2.
// The zero padding to M x M is never materialised: the first FFT stages of
// both passes see only the L non-zero inputs (folds over L <= M/2 inputs).
//
// Kernel 2 (fftcorr_finalize) sums the chunk spectra (FP64), inverse-DFTs
// the (2L-1)^2 lags that exist, and divides by T N_d.  For M = 256 the
// spectrum no longer fits one CTA's shared memory and the inverse DFT runs as
// two passes (fftcorr_finalize_rows / fftcorr_finalize_cols) through global
// memory.
//
// Voltage formats: complex64 (8 B), binary16 pairs (4 B; the FP16-storage
// variant, FP32 arithmetic) and 4+4-bit integers (1 B).
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "gc_fft_reg.h"
#include "gc_internal.h"

namespace {

// ----------------------------------------------------------------- config
template <int M_, int R_, int F1_, int F2_, int NT_, int G_, int VF_, int MINB_ = 1>
struct Cfg {
    static constexpr int M = M_, R = R_, F1 = F1_, F2 = F2_, NT = NT_, G = G_, VF = VF_;
    static constexpr int MINB = MINB_;                  // resident CTAs per SM the registers must allow
    static constexpr int LMAX = M / 2;
    static constexpr int MX = M / R;                    // k_x values per work item
    static constexpr int S1 = MX / F1;                  // row residues
    static constexpr int J1 = (LMAX + F1 - 1) / F1;     // row folds
    static constexpr int S2 = M / F2;                   // column residues
    static constexpr int J2 = (LMAX + F2 - 1) / F2;     // column folds
    static constexpr int NCOL = MX * S2;                // column items per group
    static constexpr int NTHREADS = G * NCOL;
    static constexpr int GNT = G * NT;                  // samples per iteration
    static constexpr int ESZ = VF == GC_C64 ? 8 : (VF == GC_C32H ? 4 : 1);   // bytes per antenna-sample
    // padded stage row (bytes): the smallest odd number of 16-byte units
    // holding LMAX elements, so rows read by consecutive lanes hit distinct banks
    static constexpr int ROWU = (LMAX * ESZ + 15) / 16;
    static constexpr int ROWB = 16 * (ROWU % 2 == 1 ? ROWU : ROWU + 1);
    static constexpr int ROWE = ROWB / ESZ;             // elements per stage row
    static constexpr int CROW = LMAX + 2;               // coefficient row (float2)
    static constexpr int IROW = MX + 1;                 // intermediate row (float2)
    static constexpr int STAGE_BYTES = GNT * LMAX * ROWB;
    static constexpr int NSTAGE = 2;
    // shared memory layout (bytes)
    static constexpr int OFF_BAR = 0;
    static constexpr int OFF_TW = 128;
    static constexpr int OFF_COEF = OFF_TW + ((M * 8 + 127) / 128) * 128;
    static constexpr int OFF_STAGE = OFF_COEF + ((LMAX * CROW * 8 + 127) / 128) * 128;
    static constexpr int OFF_INTER = OFF_STAGE + NSTAGE * ((STAGE_BYTES + 127) / 128) * 128;
    static constexpr int SMEM = OFF_INTER + GNT * LMAX * IROW * 8;
    static_assert(MX % F1 == 0 && M % F2 == 0, "bad FFT split");
    static_assert(ROWB % 16 == 0 && (ROWB / 16) % 2 == 1, "stage row must be an odd number of 16B");
    static_assert(F1 % 4 == 0 && (VF != GC_I4C || F1 % 16 == 0 || LMAX <= 16), "row reads");
    static_assert((G - 1) * NCOL * F2 * 4 <= GNT * LMAX * IROW * 8, "group partial spectra must fit the intermediate");
};

struct Params {
    const void *volt;        // [C][T][L*L]
    const float2 *gains;     // [C][L*L]
    float *ppart;            // [C][n_chunks][M][M]
    unsigned int *status;
    int L, C, T;
    int chunk_len;           // multiple of G*NT
    int n_chunks;
    int n_items;             // C * R * n_chunks
    const unsigned char *mask = nullptr;   // [L*L] occupied lattice points, or null (all)
};

// Copy the G*NT samples starting at t into stage (plain-load fallback for
// strides that TMA cannot describe).  Rows/columns beyond L and samples
// beyond T are zero.
template <class K>
__device__ void stage_plain(const Params &p, unsigned char *stage, int c, int t) {
    const int L = p.L, N = L * L;
    const int total = K::GNT * K::LMAX * K::ROWE;
    for (int idx = threadIdx.x; idx < total; idx += K::NTHREADS) {
        const int x = idx % K::ROWE;
        const int rest = idx / K::ROWE;
        const int y = rest % K::LMAX;
        const int u = rest / K::LMAX;
        const int tt = t + u;
        const bool ok = x < L && y < L && tt < p.T;
        const size_t src = ((size_t)c * p.T + (ok ? tt : 0)) * N + (ok ? y * L + x : 0);
        if (K::VF == GC_C64) {
            float2 v = make_float2(0.f, 0.f);
            if (ok) v = reinterpret_cast<const float2 *>(p.volt)[src];
            reinterpret_cast<float2 *>(stage)[(u * K::LMAX + y) * K::ROWE + x] = v;
        } else if (K::VF == GC_C32H) {
            unsigned int v = 0u;
            if (ok) v = reinterpret_cast<const unsigned int *>(p.volt)[src];
            reinterpret_cast<unsigned int *>(stage)[(u * K::LMAX + y) * K::ROWE + x] = v;
        } else {
            unsigned char v = 0;
            if (ok) v = reinterpret_cast<const unsigned char *>(p.volt)[src];
            stage[(u * K::LMAX + y) * K::ROWB + x] = v;
        }
    }
}

__device__ __forceinline__ float2 h2_to_f2(unsigned int bits) {
    __half2 h;
    *reinterpret_cast<unsigned int *>(&h) = bits;
    return __half22float2(h);
}

// One row input into the fold: b += v c omega_M^{k x}.  With one row residue
// per item (S1 == 1) the coefficient already carries the twiddle.
template <class K>
__device__ __forceinline__ void row_in(float2 &b, float2 v, float2 c, const float2 *tws, int k, int x) {
    if constexpr (K::S1 == 1) b = cfma(b, v, c);
    else b = cfma(b, cmul(v, c), tws[(k * x) & (K::M - 1)]);
}

// multiply by (-i)^R
template <int R>
__device__ __forceinline__ float2 rot_mi(float2 a) {
    if (R == 0) return a;
    if (R == 1) return make_float2(a.y, -a.x);
    if (R == 2) return make_float2(-a.x, -a.y);
    return make_float2(-a.y, a.x);
}

// Column fold for two folds (J2 == 2) and four column residues (M = 4 F2):
// omega_M^{s2 (y + F2)} = omega_M^{s2 y} (-i)^{s2}, so the two inputs combine
// with a trivial rotation before one twiddle multiply (none for s2 = 0).
template <class K, int S2V>
__device__ __forceinline__ void col_fold2(float2 (&b)[K::F2], const float2 *icol, const float2 *tws) {
#pragma unroll
    for (int yp = 0; yp < K::F2; ++yp) {
        const float2 a0 = icol[yp * K::IROW], a1 = icol[(yp + K::F2) * K::IROW];
        float2 t;
        if constexpr (S2V == 0) t = add2(a0, a1);
        else if constexpr (S2V == 2) t = sub2(a0, a1);
        else {
            const float2 r = rot_mi<S2V>(a1);
            t = make_float2(a0.x + r.x, a0.y + r.y);
        }
        b[yp] = S2V == 0 ? t : cmul(t, tws[(S2V * yp) & (K::M - 1)]);
    }
}

template <class K, bool kTMA>
__global__ void __launch_bounds__(K::NTHREADS, K::MINB)
fftcorr_accumulate(const __grid_constant__ CUtensorMap tmap, const Params p) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + K::OFF_BAR);
    float2 *tws = reinterpret_cast<float2 *>(smem + K::OFF_TW);
    float2 *coef = reinterpret_cast<float2 *>(smem + K::OFF_COEF);
    unsigned char *stage0 = smem + K::OFF_STAGE;
    float2 *inter = reinterpret_cast<float2 *>(smem + K::OFF_INTER);
    __shared__ int s_err;

    const int tid = threadIdx.x;
    const int L = p.L;
    constexpr int kStageStride = ((K::STAGE_BYTES + 127) / 128) * 128;

    // one-time set-up: twiddles omega_M^e, zero pads and unused rows
    for (int e = tid; e < K::M; e += K::NTHREADS) {
        const cf w = c_tw.v[e * (256 / K::M)];
        tws[e] = make_float2(w.x, w.y);
    }
    for (int i = tid; i < K::GNT * K::LMAX * K::IROW; i += K::NTHREADS) inter[i] = make_float2(0.f, 0.f);
    if (tid == 0) {
        s_err = 0;
        if (kTMA) {
            gc_mbar_init(&bars[0], 1);
            gc_mbar_init(&bars[1], 1);
            gc_fence_mbar_init();
        }
    }
    __syncthreads();

    // column item owned by this thread (fixed for the whole kernel)
    const int g = tid / K::NCOL;
    const int col = tid % K::NCOL;
    const int kxl = col % K::MX;
    const int s2 = col / K::MX;
    const int n_it = p.chunk_len / K::GNT;
    const int rows_per_it = K::GNT * L * K::S1;
    uint32_t ld_count = 0, use_count = 0;   // TMA loads issued / consumed (phase tracking)

    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        const int q = item % K::R;
        const int chunk = (item / K::R) % p.n_chunks;
        const int c = item / (K::R * p.n_chunks);
        const int t0 = chunk * p.chunk_len;

        // calibration coefficients 1/g_i = conj(g)/|g|^2 in the padded layout
        for (int i = tid; i < K::LMAX * K::CROW; i += K::NTHREADS) {
            const int x = i % K::CROW, y = i / K::CROW;
            float2 cc = make_float2(0.f, 0.f);
            if (x < L && y < L && (!p.mask || p.mask[y * L + x])) {
                const float2 gg = p.gains[(size_t)c * L * L + y * L + x];
                const float d = gg.x * gg.x + gg.y * gg.y;
                if (d > 0.f && isfinite(d)) {
                    cc = make_float2(gg.x / d, -gg.y / d);
                } else {
                    // w = v / g is undefined: report it and leave the antenna out
                    atomicOr(p.status, GC_DEV_BADINPUT);
                }
                // one row residue (k = q for the whole item): the row twiddle
                // omega_M^{k x} rides on the coefficient
                if (K::S1 == 1) cc = cmul(cc, tws[(q * x) & (K::M - 1)]);
            }
            coef[i] = cc;
        }
        if (kTMA && tid == 0) {
            for (int k = 0; k < 2 && k < n_it; ++k) {
                unsigned char *dst = stage0 + (ld_count & 1u) * kStageStride;
                gc_mbar_expect_tx(&bars[ld_count & 1u], K::STAGE_BYTES);
                gc_tma_load_4d(dst, &tmap, &bars[ld_count & 1u], 0, 0, t0 + k * K::GNT, c);
                ++ld_count;
            }
        }
        __syncthreads();

        float acc[K::F2];
#pragma unroll
        for (int i = 0; i < K::F2; ++i) acc[i] = 0.f;

        for (int it = 0; it < n_it; ++it) {
            const int t = t0 + it * K::GNT;
            unsigned char *stage;
            if (kTMA) {
                const uint32_t buf = use_count & 1u;
                stage = stage0 + buf * kStageStride;
                if (!gc_mbar_wait(&bars[buf], (use_count >> 1) & 1u, GC_WAIT_LIMIT_NS)) {
                    atomicOr(p.status, GC_DEV_TIMEOUT_FFT);
                    s_err = 1;
                } else {
                    ++use_count;
                }
                __syncthreads();
                if (s_err) break;
            } else {
                stage = stage0;
                stage_plain<K>(p, stage, c, t);
                __syncthreads();
            }

            // ---------------- row pass
            for (int r = tid; r < rows_per_it; r += K::NTHREADS) {
                const int y = r % L;
                const int rest = r / L;
                const int u = rest % K::GNT;
                const int s = rest / K::GNT;
                const int k = q + K::R * s;
                float2 b[K::F1];
#pragma unroll
                for (int i = 0; i < K::F1; ++i) b[i] = make_float2(0.f, 0.f);
                const float2 *crow = coef + y * K::CROW;
                const unsigned char *srow = stage + (u * K::LMAX + y) * K::ROWB;
#pragma unroll
                for (int j = 0; j < K::J1; ++j) {
                    if (K::VF == GC_C64) {
#pragma unroll
                        for (int xp = 0; xp < K::F1; xp += 2) {
                            const int x = xp + K::F1 * j;
                            if (x < K::LMAX) {
                                const float4 vv = *reinterpret_cast<const float4 *>(srow + x * 8);
                                const float4 cc = *reinterpret_cast<const float4 *>(crow + x);
                                row_in<K>(b[xp], make_float2(vv.x, vv.y), make_float2(cc.x, cc.y), tws, k, x);
                                row_in<K>(b[xp + 1], make_float2(vv.z, vv.w), make_float2(cc.z, cc.w), tws, k, x + 1);
                            }
                        }
                    } else if (K::VF == GC_C32H) {
#pragma unroll
                        for (int xp = 0; xp < K::F1; xp += 4) {
                            const int x = xp + K::F1 * j;
                            if (x < K::LMAX) {
                                const uint4 raw = *reinterpret_cast<const uint4 *>(srow + x * 4);
                                const float4 c01 = *reinterpret_cast<const float4 *>(crow + x);
                                const float4 c23 = *reinterpret_cast<const float4 *>(crow + x + 2);
                                row_in<K>(b[xp], h2_to_f2(raw.x), make_float2(c01.x, c01.y), tws, k, x);
                                row_in<K>(b[xp + 1], h2_to_f2(raw.y), make_float2(c01.z, c01.w), tws, k, x + 1);
                                row_in<K>(b[xp + 2], h2_to_f2(raw.z), make_float2(c23.x, c23.y), tws, k, x + 2);
                                row_in<K>(b[xp + 3], h2_to_f2(raw.w), make_float2(c23.z, c23.w), tws, k, x + 3);
                            }
                        }
                    } else {
#pragma unroll
                        for (int xp = 0; xp < K::F1; xp += 16) {
                            const int x0 = xp + K::F1 * j;
                            if (x0 < K::LMAX) {
                                const uint4 raw = *reinterpret_cast<const uint4 *>(srow + x0);
                                const unsigned int words[4] = {raw.x, raw.y, raw.z, raw.w};
                                // n + 8 of the four Re and the four Im nibbles of a word,
                                // one byte each (two and one instructions)
                                unsigned int ure[4], uim[4];
#pragma unroll
                                for (int w = 0; w < 4; ++w) {
                                    ure[w] = ((words[w] >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
                                    uim[w] = (words[w] & 0x0F0F0F0Fu) ^ 0x08080808u;
                                }
#pragma unroll
                                for (int e = 0; e < 16 && xp + e < K::F1; ++e) {
                                    const int x = x0 + e;
                                    if (x < K::LMAX) {
                                        const float2 v = i4c_bytes_to_f2(ure[e >> 2], uim[e >> 2], e & 3);
                                        row_in<K>(b[xp + e], v, crow[x], tws, k, x);
                                    }
                                }
                            }
                        }
                    }
                }
                fft_reg<K::F1>(b);
                float2 *irow = inter + (u * K::LMAX + y) * K::IROW;
#pragma unroll
                for (int i = 0; i < K::F1; ++i) irow[s + K::S1 * bitrev<K::F1>(i)] = b[i];
            }
            __syncthreads();

            // refill the consumed stage with the samples two iterations ahead
            if (kTMA && tid == 0 && it + 2 < n_it) {
                gc_fence_proxy_async();
                unsigned char *dst = stage0 + (ld_count & 1u) * kStageStride;
                gc_mbar_expect_tx(&bars[ld_count & 1u], K::STAGE_BYTES);
                gc_tma_load_4d(dst, &tmap, &bars[ld_count & 1u], 0, 0, t + 2 * K::GNT, c);
                ++ld_count;
            }

            // ---------------- column pass + power
#pragma unroll 1
            for (int u = 0; u < K::NT; ++u) {
                const float2 *icol = inter + ((g * K::NT + u) * K::LMAX) * K::IROW + kxl;
                float2 b[K::F2];
                if constexpr (K::J2 == 2 && K::S2 == 4 && K::LMAX == 2 * K::F2) {
                    // s2 is uniform over each warp (MX >= 32 threads per residue)
                    switch (s2) {
                        case 0: col_fold2<K, 0>(b, icol, tws); break;
                        case 1: col_fold2<K, 1>(b, icol, tws); break;
                        case 2: col_fold2<K, 2>(b, icol, tws); break;
                        default: col_fold2<K, 3>(b, icol, tws); break;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < K::F2; ++i) b[i] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < K::J2; ++j) {
#pragma unroll
                        for (int yp = 0; yp < K::F2; ++yp) {
                            const int y = yp + K::F2 * j;
                            if (y < K::LMAX) b[yp] = cfma(b[yp], icol[y * K::IROW], tws[(s2 * y) & (K::M - 1)]);
                        }
                    }
                }
                fft_reg<K::F2>(b);
#pragma unroll
                for (int i = 0; i < K::F2; ++i) acc[i] = fmaf(b[i].x, b[i].x, fmaf(b[i].y, b[i].y, acc[i]));
            }
            __syncthreads();
        }
        if (s_err) break;

        // chunk spectrum P[k_y][k_x]: the groups hold the same bins for
        // different samples; groups 1.. park theirs in the (now idle)
        // intermediate buffer and group 0 adds them up and stores
        if constexpr (K::G > 1) {
            float *park = reinterpret_cast<float *>(inter);
            if (g > 0) {
#pragma unroll
                for (int i = 0; i < K::F2; ++i) park[((g - 1) * K::F2 + i) * K::NCOL + col] = acc[i];
            }
            __syncthreads();
            if (g == 0) {
#pragma unroll
                for (int i = 0; i < K::F2; ++i)
                    for (int gg = 1; gg < K::G; ++gg) acc[i] += park[((gg - 1) * K::F2 + i) * K::NCOL + col];
            }
        }
        if (g == 0) {
            float *out = p.ppart + ((size_t)c * p.n_chunks + chunk) * K::M * K::M;
            const int kx = q + K::R * kxl;
#pragma unroll
            for (int i = 0; i < K::F2; ++i) out[(s2 + K::S2 * bitrev<K::F2>(i)) * K::M + kx] = acc[i];
        }
    }

    if (kTMA && s_err && tid == 0) {
        // let copies still in flight land before the CTA exits (bounded)
        while (use_count < ld_count) {
            gc_mbar_wait(&bars[use_count & 1u], (use_count >> 1) & 1u, GC_WAIT_LIMIT_NS / 10);
            ++use_count;
        }
    }
}

// ----------------------------------------------------------------- finalize
template <int M>
__global__ void __launch_bounds__(256)
fftcorr_finalize(const float *__restrict__ ppart, int n_parts, float2 *__restrict__ vunique, int L, int T,
                 const float *__restrict__ ndtab, unsigned int *status) {
    extern __shared__ __align__(128) unsigned char smem[];
    float *P = reinterpret_cast<float *>(smem);                 // [M][M]
    float2 *Q = reinterpret_cast<float2 *>(smem + M * M * 4);   // [M][W]
    float2 *tws = Q + M * (2 * L - 1);                          // [M]
    const int c = blockIdx.x, W = 2 * L - 1;
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const cf w = c_tw.v[e * (256 / M)];
        tws[e] = make_float2(w.x, w.y);
    }
    const float *src = ppart + (size_t)c * n_parts * M * M;
    for (int k = threadIdx.x; k < M * M; k += blockDim.x) {
        double s = 0.0;
        for (int pp = 0; pp < n_parts; ++pp) s += (double)src[(size_t)pp * M * M + k];
        if (!isfinite(s)) atomicOr(status, GC_DEV_BADINPUT);   // non-finite voltages
        P[k] = (float)s;
    }
    __syncthreads();
    // Q[ky][dx] = sum_kx P[ky][kx] exp(+2 pi i kx dx / M)
    for (int idx = threadIdx.x; idx < M * W; idx += blockDim.x) {
        const int ky = idx / W, dx = idx % W - (L - 1);
        float re = 0.f, im = 0.f;
        for (int kx = 0; kx < M; ++kx) {
            const float2 w = tws[(kx * dx) & (M - 1)];   // conj gives the + sign
            const float pv = P[ky * M + kx];
            re = fmaf(pv, w.x, re);
            im = fmaf(-pv, w.y, im);
        }
        Q[ky * W + (dx + L - 1)] = make_float2(re, im);
    }
    __syncthreads();
    // R[dy][dx] = (1/M^2) sum_ky Q[ky][dx] exp(+2 pi i ky dy / M); V = R / (T N_d)
    for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
        const int dyi = idx / W, dxi = idx % W;
        const int dy = dyi - (L - 1), dx = dxi - (L - 1);
        float re = 0.f, im = 0.f;
        for (int ky = 0; ky < M; ++ky) {
            const float2 w = tws[(ky * dy) & (M - 1)];
            const float2 qv = Q[ky * W + dxi];
            // qv * conj(w)
            re = fmaf(qv.x, w.x, fmaf(qv.y, w.y, re));
            im = fmaf(qv.y, w.x, fmaf(-qv.x, w.y, im));
        }
        // N_d: pairs per lag (a partly occupied lattice passes its table)
        const double nd = ndtab ? (double)ndtab[idx] : (double)((L - (dx < 0 ? -dx : dx)) * (L - (dy < 0 ? -dy : dy)));
        const float s = nd > 0.0 ? (float)(1.0 / ((double)M * M * (double)T * nd)) : 0.f;
        vunique[(size_t)c * W * W + idx] = make_float2(re * s, im * s);
    }
}

// Two-pass inverse DFT for large M (the M x M spectrum of one channel does
// not fit in shared memory beside its partial transform).
//   rows: Q[c][ky][dx] = sum_kx P[ky][kx] exp(+2 pi i kx dx / M),
//         P = FP64 sum of the chunk spectra; kFinRows k_y rows per CTA.
//   cols: V[c][dy][dx] = (1/M^2) sum_ky Q[ky][dx] exp(+2 pi i ky dy / M) / (T N_d);
//         kFinCols lag columns per CTA.
constexpr int kFinRows = 8;
constexpr int kFinCols = 16;

template <int M>
__global__ void __launch_bounds__(256)
fftcorr_finalize_rows(const float *__restrict__ ppart, int n_parts, float2 *__restrict__ Q, int L,
                      unsigned int *status) {
    __shared__ float P[kFinRows][M];
    __shared__ float2 tws[M];
    const int c = blockIdx.x, ky0 = blockIdx.y * kFinRows, W = 2 * L - 1;
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const cf w = c_tw.v[e * (256 / M)];
        tws[e] = make_float2(w.x, w.y);
    }
    const float *src = ppart + (size_t)c * n_parts * M * M + (size_t)ky0 * M;
    for (int k = threadIdx.x; k < kFinRows * M; k += blockDim.x) {
        double s = 0.0;
        for (int pp = 0; pp < n_parts; ++pp) s += (double)src[(size_t)pp * M * M + k];
        if (!isfinite(s)) atomicOr(status, GC_DEV_BADINPUT);
        P[k / M][k % M] = (float)s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kFinRows * W; idx += blockDim.x) {
        const int r = idx / W, dx = idx % W - (L - 1);
        float re = 0.f, im = 0.f;
        for (int kx = 0; kx < M; ++kx) {
            const float2 w = tws[(kx * dx) & (M - 1)];
            const float pv = P[r][kx];
            re = fmaf(pv, w.x, re);
            im = fmaf(-pv, w.y, im);
        }
        Q[((size_t)c * M + ky0 + r) * W + (dx + L - 1)] = make_float2(re, im);
    }
}

template <int M>
__global__ void __launch_bounds__(256)
fftcorr_finalize_cols(const float2 *__restrict__ Q, float2 *__restrict__ vunique, int L, int T,
                      const float *__restrict__ ndtab) {
    __shared__ float2 Qs[M][kFinCols];
    __shared__ float2 tws[M];
    const int c = blockIdx.x, dx0 = blockIdx.y * kFinCols, W = 2 * L - 1;
    const int ncol = min(kFinCols, W - dx0);
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const cf w = c_tw.v[e * (256 / M)];
        tws[e] = make_float2(w.x, w.y);
    }
    for (int k = threadIdx.x; k < M * kFinCols; k += blockDim.x) {
        const int ky = k / kFinCols, j = k % kFinCols;
        Qs[ky][j] = j < ncol ? Q[((size_t)c * M + ky) * W + dx0 + j] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < W * ncol; idx += blockDim.x) {
        const int dyi = idx / ncol, j = idx % ncol;
        const int dy = dyi - (L - 1), dxi = dx0 + j, dx = dxi - (L - 1);
        float re = 0.f, im = 0.f;
        for (int ky = 0; ky < M; ++ky) {
            const float2 w = tws[(ky * dy) & (M - 1)];
            const float2 qv = Qs[ky][j];
            re = fmaf(qv.x, w.x, fmaf(qv.y, w.y, re));
            im = fmaf(qv.y, w.x, fmaf(-qv.x, w.y, im));
        }
        const double nd = ndtab ? (double)ndtab[(size_t)dyi * W + dxi]
                                : (double)((L - (dx < 0 ? -dx : dx)) * (L - (dy < 0 ? -dy : dy)));
        const float s = nd > 0.0 ? (float)(1.0 / ((double)M * M * (double)T * nd)) : 0.f;
        vunique[(size_t)c * W * W + (size_t)dyi * W + dxi] = make_float2(re * s, im * s);
    }
}

// ----------------------------------------------------------------- host side
template <class K>
CUtensorMapDataType tma_dtype() {
    return K::VF == GC_C64 ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                           : (K::VF == GC_C32H ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT8);
}

template <class K>
struct Launcher {
    // h_mask (host, L*L, or null): a partly occupied lattice -- zero
    // coefficients at the empty points and N_d from the mask's pairs
    static gc_status run(gc_ctx *ctx, const void *volt, int L, int C, int T, const float *gains,
                         float *vunique, cudaStream_t stream, const unsigned char *h_mask = nullptr) {
        const int N = L * L;
        const bool tma = gc_aligned(volt, 16) && ((size_t)L * K::ESZ) % 16 == 0;
        auto kern = tma ? fftcorr_accumulate<K, true> : fftcorr_accumulate<K, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaFuncSetAttribute(fftcorr_accumulate)");
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, K::NTHREADS, K::SMEM);
        if (e != cudaSuccess || occ < 1) return gc_cuda_fail(ctx, e, "occupancy(fftcorr_accumulate)");
        const int slots = occ * ctx->sm_count;

        // time chunking: chunks of <= 512 samples, chosen so the work items
        // fill whole waves of the resident CTAs
        const int step = K::GNT;
        int best_n = 1, best_len = ((T + step - 1) / step) * step;
        double best_eff = -1.0;
        const int n_min = std::max(1, (T + 511) / 512);
        for (int n = n_min; n <= n_min + 64; ++n) {
            const int len = ((T + n - 1) / n + step - 1) / step * step;
            const int nn = (T + len - 1) / len;
            const long items = (long)C * K::R * nn;
            const long waves = (items + slots - 1) / slots;
            const double eff = (double)C * K::R * T / ((double)waves * slots * len);
            if (eff > best_eff + 1e-9) {
                best_eff = eff;
                best_n = nn;
                best_len = len;
            }
        }
        if (ctx->tune[GC_TUNE_FFT_CHUNK] > 0) {
            best_len = ((std::min(ctx->tune[GC_TUNE_FFT_CHUNK], 4096) + step - 1) / step) * step;
            best_n = (T + best_len - 1) / best_len;
        }
        Params p;
        p.volt = volt;
        p.gains = reinterpret_cast<const float2 *>(gains);
        p.status = ctx->status_dev;
        p.L = L;
        p.C = C;
        p.T = T;
        p.chunk_len = best_len;
        p.n_chunks = best_n;
        p.n_items = C * K::R * best_n;
        const size_t part_bytes = ((size_t)C * best_n * K::M * K::M * sizeof(float) + 255) / 256 * 256;
        const size_t q_bytes = K::M > 128 ? (size_t)C * K::M * (2 * L - 1) * sizeof(float2) : 0;
        const int Wd = 2 * L - 1;
        const size_t nd_bytes = h_mask ? ((size_t)Wd * Wd * sizeof(float) + 255) / 256 * 256 : 0;
        const size_t mask_bytes = h_mask ? ((size_t)N + 255) / 256 * 256 : 0;
        const size_t qb = (q_bytes + 255) / 256 * 256;
        gc_status st = gc_scratch_reserve(ctx, part_bytes + qb + nd_bytes + mask_bytes);
        if (st != GC_OK) return st;
        p.ppart = reinterpret_cast<float *>(ctx->scratch);
        const float *ndtab = nullptr;
        if (h_mask) {
            // N_d = number of occupied pairs per lag (host, once per call)
            std::vector<float> nd((size_t)Wd * Wd, 0.f);
            std::vector<int> occ;
            for (int i = 0; i < N; ++i)
                if (h_mask[i]) occ.push_back(i);
            for (int a : occ)
                for (int b : occ) nd[(size_t)(a / L - b / L + L - 1) * Wd + (a % L - b % L + L - 1)] += 1.f;
            char *aux = static_cast<char *>(ctx->scratch) + part_bytes + qb;
            std::vector<unsigned char> m01(N);
            for (int i = 0; i < N; ++i) m01[i] = h_mask[i] ? 1 : 0;
            // pageable sources: the calls return once the data is staged
            e = cudaMemcpyAsync(aux, nd.data(), (size_t)Wd * Wd * sizeof(float), cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(aux + nd_bytes, m01.data(), (size_t)N, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "upload lattice mask");
            ndtab = reinterpret_cast<const float *>(aux);
            p.mask = reinterpret_cast<const unsigned char *>(aux + nd_bytes);
        }

        CUtensorMap tmap;
        memset(&tmap, 0, sizeof tmap);
        if (tma) {
            const uint64_t dims[4] = {(uint64_t)L, (uint64_t)L, (uint64_t)T, (uint64_t)C};
            const uint64_t strides[3] = {(uint64_t)L * K::ESZ, (uint64_t)N * K::ESZ,
                                         (uint64_t)T * N * K::ESZ};
            const uint32_t box[4] = {(uint32_t)K::ROWE, (uint32_t)K::LMAX, (uint32_t)K::GNT, 1u};
            st = gc_encode_tiled(ctx, &tmap, tma_dtype<K>(), 4, const_cast<void *>(volt), dims, strides, box);
            if (st != GC_OK) return st;
        }
        const int grid = (int)std::min<long>(p.n_items, slots);
        int rec = gc_prof_begin(ctx, stream, "fftcorr_accumulate");
        kern<<<grid, K::NTHREADS, K::SMEM, stream>>>(tmap, p);
        gc_prof_end(ctx, stream, rec);
        e = cudaGetLastError();
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch fftcorr_accumulate");

        const int W = 2 * L - 1;
        if constexpr (K::M > 128) {
            float2 *Q = reinterpret_cast<float2 *>(static_cast<char *>(ctx->scratch) + part_bytes);
            rec = gc_prof_begin(ctx, stream, "fftcorr_finalize");
            fftcorr_finalize_rows<K::M><<<dim3(C, K::M / kFinRows), 256, 0, stream>>>(p.ppart, best_n, Q, L,
                                                                                       p.status);
            fftcorr_finalize_cols<K::M><<<dim3(C, (W + kFinCols - 1) / kFinCols), 256, 0, stream>>>(
                Q, reinterpret_cast<float2 *>(vunique), L, T, ndtab);
            gc_prof_end(ctx, stream, rec);
        } else {
            const size_t fsmem = (size_t)K::M * K::M * 4 + (size_t)K::M * W * 8 + K::M * 8;
            auto fin = fftcorr_finalize<K::M>;
            e = cudaFuncSetAttribute(fin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
            if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaFuncSetAttribute(fftcorr_finalize)");
            rec = gc_prof_begin(ctx, stream, "fftcorr_finalize");
            fin<<<C, 256, fsmem, stream>>>(p.ppart, best_n, reinterpret_cast<float2 *>(vunique), L, T, ndtab, p.status);
            gc_prof_end(ctx, stream, rec);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch fftcorr_finalize");
        return GC_OK;
    }
};

// configurations per FFT side (see the design notes for the smem budget)
using CfgC16 = Cfg<16, 1, 16, 16, 2, 8, GC_C64>;
using CfgC32 = Cfg<32, 1, 32, 32, 2, 4, GC_C64>;
using CfgC64 = Cfg<64, 1, 32, 32, 2, 1, GC_C64>;
using CfgC128 = Cfg<128, 4, 32, 32, 1, 1, GC_C64>;
using CfgI16 = Cfg<16, 1, 16, 16, 2, 8, GC_I4C>;
using CfgI32 = Cfg<32, 1, 32, 32, 2, 4, GC_I4C>;
using CfgI64 = Cfg<64, 1, 32, 32, 2, 1, GC_I4C>;
using CfgI128 = Cfg<128, 4, 32, 32, 1, 2, GC_I4C, 2>;   // two groups share the coefficients; 16 warps/SM
// alternative launch shapes ("fft.shape" = 1): one sample group of two
// samples per thread (no idle threads in the row pass, 8 warps/SM) for the
// 64x64 4+4-bit grid; two groups of one sample for the 32x32 complex64 grid
using CfgI128b = Cfg<128, 4, 32, 32, 2, 1, GC_I4C, 2>;
using CfgC64b = Cfg<64, 1, 32, 32, 1, 2, GC_C64>;
// M = 256 (L = 65..128): 4+4-bit only -- one complex64 or binary16 grid sample
// (128 rows of 1 KB / 512 B) does not fit a double-buffered stage beside the
// 133 KB coefficient table.  Eight k_x residues, one sample per iteration,
// one CTA of 256 threads per SM (201 KB shared memory).
using CfgI256 = Cfg<256, 8, 16, 32, 1, 1, GC_I4C>;
using CfgH16 = Cfg<16, 1, 16, 16, 2, 8, GC_C32H>;
using CfgH32 = Cfg<32, 1, 32, 32, 2, 4, GC_C32H>;
using CfgH64 = Cfg<64, 1, 32, 32, 2, 1, GC_C32H>;
using CfgH128 = Cfg<128, 4, 32, 32, 1, 2, GC_C32H>;

// Row stage on the tensor cores (gc_fftcorr_tc.cu), then the same finalize.
gc_status tc_correlate(gc_ctx *ctx, const void *volt, int L, int C, int T, const float *gains, float *vunique,
                       cudaStream_t stream) {
    float *ppart = nullptr;
    int n_chunks = 0;
    gc_status st = gc_fft_tc_run(ctx, volt, L, C, T, gains, &ppart, &n_chunks, stream);
    if (st != GC_OK) return st;
    const int W = 2 * L - 1;
    const size_t fsmem = (size_t)128 * 128 * 4 + (size_t)128 * W * 8 + 128 * 8;
    auto fin = fftcorr_finalize<128>;
    cudaError_t e = cudaFuncSetAttribute(fin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaFuncSetAttribute(fftcorr_finalize)");
    const int rec = gc_prof_begin(ctx, stream, "fftcorr_finalize");
    fin<<<C, 256, fsmem, stream>>>(ppart, n_chunks, reinterpret_cast<float2 *>(vunique), L, T, nullptr,
                                   ctx->status_dev);
    gc_prof_end(ctx, stream, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch fftcorr_finalize");
    return GC_OK;
}

}  // namespace

static gc_status correlate_impl(gc_ctx *ctx, const void *volt, int vfmt, int L, int C, int T, const float *gains,
                                float *vunique, void *stream, const unsigned char *h_mask) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    if (!volt || !gains || !vunique) return gc_fail(ctx, GC_EINVAL, "gc_correlate: null buffer");
    if (L < 1 || L > 128 || C < 1 || T < 1)
        return gc_fail(ctx, GC_EINVAL, "gc_correlate: need 1 <= L <= 128, C >= 1, T >= 1");
    if (vfmt != GC_C64 && vfmt != GC_I4C && vfmt != GC_C32H)
        return gc_fail(ctx, GC_EINVAL, "gc_correlate: unknown voltage format");
    if (L > 64 && vfmt != GC_I4C)
        return gc_fail(ctx, GC_EUNSUPPORTED, "gc_correlate: L > 64 is built for 4+4-bit voltages only");
    if (!gc_aligned(gains, 8) || !gc_aligned(vunique, 8) || (vfmt == GC_C64 && !gc_aligned(volt, 8)) ||
        (vfmt == GC_C32H && !gc_aligned(volt, 4)))
        return gc_fail(ctx, GC_EINVAL, "gc_correlate: misaligned buffer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    const int M = std::max(16, gc_fft_size(L));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (vfmt == GC_C64) {
        switch (M) {
            case 16: return Launcher<CfgC16>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 32: return Launcher<CfgC32>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 64:
                if (ctx->tune[GC_TUNE_FFT_SHAPE] == 1) return Launcher<CfgC64b>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
                return Launcher<CfgC64>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 128: return Launcher<CfgC128>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
        }
    } else if (vfmt == GC_C32H) {
        switch (M) {
            case 16: return Launcher<CfgH16>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 32: return Launcher<CfgH32>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 64: return Launcher<CfgH64>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 128: return Launcher<CfgH128>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
        }
    } else {
        switch (M) {
            case 16: return Launcher<CfgI16>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 32: return Launcher<CfgI32>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 64: return Launcher<CfgI64>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 128:
                if (gc_fft_tc_eligible(ctx, vfmt, L, volt, h_mask != nullptr))
                    return tc_correlate(ctx, volt, L, C, T, gains, vunique, s);
                if (ctx->tune[GC_TUNE_FFT_SHAPE] == 1) return Launcher<CfgI128b>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
                return Launcher<CfgI128>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
            case 256: return Launcher<CfgI256>::run(ctx, volt, L, C, T, gains, vunique, s, h_mask);
        }
    }
    return gc_fail(ctx, GC_EUNSUPPORTED, "gc_correlate: no kernel for this grid size");
}

extern "C" gc_status gc_correlate(gc_ctx *ctx, const void *volt, int vfmt, int L, int C, int T,
                                  const float *gains, float *vunique, void *stream) {
    return correlate_impl(ctx, volt, vfmt, L, C, T, gains, vunique, stream, nullptr);
}

extern "C" gc_status gc_correlate_masked(gc_ctx *ctx, const void *volt, int vfmt, int L, int C, int T,
                                         const uint8_t *mask, const float *gains, float *vunique, void *stream) {
    if (ctx && !mask) return gc_fail(ctx, GC_EINVAL, "gc_correlate_masked: null mask");
    return correlate_impl(ctx, volt, vfmt, L, C, T, gains, vunique, stream, mask);
}

// ============================================================================
// gc_correlate_noalloc: the FFT-correlator for callers that may not allocate
// device memory (see include/gridcorr.h).  The per-chunk power spectra live
// in a fixed, file-scope device array instead of the context workspace.
// ============================================================================
#include <mutex>

namespace {

constexpr size_t kNoallocScratchBytes = 64ull << 20;   // 64 MiB, held by every GPU that loads the library
static __device__ __align__(256) float g_noalloc_scratch[kNoallocScratchBytes / sizeof(float)];
static __device__ unsigned int g_noalloc_status;       // timeout flags when the caller passes none

struct NoallocDev {
    float *scratch = nullptr;
    unsigned int *status = nullptr;
};
std::mutex g_noalloc_mu;
void *g_noalloc_encode = nullptr;

// On every call, with the caller's device current: resolve the device
// addresses of the file-scope arrays (host code only sees a host-side
// stand-in symbol).  The lookup enqueues nothing; doing it per call keeps the
// addresses right after a device or context reset reloads the module.
gc_status noalloc_setup(NoallocDev *d) {
    void *p = nullptr, *q = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
        cudaGetLastError();
        return GC_ECUDA;
    }
    if (cudaGetSymbolAddress(&q, g_noalloc_status) != cudaSuccess) {
        cudaGetLastError();
        return GC_ECUDA;
    }
    d->scratch = static_cast<float *>(p);
    d->status = static_cast<unsigned int *>(q);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_encode) {
        cudaDriverEntryPointQueryResult qr;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            g_noalloc_encode = fn;
    }
    return GC_OK;
}

template <class K>
gc_status noalloc_run(const NoallocDev &d, const void *volt, int L, int C, int T, const float *gains,
                      float *vunique, unsigned int *status, cudaStream_t stream) {
    const int N = L * L;
    const size_t per_chunk = (size_t)C * K::M * K::M * sizeof(float);
    const int n_min = std::max(1, (T + 511) / 512);      // chunks of <= 512 samples
    if (per_chunk * n_min > kNoallocScratchBytes) return GC_EINVAL;
    const int n_cap = (int)std::min<size_t>(kNoallocScratchBytes / per_chunk, (size_t)n_min + 64);
    bool tma = gc_aligned(volt, 16) && ((size_t)L * K::ESZ) % 16 == 0 && g_noalloc_encode != nullptr;
    auto kern = tma ? fftcorr_accumulate<K, true> : fftcorr_accumulate<K, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM) != cudaSuccess)
        return GC_ECUDA;
    int occ = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, K::NTHREADS, K::SMEM) != cudaSuccess ||
        occ < 1 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GC_ECUDA;
    const int slots = occ * sms;
    const int step = K::GNT;
    int best_n = n_min, best_len = ((T + n_min - 1) / n_min + step - 1) / step * step;
    double best_eff = -1.0;
    for (int n = n_min; n <= n_cap; ++n) {
        const int len = ((T + n - 1) / n + step - 1) / step * step;
        const int nn = (T + len - 1) / len;
        if (nn > n_cap) continue;
        const long items = (long)C * K::R * nn;
        const long waves = (items + slots - 1) / slots;
        const double eff = (double)C * K::R * T / ((double)waves * slots * len);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best_n = nn;
            best_len = len;
        }
    }
    Params p;
    p.volt = volt;
    p.gains = reinterpret_cast<const float2 *>(gains);
    p.ppart = d.scratch;
    p.status = status ? status : d.status;
    p.L = L;
    p.C = C;
    p.T = T;
    p.chunk_len = best_len;
    p.n_chunks = best_n;
    p.n_items = C * K::R * best_n;

    CUtensorMap tmap;
    memset(&tmap, 0, sizeof tmap);
    if (tma) {
        using Fn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                CUtensorMapFloatOOBfill);
        const cuuint64_t dims[4] = {(cuuint64_t)L, (cuuint64_t)L, (cuuint64_t)T, (cuuint64_t)C};
        const cuuint64_t strides[3] = {(cuuint64_t)L * K::ESZ, (cuuint64_t)N * K::ESZ,
                                       (cuuint64_t)T * N * K::ESZ};
        const cuuint32_t box[4] = {(cuuint32_t)K::ROWE, (cuuint32_t)K::LMAX, (cuuint32_t)K::GNT, 1u};
        const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
        CUresult r = reinterpret_cast<Fn>(g_noalloc_encode)(
            &tmap, tma_dtype<K>(), 4,
            const_cast<void *>(volt), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return GC_ECUDA;
    }
    const int grid = (int)std::min<long>(p.n_items, slots);
    kern<<<grid, K::NTHREADS, K::SMEM, stream>>>(tmap, p);
    if (cudaGetLastError() != cudaSuccess) return GC_ECUDA;
    const int W = 2 * L - 1;
    const size_t fsmem = (size_t)K::M * K::M * 4 + (size_t)K::M * W * 8 + K::M * 8;
    auto fin = fftcorr_finalize<K::M>;
    if (cudaFuncSetAttribute(fin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem) != cudaSuccess)
        return GC_ECUDA;
    fin<<<C, 256, fsmem, stream>>>(p.ppart, best_n, reinterpret_cast<float2 *>(vunique), L, T, nullptr,
                                   p.status);
    if (cudaGetLastError() != cudaSuccess) return GC_ECUDA;
    return GC_OK;
}

}  // namespace

extern "C" gc_status gc_correlate_noalloc(const void *volt, int vfmt, int L, int C, int T, const float *gains,
                                          float *vunique, unsigned int *status, void *stream) {
    if (!volt || !gains || !vunique) return GC_EINVAL;
    if (L < 1 || L > 64 || C < 1 || T < 1) return GC_EINVAL;
    if (vfmt != GC_C64 && vfmt != GC_I4C && vfmt != GC_C32H) return GC_EINVAL;
    if (!gc_aligned(gains, 8) || !gc_aligned(vunique, 8) || (vfmt == GC_C64 && !gc_aligned(volt, 8)) ||
        (vfmt == GC_C32H && !gc_aligned(volt, 4)) || (status && !gc_aligned(status, 4)))
        return GC_EINVAL;
    NoallocDev dd;
    gc_status st = noalloc_setup(&dd);
    if (st != GC_OK) return st;
    const NoallocDev *d = &dd;
    const int M = std::max(16, gc_fft_size(L));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (vfmt == GC_C64) {
        switch (M) {
            case 16: return noalloc_run<CfgC16>(*d, volt, L, C, T, gains, vunique, status, s);
            case 32: return noalloc_run<CfgC32>(*d, volt, L, C, T, gains, vunique, status, s);
            case 64: return noalloc_run<CfgC64>(*d, volt, L, C, T, gains, vunique, status, s);
            case 128: return noalloc_run<CfgC128>(*d, volt, L, C, T, gains, vunique, status, s);
        }
    } else if (vfmt == GC_C32H) {
        switch (M) {
            case 16: return noalloc_run<CfgH16>(*d, volt, L, C, T, gains, vunique, status, s);
            case 32: return noalloc_run<CfgH32>(*d, volt, L, C, T, gains, vunique, status, s);
            case 64: return noalloc_run<CfgH64>(*d, volt, L, C, T, gains, vunique, status, s);
            case 128: return noalloc_run<CfgH128>(*d, volt, L, C, T, gains, vunique, status, s);
        }
    } else {
        switch (M) {
            case 16: return noalloc_run<CfgI16>(*d, volt, L, C, T, gains, vunique, status, s);
            case 32: return noalloc_run<CfgI32>(*d, volt, L, C, T, gains, vunique, status, s);
            case 64: return noalloc_run<CfgI64>(*d, volt, L, C, T, gains, vunique, status, s);
            case 128: return noalloc_run<CfgI128>(*d, volt, L, C, T, gains, vunique, status, s);
        }
    }
    return GC_EUNSUPPORTED;
}
