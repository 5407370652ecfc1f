// FFT-correlator with the row stage of the spatial FFT on the tensor cores
// (paper Fig. 1b, Sec. 1 convolution theorem, Eq. modelvis), for 4+4-bit
// voltages on grids of 33..64 antennas a side (M = 128).
//
// Per time sample the zero-padded 2-D DFT X(k_y, k_x) of the calibrated
// voltages w = v / g splits into a row stage over x and a column stage over
// y.  The row stage is a matrix product with one matrix for every row and
// sample:
//   X1[k_x][y] = sum_x w[y][x] exp(-2 pi i k_x x / 128),  x < 64, k_x < 128
// written in real form with A = [C | S] (C = cos, S = sin of 2 pi k_x x / 128;
// M = 128 rows k_x, K = 128 = Re and Im parts of 64 inputs) and
// B[k][y] = (Re w[y][k], Im w[y][k - 64]):
//   Re X1 = A B,   Im X1 = sum_{k < 64} S.. : C Im w - S Re w,
// i.e. the Im product pairs the C half of A with the Im half of B and the S
// half of A, negated, with the Re half of B (the negate-A bit of the
// instruction), so one A serves both products.  The products run as
// tcgen05.mma kind::f16 (FP32 accumulation in tensor memory) on a split of
// every FP32 value into two binary16 parts, hi = fp16(v) and
// lo = fp16(v - hi) (22 significant bits together): A_hi B_hi + A_hi B_lo +
// A_lo B_hi, the dropped A_lo B_lo term is below 2^-22 of the product.  The
// zero padding to 128 never appears: x and y stop at 64.
//
// The column stage stays on the CUDA cores, with tensor-memory lane = k_x:
// thread (k_x, s2) reads the 64 values X1[k_x][y] of its lane (the D columns),
// folds them for the column residue s2 (k_y = s2 + 4 m: the first radix-4
// stage of a 128-point FFT whose upper 64 inputs are zero), runs a 32-point
// FFT in registers and adds |X|^2 into its power-spectrum columns in tensor
// memory.  At the end of a time chunk the power spectrum goes to the chunk
// spectra [C][chunks][128][128] that fftcorr_finalize inverts.
//
// Warp roles (one CTA per SM, persistent over (channel, time chunk) items):
//   warps 0-7   column stage: warp w takes tensor-memory lanes 32 (w % 4) ..
//               +31 and the column residues w / 4 and w / 4 + 2 (one load of
//               the D columns feeds both folds);
//   warps 8-9   converters: raw 4+4-bit samples -> w = v / g -> hi / lo
//               binary16 B operands in shared memory (K-major, no swizzle),
//               two samples per stage;
//   warp 10     bulk copies of raw samples (two per stage) into a ring;
//   warp 11     MMA issue (one thread), completion committed to the rings.
// Tensor memory (512 columns): D (two buffers of Re 64 + Im 64 columns),
// A_hi, A_lo (64 columns each: two binary16 of K per column), the power
// spectrum (128 columns: 4 residues x 32 bins).  Every wait is bounded; a
// wait that runs out sets GC_DEV_TIMEOUT_FFT and the CTA winds down.
#include <cuda_fp16.h>

#include <algorithm>

#include "gc_fft_reg.h"
#include "gc_internal.h"
#include "gc_tcgen05.h"

namespace {

constexpr int kTM = 128;                 // FFT side
constexpr int kTL = 64;                  // largest grid side (rows y and inputs x of the row stage)
// 12 warps: column stage 0-7 (warp w: tensor-memory lanes 32 (w % 4) .. +31,
// column residues s2 = (w / 4) and (w / 4) + 2, which share their fold
// inputs), converters 8-9, bulk copies 10, MMA issue 11.
constexpr int kThreadsTC = 384;
constexpr int kEpiWarps = 8;
constexpr int kWarpConv0 = 8, kConvWarps = 2, kWarpTma = 10, kWarpMma = 11;
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kTasks = kTL * 8 / kConvThreads;   // (row, group of 8 inputs) tasks per converter thread
static_assert(kConvWarps == 2 && kTasks == 8, "the converter task map covers 64 rows x 8 input groups with 64 threads");
constexpr int kSamp = 2;                          // samples per raw stage and per B stage
constexpr int kBStages = 2;
constexpr int kBPlane = kSamp * kTL * kTM * 2;    // one binary16 B operand of kSamp samples: 32 KB
constexpr int kBSample = kTL * kTM * 2;           // one sample's rows within a plane: 16 KB
constexpr int kBStage = 2 * kBPlane;              // hi, lo
constexpr int kRawSamp = kSamp;
constexpr int kRawStages = 3;
constexpr int kRawStride = kRawSamp * kTL * kTL + 128;   // + slack for the last row's 8-byte reads
constexpr int kCoefBytes = kTasks * 8 * kConvThreads * 8;   // [task i][input e][converter thread] float2
constexpr int kTwBytes = 2 * 2 * 32 * 8;                   // [pr][residue][y] float2
constexpr size_t kSmemTC = (size_t)kBStages * kBStage + (size_t)kRawStages * kRawStride + kCoefBytes + kTwBytes;
constexpr uint32_t kColD = 0, kColAHi = 256, kColALo = 320, kColP = 384;
constexpr uint32_t kLBO = 128, kSBO = 2048;   // K-adjacent / N-adjacent core-matrix strides

struct TcFftParams {
    const unsigned char *volt;   // [C][T][L*L] 4+4-bit
    const float2 *gains;         // [C][L*L]
    float *ppart;                // [C][n_chunks][128][128]
    unsigned int *status;
    int L, C, T;
    int chunk_len;               // multiple of kRawSamp
    int n_chunks, n_items;
};

// multiply by (-i)^R
template <int R>
__device__ __forceinline__ float2 rot_mi_tc(float2 a) {
    if (R == 0) return a;
    if (R == 1) return make_float2(a.y, -a.x);
    if (R == 2) return make_float2(-a.x, -a.y);
    return make_float2(-a.y, a.x);
}

// binary16 hi / lo parts of two floats, packed (lower K index in the low half)
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// |X|^2 of one residue's 32 bins into its power columns (first sample of a
// chunk: stored, later: added), 16 columns at a time
__device__ __forceinline__ void power_update(const float2 (&b)[32], uint32_t pcol, bool first) {
    if (!first) gc_tmem_wait_st();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t pv[16];
        if (!first) {
            gc_tmem_ld4_nowait(pcol + 16 * h, pv);
            gc_tmem_ld4_nowait(pcol + 16 * h + 4, pv + 4);
            gc_tmem_ld4_nowait(pcol + 16 * h + 8, pv + 8);
            gc_tmem_ld4_nowait(pcol + 16 * h + 12, pv + 12);
            gc_tmem_wait_ld16_regs(pv);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float2 v = b[16 * h + i];
            const float p0 = first ? 0.f : __uint_as_float(pv[i]);
            pv[i] = __float_as_uint(fmaf(v.x, v.x, fmaf(v.y, v.y, p0)));
        }
        gc_tmem_st16(pcol + 16 * h, pv);
    }
}

// The column stage of one sample for the residue pair pr: (0, 2) or (1, 3).
// For each of the two residues the 64 values X1[k_x][y] of this lane come in
// with one load of the Re and one of the Im columns (tensor memory is read
// twice rather than holding both folds in registers); y and y + 32 give the
// fold input
//   s2 = pr + 2 h:  (a0 + (-1)^h (-i)^pr a1) omega_128^((pr + 2 h) y)
// (twiddles from the table tw[h][y]), then a 32-point FFT and |X|^2 -- one
// copy of the code for both residues and both pairs, so that the
// instruction cache holds the whole column stage.
__device__ __forceinline__ void column_pair(uint32_t dre, uint32_t dim, uint32_t pcol_a, uint32_t pcol_b,
                                            bool first, int pr, const float2 *tw) {
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const float sg = h ? -1.f : 1.f;
        float2 b[32];
        {
            uint32_t re[64], im[64];
            gc_tmem_ld64_nowait(dre, re);
            gc_tmem_ld64_nowait(dim, im);
            gc_tmem_wait_ld();
            gc_reg_tie32(re);
            gc_reg_tie32(re + 32);
            gc_reg_tie32(im);
            gc_reg_tie32(im + 32);
#pragma unroll
            for (int y = 0; y < 32; ++y) {
                const float2 a0 = make_float2(__uint_as_float(re[y]), __uint_as_float(im[y]));
                const float2 a1 = make_float2(__uint_as_float(re[y + 32]), __uint_as_float(im[y + 32]));
                const float2 r = pr ? make_float2(a1.y, -a1.x) : a1;   // (-i)^pr a1
                b[y] = cmul(make_float2(fmaf(sg, r.x, a0.x), fmaf(sg, r.y, a0.y)), tw[32 * h + y]);
            }
        }
        fft_reg<32>(b);
        power_update(b, h ? pcol_b : pcol_a, first);
    }
}

struct ItemTC {
    int c, chunk, t0, nt;
};
__device__ __forceinline__ ItemTC decode_tc(const TcFftParams &p, int item) {
    ItemTC it;
    it.c = item / p.n_chunks;
    it.chunk = item % p.n_chunks;
    it.t0 = it.chunk * p.chunk_len;
    it.nt = min(p.chunk_len, p.T - it.t0);
    return it;
}

__global__ void __launch_bounds__(kThreadsTC, 1) fftcorr_tc_accumulate(const TcFftParams p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *bring = smem;
    unsigned char *raw = smem + (size_t)kBStages * kBStage;
    float2 *coef = reinterpret_cast<float2 *>(raw + (size_t)kRawStages * kRawStride);
    float2 *tws = coef + kCoefBytes / 8;   // column-fold twiddles omega_128^((pr + 2 r) y)
    __shared__ uint64_t full_raw[kRawStages], empty_raw[kRawStages], full_b[kBStages], empty_b[kBStages];
    __shared__ uint64_t full_d[2], empty_d[2], mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = p.L, N = L * L;

    // ---- set-up: rings, barriers, tensor memory, the DFT matrix A
    for (int i = tid; i < kBStages * kBStage / 16; i += kThreadsTC)
        reinterpret_cast<uint4 *>(bring)[i] = make_uint4(0u, 0u, 0u, 0u);   // rows y >= L stay zero
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < kRawStages; ++i) {
            gc_mbar_init(&full_raw[i], 1);
            gc_mbar_init(&empty_raw[i], kConvWarps);
        }
        for (int i = 0; i < kBStages; ++i) {
            gc_mbar_init(&full_b[i], kConvWarps);
            gc_mbar_init(&empty_b[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            gc_mbar_init(&full_d[i], 1);
            gc_mbar_init(&empty_d[i], kEpiWarps);
        }
        gc_mbar_init(&mma_done, 1);
        gc_fence_mbar_init();
    }
    for (int i = tid; i < 2 * 2 * 32; i += kThreadsTC) {
        const int pr = i >> 6, r = (i >> 5) & 1, y = i & 31;
        const cf w = c_tw.v[(2 * (pr + 2 * r) * y) & 255];
        tws[i] = make_float2(w.x, w.y);
    }
    if (warp == 0) gc_tmem_alloc(&tmem_slot, 512);
    gc_tc_fence_before();
    __syncthreads();
    gc_tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (warp < 4) {
        // A row k_x = lane of this warp's quarter: K = 2j, 2j + 1 in column j
        const int kx = 32 * warp + lane;
        const uint32_t lb = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                float v[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 2 * (16 * q + j) + h;
                    const int x = k & 63;
                    const cf w = c_tw.v[2 * ((kx * x) & 127)];   // (cos, -sin) of 2 pi k_x x / 128
                    v[h] = k < 64 ? w.x : -w.y;
                }
                split2(v[0], v[1], hi[j], lo[j]);
            }
            gc_tmem_st16(lb + kColAHi + 16 * q, hi);
            gc_tmem_st16(lb + kColALo + 16 * q, lo);
        }
        gc_tmem_wait_st();
    }
    gc_fence_proxy_async();
    gc_tc_fence_before();
    __syncthreads();
    gc_tc_fence_after();
    bool ok = true;

    if (warp == kWarpTma) {
        // ---------------------------------------------------------------- bulk copies of raw samples
        if (lane == 0) {
            uint32_t rs = 0, rph = 0;
            int last_round[kRawStages];
            for (int i = 0; i < kRawStages; ++i) last_round[i] = -1;
            int round = 0;
            for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
                const ItemTC it = decode_tc(p, item);
                for (int s = 0; s < it.nt; s += kSamp) {
                    if (!gc_mbar_wait_abort(&empty_raw[rs], rph ^ 1u, &s_abort, GC_WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    const int ns = min(kSamp, it.nt - s);
                    const uint32_t bytes = (uint32_t)(ns * N);
                    gc_mbar_expect_tx(&full_raw[rs], bytes);
                    gc_bulk_load(raw + (size_t)rs * kRawStride,
                                 p.volt + ((size_t)it.c * p.T + it.t0 + s) * (size_t)N, bytes, &full_raw[rs]);
                    last_round[rs] = round;
                    if (++rs == kRawStages) {
                        rs = 0;
                        rph ^= 1u;
                        ++round;
                    }
                }
            }
            if (!ok) {
                s_abort = 1;
                atomicOr(p.status, GC_DEV_TIMEOUT_FFT);
            }
            // no copy may still be landing when the CTA exits
            for (int i = 0; i < kRawStages; ++i)
                if (last_round[i] >= 0)
                    gc_mbar_wait(&full_raw[i], (uint32_t)(last_round[i] & 1), GC_WAIT_LIMIT_NS / 10);
        }
        __syncwarp();
    } else if (warp == kWarpMma) {
        // ---------------------------------------------------------------- MMA issue
        if (lane == 0) {
            const uint32_t idesc = gc_tc_idesc(128, kTL, false, false);
            const uint32_t bbase = gc_smem_addr(bring);
            uint32_t bs = 0, bph = 0, db = 0, dph = 0;
            for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
                const ItemTC it = decode_tc(p, item);
                for (int s = 0; s < it.nt && ok; s += kSamp) {
                    if (!gc_mbar_wait_abort(&full_b[bs], bph, &s_abort, GC_WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    const int ns = min(kSamp, it.nt - s);
                    for (int j = 0; j < ns; ++j) {
                        if (!gc_mbar_wait_abort(&empty_d[db], dph ^ 1u, &s_abort, GC_WAIT_LIMIT_NS)) {
                            ok = false;
                            break;
                        }
                        gc_tc_fence_after();
                        const uint32_t dre = tmem + kColD + 128 * db, dim = dre + 64;
                        const uint32_t b0 = bbase + (uint32_t)(bs * kBStage + j * kBSample);
#pragma unroll 1
                        for (int term = 0; term < 3; ++term) {
                            const uint32_t a = tmem + (term == 2 ? kColALo : kColAHi);
                            const uint32_t b = b0 + (term == 1 ? (uint32_t)kBPlane : 0u);
#pragma unroll
                            for (int k = 0; k < 8; ++k)
                                gc_tc_mma_f16_ts(dre, a + 8 * k, gc_tc_sdesc(b + 256 * k, kLBO, kSBO), idesc,
                                                 (term | k) != 0);
                            // Im: C with Im w, then -S with Re w
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                gc_tc_mma_f16_ts(dim, a + 8 * k, gc_tc_sdesc(b + 256 * (k + 4), kLBO, kSBO), idesc,
                                                 (term | k) != 0);
#pragma unroll
                            for (int k = 4; k < 8; ++k)
                                gc_tc_mma_f16_ts(dim, a + 8 * k, gc_tc_sdesc(b + 256 * (k - 4), kLBO, kSBO),
                                                 idesc | GC_TC_NEGATE_A, 1u);
                        }
                        gc_tc_commit(&full_d[db]);
                        if (++db == 2) {
                            db = 0;
                            dph ^= 1u;
                        }
                    }
                    gc_tc_commit(&empty_b[bs]);
                    if (++bs == kBStages) {
                        bs = 0;
                        bph ^= 1u;
                    }
                }
            }
            if (!ok) {
                s_abort = 1;
                atomicOr(p.status, GC_DEV_TIMEOUT_FFT);
            }
            // every MMA issued has completed before tensor memory is released
            gc_tc_commit(&mma_done);
            gc_mbar_wait(&mma_done, 0, GC_WAIT_LIMIT_NS / 10);
        }
        __syncwarp();
    } else if (warp >= kWarpConv0) {
        // ---------------------------------------------------------------- converters
        // task i of this thread: row y = 8 i + ((kg + g) & 7), inputs 8 kg ..
        // 8 kg + 7, with kg = lane & 7 and g = lane / 8 + 4 (converter warp):
        // the 8 lanes of a group write 8 different rows of a core-matrix
        // column, so the 16-byte operand stores are free of bank conflicts
        const int ct = tid - 32 * kWarpConv0;
        const int kg = ct & 7;
        const int ylo = (kg + ((ct & 31) >> 3) + 4 * (ct >> 5)) & 7;
        uint32_t rs = 0, rph = 0, bs = 0, bph = 0;
        for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
            const ItemTC it = decode_tc(p, item);
            // calibration coefficients 1/g = conj(g) / |g|^2 of this thread's
            // antennas, in shared memory that only this thread reads
#pragma unroll 1
            for (int i = 0; i < kTasks; ++i) {
                const int y = 8 * i + ylo;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int x = 8 * kg + e;
                    float2 cc = make_float2(0.f, 0.f);
                    if (x < L && y < L) {
                        const float2 gg = p.gains[(size_t)it.c * N + y * L + x];
                        const float d = gg.x * gg.x + gg.y * gg.y;
                        if (d > 0.f && isfinite(d)) cc = make_float2(gg.x / d, -gg.y / d);
                        else atomicOr(p.status, GC_DEV_BADINPUT);   // w = v / g undefined: antenna left out
                    }
                    coef[(i * 8 + e) * kConvThreads + ct] = cc;
                }
            }
            for (int s = 0; s < it.nt; s += kSamp) {
                if (!gc_mbar_wait_abort(&full_raw[rs], rph, &s_abort, GC_WAIT_LIMIT_NS)) ok = false;
                if (ok && !gc_mbar_wait_abort(&empty_b[bs], bph ^ 1u, &s_abort, GC_WAIT_LIMIT_NS)) ok = false;
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const int ns = min(kSamp, it.nt - s);
                for (int j = 0; j < ns; ++j) {
                    const unsigned char *rb = raw + (size_t)rs * kRawStride + (size_t)j * N;
                    unsigned char *bhi = bring + (size_t)bs * kBStage + (size_t)j * kBSample, *blo = bhi + kBPlane;
#pragma unroll 2
                    for (int i = 0; i < kTasks; ++i) {
                        const int y = 8 * i + ylo;
                        if (y >= L) continue;
                        const uint2 word = *reinterpret_cast<const uint2 *>(rb + y * L + 8 * kg);
                        // n + 8 of the Re and Im nibbles, one byte each
                        const uint32_t ure0 = ((word.x >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
                        const uint32_t ure1 = ((word.y >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
                        const uint32_t uim0 = (word.x & 0x0F0F0F0Fu) ^ 0x08080808u;
                        const uint32_t uim1 = (word.y & 0x0F0F0F0Fu) ^ 0x08080808u;
                        uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            float2 w[2];
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int ee = e + h;
                                const float2 v = i4c_bytes_to_f2(ee < 4 ? ure0 : ure1, ee < 4 ? uim0 : uim1, ee & 3);
                                w[h] = cmul(v, coef[(i * 8 + ee) * kConvThreads + ct]);
                            }
                            split2(w[0].x, w[1].x, rh[e >> 1], rl[e >> 1]);
                            split2(w[0].y, w[1].y, ih[e >> 1], il[e >> 1]);
                        }
                        // B[n = y][k]: Re at k = 8 kg .., Im at k = 64 + 8 kg ..
                        const int off = (y >> 3) * (int)kSBO + (y & 7) * 16;
                        *reinterpret_cast<uint4 *>(bhi + off + kg * (int)kLBO) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                        *reinterpret_cast<uint4 *>(bhi + off + (8 + kg) * (int)kLBO) =
                            make_uint4(ih[0], ih[1], ih[2], ih[3]);
                        *reinterpret_cast<uint4 *>(blo + off + kg * (int)kLBO) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                        *reinterpret_cast<uint4 *>(blo + off + (8 + kg) * (int)kLBO) =
                            make_uint4(il[0], il[1], il[2], il[3]);
                    }
                }
                gc_fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    gc_mbar_arrive(&full_b[bs]);
                    gc_mbar_arrive(&empty_raw[rs]);
                }
                if (++rs == kRawStages) {
                    rs = 0;
                    rph ^= 1u;
                }
                if (++bs == kBStages) {
                    bs = 0;
                    bph ^= 1u;
                }
            }
        }
        if (!ok) {
            s_abort = 1;
            if (lane == 0) atomicOr(p.status, GC_DEV_TIMEOUT_FFT);
        }
    } else {
        // ---------------------------------------------------------------- column stage (warps 0-7)
        const int lq = warp & 3, pr = warp >> 2;
        const int kx = 32 * lq + lane;
        const uint32_t lb = tmem + ((uint32_t)(32 * lq) << 16);
        const uint32_t pa = lb + kColP + 32 * pr, pb = lb + kColP + 32 * (pr + 2);
        uint32_t db = 0, dph = 0;
        for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
            const ItemTC it = decode_tc(p, item);
            for (int s = 0; s < it.nt; ++s) {
                if (!gc_mbar_wait_abort(&full_d[db], dph, &s_abort, GC_WAIT_LIMIT_NS)) ok = false;
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                gc_tc_fence_after();
                const uint32_t dre = lb + kColD + 128 * db, dim = dre + 64;
                const bool first = s == 0;
                column_pair(dre, dim, pa, pb, first, pr, tws + 64 * pr);
                gc_tc_fence_before();
                __syncwarp();
                if (lane == 0) gc_mbar_arrive(&empty_d[db]);
                if (++db == 2) {
                    db = 0;
                    dph ^= 1u;
                }
            }
            if (!ok) break;
            // chunk spectrum P[k_y][k_x], k_y = s2 + 4 bitrev(i)
            gc_tmem_wait_st();
            float *out = p.ppart + ((size_t)it.c * p.n_chunks + it.chunk) * kTM * kTM;
#pragma unroll 1
            for (int r = 0; r < 2; ++r) {
                const int s2 = pr + 2 * r;
                uint32_t pv[32];
                gc_tmem_ld32_nowait(lb + kColP + 32 * s2, pv);
                gc_tmem_wait_ld_regs(pv);
#pragma unroll
                for (int i = 0; i < 32; ++i) out[(s2 + 4 * bitrev<32>(i)) * kTM + kx] = __uint_as_float(pv[i]);
            }
        }
        if (!ok) {
            s_abort = 1;
            if (lane == 0) atomicOr(p.status, GC_DEV_TIMEOUT_FFT);
        }
    }

    gc_tc_fence_before();
    __syncthreads();
    gc_tc_fence_after();
    if (warp == 0) gc_tmem_dealloc(tmem, 512);
}

}  // namespace

bool gc_fft_tc_eligible(const gc_ctx *ctx, int vfmt, int L, const void *volt, bool masked) {
    return ctx->tune[GC_TUNE_FFT_PATH] != 1 && vfmt == GC_I4C && !masked && L > 32 && L <= kTL && L % 8 == 0 &&
           gc_aligned(volt, 16);
}

// Chunk spectra of one launch: ppart [C][n_chunks][128][128] in the context
// workspace (returned with n_chunks for fftcorr_finalize).
gc_status gc_fft_tc_run(gc_ctx *ctx, const void *volt, int L, int C, int T, const float *gains, float **ppart,
                        int *n_chunks, cudaStream_t stream) {
    cudaError_t e = cudaFuncSetAttribute(fftcorr_tc_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemTC);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaFuncSetAttribute(fftcorr_tc_accumulate)");
    const int slots = ctx->sm_count;   // one CTA per SM (all 512 tensor-memory columns)
    // time chunks (even lengths) chosen so that the items fill whole waves
    int best_n = 1, best_len = (T + kRawSamp - 1) / kRawSamp * kRawSamp;
    double best_eff = -1.0;
    const int n_min = std::max(1, (T + 2047) / 2048);
    for (int n = n_min; n <= n_min + 64; ++n) {
        const int len = ((T + n - 1) / n + kRawSamp - 1) / kRawSamp * kRawSamp;
        const int nn = (T + len - 1) / len;
        const long items = (long)C * nn;
        const long waves = (items + slots - 1) / slots;
        const double eff = (double)C * T / ((double)waves * slots * len);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best_n = nn;
            best_len = len;
        }
    }
    if (ctx->tune[GC_TUNE_FFT_CHUNK] > 0) {
        best_len = (std::min(ctx->tune[GC_TUNE_FFT_CHUNK], 8192) + kRawSamp - 1) / kRawSamp * kRawSamp;
        best_n = (T + best_len - 1) / best_len;
    }
    TcFftParams p;
    p.volt = static_cast<const unsigned char *>(volt);
    p.gains = reinterpret_cast<const float2 *>(gains);
    p.status = ctx->status_dev;
    p.L = L;
    p.C = C;
    p.T = T;
    p.chunk_len = best_len;
    p.n_chunks = best_n;
    p.n_items = C * best_n;
    const size_t part_bytes = ((size_t)C * best_n * kTM * kTM * sizeof(float) + 255) / 256 * 256;
    gc_status st = gc_scratch_reserve(ctx, part_bytes);
    if (st != GC_OK) return st;
    p.ppart = static_cast<float *>(ctx->scratch);
    const int grid = std::min(p.n_items, slots);
    int rec = gc_prof_begin(ctx, stream, "fftcorr_tc_accumulate");
    fftcorr_tc_accumulate<<<grid, kThreadsTC, kSmemTC, stream>>>(p);
    gc_prof_end(ctx, stream, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch fftcorr_tc_accumulate");
    *ppart = p.ppart;
    *n_chunks = best_n;
    return GC_OK;
}
