// Reduced X-engine on the tensor cores (paper Fig. 1, calibrator step (a)),
// for 4+4-bit voltages and selections whose types share one integration
// window (subset calibration, Sec. 5).
//
// The pairs of a subset selection join every antenna to its neighbours at a
// handful of short separations d = (dx, dy), dy >= 0.  A block of 128
// consecutive antennas (own antennas j, whole grid rows) and the H antennas
// from its first row up to dy_max rows past its last (the halo, containing
// every partner i = j + d) are correlated densely on the tensor cores:
//   D[j][i] = sum_t v_j(t) conj(v_i(t))       (128 x H complex sums)
// and each type's pairs are the diagonal i - j = dy L + dx of D.
//
// Exact integer arithmetic through FP8: a 4-bit two's-complement nibble n in
// [-8, 7] gives u = n + 8 in [0, 15] by flipping its top bit, and the byte u
// (exponent field 000u3, mantissa u2u1u0) is the e4m3 code of u * 2^-9 --
// subnormal for u < 8, normal above.  So the raw nibble XOR 8, in a byte of its
// own, is an exact e4m3 operand with no table and no conversion.  The MMA
// (kind::f8f6f4, FP32 accumulator) sums products u_a u_b 2^-18; every partial
// sum is an integer multiple of 2^-18 below 2^24 of them (|sum| <= 450 per
// sample: windows up to 32768 samples), so FP32 holds it exactly.  With
// U_a = sum_t u_a (per part and antenna) the integer sums follow exactly:
//   Re = D1 - 8 (Ure_a + Uim_a + Ure_b + Uim_b) + 128 t_w
//   Im = D2 - 8 (Uim_a - Ure_a) - 8 (Ure_b - Uim_b)
// for D1 = sum (ure_a ure_b + uim_a uim_b), D2 = sum (uim_a ure_b - ure_a uim_b),
// a = own antenna, b = partner, t_w = samples in the window.
//
// Operands need no transpose: the voltages are [t][antenna] bytes, which is
// the MN-major operand layout (antennas contiguous, K = time strided).  Each
// 32-sample stage holds an RE and an IM plane of the halo (e4m3 codes);
// four MMAs (M = 128, N = H, K = 32) per stage:
//   D1 += RE.RE + IM.IM,   D2 += IM.RE - RE.IM (negate-A bit)
// where the A operand is the first 128 antennas of the same plane (the own
// rows are the first rows of the halo).  D1 and D2 stay in tensor memory
// (2 x 256 of the 512 columns) over the whole window.
//
// Warp roles (one CTA per SM, persistent over (channel, block, time slice)
// items): warp 4 issues 2-D TMA copies of the raw halo rows (32 samples per
// stage, row pitch padded by 16 bytes so that the converters' 16-byte reads
// are conflict-free) into a ring; warps 0-3 turn raw stages into operand
// planes (two LOP3 per 4 bytes), accumulate the per-antenna sums U in
// byte-parallel registers, and after the last stage read the diagonals out of
// tensor memory (the epilogue: tensor-memory lane = own antenna); warp 5
// issues the MMAs and commits their completion to the operand ring and the
// accumulator barrier.  Every wait is bounded (GC_DEV_TIMEOUT_XENG).
#include <algorithm>

#include "gc_sel.h"
#include "gc_tcgen05.h"

namespace {

constexpr int kH = 256;          // halo antennas = MMA N
constexpr int kST = 32;          // samples per stage (K of one MMA)
constexpr int kMaxTypes = 16;
constexpr int kNSeg = kH / 16;   // 16-antenna segments of the halo
constexpr int kRawPitch = kH + 16;
constexpr int kRawBytes = kST * kRawPitch;        // 8704 (68 x 128)
constexpr int kPlane = kST * kH;                  // one operand plane
constexpr int kOpBytes = 2 * kPlane;              // RE plane, IM plane
constexpr uint32_t kLBO = 128;                    // K-group stride: 8 samples x 16 bytes
constexpr uint32_t kSBO = 512;                    // MN-group stride: 16 antennas x 32 samples
constexpr int kTilePitch = 36;                    // words per row of the epilogue tile
constexpr int kTileWords = 2 * 32 * kTilePitch;   // D1 and D2 tiles of one warp
constexpr int kSliceMax = 32768;                  // samples per item (exact FP32 sums)

// Launch shape: CW converter warps (4 or 8; warps 0-3 also read tensor memory
// back), then a TMA warp and an MMA warp; RS raw and OS operand stages.
template <int CW, int RS, int OS>
struct TcShape {
    static constexpr int kConvWarps = CW, kRawStages = RS, kOpStages = OS;
    static constexpr int kThreads = 32 * (CW + 2);
    static constexpr int kOStep = CW / 4;        // stride between a thread's 8-sample groups
    static constexpr int kParts = CW / 4;        // partial per-antenna sums (one per octet phase)
    static constexpr size_t kSmemOp = 0;
    static constexpr size_t kSmemRaw = kSmemOp + (size_t)OS * kOpBytes;
    static constexpr size_t kSmemTile = kSmemRaw + (size_t)RS * kRawBytes;
    static constexpr size_t kSmemU = kSmemTile + (size_t)4 * kTileWords * 4;
    static constexpr size_t kSmemBytes = kSmemU + (size_t)kParts * 2 * kH * 4;
};

struct TcParams {
    int L, N, C, T;
    int n_blk;        // blocks of 128 own antennas per channel
    int n_tsplit;     // time slices of the window
    int w0, w1;       // the integration window
    int n_items;
    int ntypes;
    int P;
    const int32_t *types, *type_ptr;
    int2 *part;       // [n_tsplit][C][P]
    int *apart;       // [n_tsplit][C][N] or null
    unsigned int *status;
};

struct Item {
    int blk, c, ts, ta, tb, nst;
};

__device__ __forceinline__ Item decode(const TcParams &p, int item) {
    Item it;
    it.blk = item % p.n_blk;
    it.c = (item / p.n_blk) % p.C;
    it.ts = item / (p.n_blk * p.C);
    const int len = (p.w1 - p.w0 + p.n_tsplit - 1) / p.n_tsplit;
    it.ta = min(p.w1, p.w0 + it.ts * len);
    it.tb = min(p.w1, it.ta + len);
    it.nst = (it.tb - it.ta + kST - 1) / kST;
    return it;
}

__device__ __forceinline__ void conv_sync(uint64_t *bar, uint32_t &phase, volatile int *abort, bool &ok) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) gc_mbar_arrive(bar);
    if (!gc_mbar_wait_abort(bar, phase, abort, GC_WAIT_LIMIT_NS)) ok = false;
    phase ^= 1u;
    ok = __all_sync(0xffffffffu, ok);
}

template <class S>
__global__ void __launch_bounds__(S::kThreads, 1)
xeng_tc_accumulate(const __grid_constant__ CUtensorMap tmap, const TcParams p) {
    constexpr int kRawStages = S::kRawStages, kOpStages = S::kOpStages, CW = S::kConvWarps;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *op = smem + S::kSmemOp;
    unsigned char *raw = smem + S::kSmemRaw;
    uint32_t *tiles = reinterpret_cast<uint32_t *>(smem + S::kSmemTile);
    int *usum = reinterpret_cast<int *>(smem + S::kSmemU);   // [parts][re, im][kH]
    __shared__ uint64_t full_raw[kRawStages], empty_raw[kRawStages], full_op[kOpStages], empty_op[kOpStages];
    __shared__ uint64_t acc_full, acc_empty, conv_bar, mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_dx[kMaxTypes], s_dy[kMaxTypes], s_off[kMaxTypes], s_base[kMaxTypes];
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = p.L;
    if (tid < p.ntypes) {
        s_dx[tid] = p.types[2 * tid];
        s_dy[tid] = p.types[2 * tid + 1];
        s_off[tid] = s_dy[tid] * L + s_dx[tid];
        s_base[tid] = p.type_ptr[tid];
    }
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < kRawStages; ++i) {
            gc_mbar_init(&full_raw[i], 1);
            gc_mbar_init(&empty_raw[i], CW);
        }
        for (int i = 0; i < kOpStages; ++i) {
            gc_mbar_init(&full_op[i], CW);
            gc_mbar_init(&empty_op[i], 1);
        }
        gc_mbar_init(&acc_full, 1);
        gc_mbar_init(&acc_empty, 4);
        gc_mbar_init(&conv_bar, CW);
        gc_mbar_init(&mma_done, 1);
        gc_fence_mbar_init();
    }
    if (warp == 0) gc_tmem_alloc(&tmem_slot, 512);
    gc_tc_fence_before();
    __syncthreads();
    gc_tc_fence_after();
    const uint32_t tmem = tmem_slot;
    bool ok = true;

    if (warp == CW) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            uint32_t rs = 0, rph = 0;
            int last_round[kRawStages];
            for (int i = 0; i < kRawStages; ++i) last_round[i] = -1;
            int round = 0;
            for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
                const Item it = decode(p, item);
                for (int s = 0; s < it.nst; ++s) {
                    if (!gc_mbar_wait_abort(&empty_raw[rs], rph ^ 1u, &s_abort, GC_WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    gc_mbar_expect_tx(&full_raw[rs], (uint32_t)kRawBytes);
                    gc_tma_load_2d(raw + (size_t)rs * kRawBytes, &tmap, &full_raw[rs], it.blk * 32,
                                   it.c * p.T + it.ta + s * kST);
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
                atomicOr(p.status, GC_DEV_TIMEOUT_XENG);
            }
            // no copy may still be landing when the CTA exits
            for (int i = 0; i < kRawStages; ++i)
                if (last_round[i] >= 0)
                    gc_mbar_wait(&full_raw[i], (uint32_t)(last_round[i] & 1), GC_WAIT_LIMIT_NS / 10);
        }
        __syncwarp();
    } else if (warp == CW + 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = gc_tc_idesc(128, kH, true, true);
            uint32_t os = 0, oph = 0, aph = 0;
            bool first = true;
            for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
                const Item it = decode(p, item);
                if (it.nst == 0) continue;
                if (!first) {
                    if (!gc_mbar_wait_abort(&acc_empty, aph, &s_abort, GC_WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    aph ^= 1u;
                }
                first = false;
                gc_tc_fence_after();
                for (int s = 0; s < it.nst; ++s) {
                    if (!gc_mbar_wait_abort(&full_op[os], oph, &s_abort, GC_WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    gc_tc_fence_after();
                    const uint32_t base = gc_smem_addr(op + (size_t)os * kOpBytes);
                    const uint64_t re = gc_tc_sdesc(base, kLBO, kSBO), im = gc_tc_sdesc(base + kPlane, kLBO, kSBO);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    gc_tc_mma_f8(tmem, re, re, idesc, acc);
                    gc_tc_mma_f8(tmem, im, im, idesc, 1u);
                    gc_tc_mma_f8(tmem + 256, im, re, idesc, acc);
                    gc_tc_mma_f8(tmem + 256, re, im, idesc | GC_TC_NEGATE_A, 1u);
                    gc_tc_commit(&empty_op[os]);
                    if (++os == kOpStages) {
                        os = 0;
                        oph ^= 1u;
                    }
                }
                if (!ok) break;
                gc_tc_commit(&acc_full);
            }
            if (!ok) {
                s_abort = 1;
                atomicOr(p.status, GC_DEV_TIMEOUT_XENG);
            }
            // every MMA issued has completed before tensor memory is released
            gc_tc_commit(&mma_done);
            gc_mbar_wait(&mma_done, 0, GC_WAIT_LIMIT_NS / 10);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- converters + epilogue
        const int rl = tid & 7;              // sample within an 8-sample group
        const int g = (tid >> 3) % kNSeg;    // 16-antenna segment of the halo
        const int o0 = tid >> 7;             // first 8-sample group of the stage (octet phase)
        uint32_t rs = 0, rph = 0, os = 0, oph = 0, afph = 0, cph = 0;
        uint32_t *tile1 = tiles + warp * kTileWords, *tile2 = tile1 + 32 * kTilePitch;
        for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
            const Item it = decode(p, item);
            uint32_t a8re[4] = {0u, 0u, 0u, 0u}, a8im[4] = {0u, 0u, 0u, 0u};
            uint32_t a16re[8], a16im[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a16re[i] = a16im[i] = 0u;
            auto flush = [&]() {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    a16re[2 * i] += __byte_perm(a8re[i], 0u, 0x4240);
                    a16re[2 * i + 1] += __byte_perm(a8re[i], 0u, 0x4341);
                    a16im[2 * i] += __byte_perm(a8im[i], 0u, 0x4240);
                    a16im[2 * i + 1] += __byte_perm(a8im[i], 0u, 0x4341);
                    a8re[i] = 0u;
                    a8im[i] = 0u;
                }
            };
            for (int s = 0; s < it.nst; ++s) {
                if (!gc_mbar_wait_abort(&full_raw[rs], rph, &s_abort, GC_WAIT_LIMIT_NS)) ok = false;
                if (ok && !gc_mbar_wait_abort(&empty_op[os], oph ^ 1u, &s_abort, GC_WAIT_LIMIT_NS)) ok = false;
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const unsigned char *rb = raw + (size_t)rs * kRawBytes;
                unsigned char *ob = op + (size_t)os * kOpBytes;
                const int t0 = it.ta + s * kST;
#pragma unroll
                for (int oo = 0; oo < 4; oo += S::kOStep) {
                    const int o = oo + o0;
                    const int r = 8 * o + rl;
                    uint4 X = *reinterpret_cast<const uint4 *>(rb + r * kRawPitch + 16 * g);
                    // samples past the slice: raw 0x88 gives code 0 in both parts
                    if (t0 + r >= it.tb) X = make_uint4(0x88888888u, 0x88888888u, 0x88888888u, 0x88888888u);
                    uint4 re, im;
                    im.x = (X.x & 0x0F0F0F0Fu) ^ 0x08080808u;
                    im.y = (X.y & 0x0F0F0F0Fu) ^ 0x08080808u;
                    im.z = (X.z & 0x0F0F0F0Fu) ^ 0x08080808u;
                    im.w = (X.w & 0x0F0F0F0Fu) ^ 0x08080808u;
                    re.x = ((X.x >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
                    re.y = ((X.y >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
                    re.z = ((X.z >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
                    re.w = ((X.w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
                    a8re[0] += re.x;
                    a8re[1] += re.y;
                    a8re[2] += re.z;
                    a8re[3] += re.w;
                    a8im[0] += im.x;
                    a8im[1] += im.y;
                    a8im[2] += im.z;
                    a8im[3] += im.w;
                    unsigned char *dst = ob + o * kLBO + g * kSBO + rl * 16;
                    *reinterpret_cast<uint4 *>(dst) = re;
                    *reinterpret_cast<uint4 *>(dst + kPlane) = im;
                }
                gc_fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    gc_mbar_arrive(&full_op[os]);
                    gc_mbar_arrive(&empty_raw[rs]);
                }
                if (++rs == kRawStages) {
                    rs = 0;
                    rph ^= 1u;
                }
                if (++os == kOpStages) {
                    os = 0;
                    oph ^= 1u;
                }
                // byte sums hold 16 samples of codes <= 15 (4 / kOStep per stage)
                if ((s & (4 * S::kOStep - 1)) == 4 * S::kOStep - 1) flush();
            }
            if (!ok) break;
            flush();
            // per-antenna sums of the halo over the slice: the 8 threads of a
            // segment are lanes 8k..8k+7 of one warp
            {
                int sre[16], sim[16];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    sre[4 * i + 0] = (int)(a16re[2 * i] & 0xFFFFu);
                    sre[4 * i + 2] = (int)(a16re[2 * i] >> 16);
                    sre[4 * i + 1] = (int)(a16re[2 * i + 1] & 0xFFFFu);
                    sre[4 * i + 3] = (int)(a16re[2 * i + 1] >> 16);
                    sim[4 * i + 0] = (int)(a16im[2 * i] & 0xFFFFu);
                    sim[4 * i + 2] = (int)(a16im[2 * i] >> 16);
                    sim[4 * i + 1] = (int)(a16im[2 * i + 1] & 0xFFFFu);
                    sim[4 * i + 3] = (int)(a16im[2 * i + 1] >> 16);
                }
#pragma unroll
                for (int m = 1; m < 8; m <<= 1) {
#pragma unroll
                    for (int a = 0; a < 16; ++a) {
                        sre[a] += __shfl_xor_sync(0xffffffffu, sre[a], m);
                        sim[a] += __shfl_xor_sync(0xffffffffu, sim[a], m);
                    }
                }
                // lane rl stores antennas 2 rl, 2 rl + 1 of the segment (partial o0)
                int *up = usum + o0 * 2 * kH;
#pragma unroll
                for (int a = 0; a < 16; ++a) {
                    if ((a >> 1) == rl) {
                        up[16 * g + a] = sre[a];
                        up[kH + 16 * g + a] = sim[a];
                    }
                }
            }
            conv_sync(&conv_bar, cph, &s_abort, ok);
            if (!ok) break;
            if (warp >= 4) {   // extra converter warps: no tensor-memory lanes of their own
                conv_sync(&conv_bar, cph, &s_abort, ok);
                continue;
            }
            auto usum_at = [&](int part, int a) {
                int v = usum[part * kH + a];
#pragma unroll
                for (int q = 1; q < S::kParts; ++q) v += usum[q * 2 * kH + part * kH + a];
                return v;
            };
            // ---- epilogue: lane l of tensor memory = own antenna blk * 128 + l
            const int l = tid;
            const int j = it.blk * 128 + l;
            const int x = j % L, y = j / L;
            const int ure_l = usum_at(0, l), uim_l = usum_at(1, l);
            uint32_t d1[kMaxTypes], d2[kMaxTypes], dauto = 0u;
#pragma unroll
            for (int k = 0; k < kMaxTypes; ++k) d1[k] = d2[k] = 0u;
            if (it.nst > 0) {
                if (!gc_mbar_wait_abort(&acc_full, afph, &s_abort, GC_WAIT_LIMIT_NS)) ok = false;
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                afph ^= 1u;
                gc_tc_fence_after();
                const uint32_t lanebase = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
                for (int q = 0; q < kH / 32; ++q) {
                    uint32_t r[32];
                    gc_tmem_ld32(lanebase + 32 * q, r);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        *reinterpret_cast<uint4 *>(tile1 + lane * kTilePitch + 4 * i) =
                            make_uint4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
                    gc_tmem_ld32(lanebase + 256 + 32 * q, r);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        *reinterpret_cast<uint4 *>(tile2 + lane * kTilePitch + 4 * i) =
                            make_uint4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < kMaxTypes; ++k) {
                        if (k < p.ntypes) {
                            const int col = l + s_off[k];
                            if ((col >> 5) == q) {
                                d1[k] = tile1[lane * kTilePitch + (col & 31)];
                                d2[k] = tile2[lane * kTilePitch + (col & 31)];
                            }
                        }
                    }
                    if (q == warp) dauto = tile1[lane * kTilePitch + lane];
                    __syncwarp();
                }
                gc_tc_fence_before();
                __syncwarp();
                if (lane == 0) gc_mbar_arrive(&acc_empty);   // tensor memory free for the next item
            }
            const int tw = it.tb - it.ta;
            int2 *out = p.part + ((size_t)it.ts * p.C + it.c) * p.P;
#pragma unroll
            for (int k = 0; k < kMaxTypes; ++k) {
                if (k < p.ntypes) {
                    const int dx = s_dx[k], dy = s_dy[k];
                    const int xi = x + dx, yi = y + dy;
                    if (xi >= 0 && xi < L && yi < L) {
                        const int col = l + s_off[k];
                        const int ure_c = usum_at(0, col), uim_c = usum_at(1, col);
                        const int s1 = __float2int_rn(__uint_as_float(d1[k]) * 262144.0f);
                        const int s2 = __float2int_rn(__uint_as_float(d2[k]) * 262144.0f);
                        const int re = s1 - 8 * (ure_l + uim_l + ure_c + uim_c) + 128 * tw;
                        const int imd = s2 - 8 * (uim_l - ure_l) - 8 * (ure_c - uim_c);
                        const int o = s_base[k] + y * (L - abs(dx)) + (x - max(0, -dx));
                        out[o] = make_int2(re, -imd);   // S_p = conj(sum v_j conj v_i)
                    }
                }
            }
            if (p.apart) {
                const int sa = __float2int_rn(__uint_as_float(dauto) * 262144.0f);
                p.apart[((size_t)it.ts * p.C + it.c) * p.N + j] = sa - 16 * (ure_l + uim_l) + 128 * tw;
            }
            // the sums and tiles are rewritten by the next item
            conv_sync(&conv_bar, cph, &s_abort, ok);
        }
        if (!ok) {
            s_abort = 1;
            if (lane == 0) atomicOr(p.status, GC_DEV_TIMEOUT_XENG);
        }
    }
    gc_tc_fence_before();
    __syncthreads();
    if (warp == 0) gc_tmem_dealloc(tmem, 512);
}

}  // namespace

// Whether the tensor-core X-engine covers this call: 4+4-bit voltages, an
// unmasked selection with one integration window and at most 16 types, a grid
// whose blocks of 128 antennas are whole rows (L = 16, 32 or 64), a halo of at
// most 256 antennas (128 + dy_max L), and a 16-byte aligned buffer for TMA.
bool gc_xeng_tc_eligible(const gc_sel *sel, int vfmt, const void *volt, int L) {
    if (vfmt != GC_I4C || sel->masked || sel->n_windows != 1 || sel->n_ubl > kMaxTypes || sel->n_ubl < 1) return false;
    if (L != 16 && L != 32 && L != 64) return false;
    if (!gc_aligned(volt, 16)) return false;
    int dymax = 0;
    for (int k = 0; k < sel->n_ubl; ++k) {
        if (sel->types[2 * k + 1] < 0) return false;
        dymax = std::max(dymax, sel->types[2 * k + 1]);
    }
    return 128 + dymax * L <= kH;
}

int gc_xeng_tc_slices(const gc_ctx *ctx, const gc_sel *sel, int L, int C) {
    const long items = (long)C * (L * L / 128);
    const int w = sel->grp_t1[0] - sel->grp_t0[0];
    const int min_ts = (w + kSliceMax - 1) / kSliceMax;
    int best_ts = std::max(1, min_ts);
    double best = -1.0;
    for (int ts = best_ts; ts <= 64; ++ts) {
        if (ts > best_ts && w / ts < 256) break;
        const long n = items * ts;
        const long waves = (n + ctx->sm_count - 1) / ctx->sm_count;
        const double eff = (double)n / ((double)waves * ctx->sm_count) - 0.01 * ts;
        if (eff > best) {
            best = eff;
            best_ts = ts;
        }
    }
    return best_ts;
}

template <class S>
gc_status tc_launch(gc_ctx *ctx, const CUtensorMap &tmap, const TcParams &p, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(xeng_tc_accumulate<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::kSmemBytes);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaFuncSetAttribute(xeng_tc_accumulate)");
    const int grid = std::min(p.n_items, ctx->sm_count);
    int rec = gc_prof_begin(ctx, s, "xeng_tc_accumulate");
    xeng_tc_accumulate<S><<<grid, S::kThreads, S::kSmemBytes, s>>>(tmap, p);
    gc_prof_end(ctx, s, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch xeng_tc_accumulate");
    return GC_OK;
}

gc_status gc_xeng_tc_launch(gc_ctx *ctx, const void *volt, int L, int C, int T, const gc_sel *sel, void *part,
                            void *apart, int n_tsplit, cudaStream_t s) {
    const int N = L * L;
    CUtensorMap tmap;
    // the voltages as a 2-D array of 32-bit words: N / 4 per sample row, C T rows;
    // a box is the halo (kH bytes) plus 16 bytes of row padding, 32 samples deep
    const uint64_t dims[2] = {(uint64_t)N / 4, (uint64_t)C * T};
    const uint64_t strides[1] = {(uint64_t)N};
    const uint32_t box[2] = {(uint32_t)(kRawPitch / 4), (uint32_t)kST};
    gc_status st = gc_encode_tiled(ctx, &tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(volt), dims,
                                   strides, box);
    if (st != GC_OK) return st;
    TcParams p;
    p.L = L;
    p.N = N;
    p.C = C;
    p.T = T;
    p.n_blk = N / 128;
    p.n_tsplit = n_tsplit;
    p.w0 = sel->grp_t0[0];
    p.w1 = sel->grp_t1[0];
    p.n_items = C * p.n_blk * n_tsplit;
    p.ntypes = sel->n_ubl;
    p.P = sel->P;
    p.types = sel->d_types;
    p.type_ptr = sel->d_type_ptr;
    p.part = static_cast<int2 *>(part);
    p.apart = static_cast<int *>(apart);
    p.status = ctx->status_dev;
    // "xeng.tc_shape": converter warps / raw stages / operand stages.  The
    // kernel is bound by shared-memory bandwidth (the MMAs read 48 KB of
    // operands per stage beside the converters' 25 KB and the copies' 9 KB),
    // so more converter warps help by hiding latency, deeper rings do not.
    switch (ctx->tune[GC_TUNE_XENG_TC_SHAPE]) {
        case 1: return tc_launch<TcShape<4, 6, 3>>(ctx, tmap, p, s);
        case 2: return tc_launch<TcShape<4, 8, 4>>(ctx, tmap, p, s);
        case 4: return tc_launch<TcShape<8, 8, 4>>(ctx, tmap, p, s);
        default: return tc_launch<TcShape<8, 6, 3>>(ctx, tmap, p, s);
    }
}
