// Reduced X-engine (paper Fig. 1, calibrator step (a)): cross-correlate only
// the antenna pairs of the selection, each over its own integration window
// (low-cadence cycles, Sec. 4; the whole integration for subset, Sec. 5).
//
// xeng_accumulate: one CTA per (channel, type group, block of reference
// antennas, time slice).  Samples of the whole grid are staged in shared
// memory by 1-D bulk TMA copies (double-buffered); each thread owns one
// reference antenna j and accumulates v_{j+d} conj(v_j) for every type d of
// its group in registers.  complex64 and binary16 voltages accumulate in
// FP32.  4+4-bit voltages take an integer path: each staged byte pair
// (samples t, t+1 of one antenna) is expanded by byte-parallel integer ops
// into two words of signed bytes
//   W  = (re_t, im_t, re_t1, im_t1),   Wx = (-im_t, re_t, -im_t1, re_t1),
// and one 4-way byte dot product with int32 accumulation (dp4a) gives two
// samples of each part of v_i conj(v_j):
//   Re = re_i re_j + im_i im_j = dp4a(W_i, W_j),
//   Im = im_i re_j - re_i im_j = dp4a(W_i, Wx_j),
// so a neighbour contributes its W words unchanged -- bit-exact sums.
// xeng_reduce: sums the time slices (FP64) into V^reduced and the autos.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>

#include "gc_sel.h"

namespace {

constexpr int kXThreads = 256;

struct XParams {
    const void *volt;         // [C][T][N]
    int vfmt, L, N, C, T;
    int n_groups, n_rowblk, n_tsplit;
    int n_items;
    int ns;                   // samples per stage
    const int32_t *types, *type_ptr, *grp_types, *grp_off, *grp_t0, *grp_t1, *grp_first;
    int P;
    float2 *part;             // [n_tsplit][C][P] (int2 for 4+4-bit voltages)
    float *apart;             // [n_windows * n_tsplit][C][N] (int for 4+4-bit; may be null)
    const int32_t *grp_win;   // window index per group
    const int32_t *grp_dymax; // largest dy among the group's types
    unsigned int *status;
    int use_tma;
    int rows_stage;           // 1: stage only the block's rows plus the dy halo
    size_t stage_stride;      // bytes per stage buffer (ns staged samples)
    int conv_recs;            // 4+4-bit: expanded antenna records (staged antennas + a zero record)
    // partly occupied lattice: pair index of (r_j + d_k, r_j) by [type][j],
    // -1 where either point is empty (null: every pair of the grid is in
    // the selection, at its arithmetic index)
    const int32_t *pair_of;
};

template <int VF>
__device__ __forceinline__ float2 ld_volt(const unsigned char *s, int idx) {
    if (VF == GC_C64) return reinterpret_cast<const float2 *>(s)[idx];
    if (VF == GC_C32H) return __half22float2(reinterpret_cast<const __half2 *>(s)[idx]);
    const int b = (int)(signed char)s[idx];
    return make_float2((float)(b >> 4), (float)((int)(signed char)(b << 4) >> 4));
}

// VF: voltage format; NTY: type slots per thread (>= the largest group);
// NP: sample pairs per stage for 4+4-bit voltages (8 with 16-sample stages, 1
// with 2-sample stages for wide staged regions; 1 for the other formats).
template <int VF, int NTY, int NP>
__global__ void __launch_bounds__(kXThreads, 2) xeng_accumulate(const XParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[2];
    __shared__ int s_dx[GC_XENG_NTY], s_dy[GC_XENG_NTY], s_base[GC_XENG_NTY], s_type[GC_XENG_NTY];
    __shared__ int s_err;
    constexpr bool kI4 = VF == GC_I4C;
    const int tid = threadIdx.x;
    constexpr int esz = VF == GC_C64 ? 8 : (VF == GC_C32H ? 4 : 1);
    const size_t sample_bytes = (size_t)p.N * esz;
    const size_t stage_stride = p.stage_stride;
    const int L = p.L;
    // 4+4-bit: one record per staged antenna after the raw stages,
    // [W of NP pairs | Wx of NP pairs | pad]; the pad makes the 16-byte record
    // reads of consecutive antennas conflict-free.  The last record stays zero
    // and stands in for neighbours outside the grid.
    constexpr int kRec = NP == 8 ? 20 : 2;
    uint32_t *conv = reinterpret_cast<uint32_t *>(smem + 2 * stage_stride);
    if (kI4) {
        for (int i = tid; i < kRec; i += kXThreads) conv[(size_t)(p.conv_recs - 1) * kRec + i] = 0u;
    }
    if (tid == 0) {
        s_err = 0;
        gc_mbar_init(&bars[0], 1);
        gc_mbar_init(&bars[1], 1);
        gc_fence_mbar_init();
    }
    __syncthreads();
    uint32_t ld_count = 0, use_count = 0;

    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        // item order: row block fastest, then group, time slice, channel
        const int rb = item % p.n_rowblk;
        const int g = (item / p.n_rowblk) % p.n_groups;
        const int ts = (item / (p.n_rowblk * p.n_groups)) % p.n_tsplit;
        const int c = item / (p.n_rowblk * p.n_groups * p.n_tsplit);
        const int w0 = p.grp_t0[g], w1 = p.grp_t1[g];
        const int len = (w1 - w0 + p.n_tsplit - 1) / p.n_tsplit;
        const int ta = min(w1, w0 + ts * len), tb = min(w1, ta + len);
        const int ntype = p.grp_off[g + 1] - p.grp_off[g];
        if (tid < ntype) {
            const int k = p.grp_types[p.grp_off[g] + tid];
            s_dx[tid] = p.types[2 * k];
            s_dy[tid] = p.types[2 * k + 1];
            s_base[tid] = p.type_ptr[k];
            s_type[tid] = k;
        }
        const int j = rb * kXThreads + tid;
        const int x = j % L, y = j / L;
        const bool own = j < p.N;
        const unsigned char *vc = static_cast<const unsigned char *>(p.volt) + (size_t)c * p.T * sample_bytes;
        const int n_st = (tb - ta + p.ns - 1) / p.ns;
        // staged part of each sample: rows [y_lo, y_hi) (whole sample without row staging)
        const int y_lo = p.rows_stage ? (rb * kXThreads) / L : 0;
        const int y_hi = p.rows_stage ? min(L, (min(p.N, (rb + 1) * kXThreads) - 1) / L + 1 + p.grp_dymax[g]) : L;
        const size_t part_bytes = (size_t)(y_hi - y_lo) * L * esz;   // staged bytes per sample
        const size_t src_off = (size_t)y_lo * L * esz;
        auto issue = [&](int t, int cnt, uint32_t b) {
            unsigned char *dst = smem + b * stage_stride;
            gc_mbar_expect_tx(&bars[b], (uint32_t)(cnt * part_bytes));
            if (part_bytes == sample_bytes) {
                gc_bulk_load(dst, vc + (size_t)t * sample_bytes, (uint32_t)(cnt * sample_bytes), &bars[b]);
            } else {
                for (int u = 0; u < cnt; ++u)
                    gc_bulk_load(dst + u * part_bytes, vc + (size_t)(t + u) * sample_bytes + src_off,
                                 (uint32_t)part_bytes, &bars[b]);
            }
        };
        if (p.use_tma && tid == 0) {
            for (int k = 0; k < 2 && k < n_st; ++k) {
                const int t = ta + k * p.ns;
                issue(t, min(p.ns, tb - t), ld_count & 1u);
                ++ld_count;
            }
        }
        __syncthreads();

        float2 acc[kI4 ? 1 : NTY];
        int ire[kI4 ? NTY : 1], iim[kI4 ? NTY : 1];
        int nb[NTY];   // neighbour antenna r_j + d_k, or -1 (fixed for the item)
        const bool do_autos = p.apart && p.grp_first[g];
#pragma unroll
        for (int k = 0; k < NTY; ++k) {
            if (kI4) {
                ire[k] = 0;
                iim[k] = 0;
            } else {
                acc[k] = make_float2(0.f, 0.f);
            }
            nb[k] = -1;
            if (k < ntype && own) {
                const int xi = x + s_dx[k], yi = y + s_dy[k];
                if (xi >= 0 && xi < L && yi >= 0 && yi < L) nb[k] = (yi - y_lo) * L + xi;
            }
        }
        float aut = 0.f;
        int iaut = 0;
        auto refill = [&](int st) {
            if (p.use_tma && tid == 0 && st + 2 < n_st) {
                gc_fence_proxy_async();
                const int t2 = ta + (st + 2) * p.ns;
                issue(t2, min(p.ns, tb - t2), ld_count & 1u);
                ++ld_count;
            }
        };

        for (int st = 0; st < n_st; ++st) {
            const int t = ta + st * p.ns;
            const int cnt = min(p.ns, tb - t);
            const unsigned char *stage;
            if (p.use_tma) {
                const uint32_t b = use_count & 1u;
                stage = smem + b * stage_stride;
                if (!gc_mbar_wait(&bars[b], (use_count >> 1) & 1u, GC_WAIT_LIMIT_NS)) {
                    atomicOr(p.status, GC_DEV_TIMEOUT_XENG);
                    s_err = 1;
                } else {
                    ++use_count;
                }
                __syncthreads();
                if (s_err) break;
            } else {
                // plain staging (sizes or alignment TMA cannot take)
                for (size_t i = tid; i < cnt * part_bytes; i += kXThreads) {
                    const size_t u = i / part_bytes, o = i - u * part_bytes;
                    smem[i] = vc[(size_t)(t + u) * sample_bytes + src_off + o];
                }
                stage = smem;
                __syncthreads();
            }
            if constexpr (kI4) {
                // expand every staged antenna's bytes, sample pair by pair
                // (samples beyond the copied count are zero)
                // work unit = (antenna, two sample pairs); consecutive threads
                // take consecutive antennas of one sample row
                const int n_ant = (int)part_bytes;
                constexpr int kQ = NP == 8 ? 4 : 1;   // units per antenna
                for (int u = tid; u < kQ * n_ant; u += kXThreads) {
                    const int qu = kQ == 1 ? 0 : u / n_ant;
                    const int a = u - qu * n_ant;
                    const int s0 = 4 * qu;             // first sample of the unit
                    uint32_t X = 0u;                   // bytes of samples s0..s0+3 (0 past cnt)
#pragma unroll
                    for (int i = 0; i < (NP == 8 ? 4 : 2); ++i)
                        if (s0 + i < cnt) X |= (uint32_t)stage[(size_t)(s0 + i) * part_bytes + a] << (8 * i);
                    // sign-extend the nibbles byte-parallel: (n ^ 8) + 0x78 never
                    // carries out of a byte and ^ 0x80 turns it into n as int8;
                    // 0x88 - (n ^ 8), then ^ 0x80, gives -n
                    const uint32_t ux = (X & 0x0F0F0F0Fu) ^ 0x08080808u;
                    const uint32_t vx = ((X >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
                    const uint32_t im = (ux + 0x78787878u) ^ 0x80808080u;
                    const uint32_t nim = (0x88888888u - ux) ^ 0x80808080u;
                    const uint32_t re = (vx + 0x78787878u) ^ 0x80808080u;
                    uint32_t *rec = conv + (size_t)a * kRec;
                    if constexpr (NP == 8) {
                        *reinterpret_cast<uint2 *>(rec + 2 * qu) =
                            make_uint2(__byte_perm(re, im, 0x5140), __byte_perm(re, im, 0x7362));
                        *reinterpret_cast<uint2 *>(rec + 8 + 2 * qu) =
                            make_uint2(__byte_perm(nim, re, 0x5140), __byte_perm(nim, re, 0x7362));
                    } else {
                        *reinterpret_cast<uint2 *>(rec) =
                            make_uint2(__byte_perm(re, im, 0x5140), __byte_perm(nim, re, 0x5140));
                    }
                }
                __syncthreads();
                refill(st);   // the raw stage is free again
                if (own) {
                    const int jl = j - y_lo * L;
                    uint32_t wj[NP], wxj[NP];
                    const uint32_t *rj = conv + (size_t)jl * kRec;
                    if constexpr (NP == 8) {
                        const uint4 *r4 = reinterpret_cast<const uint4 *>(rj);
                        const uint4 a0 = r4[0], a1 = r4[1], b0 = r4[2], b1 = r4[3];
                        wj[0] = a0.x; wj[1] = a0.y; wj[2] = a0.z; wj[3] = a0.w;
                        wj[4] = a1.x; wj[5] = a1.y; wj[6] = a1.z; wj[7] = a1.w;
                        wxj[0] = b0.x; wxj[1] = b0.y; wxj[2] = b0.z; wxj[3] = b0.w;
                        wxj[4] = b1.x; wxj[5] = b1.y; wxj[6] = b1.z; wxj[7] = b1.w;
                    } else {
                        const uint2 r = *reinterpret_cast<const uint2 *>(rj);
                        wj[0] = r.x;
                        wxj[0] = r.y;
                    }
                    if (do_autos) {
#pragma unroll
                        for (int q = 0; q < NP; ++q) iaut = __dp4a((int)wj[q], (int)wj[q], iaut);
                    }
                    // straight-line over the type slots (absent neighbours and
                    // unused slots read the zero record) so that loads and the
                    // dp4a chains of different types interleave
#pragma unroll
                    for (int k = 0; k < NTY; ++k) {
                        const uint32_t *ri = conv + (size_t)(nb[k] >= 0 ? nb[k] : p.conv_recs - 1) * kRec;
                        uint32_t wi[NP];
                        if constexpr (NP == 8) {
                            const uint4 *r4 = reinterpret_cast<const uint4 *>(ri);
                            const uint4 a0 = r4[0], a1 = r4[1];
                            wi[0] = a0.x; wi[1] = a0.y; wi[2] = a0.z; wi[3] = a0.w;
                            wi[4] = a1.x; wi[5] = a1.y; wi[6] = a1.z; wi[7] = a1.w;
                        } else {
                            wi[0] = ri[0];
                        }
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            ire[k] = __dp4a((int)wi[q], (int)wj[q], ire[k]);
                            iim[k] = __dp4a((int)wi[q], (int)wxj[q], iim[k]);
                        }
                    }
                }
                __syncthreads();
            } else {
                if (own) {
                    const int jl = j - y_lo * L;   // own antenna within the staged rows
                    for (int u = 0; u < cnt; ++u) {
                        const unsigned char *sv = stage + u * part_bytes;
                        const float2 b = ld_volt<VF>(sv, jl);
                        if (do_autos) aut = fmaf(b.x, b.x, fmaf(b.y, b.y, aut));
#pragma unroll
                        for (int k = 0; k < NTY; ++k) {
                            if (nb[k] >= 0) {
                                const float2 a = ld_volt<VF>(sv, nb[k]);
                                // a * conj(b)
                                acc[k].x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc[k].x));
                                acc[k].y = fmaf(a.y, b.x, fmaf(-a.x, b.y, acc[k].y));
                            }
                        }
                    }
                }
                __syncthreads();
                refill(st);
            }
        }
        if (s_err) break;
        if (own) {
            float2 *out = p.part + ((size_t)ts * p.C + c) * p.P;
#pragma unroll
            for (int k = 0; k < NTY; ++k) {
                if (k < ntype) {
                    const int dx = s_dx[k], dy = s_dy[k];
                    const int xlo = max(0, -dx), ylo = max(0, -dy);
                    const int xi = x + dx, yi = y + dy;
                    if (xi >= 0 && xi < L && yi >= 0 && yi < L) {
                        long o = s_base[k] + (y - ylo) * (L - abs(dx)) + (x - xlo);
                        if (p.pair_of) o = p.pair_of[(size_t)s_type[k] * p.N + j];
                        if (o >= 0) {
                            if constexpr (kI4) reinterpret_cast<int2 *>(out)[o] = make_int2(ire[k], iim[k]);
                            else out[o] = acc[k];
                        }
                    }
                }
            }
            if (do_autos) {
                const int slot = p.grp_win[g] * p.n_tsplit + ts;
                const size_t o = ((size_t)slot * p.C + c) * p.N + j;
                if constexpr (kI4) reinterpret_cast<int *>(p.apart)[o] = iaut;
                else p.apart[o] = aut;
            }
        }
        __syncthreads();
    }
    if (p.use_tma && s_err && tid == 0) {
        while (use_count < ld_count) {
            gc_mbar_wait(&bars[use_count & 1u], (use_count >> 1) & 1u, GC_WAIT_LIMIT_NS / 10);
            ++use_count;
        }
    }
}

// Sum the time slices: V^reduced (c64: float2, i4c: exact int32 pairs) and autos.
__global__ void xeng_reduce(const float2 *__restrict__ part, int n_tsplit, int C, int P, int vfmt, void *vred,
                            const float *__restrict__ apart, int n_aslots, int N, void *autos,
                            unsigned int *status) {
    const size_t total = (size_t)C * P;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total + (size_t)C * N;
         idx += (size_t)gridDim.x * blockDim.x) {
        if (idx < total) {
            if (vfmt != GC_I4C) {
                double re = 0.0, im = 0.0;
                for (int s = 0; s < n_tsplit; ++s) {
                    const float2 v = part[(size_t)s * total + idx];
                    re += v.x;
                    im += v.y;
                }
                if (!isfinite(re) || !isfinite(im)) atomicOr(status, GC_DEV_BADINPUT);   // non-finite voltages
                reinterpret_cast<float2 *>(vred)[idx] = make_float2((float)re, (float)im);
            } else {
                int re = 0, im = 0;
                for (int s = 0; s < n_tsplit; ++s) {
                    const int2 v = reinterpret_cast<const int2 *>(part)[(size_t)s * total + idx];
                    re += v.x;
                    im += v.y;
                }
                reinterpret_cast<int2 *>(vred)[idx] = make_int2(re, im);
            }
        } else if (autos) {
            const size_t a = idx - total;
            if (vfmt != GC_I4C) {
                double s = 0.0;
                for (int k = 0; k < n_aslots; ++k) s += apart[(size_t)k * C * N + a];
                reinterpret_cast<float *>(autos)[a] = (float)s;
            } else {
                int s = 0;
                for (int k = 0; k < n_aslots; ++k) s += reinterpret_cast<const int *>(apart)[(size_t)k * C * N + a];
                reinterpret_cast<int *>(autos)[a] = s;
            }
        }
    }
}

template <int VF, int NP>
const void *pick_xeng(int nty) {
    return nty == 4 ? (const void *)xeng_accumulate<VF, 4, NP> : nty == 8 ? (const void *)xeng_accumulate<VF, 8, NP>
         : nty == 12 ? (const void *)xeng_accumulate<VF, 12, NP> : (const void *)xeng_accumulate<VF, 16, NP>;
}

}  // namespace

extern "C" gc_status gc_reduce(gc_ctx *ctx, const void *volt, int vfmt, int L, int C, int T, const gc_sel *csel,
                               void *vreduced, void *autos, void *stream) {
    if (!ctx) return GC_EINVAL;
    ctx->last_error.clear();
    gc_sel *sel = const_cast<gc_sel *>(csel);   // device copies are a cache of the immutable selection
    if (!volt || !sel || !vreduced) return gc_fail(ctx, GC_EINVAL, "gc_reduce: null argument");
    if (vfmt != GC_C64 && vfmt != GC_I4C && vfmt != GC_C32H)
        return gc_fail(ctx, GC_EINVAL, "gc_reduce: unknown voltage format");
    if (L != sel->L || T < sel->T || C < 1)
        return gc_fail(ctx, GC_EINVAL, "gc_reduce: grid or integration does not match the selection");
    if (!gc_aligned(vreduced, 8) || (autos && !gc_aligned(autos, 4)) || (vfmt == GC_C64 && !gc_aligned(volt, 8)) ||
        (vfmt == GC_C32H && !gc_aligned(volt, 4)))
        return gc_fail(ctx, GC_EINVAL, "gc_reduce: misaligned buffer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaSetDevice");
    gc_status st = gc_sel_upload(ctx, sel);
    if (st != GC_OK) return st;
    const int N = L * L;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // tensor cores for 4+4-bit subset selections ("xeng.path": 0 automatic,
    // 1 integer SIMT path, 2 tensor cores only)
    const int path = ctx->tune[GC_TUNE_XENG_PATH];
    const bool tc_ok = gc_xeng_tc_eligible(sel, vfmt, volt, L);
    if (path == 2 && !tc_ok)
        return gc_fail(ctx, GC_EUNSUPPORTED, "gc_reduce: the tensor-core X-engine does not cover this call");
    if (tc_ok && path != 1) {
        int n_tsplit = gc_xeng_tc_slices(ctx, sel, L, C);
        if (ctx->tune[GC_TUNE_XENG_TSPLIT] > 0) n_tsplit = std::max(n_tsplit, std::min(ctx->tune[GC_TUNE_XENG_TSPLIT], 64));
        const size_t part_bytes = (size_t)n_tsplit * C * sel->P * sizeof(int2);
        const size_t apart_bytes = autos ? (size_t)n_tsplit * C * N * sizeof(int) : 0;
        st = gc_scratch_reserve(ctx, part_bytes + apart_bytes + 512);
        if (st != GC_OK) return st;
        char *scr = static_cast<char *>(ctx->scratch);
        void *part = scr;
        int *apart = autos ? reinterpret_cast<int *>(scr + ((part_bytes + 255) / 256) * 256) : nullptr;
        st = gc_xeng_tc_launch(ctx, volt, L, C, T, sel, part, apart, n_tsplit, s);
        if (st != GC_OK) return st;
        const size_t work = (size_t)C * sel->P + (autos ? (size_t)C * N : 0);
        const int rgrid = (int)std::min<size_t>((work + 255) / 256, (size_t)ctx->sm_count * 8);
        int rec = gc_prof_begin(ctx, s, "xeng_reduce");
        xeng_reduce<<<rgrid, 256, 0, s>>>(static_cast<const float2 *>(part), n_tsplit, C, sel->P, vfmt, vreduced,
                                          reinterpret_cast<const float *>(apart), n_tsplit, N, autos,
                                          ctx->status_dev);
        gc_prof_end(ctx, s, rec);
        e = cudaGetLastError();
        if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch xeng_reduce");
        return GC_OK;
    }
    const int esz = vfmt == GC_C64 ? 8 : (vfmt == GC_C32H ? 4 : 1);
    const size_t sample_bytes = (size_t)N * esz;
    const bool tma = gc_aligned(volt, 16) && sample_bytes % 16 == 0;
    const int n_rowblk = (N + kXThreads - 1) / kXThreads;
    // stage row ranges when the halo is small (subset selections); a bulk copy
    // per row range needs 16-byte aligned rows
    int dymax_all = 0, ntmax = 0;
    for (int k = 0; k < sel->n_ubl; ++k) dymax_all = std::max(dymax_all, sel->types[2 * k + 1]);
    for (int g = 0; g < sel->n_groups; ++g) ntmax = std::max(ntmax, sel->grp_off[g + 1] - sel->grp_off[g]);
    const int rows_stage = (n_rowblk > 1 && (kXThreads / L + 1 + dymax_all) < L &&
                            (!tma || ((size_t)L * esz) % 16 == 0)) ? 1 : 0;
    const size_t staged = rows_stage ? (size_t)std::min(L, kXThreads / L + 2 + dymax_all) * L * esz : sample_bytes;
    int ns = (int)std::max<size_t>(1, std::min<size_t>(16, (32u << 10) / staged));
    if (vfmt == GC_I4C) ns = ns == 16 ? 16 : 2;   // 8 sample pairs per stage, or 1 for wide regions
    const size_t stage_stride = ((staged * ns + 127) / 128) * 128;
    // 4+4-bit: one expanded record per staged antenna plus the zero record
    const int conv_recs = vfmt == GC_I4C ? (int)staged + 1 : 0;
    const size_t smem = 2 * stage_stride + (size_t)conv_recs * (ns == 16 ? 20 : 2) * 4;
    if (smem > 200u * 1024u) return gc_fail(ctx, GC_EUNSUPPORTED, "gc_reduce: grid too large for the stage");
    const int nty = ntmax <= 4 ? 4 : (ntmax <= 8 ? 8 : (ntmax <= 12 ? 12 : 16));
    const void *kern;
    if (vfmt == GC_C64)
        kern = pick_xeng<GC_C64, 1>(nty);
    else if (vfmt == GC_C32H)
        kern = pick_xeng<GC_C32H, 1>(nty);
    else
        kern = ns == 16 ? pick_xeng<GC_I4C, 8>(nty) : pick_xeng<GC_I4C, 1>(nty);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "cudaFuncSetAttribute(xeng_accumulate)");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kXThreads, smem);
    if (e != cudaSuccess || occ < 1) return gc_cuda_fail(ctx, e, "occupancy(xeng_accumulate)");
    const int slots = occ * ctx->sm_count;
    const long base_items = (long)C * sel->n_groups * n_rowblk;
    // split long windows in time so that the items fill whole waves of the
    // resident CTAs (slices of at least 64 samples)
    int max_win = 0;
    for (int g = 0; g < sel->n_groups; ++g) max_win = std::max(max_win, sel->grp_t1[g] - sel->grp_t0[g]);
    int n_tsplit = 1;
    double best = -1.0;
    for (int ts = 1; ts <= 16; ++ts) {
        if (ts > 1 && max_win / ts < 64) break;
        const long items = base_items * ts;
        const long waves = (items + slots - 1) / slots;
        const double eff = (double)items / ((double)waves * slots) - 0.01 * ts;   // prefer fewer slices
        if (eff > best) {
            best = eff;
            n_tsplit = ts;
        }
    }
    if (ctx->tune[GC_TUNE_XENG_TSPLIT] > 0) n_tsplit = std::min(ctx->tune[GC_TUNE_XENG_TSPLIT], 64);
    const size_t part_bytes = (size_t)n_tsplit * C * sel->P * sizeof(float2);
    const size_t apart_bytes = autos ? (size_t)sel->n_windows * n_tsplit * C * N * sizeof(float) : 0;
    st = gc_scratch_reserve(ctx, part_bytes + apart_bytes + 512);
    if (st != GC_OK) return st;
    char *scr = static_cast<char *>(ctx->scratch);
    float2 *part = reinterpret_cast<float2 *>(scr);
    float *apart = autos ? reinterpret_cast<float *>(scr + ((part_bytes + 255) / 256) * 256) : nullptr;

    XParams p;
    p.volt = volt;
    p.vfmt = vfmt;
    p.L = L;
    p.N = N;
    p.C = C;
    p.T = T;
    p.n_groups = sel->n_groups;
    p.n_rowblk = n_rowblk;
    p.n_tsplit = n_tsplit;
    p.n_items = (int)(base_items * n_tsplit);
    p.ns = ns;
    p.types = sel->d_types;
    p.type_ptr = sel->d_type_ptr;
    p.grp_types = sel->d_grp_types;
    p.grp_off = sel->d_grp_off;
    p.grp_t0 = sel->d_grp_t0;
    p.grp_t1 = sel->d_grp_t1;
    p.grp_first = sel->d_grp_first;
    p.P = sel->P;
    p.part = part;
    p.apart = apart;
    p.grp_win = sel->d_grp_win;
    p.grp_dymax = sel->d_grp_dymax;
    p.status = ctx->status_dev;
    p.use_tma = tma ? 1 : 0;
    p.rows_stage = rows_stage;
    p.stage_stride = stage_stride;
    p.conv_recs = conv_recs;
    p.pair_of = nullptr;
    if (sel->masked) {
        if (!sel->d_nbr) return gc_fail(ctx, GC_EUNSUPPORTED, "gc_reduce: masked selection without pair table");
        p.pair_of = sel->d_nbr + (size_t)sel->n_ubl * N;   // antenna as the second member
    }
    const int grid = (int)std::min<long>(p.n_items, slots);
    int rec = gc_prof_begin(ctx, s, "xeng_accumulate");
    void *args[] = {&p};
    e = cudaLaunchKernel(kern, dim3(grid), dim3(kXThreads), args, smem, s);
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch xeng_accumulate");
    gc_prof_end(ctx, s, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch xeng_accumulate");
    const size_t work = (size_t)C * sel->P + (autos ? (size_t)C * N : 0);
    const int rgrid = (int)std::min<size_t>((work + 255) / 256, (size_t)ctx->sm_count * 8);
    rec = gc_prof_begin(ctx, s, "xeng_reduce");
    xeng_reduce<<<rgrid, 256, 0, s>>>(part, n_tsplit, C, sel->P, vfmt, vreduced, apart,
                                      sel->n_windows * n_tsplit, N, autos, ctx->status_dev);
    gc_prof_end(ctx, s, rec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gc_cuda_fail(ctx, e, "launch xeng_reduce");
    return GC_OK;
}
