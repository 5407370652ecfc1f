// Register-level FFT helpers shared by the FFT-correlator kernels: the
// omega_256 twiddle table (built at compile time), packed two-lane FP32 adds,
// complex multiplies and the in-register radix-2 FFT.  Each translation unit
// gets its own copy (anonymous namespace).
#pragma once

#include "gc_internal.h"

#ifdef __CUDACC__
namespace {

// ----------------------------------------------------------------- twiddles
// omega_256^e = exp(-2 pi i e / 256), built at compile time from a Taylor
// series (double) and rounded to float; exact at multiples of pi/4.
struct cf {
    float x, y;
};
struct Tw256 {
    cf v[256];
};
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double cx_sin(double x) {
    double t = x, s = x;
    for (int n = 1; n < 40; ++n) {
        t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        s += t;
    }
    return s;
}
constexpr double cx_cos(double x) {
    double t = 1.0, s = 1.0;
    for (int n = 1; n < 40; ++n) {
        t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        s += t;
    }
    return s;
}
constexpr Tw256 make_tw256() {
    Tw256 t{};
    const double h = 0.70710678118654752440084436210484903928;
    for (int e = 0; e < 256; ++e) {
        double c = 0.0, s = 0.0;
        if (e % 64 == 0) {
            const int q = e / 64;
            c = q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0);
            s = q == 1 ? 1.0 : (q == 3 ? -1.0 : 0.0);
        } else if (e % 32 == 0) {
            const int q = e / 32;  // 1, 3, 5, 7
            c = (q == 1 || q == 7) ? h : -h;
            s = (q == 1 || q == 3) ? h : -h;
        } else {
            double th = 2.0 * kPi * e / 256.0;
            if (th > kPi) th -= 2.0 * kPi;
            c = cx_cos(th);
            s = cx_sin(th);
        }
        t.v[e].x = (float)c;
        t.v[e].y = (float)(-s);
    }
    return t;
}
__constant__ Tw256 c_tw = make_tw256();

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// Packed two-lane FP32 add / subtract (one instruction for both parts of a
// complex number; each lane rounds as the scalar operation does).
__device__ __forceinline__ unsigned long long pk2(float2 a) { return *reinterpret_cast<unsigned long long *>(&a); }
__device__ __forceinline__ float2 up2(unsigned long long a) { return *reinterpret_cast<float2 *>(&a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return up2(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return up2(d);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 w) {
    acc.x = fmaf(a.x, w.x, fmaf(-a.y, w.y, acc.x));
    acc.y = fmaf(a.x, w.y, fmaf(a.y, w.x, acc.y));
    return acc;
}

// multiply by omega_256^e; e is a compile-time constant after unrolling
__device__ __forceinline__ float2 tw_apply(float2 d, int e) {
    const float h = 0.70710678118654752f;
    if (e == 0) return d;
    if (e == 64) return make_float2(d.y, -d.x);                     // * (-i)
    if (e == 32) return make_float2((d.x + d.y) * h, (d.y - d.x) * h);   // * (1-i)/sqrt2
    if (e == 96) return make_float2((d.y - d.x) * h, -(d.x + d.y) * h);  // * (-1-i)/sqrt2
    const cf w = c_tw.v[e];
    return cmul(d, make_float2(w.x, w.y));
}

// In-register radix-2 decimation-in-frequency FFT of F points (forward,
// omega = exp(-2 pi i / F)); output in bit-reversed order: a[i] = X[rev(i)].
template <int F>
__device__ __forceinline__ void fft_reg(float2 (&a)[F]) {
#pragma unroll
    for (int len = F; len >= 2; len >>= 1) {
#pragma unroll
        for (int blk = 0; blk < F; blk += len) {
#pragma unroll
            for (int j = 0; j < len / 2; ++j) {
                const float2 u = a[blk + j], v = a[blk + j + len / 2];
                a[blk + j] = add2(u, v);
                a[blk + j + len / 2] = tw_apply(sub2(u, v), j * (256 / len));
            }
        }
    }
}

template <int F>
__host__ __device__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1; b < F; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

// 4+4-bit voltages without an int-to-float conversion: flipping a nibble's
// sign bit gives n + 8 in [0, 15], one byte each in the words ure / uim (Re /
// Im codes of four antennas); byte e placed under the exponent of 2^23 is the
// float 2^23 + n + 8 (one byte permute), and subtracting 2^23 + 8 leaves n.
__device__ __forceinline__ float2 i4c_bytes_to_f2(unsigned int ure, unsigned int uim, int e) {
    const unsigned int sel = 0x7440u | (unsigned int)e;
    const float re = __uint_as_float(__byte_perm(ure, 0x4B000000u, sel)) - 8388616.0f;
    const float im = __uint_as_float(__byte_perm(uim, 0x4B000000u, sel)) - 8388616.0f;
    return make_float2(re, im);
}

}  // namespace
#endif  // __CUDACC__
