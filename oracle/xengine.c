/*
 * Oracle: reduced X-engine and the 4+4-bit quantiser.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Paper basis: Sec. 1 and Fig. 1 (the calibrator's first function is to
 * cross-correlate only the antenna pairs that the reduced calibration scheme
 * needs); Sec. 4 (low-cadence: each pair integrated over its own cycle).
 * The quantiser is the precision variant of the voltage path; the paper
 * itself does not quantise.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>

void orc_xeng_c64(int N, int T, const double *volt, int P, const int32_t *pi,
                  const int32_t *pj, const int32_t *t0, const int32_t *t1,
                  double *vred) {
    for (int p = 0; p < P; ++p) {
        double re = 0.0, im = 0.0;
        for (int t = t0[p]; t < t1[p] && t < T; ++t) {
            const double *a = volt + 2 * ((size_t)t * N + pi[p]);
            const double *b = volt + 2 * ((size_t)t * N + pj[p]);
            /* a * conj(b) */
            re += a[0] * b[0] + a[1] * b[1];
            im += a[1] * b[0] - a[0] * b[1];
        }
        vred[2 * p] = re;
        vred[2 * p + 1] = im;
    }
}

/* signed 4-bit two's complement nibble -> int */
static int nib(int v) { return (v & 8) ? (v & 15) - 16 : (v & 15); }

void orc_xeng_i4c(int N, int T, const uint8_t *volt, int P, const int32_t *pi,
                  const int32_t *pj, const int32_t *t0, const int32_t *t1,
                  int64_t *vred) {
    for (int p = 0; p < P; ++p) {
        int64_t re = 0, im = 0;
        for (int t = t0[p]; t < t1[p] && t < T; ++t) {
            int a = volt[(size_t)t * N + pi[p]], b = volt[(size_t)t * N + pj[p]];
            int ar = nib(a >> 4), ai = nib(a), br = nib(b >> 4), bi = nib(b);
            re += (int64_t)(ar * br + ai * bi);
            im += (int64_t)(ai * br - ar * bi);
        }
        vred[2 * p] = re;
        vred[2 * p + 1] = im;
    }
}

/* round half away from zero, written out */
static float round_half_away(float x) {
    float a = fabsf(x);
    float f = floorf(a);
    if (a - f >= 0.5f) f += 1.0f;
    return x < 0.0f ? -f : f;
}

static int clip7(float q) {
    if (q > 7.0f) return 7;
    if (q < -7.0f) return -7;
    return (int)q;
}

float orc_quantize(int T, int N, const float *volt, uint8_t *out) {
    double ss = 0.0;
    size_t n = (size_t)T * N;
    for (size_t k = 0; k < 2 * n; ++k) ss += (double)volt[k] * (double)volt[k];
    double rms = sqrt(ss / (double)(2 * n));
    float scale = rms > 0.0 ? (float)(3.0 / rms) : 0.0f;
    for (size_t k = 0; k < n; ++k) {
        /* product rounded to float, as written */
        volatile float xr = volt[2 * k] * scale;
        volatile float xi = volt[2 * k + 1] * scale;
        int qr = clip7(round_half_away(xr)), qi = clip7(round_half_away(xi));
        out[k] = (uint8_t)(((qr & 15) << 4) | (qi & 15));
    }
    return scale;
}
