/*
 * FP64 reference implementation ("oracle") of the FFT-correlator system of
 * Gorthi, Parsons & Dillon (2020), "Calibration schemes with O(N log N)
 * scaling for large-N radio interferometers built on a regular grid".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path includes,
 * links or calls this code; only the test-suite, the smoke check and the CPU
 * baseline of the benchmark do.  It shares no source with the CUDA path.
 *
 * Conventions (the paper's Sec. 2 and Eq. modelvis, read as stated in the
 * design notes):
 *   - antenna i sits at r_i = (x, y) on an L x L unit grid, i = y*L + x;
 *   - complex numbers are stored interleaved (re, im) as double;
 *   - voltages of one channel are [T][N] complex;
 *   - a visibility of the ordered pair (i, j) is <v_i v_j^*>, of separation
 *     d = r_i - r_j (Eq. redcal: d_alpha = r_0 - r_1);
 *   - V^unique is indexed [dy + L - 1][dx + L - 1] over |dx|, |dy| <= L-1.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* FX correlator (Fig. 1a): V_ij = (1/T) sum_t w_i w_j^*, w_i = v_i / g_i, for
 * all ordered pairs, then Eq. modelvis: V^unique(d) = (1/N_d) sum_{r_i-r_j=d}
 * V_ij.  vfull may be NULL; otherwise it receives the [N][N] matrix.
 * volt: [T][N] complex, gains: [N] complex (NULL means all ones),
 * vunique: [(2L-1)^2] complex. */
void orc_fx(int L, int T, const double *volt, const double *gains,
            double *vunique, double *vfull);

/* Multi-channel FX, OpenMP over channels.  volt [C][T][N], gains [C][N],
 * vunique [C][(2L-1)^2]. Returns the number of threads used. */
int orc_fx_multi(int C, int L, int T, const double *volt, const double *gains,
                 double *vunique);
/* orc_fx's V^unique for one channel with the pair loop over OpenMP threads
 * (fixed-order reduction); returns the thread count. */
int orc_fx_par(int L, int T, const double *volt, const double *gains, double *vunique);

/* FFT-correlator written as direct DFTs (Fig. 1b, Sec. 1): per sample
 * X(k) = sum_r w(r) e^{-2 pi i k.r / M} on an M x M zero-padded grid,
 * P(k) = sum_t |X(k)|^2, R(d) = (1/M^2) sum_k P(k) e^{+2 pi i k.d/M},
 * V^unique(d) = R(d) / (T N_d).  Requires M >= 2L-1.  pk (may be NULL)
 * receives P(k) as [M][M] doubles (k_y major). */
void orc_dft(int L, int M, int T, const double *volt, const double *gains,
             double *vunique, double *pk);

/* One lag of V^unique by its definition (Eq. modelvis), for sampled checks
 * at sizes where the full oracle would be too slow. out: 1 complex. */
void orc_lag(int L, int T, const double *volt, const double *gains,
             int dx, int dy, double *out);

/* Reduced X-engine (Fig. 1 blue box, step (a)): for each selected pair p,
 * S_p = sum_{t in [t0_p, t1_p)} v_{i_p}(t) v_{j_p}(t)^*  (raw sums, no
 * gains).  vred: [P] complex. */
void orc_xeng_c64(int N, int T, const double *volt, int P, const int32_t *pi,
                  const int32_t *pj, const int32_t *t0, const int32_t *t1,
                  double *vred);

/* Same on 4+4-bit voltages (high nibble = Re, low nibble = Im, two's
 * complement); exact int64 sums.  volt: [T][N] bytes, vred: [P][2] int64. */
void orc_xeng_i4c(int N, int T, const uint8_t *volt, int P, const int32_t *pi,
                  const int32_t *pj, const int32_t *t0, const int32_t *t1,
                  int64_t *vred);

/* Auto-correlation sums A_i = sum_{t in [t0,t1)} |v_i(t)|^2. */
void orc_autos_c64(int N, int T, const double *volt, int t0, int t1, double *autos);

/* 4+4-bit quantiser of one channel (precision pattern of the voltage path):
 * rms = sqrt(sum(re^2 + im^2) / (2 T N)) in FP64, scale = (float)(3 / rms),
 * q = clip(round_half_away(x * scale computed in float), -7, 7), byte =
 * (q_re << 4) | (q_im & 15).  volt: [T][N] complex64 as float pairs.
 * Returns the float scale used. */
float orc_quantize(int T, int N, const float *volt, uint8_t *out);

#ifdef __cplusplus
}
#endif
#endif
