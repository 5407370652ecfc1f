/*
 * Oracle: FX correlator, direct-DFT FFT-correlator and single-lag V^unique.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain loops, FP64, no blocking.
 *
 * Paper basis: Sec. 1 (FX vs FFT correlator, convolution theorem, Fig. 1),
 * Sec. 2 Eq. modelvis (redundant averaging of calibrated visibilities).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* w = v / g for one antenna (g == NULL means unit gains). */
static void calibrated(const double *v, const double *g, double *w) {
    if (!g) { w[0] = v[0]; w[1] = v[1]; return; }
    double d = g[0] * g[0] + g[1] * g[1];
    /* v * conj(g) / |g|^2 */
    w[0] = (v[0] * g[0] + v[1] * g[1]) / d;
    w[1] = (v[1] * g[0] - v[0] * g[1]) / d;
}

/* N_d = number of ordered pairs (i, j) with r_i - r_j = d on an L x L grid. */
static int n_redundant(int L, int dx, int dy) {
    return (L - abs(dx)) * (L - abs(dy));
}

void orc_fx(int L, int T, const double *volt, const double *gains,
            double *vunique, double *vfull) {
    const int N = L * L, W = 2 * L - 1;
    double *w = (double *)malloc(sizeof(double) * 2 * (size_t)N * T);
    for (int t = 0; t < T; ++t)
        for (int i = 0; i < N; ++i)
            calibrated(volt + 2 * ((size_t)t * N + i), gains ? gains + 2 * i : NULL,
                       w + 2 * ((size_t)t * N + i));
    memset(vunique, 0, sizeof(double) * 2 * W * W);
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j < N; ++j) {
            /* V_ij = (1/T) sum_t w_i w_j^* */
            double re = 0.0, im = 0.0;
            for (int t = 0; t < T; ++t) {
                const double *a = w + 2 * ((size_t)t * N + i);
                const double *b = w + 2 * ((size_t)t * N + j);
                re += a[0] * b[0] + a[1] * b[1];
                im += a[1] * b[0] - a[0] * b[1];
            }
            re /= T;
            im /= T;
            if (vfull) {
                vfull[2 * ((size_t)i * N + j)] = re;
                vfull[2 * ((size_t)i * N + j) + 1] = im;
            }
            int dx = (i % L) - (j % L), dy = (i / L) - (j / L);
            int o = (dy + L - 1) * W + (dx + L - 1);
            vunique[2 * o] += re;
            vunique[2 * o + 1] += im;
        }
    }
    /* Eq. modelvis: divide each redundant sum by N_alpha */
    for (int dy = -(L - 1); dy <= L - 1; ++dy)
        for (int dx = -(L - 1); dx <= L - 1; ++dx) {
            int o = (dy + L - 1) * W + (dx + L - 1);
            double n = (double)n_redundant(L, dx, dy);
            vunique[2 * o] /= n;
            vunique[2 * o + 1] /= n;
        }
    free(w);
}

/* orc_fx's V^unique with its pair loop split over threads, for one large
 * channel: the calibrated voltages are copied antenna-major so that each
 * pair's time sum walks contiguous memory (the same sum over t as orc_fx),
 * every thread adds its first antennas' pairs into its own lag array, and
 * the arrays are added in thread order before the division by N_alpha
 * (Eq. modelvis).  Returns the number of threads. */
int orc_fx_par(int L, int T, const double *volt, const double *gains, double *vunique) {
    const int N = L * L, W = 2 * L - 1;
    double *w = (double *)malloc(sizeof(double) * 2 * (size_t)N * T);
    for (int t = 0; t < T; ++t)
        for (int i = 0; i < N; ++i)
            calibrated(volt + 2 * ((size_t)t * N + i), gains ? gains + 2 * i : NULL,
                       w + 2 * ((size_t)i * T + t));
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nthreads * 2 * W * W, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *a = acc + (size_t)tid * 2 * W * W;
#pragma omp for schedule(static)
        for (int i = 0; i < N; ++i) {
            const double *wi = w + 2 * (size_t)i * T;
            for (int j = 0; j < N; ++j) {
                const double *wj = w + 2 * (size_t)j * T;
                double re = 0.0, im = 0.0;
                for (int t = 0; t < T; ++t) {
                    re += wi[2 * t] * wj[2 * t] + wi[2 * t + 1] * wj[2 * t + 1];
                    im += wi[2 * t + 1] * wj[2 * t] - wi[2 * t] * wj[2 * t + 1];
                }
                const int dx = (i % L) - (j % L), dy = (i / L) - (j / L);
                const int o = (dy + L - 1) * W + (dx + L - 1);
                a[2 * o] += re / T;
                a[2 * o + 1] += im / T;
            }
        }
    }
    memset(vunique, 0, sizeof(double) * 2 * W * W);
    for (int u = 0; u < nthreads; ++u)
        for (int o = 0; o < 2 * W * W; ++o) vunique[o] += acc[(size_t)u * 2 * W * W + o];
    for (int dy = -(L - 1); dy <= L - 1; ++dy)
        for (int dx = -(L - 1); dx <= L - 1; ++dx) {
            const int o = (dy + L - 1) * W + (dx + L - 1);
            const double n = (double)n_redundant(L, dx, dy);
            vunique[2 * o] /= n;
            vunique[2 * o + 1] /= n;
        }
    free(acc);
    free(w);
    return nthreads;
}

int orc_fx_multi(int C, int L, int T, const double *volt, const double *gains,
                 double *vunique) {
    const int N = L * L, W = 2 * L - 1;
    int nthreads = 1;
#pragma omp parallel
    {
#ifdef _OPENMP
#pragma omp single
        nthreads = omp_get_num_threads();
#endif
#pragma omp for schedule(dynamic, 1)
        for (int c = 0; c < C; ++c)
            orc_fx(L, T, volt + 2 * (size_t)c * T * N, gains ? gains + 2 * (size_t)c * N : NULL,
                   vunique + 2 * (size_t)c * W * W, NULL);
    }
    return nthreads;
}

void orc_dft(int L, int M, int T, const double *volt, const double *gains,
             double *vunique, double *pk) {
    const int N = L * L, W = 2 * L - 1;
    double *P = (double *)calloc((size_t)M * M, sizeof(double));
    double *w = (double *)malloc(sizeof(double) * 2 * N);
    for (int t = 0; t < T; ++t) {
        for (int i = 0; i < N; ++i)
            calibrated(volt + 2 * ((size_t)t * N + i), gains ? gains + 2 * i : NULL, w + 2 * i);
        /* X(k) = sum_r w(r) exp(-2 pi i k.r / M), accumulate |X|^2 */
        for (int ky = 0; ky < M; ++ky)
            for (int kx = 0; kx < M; ++kx) {
                double xr = 0.0, xi = 0.0;
                for (int y = 0; y < L; ++y)
                    for (int x = 0; x < L; ++x) {
                        double ph = -2.0 * ORC_PI * (double)((kx * x + ky * y) % M) / (double)M;
                        double c = cos(ph), s = sin(ph);
                        const double *a = w + 2 * (y * L + x);
                        xr += a[0] * c - a[1] * s;
                        xi += a[0] * s + a[1] * c;
                    }
                P[ky * M + kx] += xr * xr + xi * xi;
            }
    }
    /* R(d) = (1/M^2) sum_k P(k) exp(+2 pi i k.d / M); V(d) = R(d)/(T N_d) */
    for (int dy = -(L - 1); dy <= L - 1; ++dy)
        for (int dx = -(L - 1); dx <= L - 1; ++dx) {
            double rr = 0.0, ri = 0.0;
            for (int ky = 0; ky < M; ++ky)
                for (int kx = 0; kx < M; ++kx) {
                    int e = ((kx * dx + ky * dy) % M + M) % M;
                    double ph = 2.0 * ORC_PI * (double)e / (double)M;
                    rr += P[ky * M + kx] * cos(ph);
                    ri += P[ky * M + kx] * sin(ph);
                }
            double s = 1.0 / ((double)M * M * (double)T * n_redundant(L, dx, dy));
            int o = (dy + L - 1) * W + (dx + L - 1);
            vunique[2 * o] = rr * s;
            vunique[2 * o + 1] = ri * s;
        }
    if (pk) memcpy(pk, P, sizeof(double) * M * M);
    free(w);
    free(P);
}

void orc_lag(int L, int T, const double *volt, const double *gains, int dx, int dy,
             double *out) {
    const int N = L * L;
    double re = 0.0, im = 0.0;
    int n = 0;
    /* pairs with r_i - r_j = (dx, dy): r_j = (x, y), r_i = (x + dx, y + dy) */
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int xi_ = x + dx, yi_ = y + dy;
            if (xi_ < 0 || xi_ >= L || yi_ < 0 || yi_ >= L) continue;
            int i = yi_ * L + xi_, j = y * L + x;
            ++n;
            for (int t = 0; t < T; ++t) {
                double a[2], b[2];
                calibrated(volt + 2 * ((size_t)t * N + i), gains ? gains + 2 * i : NULL, a);
                calibrated(volt + 2 * ((size_t)t * N + j), gains ? gains + 2 * j : NULL, b);
                re += a[0] * b[0] + a[1] * b[1];
                im += a[1] * b[0] - a[0] * b[1];
            }
        }
    out[0] = n ? re / ((double)T * n) : 0.0;
    out[1] = n ? im / ((double)T * n) : 0.0;
}

void orc_autos_c64(int N, int T, const double *volt, int t0, int t1, double *autos) {
    for (int i = 0; i < N; ++i) {
        double s = 0.0;
        for (int t = t0; t < t1 && t < T; ++t) {
            const double *a = volt + 2 * ((size_t)t * N + i);
            s += a[0] * a[0] + a[1] * a[1];
        }
        autos[i] = s;
    }
}
