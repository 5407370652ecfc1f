/*
 * gridcorr -- C ABI of a GB300 (sm_103a) implementation of the self-contained
 * O(N log N) correlator system for redundant arrays on a regular grid
 * (Gorthi, Parsons & Dillon 2020, "Calibration schemes with O(N log N)
 * scaling for large-N radio interferometers built on a regular grid").
 *
 * The system (paper Fig. 1b) has three data-parallel parts:
 *   correlate : gains + antenna voltages -> V^unique  (FFT-correlator)
 *   reduce    : voltages + selection      -> V^reduced (calibrator step (a))
 *   calibrate : V^reduced + redundancy    -> gains      (calibrator step (b))
 *
 * Conventions used by every entry point:
 *   - antennas sit on an L x L unit grid; antenna i is at r_i = (x, y) with
 *     i = y*L + x (row major);
 *   - complex numbers are interleaved (re, im) float32 ("c64");
 *   - a 4+4-bit complex ("i4c") is one byte: high nibble = Re, low nibble =
 *     Im, both two's complement in [-8, 7] (the quantiser emits [-7, 7]);
 *   - voltages are [C][T][N] (channel, time sample, antenna), contiguous;
 *   - the visibility of the ordered pair (i, j) is <v_i v_j^*> and belongs
 *     to the baseline-type d = r_i - r_j (paper Eq. redcal, d = r_0 - r_1);
 *   - every data buffer is caller-owned DEVICE memory unless a comment says
 *     HOST; the library never frees caller memory;
 *   - calls are asynchronous on the CUDA stream passed as `stream`
 *     (a cudaStream_t; NULL = the legacy default stream).  The returned
 *     status covers argument validation and launch errors; errors detected
 *     by the device (a bounded wait that ran out) are reported by
 *     gc_device_status().
 *   - no call allocates device memory except where stated (the context's
 *     scratch workspace grows on demand and is released by gc_destroy).
 */
#ifndef GRIDCORR_H
#define GRIDCORR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GC_API __attribute__((visibility("default")))
#else
#define GC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gc_status {
    GC_OK = 0,
    GC_EINVAL = 1,        /* bad argument (null pointer, size, alignment) */
    GC_ENOMEM = 2,        /* device workspace allocation failed */
    GC_ECUDA = 3,         /* a CUDA runtime / driver call failed */
    GC_ENOCONV = 4,       /* a solver hit its iteration cap */
    GC_ETIMEOUT = 5,      /* a device-side bounded wait ran out */
    GC_EDEGEN = 6,        /* selection does not meet the degeneracy criterion */
    GC_EUNSUPPORTED = 7   /* size / format combination not built */
} gc_status;

typedef enum gc_vfmt {
    GC_C64 = 0,           /* complex64: 8 bytes per antenna-sample */
    GC_I4C = 1,           /* 4+4-bit complex: 1 byte per antenna-sample
                             (two's-complement Re in the high nibble, Im in the low) */
    GC_C32H = 2           /* binary16 pair (Re, Im): 4 bytes per antenna-sample; the
                             FP16-storage variant -- arithmetic stays FP32.
                             Accepted by the correlators and gc_reduce. */
} gc_vfmt;

typedef struct gc_ctx gc_ctx;

/* Create a context bound to CUDA device `device`.  Allocates a 4-byte device
 * status word (cudaMalloc).  *out is set to NULL on failure. */
GC_API gc_status gc_create(gc_ctx **out, int device);

/* Release the context and its workspace.  Safe on NULL. */
GC_API void gc_destroy(gc_ctx *ctx);

/* Human-readable description of the last error on this context ("" if none).
 * The pointer stays valid until the next call on the context. */
GC_API const char *gc_last_error(const gc_ctx *ctx);

/* Synchronise `stream`, read and clear the device-side error word.  Returns
 * GC_ETIMEOUT if a kernel gave up a bounded wait since the last check, and
 * GC_EINVAL if a kernel met a zero or non-finite gain, or voltages whose
 * sums were not finite (NaN or infinity in the input). */
GC_API gc_status gc_device_status(gc_ctx *ctx, void *stream);

/* Launch timing (not part of the paper's method; used by benchmarks).
 * When enabled, the library records a CUDA event pair on the launching
 * stream around every kernel it enqueues.  gc_profile_read synchronises on
 * those events, writes per-kernel-kind totals (names: 64-byte slots,
 * NUL-terminated; total milliseconds; launch counts) for up to max_kinds
 * kinds, clears the records and returns the number of kinds (-1 on a bad
 * argument).  Any of names / total_ms / launches may be NULL. */
GC_API gc_status gc_profile_enable(gc_ctx *ctx, int enable);
GC_API int gc_profile_read(gc_ctx *ctx, char *names, double *total_ms, int *launches,
                           int max_kinds);

/* Arithmetic throughput probe (not part of the paper's method; used for
 * roofline denominators).  kind 0: FP32 FMA, kind 1: FP64 FMA, kind 2: 4-way
 * signed 8-bit dot product with int32 accumulate (dp4a), kind 3: dense FP8
 * tensor-core MMA (tcgen05 kind::f8f6f4, e4m3 x e4m3 -> FP32, M = 128,
 * N = 256, K = 32, one CTA per SM, operands resident in shared memory),
 * kind 4: warp-level int8 MMA (mma.sync m16n8k32 s8 x s8 -> s32).
 * Launches a kernel on the context's device (legacy default stream),
 * synchronises, and writes the achieved tera-operations per second (FMA = 2
 * flops; dp4a = 8 integer ops; MMA = 2 M N K).  GC_EINVAL for another kind. */
GC_API gc_status gc_peak_probe(gc_ctx *ctx, int kind, double *tflops);

/* Smallest FFT side M for an L x L grid: the smallest power of two >= 2L - 1,
 * so that the circular correlation of the zero-padded grid equals the
 * linear one (paper Sec. 1, convolution theorem).  gc_correlate uses
 * max(16, gc_fft_size(L)).  0 if L is out of range. */
GC_API int gc_fft_size(int L);

/*
 * FFT-correlator (paper Fig. 1b yellow box; Sec. 1; Eq. modelvis).
 *
 * For every channel c: calibrate the voltages with the gains (w_i = v_i /
 * g_i), take the zero-padded M x M spatial FFT of w at every time sample,
 * integrate |X(k)|^2 over the T samples, inverse-FFT, and normalise each lag
 * by T * N_d, giving the redundant average of Eq. modelvis:
 *
 *   V^unique_c(d) = 1/(T N_d) sum_t sum_{r_i - r_j = d} w_i(t) w_j(t)^*,
 *   N_d = (L - |dx|)(L - |dy|).
 *
 *   volt     [C][T][L*L] c64 (8-byte aligned), c32h (4-byte aligned) or
 *            i4c (device)
 *   gains    [C][L*L]    c64 (device); a zero or non-finite gain leaves
 *            that antenna out of the sums and makes gc_device_status return
 *            GC_EINVAL, as do voltages whose spectra are not finite
 *   vunique  [C][2L-1][2L-1] c64 (device), index [dy + L - 1][dx + L - 1]
 *   1 <= L <= 128, C >= 1, T >= 1 (GC_EINVAL otherwise); L > 64 (M = 256)
 *   is built for i4c only (GC_EUNSUPPORTED for c64 / c32h).
 * Voltages are staged by TMA when the buffer is 16-byte aligned and a grid
 * row is a multiple of 16 bytes (c64: L even; c32h: L % 4 == 0; i4c:
 * L % 16 == 0), by plain loads otherwise.
 * 4+4-bit voltages on grids of L = 40, 48, 56 or 64 (M = 128, 16-byte
 * aligned, unmasked) take the row stage of the FFT on the tensor cores
 * (tcgen05 kind::f16 products of binary16 hi/lo splits of the DFT matrix and
 * of w, FP32 accumulation; the column stage and |X|^2 on the CUDA cores);
 * the knob "fft.path" = 1 keeps them on the CUDA-core kernel.  Both meet the
 * same accuracy (lag sums within 1e-5 of the zero-lag power, FP64
 * reference).
 *
 * Uses the context's scratch workspace for per-time-chunk power spectra
 * (C * chunks * M^2 * 4 bytes, plus C * M * (2L-1) * 8 bytes for M = 256;
 * grown with cudaMalloc on first need, which synchronises the device).  Two
 * kernels (three for M = 256) are enqueued on `stream`.
 */
GC_API gc_status gc_correlate(gc_ctx *ctx, const void *volt, int vfmt, int L, int C, int T,
                       const float *gains, float *vunique, void *stream);

/*
 * Reduced redundant-baseline calibration selections (paper Sec. 4 and 5).
 *
 * A selection lists the baseline-types (d = (dx, dy), canonical half-plane
 * dy > 0 or dy == 0 and dx > 0, ordered by |d|^2 then by angle in [0, pi))
 * and, per type, its redundant pairs (i = r_j + d, j = r_j, reference
 * antenna r_j in row-major order) and the integration window [t0, t1) in
 * which they are correlated.  It doubles as the redundancy map of the
 * calibration.  Host objects; created without a GPU; device copies are made
 * on first use by gc_reduce / gc_calibrate (cudaMalloc, freed by
 * gc_sel_free).
 *
 * gc_selection_subset  (Sec. 5, Eq. subredcal_frac_bls, Sec. 6.1): whole
 *   types, shortest first, stopping at the cumulative pair count closest to
 *   p N log N (log to base `log_base`; 0 = natural); extended until the
 *   degeneracy criterion of Sec. 5.2 holds (null space = 4).  Window [0, T).
 *   GC_EDEGEN for L = 2 (never satisfiable), GC_EINVAL for L < 2, L > 256.
 * gc_selection_lowcad  (Sec. 4, Eq. lowcadcal_inttime): every type; types
 *   are packed first-fit, shortest first, into cycles of floor(p N log N)
 *   pairs; N_cycle cycles of t_int = floor(T / N_cycle) samples; the types of
 *   cycle c are integrated over [c t_int, (c + 1) t_int).  Holding every
 *   pair, it is refused with GC_EUNSUPPORTED past 2^28 pairs
 *   (N (N - 1) / 2 > 2^28: about 23 000 antennas, L > 152).
 * Every builder returns GC_ENOMEM when host memory runs out; no C++
 * exception leaves the library.
 */
typedef struct gc_sel gc_sel;
GC_API gc_status gc_selection_subset(int L, int T, double p, double log_base, gc_sel **out);
GC_API gc_status gc_selection_lowcad(int L, int T, double p, double log_base, gc_sel **out);

/*
 * The FFT-correlator for an array on a partly occupied lattice (layout as
 * gc_selection_subset_masked; the paper's hexagonal arrays, Sec. 3): as
 * gc_correlate on the L x L grid of lattice points, with the points where
 * mask[i] == 0 (host, L*L bytes) contributing nothing (their gains are not
 * read), and V^unique(d) = R(d) / (T N_d) with N_d the number of pairs of
 * occupied points at lattice separation d (computed on the host per call,
 * O(antennas^2)); lags without a pair are 0.  Uses the context workspace.
 */
GC_API gc_status gc_correlate_masked(gc_ctx *ctx, const void *volt, int vfmt, int L, int C, int T,
                                     const uint8_t *mask, const float *gains, float *vunique, void *stream);

/*
 * Subset selection for an array on a partly occupied lattice -- the paper's
 * own arrays are hexagonal (Sec. 3; Fig. 13's 331 antennas).  The array is
 * held as the L x L bounding grid of lattice points (point i = y L + x) with
 * mask[i] = 1 where an antenna sits (host, L*L bytes); voltages and gains
 * keep the grid layout, with anything at unoccupied points ignored.
 * lattice GC_LATTICE_SQUARE: unit spacing; GC_LATTICE_TRIANGULAR: basis
 * (1, 0), (1/2, sqrt(3)/2), so type (dx, dy) has squared length
 * dx^2 + dx dy + dy^2.  Types with a pair between occupied points are taken
 * whole, shortest first (ties by angle in [0, pi)), stopping at the count
 * closest to p N log N with N the occupied points, then extended until the
 * criterion of Sec. 5.2 holds: both axis types, and dx + dy even (square) or
 * (-1, 1) (triangular).  GC_EDEGEN when no prefix satisfies it or the axis
 * types do not connect the array; GC_EINVAL for a NULL mask, fewer than 3
 * antennas or the size limits of gc_selection_subset.  Works with
 * gc_reduce, gc_calibrate (GC_LINCAL_CG), gc_chi2 and gc_correlate_masked.
 */
typedef enum gc_lattice { GC_LATTICE_SQUARE = 0, GC_LATTICE_TRIANGULAR = 1 } gc_lattice;
GC_API gc_status gc_selection_subset_masked(int L, int T, double p, double log_base, const uint8_t *mask,
                                            int lattice, gc_sel **out);
/* Low-cadence selection (Sec. 4) on a partly occupied lattice: every type
 * with a pair between occupied points, packed as gc_selection_lowcad with
 * N the occupied points.  GC_EDEGEN when the axis types do not connect the
 * array; other errors (and the 2^28-pair limit) as gc_selection_lowcad. */
GC_API gc_status gc_selection_lowcad_masked(int L, int T, double p, double log_base, const uint8_t *mask,
                                            int lattice, gc_sel **out);
GC_API void gc_sel_free(gc_sel *sel);
/* info[11] = {L, T, P (pairs), n_ubl (types), n_cycle, t_int, null_dim,
 *             scheme (0 subset, 1 low-cadence), masked, lattice, antennas} */
GC_API gc_status gc_sel_info(const gc_sel *sel, int32_t *info);
/* Edge antennas of the selection's array (Sec. 5.4): edge[i] = 1 for an
 * occupied point with an unoccupied or outside nearest neighbour (4 on the
 * square lattice, 6 on the triangular one), else 0.  edge: host [L*L]. */
GC_API gc_status gc_sel_edge(const gc_sel *sel, uint8_t *edge);
/* Host arrays owned by the selection (valid until gc_sel_free): types [n_ubl][2],
 * type_ptr [n_ubl + 1] (pairs of type k are [type_ptr[k], type_ptr[k+1])),
 * pair_i, pair_j [P], win_t0, win_t1 [n_ubl].  Any output may be NULL. */
GC_API gc_status gc_sel_arrays(const gc_sel *sel, const int32_t **types, const int32_t **type_ptr,
                               const int32_t **pair_i, const int32_t **pair_j,
                               const int32_t **win_t0, const int32_t **win_t1);

/*
 * Reduced X-engine (paper Fig. 1 calibrator step (a); Sec. 4 windows).
 *
 *   S_p = sum_{t in [t0_p, t1_p)} v_{i_p}(t) v_{j_p}(t)^*     (raw sums)
 *   A_i = sum_{t in [0, N_cycle t_int)} |v_i(t)|^2            (autos)
 *
 *   volt      [C][T][L*L] c64, c32h or i4c (device), T >= the selection's T
 *   vreduced  c64 / c32h: [C][P] c64 (FP32 sums); i4c: [C][P][2] int32, exact
 *   autos     c64 / c32h: [C][L*L] float; i4c: [C][L*L] int32; may be NULL
 * Non-finite complex64 / binary16 sums make gc_device_status return
 * GC_EINVAL.
 * 4+4-bit voltages of a subset selection (one window, at most 16 types) on
 * an L = 16, 32 or 64 grid whose halo 128 + dy_max L is at most 256 antennas
 * run on the tensor cores (tcgen05 FP8 MMAs on exact integer codes, equal bit
 * for bit to the SIMT path); the tuning knob "xeng.path" forces the SIMT
 * path (1) or the tensor cores (2; GC_EUNSUPPORTED where they do not apply).
 * Uses the context workspace (time-slice partial sums).  Two kernels.
 */
GC_API gc_status gc_reduce(gc_ctx *ctx, const void *volt, int vfmt, int L, int C, int T,
                           const gc_sel *sel, void *vreduced, void *autos, void *stream);

/*
 * 4+4-bit quantiser (the precision variant of the voltage path; the paper
 * does not quantise).  Per channel c: rms_c = sqrt(sum (re^2 + im^2) /
 * (2 T N)) in FP64, scale_c = (float)(3 / rms_c) (RMS of 3 levels per
 * component), q = clip(round_half_away(x * scale_c rounded to float), -7, 7),
 * byte = (q_re << 4) | (q_im & 15).
 *   volt   [C][T][N] c64 (device, 16-byte aligned), T * N even
 *   out    [C][T][N] bytes (device)
 *   scales [C] float (device) or NULL
 */
GC_API gc_status gc_quantize(gc_ctx *ctx, const float *volt, int C, int T, int N, uint8_t *out,
                             float *scales, void *stream);

/*
 * Per-channel redundant-baseline calibration (paper Sec. 2 Eq. redcal;
 * lincal and omnical, Sec. 2 and Sec. 3; degeneracies Sec. 5.2; chi^2_r and
 * DoF, Eq. redchi / Eq. dof).
 *
 * For every channel, V_p = S_p / t_p (the X-engine sums divided by the
 * pair's window length) and the model V_p ~ g_i conj(g_j) V_alpha(p) is
 * fitted by least squares with uniform weights (Eq. noisecov):
 *   GC_LINCAL  Gauss-Newton on (Re, Im) of every gain and model visibility;
 *              banded normal equations (antennas row-major), FP64 (GC_FP64)
 *              or FP32 (GC_FP32); the four degeneracies are projected out
 *              of each step; up to 64 baseline-types (subset selections).
 *   GC_OMNICAL damped simultaneous least-squares fixed point (damping 0.3
 *              by default, Sec. 3), FP32; any selection (low-cadence).
 *   GC_LINCAL_CG Gauss-Newton with the step from conjugate gradients on
 *              J^T J, preconditioned by Jacobi plus a patch-level coarse
 *              space, matrix-free (per-antenna gather over the grid, or a
 *              scatter over the pair list: "cal.operator"), FP32 products
 *              with FP64 reductions; inexact-Newton CG tolerance
 *              min(0.05, (|grad| / |grad_0|)^(1/4)) relative residual (at
 *              least 1e-4), at most 500 CG iterations per step; channels are
 *              taken from a device counter (the call enqueues a memset before
 *              the kernel); any selection, and the only solver for partly
 *              occupied lattices.
 * Start point (unless warm_start): spanning-tree phases over the (1,0) and
 * (0,1) types, unit amplitudes, group-mean model visibilities.  Warm start
 * reads gains and vmodel as given.
 * Output convention for the degeneracies: mean ln|g| = 0, arg g_0 = 0,
 * arg V_(1,0) = arg V_(0,1) = 0.
 *
 *   vreduced  gc_reduce output (c64 [C][P] or i4c [C][P][2] int32)
 *   autos     gc_reduce autos or NULL (then chi2r = -1)
 *   gains     [C][L*L] c64 (device, out; in for warm start)
 *   vmodel    [C][n_ubl] c64 (device, out; in for warm start)
 *   stats     [C] gc_calstats (device): chi2 = sum |V_p - model|^2,
 *             chi2r = sum |r|^2 / sigma_p^2 / DoF with the radiometer
 *             sigma_p^2 = (A_i/T_a)(A_j/T_a)/t_p, DoF = P - N - n_ubl + 2,
 *             iters, status (GC_OK, GC_ENOCONV at max_iter, GC_ETIMEOUT past
 *             time_limit_ms, GC_EDEGEN on a non-positive pivot, GC_EINVAL
 *             when the channel's V^reduced or its solution is not finite).
 * Zero-valued option fields select the defaults: max_iter 50 (lincal) /
 * 20000 (omnical), tol 1e-10 (lincal FP64) / 1e-6 (otherwise), damping
 * 0.3, time_limit_ms 10000 per channel.  Uses the context workspace.
 */
typedef enum gc_solver { GC_LINCAL = 0, GC_OMNICAL = 1, GC_LINCAL_CG = 2 } gc_solver;
typedef enum gc_precision { GC_FP64 = 0, GC_FP32 = 1 } gc_precision;
typedef struct gc_calopts {
    int solver;        /* gc_solver */
    int precision;     /* gc_precision (lincal) */
    int max_iter;
    int warm_start;
    double tol;        /* relative step / change */
    double damping;    /* omnical */
    int time_limit_ms; /* per channel, device-side */
    int fp32_reductions; /* GC_LINCAL_CG with the grid-gather operator: 1 = every
                            reduction in FP32 too (the plain-FP32 form), 0 = the
                            chi^2 and step norms in FP64 (default) */
} gc_calopts;
typedef struct gc_calstats {
    double chi2;
    double chi2r;
    int dof;
    int iters;
    int status;
    int inner;   /* GC_LINCAL_CG: total conjugate-gradient iterations; else 0 */
} gc_calstats;
GC_API gc_status gc_calibrate(gc_ctx *ctx, const void *vreduced, int vfmt, const gc_sel *sel, int C,
                              const void *autos, const gc_calopts *opts, float *gains, float *vmodel,
                              gc_calstats *stats, void *stream);

/*
 * Batched calibration: several arrays of different size (each with its own
 * selection, channel count and buffers, as for gc_calibrate) in one
 * persistent launch.  CTAs take (array, channel) work items from a device
 * counter, arrays ordered by decreasing cost (pairs + 4 N) unless the
 * "cal.order" tuning knob is 1.  The solver is GC_LINCAL_CG (other solver
 * fields of opts are ignored); results equal those of gc_calibrate with
 * GC_LINCAL_CG.  At most 32 arrays.  Enqueues a memset and one kernel, so
 * after a first call that has sized the workspace the call can be captured
 * into a CUDA graph.
 */
typedef struct gc_batch_item {
    const gc_sel *sel;
    int C;
    int vfmt;
    const void *vreduced;
    const void *autos;
    float *gains;
    float *vmodel;
    gc_calstats *stats;
} gc_batch_item;
GC_API gc_status gc_calibrate_batched(gc_ctx *ctx, int n_arrays, const gc_batch_item *items,
                                      const gc_calopts *opts, void *stream);

/*
 * Predicted calibration variances of a selection (Eq. gaincov, the
 * uniform-noise form of Eq. noisecov): for every unknown u -- antennas
 * u < L*L, then model visibilities u = L*L + k -- the diagonal entry of the
 * pseudo-inverse of Eq. logcal's normal matrices, amplitude [(A^T A)^+]_uu
 * into var_amp[u] and phase [(B^T B)^+]_uu into var_phase[u] (device float
 * arrays of L*L + n_ubl; the four degeneracies of Sec. 5.2 are left out,
 * empty points of a partly occupied lattice get 0).  With per-visibility
 * noise variance sigma^2 the gain variance is sigma^2 (var_amp + var_phase)
 * / 2 per unit gain (|V| = 1); sum over antennas for the array mean, or
 * leave out edge antennas as the paper's Sec. 5.4 does.  One FP64
 * Jacobi-preconditioned conjugate-gradient solve per unknown on the GPU
 * (relative residual 1e-8, at most 4000 iterations; an unknown whose solve
 * does not get there reads NaN).  The cost grows as unknowns x iterations x
 * pairs: meant for arrays of hundreds of antennas.  GC_EDEGEN for a
 * selection with more than the four degeneracies.  Uses the context
 * workspace.
 */
GC_API gc_status gc_gain_variance(gc_ctx *ctx, const gc_sel *sel, float *var_amp, float *var_phase,
                                  void *stream);

/*
 * Gain covariance rows (Eq. gaincov; covariance rows and matrices of
 * Sec. 5.3, Figs. 7-8), in the units of gc_gain_variance (per unit noise;
 * multiply by sigma^2 / 2 for the covariance of the log-amplitude and phase
 * errors).
 *   fixed = 0: rows[r] is an unknown (antenna < L*L, then types); row r of
 *              the pseudo-inverses, cov_amp[r][u] = [(A^T A)^+]_{rows[r],u}
 *              and cov_phase[r][u] = [(B^T B)^+]_{rows[r],u},
 *              u < L*L + n_ubl;
 *   fixed = 1: rows[r] is an antenna; the antenna covariance after the
 *              four degeneracies are fixed against the true gains by least
 *              squares over the antennas (how the paper's simulations
 *              compare gains, Sec. 3): P (A^T A)^+ P and P (B^T B)^+ P
 *              restricted to the antennas, P the projector off the
 *              antenna-space degeneracy directions (amplitude: constant;
 *              phase: constant, x, y), u < L*L.
 * rows: host [n_rows], read before the call returns.  cov_amp, cov_phase:
 * device float [n_rows][row length].  Empty points of a partly occupied
 * lattice read 0; a row whose solve does not converge reads NaN (same
 * solver and limits as gc_gain_variance, one solve per row).  The amplitude
 * plus phase sum of a row is the quantity Figs. 7-8 plot.  GC_EINVAL for a
 * row out of range, GC_EDEGEN as gc_gain_variance.  Uses the context
 * workspace.
 */
GC_API gc_status gc_gain_covariance(gc_ctx *ctx, const gc_sel *sel, int fixed, int n_rows,
                                    const int32_t *rows, float *cov_amp, float *cov_phase, void *stream);

/*
 * Variance of calibrated redundant visibilities (Sec. 6.2): for every lag
 * alpha = (dx, dy) of the full array (plane [(2L-1)^2], index
 * (dy + L - 1)(2L - 1) + dx + L - 1), the relative variance SNR^-2 of
 * V^unique_alpha, the redundant average of the N_alpha full-array pairs
 * (i, j = i + alpha) calibrated with gains from this selection's
 * calibrator.  Gains and visibilities of unit amplitude (the paper's own
 * simplification before Eq. visvar); each full-array visibility has
 * SNR^-2 = snr_full_inv2; the calibrator's visibilities have noise
 * variance sigma_cal2 (relative), independent of the former, so that the
 * log-gain errors a = eta + i phi have covariance (sigma_cal2 / 2) C_a and
 * (sigma_cal2 / 2) C_p, with C the fixed-degeneracy antenna covariance of
 * gc_gain_covariance (fixed = 1).
 *   var_pair[alpha]  = (1 / N_a^2) sum_{(i,j) in alpha} [snr_full_inv2
 *                      + s_i + s_j + 2 rho_ij], the per-pair form before
 *                      Eq. visvar, s_i = E|a_i|^2 and rho_ij =
 *                      Re E[a_i a_j] = Cov(eta_i, eta_j) - Cov(phi_i, phi_j)
 *                      (the covariance term of a calibrated visibility
 *                      V_ij / (g_i conj(g_j)));
 *   var_exact[alpha] = (1 / N_a^2) [N_a snr_full_inv2 + (sigma_cal2 / 2)
 *                      (u^T C_a u + w^T C_p w)], u = sum (e_i + e_j),
 *                      w = sum (e_i - e_j) over the lag's pairs: the full
 *                      linearised variance, with the covariance between
 *                      different pairs that the paper's form leaves out
 *                      (NULL to skip);
 *   n_pairs[alpha]   = N_alpha (NULL to skip).
 * Outputs are device arrays; lag 0 and lags without pairs read NaN (n 0).
 * Cost: L*L covariance solves, then (2L-1)^2 x (L*L)^2 multiply-adds; meant
 * for arrays up to about a thousand antennas.  Workspace: 8 (L*L)^2 bytes
 * plus the solver's.  GC_EINVAL for negative or NaN variances, GC_EDEGEN as
 * gc_gain_variance.
 */
GC_API gc_status gc_visibility_variance(gc_ctx *ctx, const gc_sel *sel, double snr_full_inv2,
                                        double sigma_cal2, double *var_pair, double *var_exact,
                                        int32_t *n_pairs, void *stream);

/*
 * Tuning knobs of a context (0 = automatic), set by the autotuner:
 *   "fft.chunk_len"    time samples per FFT-correlator work item
 *   "xeng.tsplit"      time slices per X-engine window
 *   "cal.ctas_per_sm"  resident calibration CTAs per SM (cap)
 *   "cal.order"        batched work order: 0 largest first, 1 as given
 *   "cal.operator"     GC_LINCAL_CG operator: 0 per-antenna gather over the
 *                      grid (selections of <= 16 baseline-types; others
 *                      fall back to 1), 1 scatter over the pair list
 *   "xeng.path"        gc_reduce for 4+4-bit voltages: 0 tensor cores where
 *                      they apply, 1 integer SIMT (dp4a), 2 tensor cores only
 *   "xeng.tc_shape"    tensor-core X-engine launch shape (0 default; 1-4:
 *                      converter warps and ring depths)
 *   "fft.shape"        FFT-correlator launch shape: 0 default, 1 the
 *                      alternative sample grouping built for the 64x64
 *                      4+4-bit and 32x32 complex64 grids (others ignore it)
 *   "fft.path"         FFT-correlator for 4+4-bit voltages with M = 128: 0
 *                      row stage on the tensor cores where it applies, 1
 *                      CUDA cores only
 * GC_EINVAL for an unknown name or a negative value.
 */
GC_API gc_status gc_set_tuning(gc_ctx *ctx, const char *name, int value);
GC_API gc_status gc_get_tuning(const gc_ctx *ctx, const char *name, int *value);

/*
 * chi^2 of the redundant model and its adjoint (numerator of Eq. redchi;
 * the differentiable form of the calibration objective).
 *
 *   chi2[c] = sum_p w_p |V_p - g_i conj(g_j) V_alpha(p)|^2,  V_p = S_p / t_p
 *
 *   vreduced  gc_reduce output for `sel`; gains [C][L*L] c64; vmodel
 *   [C][n_ubl] c64; weights [C][P] float or NULL (uniform); chi2 [C] double.
 * gc_chi2_backward writes, scaled by grad_out[c] (dL/dchi2_c; NULL = 1):
 *   grad_gains[c][k]  = dchi2/dRe g_k + i dchi2/dIm g_k
 *                     = -2 [sum_{i_p=k} w r g_j conj(V) + sum_{j_p=k} w conj(r) g_i V]
 *   grad_vmodel[c][a] = -2 sum_{p in a} w r conj(g_i) g_j
 * recomputing the residuals from (gains, vmodel).  FP32 products; sums of at
 * most 32 terms in FP32, longer sums in FP64.  Selections of at most 16
 * baseline-types on a full grid split each channel's antennas over several
 * CTAs and keep their partial sums in the context workspace (a second small
 * kernel adds them in a fixed order, so results do not vary between runs).
 */
GC_API gc_status gc_chi2(gc_ctx *ctx, const void *vreduced, int vfmt, const gc_sel *sel, int C,
                         const float *gains, const float *vmodel, const float *weights, double *chi2,
                         void *stream);
GC_API gc_status gc_chi2_backward(gc_ctx *ctx, const void *vreduced, int vfmt, const gc_sel *sel,
                                  int C, const float *gains, const float *vmodel,
                                  const float *weights, const double *grad_out, float *grad_gains,
                                  float *grad_vmodel, void *stream);

/*
 * Checkpointed form of the pair above: gc_chi2_ckpt also stores the
 * residuals r_p = V_p - g_i conj(g_j) V_alpha (unweighted, c64 [C][P],
 * device, 8-byte aligned), and gc_chi2_backward_ckpt computes the same
 * gradients from them instead of re-evaluating the model (V^reduced is not
 * read).  The residuals cost 8 * P * C bytes, e.g. 0.92 GB for 512 channels
 * of the 128x128 subset selection.  GC_EINVAL for null outputs.
 */
GC_API gc_status gc_chi2_ckpt(gc_ctx *ctx, const void *vreduced, int vfmt, const gc_sel *sel, int C,
                              const float *gains, const float *vmodel, const float *weights, double *chi2,
                              float *residuals, void *stream);
GC_API gc_status gc_chi2_backward_ckpt(gc_ctx *ctx, const float *residuals, const gc_sel *sel, int C,
                                       const float *gains, const float *vmodel, const float *weights,
                                       const double *grad_out, float *grad_gains, float *grad_vmodel,
                                       void *stream);

/*
 * One integration of HOST-resident voltages through the whole cycle of the
 * paper's Fig. 1: FFT-correlator (gc_correlate), reduced X-engine
 * (gc_reduce) and calibration (gc_calibrate), streamed in chunks of
 * `chunk` channels (0: automatic, about eight chunks; the first chunk is a
 * quarter of `chunk`, so that little copy time precedes the first kernel).
 * The host->device copy of the next chunk, on a copy stream owned by the
 * context, overlaps the kernels of the current one on `stream`; one
 * calibration launch over all C channels follows the last chunk.  A staging
 * buffer is refilled as soon as the last kernel that read it has finished,
 * so the first copies of the next call overlap this call's calibration.  (No
 * paper counterpart: this is the data path of a correlator whose voltages
 * arrive from the host.)
 *
 *   h_volt    [C][T][L*L] host memory, c64 / c32h / i4c as gc_correlate;
 *             page-locked memory lets the copies overlap (pageable memory
 *             works, with synchronous copies)
 *   gains_in  [C][L*L] c64: the gains the correlator applies, in device
 *             memory or in HOST memory (page-locked for an asynchronous
 *             copy); host gains are copied on the copy stream ahead of the
 *             first chunk into a context buffer (allocated on first need)
 *   vunique   [C][2L-1][2L-1] c64 device (output)
 *   vreduced, autos  device outputs as gc_reduce (autos may be NULL)
 *   opts      calibration options (NULL: defaults); gains_out [C][L*L],
 *             vmodel [C][n_ubl], stats [C]: device outputs as gc_calibrate
 * The context allocates three device staging buffers of chunk * T * L*L
 * voltage elements on first need (cudaMalloc, which synchronises the
 * device) and keeps them.  Everything is enqueued; the call returns when
 * the work is queued.  The staging buffers and h_volt must not be modified
 * until `stream` has completed the call's work.  Errors as the three calls.
 * With gc_profile_enable, each chunk's host->device copy is recorded as
 * "h2d_chunk" (events on the copy stream).
 */
GC_API gc_status gc_integrate_host(gc_ctx *ctx, const void *h_volt, int vfmt, int L, int C, int T,
                                   const gc_sel *sel, const float *gains_in, float *vunique, void *vreduced,
                                   void *autos, const gc_calopts *opts, float *gains_out, float *vmodel,
                                   gc_calstats *stats, int chunk, void *stream);

/*
 * FFT-correlator that allocates no device memory.  The paper has no
 * counterpart: this is an interface for callers that cannot call cudaMalloc
 * -- for example a real-time correlator process whose device memory is
 * fixed when the observation starts (cudaMalloc and cudaFree can
 * synchronise the whole device and stall the streams that keep up with the
 * telescope), or a host framework that owns every device allocation and
 * hands the library only the buffers it already holds.
 *
 * Same computation, arguments and layouts as gc_correlate (for 1 <= L <= 64),
 * with no context:
 * the per-chunk power spectra live in a fixed 64 MiB array in the library's
 * device memory (every GPU that loads the library holds it until the
 * process exits).  The call is rejected with GC_EINVAL when
 *     C * ceil(T / 512) * M^2 * 4 bytes > 64 MiB
 * (M = max(16, gc_fft_size(L)));
 * e.g. L = 32, T = 4096 allows up to 512 channels per call.
 *
 * Every call looks up the device address of that array on the current
 * device (cudaGetSymbolAddress, which enqueues nothing; the first call on a
 * device also loads the library's device code and the tensor-map encoder, so
 * make that first call before any stream capture).  Apart from the lookup a
 * call only enqueues two kernels on `stream`.
 *
 * `status` (optional, device, caller-zeroed) receives the device-side error
 * bits of the call (non-zero = a bounded wait ran out and the output is
 * incomplete, or a gain or voltage was zero or not finite); NULL sends them to
 * a word of the library that is not reported, so with NULL such a call still
 * returns GC_OK and its output can hold spectra an earlier call left in the
 * shared array.  All calls on a device share the one scratch array, and each
 * call overwrites every element it later reads, so nothing has to be cleared
 * between calls; calls that overlap on the GPU (different streams without
 * ordering between them) race on the array and give wrong results.
 *
 * Returns GC_EINVAL for bad arguments or sizes beyond the fixed scratch,
 * GC_ECUDA when a CUDA call fails, GC_EUNSUPPORTED for an unbuilt size.
 */
GC_API gc_status gc_correlate_noalloc(const void *volt, int vfmt, int L, int C, int T,
                                      const float *gains, float *vunique, unsigned int *status,
                                      void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GRIDCORR_H */
