"""Oracle: gain covariance and the variance of calibrated redundant
visibilities, in FP64 numpy.

TEST INFRASTRUCTURE ONLY: the library's product path never imports this
module, and this module imports nothing from the library.

Paper basis:
  * gain covariance (Eq. cov, Eq. noisecov, Eq. gaincov): with noise of
    variance sigma^2 on every complex visibility (|V| = 1), Eq. logcal's
    real and imaginary parts each carry sigma^2 / 2, so the log-amplitude
    errors eta have covariance (sigma^2 / 2) (A^T A)^+ and the phase errors
    phi (sigma^2 / 2) (B^T B)^+, the four degeneracies (Sec. 5.2) left out
    by the pseudo-inverse;
  * covariance rows and matrices (Sec. 5.3, Figs. 7 and 8): the sum of the
    amplitude and phase covariance of one antenna with every other;
  * edge antennas (Sec. 5.4): antennas on the rim of the array take part in
    fewer cross-correlations and get larger variances; the statistic leaves
    them out;
  * variance of calibrated redundant visibilities (Sec. 6.2): the general
    per-pair form (the equation before Eq. visvar), Eq. visvar,
    Eq. visvar_lowcadcal and Eq. visvar_subredcal.

Readings where the paper is loose (stated in the design notes):
  * rho_{g_i g_j}.  A calibrated visibility is V_ij / (g_i conj(g_j)); with
    a = delta g / g = eta + i phi its relative error is -(a_i + conj(a_j)),
    whose variance is E|a_i|^2 + E|a_j|^2 + 2 Re E[a_i a_j].  The covariance
    term that makes the paper's bracket this variance is
    rho_ij = Re E[a_i a_j] = Cov(eta_i, eta_j) - Cov(phi_i, phi_j),
    and that is the reading here (for Figs. 7-8, which plot the plain sum of
    the amplitude and phase covariance, gain_covariance returns both parts);
  * the per-pair form keeps only the terms of one pair at a time, as the
    paper writes it; visvar_exact adds the covariances between different
    pairs of the same baseline-type (the full linearised variance of the
    redundant average), which the paper's "approximately" leaves out;
  * gains and visibilities have unit amplitude (the paper's own
    simplification before Eq. visvar), the full-array pairs all have the
    same SNR, and the calibrator's noise is independent of the noise in the
    visibilities that the gains are applied to;
  * an edge antenna is an occupied lattice point with at least one
    unoccupied (or outside) nearest-neighbour point: 4 neighbours on the
    square lattice, 6 on the triangular lattice of hexagonal arrays;
  * log N in Eq. visvar_lowcadcal and Eq. visvar_subredcal is to base 2,
    as in the selections' pair budget p N log2 N.
"""
from __future__ import annotations

import numpy as np

from . import calib


# ----------------------------------------------------------- gain covariance
def gain_covariance(L, types, pi, pj, alpha, N=None):
    """(A^T A)^+ and (B^T B)^+ of Eq. logcal for a selection: the full
    (N + n_ubl) x (N + n_ubl) matrices whose (sigma^2 / 2)-multiples are the
    covariances of the log-amplitude and phase errors (Eq. gaincov).
    Unknowns: antennas 0..N-1, then baseline-types."""
    N = L * L if N is None else N
    AtA, BtB = calib.logcal_normal_matrices(N, types, pi, pj, alpha)
    # the four exact degeneracies are singular values at rounding level;
    # the cut-off leaves them out (as in calib.gain_variance_prediction)
    ca = np.linalg.pinv(AtA, rcond=1e-9, hermitian=True)
    cb = np.linalg.pinv(BtB, rcond=1e-9, hermitian=True)
    return ca, cb


def covariance_rows(ca, cb, rows):
    """Rows of the gain covariance for the unknowns `rows`: the amplitude and
    phase parts, and their sum as plotted in Figs. 7-8."""
    rows = np.asarray(rows, np.int64)
    return ca[rows], cb[rows], ca[rows] + cb[rows]


# ---------------------------------------------------------------- lags
def lattice_neighbours(lattice="square"):
    """Unit steps to the nearest lattice neighbours (grid coordinates; the
    triangular lattice is stored sheared, its sixth neighbours at (1, -1)
    and (-1, 1))."""
    if lattice == "square":
        return [(1, 0), (-1, 0), (0, 1), (0, -1)]
    return [(1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1)]


def lag_index(L, dx, dy):
    """Position of lag (dx, dy) in a (2L-1) x (2L-1) plane, dy-major."""
    return (dy + L - 1) * (2 * L - 1) + (dx + L - 1)


def full_array_pairs(L, dx, dy, mask=None):
    """All pairs (i, j) of the full array with pos(j) - pos(i) = (dx, dy),
    both points occupied: the N_alpha redundant baselines of one type."""
    occ = np.ones(L * L, bool) if mask is None else np.asarray(mask, bool).reshape(-1)
    ii, jj = [], []
    for y in range(L):
        for x in range(L):
            x2, y2 = x + dx, y + dy
            if 0 <= x2 < L and 0 <= y2 < L:
                i, j = y * L + x, y2 * L + x2
                if occ[i] and occ[j]:
                    ii.append(i)
                    jj.append(j)
    return np.array(ii, np.int64), np.array(jj, np.int64)


# ------------------------------------------------------ visibility variance
def visvar_planes(ca, cb, L, snr_full_inv2, sigma_cal2, mask=None):
    """Relative variance (SNR^-2) of every unique visibility V^unique_alpha
    of the full L x L array, calibrated with gains whose log errors have
    covariance (sigma_cal2 / 2) (ca, cb) (Eq. gaincov; pass the antenna
    covariance of fixed_gain_covariance for the paper's comparison against
    the truth, or the raw pseudo-inverses), applied to
    visibilities of SNR^-2 = snr_full_inv2 each (Sec. 6.2).

    Returns (paper, exact, n_pairs), planes of (2L-1)^2 indexed by
    lag_index: `paper` is the per-pair form before Eq. visvar with
    |g| = |V| = 1,
        (1 / N_a^2) sum_{(i,j) in a} [SNR^-2 + s_i + s_j + 2 rho_ij],
    s_i = E|a_i|^2, rho_ij the reading in the module header; `exact` is the
    linearised variance of the redundant average including the covariance
    between different pairs,
        (1 / N_a^2) [N_a SNR^-2 + (sigma_cal2 / 2)(u^T ca u + w^T cb w)],
    u = sum_{(i,j) in a} (e_i + e_j), w = sum_{(i,j) in a} (e_i - e_j).
    Lag 0 and lags with no pair read NaN."""
    n = 2 * L - 1
    paper = np.full(n * n, np.nan)
    exact = np.full(n * n, np.nan)
    npairs = np.zeros(n * n, np.int64)
    N = L * L
    h = 0.5 * sigma_cal2
    A = ca[:N, :N]
    B = cb[:N, :N]
    for dy in range(-(L - 1), L):
        for dx in range(-(L - 1), L):
            if dx == 0 and dy == 0:
                continue
            i, j = full_array_pairs(L, dx, dy, mask)
            k = lag_index(L, dx, dy)
            npairs[k] = len(i)
            if len(i) == 0:
                continue
            Na = float(len(i))
            per_pair = (snr_full_inv2 + h * (A[i, i] + B[i, i] + A[j, j] + B[j, j])
                        + 2.0 * h * (A[i, j] - B[i, j]))
            paper[k] = np.sum(per_pair) / Na ** 2
            u = np.zeros(N)
            w = np.zeros(N)
            np.add.at(u, i, 1.0)
            np.add.at(u, j, 1.0)
            np.add.at(w, i, 1.0)
            np.add.at(w, j, -1.0)
            exact[k] = (Na * snr_full_inv2 + h * (u @ A @ u + w @ B @ w)) / Na ** 2
    return paper, exact, npairs


def visvar_eq(n_alpha, snr_full_inv2, sigma_g2, rho_sum=0.0):
    """Eq. visvar: (1 / N_a) [SNR_full^-2 + 2 sigma_g^2 + (2 / N_a) sum rho]."""
    return (snr_full_inv2 + 2.0 * sigma_g2 + 2.0 * rho_sum / n_alpha) / n_alpha


def visvar_lowcadcal(n_alpha, snr_full_inv2, p, N):
    """Eq. visvar_lowcadcal (calibration interval = correlator integration,
    covariance dropped): (SNR_full^-2 / N_a) [1 + 2 / (p log N)]."""
    return snr_full_inv2 / n_alpha * (1.0 + 2.0 / (p * np.log2(N)))


def visvar_subredcal(n_alpha, snr_full_inv2, p, N, rho_sum_rel=0.0):
    """Eq. visvar_subredcal: (SNR_full^-2 / N_a) [1 + 2 / (p log N)
    + (2 / N_a) sum rho], the covariance sum in units of SNR_full^-2."""
    return snr_full_inv2 / n_alpha * (1.0 + 2.0 / (p * np.log2(N)) + 2.0 * rho_sum_rel / n_alpha)


# ------------------------------------------------------------ edge antennas
def edge_antennas(L, mask=None, lattice="square"):
    """Boolean [L*L]: occupied points with an unoccupied or outside nearest
    neighbour (Sec. 5.4)."""
    occ = np.ones(L * L, bool) if mask is None else np.asarray(mask, bool).reshape(-1)
    edge = np.zeros(L * L, bool)
    for y in range(L):
        for x in range(L):
            i = y * L + x
            if not occ[i]:
                continue
            for dx, dy in lattice_neighbours(lattice):
                x2, y2 = x + dx, y + dy
                if not (0 <= x2 < L and 0 <= y2 < L) or not occ[y2 * L + x2]:
                    edge[i] = True
                    break
    return edge


def variance_distribution(var, keep):
    """Antenna-to-antenna distribution of per-antenna gain variances over the
    antennas where `keep` is true: mean, standard deviation (the
    antenna-to-antenna variation), quartiles and range (the boxes of the
    paper's variance figures)."""
    v = np.asarray(var, np.float64)[np.asarray(keep, bool)]
    q25, q50, q75 = np.percentile(v, [25, 50, 75])
    return dict(n=int(v.size), mean=float(v.mean()), std=float(v.std()), min=float(v.min()),
                max=float(v.max()), q25=float(q25), median=float(q50), q75=float(q75))


# --------------------------------------------------- fixing against the truth
def fixed_log_errors(g_est, g_true, L, mask=None):
    """Log-gain errors a = ln(g_est / g_true) with the four degeneracies
    fixed against the truth by least squares over the antennas (Sec. 3): the
    real parts lose their mean, the imaginary parts their best plane
    c0 + c1 x + c2 y (lattice coordinates).  Entries of empty points are 0.
    Small errors: the principal logarithm is the linearised error."""
    occ = np.ones(L * L, bool) if mask is None else np.asarray(mask, bool).reshape(-1)
    idx = np.nonzero(occ)[0]
    x, y = (idx % L).astype(float), (idx // L).astype(float)
    q = np.ones(L * L, np.complex128)
    q[idx] = np.asarray(g_est, np.complex128)[idx] / np.asarray(g_true, np.complex128)[idx]
    # the estimate may differ from the truth by any phase slope and offset:
    # take those out wrap-free first (mean increments between occupied
    # neighbours), so that the logarithm below sees a small error
    qq = q.reshape(L, L)
    oo = occ.reshape(L, L)
    kx = np.angle(np.sum((qq[:, 1:] * np.conj(qq[:, :-1]))[oo[:, 1:] & oo[:, :-1]]))
    ky = np.angle(np.sum((qq[1:, :] * np.conj(qq[:-1, :]))[oo[1:, :] & oo[:-1, :]]))
    q[idx] *= np.exp(-1j * (kx * x + ky * y))
    q[idx] *= np.exp(-1j * np.angle(np.sum(q[idx])))
    a = np.zeros(L * L, np.complex128)
    a[idx] = np.log(q[idx])
    re = a.real[idx] - a.real[idx].mean()
    Q = np.stack([np.ones_like(x), x, y], 1)
    coef, *_ = np.linalg.lstsq(Q, a.imag[idx], rcond=None)
    im = a.imag[idx] - Q @ coef
    out = np.zeros(L * L, np.complex128)
    out[idx] = re + 1j * im
    return out


def fixed_gain_covariance(ca, cb, L, mask=None):
    """The antenna covariance after the degeneracies are fixed against the
    truth by least squares over the antennas: P_a ca P_a and P_p cb P_p on
    the L*L antennas (P the orthogonal projectors that fixed_log_errors
    applies; empty points get 0 rows and columns)."""
    occ = np.ones(L * L, bool) if mask is None else np.asarray(mask, bool).reshape(-1)
    N = L * L
    idx = np.nonzero(occ)[0]
    x, y = (idx % L).astype(float), (idx // L).astype(float)

    def projector(Q):
        return np.eye(len(idx)) - Q @ np.linalg.solve(Q.T @ Q, Q.T)

    Pa = projector(np.ones((len(idx), 1)))
    Pp = projector(np.stack([np.ones_like(x), x, y], 1))
    fa = np.zeros((N, N))
    fp = np.zeros((N, N))
    fa[np.ix_(idx, idx)] = Pa @ ca[np.ix_(idx, idx)] @ Pa
    fp[np.ix_(idx, idx)] = Pp @ cb[np.ix_(idx, idx)] @ Pp
    return fa, fp
