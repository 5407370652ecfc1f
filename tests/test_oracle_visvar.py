"""Pins of the covariance and visibility-variance oracle (oracle/visvar.py;
Sec. 5.3-5.4 and Sec. 6.2), against things other than itself:

  * Monte Carlo of the whole chain on a 5 x 5 array: noisy V^reduced ->
    the oracle's lincal -> degeneracies fixed against the truth -> gains
    applied to independently noisy full-array visibilities -> redundant
    average.  The measured gain covariance and the measured variance of
    every V^unique lag agree with the predictions;
  * with noiseless gains the variance is that of a mean of N_a samples, and
    N_a = (L - |dx|)(L - |dy|) on a full grid (textbook);
  * under the paper's stated assumptions (equal gain variances, a common
    covariance) the per-pair form reduces to Eq. visvar, Eq.
    visvar_lowcadcal and Eq. visvar_subredcal, and the full form to its own
    closed form;
  * edge antennas of small square and hexagonal arrays, counted by hand;
  * the pseudo-inverse rows are orthogonal to the exact degeneracies.
"""
import numpy as np
import pytest

from oracle import calib as oc
from oracle import select as osel
from oracle import visvar as ov


def _sel(L):
    s = osel.subset(L, 1024)
    return s, [tuple(t) for t in s.types], np.asarray(s.pair_i), np.asarray(s.pair_j), s.pair_type()


@pytest.fixture(scope="module")
def monte_carlo():
    L, K = 5, 1500
    sigma_cal2, snr_full_inv2 = 0.03 ** 2, 0.05 ** 2
    s, types, pi, pj, pt = _sel(L)
    N = L * L
    rng = np.random.default_rng(20200506)
    # unit-amplitude gains: the setting in which Eq. gaincov holds exactly
    # (with |g| != 1 each pair's relative noise scales as 1 / |g_i g_j|)
    g = np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    Vt = np.exp(1j * rng.uniform(-np.pi, np.pi, len(types)))
    m = g[pi] * np.conj(g[pj]) * Vt[pt]
    # true unique visibilities of every lag of the full array (Hermitian)
    n = 2 * L - 1
    Vfull = np.zeros(n * n, np.complex128)
    for dy in range(0, L):
        for dx in range(-(L - 1), L):
            if dy == 0 and dx <= 0:
                continue
            v = np.exp(1j * rng.uniform(-np.pi, np.pi))
            Vfull[ov.lag_index(L, dx, dy)] = v
            Vfull[ov.lag_index(L, -dx, -dy)] = np.conj(v)
    lags = [(dx, dy) for dy in range(-(L - 1), L) for dx in range(-(L - 1), L) if (dx, dy) != (0, 0)]
    pairs = {d: ov.full_array_pairs(L, *d) for d in lags}
    errs = np.zeros((K, N), np.complex128)
    verr = np.zeros((K, n * n), np.complex128)
    for k in range(K):
        noise = np.sqrt(sigma_cal2 / 2) * (rng.standard_normal(len(m)) + 1j * rng.standard_normal(len(m)))
        ge, _, _, ok = oc.calibrate(m + noise, pi, pj, pt, types, L)
        assert ok
        a = ov.fixed_log_errors(ge, g, L)
        errs[k] = a
        gf = g * np.exp(a)
        for d in lags:
            i, j = pairs[d]
            idx = ov.lag_index(L, *d)
            nf = np.sqrt(snr_full_inv2 / 2) * (rng.standard_normal(len(i)) + 1j * rng.standard_normal(len(i)))
            vobs = g[i] * np.conj(g[j]) * Vfull[idx] + nf
            vu = np.mean(vobs / (gf[i] * np.conj(gf[j])))
            verr[k, idx] = vu / Vfull[idx] - 1.0
    ca, cb = ov.gain_covariance(L, types, pi, pj, pt)
    fa, fp = ov.fixed_gain_covariance(ca, cb, L)
    paper, exact, npairs = ov.visvar_planes(fa, fp, L, snr_full_inv2, sigma_cal2)
    return dict(L=L, K=K, errs=errs, verr=verr, fa=fa, fp=fp, paper=paper, exact=exact, npairs=npairs,
                sigma_cal2=sigma_cal2, snr=snr_full_inv2)


def test_gain_covariance_matches_monte_carlo(monte_carlo):
    mc = monte_carlo
    h = mc["sigma_cal2"] / 2
    ca_mc = np.cov(mc["errs"].real.T, bias=True)
    cp_mc = np.cov(mc["errs"].imag.T, bias=True)
    for meas, pred in ((ca_mc, h * mc["fa"]), (cp_mc, h * mc["fp"])):
        # variances: each within the sampling error of K draws
        ratio = np.diag(meas) / np.diag(pred)
        assert 0.95 < ratio.mean() < 1.05 and np.all(np.abs(ratio - 1) < 0.15), ratio
        # covariances (the rows of Figs. 7-8): same pattern, unit slope
        off = ~np.eye(len(pred), dtype=bool)
        assert np.corrcoef(meas[off], pred[off])[0, 1] > 0.9
        slope = np.sum(meas[off] * pred[off]) / np.sum(pred[off] ** 2)
        assert 0.9 < slope < 1.1, slope


def test_visibility_variance_matches_monte_carlo(monte_carlo):
    mc = monte_carlo
    ok = mc["npairs"] > 0
    meas = np.mean(np.abs(mc["verr"][:, ok]) ** 2, axis=0)
    ratio = meas / mc["exact"][ok]
    assert 0.95 < np.mean(ratio) < 1.05, np.mean(ratio)
    assert np.all((ratio > 0.8) & (ratio < 1.2)), (ratio.min(), ratio.max())
    # the per-pair form leaves out the covariance between pairs; here it
    # is the worse description of the simulation, at every lag with 2+ pairs
    multi = mc["npairs"][ok] > 1
    err_exact = np.abs(np.log(meas / mc["exact"][ok]))[multi]
    err_paper = np.abs(np.log(meas / mc["paper"][ok]))[multi]
    assert np.mean(err_exact) < np.mean(err_paper)


@pytest.mark.parametrize("L", [3, 6])
def test_noiseless_gains_give_the_mean_of_n_samples(L):
    s, types, pi, pj, pt = _sel(L)
    ca, cb = ov.gain_covariance(L, types, pi, pj, pt)
    fa, fp = ov.fixed_gain_covariance(ca, cb, L)
    snr = 0.01
    paper, exact, npairs = ov.visvar_planes(fa, fp, L, snr, 0.0)
    for dy in range(-(L - 1), L):
        for dx in range(-(L - 1), L):
            k = ov.lag_index(L, dx, dy)
            if (dx, dy) == (0, 0):
                assert np.isnan(paper[k]) and np.isnan(exact[k])
                continue
            nd = (L - abs(dx)) * (L - abs(dy))
            assert npairs[k] == nd
            assert paper[k] == pytest.approx(snr / nd, rel=1e-12)
            assert exact[k] == pytest.approx(snr / nd, rel=1e-12)


def test_general_form_reduces_to_the_numbered_equations():
    L, c = 6, 0.3
    N = L * L
    snr, p = 0.02, 1.0
    ca = np.eye(N) + c * np.ones((N, N))
    cb = np.eye(N)
    # equal gain variances sigma_g^2 = Eq. visvar_subredcal's 1 / (p log N)
    # in units of SNR^-2, and a common covariance rho = h c
    sg2 = snr / (p * np.log2(N))
    h = sg2 / (2.0 + c)
    paper, exact, npairs = ov.visvar_planes(ca, cb, L, snr, 2.0 * h)
    ok = npairs > 0
    na = npairs[ok].astype(float)
    np.testing.assert_allclose(paper[ok], ov.visvar_eq(na, snr, sg2, rho_sum=na * h * c), rtol=1e-12)
    np.testing.assert_allclose(paper[ok], ov.visvar_subredcal(na, snr, p, N, rho_sum_rel=na * h * c / snr),
                               rtol=1e-12)
    # full form: |u|^2 + |w|^2 = 4 N_a and sum(u) = 2 N_a for any pair layout
    np.testing.assert_allclose(exact[ok], (snr + 4 * h) / na + 4 * h * c, rtol=1e-12)
    # a common phase covariance enters with the opposite sign: the phases of
    # g_i and conj(g_j) cancel in a calibrated visibility
    paper_p, exact_p, _ = ov.visvar_planes(cb, ca, L, snr, 2.0 * h)
    np.testing.assert_allclose(paper_p[ok], ov.visvar_eq(na, snr, sg2, rho_sum=-na * h * c), rtol=1e-12)
    np.testing.assert_allclose(exact_p[ok], (snr + 4 * h) / na, rtol=1e-12)
    # no covariance: Eq. visvar_lowcadcal
    paper0, _, _ = ov.visvar_planes(np.eye(N), np.eye(N), L, snr, sg2)
    np.testing.assert_allclose(paper0[ok], ov.visvar_lowcadcal(na, snr, p, N), rtol=1e-12)


def test_edge_antennas_by_hand():
    e3 = ov.edge_antennas(3)
    assert e3.sum() == 8 and not e3[4]
    e4 = ov.edge_antennas(4)
    assert sorted(np.nonzero(~e4)[0]) == [5, 6, 9, 10]
    # hexagonal arrays of side 2 (7 antennas) and 3 (19): 1 and 7 inside
    for s, inner in ((2, 1), (3, 7)):
        L = 2 * s - 1
        y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
        m = ((x + y >= s - 1) & (x + y <= 3 * s - 3)).reshape(-1)
        e = ov.edge_antennas(L, m, "triangular")
        assert m.sum() == 3 * s * (s - 1) + 1
        assert int((m & ~e).sum()) == inner
        assert not e[~m].any()
    d = ov.variance_distribution(np.arange(9.0), ~e3)
    assert d["n"] == 1 and d["mean"] == 4.0 and d["std"] == 0.0


def test_pinv_rows_are_orthogonal_to_the_degeneracies():
    L = 6
    s, types, pi, pj, pt = _sel(L)
    ca, cb = ov.gain_covariance(L, types, pi, pj, pt)
    N = L * L
    td = np.asarray(types, float)
    na = np.concatenate([np.ones(N), -2.0 * np.ones(len(types))])
    x, y = np.arange(N) % L, np.arange(N) // L
    n1 = np.concatenate([np.ones(N), np.zeros(len(types))])
    nx = np.concatenate([x, -td[:, 0]])
    ny = np.concatenate([y, -td[:, 1]])
    scale = np.abs(ca).max()
    assert np.abs(ca @ na).max() < 1e-9 * scale * len(na)
    for v in (n1, nx, ny):
        assert np.abs(cb @ v).max() < 1e-9 * np.abs(cb).max() * len(v)
