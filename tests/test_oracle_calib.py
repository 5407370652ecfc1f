"""Pins of the calibration oracle against what the paper and the mathematics
fix: exact recovery up to the four degeneracies (Sec. 5.2), solver
independence of the chi^2 minimum (Sec. 2), Eq. gaincov at high SNR,
Eq. dof / Eq. redchi (chi^2_r ~ 1), and the chi^2 gradient against finite
differences."""
import numpy as np
import pytest

from oracle import calib as oc
from oracle import select as osel


def _problem(L, seed, sigma=0.0, unit_amp=False, sel=None):
    rng = np.random.default_rng(seed)
    N = L * L
    sel = sel or osel.subset(L, 100)
    alpha = sel.pair_type()
    amp = np.ones(N) if unit_amp else 1.0 + 0.05 * rng.standard_normal(N)
    g = amp * np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    V = (1.0 if unit_amp else (0.5 + rng.uniform(0, 1, sel.n_ubl))) * \
        np.exp(1j * rng.uniform(-np.pi, np.pi, sel.n_ubl))
    m = oc.model(g, V, sel.pair_i, sel.pair_j, alpha)
    n = sigma * np.sqrt(0.5) * (rng.standard_normal(len(m)) + 1j * rng.standard_normal(len(m)))
    return sel, alpha, g, V, m + n


@pytest.mark.parametrize("solver", ["lincal", "omnical"])
@pytest.mark.parametrize("L", [3, 5])
def test_noise_free_recovery(L, solver):
    sel, alpha, g, V, vobs = _problem(L, 10 + L)
    ge, Ve, it, ok = oc.calibrate(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L, solver)
    assert ok
    assert oc.chi2(vobs, ge, Ve, sel.pair_i, sel.pair_j, alpha) < 1e-18 * len(vobs)
    gf = oc.fit_degeneracies(ge, g, L)
    assert np.max(np.abs(gf - g) / np.abs(g)) < 1e-8


def test_degeneracies_leave_chi2_unchanged():
    L = 4
    sel, alpha, g, V, vobs = _problem(L, 3, sigma=0.1)
    base = oc.chi2(vobs, g, V, sel.pair_i, sel.pair_j, alpha)
    pos = np.stack([np.arange(L * L) % L, np.arange(L * L) // L], 1).astype(float)
    d = np.asarray(sel.types, float)
    k = np.array([0.3, -0.7])
    for g2, V2 in [(1.7 * g, V / 1.7 ** 2),
                   (g * np.exp(0.4j), V),
                   (g * np.exp(1j * pos @ k), V * np.exp(-1j * d @ k))]:
        assert oc.chi2(vobs, g2, V2, sel.pair_i, sel.pair_j, alpha) == pytest.approx(base, rel=1e-12)
    # the projection keeps chi^2 and meets the output convention
    gp, Vp = oc.project(g, V, sel.types, L)
    assert oc.chi2(vobs, gp, Vp, sel.pair_i, sel.pair_j, alpha) == pytest.approx(base, rel=1e-12)
    assert abs(np.mean(np.log(np.abs(gp)))) < 1e-14
    assert abs(np.angle(gp[0])) < 1e-14
    assert abs(np.angle(Vp[sel.types.index((1, 0))])) < 1e-14
    assert abs(np.angle(Vp[sel.types.index((0, 1))])) < 1e-14


def test_lincal_and_omnical_reach_same_minimum():
    """Sec. 2: results do not depend on the solving technique."""
    L = 4
    sel, alpha, g, V, vobs = _problem(L, 7, sigma=0.05)
    a = oc.calibrate(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L, "lincal")
    b = oc.calibrate(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L, "omnical")
    assert a[3] and b[3]
    ca = oc.chi2(vobs, a[0], a[1], sel.pair_i, sel.pair_j, alpha)
    cb = oc.chi2(vobs, b[0], b[1], sel.pair_i, sel.pair_j, alpha)
    assert ca == pytest.approx(cb, rel=1e-8)
    assert np.max(np.abs(a[0] - b[0])) < 1e-6


def test_gradient_matches_finite_differences():
    L = 3
    rng = np.random.default_rng(4)
    sel, alpha, g, V, vobs = _problem(L, 5, sigma=0.3)
    g = g * (1 + 0.1 * rng.standard_normal(len(g)))
    dg, dV = oc.chi2_grad(vobs, g, V, sel.pair_i, sel.pair_j, alpha)
    f = lambda gg, VV: oc.chi2(vobs, gg, VV, sel.pair_i, sel.pair_j, alpha)
    h = 1e-6
    for k in range(len(g)):
        for unit, comp in ((1.0, "re"), (1j, "im")):
            e = np.zeros(len(g), complex)
            e[k] = unit * h
            fd = (f(g + e, V) - f(g - e, V)) / (2 * h)
            an = dg[k].real if comp == "re" else dg[k].imag
            assert fd == pytest.approx(an, rel=1e-6, abs=1e-8)
    for a in range(len(V)):
        for unit, comp in ((1.0, "re"), (1j, "im")):
            e = np.zeros(len(V), complex)
            e[a] = unit * h
            fd = (f(g, V + e) - f(g, V - e)) / (2 * h)
            an = dV[a].real if comp == "re" else dV[a].imag
            assert fd == pytest.approx(an, rel=1e-6, abs=1e-8)


def test_gain_variance_follows_eq_gaincov():
    """Eq. gaincov at high SNR: per-antenna variance of the gain error after
    fixing the degeneracies against the truth equals SNR^-2 diag[(A^T A)^+],
    amplitude and phase parts (Fig. 3, high-SNR regime)."""
    L, sigma, nsim = 4, 0.02, 300
    sel = osel.subset(L, 100)
    alpha = sel.pair_type()
    pa, pp = oc.gain_variance_prediction(L, sel.types, sel.pair_i, sel.pair_j, alpha)
    pred = 0.5 * sigma ** 2 * (pa + pp)
    errs, e_amp, e_ph = [], [], []
    for s in range(nsim):
        _, _, g, V, vobs = _problem(L, 1000 + s, sigma=sigma, unit_amp=True, sel=sel)
        ge, Ve, it, ok = oc.calibrate(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L, "lincal")
        assert ok
        gf = oc.fit_degeneracies(ge, g, L)
        errs.append(np.abs(gf / g - 1.0) ** 2)
        e_amp.append(np.log(np.abs(gf / g)) ** 2)
        e_ph.append(np.angle(gf / g) ** 2)
    meas = np.mean(errs, axis=0)
    ratio = np.mean(meas) / np.mean(pred)
    assert 0.85 < ratio < 1.15, ratio
    # the parts separately: ln|g| follows the amplitude system (A, one null
    # direction), arg g the phase system (B, three); on this array the two
    # predictions differ by ~1.5x, so exchanging them fails
    r_amp = np.mean(e_amp) / np.mean(0.5 * sigma ** 2 * pa)
    r_ph = np.mean(e_ph) / np.mean(0.5 * sigma ** 2 * pp)
    assert 0.9 < r_amp < 1.1 and 0.9 < r_ph < 1.1, (r_amp, r_ph)


def test_dof_is_the_expected_residual():
    """Eq. dof from the statistics of least squares rather than from its
    formula: at high SNR the fit is linear, and the residual chi^2 of complex
    noise of variance sigma^2 has expectation sigma^2 (N_obs - N - N_ubl + 2)
    -- 2 N_obs real observations less 2 (N + N_ubl) - 4 effective real
    parameters (four degeneracies, Sec. 5.2), halved per real component.  A
    3 x 3 array keeps DoF small so that 800 draws resolve a unit error."""
    L, sigma, nsim = 3, 1e-3, 800
    sel = osel.subset(L, 100)
    alpha = sel.pair_type()
    vals = []
    for s in range(nsim):
        _, _, g, V, vobs = _problem(L, 90000 + s, sigma=sigma, sel=sel)
        ge, Ve, it, ok = oc.calibrate(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L, "lincal")
        assert ok
        vals.append(oc.chi2(vobs, ge, Ve, sel.pair_i, sel.pair_j, alpha) / sigma ** 2)
    d = oc.dof(sel.P, L * L, sel.n_ubl)
    # std of the mean: sqrt(DoF / nsim) (chi^2 / sigma^2 is half a chi-square of 2 DoF)
    assert abs(np.mean(vals) - d) < 4.0 * np.sqrt(d / nsim), (np.mean(vals), d)


def test_start_point_is_exact_without_noise():
    """The logcal start (Eq. logcal: ln|V_p| = eta_i + eta_j + a_alpha and
    arg V_p = phi_i - phi_j + theta_alpha) is exact on noise-free data: its
    model reproduces every visibility before any lincal or omnical step."""
    for L, seed in ((3, 4), (5, 8)):
        sel, alpha, g, V, vobs = _problem(L, seed)
        g0, V0 = oc.initial_solution(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L)
        m0 = oc.model(g0, V0, sel.pair_i, sel.pair_j, alpha)
        assert np.max(np.abs(m0 - vobs)) < 1e-10 * np.max(np.abs(vobs))
    # with noise the start is the logcal estimate itself, which is where Eq.
    # gaincov comes from: at high SNR and |g| = |V| = 1 its ln|g| and arg g
    # errors have the variances 0.5 sigma^2 diag[(A^T A)^+] and diag[(B^T B)^+]
    L, sigma, nsim = 4, 0.02, 300
    sel = osel.subset(L, 100)
    alpha = sel.pair_type()
    pa, pp = oc.gain_variance_prediction(L, sel.types, sel.pair_i, sel.pair_j, alpha)
    e_amp, e_ph = [], []
    for s in range(nsim):
        _, _, g, V, vobs = _problem(L, 7000 + s, sigma=sigma, unit_amp=True, sel=sel)
        g0, _ = oc.initial_solution(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L)
        q = oc.fit_degeneracies(g0, g, L) / g
        e_amp.append(np.log(np.abs(q)) ** 2)
        e_ph.append(np.angle(q) ** 2)
    r_amp = np.mean(e_amp) / np.mean(0.5 * sigma ** 2 * pa)
    r_ph = np.mean(e_ph) / np.mean(0.5 * sigma ** 2 * pp)
    assert 0.9 < r_amp < 1.1 and 0.9 < r_ph < 1.1, (r_amp, r_ph)


def test_full_redcal_variance_scales_as_one_over_n():
    """Eq. gainvar_redcal: with the full visibility matrix every antenna sits
    in N - 1 equations and the diagonal of (A^T A)^+ approaches 1/N for the
    amplitude and for the phase part alike; N times the mean predicted
    variance falls towards 1 as the grid grows (every pair, unit noise)."""
    prev = None
    for L in (4, 6, 8, 12):
        sel = osel.lowcad(L, 10 ** 6)            # every baseline-type, i.e. every pair
        assert sel.P == L * L * (L * L - 1) // 2
        pa, pp = oc.gain_variance_prediction(L, sel.types, sel.pair_i, sel.pair_j, sel.pair_type())
        na, npp = L * L * pa.mean(), L * L * pp.mean()
        assert na > 1.0 and npp > 0.95
        if prev is not None:
            assert na < prev
        prev = na
    assert na == pytest.approx(1.0, abs=0.05) and npp == pytest.approx(1.0, abs=0.05)


@pytest.mark.parametrize("scheme", ["subset", "lowcad"])
def test_gains_are_unbiased(scheme):
    """Sec. 6.3 / Fig. 11: with the gains and visibilities held fixed and the
    noise redrawn, the gain solutions averaged over N_sim realisations
    deviate from the truth by a factor 1/N_sim less (in squared deviation)
    than one solution does -- the estimates differ from the truth only by
    noise.  D(N_sim) N_sim / sigma_g^2 stays at 1 for N_sim = 1 .. 256,
    within three standard deviations of its scatter over the 2 N - 4 real
    components of each of the 256 / N_sim averages; a bias b would lift it
    by N_sim |b|^2 / sigma_g^2 (detectable down to |b| ~ 0.06 sigma_g)."""
    L, sigma, nsim = 4, 0.05, 256
    sel = osel.subset(L, 100) if scheme == "subset" else osel.lowcad(L, 100)
    alpha = sel.pair_type()
    rng = np.random.default_rng(77)
    g = (1.0 + 0.05 * rng.standard_normal(L * L)) * np.exp(1j * rng.uniform(-np.pi, np.pi, L * L))
    V = (0.5 + rng.uniform(0, 1, sel.n_ubl)) * np.exp(1j * rng.uniform(-np.pi, np.pi, sel.n_ubl))
    m = oc.model(g, V, sel.pair_i, sel.pair_j, alpha)
    q = []
    for s in range(nsim):
        n = sigma * np.sqrt(0.5) * (rng.standard_normal(len(m)) + 1j * rng.standard_normal(len(m)))
        ge, _, _, ok = oc.calibrate(m + n, sel.pair_i, sel.pair_j, alpha, sel.types, L, "lincal")
        assert ok
        q.append(oc.fit_degeneracies(ge, g, L) / g - 1.0)
    q = np.asarray(q)
    var1 = np.mean(np.abs(q) ** 2)                        # one realisation
    for k in (4, 16, 64, 256):
        groups = q[: (nsim // k) * k].reshape(nsim // k, k, -1).mean(axis=1)
        d = np.mean(np.abs(groups) ** 2)                  # squared deviation of a k-average
        n_eff = (nsim // k) * (2 * L * L - 4)
        assert abs(d * k / var1 - 1.0) < 3.0 * np.sqrt(2.0 / n_eff), (k, d * k / var1)


def test_reduced_chi2_is_one():
    """Eq. redchi / Eq. dof: with the true noise variance chi^2_r ~ 1."""
    L, sigma, nsim = 4, 0.05, 200
    sel = osel.subset(L, 100)
    alpha = sel.pair_type()
    vals = []
    for s in range(nsim):
        _, _, g, V, vobs = _problem(L, 5000 + s, sigma=sigma, sel=sel)
        ge, Ve, it, ok = oc.calibrate(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L, "lincal")
        vals.append(oc.chi2_r(vobs, ge, Ve, sel.pair_i, sel.pair_j, alpha, sigma ** 2))
    assert np.mean(vals) == pytest.approx(1.0, abs=0.05)


@pytest.mark.parametrize("solver", ["lincal", "omnical"])
def test_voltages_to_gains_end_to_end(orc, solver):
    """Fig. 1 cycle on the oracle: voltages v_i = g_i s_i of one noise-free
    point source (exactly redundant), X-engine sums over the subset pairs,
    calibration, and recovery of the injected gains up to the degeneracies.
    Fixes the conjugation convention shared by Eq. redcal and the X-engine."""
    import torch
    from paper_2005_03060_gb300 import synth
    L, T = 5, 64
    volt, gains, _ = synth.make_voltages(21, L, 1, T, n_src=1, noise=False)
    v = volt[0].numpy().astype(np.complex128)
    g_true = gains[0].numpy().astype(np.complex128)
    sel = osel.subset(L, T)
    alpha = sel.pair_type()
    s = orc.xengine_c64(v, sel.pair_i, sel.pair_j, sel.win_t0[alpha], sel.win_t1[alpha])
    ge, Ve, it, ok = oc.calibrate(s / T, sel.pair_i, sel.pair_j, alpha, sel.types, L, solver)
    assert ok
    gf = oc.fit_degeneracies(ge, g_true, L)
    # float32 voltages: recovery to single precision
    assert np.max(np.abs(gf - g_true) / np.abs(g_true)) < 1e-5


@pytest.mark.parametrize("L,sigma", [(4, 0.05), (6, 0.1), (8, 0.02)])
def test_sparse_lincal_equals_dense(L, sigma):
    """The sparse form of lincal solves the same Gauss-Newton normal
    equations: same minimum, same gains after the output convention."""
    sel, alpha, g, V, vobs = _problem(L, 40 + L, sigma=sigma)
    a = oc.calibrate(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L, "lincal")
    b = oc.calibrate(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L, "lincal", sparse=True)
    assert a[3] and b[3]
    assert np.max(np.abs(a[0] - b[0]) / np.abs(a[0])) < 1e-9
    assert np.max(np.abs(a[1] - b[1]) / np.abs(a[1])) < 1e-9


def test_sparse_lincal_noise_free_recovery_24x24():
    """Exact recovery up to the four degeneracies (Sec. 5.2) on an array
    the dense form would handle only slowly."""
    L = 24
    sel, alpha, g, V, vobs = _problem(L, 77, sel=osel.subset(L, 100))
    ge, Ve, it, ok = oc.calibrate(vobs, sel.pair_i, sel.pair_j, alpha, sel.types, L, "lincal", sparse=True)
    assert ok
    assert oc.chi2(vobs, ge, Ve, sel.pair_i, sel.pair_j, alpha) < 1e-18 * len(vobs)
    gf = oc.fit_degeneracies(ge, g, L)
    assert np.max(np.abs(gf - g) / np.abs(g)) < 1e-8
