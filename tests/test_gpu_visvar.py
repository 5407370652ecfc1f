"""The covariance and visibility-variance tool on the GPU (Sec. 5.3-5.4,
Sec. 6.2) against the oracle (oracle/visvar.py):

  * gc_gain_covariance rows of the pseudo-inverses (Figs. 7-8) and the rows
    with the degeneracies fixed against the truth, on square grids (subset
    and low-cadence) and a hexagonal array;
  * gc_visibility_variance, both the paper's per-pair form and the full
    linearised variance, and the pair counts N_alpha, for every lag;
  * the edge-excluded gain-variance statistic of Sec. 5.4 (edge antennas
    from gc_sel_edge), with the table of how much leaving the rim out
    lowers the antenna-to-antenna variation (run with -s to see it);
  * the visibility-variance factor N_alpha SNR^2 var against the closed
    forms Eq. visvar_lowcadcal / Eq. visvar_subredcal (table).
"""
import numpy as np
import pytest

from oracle import select as osel
from oracle import visvar as ov

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


@pytest.fixture(scope="module")
def ctx(gc):
    return gc.Context(0)


def _case(gc, kind, L_or_s, p=1.0):
    """(library selection, L, mask or None, lattice, oracle types, pair_i,
    pair_j, pair_type in grid numbering)."""
    from paper_2005_03060_gb300 import synth
    if kind == "hex":
        L, m = synth.hex_mask(L_or_s)
        sel = gc.Selection("subset", L, 256, p=p, mask=m, lattice="triangular")
        ref = osel.subset_layout(L, m, "triangular", 256, p=p)
        return sel, L, m, "triangular", ref
    L = L_or_s
    sel = gc.Selection(kind, L, 256, p=p)
    ref = osel.subset(L, 256, p=p) if kind == "subset" else osel.lowcad(L, 256, p=p)
    return sel, L, None, "square", ref


def _oracle_cov(L, ref, mask):
    types = [tuple(t) for t in ref.types]
    return ov.gain_covariance(L, types, np.asarray(ref.pair_i), np.asarray(ref.pair_j), ref.pair_type())


CASES = [("subset", 8), ("lowcad", 8), ("subset", 12), ("hex", 4)]


@pytest.mark.parametrize("kind,size", CASES)
def test_covariance_rows(gc, ctx, kind, size):
    sel, L, m, lat, ref = _case(gc, kind, size)
    N = L * L
    ca, cb = _oracle_cov(L, ref, m)
    occ = np.arange(N) if m is None else np.flatnonzero(m)
    rows = [int(occ[0]), int(occ[len(occ) // 2]), int(occ[-1]), N, N + sel.n_ubl - 1]
    ga, gp = ctx.gain_covariance(sel, rows)
    ctx.device_status()
    ga, gp = ga.cpu().numpy(), gp.cpu().numpy()
    for k, r in enumerate(rows):
        for got, ref_row in ((ga[k], ca[r]), (gp[k], cb[r])):
            np.testing.assert_allclose(got, ref_row, rtol=0, atol=2e-4 * np.abs(ref_row).max())
    # fixed against the truth: every antenna row
    fa, fp = ov.fixed_gain_covariance(ca, cb, L, m)
    arows = occ.astype(np.int32)
    ga, gp = ctx.gain_covariance(sel, arows, fixed=True)
    ctx.device_status()
    ga, gp = ga.cpu().numpy(), gp.cpu().numpy()
    np.testing.assert_allclose(ga, fa[arows], rtol=0, atol=2e-4 * np.abs(fa).max())
    np.testing.assert_allclose(gp, fp[arows], rtol=0, atol=2e-4 * np.abs(fp).max())


@pytest.mark.parametrize("kind,size", CASES)
def test_visibility_variance(gc, ctx, kind, size):
    sel, L, m, lat, ref = _case(gc, kind, size)
    snr, scal = 1.0 / 50.0, 1.0 / 30.0
    vp, ve, npr = ctx.visibility_variance(sel, snr, scal)
    ctx.device_status()
    ca, cb = _oracle_cov(L, ref, m)
    fa, fp = ov.fixed_gain_covariance(ca, cb, L, m)
    paper, exact, npairs = ov.visvar_planes(fa, fp, L, snr, scal, m)
    n = 2 * L - 1
    assert np.array_equal(npr.cpu().numpy().reshape(-1), npairs)
    ok = npairs > 0
    for got, want in ((vp, paper), (ve, exact)):
        got = got.cpu().numpy().reshape(-1)
        assert np.all(np.isnan(got[~ok])) and np.all(np.isnan(want[~ok]))
        np.testing.assert_allclose(got[ok], want[ok], rtol=1e-4)
    assert got.shape == (n * n,)


@pytest.mark.parametrize("kind,size", [("subset", 8), ("hex", 5)])
def test_edge_mask_matches_oracle(gc, kind, size):
    sel, L, m, lat, ref = _case(gc, kind, size)
    assert np.array_equal(sel.edge_mask().astype(bool), ov.edge_antennas(L, m, lat))


def test_edge_excluded_statistic_table(gc, ctx):
    """Sec. 5.4: the antenna-to-antenna spread of gain variance with and
    without the edge antennas, subset selections of several sizes p on a
    16 x 16 grid and a hexagonal array of side 6 (91 antennas)."""
    rows = []
    for kind, size, p in (("subset", 16, 0.5), ("subset", 16, 1.0), ("subset", 16, 2.0), ("subset", 16, 4.0),
                          ("hex", 6, 1.0), ("hex", 6, 2.0)):
        sel, L, m, lat, ref = _case(gc, kind, size, p)
        occ = np.arange(L * L) if m is None else np.flatnonzero(m)
        ga, gp = ctx.gain_covariance(sel, occ.astype(np.int32), fixed=True)
        ctx.device_status()
        var_gpu = np.zeros(L * L)
        var_gpu[occ] = (ga.cpu().numpy()[np.arange(len(occ)), occ] + gp.cpu().numpy()[np.arange(len(occ)), occ])
        ca, cb = _oracle_cov(L, ref, m)
        fa, fp = ov.fixed_gain_covariance(ca, cb, L, m)
        var_orc = np.diag(fa) + np.diag(fp)
        edge = sel.edge_mask().astype(bool)
        keep_all = np.zeros(L * L, bool)
        keep_all[occ] = True
        st = {}
        for name, v in (("gpu", var_gpu), ("oracle", var_orc)):
            st[name] = (ov.variance_distribution(v, keep_all), ov.variance_distribution(v, keep_all & ~edge))
        for a, b in zip(st["gpu"], st["oracle"]):
            for key in ("mean", "std", "min", "max", "median"):
                assert a[key] == pytest.approx(b[key], rel=1e-3), (kind, size, p, key)
        full, inner = st["gpu"]
        rows.append((kind, size, p, sel.P, full["n"], inner["n"], full["mean"], inner["mean"], full["std"],
                     inner["std"]))
        # leaving the rim out lowers both the mean and the spread
        assert inner["mean"] < full["mean"] and inner["std"] < full["std"]
    print("\narray      p      P    N  N_in   mean(all)  mean(in)   std(all)   std(in)  spread drop")
    for r in rows:
        print(f"{r[0]:6s}{r[1]:3d} {r[2]:4.1f} {r[3]:6d} {r[4]:4d} {r[5]:4d}  {r[6]:.4e} {r[7]:.4e} "
              f"{r[8]:.4e} {r[9]:.4e}  {100 * (1 - r[9] / r[8]):5.1f} %")


def test_visibility_variance_against_closed_forms(gc, ctx):
    """Sec. 6.2: N_alpha SNR_full^2 var(V^unique) against the bracket of
    Eq. visvar_lowcadcal and Eq. visvar_subredcal, per scheme and size.
    The calibrator's noise: the same integration as the correlator for
    subset calibration; 1 / (time share of a type) more for low-cadence
    calibration (Eq. SNR_lowcadcal with t_cal = t_int)."""
    snr = 1.0 / 100.0
    rows = []
    for kind in ("subset", "lowcad"):
        for L in (8, 12, 16):
            sel, _, _, _, ref = _case(gc, kind, L)
            t_share = float(np.mean(sel.win_t1 - sel.win_t0)) / sel.T
            scal = snr / t_share
            vp, ve, npr = ctx.visibility_variance(sel, snr, scal)
            ctx.device_status()
            vp, ve, npr = vp.cpu().numpy(), ve.cpu().numpy(), npr.cpu().numpy()
            ok = npr > 0
            f_pair = np.median(vp[ok] * npr[ok] / snr)
            f_exact = np.median(ve[ok] * npr[ok] / snr)
            f_eq = 1.0 + 2.0 / (1.0 * np.log2(L * L))
            rows.append((kind, L, sel.P, f_pair, f_exact, f_eq))
            # the gain-variance terms add to the thermal term, never remove
            assert f_pair > 1.0 and f_exact > 1.0
    print("\nscheme   L      P   N_a SNR^2 var: per-pair form  full form   Eq. visvar_* bracket")
    for r in rows:
        print(f"{r[0]:7s}{r[1]:3d} {r[2]:6d}   {r[3]:14.4f} {r[4]:10.4f}   {r[5]:10.4f}")
