"""Hexagonal arrays -- the paper's own layout (Sec. 3; Fig. 13's 331-antenna
array) -- through the whole path on the GPU, as a partly occupied triangular
lattice, against the FP64 oracle:

* gc_correlate_masked against the masked FX definition (lag-sum bound
  max_d |dV(d)| N_d / (N |V(0)|) <= 1e-5, as for full grids);
* gc_reduce on the masked subset selection: FP32 sums within 1e-5
  sqrt(A_i A_j), 4+4-bit sums bit-exact;
* gc_calibrate (matrix-free lincal) against the oracle's lincal in lattice
  coordinates: gains within 1e-3 after both are in the output convention,
  DoF = P - N - n_ubl + 2 with N the antennas; empty points return g = 0;
* noise-free visibilities: injected gains recovered up to the degeneracies;
* gc_chi2 / gc_chi2_backward against the oracle chi^2 and its gradient.
"""
import numpy as np
import pytest
import torch

from oracle import calib as oc
from oracle import select as osel
from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


@pytest.fixture(scope="module")
def ctx(gc):
    return gc.Context(0)


def _lagsum_err(got, ref, nd, n_ant):
    c = (got.shape[0] - 1) // 2
    return float(np.max(np.abs(got - ref) * nd) / (n_ant * abs(ref[c, c])))


@pytest.mark.parametrize("s,C,T", [(3, 3, 200), (6, 2, 300), (11, 2, 256)])
def test_correlate_masked(gc, ctx, orc, s, C, T):
    L, m = synth.hex_mask(s)
    volt, gains, _ = synth.make_voltages(20 + s, L, C, T, n_src=20, lattice="triangular")
    got = ctx.correlate(volt.cuda(), gains.cuda(), mask=m).cpu().numpy()
    ctx.device_status()
    for c in range(C):
        ref, nd = orc.fx_masked(volt[c].numpy(), gains[c].numpy(), m, L)
        assert _lagsum_err(got[c], ref, nd, int(m.sum())) < 1e-5, (s, c)
        assert np.all(got[c][nd == 0] == 0)


def test_correlate_masked_i4c(gc, ctx, orc):
    s, C, T = 11, 2, 512
    L, m = synth.hex_mask(s)
    volt, gains, _ = synth.make_voltages(41, L, C, T, n_src=20, lattice="triangular")
    q = np.stack([orc.quantize(volt[c].numpy())[0] for c in range(C)])
    got = ctx.correlate(torch.from_numpy(q).cuda(), gains.cuda(), mask=m).cpu().numpy()
    ctx.device_status()
    for c in range(C):
        vq = orc.unpack_i4c(q[c])
        ref, nd = orc.fx_masked(vq, gains[c].numpy(), m, L)
        assert _lagsum_err(got[c], ref, nd, int(m.sum())) < 1e-5


def test_reduce_masked(gc, ctx, orc):
    s, C, T = 11, 2, 300
    L, m = synth.hex_mask(s)
    volt, _, _ = synth.make_voltages(42, L, C, T, n_src=20, lattice="triangular")
    sel = gc.Selection("subset", L, T, mask=m, lattice="triangular")
    ref_sel = osel.subset_layout(L, m, "triangular", T)
    assert np.array_equal(sel.pair_i, ref_sel.pair_i) and np.array_equal(sel.pair_j, ref_sel.pair_j)
    vr, au = ctx.reduce(volt.cuda(), sel)
    vr = vr.cpu().numpy()
    t0, t1 = ref_sel.pair_windows()
    for c in range(C):
        v = volt[c].numpy()
        ref = orc.xengine_c64(v, ref_sel.pair_i, ref_sel.pair_j, t0, t1)
        a = orc.autos(v)
        err = np.max(np.abs(vr[c] - ref) / np.sqrt(a[ref_sel.pair_i] * a[ref_sel.pair_j]))
        assert err < 1e-5
    # 4+4-bit: exact integer sums
    q = np.stack([orc.quantize(volt[c].numpy())[0] for c in range(C)])
    vri, _ = ctx.reduce(torch.from_numpy(q).cuda(), sel)
    vri = vri.cpu().numpy()
    for c in range(C):
        ref = orc.xengine_i4c(q[c], ref_sel.pair_i, ref_sel.pair_j, t0, t1)
        assert np.array_equal(vri[c], ref)


def _oracle_cal(vobs, ref_sel, m):
    pi, pj, pos = osel.compact(ref_sel, m)
    g, V, it, ok = oc.calibrate(vobs, pi, pj, ref_sel.pair_type(), ref_sel.types, pos, "lincal")
    assert ok
    return g, V, pi, pj, pos


def test_calibrate_331_matches_oracle(gc, ctx, orc):
    """Fig. 13's array: hexagon of side 11 (331 antennas), voltages at SNR 10."""
    s, C, T = 11, 3, 1024
    L, m = synth.hex_mask(s)
    occ = np.flatnonzero(m)
    volt, gains, _ = synth.make_voltages(43, L, C, T, n_src=20, lattice="triangular")
    sel = gc.Selection("subset", L, T, mask=m, lattice="triangular")
    assert sel.n_ant == 331
    vr, au = ctx.reduce(volt.cuda(), sel)
    g, V, st = ctx.calibrate(vr, sel, au, solver="lincal_cg")
    ctx.device_status()
    stats = gc.decode_stats(st)
    assert np.all(stats["status"] == gc.GC_OK), stats["status"]
    dof = sel.P - 331 - sel.n_ubl + 2
    assert np.all(stats["dof"] == dof)
    g = g.cpu().numpy().astype(np.complex128)
    ref_sel = osel.subset_layout(L, m, "triangular", T)
    t0, t1 = ref_sel.pair_windows()
    for c in range(C):
        s_ref = orc.xengine_c64(volt[c].numpy(), ref_sel.pair_i, ref_sel.pair_j, t0, t1)
        gr, Vr, pi, pj, pos = _oracle_cal(s_ref / (t1 - t0), ref_sel, m)
        assert np.max(np.abs(g[c][occ] - gr) / np.abs(gr)) < 1e-3
        assert np.all(g[c][m == 0] == 0)
        chi2_ref = oc.chi2(s_ref / (t1 - t0), gr, Vr, pi, pj, ref_sel.pair_type())
        assert stats["chi2"][c] == pytest.approx(chi2_ref, rel=1e-2)
        # Eq. redchi with the radiometer variance sigma_p^2 = (A_i/T)(A_j/T)/t_p
        a = orc.autos(volt[c].numpy())
        sig2 = (a[ref_sel.pair_i] / T) * (a[ref_sel.pair_j] / T) / (t1 - t0)
        r = s_ref / (t1 - t0) - oc.model(gr, Vr, pi, pj, ref_sel.pair_type())
        assert stats["chi2r"][c] == pytest.approx(np.sum(np.abs(r) ** 2 / sig2) / dof, rel=1e-2)


def test_calibrate_noise_free_hex(gc, ctx):
    s, C, T = 6, 3, 256
    L, m = synth.hex_mask(s)
    occ = np.flatnonzero(m)
    sel = gc.Selection("subset", L, T, mask=m, lattice="triangular")
    pt = sel.pair_type()
    tp = (sel.win_t1 - sel.win_t0)[pt]
    sums, gtrue, _ = synth.make_visibilities(44, L, C, sel.pair_i, sel.pair_j, pt, sel.n_ubl, tp,
                                             snr=1e12)
    g, V, st = ctx.calibrate(sums.cuda(), sel, solver="lincal_cg")
    ctx.device_status()
    assert np.all(gc.decode_stats(st)["status"] == gc.GC_OK)
    g = g.cpu().numpy().astype(np.complex128)
    pos = np.stack([occ % L, occ // L], 1).astype(float)
    for c in range(C):
        gt = gtrue[c].numpy().astype(np.complex128)[occ]
        gf = oc.fit_degeneracies(g[c][occ], gt, pos)
        assert np.max(np.abs(gf - gt) / np.abs(gt)) < 1e-4


def test_chi2_and_gradient_masked(gc, ctx):
    s, C, T = 5, 2, 128
    L, m = synth.hex_mask(s)
    occ = np.flatnonzero(m)
    sel = gc.Selection("subset", L, T, mask=m, lattice="triangular")
    pt = sel.pair_type()
    tp = (sel.win_t1 - sel.win_t0)[pt]
    sums, _, _ = synth.make_visibilities(45, L, C, sel.pair_i, sel.pair_j, pt, sel.n_ubl, tp, snr=10.0)
    rng = np.random.default_rng(5)
    N = L * L
    g = (rng.standard_normal((C, N)) + 1j * rng.standard_normal((C, N))).astype(np.complex64)
    V = (rng.standard_normal((C, sel.n_ubl)) + 1j * rng.standard_normal((C, sel.n_ubl))).astype(np.complex64)
    gt, Vt = torch.from_numpy(g).cuda(), torch.from_numpy(V).cuda()
    chi = ctx.chi2(sums.cuda(), sel, gt, Vt).cpu().numpy()
    dg, dV = ctx.chi2_backward(sums.cuda(), sel, gt, Vt)
    dg, dV = dg.cpu().numpy(), dV.cpu().numpy()
    ref_sel = osel.subset_layout(L, m, "triangular", T)
    pi, pj, _ = osel.compact(ref_sel, m)
    alpha = ref_sel.pair_type()
    for c in range(C):
        vobs = sums[c].numpy().astype(np.complex128) / tp
        gc_ = g[c].astype(np.complex128)[occ]
        Vc = V[c].astype(np.complex128)
        ref = oc.chi2(vobs, gc_, Vc, pi, pj, alpha)
        assert chi[c] == pytest.approx(ref, rel=1e-4)
        rg, rV = oc.chi2_grad(vobs, gc_, Vc, pi, pj, alpha)
        scale = np.max(np.abs(rg))
        assert np.max(np.abs(dg[c][occ] - rg)) < 1e-3 * scale
        assert np.max(np.abs(dV[c] - rV)) < 1e-3 * np.max(np.abs(rV))
        assert np.all(dg[c][m == 0] == 0)
