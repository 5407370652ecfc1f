"""Parity of the CUDA calibration (gc_calibrate) with the FP64 oracle.

The oracle computes its own V^reduced from the same voltages (its X-engine)
and calibrates it (lincal to 1e-10); the GPU path runs gc_reduce then
gc_calibrate.  Both outputs are in the same degeneracy convention (mean
ln|g| = 0, arg g_0 = 0, arg V_(1,0) = arg V_(0,1) = 0) and must agree to
max_i |g_gpu - g_ref| / |g_ref| <= 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import calib as oc
from oracle import select as osel
from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu
GTOL = 1e-3


@pytest.fixture(scope="module")
def gc():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


@pytest.fixture(scope="module")
def ctx(gc):
    return gc.Context(0)


def oracle_gains(orc, v, scheme, L, T, quantised=None):
    sel = osel.subset(L, T) if scheme == "subset" else osel.lowcad(L, T)
    pt = sel.pair_type()
    t0, t1 = sel.win_t0[pt], sel.win_t1[pt]
    if quantised is None:
        s = orc.xengine_c64(v, sel.pair_i, sel.pair_j, t0, t1)
    else:
        raw = orc.xengine_i4c(quantised, sel.pair_i, sel.pair_j, t0, t1)
        s = raw[:, 0] + 1j * raw[:, 1]
    vobs = s / (t1 - t0)
    g, V, it, ok = oc.calibrate(vobs, sel.pair_i, sel.pair_j, pt, sel.types, L, "lincal")
    assert ok
    return g, V, vobs, sel


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


SOLVERS = [("lincal", "fp64"), ("lincal", "fp32"), ("lincal_cg", "fp32"), ("omnical", "fp32")]


@pytest.mark.parametrize("solver,precision", SOLVERS)
def test_noise_free_recovers_injected_gains(gc, ctx, solver, precision):
    """One noise-free point source is exactly redundant: the injected gains
    come back up to the four degeneracies (Sec. 5.2)."""
    L, C, T = 6, 3, 64
    volt, gains, _ = synth.make_voltages(31, L, C, T, n_src=1, noise=False)
    sel = gc.Selection("subset", L, T)
    vr, au = ctx.reduce(volt.cuda(), sel)
    g, V, st = ctx.calibrate(vr, sel, au, solver=solver, precision=precision)
    ctx.device_status()
    stats = gc.decode_stats(st)
    assert np.all(stats["status"] == gc.GC_OK), stats
    g = g.cpu().numpy().astype(np.complex128)
    for c in range(C):
        gt = gains[c].numpy().astype(np.complex128)
        gf = oc.fit_degeneracies(g[c], gt, L)
        assert rel_err(gf, gt) < GTOL


@pytest.mark.parametrize("solver,precision", SOLVERS)
def test_tiny_config_matches_oracle(gc, ctx, orc, solver, precision):
    """8x8 grid, 32 channels, 256 samples, 20 sources, subset selection."""
    L, C, T = 8, 32, 256
    volt, gains, _ = synth.make_voltages(1, L, C, T, n_src=20)
    sel = gc.Selection("subset", L, T)
    vr, au = ctx.reduce(volt.cuda(), sel)
    g, V, st = ctx.calibrate(vr, sel, au, solver=solver, precision=precision)
    ctx.device_status()
    stats = gc.decode_stats(st)
    assert np.all(stats["status"] == gc.GC_OK), stats["status"]
    g = g.cpu().numpy().astype(np.complex128)
    for c in range(0, C, 4):
        v = volt[c].numpy().astype(np.complex128)
        gr, Vr, vobs, osl = oracle_gains(orc, v, "subset", L, T)
        assert rel_err(g[c], gr) < GTOL, (c, rel_err(g[c], gr))
        chi2_ref = oc.chi2(vobs, gr, Vr, osl.pair_i, osl.pair_j, osl.pair_type())
        assert stats["chi2"][c] == pytest.approx(chi2_ref, rel=1e-2)
        assert stats["dof"][c] == osl.P - L * L - osl.n_ubl + 2
    # Eq. redchi: with the radiometer noise variance chi^2_r is near one
    assert 0.7 < float(np.median(stats["chi2r"])) < 1.4


@pytest.mark.parametrize("solver", ["omnical", "lincal_cg"])
def test_lowcad_matches_oracle(gc, ctx, orc, solver):
    L, C, T = 6, 4, 400
    volt, gains, _ = synth.make_voltages(3, L, C, T, n_src=20)
    sel = gc.Selection("lowcad", L, T)
    vr, au = ctx.reduce(volt.cuda(), sel)
    g, V, st = ctx.calibrate(vr, sel, au, solver=solver)
    ctx.device_status()
    stats = gc.decode_stats(st)
    assert np.all(stats["status"] == gc.GC_OK), stats["status"]
    g = g.cpu().numpy().astype(np.complex128)
    for c in range(C):
        gr, _, _, _ = oracle_gains(orc, volt[c].numpy().astype(np.complex128), "lowcad", L, T)
        assert rel_err(g[c], gr) < GTOL


def test_i4c_path_matches_oracle(gc, ctx, orc):
    """Quantised voltages: exact X-engine sums feed the same calibration."""
    L, C, T = 8, 4, 512
    volt, gains, _ = synth.make_voltages(8, L, C, T, n_src=20)
    q = np.stack([orc.quantize(volt[c].numpy())[0] for c in range(C)])
    sel = gc.Selection("subset", L, T)
    vr, au = ctx.reduce(torch.from_numpy(q).cuda(), sel)
    g, V, st = ctx.calibrate(vr, sel, au)
    ctx.device_status()
    g = g.cpu().numpy().astype(np.complex128)
    for c in range(C):
        gr, _, _, _ = oracle_gains(orc, None, "subset", L, T, quantised=q[c])
        assert rel_err(g[c], gr) < GTOL


def test_warm_start_converges_immediately(gc, ctx):
    L, C, T = 8, 4, 256
    volt, gains, _ = synth.make_voltages(9, L, C, T, n_src=20)
    sel = gc.Selection("subset", L, T)
    vr, au = ctx.reduce(volt.cuda(), sel)
    g, V, st = ctx.calibrate(vr, sel, au)
    g2, V2, st2 = ctx.calibrate(vr, sel, au, gains=g.clone(), vmodel=V.clone(), warm_start=True)
    ctx.device_status()
    s1, s2 = gc.decode_stats(st), gc.decode_stats(st2)
    # the float32 output point is one rounding away from the FP64 minimum
    assert np.all(s2["iters"] <= 3) and np.all(s2["iters"] < s1["iters"])
    assert np.allclose(g.cpu().numpy(), g2.cpu().numpy(), atol=1e-5)


def test_time_limit_reports_timeout(gc, ctx):
    """A solve that cannot converge (tolerance below rounding) stops at its
    device-side time limit and reports GC_ETIMEOUT, leaving the context usable."""
    L, C, T = 8, 2, 256
    volt, gains, _ = synth.make_voltages(10, L, C, T, n_src=20)
    sel = gc.Selection("subset", L, T)
    vr, au = ctx.reduce(volt.cuda(), sel)
    g, V, st = ctx.calibrate(vr, sel, au, solver="omnical", tol=1e-300, max_iter=10 ** 9,
                             time_limit_ms=20)
    with pytest.raises(gc.GridcorrError) as e:
        ctx.device_status()
    assert e.value.status == gc.GC_ETIMEOUT
    assert np.all(gc.decode_stats(st)["status"] == gc.GC_ETIMEOUT)
    ctx.device_status()   # cleared, context still works
    g, V, st = ctx.calibrate(vr, sel, au)
    ctx.device_status()
    assert np.all(gc.decode_stats(st)["status"] == gc.GC_OK)


def test_paper_scale_channel_matches_oracle(gc, ctx, orc):
    """32x32 grid, 256 channels, 4096 samples, 200 sources: the full GPU run
    (the benchmark's configuration, every solver) against the oracle on one
    channel."""
    L, C, T = 32, 256, 4096
    sel = gc.Selection("subset", L, T)
    volt = torch.empty(C, T, L * L, dtype=torch.complex64, device="cuda")
    volt, gains, _ = synth.make_voltages(2, L, C, T, n_src=200, device="cuda", out=volt)
    vr, au = ctx.reduce(volt, sel)
    c = 77
    gr, _, _, _ = oracle_gains(orc, volt[c].cpu().numpy().astype(np.complex128), "subset", L, T)
    for solver, precision in SOLVERS:
        g, V, st = ctx.calibrate(vr, sel, au, solver=solver, precision=precision)
        ctx.device_status()
        stats = gc.decode_stats(st)
        assert np.all(stats["status"] == gc.GC_OK), solver
        assert rel_err(g[c].cpu().numpy().astype(np.complex128), gr) < GTOL, solver
    del volt
    torch.cuda.empty_cache()


@pytest.mark.parametrize("L,C", [(8, 4), (32, 3), (64, 2), (128, 1)])
def test_gather_operator_equals_pair_scatter(gc, ctx, L, C):
    """The matrix-free Gauss-Newton operator J^T J has two forms: a gather
    over the grid (each antenna evaluates its own pairs; the default for
    selections of <= 16 baseline-types) and a scatter over the pair list
    ("cal.operator" = 1).  Both must land on the same solution.  The sizes
    cover every placement of the gathered vectors: shared memory with the
    coarse operators (8, 32), shared memory alone (64), global memory (128).
    Inputs: the paper's visibility-level simulation (Sec. 3) at SNR 10."""
    T = 2048
    sel = gc.Selection("subset", L, T)
    assert sel.n_ubl <= 16
    pt = sel.pair_type()
    tp = (sel.win_t1 - sel.win_t0)[pt]
    s, _, _ = synth.make_visibilities(50 + L, L, C, sel.pair_i, sel.pair_j, pt, sel.n_ubl, tp,
                                      snr=10.0, device="cuda")
    s = s.contiguous()
    assert ctx.get_tuning("cal.operator") == 0
    g0, v0, st0 = ctx.calibrate(s, sel, solver="lincal_cg")
    ctx.set_tuning("cal.operator", 1)
    try:
        g1, v1, st1 = ctx.calibrate(s, sel, solver="lincal_cg")
    finally:
        ctx.set_tuning("cal.operator", 0)
    ctx.device_status()
    for st in (st0, st1):
        stats = gc.decode_stats(st)
        assert np.all(stats["status"] == gc.GC_OK), (L, stats["status"])
    s0, s1 = gc.decode_stats(st0), gc.decode_stats(st1)
    assert np.allclose(s0["chi2"], s1["chi2"], rtol=1e-4)
    d = ((g0 - g1).abs() / g1.abs()).max().item()
    assert d < 1e-4, (L, d)
    dv = ((v0 - v1).abs() / v1.abs()).max().item()
    assert dv < 1e-4, (L, dv)
