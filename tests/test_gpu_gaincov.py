"""gc_gain_variance (Eq. gaincov: diagonal of the pseudo-inverse of Eq.
logcal's normal matrices, the four degeneracies of Sec. 5.2 left out)
against the oracle's dense pseudo-inverse, per antenna and per baseline-type,
on square grids (subset and low-cadence) and hexagonal arrays."""
import numpy as np
import pytest

from oracle import calib as oc
from oracle import select as osel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


@pytest.fixture(scope="module")
def ctx(gc):
    return gc.Context(0)


def _oracle_full(N, types, pi, pj, alpha):
    AtA, BtB = oc.logcal_normal_matrices(N, types, pi, pj, alpha)
    ca = np.diag(np.linalg.pinv(AtA, rcond=1e-9, hermitian=True))
    cb = np.diag(np.linalg.pinv(BtB, rcond=1e-9, hermitian=True))
    return ca, cb


@pytest.mark.parametrize("scheme,L", [("subset", 6), ("subset", 12), ("lowcad", 6)])
def test_gain_variance_square(gc, ctx, scheme, L):
    sel = gc.Selection(scheme, L, 256)
    va, vp = ctx.gain_variance(sel)
    ctx.device_status()
    osl = osel.subset(L, 256) if scheme == "subset" else osel.lowcad(L, 256)
    ca, cb = _oracle_full(L * L, osl.types, osl.pair_i, osl.pair_j, osl.pair_type())
    np.testing.assert_allclose(va.cpu().numpy(), ca, rtol=2e-3)
    np.testing.assert_allclose(vp.cpu().numpy(), cb, rtol=2e-3)
    # the antenna part equals the oracle's Eq. gaincov prediction
    pa, pp = oc.gain_variance_prediction(L, osl.types, osl.pair_i, osl.pair_j, osl.pair_type())
    np.testing.assert_allclose(va.cpu().numpy()[:L * L], pa, rtol=2e-3)


@pytest.mark.parametrize("s", [3, 5])
def test_gain_variance_hex(gc, ctx, s):
    from paper_2005_03060_gb300 import synth
    L, m = synth.hex_mask(s)
    sel = gc.Selection("subset", L, 256, mask=m, lattice="triangular")
    va, vp = ctx.gain_variance(sel)
    ctx.device_status()
    va, vp = va.cpu().numpy(), vp.cpu().numpy()
    ref = osel.subset_layout(L, m, "triangular", 256)
    pi, pj, pos = osel.compact(ref, m)
    n = len(pos)
    ca, cb = _oracle_full(n, ref.types, pi, pj, ref.pair_type())
    occ = np.flatnonzero(m)
    np.testing.assert_allclose(va[occ], ca[:n], rtol=2e-3)
    np.testing.assert_allclose(vp[occ], cb[:n], rtol=2e-3)
    np.testing.assert_allclose(va[L * L:], ca[n:], rtol=2e-3)     # model visibilities (Eq. visvar form)
    np.testing.assert_allclose(vp[L * L:], cb[n:], rtol=2e-3)
    assert np.all(va[:L * L][m == 0] == 0) and np.all(vp[:L * L][m == 0] == 0)


def test_gain_variance_331(gc, ctx):
    """Fig. 13's 331-antenna hexagon: every unknown converges and matches the
    oracle; prints the time (run with -s)."""
    import torch
    from paper_2005_03060_gb300 import synth
    L, m = synth.hex_mask(11)
    sel = gc.Selection("subset", L, 1024, mask=m, lattice="triangular")
    ctx.gain_variance(sel)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    va, vp = ctx.gain_variance(sel)
    b.record()
    torch.cuda.synchronize()
    ctx.device_status()
    va, vp = va.cpu().numpy(), vp.cpu().numpy()
    ref = osel.subset_layout(L, m, "triangular", 1024)
    pi, pj, pos = osel.compact(ref, m)
    n = len(pos)
    ca, cb = _oracle_full(n, ref.types, pi, pj, ref.pair_type())
    occ = np.flatnonzero(m)
    assert np.all(np.isfinite(va)) and np.all(np.isfinite(vp))
    np.testing.assert_allclose(va[occ], ca[:n], rtol=2e-3)
    np.testing.assert_allclose(vp[occ], cb[:n], rtol=2e-3)
    print(f"\ngc_gain_variance hexagon 331 ({sel.P} pairs, {n + sel.n_ubl} unknowns): {a.elapsed_time(b):.1f} ms; "
          f"mean antenna variance (amp + phase) {np.mean(va[occ] + vp[occ]):.4e}")
