"""Parity of the reduced X-engine (gc_reduce) and the quantiser (gc_quantize)
with the FP64 oracle.

Tolerances: the 4+4-bit X-engine and its autos are bit-exact (int32 ==
oracle int64); the FP32 complex64 X-engine is bounded per pair by the
Cauchy-Schwarz scale of the sum, |S_gpu - S_ref| <= 1e-5 sqrt(A_i A_j) with
A the autos over the pair's window; the quantiser is bit-exact (codes and
per-channel scale).
"""
import numpy as np
import pytest
import torch

from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def gc():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


@pytest.fixture(scope="module")
def ctx(gc):
    return gc.Context(0)


def _pack(re, im):
    return ((np.asarray(re) & 15) << 4 | (np.asarray(im) & 15)).astype(np.uint8)


def _check_c64(orc, v, sel, got):
    """max over pairs of |S_gpu - S_ref| / sqrt(A_i A_j) (autos over the pair's window)."""
    pt = sel.pair_type()
    t0, t1 = sel.win_t0[pt], sel.win_t1[pt]
    ref = orc.xengine_c64(v, sel.pair_i, sel.pair_j, t0, t1)
    wins = {}
    for a, b in set(zip(t0.tolist(), t1.tolist())):
        wins[(a, b)] = orc.autos(v, a, b)
    ai = np.array([wins[(a, b)][i] for i, a, b in zip(sel.pair_i, t0, t1)])
    aj = np.array([wins[(a, b)][j] for j, a, b in zip(sel.pair_j, t0, t1)])
    return float(np.max(np.abs(got - ref) / np.sqrt(ai * aj)))


@pytest.mark.parametrize("scheme,L,C,T", [("subset", 3, 2, 40), ("subset", 8, 3, 256),
                                          ("subset", 12, 1, 500), ("lowcad", 4, 2, 120),
                                          ("lowcad", 8, 2, 256), ("subset", 32, 1, 300)])
def test_reduce_c64(gc, ctx, orc, scheme, L, C, T):
    sel = gc.Selection(scheme, L, T)
    volt, gains, _ = synth.make_voltages(400 + L, L, C, T, n_src=20)
    vr, au = ctx.reduce(volt.cuda(), sel)
    ctx.device_status()
    vr, au = vr.cpu().numpy(), au.cpu().numpy()
    used = sel.n_cycle * sel.t_int
    for c in range(C):
        v = volt[c].numpy().astype(np.complex128)
        assert _check_c64(orc, v, sel, vr[c]) < TOL
        ref_a = orc.autos(v, 0, used)
        assert np.max(np.abs(au[c] - ref_a) / ref_a) < TOL


@pytest.mark.parametrize("scheme,L,C,T", [("subset", 8, 2, 256), ("lowcad", 8, 1, 256),
                                          ("subset", 13, 1, 200), ("subset", 32, 1, 300)])
def test_reduce_c32h(gc, ctx, orc, scheme, L, C, T):
    """binary16-stored voltages (FP32 products and sums) against the oracle on
    the stored values, with the complex64 bound; L = 13 takes the plain
    staging path (a grid sample of 676 bytes is no multiple of 16)."""
    sel = gc.Selection(scheme, L, T)
    volt, gains, _ = synth.make_voltages(450 + L, L, C, T, n_src=20)
    h = torch.view_as_real(volt).to(torch.float16).contiguous()
    held = torch.view_as_complex(h.to(torch.float64)).numpy()
    vr, au = ctx.reduce(h.cuda(), sel)
    ctx.device_status()
    assert vr.dtype == torch.complex64 and au.dtype == torch.float32
    vr, au = vr.cpu().numpy(), au.cpu().numpy()
    used = sel.n_cycle * sel.t_int
    for c in range(C):
        assert _check_c64(orc, held[c], sel, vr[c]) < TOL
        ref_a = orc.autos(held[c], 0, used)
        assert np.max(np.abs(au[c] - ref_a) / ref_a) < TOL


@pytest.mark.parametrize("scheme,L,C,T", [("subset", 4, 2, 50), ("subset", 8, 2, 300),
                                          ("subset", 16, 1, 1000), ("lowcad", 8, 2, 256),
                                          ("lowcad", 16, 1, 2000), ("subset", 64, 1, 64)])
def test_reduce_i4c_exact(gc, ctx, orc, scheme, L, C, T):
    sel = gc.Selection(scheme, L, T)
    rng = np.random.default_rng(L * 7 + T)
    b = _pack(rng.integers(-7, 8, (C, T, L * L)), rng.integers(-7, 8, (C, T, L * L)))
    vr, au = ctx.reduce(torch.from_numpy(b).cuda(), sel)
    ctx.device_status()
    vr, au = vr.cpu().numpy(), au.cpu().numpy()
    pt = sel.pair_type()
    used = sel.n_cycle * sel.t_int
    for c in range(C):
        ref = orc.xengine_i4c(b[c], sel.pair_i, sel.pair_j, sel.win_t0[pt], sel.win_t1[pt])
        assert np.array_equal(vr[c].astype(np.int64), ref)
        q = orc.unpack_i4c(b[c])
        ref_a = np.sum(q[:used].real ** 2 + q[:used].imag ** 2, axis=0)
        assert np.array_equal(au[c].astype(np.int64), ref_a.astype(np.int64))


def test_reduce_i4c_worst_case_magnitude(gc, ctx, orc):
    """All voltages -7-7i over 8192 samples: |sum| = 802816 per pair, the
    largest the int32/FP32 path must hold exactly."""
    L, T = 8, 8192
    sel = gc.Selection("subset", L, T)
    b = np.full((1, T, L * L), _pack(-7, -7), np.uint8)
    vr = ctx.reduce(torch.from_numpy(b).cuda(), sel, autos=False).cpu().numpy()
    assert np.all(vr[0, :, 0] == 98 * T) and np.all(vr[0, :, 1] == 0)


def test_reduce_paper_scale_sampled(gc, ctx, orc):
    """32x32 grid, 256 channels, 4096 samples, subset selection (10446 pairs):
    every pair of two channels against the oracle."""
    L, C, T = 32, 256, 4096
    sel = gc.Selection("subset", L, T)
    volt = torch.empty(C, T, L * L, dtype=torch.complex64, device="cuda")
    volt, gains, _ = synth.make_voltages(2, L, C, T, n_src=200, device="cuda", out=volt)
    vr, au = ctx.reduce(volt, sel)
    ctx.device_status()
    vr = vr.cpu().numpy()
    for c in (3, 200):
        v = volt[c].cpu().numpy().astype(np.complex128)
        assert _check_c64(orc, v, sel, vr[c]) < TOL
    del volt
    torch.cuda.empty_cache()


@pytest.mark.parametrize("C,T,N", [(3, 100, 64), (2, 1000, 1024), (1, 7, 16)])
def test_quantize_exact(ctx, orc, C, T, N):
    volt, _, _ = synth.make_voltages(500 + N, int(round(N ** 0.5)), C, T, n_src=20)
    q, s = ctx.quantize(volt.cuda())
    q, s = q.cpu().numpy(), s.cpu().numpy()
    for c in range(C):
        ref, sc = orc.quantize(volt[c].numpy())
        assert np.float32(sc) == s[c]
        assert np.array_equal(q[c], ref)
