"""Parity of the tensor-core reduced X-engine (xeng_tc_accumulate: tcgen05
kind::f8f6f4 MMAs on offset-coded 4+4-bit voltages) with the FP64 oracle.

Bar: bit-exact.  V^reduced and the autos must equal the oracle's int64 sums
(orc_xeng_i4c) element by element, on grids whose 128-antenna blocks are whole
rows (L = 16, 32, 64), ragged integrations (T not a multiple of the 32-sample
stage), several time slices, the full 4-bit range [-8, 7] and the largest sums
a 32768-sample slice can hold.  The SIMT dp4a path ("xeng.path" = 1) is run
on the same inputs and must agree too.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


@pytest.fixture(scope="module")
def ctx(gc):
    c = gc.Context(0)
    yield c
    c.set_tuning("xeng.path", 0)
    c.set_tuning("xeng.tsplit", 0)


def _pack(re, im):
    return ((np.asarray(re) & 15) << 4 | (np.asarray(im) & 15)).astype(np.uint8)


def _oracle(orc, b, sel):
    pt = sel.pair_type()
    return orc.xengine_i4c(b, sel.pair_i, sel.pair_j, sel.win_t0[pt], sel.win_t1[pt])


def _autos(orc, b, t1):
    q = orc.unpack_i4c(b)[:t1]
    return np.sum(q.real ** 2 + q.imag ** 2, axis=0).astype(np.int64)


def _run(ctx, b, sel, path, tsplit=0):
    ctx.set_tuning("xeng.path", path)
    ctx.set_tuning("xeng.tsplit", tsplit)
    try:
        ctx.profile(True)
        vr, au = ctx.reduce(torch.from_numpy(b).cuda(), sel)
        ctx.device_status()
        kinds = ctx.profile_read()
    finally:
        ctx.profile(False)
        ctx.set_tuning("xeng.path", 0)
        ctx.set_tuning("xeng.tsplit", 0)
    return vr.cpu().numpy().astype(np.int64), au.cpu().numpy().astype(np.int64), kinds


@pytest.mark.parametrize("L,C,T,Tsel,lo,hi", [
    (16, 2, 1000, 1000, -7, 8),     # ragged: 31 stages + 8 samples
    (16, 3, 64, 50, -8, 8),         # buffer longer than the window, full 4-bit range
    (32, 2, 300, 300, -8, 8),
    (64, 2, 512, 512, -7, 8),
    (64, 1, 33, 33, -8, 8),         # one full stage + one sample
    (64, 2, 4096, 4000, -7, 8),
])
def test_tc_matches_oracle(gc, ctx, orc, L, C, T, Tsel, lo, hi):
    sel = gc.Selection("subset", L, Tsel)
    rng = np.random.default_rng(L * 31 + T)
    b = _pack(rng.integers(lo, hi, (C, T, L * L)), rng.integers(lo, hi, (C, T, L * L)))
    vr, au, kinds = _run(ctx, b, sel, 2)
    assert "xeng_tc_accumulate" in kinds
    for c in range(C):
        assert np.array_equal(vr[c], _oracle(orc, b[c], sel))
        assert np.array_equal(au[c], _autos(orc, b[c], Tsel))
    vr1, au1, kinds1 = _run(ctx, b, sel, 1)
    assert "xeng_tc_accumulate" not in kinds1
    assert np.array_equal(vr, vr1) and np.array_equal(au, au1)


@pytest.mark.parametrize("tsplit", [2, 5, 16])
def test_tc_time_slices(gc, ctx, orc, tsplit):
    """The window split into slices (partial sums per slice, summed by
    xeng_reduce) gives the same exact sums; slice edges fall inside stages."""
    L, C, T = 32, 2, 2100
    sel = gc.Selection("subset", L, T)
    rng = np.random.default_rng(tsplit)
    b = _pack(rng.integers(-8, 8, (C, T, L * L)), rng.integers(-8, 8, (C, T, L * L)))
    vr, au, _ = _run(ctx, b, sel, 2, tsplit)
    for c in range(C):
        assert np.array_equal(vr[c], _oracle(orc, b[c], sel))
        assert np.array_equal(au[c], _autos(orc, b[c], T))


@pytest.mark.parametrize("re,im", [(-7, -7), (7, 7), (-8, -8), (7, -8), (0, 0)])
def test_tc_extreme_constant_voltages(gc, ctx, re, im):
    """Constant voltages over 8192 samples: every pair sum is |v|^2 T, up to
    (64 + 64) 8192 = 1 048 576 -- the extremes of the codes (u = 0 and
    u = 15) and of the FP32 accumulator (|D1| up to 450 T)."""
    L, T = 64, 8192
    sel = gc.Selection("subset", L, T)
    b = np.full((1, T, L * L), _pack(re, im), np.uint8)
    vr, au, kinds = _run(ctx, b, sel, 2)
    assert "xeng_tc_accumulate" in kinds
    p2 = re * re + im * im
    assert np.all(vr[0, :, 0] == p2 * T) and np.all(vr[0, :, 1] == 0)
    assert np.all(au[0] == p2 * T)


def test_tc_alternating_extremes(gc, ctx, orc):
    """Samples alternating between -8-8i and 7+7i, antennas out of phase by
    row parity: partial sums swing through the largest magnitudes and
    cancel, exercising exactness of every intermediate sum."""
    L, T = 16, 4096
    sel = gc.Selection("subset", L, T)
    t = np.arange(T)[:, None]
    y = (np.arange(L * L) // L)[None, :]
    hi = ((t + y) % 2 == 0)
    q = np.where(hi, 7, -8)
    b = _pack(q, q)[None]
    vr, au, _ = _run(ctx, b, sel, 2)
    assert np.array_equal(vr[0], _oracle(orc, b[0], sel))
    assert np.array_equal(au[0], _autos(orc, b[0], T))


def test_tc_not_taken_where_not_covered(gc, ctx):
    """Low-cadence selections (one window per cycle), complex64 voltages and
    grids whose blocks are not whole rows keep the SIMT path under the
    automatic choice, and the forced tensor path refuses them."""
    L, T = 16, 256
    low = gc.Selection("lowcad", L, T)
    b = torch.zeros(1, T, L * L, dtype=torch.uint8, device="cuda")
    ctx.profile(True)
    ctx.reduce(b, low)
    kinds = ctx.profile_read()
    ctx.profile(False)
    assert "xeng_tc_accumulate" not in kinds
    ctx.set_tuning("xeng.path", 2)
    try:
        with pytest.raises(gc.GridcorrError):
            ctx.reduce(b, low)
        sub12 = gc.Selection("subset", 12, T)
        with pytest.raises(gc.GridcorrError):
            ctx.reduce(torch.zeros(1, T, 144, dtype=torch.uint8, device="cuda"), sub12)
    finally:
        ctx.set_tuning("xeng.path", 0)
