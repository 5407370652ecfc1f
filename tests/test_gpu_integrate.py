"""gc_integrate_host: one integration of host-resident voltages streamed in
channel chunks (copy of chunk i+1 overlapping the kernels of chunk i,
calibration on groups of chunks) gives what the three device calls give on
the whole integration: V^unique within the FP32 lag-sum bound, V^reduced
bit-exact for 4+4-bit voltages (FP32 bound for complex64), gains within the
solver tolerance."""
import numpy as np
import pytest
import torch

from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


@pytest.fixture(scope="module")
def ctx(gc):
    return gc.Context(0)


@pytest.mark.parametrize("vfmt,L,C,T,chunk", [("i4c", 16, 40, 300, 16), ("c64", 12, 37, 200, 0),
                                              ("i4c", 32, 9, 500, 4)])
def test_streamed_cycle_equals_device_calls(gc, ctx, vfmt, L, C, T, chunk):
    N, W = L * L, 2 * L - 1
    volt, gains, _ = synth.make_voltages(60 + L, L, C, T, n_src=20, device="cuda")
    if vfmt == "i4c":
        volt = ctx.quantize(volt)[0]
    sel = gc.Selection("subset", L, T)
    # reference: the three calls on the device-resident integration
    vu_ref = ctx.correlate(volt, gains)
    vr_ref, au_ref = ctx.reduce(volt, sel)
    g_ref, V_ref, st_ref = ctx.calibrate(vr_ref, sel, au_ref, solver="lincal_cg", precision="fp32")
    # streamed from pinned host memory
    h = torch.empty(volt.shape, dtype=volt.dtype, pin_memory=True)
    h.copy_(volt)
    vu = torch.empty(C, W, W, dtype=torch.complex64, device="cuda")
    vr = torch.empty_like(vr_ref)
    au = torch.empty_like(au_ref)
    g = torch.empty_like(gains)
    V = torch.empty_like(V_ref)
    st = torch.empty_like(st_ref)
    ctx.integrate_host(h, sel, gains, vu, vr, au, g, V, st, chunk=chunk)
    ctx.device_status()
    assert np.all(gc.decode_stats(st)["status"] == gc.GC_OK)
    a, b = vu.cpu().numpy(), vu_ref.cpu().numpy()
    r = np.arange(-(L - 1), L)
    nd = (L - np.abs(r))[:, None] * (L - np.abs(r))[None, :]
    for c in range(C):
        assert np.max(np.abs(a[c] - b[c]) * nd) / (N * abs(b[c, L - 1, L - 1])) < 1e-5
    if vfmt == "i4c":
        assert torch.equal(vr, vr_ref) and torch.equal(au, au_ref)
    else:
        assert ((vr - vr_ref).abs().max() / vr_ref.abs().max()).item() < 1e-5
    assert ((g - g_ref).abs() / g_ref.abs()).max().item() < 1e-4


def test_streamed_cycle_rejects_device_voltages(gc, ctx):
    L, C, T = 8, 2, 64
    volt, gains, _ = synth.make_voltages(1, L, C, T, n_src=3, device="cuda")
    sel = gc.Selection("subset", L, T)
    e = torch.empty(1, device="cuda")
    with pytest.raises(ValueError):
        ctx.integrate_host(volt, sel, gains, e, e, None, e, e, e)


@pytest.mark.parametrize("pinned", [True, False])
def test_streamed_cycle_with_host_gains(gc, ctx, pinned):
    """Gains handed over in host memory (page-locked or pageable) are copied
    by the library on its copy stream; two integrations in a row with
    different gains give what device-resident gains give (the gains buffer is
    not overwritten while the previous call's correlator still reads it)."""
    L, C, T = 16, 24, 256
    N, W = L * L, 2 * L - 1
    volt, _, _ = synth.make_voltages(71, L, C, T, n_src=20, device="cuda")
    volt = ctx.quantize(volt)[0]
    sel = gc.Selection("subset", L, T)
    h = torch.empty(volt.shape, dtype=volt.dtype, pin_memory=True)
    h.copy_(volt)
    outs = []
    for seed in (1, 2):
        _, gains, _ = synth.make_voltages(seed, L, C, 1, n_src=1)
        hg = torch.empty(gains.shape, dtype=gains.dtype, pin_memory=pinned)
        hg.copy_(gains)
        vu = torch.empty(C, W, W, dtype=torch.complex64, device="cuda")
        vr, au = ctx.reduce(volt, sel)
        g = torch.empty(C, N, dtype=torch.complex64, device="cuda")
        V = torch.empty(C, sel.n_ubl, dtype=torch.complex64, device="cuda")
        st = torch.empty(C, 32, dtype=torch.uint8, device="cuda")
        ctx.integrate_host(h, sel, hg, vu, vr, au, g, V, st, chunk=8)
        outs.append((vu, gains.cuda()))
    ctx.device_status()
    r = np.arange(-(L - 1), L)
    nd = (L - np.abs(r))[:, None] * (L - np.abs(r))[None, :]
    for vu, gd in outs:
        ref = ctx.correlate(volt, gd).cpu().numpy()
        a = vu.cpu().numpy()
        for c in range(C):
            assert np.max(np.abs(a[c] - ref[c]) * nd) / (N * abs(ref[c, L - 1, L - 1])) < 1e-5
