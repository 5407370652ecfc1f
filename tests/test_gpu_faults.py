"""Host-visible fault cases of the hot path, made on the host (bad inputs,
a tiny iteration cap); none of them traps, faults or hangs the GPU.

  * a zero or non-finite gain: w = v / g is undefined (Eq. modelvis); the
    correlator leaves the antenna out and gc_device_status reports GC_EINVAL;
  * NaN voltages: the correlator's spectra and the X-engine's FP32 sums are
    not finite; gc_device_status reports GC_EINVAL;
  * V^reduced with a NaN: that channel's calibration status is GC_EINVAL,
    the other channels are unaffected;
  * max_iter = 1: the solvers stop at the cap with GC_ENOCONV;
and after each, the context is clean again: the next good call succeeds.
"""
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


def _expect_einval(gc, ctx):
    with pytest.raises(gc.GridcorrError) as ei:
        ctx.device_status()
    assert ei.value.status == gc.GC_EINVAL


@pytest.mark.parametrize("bad", [0.0, float("inf"), float("nan")])
@pytest.mark.parametrize("fmt", ["c64", "i4c"])
def test_bad_gain_is_reported(gc, ctx, bad, fmt):
    L, C, T = 8, 2, 256
    volt, gains, _ = synth.make_voltages(11, L, C, T, n_src=20)
    v = volt.cuda()
    if fmt == "i4c":
        v, _ = ctx.quantize(v)
    g = gains.clone()
    g[1, 13] = complex(bad, 0.0)
    ctx.correlate(v, g.cuda())
    _expect_einval(gc, ctx)
    # the good channel is untouched by the bad antenna of channel 1, and the
    # word is clear again for the next call
    vu = ctx.correlate(v, gains.cuda())
    ctx.device_status()
    assert torch.isfinite(torch.view_as_real(vu)).all()


def test_nan_voltage_is_reported_by_correlator_and_xengine(gc, ctx):
    L, C, T = 8, 2, 256
    volt, gains, _ = synth.make_voltages(12, L, C, T, n_src=20)
    volt[0, 100, 5] = complex(float("nan"), 0.0)
    v = volt.cuda()
    ctx.correlate(v, gains.cuda())
    _expect_einval(gc, ctx)
    sel = gc.Selection("subset", L, T)
    ctx.reduce(v, sel)
    _expect_einval(gc, ctx)


def test_nonfinite_vreduced_fails_only_its_channel(gc, ctx):
    L, C, T = 8, 3, 256
    sel = gc.Selection("subset", L, T)
    volt, gains, _ = synth.make_voltages(13, L, C, T, n_src=20)
    vr, au = ctx.reduce(volt.cuda(), sel)
    ctx.device_status()
    vr[1, 7] = complex(float("nan"), 0.0)
    for solver in ("lincal_cg", "omnical", "lincal"):
        _, _, st = ctx.calibrate(vr, sel, au, solver=solver)
        s = gc.decode_stats(st)
        assert s["status"][1] == gc.GC_EINVAL, solver
        assert s["status"][0] == gc.GC_OK and s["status"][2] == gc.GC_OK, solver


@pytest.mark.parametrize("solver", ["lincal_cg", "omnical", "lincal"])
def test_iteration_cap_gives_enoconv(gc, ctx, solver):
    L, C, T = 8, 2, 256
    sel = gc.Selection("subset", L, T)
    volt, gains, _ = synth.make_voltages(14, L, C, T, n_src=20)
    vr, au = ctx.reduce(volt.cuda(), sel)
    _, _, st = ctx.calibrate(vr, sel, au, solver=solver, max_iter=1)
    s = gc.decode_stats(st)
    assert np.all(s["status"] == gc.GC_ENOCONV), (solver, s["status"])
    assert np.all(s["iters"] <= 1)
    # the default cap converges on the same data
    _, _, st = ctx.calibrate(vr, sel, au, solver=solver)
    assert np.all(gc.decode_stats(st)["status"] == gc.GC_OK)
