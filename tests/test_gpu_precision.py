"""The 64 x 64 precision workload at full size (4096 antennas, 1024
channels, 8192 samples, 4+4-bit voltages) in the launch configuration the
benchmark times, checked on two sampled channels against the FP64 oracle:

* quantiser: the device bytes equal the oracle quantiser's bytes of the same
  complex64 draw (bit-exact); the oracle then works from its own bytes;
* FFT-correlator: sampled lags of V^unique against the oracle's one-lag
  definition (Eq. modelvis), lag-sum bound 1e-5;
* X-engine: every selected pair and every auto, bit-exact (int32 == int64);
* calibration (matrix-free lincal, FP32 products): gains within 1e-3 of the
  oracle's lincal (sparse form of the same normal equations) after the
  output convention.
"""
import numpy as np
import pytest
import torch

from oracle import calib as oc
from oracle import select as osel
from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu

L, C, T, N_SRC, SEED = 64, 1024, 8192, 200, 3
N = L * L
CHANNELS = (0, 777)


@pytest.fixture(scope="module")
def run():
    from paper_2005_03060_gb300 import gridcorr
    ctx = gridcorr.Context(0)
    dev = torch.device("cuda", 0)
    gains = synth.make_gains(SEED, C, N, device=dev)
    q = torch.empty(C, T, N, dtype=torch.uint8, device=dev)
    scales = torch.empty(C, dtype=torch.float32, device=dev)
    for c0 in range(0, C, 8):
        v, _, _ = synth.make_voltages(SEED, L, 8, T, n_src=N_SRC, device=dev, gains=gains[c0:c0 + 8], channel0=c0)
        ctx.quantize(v, out=q[c0:c0 + 8], scales=scales[c0:c0 + 8])
        del v
    sel = gridcorr.Selection("subset", L, T)
    vu = ctx.correlate(q, gains)
    vr, au = ctx.reduce(q, sel)
    g, V, st = ctx.calibrate(vr, sel, au, solver="lincal_cg", precision="fp32")
    ctx.device_status()
    out = {"sel": sel, "stats": gridcorr.decode_stats(st), "ch": {}}
    for c in CHANNELS:
        # the same channel's complex64 draw, on its own (the draws do not
        # depend on how the channels are chunked)
        v, _, _ = synth.make_voltages(SEED, L, 1, T, n_src=N_SRC, device=dev, gains=gains[c:c + 1], channel0=c)
        out["ch"][c] = {"volt": v[0].cpu().numpy(), "bytes": q[c].cpu().numpy(), "gains": gains[c].cpu().numpy(),
                        "vu": vu[c].cpu().numpy(), "vr": vr[c].cpu().numpy(), "au": au[c].cpu().numpy(),
                        "g": g[c].cpu().numpy().astype(np.complex128)}
        del v
    del q
    torch.cuda.empty_cache()
    return out


@pytest.fixture(scope="module")
def oracle_bytes(run, orc):
    return {c: orc.quantize(run["ch"][c]["volt"])[0] for c in CHANNELS}


def test_quantiser_bit_exact(run, oracle_bytes):
    for c in CHANNELS:
        assert np.array_equal(run["ch"][c]["bytes"], oracle_bytes[c]), c


def test_vunique_sampled_lags(run, orc, oracle_bytes):
    rng = np.random.default_rng(5)
    for c in CHANNELS:
        v = orc.unpack_i4c(oracle_bytes[c])
        g = run["ch"][c]["gains"]
        got = run["ch"][c]["vu"]
        r0 = orc.lag(v, g, L, 0, 0)
        lags = [(0, 0), (1, 0), (0, 1), (-63, 63), (63, 0), (0, -63)] + \
            [tuple(rng.integers(-(L - 1), L, 2)) for _ in range(14)]
        for dx, dy in lags:
            ref = orc.lag(v, g, L, int(dx), int(dy))
            nd = (L - abs(dx)) * (L - abs(dy))
            e = abs(got[dy + L - 1, dx + L - 1] - ref) * nd / (N * abs(r0))
            assert e < 1e-5, (c, dx, dy, e)


def test_xengine_all_pairs_bit_exact(run, orc, oracle_bytes):
    osl = osel.subset(L, T)
    pt = osl.pair_type()
    for c in CHANNELS:
        ref = orc.xengine_i4c(oracle_bytes[c], osl.pair_i, osl.pair_j, osl.win_t0[pt], osl.win_t1[pt])
        assert np.array_equal(run["ch"][c]["vr"].astype(np.int64), ref), c
        q = orc.unpack_i4c(oracle_bytes[c])
        ref_a = np.rint(np.sum(q.real ** 2 + q.imag ** 2, axis=0)).astype(np.int64)
        assert np.array_equal(run["ch"][c]["au"].astype(np.int64), ref_a), c


def test_calibration_matches_oracle(run, orc, oracle_bytes):
    assert np.all(run["stats"]["status"] == 0)
    osl = osel.subset(L, T)
    pt = osl.pair_type()
    for c in CHANNELS:
        raw = orc.xengine_i4c(oracle_bytes[c], osl.pair_i, osl.pair_j, osl.win_t0[pt], osl.win_t1[pt])
        vobs = (raw[:, 0] + 1j * raw[:, 1]) / T
        gr, Vr, it, ok = oc.calibrate(vobs, osl.pair_i, osl.pair_j, pt, osl.types, L, "lincal", sparse=True)
        assert ok, c
        e = float(np.max(np.abs(run["ch"][c]["g"] - gr) / np.abs(gr)))
        assert e < 1e-3, (c, e)


def test_vunique_all_lags_one_channel(run, orc, oracle_bytes):
    """Every one of the (2L-1)^2 = 16 129 lags of channel 0 at full size
    (4096 antennas x 8192 samples) against the FX definition (orc_fx_par,
    Eq. modelvis).  Bound: the lag-sum form, max_d |dV(d)| N_d / (N |V(0)|)
    <= 1e-5.  Also reported (printed): max_d |dV(d)| / |V(0)| and the relative
    L2 error over all lags; at the longest lags N_d is 1, so the FP32 FFT's
    rounding, spread evenly over the lag sums R(d) = T N_d V(d), shows there
    up to N / N_d times larger relative to V(0)."""
    c = CHANNELS[0]
    v = orc.unpack_i4c(oracle_bytes[c])
    ref, threads = orc.fx_par(v, run["ch"][c]["gains"], L)
    got = run["ch"][c]["vu"].astype(np.complex128)
    r = np.arange(-(L - 1), L)
    nd = (L - np.abs(r))[:, None] * (L - np.abs(r))[None, :]
    v0 = abs(ref[L - 1, L - 1])
    d = np.abs(got - ref)
    lag_sum = float(np.max(d * nd) / (N * v0))
    inf_rel = float(np.max(d) / v0)
    l2_rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    print(f"\nV^unique, channel {c}, all {ref.size} lags (oracle on {threads} threads): lag-sum "
          f"{lag_sum:.3e}, max|dV|/|V(0)| {inf_rel:.3e}, relative L2 {l2_rel:.3e}")
    assert lag_sum < 1e-5, lag_sum
