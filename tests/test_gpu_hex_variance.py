"""Gain variance of both reduced calibration schemes on hexagonal arrays --
the paper's own layout and its Fig. 13 comparison on 331 antennas -- from
the GPU calibration of the paper's visibility-level simulation (Sec. 3):
64 realisations (channels) per size, T = 4096, SNR 10, every baseline-type
at |V| = 1.  Pins per scheme and size: the measured variance of the gain
error after fixing the degeneracies against the truth agrees with Eq.
gaincov ((1 / (2 SNR^2 t)) diag[(A^T A)^+], amplitude + phase, in the
occupied-antenna numbering) within 15 %, and follows its trend with N; on
the 331-antenna array low-cadence beats subset calibration.  The table is
printed (-s)."""
import math

import numpy as np
import pytest

from oracle import calib as oc
from oracle import select as osel
from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu

SIDES = [4, 6, 8, 11]
C, T, SNR = 64, 4096, 10.0


@pytest.fixture(scope="module")
def sweep():
    from paper_2005_03060_gb300 import gridcorr
    ctx = gridcorr.Context(0)
    rows = []
    for scheme in ("subset", "lowcad"):
        for s in SIDES:
            L, m = synth.hex_mask(s)
            occ = np.flatnonzero(m)
            sel = gridcorr.Selection(scheme, L, T, mask=m, lattice="triangular")
            pt = sel.pair_type()
            tp = (sel.win_t1 - sel.win_t0)[pt]
            S, g_true, _ = synth.make_visibilities(700 + s, L, C, sel.pair_i, sel.pair_j, pt, sel.n_ubl, tp,
                                                   snr=SNR, device="cuda", unit_amp=True)
            g, V, st = ctx.calibrate(S.contiguous(), sel, solver="lincal_cg", precision="fp32")
            ctx.device_status()
            stats = gridcorr.decode_stats(st)
            ge = g.cpu().numpy().astype(np.complex128)[:, occ]
            gt = g_true.cpu().numpy().astype(np.complex128)[:, occ]
            pos = np.stack([occ % L, occ // L], 1).astype(float)
            err = np.mean([np.mean(np.abs(oc.fit_degeneracies(ge[c], gt[c], pos) / gt[c] - 1.0) ** 2)
                           for c in range(C)])
            osl = (osel.subset_layout if scheme == "subset" else osel.lowcad_layout)(L, m, "triangular", T)
            pi, pj, _ = osel.compact(osl, m)
            pa, pp = oc.gain_variance_prediction(None, osl.types, pi, pj, osl.pair_type(), N=len(occ))
            t = float(np.mean(osl.win_t1 - osl.win_t0))
            pred = float(np.mean(pa + pp)) / (2.0 * SNR ** 2 * t)
            rows.append(dict(scheme=scheme, s=s, N=len(occ), P=sel.P, t=t, measured=err, predicted=pred,
                             converged=int(np.sum(stats["status"] == 0))))
    print("\nscheme   side    N      P       t    sigma_g^2    Eq.gaincov   ratio  sigma_g^2*log2(N)")
    for r in rows:
        print(f"{r['scheme']:7s} {r['s']:4d} {r['N']:5d} {r['P']:7d} {r['t']:6.0f} {r['measured']:.3e}  "
              f"{r['predicted']:.3e}  {r['measured'] / r['predicted']:.3f}  {r['measured'] * math.log2(r['N']):.3e}")
    return rows


def test_hex_all_channels_converge(sweep):
    for r in sweep:
        assert r["converged"] == C, r


def test_hex_variance_follows_eq_gaincov(sweep):
    for r in sweep:
        assert 0.85 < r["measured"] / r["predicted"] < 1.15, r


def test_hex_variance_trend_follows_eq_gaincov(sweep):
    """Where Eq. gaincov predicts a change of more than 5 % between sizes, the
    measured variance moves the same way (on hexagons the subset prediction
    flattens between 169 and 331 antennas, the deviation from the 1/log N
    approximation the paper notes for subset calibration)."""
    for scheme in ("subset", "lowcad"):
        rs = [r for r in sweep if r["scheme"] == scheme]
        for a, b in zip(rs, rs[1:]):
            dp = b["predicted"] / a["predicted"] - 1.0
            if abs(dp) > 0.05:
                assert (b["measured"] - a["measured"]) * dp > 0, (scheme, a, b)


def test_lowcad_beats_subset_on_331_antennas(sweep):
    """Fig. 13's array: with the same correlation budget (p N log N pairs per
    cycle), low-cadence calibration gives the lower gain variance, as Eq.
    gaincov predicts."""
    sub = [r for r in sweep if r["scheme"] == "subset" and r["s"] == 11][0]
    low = [r for r in sweep if r["scheme"] == "lowcad" and r["s"] == 11][0]
    assert low["predicted"] < sub["predicted"] and low["measured"] < sub["measured"]
