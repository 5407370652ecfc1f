"""Gain variance against array size for both reduced calibration schemes
(Sec. 4, Eq. for sigma_g^2 of low-cadence calibration; Sec. 5 / Sec. 6.1
for subset redundant calibration): the GPU calibration of the paper's own
visibility-level simulation (Sec. 3) on L x L grids, 64 realisations
(channels) per size, T = 4096 samples, SNR 10.

Pins, per scheme and size:
* the measured variance of the gain error after fixing the degeneracies
  against the truth agrees with Eq. gaincov's prediction
  (1 / (2 SNR^2 t)) diag[(A^T A)^+] (amplitude + phase), t the pair's
  integration time, within 15 %.  Every baseline-type has the same SNR
  (|V| = 1), the setting of the paper's variance curves, so that the
  uniform-weight solve is the optimal one Eq. gaincov describes (with
  visibility amplitudes spread over [0.5, 1.5] the uniform weights cost
  ~28 % extra variance, oracle and GPU alike);
* the variance decreases with N, as the paper's 1/log N scaling says
  (sigma_g^2 ~ 1 / (p log N t_cal)); the table of variance x log2 N is
  printed (run with -s to see it).
"""
import math

import numpy as np
import pytest
import torch

from oracle import calib as oc
from oracle import select as osel
from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu

GRIDS = [8, 12, 16, 24, 32]
C, T, SNR = 64, 4096, 10.0


@pytest.fixture(scope="module")
def sweep():
    from paper_2005_03060_gb300 import gridcorr
    ctx = gridcorr.Context(0)
    rows = []
    for scheme in ("subset", "lowcad"):
        for L in GRIDS:
            sel = gridcorr.Selection(scheme, L, T)
            pt = sel.pair_type()
            tp = (sel.win_t1 - sel.win_t0)[pt]
            S, g_true, _ = synth.make_visibilities(900 + L, L, C, sel.pair_i, sel.pair_j, pt, sel.n_ubl, tp,
                                                   snr=SNR, device="cuda", unit_amp=True)
            g, V, st = ctx.calibrate(S.contiguous(), sel, solver="lincal_cg", precision="fp32")
            ctx.device_status()
            stats = gridcorr.decode_stats(st)
            ge = g.cpu().numpy().astype(np.complex128)
            gt = g_true.cpu().numpy().astype(np.complex128)
            err = np.mean([np.mean(np.abs(oc.fit_degeneracies(ge[c], gt[c], L) / gt[c] - 1.0) ** 2)
                           for c in range(C)])
            osl = osel.subset(L, T) if scheme == "subset" else osel.lowcad(L, T)
            opt = osl.pair_type()
            pa, pp = oc.gain_variance_prediction(L, osl.types, osl.pair_i, osl.pair_j, opt)
            t = float(np.mean((osl.win_t1 - osl.win_t0)))
            pred = float(np.mean(pa + pp)) / (2.0 * SNR ** 2 * t)
            rows.append(dict(scheme=scheme, L=L, N=L * L, P=sel.P, t=t, measured=err, predicted=pred,
                             converged=int(np.sum(stats["status"] == 0))))
    print("\nscheme   L     N      P       t    sigma_g^2    Eq.gaincov   ratio  sigma_g^2*log2(N)")
    for r in rows:
        print(f"{r['scheme']:7s} {r['L']:3d} {r['N']:5d} {r['P']:7d} {r['t']:6.0f} {r['measured']:.3e}  "
              f"{r['predicted']:.3e}  {r['measured'] / r['predicted']:.3f}  {r['measured'] * math.log2(r['N']):.3e}")
    return rows


def test_all_channels_converge(sweep):
    for r in sweep:
        assert r["converged"] == C, r


def test_variance_follows_eq_gaincov(sweep):
    for r in sweep:
        assert 0.85 < r["measured"] / r["predicted"] < 1.15, r


def test_variance_decreases_with_array_size(sweep):
    for scheme in ("subset", "lowcad"):
        v = [r["measured"] for r in sweep if r["scheme"] == scheme]
        assert all(b < a for a, b in zip(v, v[1:])), (scheme, v)
