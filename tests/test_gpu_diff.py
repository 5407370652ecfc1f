"""The differentiation workload at full size: 128 x 128 grid (16 384
antennas), 512 channels, 4096 samples, 4+4-bit voltages, subset selection
(224 786 pairs).  The chi^2 of the redundant model over V^reduced (Eq.
redchi numerator) through the autograd Function, in both forms (residuals
recomputed in the backward pass, or checkpointed by the forward pass):

* forward: two sampled channels against the FP64 oracle chi^2 (relative 1e-5);
* backward: against the FP64 oracle gradient (1e-4 of the largest component);
  the checkpointed and recomputed backward passes agree;
* central finite differences (step 1e-4 relative) of the GPU forward;
* a gradient-driven solve (L-BFGS on the autograd Function, checkpointed
  form) started from the Gauss-Newton solution with 1 % phase noise returns
  to the Gauss-Newton minimum (Sec. 2: the result does not depend on the
  solver).
The evaluation point is the true gains with 1 % phase noise and the group
means of V_p / (g_i conj g_j); for the sampled channels the oracle builds it
from its own quantiser and X-engine (whose sums equal the device's bit for
bit).
"""
import numpy as np
import pytest
import torch

from oracle import calib as oc
from oracle import select as osel
from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu

L, C, T, N_SRC, SEED = 128, 512, 4096, 200, 5
N = L * L
CHANNELS = (0, 301)


@pytest.fixture(scope="module")
def run(orc):
    from paper_2005_03060_gb300 import gridcorr
    ctx = gridcorr.Context(0)
    dev = torch.device("cuda", 0)
    gains = synth.make_gains(SEED, C, N, device=dev)
    q = torch.empty(C, T, N, dtype=torch.uint8, device=dev)
    for c0 in range(0, C, 8):
        v, _, _ = synth.make_voltages(SEED, L, 8, T, n_src=N_SRC, device=dev, gains=gains[c0:c0 + 8], channel0=c0)
        ctx.quantize(v, out=q[c0:c0 + 8])
        del v
    sel = gridcorr.Selection("subset", L, T)
    vr, au = ctx.reduce(q, sel)
    del q
    torch.cuda.empty_cache()
    g_gn, V_gn, st = ctx.calibrate(vr, sel, au, solver="lincal_cg", precision="fp32")
    ctx.device_status()
    assert np.all(gridcorr.decode_stats(st)["status"] == 0)
    # evaluation point: the true gains with 1 % phase noise, model visibilities
    # the group means of V_p / (g_i conj g_j) there
    rng = torch.Generator(device=dev)
    rng.manual_seed(11)
    ph = 0.01 * torch.randn(C, N, generator=rng, device=dev)
    g0 = (gains * torch.polar(torch.ones_like(ph), ph)).contiguous()
    osl = osel.subset(L, T)
    pt = osl.pair_type()
    t = (osl.win_t1 - osl.win_t0)[pt]
    pi_, pj_, pt_ = (torch.as_tensor(a, device=dev, dtype=torch.long) for a in (osl.pair_i, osl.pair_j, pt))
    vobs_all = torch.complex(vr[..., 0].double(), vr[..., 1].double()) / torch.as_tensor(t, device=dev)
    e = g0[:, pi_].to(torch.complex128) * g0[:, pj_].to(torch.complex128).conj()
    V0 = torch.zeros(C, sel.n_ubl, dtype=torch.complex128, device=dev)
    V0.index_add_(1, pt_, vobs_all / e)
    V0 = (V0 / torch.bincount(pt_, minlength=sel.n_ubl).to(dev)).to(torch.complex64)
    ora = {}
    for c in CHANNELS:
        # the oracle's own inputs for this channel: its quantiser on the same
        # complex64 draw, its X-engine, its evaluation point
        v, _, _ = synth.make_voltages(SEED, L, 1, T, n_src=N_SRC, device=dev, gains=gains[c:c + 1], channel0=c)
        b, _ = orc.quantize(v[0].cpu().numpy())
        del v
        raw = orc.xengine_i4c(b, osl.pair_i, osl.pair_j, osl.win_t0[pt], osl.win_t1[pt])
        assert np.array_equal(raw, vr[c].cpu().numpy().astype(np.int64)), c
        vobs = (raw[:, 0] + 1j * raw[:, 1]) / t
        g = g0[c].cpu().numpy().astype(np.complex128)
        Vs = np.zeros(sel.n_ubl, np.complex128)
        np.add.at(Vs, pt, vobs / (g[osl.pair_i] * np.conj(g[osl.pair_j])))
        Vs = (Vs / np.bincount(pt, minlength=sel.n_ubl)).astype(np.complex64)
        V0[c] = torch.from_numpy(Vs).to(dev)
        ora[c] = (vobs, g, Vs.astype(np.complex128))
    V0 = V0.contiguous()
    out = {"ctx": ctx, "sel": sel, "vr": vr, "g_gn": g_gn, "V_gn": V_gn, "g0": g0, "V0": V0, "gc": gridcorr,
           "ora": ora, "osl": osl, "pt": pt}
    for ckpt in (False, True):
        g = g0.clone().requires_grad_(True)
        V = V0.clone().requires_grad_(True)
        c2 = gridcorr.chi2(g, V, vr, sel, ctx, checkpoint=ckpt)
        c2.sum().backward()
        out[ckpt] = (c2.detach(), g.grad.detach(), V.grad.detach())
    ctx.device_status()
    return out


def _oracle(run, orc, c):
    vobs, g, V = run["ora"][c]
    osl, pt = run["osl"], run["pt"]
    args = (vobs, g, V, osl.pair_i, osl.pair_j, pt)
    return oc.chi2(*args), oc.chi2_grad(*args)


def test_forward_and_gradient_match_oracle(run, orc):
    for ckpt in (False, True):
        c2, dg, dv = run[ckpt]
        for c in CHANNELS:
            ref, (rg, rv) = _oracle(run, orc, c)
            assert float(c2[c]) == pytest.approx(ref, rel=1e-5), (ckpt, c)
            scale = max(np.max(np.abs(rg)), np.max(np.abs(rv)))
            assert np.max(np.abs(dg[c].cpu().numpy() - rg)) < 1e-4 * scale, (ckpt, c)
            assert np.max(np.abs(dv[c].cpu().numpy() - rv)) < 1e-4 * scale, (ckpt, c)


def test_checkpointed_equals_recomputed(run):
    a, b = run[False], run[True]
    assert torch.equal(a[0], b[0])
    for x, y in zip(a[1:], b[1:]):
        assert ((x - y).abs().max() / x.abs().max()).item() < 1e-6


def test_central_finite_differences(run):
    ctx, sel, vr, gc = run["ctx"], run["sel"], run["vr"], run["gc"]
    c = CHANNELS[1]
    vr1 = vr[c:c + 1].contiguous()
    g0 = run["g0"][c:c + 1].contiguous()
    V0 = run["V0"][c:c + 1].contiguous()
    _, dg, dv = run[False]
    rng = np.random.default_rng(3)
    for _ in range(6):
        which = int(rng.integers(0, 2))
        k = int(rng.integers(0, N if which == 0 else sel.n_ubl))
        for unit in (1.0, 1j):
            base = (g0 if which == 0 else V0)
            h = 1e-4 * abs(base[0, k].item())
            f = []
            for sgn in (1.0, -1.0):
                x = base.clone()
                x[0, k] += sgn * unit * h
                gg, vv = (x, V0) if which == 0 else (g0, x)
                f.append(float(ctx.chi2(vr1, sel, gg, vv)[0]))
            fd = (f[0] - f[1]) / (2 * h)
            grad = (dg if which == 0 else dv)[c, k].item()
            an = grad.real if unit == 1.0 else grad.imag
            assert fd == pytest.approx(an, rel=2e-2, abs=2e-2 * abs(grad)), (which, k, unit)


def test_gradient_driven_solve_reaches_gauss_newton(run):
    ctx, sel, vr, gc = run["ctx"], run["sel"], run["vr"], run["gc"]
    cs = slice(0, 2)
    vr2 = vr[cs].contiguous()
    g_gn, V_gn = run["g_gn"][cs].contiguous(), run["V_gn"][cs].contiguous()
    c2_gn = ctx.chi2(vr2, sel, g_gn, V_gn).cpu().numpy()
    # start: the Gauss-Newton point with 1 % phase noise on every gain
    rng = torch.Generator(device=g_gn.device)
    rng.manual_seed(21)
    ph = 0.01 * torch.randn(g_gn.shape, generator=rng, device=g_gn.device)
    gr = torch.view_as_real((g_gn * torch.polar(torch.ones_like(ph), ph)).contiguous()).clone().requires_grad_(True)
    Vr = torch.view_as_real(V_gn.clone()).clone().requires_grad_(True)
    opt = torch.optim.LBFGS([gr, Vr], lr=1.0, max_iter=1500, tolerance_grad=1e-14, tolerance_change=1e-16,
                            history_size=50, line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        loss = gc.chi2(torch.view_as_complex(gr), torch.view_as_complex(Vr), vr2, sel, ctx,
                       checkpoint=True).sum()
        loss.backward()
        return loss

    opt.step(closure)
    g = torch.view_as_complex(gr.detach())
    V = torch.view_as_complex(Vr.detach())
    c2 = ctx.chi2(vr2, sel, g, V).cpu().numpy()
    assert np.all(np.abs(c2 - c2_gn) <= 1e-3 * c2_gn), (c2, c2_gn)
    osl = osel.subset(L, T)
    for c in range(2):
        gp, _ = oc.project(g[c].cpu().numpy().astype(np.complex128), V[c].cpu().numpy().astype(np.complex128),
                           osl.types, L)
        ref = g_gn[c].cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(gp - ref) / np.abs(ref)) < 5e-3
