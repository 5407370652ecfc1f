"""chi^2 forward / adjoint kernels and the autograd Function against the FP64
oracle (oracle.calib.chi2 / chi2_grad, whose gradient is pinned to finite
differences in test_oracle_calib), central finite differences of the GPU
forward, and a gradient-driven solve compared with Gauss-Newton lincal.

Tolerances: chi^2 relative 1e-5 (FP32 residuals, FP64 sums); gradients
1e-4 of the largest component (FP32 products); finite differences 2e-2
(step 1e-3 relative on an FP32 forward)."""
import numpy as np
import pytest
import torch

from oracle import calib as oc
from oracle import select as osel
from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


@pytest.fixture(scope="module")
def ctx(gc):
    return gc.Context(0)


def _problem(gc, scheme, L, T, C, seed, weights=False):
    rng = np.random.default_rng(seed)
    sel = gc.Selection(scheme, L, T)
    osl = osel.subset(L, T) if scheme == "subset" else osel.lowcad(L, T)
    N = L * L
    S = (rng.standard_normal((C, sel.P)) + 1j * rng.standard_normal((C, sel.P))).astype(np.complex64) * 50
    g = ((1 + 0.1 * rng.standard_normal((C, N))) * np.exp(1j * rng.uniform(-np.pi, np.pi, (C, N)))).astype(
        np.complex64)
    V = (rng.standard_normal((C, sel.n_ubl)) + 1j * rng.standard_normal((C, sel.n_ubl))).astype(np.complex64)
    w = rng.uniform(0.5, 2.0, (C, sel.P)).astype(np.float32) if weights else None
    return sel, osl, S, g, V, w


def _oracle(osl, S, g, V, w, c):
    pt = osl.pair_type()
    t = (osl.win_t1 - osl.win_t0)[pt]
    vobs = S[c].astype(np.complex128) / t
    ww = None if w is None else w[c].astype(np.float64)
    args = (vobs, g[c].astype(np.complex128), V[c].astype(np.complex128), osl.pair_i, osl.pair_j, pt)
    return oc.chi2(*args, w=ww), oc.chi2_grad(*args, w=ww)


@pytest.mark.parametrize("scheme,L,T,weights", [("subset", 6, 100, False), ("subset", 8, 256, True),
                                                ("lowcad", 5, 300, True), ("subset", 32, 4096, False)])
def test_forward_backward_match_oracle(gc, ctx, scheme, L, T, weights):
    C = 3
    sel, osl, S, g, V, w = _problem(gc, scheme, L, T, C, L + T, weights)
    dev = "cuda"
    vr = torch.from_numpy(S).to(dev)
    gt, Vt = torch.from_numpy(g).to(dev), torch.from_numpy(V).to(dev)
    wt = torch.from_numpy(w).to(dev) if w is not None else None
    c2 = ctx.chi2(vr, sel, gt, Vt, wt).cpu().numpy()
    go = torch.tensor([1.0, -0.5, 2.0], dtype=torch.float64, device=dev)
    dg, dv = ctx.chi2_backward(vr, sel, gt, Vt, go, wt)
    ctx.device_status()
    dg, dv = dg.cpu().numpy(), dv.cpu().numpy()
    for c in range(C):
        ref, (rg, rv) = _oracle(osl, S, g, V, w, c)
        assert c2[c] == pytest.approx(ref, rel=1e-5)
        s = float(go[c])
        scale = max(np.max(np.abs(rg)), np.max(np.abs(rv))) * abs(s)
        assert np.max(np.abs(dg[c] - s * rg)) < 1e-4 * scale
        assert np.max(np.abs(dv[c] - s * rv)) < 1e-4 * scale


def test_autograd_matches_finite_differences(gc, ctx):
    L, T, C = 5, 50, 2
    sel, osl, S, g, V, w = _problem(gc, "subset", L, T, C, 77)
    vr = torch.from_numpy(S).cuda()
    gt = torch.from_numpy(g).cuda().requires_grad_(True)
    Vt = torch.from_numpy(V).cuda().requires_grad_(True)
    loss = gc.chi2(gt, Vt, vr, sel, ctx).sum()
    loss.backward()
    rng = np.random.default_rng(3)
    for _ in range(8):
        which = rng.integers(0, 2)
        c = int(rng.integers(0, C))
        k = int(rng.integers(0, L * L if which == 0 else sel.n_ubl))
        for unit in (1.0, 1j):
            base = (g if which == 0 else V).copy()
            h = 1e-3 * abs(base[c, k])
            plus, minus = base.copy(), base.copy()
            plus[c, k] += unit * h
            minus[c, k] -= unit * h
            f = []
            for arr in (plus, minus):
                gg = torch.from_numpy(arr if which == 0 else g).cuda()
                vv = torch.from_numpy(V if which == 0 else arr).cuda()
                f.append(float(ctx.chi2(vr, sel, gg, vv)[c]))
            fd = (f[0] - f[1]) / (2 * h)
            grad = (gt.grad if which == 0 else Vt.grad)[c, k].item()
            an = grad.real if unit == 1.0 else grad.imag
            assert fd == pytest.approx(an, rel=2e-2, abs=2e-2 * abs(grad))


def test_gradient_driven_solve_matches_gauss_newton(gc, ctx):
    """chi^2 minimised through the autograd Function (L-BFGS) reaches the
    Gauss-Newton lincal minimum (Sec. 2: results do not depend on the solver)."""
    L, C, T = 6, 2, 512
    volt, gains, _ = synth.make_voltages(12, L, C, T, n_src=20)
    sel = gc.Selection("subset", L, T)
    vr, au = ctx.reduce(volt.cuda(), sel)
    g_gn, V_gn, st = ctx.calibrate(vr, sel, au, solver="lincal", precision="fp64")
    c2_gn = ctx.chi2(vr, sel, g_gn, V_gn).cpu().numpy()
    rng = np.random.default_rng(5)
    g0 = g_gn.cpu().numpy() * np.exp(1j * 0.05 * rng.standard_normal(g_gn.shape))
    V0 = V_gn.cpu().numpy() * (1 + 0.05 * rng.standard_normal(V_gn.shape))
    # optimise real views of the complex parameters
    gr = torch.view_as_real(torch.from_numpy(g0.astype(np.complex64))).clone().cuda().requires_grad_(True)
    Vr = torch.view_as_real(torch.from_numpy(V0.astype(np.complex64))).clone().cuda().requires_grad_(True)
    opt = torch.optim.LBFGS([gr, Vr], lr=1.0, max_iter=400, tolerance_grad=1e-12, tolerance_change=1e-15,
                            history_size=50, line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        loss = gc.chi2(torch.view_as_complex(gr), torch.view_as_complex(Vr), vr, sel, ctx).sum()
        loss.backward()
        return loss

    opt.step(closure)
    g = torch.view_as_complex(gr.detach())
    V = torch.view_as_complex(Vr.detach())
    c2 = ctx.chi2(vr, sel, g.detach(), V.detach()).cpu().numpy()
    assert np.all(np.abs(c2 - c2_gn) <= 1e-3 * c2_gn)
    # same point up to the degeneracies
    osl = osel.subset(L, T)
    for c in range(C):
        gp, _ = oc.project(g.detach()[c].cpu().numpy().astype(np.complex128),
                           V.detach()[c].cpu().numpy().astype(np.complex128), osl.types, L)
        gr = g_gn[c].cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(gp - gr) / np.abs(gr)) < 5e-3



@pytest.mark.parametrize("L,weights,i4c", [(17, True, False), (64, False, True), (128, True, True)])
def test_adjoint_is_deterministic(gc, ctx, L, weights, i4c):
    """The adjoint's sums have a fixed order (slots ordered by a barrier per
    type, CTA partials added in range order, the halo terms after): two runs
    give the same bits.  One and several antenna ranges per channel."""
    C = 3
    sel, osl, S, g, V, w = _problem(gc, "subset", L, 256, C, 700 + L, weights)
    dev = "cuda"
    if i4c:
        vr = torch.from_numpy(np.stack([np.round(S.real), np.round(S.imag)], -1).astype(np.int32)).to(dev)
    else:
        vr = torch.from_numpy(S).to(dev)
    gt, Vt = torch.from_numpy(g).to(dev), torch.from_numpy(V).to(dev)
    wt = torch.from_numpy(w).to(dev) if w is not None else None
    go = torch.tensor([1.0, -0.5, 2.0], dtype=torch.float64, device=dev)
    a = [t.cpu().numpy() for t in ctx.chi2_backward(vr, sel, gt, Vt, go, wt)]
    b = [t.cpu().numpy() for t in ctx.chi2_backward(vr, sel, gt, Vt, go, wt)]
    ctx.device_status()
    assert np.isfinite(a[0]).all() and np.isfinite(a[1]).all()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
