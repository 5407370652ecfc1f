"""Oracle pins for arrays on a partly occupied lattice -- the paper's
hexagonal arrays (Sec. 3, Fig. 13's 331-antenna array) -- held as a masked
L x L grid of triangular-lattice points.

Pinned against: the hexagon's antenna count 3 s (s - 1) + 1 and its six-fold
symmetry; the count 3 s^2 - 5 s + 2 of unit-length pairs per direction; the
degeneracy criterion of Sec. 5.2 by exact rank (two unit directions leave a
fifth, checkerboard-amplitude degeneracy, the third removes it); the masked
FX correlator against the grid FX oracle (all points occupied) and against
pair-by-pair sums; exact recovery of injected gains from noise-free
redundant data on a hexagonal array (Sec. 3 procedure, up to the four
degeneracies)."""
import numpy as np
import pytest

from oracle import calib as oc
from oracle import select as osel
from paper_2005_03060_gb300 import synth


@pytest.mark.parametrize("s", range(2, 12))
def test_hex_mask_count_and_symmetry(s):
    L, m = osel.hex_mask(s)
    assert L == 2 * s - 1 and int(m.sum()) == 3 * s * (s - 1) + 1
    occ = {(i % L - (s - 1), i // L - (s - 1)) for i in np.flatnonzero(m)}
    assert {(-b, a + b) for a, b in occ} == occ          # 60-degree rotation in axial coordinates


@pytest.mark.parametrize("s", [3, 6, 11])
def test_hex_types_and_unit_pair_counts(s):
    L, m = osel.hex_mask(s)
    ts, cnt = osel.layout_types(L, m, "triangular")
    assert ts[:3] == [(1, 0), (0, 1), (-1, 1)]
    assert cnt[:3] == [3 * s * s - 5 * s + 2] * 3
    assert ts[3:6] == [(1, 1), (-1, 2), (-2, 1)]           # length sqrt(3), by angle 30, 90, 150 degrees
    lens = [osel.type_length2(d, "triangular") for d in ts]
    assert lens == sorted(lens)


@pytest.mark.parametrize("s", [3, 4, 5])
def test_hex_degeneracy_criterion(s):
    L, m = osel.hex_mask(s)
    assert osel.masked_null_space_dim(L, m, [(1, 0), (0, 1)]) == 5
    assert osel.masked_null_space_dim(L, m, [(1, 0), (0, 1), (-1, 1)]) == 4


def test_fx_masked_all_occupied_equals_grid_fx(orc):
    L = 5
    v, g, _ = synth.make_voltages(4, L, 1, 64, n_src=3)
    a = orc.fx(v[0].numpy(), g[0].numpy(), L)
    b, nd = orc.fx_masked(v[0].numpy(), g[0].numpy(), np.ones(L * L, np.uint8), L)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-12 * abs(a[L - 1, L - 1]))
    assert nd[L - 1, L - 1] == L * L and nd[0, 0] == 1


def test_fx_masked_pair_by_pair(orc):
    L, m = osel.hex_mask(2)
    v, g, _ = synth.make_voltages(5, L, 1, 32, n_src=2)
    v, g = v[0].numpy().astype(np.complex128), g[0].numpy().astype(np.complex128)
    got, nd = orc.fx_masked(v, g, m, L)
    w = v / g[None, :]
    occ = np.flatnonzero(m)
    for dy in range(-(L - 1), L):
        for dx in range(-(L - 1), L):
            acc, n = 0j, 0
            for i in occ:
                for j in occ:
                    if (i % L - j % L, i // L - j // L) == (dx, dy):
                        acc += np.mean(w[:, i] * np.conj(w[:, j]))
                        n += 1
            assert nd[dy + L - 1, dx + L - 1] == n
            assert abs(got[dy + L - 1, dx + L - 1] - (acc / n if n else 0)) < 1e-12


@pytest.mark.parametrize("solver", ["lincal", "omnical"])
def test_hex_noise_free_recovery(solver):
    L, m = osel.hex_mask(4)
    sel = osel.subset_layout(L, m, "triangular", 64)
    pi, pj, pos = osel.compact(sel, m)
    N = len(pos)
    rng = np.random.default_rng(3)
    g = (1 + 0.05 * rng.standard_normal(N)) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    V = rng.standard_normal(sel.n_ubl) + 1j * rng.standard_normal(sel.n_ubl)
    alpha = sel.pair_type()
    vobs = g[pi] * np.conj(g[pj]) * V[alpha]
    ge, Ve, it, ok = oc.calibrate(vobs, pi, pj, alpha, sel.types, pos, solver)
    assert ok
    gf = oc.fit_degeneracies(ge, g, pos)
    assert np.max(np.abs(gf - g) / np.abs(g)) < 1e-8
    assert oc.chi2(vobs, ge, Ve, pi, pj, alpha) < 1e-16 * np.sum(np.abs(vobs) ** 2)


def test_hex_subset_331():
    L, m = osel.hex_mask(11)
    sel = osel.subset_layout(L, m, "triangular", 1024)
    assert sel.extra["N"] == 331
    # whole groups, count closest to N log2 N among the prefixes
    ts, cnt = osel.layout_types(L, m, "triangular")
    cums = np.cumsum(cnt)
    k = int(np.argmin(np.abs(cums - 331 * np.log2(331)))) + 1
    assert sel.n_ubl == k and sel.P == cums[k - 1]
    assert sel.types == ts[:k]


def test_normal_matrices_equal_design_products():
    """Eq. logcal's normal matrices summed pair by pair equal A^T A, B^T B."""
    L = 6
    sel = osel.subset(L, 64)
    A, B = oc.logcal_matrices(L, sel.types, sel.pair_i, sel.pair_j, sel.pair_type())
    AtA, BtB = oc.logcal_normal_matrices(L * L, sel.types, sel.pair_i, sel.pair_j, sel.pair_type())
    assert np.array_equal(AtA, A.T @ A) and np.array_equal(BtB, B.T @ B)


def test_hex_gain_variance_prediction_is_finite_and_positive():
    L, m = osel.hex_mask(4)
    for sel in (osel.subset_layout(L, m, "triangular", 256), osel.lowcad_layout(L, m, "triangular", 256)):
        pi, pj, pos = osel.compact(sel, m)
        pa, pp = oc.gain_variance_prediction(None, sel.types, pi, pj, sel.pair_type(), N=len(pos))
        assert np.all(pa > 0) and np.all(pp > 0) and np.all(np.isfinite(pa + pp))
    # at equal visibility noise, more pairs per antenna (low-cadence: all of them) predict less variance
    sub = osel.subset_layout(L, m, "triangular", 256)
    low = osel.lowcad_layout(L, m, "triangular", 256)
    a = [oc.gain_variance_prediction(None, s.types, *osel.compact(s, m)[:2], s.pair_type(), N=int(m.sum()))
         for s in (sub, low)]
    assert np.mean(a[1][0] + a[1][1]) < np.mean(a[0][0] + a[0][1])
