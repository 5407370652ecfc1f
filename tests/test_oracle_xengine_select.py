"""Pins of the X-engine, quantiser and selection oracles."""
import json
import math
import os

import numpy as np
import pytest

from oracle import select as osel

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pack(re, im):
    return ((np.asarray(re) & 15) << 4 | (np.asarray(im) & 15)).astype(np.uint8)


def test_i4c_hand_example(orc):
    d = json.load(open(os.path.join(GOLD, "xengine_i4c_hand.json")))
    v = np.array(d["voltages_re_im"])             # [T, N, 2]
    b = _pack(v[..., 0], v[..., 1])
    pr = np.array(d["pairs"])
    T = v.shape[0]
    out = orc.xengine_i4c(b, pr[:, 0], pr[:, 1], [0] * len(pr), [T] * len(pr))
    assert out.tolist() == d["expected_sums_re_im"]


def test_i4c_equals_c64_on_integers(orc):
    """The exact int64 path and the FP64 path agree on integer voltages."""
    rng = np.random.default_rng(2)
    T, N, P = 50, 20, 40
    re = rng.integers(-7, 8, (T, N))
    im = rng.integers(-7, 8, (T, N))
    b = _pack(re, im)
    pi = rng.integers(0, N, P)
    pj = rng.integers(0, N, P)
    t0 = rng.integers(0, T // 2, P)
    t1 = t0 + rng.integers(0, T // 2, P)
    a = orc.xengine_i4c(b, pi, pj, t0, t1)
    c = orc.xengine_c64(re + 1j * im, pi, pj, t0, t1)
    assert np.array_equal(a[:, 0], c.real.astype(np.int64))
    assert np.array_equal(a[:, 1], c.imag.astype(np.int64))
    assert np.array_equal(orc.unpack_i4c(b), re + 1j * im)


def test_xengine_matches_fx_full_matrix(orc):
    """Full-window pair sums equal T * V^full_ij of the FX oracle."""
    rng = np.random.default_rng(3)
    L, T = 3, 6
    v = rng.standard_normal((T, L * L)) + 1j * rng.standard_normal((T, L * L))
    _, vf = orc.fx(v, None, L, full=True)
    pi = np.arange(L * L).repeat(L * L)
    pj = np.tile(np.arange(L * L), L * L)
    s = orc.xengine_c64(v, pi, pj, [0] * len(pi), [T] * len(pi))
    assert np.allclose(s, T * vf[pi, pj], atol=1e-12)


def test_subset_tie_goes_to_the_shorter_prefix():
    """Sec. 6.1 takes the whole number of groups closest to p N log N and
    leaves ties open; the reading here is the shorter prefix.  On a 4 x 4
    grid the prefixes hold 12, 24, 33, 42 pairs; p = 0.5859375 puts the
    budget at 37.5, exactly between 33 and 42."""
    sel = osel.subset(4, 64, p=0.5859375)
    assert sel.extra["target"] == 37.5
    assert sel.P == 33 and sel.types == [(1, 0), (0, 1), (1, 1)]
    assert osel.subset(4, 64, p=0.5859375 + 1e-6).P == 42


def test_autos_are_windowed_self_pairs(orc):
    """A_i over [t0, t1) equals the X-engine's sum of the pair (i, i) over the
    same window (real, |v_i|^2 summed) and T V^full_ii of the FX oracle for
    the full window; a window that starts late drops the early samples."""
    rng = np.random.default_rng(5)
    L, T = 3, 10
    N = L * L
    v = rng.standard_normal((T, N)) + 1j * rng.standard_normal((T, N))
    ii = np.arange(N)
    for t0, t1 in ((0, T), (3, 8), (4, 4)):
        a = orc.autos(v, t0, t1)
        s = orc.xengine_c64(v, ii, ii, [t0] * N, [t1] * N)
        assert np.allclose(a, s.real, atol=1e-12) and np.all(s.imag == 0)
    _, vf = orc.fx(v, None, L, full=True)
    assert np.allclose(orc.autos(v), T * np.diag(vf).real, atol=1e-12)
    assert np.allclose(orc.autos(v, 3, 8), np.sum(np.abs(v[3:8]) ** 2, axis=0), atol=1e-12)


def _round_half_away32(x):
    a = np.abs(x).astype(np.float32)
    f = np.floor(a)
    f = f + (a - f >= np.float32(0.5))
    return np.sign(x) * f


def test_quantiser_rules(orc):
    """Round half away from zero, clip to +-7, high nibble = Re, one scale per
    channel giving a per-component RMS of 3 levels."""
    rng = np.random.default_rng(1)
    T, N = 64, 16
    v = (rng.standard_normal((T, N)) + 1j * rng.standard_normal((T, N))).astype(np.complex64)
    v[0, :4] = np.complex64(40 + 40j)              # far beyond 7 levels: must clip
    v[1, :4] = np.complex64(-40 - 40j)
    b, s = orc.quantize(v)
    q = orc.unpack_i4c(b)
    assert np.all(np.abs(q.real) <= 7) and np.all(np.abs(q.imag) <= 7)
    assert np.all(q[0, :4] == 7 + 7j) and np.all(q[1, :4] == -7 - 7j)
    # expected codes written out with float32 products and the exact rule
    xr = v.real.astype(np.float32) * np.float32(s)
    xi = v.imag.astype(np.float32) * np.float32(s)
    assert np.array_equal(q.real, np.clip(_round_half_away32(xr), -7, 7))
    assert np.array_equal(q.imag, np.clip(_round_half_away32(xi), -7, 7))
    rms = math.sqrt(np.mean(np.abs(v.astype(complex)) ** 2) / 2)
    assert s == pytest.approx(3.0 / rms, rel=1e-6)
    # halves: +-2.5 levels round to +-3, +-0.5 to +-1
    h = np.array([2.5, -2.5, 0.5, -0.5], np.float32)
    assert _round_half_away32(h).tolist() == [3.0, -3.0, 1.0, -1.0]


def test_quantiser_code_distribution_closed_form(orc):
    """For Gaussian voltages the codes follow a closed form that the quantiser's
    stated rule fixes (RMS of 3 levels per component, round to nearest, clip to
    +-7): with x ~ N(0, 3^2), P(q = k) = Phi((k + 1/2)/3) - Phi((k - 1/2)/3) for
    |k| <= 6 and P(q = +-7) = 1 - Phi(6.5/3).  A wrong scale (per complex value
    instead of per component: a factor sqrt 2), truncation instead of rounding,
    a clip at 8 or swapped nibbles fail the chi-square bound."""
    from scipy.stats import norm, chi2
    rng = np.random.default_rng(20050306)
    T, N = 4096, 64
    # Re and Im with different spreads: the scale comes from their pooled RMS
    sr, si = 1.25, 0.65
    v = (sr * rng.standard_normal((T, N)) + 1j * si * rng.standard_normal((T, N))).astype(np.complex64)
    b, s = orc.quantize(v)
    q = orc.unpack_i4c(b)
    pooled = math.sqrt((sr * sr + si * si) / 2.0)
    for comp, sig in ((q.real, 3.0 * sr / pooled), (q.imag, 3.0 * si / pooled)):
        k = np.arange(-7, 8)
        p = norm.cdf((k + 0.5) / sig) - norm.cdf((k - 0.5) / sig)
        p[0] = norm.cdf(-6.5 / sig)
        p[-1] = 1.0 - norm.cdf(6.5 / sig)
        assert abs(p.sum() - 1.0) < 1e-12
        counts = np.array([(comp == kk).sum() for kk in k], dtype=np.float64)
        assert counts.sum() == comp.size            # nothing outside [-7, 7]
        e = p * comp.size
        keep = e > 5.0
        stat = float((((counts - e) ** 2) / e)[keep].sum())
        assert stat < chi2.ppf(1.0 - 1e-6, int(keep.sum()) - 1), (sig, stat)
        # second moment of the clipped, rounded Gaussian
        assert np.mean(comp ** 2) == pytest.approx(float((p * k * k).sum()), rel=0.01)
    # byte layout: two's-complement Re in the high nibble, Im in the low
    w = np.ones((1000, 4), np.complex64)           # unit rows keep the scale near 3
    w[0] = [40 - 40j, -40 + 40j, 0, 1e-3 - 1e-3j]  # clipped, clipped, zero, rounds to zero
    bb, _ = orc.quantize(w)
    assert bb[0].tolist() == [0x79, 0x97, 0x00, 0x00]


def test_canonical_types_cover_all_pairs():
    for L in (2, 3, 5):
        N = L * L
        ts = osel.canonical_types(L)
        assert len(ts) == ((2 * L - 1) ** 2 - 1) // 2
        assert sum(osel.n_pairs(L, d) for d in ts) == N * (N - 1) // 2
        seen = set()
        for d in ts:
            for i, j in osel.type_pairs(L, d):
                key = (min(i, j), max(i, j))
                assert key not in seen
                seen.add(key)
        assert len(seen) == N * (N - 1) // 2


def test_subset_golden_L8():
    d = json.load(open(os.path.join(GOLD, "subset_L8.json")))
    sel = osel.subset(8, 256)
    assert [list(t) for t in sel.types] == d["types"]
    assert sel.P == d["P"]
    assert sel.extra["target"] == pytest.approx(d["target_pairs"])


@pytest.mark.parametrize("L", [3, 4, 6])
def test_degeneracy_criterion(L):
    """Sec. 5.2: null space = 4 (amplitude, phase, two slopes).  On a square
    grid the two axis types alone leave a fifth (checkerboard amplitude)
    mode; adding the (1,1) diagonal removes it."""
    assert osel.null_space_dim(L, [(1, 0), (0, 1)]) == 5
    assert osel.null_space_dim(L, [(1, 0), (0, 1), (1, 1)]) == 4
    assert osel.null_space_dim(L, osel.canonical_types(L)) == 4


def test_two_by_two_is_underdetermined():
    """A 2x2 array has 6 visibilities for 8 complex unknowns: no selection
    reaches the four-degeneracy criterion, so L >= 3 is required."""
    assert osel.null_space_dim(2, osel.canonical_types(2)) > 4
    with pytest.raises(ValueError):
        osel.subset(2, 10)


def test_subset_small_budget_gets_criterion():
    # L = 3: target 9 log2 9 = 28.53; cumulative 6, 12, 16, 20, 23, 26, 28, 30 (k = 7 is closest)
    sel = osel.subset(3, 10)
    assert sel.P == 28 and len(sel.types) == 7
    assert osel.null_space_dim(3, sel.types) == 4
    # a tiny budget still takes the three-type minimum
    sel = osel.subset(6, 10, p=0.05)
    assert sel.types[:3] == [(1, 0), (0, 1), (1, 1)]
    assert osel.null_space_dim(6, sel.types) == 4


@pytest.mark.parametrize("L,T", [(4, 100), (8, 256)])
def test_lowcad_schedule(L, T):
    sel = osel.lowcad(L, T)
    N = L * L
    assert sel.P == N * (N - 1) // 2
    cap = sel.extra["cap"]
    load = np.zeros(sel.n_cycle, int)
    for k, c in enumerate(sel.extra["cycle_of"]):
        load[c] += osel.n_pairs(L, sel.types[k])
    assert np.all(load <= cap)
    assert sel.n_cycle >= math.ceil(sel.P / cap)
    assert sel.t_int == T // sel.n_cycle
    assert np.all(sel.win_t1 - sel.win_t0 == sel.t_int)
    assert np.all(sel.win_t1 <= T)
