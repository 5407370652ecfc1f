"""Pins of the FX / FFT-correlator oracle against what the paper and the
mathematics fix (Sec. 1 convolution theorem; Eq. modelvis)."""
import math

import numpy as np
import pytest


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("L,T", [(2, 3), (3, 5), (4, 4)])
def test_fx_equals_fft_correlator(orc, L, T):
    """Sec. 1: averaging redundant FX visibilities equals the FFT-correlator
    (convolution theorem).  Two independent oracle algorithms must agree."""
    rng = np.random.default_rng(L * 100 + T)
    v = _rand(rng, T, L * L)
    g = _rand(rng, L * L) + 3.0
    a = orc.fx(v, g, L)
    b = orc.dft(v, g, L)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("L", [2, 3])
def test_all_ones_closed_form(orc, L):
    """Unit voltages and gains: R(d) = T N_d, so V^unique(d) = 1 for all d."""
    T = 7
    v = np.ones((T, L * L), complex)
    for f in (orc.fx, orc.dft):
        out = f(v, None, L)
        assert np.allclose(out, 1.0, atol=1e-13)


def test_two_by_two_lag_sums(orc):
    """2x2 grid: N_0 = 4, N_(+-1,0) = N_(0,+-1) = 2, N_(+-1,+-1) = 1 -- the
    redundant counts of Eq. modelvis, read off a voltage pattern that makes
    each ordered pair's product distinct."""
    L, T = 2, 1
    # w = (a, b, c, e) at (0,0), (1,0), (0,1), (1,1)
    w = np.array([[1.0, 2.0, 3.0, 5.0]], complex)
    out = orc.fx(w, None, L)
    a, b, c, e = w[0]
    W = 3
    get = lambda dx, dy: out[dy + 1, dx + 1]
    assert get(0, 0) == pytest.approx((a * a + b * b + c * c + e * e) / 4)
    assert get(1, 0) == pytest.approx((b * a + e * c) / 2)          # r_i - r_j = (1, 0)
    assert get(-1, 0) == pytest.approx((a * b + c * e) / 2)
    assert get(0, 1) == pytest.approx((c * a + e * b) / 2)
    assert get(1, 1) == pytest.approx(e * a / 1)
    assert get(-1, 1) == pytest.approx(c * b / 1)


@pytest.mark.parametrize("L", [3, 4])
def test_point_source_closed_form(orc, L):
    """One noise-free point source, unit gains: V(d) = mean|a|^2 e^{2 pi i d.l}.
    Fixes the sign convention d = r_i - r_j and the conjugation."""
    rng = np.random.default_rng(5)
    T = 9
    l = np.array([0.13, -0.31])
    a = _rand(rng, T)
    pos = np.stack([np.arange(L * L) % L, np.arange(L * L) // L], 1)
    v = a[:, None] * np.exp(2j * np.pi * (pos @ l))[None, :]
    S = np.mean(np.abs(a) ** 2)
    for f in (orc.fx, orc.dft):
        out = f(v, None, L)
        for dy in range(-(L - 1), L):
            for dx in range(-(L - 1), L):
                exp = S * np.exp(2j * np.pi * (dx * l[0] + dy * l[1]))
                assert abs(out[dy + L - 1, dx + L - 1] - exp) < 1e-12


def test_gains_are_divided_out(orc):
    """Eq. modelvis divides V_ij by g_i g_j^*: voltages g_i s_i with gains g
    give the same V^unique as s with unit gains."""
    rng = np.random.default_rng(11)
    L, T = 3, 6
    s = _rand(rng, T, L * L)
    g = _rand(rng, L * L) + 2.0
    ref = orc.fx(s, None, L)
    got = orc.fx(s * g[None, :], g, L)
    assert np.max(np.abs(ref - got)) < 1e-12 * np.max(np.abs(ref))
    got2 = orc.dft(s * g[None, :], g, L)
    assert np.max(np.abs(ref - got2)) < 1e-12 * np.max(np.abs(ref))


def test_hermitian_and_zero_lag(orc):
    """V(-d) = conj V(d); V(0) = mean |w|^2 over antennas and time."""
    rng = np.random.default_rng(3)
    L, T = 4, 5
    v = _rand(rng, T, L * L)
    out = orc.fx(v, None, L)
    assert np.allclose(out[::-1, ::-1], np.conj(out), atol=1e-13)
    assert out[L - 1, L - 1] == pytest.approx(np.mean(np.abs(v) ** 2))


def test_power_spectrum_matches_library_fft(orc):
    """The oracle's direct DFT power P(k) equals |FFT2|^2 of the zero-padded
    grid from numpy's FFT (a library routine as an independent check)."""
    rng = np.random.default_rng(8)
    L, T, M = 3, 4, 8
    v = _rand(rng, T, L * L)
    _, pk = orc.dft(v, None, L, M, return_pk=True)
    grid = np.zeros((T, M, M), complex)
    grid[:, :L, :L] = v.reshape(T, L, L)         # [t, y, x]
    ref = np.sum(np.abs(np.fft.fft2(grid)) ** 2, axis=0)   # k_y major
    assert np.max(np.abs(pk - ref)) < 1e-10 * np.max(ref)


def test_lag_matches_fx(orc):
    rng = np.random.default_rng(4)
    L, T = 4, 3
    v = _rand(rng, T, L * L)
    g = _rand(rng, L * L) + 2.0
    full = orc.fx(v, g, L)
    for dx, dy in [(0, 0), (1, 0), (-3, 2), (2, -3), (3, 3)]:
        assert abs(orc.lag(v, g, L, dx, dy) - full[dy + L - 1, dx + L - 1]) < 1e-12


def test_fx_multi_matches_single(orc):
    rng = np.random.default_rng(9)
    C, L, T = 3, 3, 4
    v = _rand(rng, C, T, L * L)
    g = _rand(rng, C, L * L) + 2.0
    out, nt = orc.fx_multi(v, g, L)
    assert nt >= 1
    for c in range(C):
        assert np.allclose(out[c], orc.fx(v[c], g[c], L), atol=1e-13)


@pytest.mark.parametrize("L,T", [(3, 17), (8, 50), (11, 23)])
def test_fx_par_equals_fx(orc, L, T):
    """The threaded FX oracle (pair loop split over threads, antenna-major
    copy of the calibrated voltages) computes the same Eq. modelvis sums as
    the plain FX loop; a planted change in either would show here and in the
    pins above."""
    rng = np.random.default_rng(L * T)
    N = L * L
    v = rng.standard_normal((T, N)) + 1j * rng.standard_normal((T, N))
    g = (1 + 0.1 * rng.standard_normal(N)) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    ref = orc.fx(v, g, L)
    got, n = orc.fx_par(v, g, L)
    assert n >= 1
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
