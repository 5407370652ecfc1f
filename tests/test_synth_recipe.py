"""The seeded input generator follows the recipe it states (the sky, gains
and noise of the paper-style workloads), on the CPU."""
import math

import numpy as np
import pytest
import torch

from paper_2005_03060_gb300 import synth


def test_sky_fluxes_follow_s_minus_two():
    """dN/dS ~ S^-2 on [0.1, 10]: CDF F(S) = (10 - 1/S) / 9.9; directions
    uniform in [-0.5, 0.5)^2.  Kolmogorov-Smirnov bounds on 20 000 draws."""
    from scipy.stats import kstest
    sky = synth.make_sky(7, 20000)
    s = sky.flux.numpy()
    assert s.min() >= 0.1 and s.max() <= 10.0
    assert kstest(s, lambda x: (10.0 - 1.0 / np.asarray(x)) / 9.9).pvalue > 1e-4
    l = sky.l.numpy()
    assert l.min() >= -0.5 and l.max() < 0.5
    assert kstest(l[:, 0] + 0.5, "uniform").pvalue > 1e-4
    assert kstest(l[:, 1] + 0.5, "uniform").pvalue > 1e-4


def test_gains_mean_one_scatter_and_uniform_phase():
    g = synth.make_gains(3, 8, 4096).numpy().astype(np.complex128)
    a = np.abs(g)
    assert a.mean() == pytest.approx(1.0, abs=0.002)
    assert a.std() == pytest.approx(0.05, rel=0.03)
    ph = np.angle(g).ravel()
    assert abs(np.mean(np.exp(1j * ph))) < 0.02          # uniform phases


def test_voltage_power_and_snr():
    """E|v_i|^2 = |g_i|^2 (sum_k S_k) (1 + 1/snr): sky power plus noise at the
    stated power ratio; without noise the ratio term drops out."""
    L, C, T, K, snr = 6, 2, 4096, 20, 10.0
    v, g, sky = synth.make_voltages(11, L, C, T, n_src=K, snr=snr)
    v0, _, _ = synth.make_voltages(11, L, C, T, n_src=K, snr=snr, noise=False)
    S = float(sky.flux.sum())
    p = (v.abs() ** 2).mean(dim=1) / (g.abs() ** 2)      # [C, N]
    p0 = (v0.abs() ** 2).mean(dim=1) / (g.abs() ** 2)
    # K sources with independent amplitudes: the per-antenna sky power is S on average
    assert float(p0.mean()) == pytest.approx(S, rel=0.03)
    assert float((p - p0).mean()) == pytest.approx(S / snr, rel=0.05)


def test_channels_do_not_depend_on_chunking():
    """A channel's draws depend on its index, not on how many channels are
    generated together: the 64x64 workload is drawn in chunks."""
    L, T, K = 5, 64, 8
    g = synth.make_gains(5, 6, L * L)
    full, _, _ = synth.make_voltages(5, L, 6, T, n_src=K, gains=g)
    part, _, _ = synth.make_voltages(5, L, 2, T, n_src=K, gains=g[3:5], channel0=3)
    assert torch.equal(full[3:5], part)


def test_triangular_lattice_geometry():
    """Point i = y L + x of the triangular lattice sits at x (1, 0) +
    y (1/2, sqrt3/2): all six neighbours of an inner point at unit distance."""
    L = 5
    p = synth.lattice_positions(L, "triangular").numpy()
    c = 2 * L + 2
    for dx, dy in ((1, 0), (0, 1), (-1, 1), (-1, 0), (0, -1), (1, -1)):
        j = (2 + dy) * L + (2 + dx)
        assert np.linalg.norm(p[j] - p[c]) == pytest.approx(1.0, abs=1e-12)
    assert np.linalg.norm(p[(2 + 1) * L + 3] - p[c]) == pytest.approx(math.sqrt(3.0), abs=1e-12)
