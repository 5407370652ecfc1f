"""Seeded synthetic antenna voltages for a regular-grid redundant array.

This module only *draws inputs*; it holds none of the correlator or
calibration arithmetic, and both the CUDA path and the FP64 oracle consume
what it returns.  The sky model follows the voltage-level recipe used for
every workload of this library:

    v_i(t) = g_i * ( sum_k a_k(t) * exp(2*pi*i * r_i . l_k) + n_i(t) )

* antenna i sits at r_i = (x, y) on an L x L unit-spaced grid, i = y*L + x;
* source directions l_k ~ U(-0.5, 0.5)^2 (direction cosines);
* source fluxes S_k follow dN/dS ~ S^-2 on [0.1, 10] (inverse-CDF draw);
* a_k(t) ~ CN(0, S_k), independent per time sample;
* n_i(t) ~ CN(0, sigma_n^2) with sigma_n^2 = sum_k S_k / snr (power ratio);
* g_i = (1 + N(0, 0.05)) * exp(i U(-pi, pi)), independent per channel.

The paper's own simulations (Sec. 3) used gains of mean amplitude 1 with a
scatter at the ~10 % level and an SNR of 10; the defaults here keep the mean
and the SNR and draw the amplitude scatter with a standard deviation of 0.05,
the figure the benchmark workloads are specified with.

Every draw comes from a torch.Generator seeded from (seed, channel, stream),
so a channel's data does not depend on how many channels are generated or in
which chunks.  CPU and CUDA generators produce different streams; a test
feeds the *same* tensor to both the GPU path and the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

_TWO_PI = 2.0 * math.pi


def _gen(device, seed: int, channel: int, stream: int) -> torch.Generator:
    g = torch.Generator(device=device)
    # distinct, reproducible 63-bit seeds per (seed, channel, stream)
    g.manual_seed((seed * 1_000_003 + channel * 7919 + stream * 104_729) & 0x7FFF_FFFF_FFFF_FFFF)
    return g


@dataclass
class Sky:
    l: torch.Tensor      # [K, 2] float64 direction cosines
    flux: torch.Tensor   # [K] float64


def make_sky(seed: int, n_src: int, device="cpu") -> Sky:
    """Point-source sky shared by all channels of one draw."""
    g = _gen("cpu", seed, 0, 1)
    l = torch.rand(n_src, 2, generator=g, dtype=torch.float64) - 0.5
    u = torch.rand(n_src, generator=g, dtype=torch.float64)
    # inverse CDF of p(S) ~ S^-2 on [0.1, 10]:  1/S = 1/0.1 - u (1/0.1 - 1/10)
    flux = 1.0 / (10.0 - u * (10.0 - 0.1))
    return Sky(l.to(device), flux.to(device))


def make_gains(seed: int, C: int, N: int, device="cpu", amp_sigma: float = 0.05) -> torch.Tensor:
    """Per-channel complex gains [C, N] complex64."""
    out = torch.empty(C, N, dtype=torch.complex64, device=device)
    for c in range(C):
        g = _gen(device, seed, c, 2)
        amp = 1.0 + amp_sigma * torch.randn(N, generator=g, device=device, dtype=torch.float64)
        ph = (torch.rand(N, generator=g, device=device, dtype=torch.float64) * 2.0 - 1.0) * math.pi
        out[c] = torch.polar(amp, ph).to(torch.complex64)
    return out


def grid_positions(L: int, device="cpu") -> torch.Tensor:
    """[N, 2] float64 positions (x, y) with antenna index i = y*L + x."""
    y, x = torch.meshgrid(torch.arange(L, device=device), torch.arange(L, device=device), indexing="ij")
    return torch.stack([x.reshape(-1), y.reshape(-1)], dim=1).to(torch.float64)


def lattice_positions(L: int, lattice: str = "square", device="cpu") -> torch.Tensor:
    """[N, 2] float64 physical positions of the L x L lattice points
    (i = y*L + x): the grid itself for "square", x (1, 0) + y (1/2, sqrt3/2)
    for "triangular" (the lattice of hexagonal arrays)."""
    p = grid_positions(L, device)
    if lattice == "triangular":
        p = torch.stack([p[:, 0] + 0.5 * p[:, 1], p[:, 1] * (math.sqrt(3.0) / 2.0)], dim=1)
    elif lattice != "square":
        raise ValueError(lattice)
    return p


def hex_mask(s: int):
    """Layout of a hexagonal array of side s (3 s (s - 1) + 1 antennas) on
    the triangular lattice: axial coordinates (a, b) with |a|, |b|, |a + b|
    <= s - 1 at grid point x = a + s - 1, y = b + s - 1 of the (2 s - 1)^2
    bounding grid.  Returns (L, mask) with mask a uint8 numpy array [L * L]."""
    import numpy as np
    L = 2 * s - 1
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    m = ((x + y >= s - 1) & (x + y <= 3 * s - 3)).astype(np.uint8)
    return L, m.reshape(-1)


def _cnormal(n_shape, var, g, device):
    """Complex normal with E|z|^2 = var (var broadcastable)."""
    re = torch.randn(*n_shape, generator=g, device=device, dtype=torch.float32)
    im = torch.randn(*n_shape, generator=g, device=device, dtype=torch.float32)
    s = torch.sqrt(torch.as_tensor(var, device=device, dtype=torch.float32) * 0.5)
    return torch.complex(re * s, im * s)


def make_voltages(seed: int, L: int, C: int, T: int, n_src: int, snr: float = 10.0,
                  device="cpu", gains: torch.Tensor | None = None, noise: bool = True,
                  out: torch.Tensor | None = None, channel0: int = 0, lattice: str = "square"):
    """Voltages [C, T, N] complex64 (row-major grid index), and the true gains.

    Returns (volt, gains, sky).  `out` may be a preallocated [C, T, N]
    complex64 tensor.  `channel0` offsets the channel index of the draws, so
    that channels c0..c0+C-1 of a large workload can be generated chunk by
    chunk (same sky for every chunk; pass that chunk's gains).
    lattice: "triangular" places point i = y*L + x at x (1, 0) + y (1/2,
    sqrt3/2) (hexagonal arrays); the voltages keep the grid layout.
    """
    N = L * L
    sky = make_sky(seed, n_src, device)
    if gains is None:
        gains = make_gains(seed, channel0 + C, N, device)[channel0:]
    pos = lattice_positions(L, lattice, device)
    # steering phases e^{2 pi i r_i . l_k}: [K, N] complex64 (draw-time geometry)
    steer = torch.polar(torch.ones((), dtype=torch.float64, device=device),
                        _TWO_PI * (sky.l @ pos.T)).to(torch.complex64)
    sigma_n2 = float(sky.flux.sum()) / snr
    volt = out if out is not None else torch.empty(C, T, N, dtype=torch.complex64, device=device)
    flux32 = sky.flux.to(torch.float32)
    for c in range(C):
        g = _gen(device, seed, channel0 + c, 3)
        a = _cnormal((T, n_src), flux32, g, device)             # [T, K]
        sig = a @ steer                                         # [T, N]
        if noise:
            sig = sig + _cnormal((T, N), sigma_n2, g, device)
        volt[c] = sig * gains[c].unsqueeze(0)
    return volt, gains, sky


def complex_to_interleaved(z: torch.Tensor) -> torch.Tensor:
    """complex64 [...] -> float32 [..., 2] view (re, im) without copying."""
    return torch.view_as_real(z)


def make_visibilities(seed: int, L: int, C: int, pair_i, pair_j, pair_type, n_ubl: int, t_pair,
                      snr: float = 10.0, amp_sigma: float = 0.05, device="cpu", unit_amp: bool = False,
                      shared_truth: bool = False):
    """Visibility-level draw in the manner of the paper's own simulations
    (Sec. 3): true visibilities of random amplitude, uncorrelated between
    baseline-types and constant in time; gains with ~5 % amplitude scatter and
    random phases; complex Gaussian noise at the given per-visibility SNR,
    reduced by sqrt(t_p) for a pair integrated over t_p samples.

    Returns (sums [C, P] complex64 = t_p * V_p, gains [C, N], vtrue [C, n_ubl])
    so that the sums stand where the X-engine output would.  unit_amp: every
    baseline-type has |V| = 1 (the same SNR for all types, the setting of the
    paper's gain-variance curves); otherwise |V| ~ U(0.5, 1.5).
    shared_truth: every channel has channel 0's gains and visibilities and
    only the noise differs (the repeated-simulation setting of the paper's
    bias study, Sec. 6.3).
    """
    N = L * L
    pi = torch.as_tensor(pair_i, dtype=torch.long, device=device)
    pj = torch.as_tensor(pair_j, dtype=torch.long, device=device)
    pt = torch.as_tensor(pair_type, dtype=torch.long, device=device)
    tp = torch.as_tensor(t_pair, dtype=torch.float64, device=device)
    P = pi.numel()
    gains = make_gains(seed, C, N, device, amp_sigma)
    if shared_truth:
        gains = gains[:1].expand(C, N).contiguous()
    out = torch.empty(C, P, dtype=torch.complex64, device=device)
    vt = torch.empty(C, n_ubl, dtype=torch.complex64, device=device)
    for c in range(C):
        g = _gen(device, seed, 0 if shared_truth else c, 4)
        amp = 0.5 + torch.rand(n_ubl, generator=g, device=device, dtype=torch.float64)
        if unit_amp:
            amp = torch.ones_like(amp)
        ph = (torch.rand(n_ubl, generator=g, device=device, dtype=torch.float64) * 2 - 1) * math.pi
        V = torch.polar(amp, ph)
        gc = gains[c].to(torch.complex128)
        m = gc[pi] * gc[pj].conj() * V[pt]
        sig = amp[pt] / snr / torch.sqrt(tp)
        if shared_truth:
            g = _gen(device, seed, c, 5)
        nre = torch.randn(P, generator=g, device=device, dtype=torch.float64)
        nim = torch.randn(P, generator=g, device=device, dtype=torch.float64)
        noise = torch.complex(nre, nim) * (sig / math.sqrt(2.0))
        out[c] = ((m + noise) * tp).to(torch.complex64)
        vt[c] = V.to(torch.complex64)
    return out, gains, vt
