"""Parity of the CUDA FFT-correlator (gc_correlate) with the FP64 oracle.

Tolerance (FP32 path): the FFT spreads its rounding error evenly over all
lags at the scale of the zero-lag power, so the bound is stated on the lag
sums R(d) = T N_d V(d) relative to R(0):
    max_d |V_gpu(d) - V_ref(d)| N_d / (N |V_ref(0)|) <= 1e-5.
"""
import numpy as np
import pytest
import torch

from paper_2005_03060_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def lag_err(got, ref, L):
    N = L * L
    r = np.arange(-(L - 1), L)
    nd = (L - np.abs(r))[:, None] * (L - np.abs(r))[None, :]
    return float(np.max(np.abs(got - ref) * nd) / (N * abs(ref[L - 1, L - 1])))


@pytest.fixture(scope="module")
def gc():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr.Context(0)


@pytest.mark.parametrize("L,C,T", [(1, 2, 5), (2, 1, 7), (3, 2, 37), (5, 1, 100), (8, 3, 64),
                                   (12, 2, 64), (16, 2, 130), (24, 1, 50), (31, 1, 33),
                                   (32, 2, 300), (40, 1, 20), (64, 1, 12)])
def test_correlate_c64(gc, orc, L, C, T):
    volt, gains, _ = synth.make_voltages(100 + L, L, C, T, n_src=20)
    out = gc.correlate(volt.cuda(), gains.cuda())
    gc.device_status()
    got = out.cpu().numpy()
    for c in range(C):
        ref = orc.fx(volt[c].numpy(), gains[c].numpy(), L)
        assert lag_err(got[c], ref, L) < TOL, (L, c)


def test_correlate_tiny_config(gc, orc):
    """8x8 grid, 32 channels, 256 samples, 20 sources, 16x16 FFT."""
    L, C, T = 8, 32, 256
    volt, gains, _ = synth.make_voltages(1, L, C, T, n_src=20)
    got = gc.correlate(volt.cuda(), gains.cuda()).cpu().numpy()
    gc.device_status()
    ref, _ = orc.fx_multi(volt.numpy(), gains.numpy(), L)
    errs = [lag_err(got[c], ref[c], L) for c in range(C)]
    assert max(errs) < TOL


def _quantised(volt):
    import oracle
    C, T, N = volt.shape
    out = np.zeros((C, T, N), np.uint8)
    for c in range(C):
        out[c], _ = oracle.quantize(volt[c].numpy())
    return out


@pytest.mark.parametrize("L,C,T", [(8, 2, 40), (16, 2, 66), (20, 1, 30), (32, 1, 48), (64, 1, 10)])
def test_correlate_i4c(gc, orc, L, C, T):
    volt, gains, _ = synth.make_voltages(200 + L, L, C, T, n_src=20)
    q = _quantised(volt)
    out = gc.correlate(torch.from_numpy(q).cuda(), gains.cuda())
    gc.device_status()
    got = out.cpu().numpy()
    for c in range(C):
        ref = orc.fx(orc.unpack_i4c(q[c]), gains[c].numpy(), L)
        assert lag_err(got[c], ref, L) < TOL, (L, c)


HALF_U = 2.0 ** -11   # unit roundoff of binary16


def _half(volt):
    """binary16 storage of complex64 voltages: float16 [C, T, N, 2] and the
    complex128 values it holds exactly."""
    h = torch.view_as_real(volt).to(torch.float16).contiguous()
    return h, torch.view_as_complex(h.to(torch.float64)).numpy()


@pytest.mark.parametrize("L,C,T", [(4, 1, 9), (8, 2, 40), (16, 1, 66), (30, 1, 20), (32, 2, 48),
                                   (61, 1, 7), (64, 1, 10)])
def test_correlate_c32h(gc, orc, L, C, T):
    """FP16-storage variant: FP32 arithmetic on binary16 voltages.  Against the
    oracle on the stored values: the FP32 bound.  Against FP64 on the
    unrounded voltages: component rounding |dv| <= u |v| moves every product
    w_i conj(w_j) by at most (2u + u^2)|w_i||w_j|, and by Cauchy-Schwarz the
    pairs of one lag sum to at most R(0), so the lag-sum error is <= 2u + u^2
    (u = 2^-11) plus the FP32 bound."""
    volt, gains, _ = synth.make_voltages(300 + L, L, C, T, n_src=20)
    h, held = _half(volt)
    got = gc.correlate(h.cuda(), gains.cuda()).cpu().numpy()
    gc.device_status()
    # complex32 tensors take the same path
    if hasattr(torch, "complex32"):
        got2 = gc.correlate(torch.view_as_complex(h.float()).to(torch.complex32).cuda(), gains.cuda())
        assert np.array_equal(got2.cpu().numpy(), got)
    for c in range(C):
        ref = orc.fx(held[c], gains[c].numpy(), L)
        assert lag_err(got[c], ref, L) < TOL, (L, c)
        ref64 = orc.fx(volt[c].numpy(), gains[c].numpy(), L)
        assert lag_err(got[c], ref64, L) < 2 * HALF_U + HALF_U ** 2 + TOL, (L, c)


@pytest.mark.parametrize("L,C,T", [(65, 1, 16), (80, 2, 8), (128, 1, 5)])
def test_correlate_i4c_m256(gc, orc, L, C, T):
    """Grids of 65..128 antennas a side (256 x 256 FFT): 4+4-bit voltages,
    plain staging (L = 65) and TMA staging (L = 80, 128)."""
    volt, gains, _ = synth.make_voltages(500 + L, L, C, T, n_src=20)
    q = _quantised(volt)
    out = gc.correlate(torch.from_numpy(q).cuda(), gains.cuda())
    gc.device_status()
    got = out.cpu().numpy()
    for c in range(C):
        ref = orc.fx(orc.unpack_i4c(q[c]), gains[c].numpy(), L)
        assert lag_err(got[c], ref, L) < TOL, (L, c)


def test_correlate_i4c_128_sampled(gc, orc):
    """128x128 grid over several time chunks (T = 1100); sampled lags against
    the oracle's one-lag definition."""
    L, C, T = 128, 2, 1100
    N = L * L
    volt, gains, _ = synth.make_voltages(9, L, C, T, n_src=50)
    qn = _quantised(volt)
    del volt
    out = gc.correlate(torch.from_numpy(qn).cuda(), gains.cuda())
    gc.device_status()
    got = out.cpu().numpy()
    rng = np.random.default_rng(1)
    for c in range(C):
        v = orc.unpack_i4c(qn[c])
        g = gains[c].numpy()
        r0 = orc.lag(v, g, L, 0, 0)
        lags = [(0, 0), (1, 0), (0, 1), (-127, 127), (127, 0), (0, -127)] + \
            [tuple(rng.integers(-(L - 1), L, 2)) for _ in range(14)]
        for dx, dy in lags:
            ref = orc.lag(v, g, L, int(dx), int(dy))
            nd = (L - abs(dx)) * (L - abs(dy))
            e = abs(got[c, dy + L - 1, dx + L - 1] - ref) * nd / (N * abs(r0))
            assert e < TOL, (c, dx, dy, e)


def test_correlate_misaligned_plain_path(gc, orc):
    """A voltage buffer that is 8- but not 16-byte aligned takes the plain
    staging path and gives the same answer."""
    L, C, T = 8, 1, 30
    volt, gains, _ = synth.make_voltages(5, L, C, T, n_src=5)
    big = torch.zeros(C * T * L * L + 1, dtype=torch.complex64, device="cuda")
    big[1:] = volt.reshape(-1).cuda()
    v = big[1:].view(C, T, L * L)
    assert v.data_ptr() % 16 == 8
    got = gc.correlate(v, gains.cuda()).cpu().numpy()
    ref = orc.fx(volt[0].numpy(), gains[0].numpy(), L)
    assert lag_err(got[0], ref, L) < TOL


def test_correlate_rejects_bad_arguments(gc):
    from paper_2005_03060_gb300 import gridcorr
    for L, dtype, status in [(65, torch.complex64, gridcorr.GC_EUNSUPPORTED),
                             (129, torch.uint8, gridcorr.GC_EINVAL)]:
        v = torch.zeros(1, 4, L * L, dtype=dtype, device="cuda")
        g = torch.ones(1, L * L, dtype=torch.complex64, device="cuda")
        with pytest.raises(gridcorr.GridcorrError) as e:
            gc.correlate(v, g)
        assert e.value.status == status


def test_correlate_paper_scale_sampled(gc, orc):
    """32x32 grid, 256 channels, 4096 samples, 200 sources, 64x64 FFT, in the
    launch configuration the benchmark times; sampled lags of two channels
    against the oracle's one-lag definition."""
    L, C, T = 32, 256, 4096
    N = L * L
    volt = torch.empty(C, T, N, dtype=torch.complex64, device="cuda")
    volt, gains, _ = synth.make_voltages(2, L, C, T, n_src=200, device="cuda", out=volt)
    out = gc.correlate(volt, gains)
    gc.device_status()
    got = out.cpu().numpy()
    rng = np.random.default_rng(0)
    for c in (0, 137):
        v = volt[c].cpu().numpy()
        g = gains[c].cpu().numpy()
        r0 = orc.lag(v, g, L, 0, 0)
        lags = [(0, 0), (1, 0), (0, 1), (-31, 31), (31, 0)] + \
            [tuple(rng.integers(-(L - 1), L, 2)) for _ in range(15)]
        for dx, dy in lags:
            ref = orc.lag(v, g, L, int(dx), int(dy))
            nd = (L - abs(dx)) * (L - abs(dy))
            e = abs(got[c, dy + L - 1, dx + L - 1] - ref) * nd / (N * abs(r0))
            assert e < TOL, (c, dx, dy, e)
    del volt
    torch.cuda.empty_cache()



@pytest.mark.parametrize("L,C,T", [(64, 2, 300), (33, 3, 77), (48, 1, 1031), (64, 5, 4)])
def test_correlate_i4c_m128_ragged(gc, orc, L, C, T):
    """M = 128 (L = 33..64) with 4+4-bit voltages over ragged sample counts
    (odd T, T below one stage copy) and rows L < 64 that stay zero."""
    volt, gains, _ = synth.make_voltages(700 + L + T, L, C, T, n_src=20)
    q = _quantised(volt)
    out = gc.correlate(torch.from_numpy(q).cuda(), gains.cuda())
    gc.device_status()
    got = out.cpu().numpy()
    for c in range(C):
        ref = orc.fx(orc.unpack_i4c(q[c]), gains[c].numpy(), L)
        assert lag_err(got[c], ref, L) < TOL, (L, c)


def test_correlate_i4c_m128_chunk_sizes_agree(gc):
    """Work items of 2..512 samples (the "fft.chunk_len" knob) over many
    channels give the same V^unique to FP32 rounding on the 64x64 grid."""
    L, C, T = 64, 12, 2048
    g = torch.Generator(device="cuda").manual_seed(3)
    q = torch.randint(0, 256, (C, T, L * L), dtype=torch.uint8, device="cuda", generator=g)
    _, gains, _ = synth.make_voltages(5, L, C, 1, n_src=1)
    gains = gains.cuda()
    outs = {}
    try:
        for chunk in (0, 2, 130, 512):
            gc.set_tuning("fft.chunk_len", chunk)
            outs[chunk] = gc.correlate(q, gains).cpu().numpy()
            gc.device_status()
    finally:
        gc.set_tuning("fft.chunk_len", 0)
    ref = outs[0]
    for key, got in outs.items():
        for c in range(C):
            assert lag_err(got[c], ref[c], L) < TOL, key
