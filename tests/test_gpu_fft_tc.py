"""The FFT-correlator with its row stage on the tensor cores (4+4-bit
voltages, L = 40..64 in steps of 8, M = 128; gc_fftcorr_tc.cu) against the
FP64 oracle (Eq. modelvis by the FX definition) and against the CUDA-core
kernel ("fft.path" = 1), at the lag-sum bound of the FP32 path:
    max_d |V_gpu(d) - V_ref(d)| N_d / (N |V_ref(0)|) <= 1e-5.
Ragged sample counts (one sample, an odd count that leaves half a raw stage,
chunks of two samples), grids smaller than the 64 x 64 operand (zero rows and
inputs), the extreme codes, and a zero gain."""
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
def gcm():
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


@pytest.fixture(scope="module")
def gc(gcm):
    return gcm.Context(0)


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _tc_ran(gc, fn):
    gc.profile(True)
    gc.profile_read()
    out = fn()
    rec = gc.profile_read()
    gc.profile(False)
    return out, rec


def _quantised(gc, volt):
    q, _ = gc.quantize(volt.cuda())
    return q


@pytest.mark.parametrize("L,C,T", [(64, 2, 257), (56, 2, 64), (48, 3, 1), (40, 2, 3)])
def test_tc_path_matches_oracle(gc, orc, L, C, T):
    volt, gains, _ = synth.make_voltages(900 + L + T, L, C, T, n_src=20)
    q = _quantised(gc, volt)
    out, rec = _tc_ran(gc, lambda: gc.correlate(q, gains.cuda()))
    gc.device_status()
    assert "fftcorr_tc_accumulate" in rec and "fftcorr_accumulate" not in rec
    got = out.cpu().numpy()
    qh = q.cpu().numpy()
    for c in range(C):
        ref = orc.fx(orc.unpack_i4c(qh[c]), gains[c].numpy(), L)
        assert lag_err(got[c], ref, L) < TOL, (L, T, c)


def test_tc_path_equals_cuda_core_path(gc):
    L, C, T = 64, 6, 1000
    g = torch.Generator(device="cuda").manual_seed(11)
    q = torch.randint(0, 256, (C, T, L * L), dtype=torch.uint8, device="cuda", generator=g)
    _, gains, _ = synth.make_voltages(12, L, C, 1, n_src=1)
    gains = gains.cuda()
    tc = gc.correlate(q, gains).cpu().numpy()
    try:
        gc.set_tuning("fft.path", 1)
        out, rec = _tc_ran(gc, lambda: gc.correlate(q, gains))
        assert "fftcorr_accumulate" in rec and "fftcorr_tc_accumulate" not in rec
        cc = out.cpu().numpy()
    finally:
        gc.set_tuning("fft.path", 0)
    gc.device_status()
    for c in range(C):
        assert lag_err(tc[c], cc[c], L) < TOL, c


@pytest.mark.parametrize("code", [0x88, 0x77, 0x87])
def test_tc_path_extreme_codes(gc, orc, code):
    """Every voltage at a corner of the 4+4-bit range (-8-8i, 7+7i, -8+7i):
    the largest B operands of the split."""
    L, C, T = 64, 1, 9
    q = torch.full((C, T, L * L), code, dtype=torch.uint8, device="cuda")
    _, gains, _ = synth.make_voltages(13, L, C, 1, n_src=1)
    got = gc.correlate(q, gains.cuda()).cpu().numpy()
    gc.device_status()
    ref = orc.fx(orc.unpack_i4c(q[0].cpu().numpy()), gains[0].numpy(), L)
    assert lag_err(got[0], ref, L) < TOL


def test_tc_path_zero_gain_is_reported(gcm, gc):
    L, C, T = 64, 2, 16
    volt, gains, _ = synth.make_voltages(14, L, C, T, n_src=5)
    q = _quantised(gc, volt)
    bad = gains.clone()
    bad[1, 100] = 0.0
    gc.correlate(q, bad.cuda())
    with pytest.raises(gcm.GridcorrError) as ei:
        gc.device_status()
    assert ei.value.status == gcm.GC_EINVAL
    out = gc.correlate(q, gains.cuda())
    gc.device_status()
    assert torch.isfinite(torch.view_as_real(out)).all()


def test_tc_path_chunk_sizes_agree(gc):
    """Work items of 2 .. 2048 samples (the "fft.chunk_len" knob)."""
    L, C, T = 64, 5, 2050
    g = torch.Generator(device="cuda").manual_seed(15)
    q = torch.randint(0, 256, (C, T, L * L), dtype=torch.uint8, device="cuda", generator=g)
    _, gains, _ = synth.make_voltages(16, L, C, 1, n_src=1)
    gains = gains.cuda()
    outs = {}
    try:
        for chunk in (0, 2, 333, 2048):
            gc.set_tuning("fft.chunk_len", chunk)
            outs[chunk] = gc.correlate(q, gains).cpu().numpy()
            gc.device_status()
    finally:
        gc.set_tuning("fft.chunk_len", 0)
    for key, got in outs.items():
        for c in range(C):
            assert lag_err(got[c], outs[0][c], L) < TOL, (key, c)
