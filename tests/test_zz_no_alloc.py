"""gc_correlate_noalloc: the FFT-correlator for callers that cannot call
cudaMalloc (e.g. a real-time pipeline whose device memory is fixed at start
of observation, or a host framework that owns every device allocation).

The entry point keeps its scratch in a fixed array inside the library, so
the test only allocates the inputs and outputs a caller would already hold.
It is called through the C ABI (ctypes) and compared with gc_correlate,
with the same tolerance as the other FFT-correlator tests, on two calls in a
row of different shapes (the shared scratch keeps the previous call's
contents, which must not matter).  This file is collected last on purpose.
"""
import ctypes

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
def api():
    from paper_2005_03060_gb300 import gridcorr
    lib = gridcorr.lib()
    f = lib.gc_correlate_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return gridcorr, f


def _noalloc(f, volt, gains, L, status):
    C, T, N = volt.shape[:3]
    W = 2 * L - 1
    out = torch.empty(C, W, W, dtype=torch.complex64, device=volt.device)
    vfmt = {torch.complex64: 0, torch.uint8: 1, torch.float16: 2}[volt.dtype]
    st = f(volt.data_ptr(), vfmt, L, C, T, gains.data_ptr(), out.data_ptr(), status.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    return st, out


def test_noalloc_matches_correlate_twice(api):
    gridcorr, f = api
    ctx = gridcorr.Context(0)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for seed, (L, C, T) in enumerate([(32, 8, 1000), (8, 4, 300)]):
        volt, gains, _ = synth.make_voltages(300 + seed, L, C, T, n_src=20)
        v, g = volt.cuda(), gains.cuda()
        st, out = _noalloc(f, v, g, L, status)
        assert st == gridcorr.GC_OK
        ref = ctx.correlate(v, g)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        for c in range(C):
            assert lag_err(a[c], b[c], L) < TOL, (L, c)


def test_noalloc_rejects_sizes_beyond_its_scratch(api):
    gridcorr, f = api
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    dummy = torch.zeros(4, dtype=torch.complex64, device="cuda")
    # 64x64 grid (M = 128), 512 channels, 4096 samples: 512 * 8 * 128^2 * 4 B = 256 MiB > 64 MiB.
    # The size check runs before any launch, so the small dummy buffers are never touched.
    st = f(dummy.data_ptr(), 0, 64, 512, 4096, dummy.data_ptr(), dummy.data_ptr(),
           status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == gridcorr.GC_EINVAL


@pytest.mark.parametrize("fmt,L,C,T", [
    ("i4c", 64, 128, 4096),   # 128 ch x 8 chunks x 128^2 x 4 B = exactly the 64 MiB of scratch
    ("c64", 7, 3, 200),       # a grid row of 56 bytes: plain loads instead of TMA
    ("c32h", 16, 4, 700),     # binary16-stored voltages
])
def test_noalloc_formats_and_bounds(api, fmt, L, C, T):
    """The other voltage formats, the non-TMA staging path and a call that
    fills the fixed scratch to its last byte (the chunk count clamped to
    what fits) equal gc_correlate within the same tolerance."""
    gridcorr, f = api
    ctx = gridcorr.Context(0)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    if fmt == "i4c":
        # random 4+4-bit codes (the full nibble range) and gains near 1
        gen = torch.Generator(device="cuda").manual_seed(L)
        v = torch.randint(0, 256, (C, T, L * L), dtype=torch.uint8, device="cuda", generator=gen)
        _, gains, _ = synth.make_voltages(900 + L, L, C, 1, n_src=1)
        g = gains.cuda()
    else:
        volt, gains, _ = synth.make_voltages(900 + L, L, C, T, n_src=20)
        g = gains.cuda()
    if fmt == "i4c":
        pass
    elif fmt == "c32h":
        v = torch.view_as_real(volt).to(torch.float16).contiguous().cuda()
    else:
        v = volt.cuda()
    st, out = _noalloc(f, v, g, L, status)
    assert st == gridcorr.GC_OK
    ref = ctx.correlate(v, g)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    a, b = out.cpu().numpy(), ref.cpu().numpy()
    for c in sorted({0, C // 2, C - 1}):
        assert lag_err(a[c], b[c], L) < TOL, (fmt, L, c)
