"""Python binding of the gridcorr C ABI (include/gridcorr.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of libgridcorr.so.  Tensors are torch CUDA tensors; the library is
handed their device pointers and the current torch stream.  There is no
CPU fallback: importing this module raises if the compiled library is
missing, and every call raises GridcorrError on a non-OK status.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgridcorr.so")

GC_OK, GC_EINVAL, GC_ENOMEM, GC_ECUDA, GC_ENOCONV, GC_ETIMEOUT, GC_EDEGEN, GC_EUNSUPPORTED = range(8)
STATUS_NAMES = ["GC_OK", "GC_EINVAL", "GC_ENOMEM", "GC_ECUDA", "GC_ENOCONV", "GC_ETIMEOUT",
                "GC_EDEGEN", "GC_EUNSUPPORTED"]
GC_C64, GC_I4C = 0, 1


class GridcorrError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                      "(there is no CPU fallback)")
_lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_i = ctypes.c_int
_lib.gc_create.argtypes = [ctypes.POINTER(_vp), _i]
_lib.gc_create.restype = _i
_lib.gc_destroy.argtypes = [_vp]
_lib.gc_destroy.restype = None
_lib.gc_last_error.argtypes = [_vp]
_lib.gc_last_error.restype = ctypes.c_char_p
_lib.gc_device_status.argtypes = [_vp, _vp]
_lib.gc_device_status.restype = _i
_lib.gc_fft_size.argtypes = [_i]
_lib.gc_fft_size.restype = _i
_lib.gc_profile_enable.argtypes = [_vp, _i]
_lib.gc_profile_enable.restype = _i
_lib.gc_profile_read.argtypes = [_vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(_i), _i]
_lib.gc_profile_read.restype = _i
_lib.gc_correlate.argtypes = [_vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp]
_lib.gc_correlate.restype = _i


def lib() -> ctypes.CDLL:
    return _lib


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class Context:
    """Owns a gc_ctx (device status word + grow-only scratch workspace)."""

    def __init__(self, device: int | torch.device | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        h = _vp()
        st = _lib.gc_create(ctypes.byref(h), self.device.index or 0)
        if st != GC_OK:
            raise GridcorrError(st, "gc_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.gc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def check(self, st: int):
        if st != GC_OK:
            raise GridcorrError(st, _lib.gc_last_error(self._h).decode())

    def device_status(self):
        """Synchronise the current stream and raise if a kernel timed out."""
        self.check(_lib.gc_device_status(self._h, _vp(_stream_ptr(self.device))))

    # ------------------------------------------------------------------ profiling
    def profile(self, enable: bool = True):
        """Record CUDA events around every kernel the library launches."""
        self.check(_lib.gc_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the last read (syncs)."""
        kmax = 32
        names = ctypes.create_string_buffer(64 * kmax)
        ms = (ctypes.c_double * kmax)()
        cnt = (_i * kmax)()
        n = _lib.gc_profile_read(self._h, names, ms, cnt, kmax)
        out = {}
        for k in range(max(0, min(n, kmax))):
            nm = names.raw[64 * k:64 * k + 64].split(b"\0", 1)[0].decode()
            out[nm] = (ms[k], cnt[k])
        return out

    # ------------------------------------------------------------------ correlate
    def correlate(self, volt: torch.Tensor, gains: torch.Tensor, L: int | None = None,
                  out: torch.Tensor | None = None) -> torch.Tensor:
        """V^unique [C, 2L-1, 2L-1] complex64 from voltages [C, T, L*L]
        (complex64, or uint8/int8 4+4-bit) and gains [C, L*L] complex64."""
        vfmt = GC_C64 if volt.dtype == torch.complex64 else GC_I4C
        if vfmt == GC_I4C and volt.dtype not in (torch.uint8, torch.int8):
            raise TypeError("voltages must be complex64 or 4+4-bit bytes (uint8/int8)")
        C, T, N = volt.shape
        L = L or int(round(N ** 0.5))
        if L * L != N:
            raise ValueError("the antenna axis must hold an L x L grid")
        if gains.dtype != torch.complex64 or tuple(gains.shape) != (C, N):
            raise ValueError("gains must be complex64 [C, L*L]")
        for t in (volt, gains):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("inputs must be contiguous CUDA tensors")
        W = 2 * L - 1
        if out is None:
            out = torch.empty(C, W, W, dtype=torch.complex64, device=volt.device)
        self.check(_lib.gc_correlate(self._h, _vp(volt.data_ptr()), vfmt, L, C, T,
                                     _vp(gains.data_ptr()), _vp(out.data_ptr()),
                                     _vp(_stream_ptr(volt.device))))
        return out


def fft_size(L: int) -> int:
    return _lib.gc_fft_size(L)


_default = {}


def default_context(device=None) -> Context:
    dev = torch.cuda.current_device() if device is None else (
        device.index if isinstance(device, torch.device) else int(device))
    if dev not in _default:
        _default[dev] = Context(dev)
    return _default[dev]


def correlate(volt, gains, L=None, out=None):
    return default_context(volt.device).correlate(volt, gains, L, out)
