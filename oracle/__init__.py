"""FP64 reference implementation (the oracle) of the FFT-correlator system.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark import this package; the library's product
path never does, and this package imports nothing from the library.

Heavy loops (FX correlator, direct-DFT correlator, X-engine, quantiser) are
plain C in this directory, compiled with gcc into liboracle.so by
`build()`; the calibration oracle (calib.py) and the selections (select.py)
are plain numpy / Python.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = ["correlate.c", "xengine.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP over channels in orc_fx_multi)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in srcs):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + \
          [os.path.join(_HERE, s) for s in _SRC] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            i = ctypes.c_int
            L.orc_fx.argtypes = [i, i, dp, dp, dp, dp]
            L.orc_fx_multi.argtypes = [i, i, i, dp, dp, dp]
            L.orc_fx_multi.restype = ctypes.c_int
            L.orc_fx_par.argtypes = [i, i, dp, dp, dp]
            L.orc_fx_par.restype = ctypes.c_int
            L.orc_dft.argtypes = [i, i, i, dp, dp, dp, dp]
            L.orc_lag.argtypes = [i, i, dp, dp, i, i, dp]
            L.orc_xeng_c64.argtypes = [i, i, dp, i, ip, ip, ip, ip, dp]
            L.orc_xeng_i4c.argtypes = [i, i, ctypes.c_void_p, i, ip, ip, ip, ip, ctypes.c_void_p]
            L.orc_autos_c64.argtypes = [i, i, dp, i, i, dp]
            L.orc_quantize.argtypes = [i, i, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_quantize.restype = ctypes.c_float
            _lib = L
    return _lib


# ----------------------------------------------------------------------------- helpers
def _c128(a) -> np.ndarray:
    """complex array -> contiguous complex128 (viewed as interleaved doubles)."""
    return np.ascontiguousarray(np.asarray(a), dtype=np.complex128)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def fx(volt, gains=None, L=None, full=False):
    """FX correlator of one channel; volt [T, N] complex. Returns V^unique
    [(2L-1), (2L-1)] (and V^full [N, N] when full=True)."""
    v = _c128(volt)
    T, N = v.shape
    L = L or int(round(N ** 0.5))
    W = 2 * L - 1
    out = np.zeros((W, W), np.complex128)
    vf = np.zeros((N, N), np.complex128) if full else None
    g = None if gains is None else _c128(gains)
    lib().orc_fx(L, T, _dp(v), _dp(g) if g is not None else None, _dp(out),
                 _dp(vf) if full else None)
    return (out, vf) if full else out


def fx_par(volt, gains, L=None):
    """V^unique of one channel by the FX definition (orc_fx's sums, the pair
    loop over OpenMP threads); volt [T, N] complex.  Returns (V^unique, threads)."""
    v = _c128(volt)
    T, N = v.shape
    L = L or int(round(N ** 0.5))
    W = 2 * L - 1
    out = np.zeros((W, W), np.complex128)
    g = None if gains is None else _c128(gains)
    n = lib().orc_fx_par(L, T, _dp(v), _dp(g) if g is not None else None, _dp(out))
    return out, n


def fx_multi(volt, gains, L):
    """FX correlator over channels (OpenMP); volt [C, T, N]. Returns
    (V^unique [C, W, W], threads used)."""
    v = _c128(volt)
    C, T, N = v.shape
    W = 2 * L - 1
    out = np.zeros((C, W, W), np.complex128)
    g = _c128(gains)
    nt = lib().orc_fx_multi(C, L, T, _dp(v), _dp(g), _dp(out))
    return out, nt


def dft(volt, gains=None, L=None, M=None, return_pk=False):
    """Direct-DFT FFT-correlator of one channel."""
    v = _c128(volt)
    T, N = v.shape
    L = L or int(round(N ** 0.5))
    M = M or 1 << (2 * L - 2).bit_length()
    W = 2 * L - 1
    out = np.zeros((W, W), np.complex128)
    pk = np.zeros((M, M), np.float64)
    g = None if gains is None else _c128(gains)
    lib().orc_dft(L, M, T, _dp(v), _dp(g) if g is not None else None, _dp(out), _dp(pk))
    return (out, pk) if return_pk else out


def lag(volt, gains, L, dx, dy):
    """One lag of V^unique by definition (Eq. modelvis)."""
    v = _c128(volt)
    T, N = v.shape
    out = np.zeros(1, np.complex128)
    g = None if gains is None else _c128(gains)
    lib().orc_lag(L, T, _dp(v), _dp(g) if g is not None else None, dx, dy, _dp(out))
    return complex(out[0])


def xengine_c64(volt, pair_i, pair_j, t0, t1):
    """Raw pair sums over each pair's window; volt [T, N] complex."""
    v = _c128(volt)
    T, N = v.shape
    pi = np.ascontiguousarray(pair_i, np.int32)
    pj = np.ascontiguousarray(pair_j, np.int32)
    a0 = np.ascontiguousarray(t0, np.int32)
    a1 = np.ascontiguousarray(t1, np.int32)
    out = np.zeros(len(pi), np.complex128)
    lib().orc_xeng_c64(N, T, _dp(v), len(pi), _ip(pi), _ip(pj), _ip(a0), _ip(a1), _dp(out))
    return out


def xengine_i4c(volt_u8, pair_i, pair_j, t0, t1):
    """Exact int64 pair sums on 4+4-bit voltages; volt [T, N] uint8/int8."""
    v = np.ascontiguousarray(np.asarray(volt_u8).view(np.uint8))
    T, N = v.shape
    pi = np.ascontiguousarray(pair_i, np.int32)
    pj = np.ascontiguousarray(pair_j, np.int32)
    a0 = np.ascontiguousarray(t0, np.int32)
    a1 = np.ascontiguousarray(t1, np.int32)
    out = np.zeros((len(pi), 2), np.int64)
    lib().orc_xeng_i4c(N, T, v.ctypes.data, len(pi), _ip(pi), _ip(pj), _ip(a0), _ip(a1),
                       out.ctypes.data)
    return out


def autos(volt, t0=0, t1=None):
    v = _c128(volt)
    T, N = v.shape
    out = np.zeros(N, np.float64)
    lib().orc_autos_c64(N, T, _dp(v), t0, T if t1 is None else t1, _dp(out))
    return out


def quantize(volt):
    """4+4-bit quantiser of one channel; volt [T, N] complex64.
    Returns (bytes [T, N] uint8, float scale)."""
    v = np.ascontiguousarray(np.asarray(volt), dtype=np.complex64)
    T, N = v.shape
    out = np.zeros((T, N), np.uint8)
    s = lib().orc_quantize(T, N, v.ctypes.data, out.ctypes.data)
    return out, float(s)


def unpack_i4c(b):
    """bytes -> complex128 integer-valued voltages (high nibble = Re)."""
    b = np.asarray(b).view(np.uint8).astype(np.int16)
    hi = (b >> 4) & 15
    lo = b & 15
    hi = np.where(hi >= 8, hi - 16, hi)
    lo = np.where(lo >= 8, lo - 16, lo)
    return hi.astype(np.float64) + 1j * lo.astype(np.float64)


def fx_masked(volt, gains, mask, L):
    """V^unique of an array on a partly occupied L x L lattice grid (Eq.
    modelvis by definition, numpy): w = v / g on the occupied points; for
    every separation d = r_i - r_j of two occupied points, the time average
    of w_i conj(w_j) summed over those pairs and divided by their number N_d.
    Returns (V [(2L-1), (2L-1)] indexed [dy + L - 1][dx + L - 1], N_d); lags
    without a pair are 0."""
    v = _c128(volt)
    T = v.shape[0]
    occ = np.flatnonzero(np.asarray(mask))
    w = v[:, occ] / _c128(gains)[occ][None, :]
    S = w.T @ np.conj(w) / T                       # S[i, j] = <w_i conj(w_j)>
    x, y = occ % L, occ // L
    dx = (x[:, None] - x[None, :]) + (L - 1)
    dy = (y[:, None] - y[None, :]) + (L - 1)
    W = 2 * L - 1
    out = np.zeros((W, W), np.complex128)
    nd = np.zeros((W, W), np.int64)
    np.add.at(out, (dy.ravel(), dx.ravel()), S.ravel())
    np.add.at(nd, (dy.ravel(), dx.ravel()), 1)
    nz = nd > 0
    out[nz] /= nd[nz]
    return out, nd
