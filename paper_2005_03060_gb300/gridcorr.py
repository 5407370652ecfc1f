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
GC_C64, GC_I4C, GC_C32H = 0, 1, 2
LATTICES = {"square": 0, "triangular": 1}


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
_lib.gc_correlate_masked.argtypes = [_vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp]
_lib.gc_correlate_masked.restype = _i
_lib.gc_gain_variance.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.gc_gain_variance.restype = _i
_lib.gc_gain_covariance.argtypes = [_vp, _vp, _i, _i, _vp, _vp, _vp, _vp]
_lib.gc_gain_covariance.restype = _i
_lib.gc_visibility_variance.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp, _vp, _vp]
_lib.gc_visibility_variance.restype = _i
_lib.gc_sel_edge.argtypes = [_vp, _vp]
_lib.gc_sel_edge.restype = _i
_lib.gc_selection_subset.argtypes = [_i, _i, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_vp)]
_lib.gc_selection_subset.restype = _i
_lib.gc_selection_lowcad.argtypes = [_i, _i, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_vp)]
_lib.gc_selection_subset_masked.argtypes = [_i, _i, ctypes.c_double, ctypes.c_double, _vp, _i, ctypes.POINTER(_vp)]
_lib.gc_selection_subset_masked.restype = _i
_lib.gc_selection_lowcad_masked.argtypes = [_i, _i, ctypes.c_double, ctypes.c_double, _vp, _i, ctypes.POINTER(_vp)]
_lib.gc_selection_lowcad_masked.restype = _i
_lib.gc_selection_lowcad.restype = _i
_lib.gc_sel_free.argtypes = [_vp]
_lib.gc_sel_free.restype = None
_lib.gc_sel_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
_lib.gc_sel_info.restype = _i
_i32pp = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
_lib.gc_sel_arrays.argtypes = [_vp] + [_i32pp] * 6
_lib.gc_sel_arrays.restype = _i
_lib.gc_reduce.argtypes = [_vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp]
_lib.gc_reduce.restype = _i
_lib.gc_calibrate.argtypes = [_vp, _vp, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.gc_calibrate.restype = _i
_lib.gc_peak_probe.argtypes = [_vp, _i, ctypes.POINTER(ctypes.c_double)]
_lib.gc_peak_probe.restype = _i
_lib.gc_chi2.argtypes = [_vp, _vp, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp]
_lib.gc_chi2.restype = _i
_lib.gc_chi2_backward.argtypes = [_vp, _vp, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.gc_chi2_backward.restype = _i
_lib.gc_calibrate_batched.argtypes = [_vp, _i, _vp, _vp, _vp]
_lib.gc_calibrate_batched.restype = _i
_lib.gc_set_tuning.argtypes = [_vp, ctypes.c_char_p, _i]
_lib.gc_set_tuning.restype = _i
_lib.gc_get_tuning.argtypes = [_vp, ctypes.c_char_p, ctypes.POINTER(_i)]
_lib.gc_get_tuning.restype = _i
_lib.gc_quantize.argtypes = [_vp, _vp, _i, _i, _i, _vp, _vp, _vp]
_lib.gc_quantize.restype = _i
_lib.gc_chi2_ckpt.argtypes = [_vp, _vp, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.gc_chi2_ckpt.restype = _i
_lib.gc_chi2_backward_ckpt.argtypes = [_vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.gc_chi2_backward_ckpt.restype = _i
_lib.gc_integrate_host.argtypes = [_vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp]
_lib.gc_integrate_host.restype = _i


def _volt_format(volt: torch.Tensor):
    """(gc_vfmt, (C, T, N)) of a voltage tensor."""
    if volt.dtype == torch.complex64 and volt.dim() == 3:
        return GC_C64, tuple(volt.shape)
    if volt.dtype in (torch.uint8, torch.int8) and volt.dim() == 3:
        return GC_I4C, tuple(volt.shape)
    if volt.dtype == torch.complex32 and volt.dim() == 3:
        return GC_C32H, tuple(volt.shape)
    if volt.dtype == torch.float16 and volt.dim() == 4 and volt.shape[-1] == 2:
        return GC_C32H, tuple(volt.shape[:3])
    raise TypeError("voltages must be complex64 [C, T, N], binary16 pairs (complex32 [C, T, N] or "
                    "float16 [C, T, N, 2]) or 4+4-bit bytes (uint8/int8 [C, T, N])")


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

    def peak_probe(self, kind: str) -> float:
        """Measured throughput in tera-ops/s: 'fp32' / 'fp64' FMA (2 flops),
        'dp4a' (8 integer ops), 'tc_f8' (dense e4m3 tensor-core MMA, 2 M N K),
        'mma_s8' (warp-level int8 MMA, 2 M N K)."""
        v = ctypes.c_double()
        self.check(_lib.gc_peak_probe(self._h, {"fp32": 0, "fp64": 1, "dp4a": 2, "tc_f8": 3, "mma_s8": 4}[kind], ctypes.byref(v)))
        return v.value

    # ------------------------------------------------------------------ correlate
    def correlate(self, volt: torch.Tensor, gains: torch.Tensor, L: int | None = None,
                  out: torch.Tensor | None = None, mask=None) -> torch.Tensor:
        """V^unique [C, 2L-1, 2L-1] complex64 from voltages [C, T, L*L]
        (complex64; binary16 pairs as complex32 [C, T, L*L] or float16
        [C, T, L*L, 2]; or uint8/int8 4+4-bit) and gains [C, L*L] complex64.
        mask: L*L occupancy of a partly occupied lattice (gc_correlate_masked)."""
        vfmt, (C, T, N) = _volt_format(volt)
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
        if mask is None:
            self.check(_lib.gc_correlate(self._h, _vp(volt.data_ptr()), vfmt, L, C, T,
                                         _vp(gains.data_ptr()), _vp(out.data_ptr()),
                                         _vp(_stream_ptr(volt.device))))
        else:
            import numpy as np
            m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
            if m.size != N:
                raise ValueError("mask must have L*L entries")
            self.check(_lib.gc_correlate_masked(self._h, _vp(volt.data_ptr()), vfmt, L, C, T,
                                                m.ctypes.data_as(_vp), _vp(gains.data_ptr()),
                                                _vp(out.data_ptr()), _vp(_stream_ptr(volt.device))))
        return out

    # ------------------------------------------------------------------ covariance
    def gain_variance(self, sel: Selection):
        """Eq. gaincov predicted variances (gc_gain_variance): (var_amp,
        var_phase), float32 CUDA tensors of L*L + n_ubl (antennas, then model
        visibilities), for unit visibility noise."""
        dev = self.device
        n = sel.L * sel.L + sel.n_ubl
        va = torch.empty(n, dtype=torch.float32, device=dev)
        vp = torch.empty(n, dtype=torch.float32, device=dev)
        self.check(_lib.gc_gain_variance(self._h, sel.handle, _vp(va.data_ptr()), _vp(vp.data_ptr()),
                                         _vp(_stream_ptr(dev))))
        return va, vp

    def gain_covariance(self, sel: Selection, rows, fixed: bool = False):
        """Gain covariance rows (gc_gain_covariance): (cov_amp, cov_phase),
        float32 CUDA tensors [len(rows), row length] -- rows of the
        pseudo-inverses over all L*L + n_ubl unknowns, or (fixed) the antenna
        covariance with the degeneracies fixed against the truth, [.., L*L]."""
        import numpy as np
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32).reshape(-1))
        dev = self.device
        n = sel.L * sel.L + (0 if fixed else sel.n_ubl)
        ca = torch.empty(r.size, n, dtype=torch.float32, device=dev)
        cp = torch.empty(r.size, n, dtype=torch.float32, device=dev)
        self.check(_lib.gc_gain_covariance(self._h, sel.handle, int(bool(fixed)), int(r.size),
                                           r.ctypes.data_as(_vp), _vp(ca.data_ptr()), _vp(cp.data_ptr()),
                                           _vp(_stream_ptr(dev))))
        return ca, cp

    def visibility_variance(self, sel: Selection, snr_full_inv2: float, sigma_cal2: float):
        """Relative variance of every V^unique lag calibrated with this
        selection's gains (gc_visibility_variance): (var_pair, var_exact,
        n_pairs), CUDA tensors [2L-1, 2L-1] indexed [dy + L - 1, dx + L - 1]."""
        dev = self.device
        n = 2 * sel.L - 1
        vp = torch.empty(n, n, dtype=torch.float64, device=dev)
        ve = torch.empty(n, n, dtype=torch.float64, device=dev)
        npr = torch.empty(n, n, dtype=torch.int32, device=dev)
        self.check(_lib.gc_visibility_variance(self._h, sel.handle, float(snr_full_inv2), float(sigma_cal2),
                                               _vp(vp.data_ptr()), _vp(ve.data_ptr()), _vp(npr.data_ptr()),
                                               _vp(_stream_ptr(dev))))
        return vp, ve, npr

    # ------------------------------------------------------------------ reduce
    def reduce(self, volt: torch.Tensor, sel: Selection, autos: bool = True, out=None, out_autos=None):
        """V^reduced raw pair sums: complex64 [C, P] for complex64 voltages,
        int32 [C, P, 2] (exact) for 4+4-bit voltages; plus autos [C, N].
        Binary16 voltages (complex32 / float16 pairs) give complex64 sums."""
        vfmt, (C, T, N) = _volt_format(volt)
        if not volt.is_cuda or not volt.is_contiguous():
            raise ValueError("voltages must be a contiguous CUDA tensor")
        if out is None:
            out = (torch.empty(C, sel.P, dtype=torch.complex64, device=volt.device) if vfmt != GC_I4C
                   else torch.empty(C, sel.P, 2, dtype=torch.int32, device=volt.device))
        a = None
        if autos:
            a = out_autos if out_autos is not None else torch.empty(
                C, N, dtype=torch.float32 if vfmt != GC_I4C else torch.int32, device=volt.device)
        self.check(_lib.gc_reduce(self._h, _vp(volt.data_ptr()), vfmt, sel.L, C, T, sel.handle,
                                  _vp(out.data_ptr()), _vp(a.data_ptr() if a is not None else None),
                                  _vp(_stream_ptr(volt.device))))
        return (out, a) if autos else out

    # ------------------------------------------------------------------ calibrate
    def calibrate(self, vred: torch.Tensor, sel: Selection, autos: torch.Tensor | None = None,
                  solver: str = "lincal", precision: str = "fp64", max_iter: int = 0,
                  tol: float = 0.0, damping: float = 0.0, time_limit_ms: int = 0,
                  gains: torch.Tensor | None = None, vmodel: torch.Tensor | None = None,
                  warm_start: bool = False, stats: torch.Tensor | None = None,
                  fp32_reductions: bool = False):
        """Per-channel redundant calibration of V^reduced (gc_reduce output).
        fp32_reductions: the matrix-free solver's plain-FP32 form (chi^2 and
        step norms summed in FP32 instead of FP64).
        Returns (gains [C, N] complex64, vmodel [C, n_ubl] complex64, stats
        as a uint8 device tensor [C, 32]; decode with `decode_stats`)."""
        vfmt = GC_C64 if vred.dtype == torch.complex64 else GC_I4C
        C = vred.shape[0]
        N = sel.L * sel.L
        dev = vred.device
        gains = gains if gains is not None else torch.empty(C, N, dtype=torch.complex64, device=dev)
        vmodel = vmodel if vmodel is not None else torch.empty(C, sel.n_ubl, dtype=torch.complex64, device=dev)
        stats = stats if stats is not None else torch.empty(C, 32, dtype=torch.uint8, device=dev)
        o = CalOpts({"lincal": GC_LINCAL, "omnical": GC_OMNICAL, "lincal_cg": GC_LINCAL_CG}[solver],
                    GC_FP64 if precision == "fp64" else GC_FP32, max_iter, 1 if warm_start else 0,
                    tol, damping, time_limit_ms, 1 if fp32_reductions else 0)
        self.check(_lib.gc_calibrate(self._h, _vp(vred.data_ptr()), vfmt, sel.handle, C,
                                     _vp(autos.data_ptr() if autos is not None else None),
                                     ctypes.byref(o), _vp(gains.data_ptr()), _vp(vmodel.data_ptr()),
                                     _vp(stats.data_ptr()), _vp(_stream_ptr(dev))))
        return gains, vmodel, stats

    def integrate_host(self, h_volt: torch.Tensor, sel: "Selection", gains_in: torch.Tensor,
                       vunique: torch.Tensor, vreduced: torch.Tensor, autos: torch.Tensor | None,
                       gains_out: torch.Tensor, vmodel: torch.Tensor, stats: torch.Tensor,
                       solver: str = "lincal_cg", precision: str = "fp32", chunk: int = 0):
        """One integration of host-resident voltages (pinned CPU tensor of
        any gc_vfmt layout) through correlate -> reduce -> calibrate,
        streamed in channel chunks (gc_integrate_host); outputs are the
        device tensors passed in, on the current stream.  gains_in may be a
        CUDA tensor or a (pinned) host tensor, which the library copies on
        its own copy stream."""
        if h_volt.is_cuda or not h_volt.is_contiguous():
            raise ValueError("h_volt must be a contiguous host tensor")
        vfmt, (C, T, N) = _volt_format(h_volt)
        dev = vunique.device
        if gains_in.dtype != torch.complex64 or not gains_in.is_contiguous() or tuple(gains_in.shape) != (C, N):
            raise ValueError("gains_in must be a contiguous complex64 [C, L*L] tensor")
        for t in (vunique, vreduced, gains_out, vmodel, stats) + ((autos,) if autos is not None else ()):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("outputs must be contiguous CUDA tensors")
        o = CalOpts({"lincal": GC_LINCAL, "omnical": GC_OMNICAL, "lincal_cg": GC_LINCAL_CG}[solver],
                    GC_FP64 if precision == "fp64" else GC_FP32, 0, 0, 0.0, 0.0, 0, 0)
        self.check(_lib.gc_integrate_host(self._h, _vp(h_volt.data_ptr()), vfmt, sel.L, C, T, sel.handle,
                                          _vp(gains_in.data_ptr()), _vp(vunique.data_ptr()),
                                          _vp(vreduced.data_ptr()),
                                          _vp(autos.data_ptr() if autos is not None else None),
                                          ctypes.byref(o), _vp(gains_out.data_ptr()), _vp(vmodel.data_ptr()),
                                          _vp(stats.data_ptr()), chunk, _vp(_stream_ptr(dev))))
        return vunique, gains_out

    def calibrate_batched(self, arrays, max_iter: int = 0, tol: float = 0.0, time_limit_ms: int = 0):
        """One persistent launch over several arrays.  `arrays` is a list of
        dicts with keys vred, sel and optionally autos, gains, vmodel, stats
        (outputs are allocated when missing).  Returns the list of
        (gains, vmodel, stats) tuples."""
        outs = []
        items = (BatchItem * len(arrays))()
        for k, a in enumerate(arrays):
            vred, sel = a["vred"], a["sel"]
            C = vred.shape[0]
            dev = vred.device
            g = a.get("gains")
            g = g if g is not None else torch.empty(C, sel.L * sel.L, dtype=torch.complex64, device=dev)
            v = a.get("vmodel")
            v = v if v is not None else torch.empty(C, sel.n_ubl, dtype=torch.complex64, device=dev)
            st = a.get("stats")
            st = st if st is not None else torch.empty(C, 32, dtype=torch.uint8, device=dev)
            au = a.get("autos")
            items[k] = BatchItem(sel.handle.value if isinstance(sel.handle, _vp) else sel.handle, C,
                                 GC_C64 if vred.dtype == torch.complex64 else GC_I4C, vred.data_ptr(),
                                 au.data_ptr() if au is not None else None, g.data_ptr(), v.data_ptr(),
                                 st.data_ptr())
            outs.append((g, v, st))
        o = CalOpts(GC_LINCAL_CG, GC_FP32, max_iter, 0, tol, 0.0, time_limit_ms, 0)
        self.check(_lib.gc_calibrate_batched(self._h, len(arrays), ctypes.cast(items, _vp), ctypes.byref(o),
                                             _vp(_stream_ptr(arrays[0]["vred"].device))))
        return outs

    def set_tuning(self, name: str, value: int):
        self.check(_lib.gc_set_tuning(self._h, name.encode(), int(value)))

    def get_tuning(self, name: str) -> int:
        v = _i()
        self.check(_lib.gc_get_tuning(self._h, name.encode(), ctypes.byref(v)))
        return v.value

    # ------------------------------------------------------------------ chi^2 and adjoint
    def chi2(self, vred, sel, gains, vmodel, weights=None, out=None, residuals=None):
        """chi^2 per channel (float64 [C]).  residuals: a complex64 [C, P]
        tensor that receives r_p (the checkpointed form, gc_chi2_ckpt)."""
        vfmt = GC_C64 if vred.dtype == torch.complex64 else GC_I4C
        C = vred.shape[0]
        out = out if out is not None else torch.empty(C, dtype=torch.float64, device=vred.device)
        w = _vp(weights.data_ptr() if weights is not None else None)
        if residuals is None:
            self.check(_lib.gc_chi2(self._h, _vp(vred.data_ptr()), vfmt, sel.handle, C,
                                    _vp(gains.data_ptr()), _vp(vmodel.data_ptr()), w,
                                    _vp(out.data_ptr()), _vp(_stream_ptr(vred.device))))
        else:
            if residuals.dtype != torch.complex64 or tuple(residuals.shape) != (C, sel.P):
                raise ValueError("residuals must be complex64 [C, P]")
            self.check(_lib.gc_chi2_ckpt(self._h, _vp(vred.data_ptr()), vfmt, sel.handle, C,
                                         _vp(gains.data_ptr()), _vp(vmodel.data_ptr()), w,
                                         _vp(out.data_ptr()), _vp(residuals.data_ptr()),
                                         _vp(_stream_ptr(vred.device))))
        return out

    def chi2_backward_ckpt(self, residuals, sel, gains, vmodel, grad_out=None, weights=None):
        """Gradients from residuals stored by chi2(..., residuals=)."""
        C = residuals.shape[0]
        dg = torch.empty_like(gains)
        dv = torch.empty_like(vmodel)
        go = grad_out.contiguous().to(torch.float64) if grad_out is not None else None
        self.check(_lib.gc_chi2_backward_ckpt(self._h, _vp(residuals.data_ptr()), sel.handle, C,
                                              _vp(gains.data_ptr()), _vp(vmodel.data_ptr()),
                                              _vp(weights.data_ptr() if weights is not None else None),
                                              _vp(go.data_ptr() if go is not None else None),
                                              _vp(dg.data_ptr()), _vp(dv.data_ptr()),
                                              _vp(_stream_ptr(residuals.device))))
        return dg, dv

    def chi2_backward(self, vred, sel, gains, vmodel, grad_out=None, weights=None):
        vfmt = GC_C64 if vred.dtype == torch.complex64 else GC_I4C
        C = vred.shape[0]
        dg = torch.empty_like(gains)
        dv = torch.empty_like(vmodel)
        go = grad_out.contiguous().to(torch.float64) if grad_out is not None else None
        self.check(_lib.gc_chi2_backward(self._h, _vp(vred.data_ptr()), vfmt, sel.handle, C,
                                         _vp(gains.data_ptr()), _vp(vmodel.data_ptr()),
                                         _vp(weights.data_ptr() if weights is not None else None),
                                         _vp(go.data_ptr() if go is not None else None),
                                         _vp(dg.data_ptr()), _vp(dv.data_ptr()),
                                         _vp(_stream_ptr(vred.device))))
        return dg, dv

    # ------------------------------------------------------------------ quantise
    def quantize(self, volt: torch.Tensor, out=None, scales=None):
        """4+4-bit bytes [C, T, N] uint8 and per-channel float scales [C]."""
        C, T, N = volt.shape
        if volt.dtype != torch.complex64 or not volt.is_cuda or not volt.is_contiguous():
            raise ValueError("voltages must be contiguous complex64 CUDA tensors")
        out = out if out is not None else torch.empty(C, T, N, dtype=torch.uint8, device=volt.device)
        scales = scales if scales is not None else torch.empty(C, dtype=torch.float32, device=volt.device)
        self.check(_lib.gc_quantize(self._h, _vp(volt.data_ptr()), C, T, N, _vp(out.data_ptr()),
                                    _vp(scales.data_ptr()), _vp(_stream_ptr(volt.device))))
        return out, scales


GC_LINCAL, GC_OMNICAL, GC_LINCAL_CG = 0, 1, 2
GC_FP64, GC_FP32 = 0, 1


class CalOpts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("precision", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("tol", ctypes.c_double), ("damping", ctypes.c_double),
                ("time_limit_ms", ctypes.c_int), ("reserved", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("sel", ctypes.c_void_p), ("C", ctypes.c_int), ("vfmt", ctypes.c_int),
                ("vreduced", ctypes.c_void_p), ("autos", ctypes.c_void_p), ("gains", ctypes.c_void_p),
                ("vmodel", ctypes.c_void_p), ("stats", ctypes.c_void_p)]


STATS_DTYPE = [("chi2", "<f8"), ("chi2r", "<f8"), ("dof", "<i4"), ("iters", "<i4"),
               ("status", "<i4"), ("inner", "<i4")]


class Selection:
    """A reduced-calibration selection (host object of the library).

    Attributes (numpy int32 copies): types [n_ubl, 2], type_ptr [n_ubl+1],
    pair_i, pair_j [P], win_t0, win_t1 [n_ubl]; scalars L, T, P, n_ubl,
    n_cycle, t_int, null_dim, scheme ('subset' or 'lowcad'), masked,
    lattice ('square' or 'triangular'), n_ant (occupied points).

    mask: for an array on a partly occupied lattice (e.g. hex_mask(s)), the
    L*L occupancy of the bounding grid.
    """

    def __init__(self, scheme: str, L: int, T: int, p: float = 1.0, log_base: float = 2.0,
                 mask=None, lattice: str = "square"):
        import numpy as np
        h = _vp()
        if mask is not None:
            m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
            if m.size != L * L:
                raise ValueError("mask must have L*L entries")
            self.mask = m
            fn = {"subset": _lib.gc_selection_subset_masked, "lowcad": _lib.gc_selection_lowcad_masked}[scheme]
            st = fn(L, T, p, log_base, m.ctypes.data_as(_vp), LATTICES[lattice], ctypes.byref(h))
        else:
            self.mask = None
            fn = {"subset": _lib.gc_selection_subset, "lowcad": _lib.gc_selection_lowcad}[scheme]
            st = fn(L, T, p, log_base, ctypes.byref(h))
        if st != GC_OK:
            raise GridcorrError(st, f"gc_selection_{scheme}(L={L}, T={T}, p={p}, masked={mask is not None})")
        self._h = h
        info = (ctypes.c_int32 * 11)()
        _lib.gc_sel_info(h, info)
        (self.L, self.T, self.P, self.n_ubl, self.n_cycle, self.t_int, self.null_dim,
         sch, self.masked, lat, self.n_ant) = list(info)
        self.lattice = "triangular" if lat == 1 else "square"
        self.scheme = "subset" if sch == 0 else "lowcad"
        ptrs = [ctypes.POINTER(ctypes.c_int32)() for _ in range(6)]
        _lib.gc_sel_arrays(h, *[ctypes.byref(q) for q in ptrs])
        sizes = [2 * self.n_ubl, self.n_ubl + 1, self.P, self.P, self.n_ubl, self.n_ubl]
        arrs = [np.ctypeslib.as_array(q, shape=(n,)).copy() if n else np.zeros(0, np.int32)
                for q, n in zip(ptrs, sizes)]
        self.types = arrs[0].reshape(-1, 2)
        self.type_ptr, self.pair_i, self.pair_j, self.win_t0, self.win_t1 = arrs[1:]

    @property
    def handle(self):
        return self._h

    def pair_type(self):
        import numpy as np
        return np.repeat(np.arange(self.n_ubl, dtype=np.int32), np.diff(self.type_ptr))

    def edge_mask(self):
        """Edge antennas (gc_sel_edge): uint8 numpy [L*L], 1 on occupied
        points with a missing nearest neighbour."""
        import numpy as np
        e = np.zeros(self.L * self.L, dtype=np.uint8)
        st = _lib.gc_sel_edge(self._h, e.ctypes.data_as(_vp))
        if st != GC_OK:
            raise GridcorrError(st, "gc_sel_edge")
        return e

    def close(self):
        if getattr(self, "_h", None):
            _lib.gc_sel_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chi2Function(torch.autograd.Function):
    """chi^2 per channel as a differentiable function of the complex gains
    [C, N] and model visibilities [C, n_ubl] (complex64), with the gradient
    from the library's adjoint kernel.  checkpoint=False saves only (gains,
    vmodel) and the backward pass recomputes the residuals; checkpoint=True
    saves the per-channel residuals (8 P bytes per channel) and the backward
    pass reads them."""

    @staticmethod
    def forward(fctx, gains, vmodel, vred, sel, ctx, weights=None, checkpoint=False):
        g = gains.detach().contiguous()
        v = vmodel.detach().contiguous()
        fctx.vred, fctx.sel, fctx.gctx, fctx.weights = vred, sel, ctx, weights
        fctx.checkpoint = checkpoint
        if checkpoint:
            r = torch.empty(vred.shape[0], sel.P, dtype=torch.complex64, device=vred.device)
            out = ctx.chi2(vred, sel, g, v, weights, residuals=r)
            fctx.save_for_backward(g, v, r)
            return out
        fctx.save_for_backward(g, v)
        return ctx.chi2(vred, sel, g, v, weights)

    @staticmethod
    def backward(fctx, grad_out):
        if fctx.checkpoint:
            g, v, r = fctx.saved_tensors
            dg, dv = fctx.gctx.chi2_backward_ckpt(r, fctx.sel, g, v, grad_out, fctx.weights)
        else:
            g, v = fctx.saved_tensors
            dg, dv = fctx.gctx.chi2_backward(fctx.vred, fctx.sel, g, v, grad_out, fctx.weights)
        return dg, dv, None, None, None, None, None


def chi2(gains, vmodel, vred, sel, ctx=None, weights=None, checkpoint=False):
    ctx = ctx or default_context(gains.device)
    return Chi2Function.apply(gains, vmodel, vred, sel, ctx, weights, checkpoint)


def decode_stats(stats: torch.Tensor):
    """uint8 [C, 32] gc_calstats -> numpy structured array."""
    import numpy as np
    return stats.cpu().numpy().reshape(-1).view(np.dtype(STATS_DTYPE))


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
