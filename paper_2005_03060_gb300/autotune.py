"""Autotuner for the launch shapes of the hot path.

Times the candidate values of each tuning knob of a context (see
gc_set_tuning in include/gridcorr.h) on the caller's own data with CUDA
events, keeps the fastest, and sets it on the context.  Knobs only change
how work is split into launches and items, never the arithmetic, so every
candidate computes the same result (the FFT chunking changes the order of
the FP32 time sums; the tests bound that).
"""
from __future__ import annotations

import torch


def _time(fn, reps: int = 3) -> float:
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _sweep(ctx, knob: str, values, fn, reps: int) -> dict:
    timings = {}
    for v in values:
        ctx.set_tuning(knob, v)
        timings[v] = _time(fn, reps)
    best = min(timings, key=timings.get)
    ctx.set_tuning(knob, best)
    return {"knob": knob, "best": best, "ms": timings}


def tune_correlator(ctx, volt, gains, L=None, reps: int = 3) -> dict:
    """FFT-correlator: the path ("fft.path": row stage on the tensor cores
    or all on the CUDA cores, where both exist), the launch shape of the
    CUDA-core kernel ("fft.shape": sample grouping of the CTA; the
    tensor-core kernel ignores it), then the time-chunk length of a work item
    ("fft.chunk_len")."""
    L = L or int(round(volt.shape[2] ** 0.5))
    out = torch.empty(volt.shape[0], 2 * L - 1, 2 * L - 1, dtype=torch.complex64, device=volt.device)
    fn = lambda: ctx.correlate(volt, gains, L, out=out)   # noqa: E731
    path = _sweep(ctx, "fft.path", [0, 1], fn, reps)
    shape = _sweep(ctx, "fft.shape", [0, 1], fn, reps)
    chunk = _sweep(ctx, "fft.chunk_len", [0, 256, 512, 1024, 2048], fn, reps)
    return {"knob": "fft.path, fft.shape, fft.chunk_len", "best": [path["best"], shape["best"], chunk["best"]],
            "ms": {"fft.path": path["ms"], "fft.shape": shape["ms"], "fft.chunk_len": chunk["ms"]}}


def tune_xengine(ctx, volt, sel, reps: int = 3) -> dict:
    """Reduced X-engine: the tensor-core launch shape ("xeng.tc_shape",
    converter warps and ring depths; ignored by the SIMT path), then the time
    slices of a window ("xeng.tsplit")."""
    vr, au = ctx.reduce(volt, sel)
    fn = lambda: ctx.reduce(volt, sel, out=vr, out_autos=au)   # noqa: E731
    shape = _sweep(ctx, "xeng.tc_shape", [0, 1, 2, 4], fn, reps)
    ts = _sweep(ctx, "xeng.tsplit", [0, 1, 2, 4, 8], fn, reps)
    return {"knob": "xeng.tc_shape, xeng.tsplit", "best": [shape["best"], ts["best"]],
            "ms": {"xeng.tc_shape": shape["ms"], "xeng.tsplit": ts["ms"]}}


def tune_calibration(ctx, arrays, reps: int = 2) -> dict:
    """arrays: as for Context.calibrate_batched (outputs are reused)."""
    outs = ctx.calibrate_batched(arrays)
    for a, (g, v, s) in zip(arrays, outs):
        a.setdefault("gains", g)
        a.setdefault("vmodel", v)
        a.setdefault("stats", s)
    res = {"order": _sweep(ctx, "cal.order", [0, 1], lambda: ctx.calibrate_batched(arrays), reps)}
    res["ctas"] = _sweep(ctx, "cal.ctas_per_sm", [0, 1, 2, 3],
                         lambda: ctx.calibrate_batched(arrays), reps)
    return res
