#!/usr/bin/env python
"""Benchmark of the FFT-correlator system hot path on GB300.

Headline workload (one step = one integration of a 64 x 64 array):
  64 x 64 regular grid (4096 antennas), 1024 channels, 8192 time samples per
  integration, voltages from 200 point sources at SNR 10 with ~5 % gain
  amplitude scatter and random phases, quantised to 4+4-bit complex (one
  scale per channel, RMS 3 levels), 128 x 128 FFT.  One step is one cycle of
  the paper's Fig. 1 system: the FFT-correlator with the current gains
  (V^unique), the reduced X-engine over the subset selection (V^reduced,
  47250 pairs, exact int32), and the per-channel calibration (Gauss-Newton
  lincal with a matrix-free PCG step, FP32 products and FP64 reductions)
  whose gains the next step's correlator applies.  The banded FP64 and FP32
  normal-equation solvers and omnical are timed on a channel subset of the
  same V^reduced and reported with their gain difference from the FP64 one.
  The paper-scale complex64 workload (32 x 32 grid, 256 channels, 4096
  samples, 64 x 64 FFT) is measured after it as a secondary line.

Prints one JSON line (rank 0).  `value` is antenna-samples per second over
the whole job (sum over ranks / max rank time); each rank processes its own
channels (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload precision64|paper32]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FFT-corr antenna-samples/s & calibrated chans/s at 64x64 grid; % roofline"
UNIT = "antenna-samples/s"
WORKLOADS = {
    "precision64": dict(
        L=64, C=1024, T=8192, n_src=200, snr=10.0, vfmt="i4c", seed=3,
        name=("precision: 64x64 grid (4096 antennas), 1024 channels, 8192 samples, 4+4-bit voltages "
              "(per-channel scale to RMS 3 levels), 200 sources, SNR 10, 128x128 FFT")),
    "paper32": dict(
        L=32, C=256, T=4096, n_src=200, snr=10.0, vfmt="c64", seed=2,
        name=("paper-scale: 32x32 grid (1024 antennas), 256 channels, 4096 samples, complex64, "
              "200 sources, SNR 10, 64x64 FFT")),
}
ESZ = {"c64": 8, "i4c": 1}


def flops_per_antenna_sample(L: int, M: int) -> float:
    """Algorithmic FP32 flops of the pruned radix-2 FFT-correlator per
    antenna-sample: row FFTs over the L non-zero rows (first stage free),
    M column FFTs, |X|^2 accumulation (4 per bin) and the gain multiply
    (6 per antenna); 10 flops per radix-2 butterfly."""
    lg = math.log2(M)
    bfly = L * (M / 2) * (lg - 1) + M * (M / 2) * lg
    return (10.0 * bfly + 4.0 * M * M + 6.0 * L * L) / (L * L)


def lincal_flops_per_iter(N: int, n_ubl: int, P: int, bw: int) -> float:
    """FP64 flops of one Gauss-Newton iteration of the banded solver:
    band Cholesky (n bw^2), forward solve of the border and rhs
    (2 (m+1) n bw), Schur complement (m^2 n), back substitution (2 n bw),
    assembly (~150 per pair-visit, two visits per pair)."""
    n, m = 2 * N, 2 * n_ubl
    return n * bw * bw + 2.0 * (m + 1) * n * bw + m * m * n + 2.0 * n * bw + 300.0 * P


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def source_hash(*rel):
    h = hashlib.sha256()
    for r in rel:
        h.update(open(os.path.join(ROOT, r), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(key: str, src_hash: str):
    """DRAM bytes per launch from a committed ncu capture (profiles/traffic.json,
    keyed "<kernel>@<workload>"), if the kernel's source has not changed since."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = d.get(key)
        if e and e.get("source_hash") == src_hash:
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "power_w_median": statistics.median(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle arm
def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_pipeline(wl: dict, Ts: int, n_ch: int):
    """The oracle's pipeline on n_ch channels x Ts samples of the workload,
    as two timed parts: corr() = (4+4-bit: the quantiser, then the integer
    voltages) FX correlator + Eq. modelvis over the channels (the oracle's
    OpenMP loop over channels) and the X-engine over the subset selection;
    cal() = lincal of the first channel's V^reduced (dense normal equations
    up to 32 x 32, the sparse form of the same equations beyond).  corr()
    returns the threads the FX correlator ran on."""
    import numpy as np

    import oracle
    from oracle import calib as oc
    from oracle import select as osel
    from paper_2005_03060_gb300 import synth

    L = wl["L"]
    volt, gains, _ = synth.make_voltages(wl["seed"], L, n_ch, Ts, n_src=wl["n_src"], snr=wl["snr"])
    v = volt.numpy()
    g = gains.numpy()
    sel = osel.subset(L, Ts)
    pt = sel.pair_type()
    t0s, t1s = sel.win_t0[pt], sel.win_t1[pt]
    i4c = wl["vfmt"] == "i4c"
    state = {}

    def corr():
        if i4c:
            vc = np.empty(v.shape, np.complex128)
            S = []
            for c in range(n_ch):
                q, _ = oracle.quantize(v[c])
                vc[c] = oracle.unpack_i4c(q)
                s = oracle.xengine_i4c(q, sel.pair_i, sel.pair_j, t0s, t1s)
                S.append(s[:, 0] + 1j * s[:, 1])
        else:
            vc = v.astype(np.complex128)
            S = [oracle.xengine_c64(vc[c], sel.pair_i, sel.pair_j, t0s, t1s) for c in range(n_ch)]
        _, threads = oracle.fx_multi(vc, g, L)
        state["S"] = S
        return threads

    def cal():
        # subset selection: every pair's window is the whole integration
        oc.calibrate(state["S"][0] / Ts, sel.pair_i, sel.pair_j, pt, sel.types, L, "lincal", sparse=L > 32)

    return corr, cal


def _oracle_desc(wl, Ts, n_ch, threads, with_cal, why=""):
    L = wl["L"]
    quant = "4+4-bit quantiser, " if wl["vfmt"] == "i4c" else ""
    form = "sparse" if L > 32 else "dense"
    return (f"{n_ch} channels x {Ts} samples of the {L * L}-antenna workload through the FP64 oracle: "
            f"{quant}FX correlator (all N^2 pairs, Eq. modelvis; OpenMP over the channels, {threads} threads), "
            f"X-engine over the subset selection"
            + (f", lincal to 1e-10 ({form} normal equations, numpy/scipy) timed on one channel and "
               f"counted once per channel" if with_cal else f"; lincal omitted{why}"))


def _oracle_corr_samples(wl, n_ch: int, budget_s: float) -> int:
    """Samples whose correlator part over n_ch channels takes about budget_s
    (the cost grows faster than T once a channel's voltages leave the
    caches, hence the margin)."""
    corr, _ = _oracle_pipeline(wl, 16, n_ch)
    t0 = time.perf_counter()
    corr()
    t16 = max(time.perf_counter() - t0, 1e-3)
    return int(max(8, min(wl["T"], 256, 0.5 * 16 * budget_s / t16)))


def cpu_baseline(wl):
    """A bounded sample of the workload through the oracle pipeline on the
    host cores (one channel per core): the correlator part on about 10 s
    worth of samples, plus the calibration of one channel for the small
    arrays (for 4096 antennas one sparse FP64 solve of a short, noisy
    integration runs for minutes, so it is left out of the bounded sample
    and said so)."""
    n_ch = _host_cores()
    Ts = _oracle_corr_samples(wl, n_ch, 10.0)
    corr, cal = _oracle_pipeline(wl, Ts, n_ch)
    with_cal = wl["L"] <= 32
    t0 = time.perf_counter()
    threads = corr()
    t1 = time.perf_counter()
    if with_cal:
        cal()
    t2 = time.perf_counter()
    L = wl["L"]
    secs = (t1 - t0) + n_ch * (t2 - t1)
    why = " (one sparse FP64 solve of this 4096-antenna sample runs for minutes on these cores)"
    return {"value": n_ch * L * L * Ts / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": _oracle_desc(wl, Ts, n_ch, threads, with_cal, why), "seconds": round(secs, 2),
            "seconds_correlator_xengine": round(t1 - t0, 2),
            "seconds_calibration": round(n_ch * (t2 - t1), 2)}


def oracle_calibration_time(w) -> dict:
    """One channel of w's V^reduced through the FP64 oracle's Gauss-Newton
    lincal (oracle/calib.py; sparse normal equations for large arrays),
    timed once: the CPU counterpart of the GPU's calibrated channels/s."""
    import numpy as np

    from oracle import calib as oc
    from oracle import select as osel
    sel = w.sel
    osl = osel.subset(w.L, w.T)
    pt = osl.pair_type()
    tp = (osl.win_t1 - osl.win_t0)[pt].astype(np.float64)
    vr = w.vr[0].cpu().numpy()
    S = vr[..., 0].astype(np.float64) + 1j * vr[..., 1].astype(np.float64) if vr.ndim == 2 else vr.astype(np.complex128)
    t0 = time.perf_counter()
    g, _, _, ok = oc.calibrate(S / tp, osl.pair_i, osl.pair_j, pt, osl.types, w.L, "lincal", sparse=w.N > 1024)
    dt = time.perf_counter() - t0
    gg = w.gbuf[w.k % 2][0].cpu().numpy().astype(np.complex128)   # the GPU's gains of this channel
    return {"chans_per_s": 1.0 / dt, "seconds_one_channel": dt, "converged": bool(ok),
            "max_rel_gain_diff_gpu_vs_oracle": float(np.max(np.abs(gg - g) / np.abs(g))),
            "sample": (f"channel 0 of the workload's V^reduced ({sel.P} pairs, {w.N} antennas): FP64 "
                       "Gauss-Newton lincal of the oracle (scipy sparse normal equations), tolerance 1e-10")}


def run_reference(args, rank):
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    L = wl["L"]
    n_ch = _host_cores()
    budget = 150.0 / (args.steps + args.warmup)     # seconds per step
    Ts = _oracle_corr_samples(wl, n_ch, 0.5 * budget)
    corr, cal = _oracle_pipeline(wl, Ts, n_ch)
    with_cal = False
    why = " (one sparse FP64 solve of this 4096-antenna sample runs for minutes on these cores)"
    threads = corr()
    if L <= 32:
        t0 = time.perf_counter()
        cal()
        t_cal = time.perf_counter() - t0
        with_cal = t_cal <= 0.5 * budget
        why = f" (one channel's solve takes {t_cal:.1f} s, over half the {budget:.1f} s per-step budget)"

    def run():
        t0 = time.perf_counter()
        corr()
        t1 = time.perf_counter()
        if with_cal:
            cal()
        # the calibration is timed on one channel and counted once per channel
        return (t1 - t0) + n_ch * (time.perf_counter() - t1)

    desc = _oracle_desc(wl, Ts, n_ch, threads, with_cal, why) + " per step"
    for _ in range(args.warmup):
        run()
    dt = sum(run() for _ in range(args.steps)) / args.steps
    value = n_ch * L * L * Ts / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
class Workload:
    """Device buffers and the step closure of one workload on one GPU."""

    def __init__(self, wl: dict, C: int, dev, ctx, rank: int):
        import torch

        from paper_2005_03060_gb300 import gridcorr, shard, synth

        self.wl, self.C, self.dev, self.ctx = wl, C, dev, ctx
        L, T = wl["L"], wl["T"]
        N = L * L
        self.L, self.T, self.N = L, T, N
        self.M = max(16, gridcorr.fft_size(L))
        seed = shard.rank_seed(wl["seed"], rank)
        gains = synth.make_gains(seed, C, N, device=dev)
        if wl["vfmt"] == "i4c":
            volt = torch.empty(C, T, N, dtype=torch.uint8, device=dev)
            self.scales = torch.empty(C, dtype=torch.float32, device=dev)
            for c0 in range(0, C, 8):
                n = min(8, C - c0)
                v, _, _ = synth.make_voltages(seed, L, n, T, n_src=wl["n_src"], snr=wl["snr"], device=dev,
                                              gains=gains[c0:c0 + n], channel0=c0)
                ctx.quantize(v, out=volt[c0:c0 + n], scales=self.scales[c0:c0 + n])
                del v
        else:
            volt = torch.empty(C, T, N, dtype=torch.complex64, device=dev)
            synth.make_voltages(seed, L, C, T, n_src=wl["n_src"], snr=wl["snr"], device=dev, gains=gains,
                                out=volt)
        torch.cuda.synchronize(dev)
        self.volt, self.gains = volt, gains
        self.sel = gridcorr.Selection("subset", L, T)
        W = 2 * L - 1
        self.vu = torch.empty(C, W, W, dtype=torch.complex64, device=dev)
        if wl["vfmt"] == "i4c":
            self.vr = torch.empty(C, self.sel.P, 2, dtype=torch.int32, device=dev)
            self.au = torch.empty(C, N, dtype=torch.int32, device=dev)
        else:
            self.vr = torch.empty(C, self.sel.P, dtype=torch.complex64, device=dev)
            self.au = torch.empty(C, N, dtype=torch.float32, device=dev)
        self.gbuf = [gains.clone(), torch.empty_like(gains)]
        self.vmod = torch.zeros(C, self.sel.n_ubl, dtype=torch.complex64, device=dev)
        self.stats = torch.empty(C, 32, dtype=torch.uint8, device=dev)
        self.k = 0

    @property
    def g_cur(self):
        return self.gbuf[self.k % 2]

    def step(self):
        g_in, g_out = self.gbuf[self.k % 2], self.gbuf[(self.k + 1) % 2]
        self.ctx.correlate(self.volt, g_in, self.L, out=self.vu)
        self.ctx.reduce(self.volt, self.sel, out=self.vr, out_autos=self.au)
        self.ctx.calibrate(self.vr, self.sel, self.au, solver="lincal_cg", precision="fp32", gains=g_out,
                           vmodel=self.vmod, stats=self.stats)
        self.k += 1

    @property
    def units(self):
        return self.N * self.C * self.T


def _timed(step, steps, stream, barrier):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1)


def rooflines(w: Workload, kern: dict, st_last, peaks: dict, probes: dict):
    import numpy as np
    L, N, C, T, M, sel = w.L, w.N, w.C, w.T, w.M, w.sel
    esz = ESZ[w.wl["vfmt"]]
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    key = "@" + [k for k, v in WORKLOADS.items() if v is w.wl][0]
    rl = {}
    if "fftcorr_accumulate" in kern:
        ms, n = kern["fftcorr_accumulate"]
        dur = ms / n * 1e-3
        flops = flops_per_antenna_sample(L, M) * N * C * T
        by = float(esz) * N * C * T
        rl["fftcorr_accumulate"] = {
            "bound": "alu", "achieved": flops / dur / 1e12, "peak": probes["fp32"], "unit": "TFLOP/s",
            "frac": flops / dur / 1e12 / probes["fp32"],
            "traffic": recorded_traffic("fftcorr_accumulate" + key,
                                        source_hash("paper_2005_03060_gb300/csrc/gc_fftcorr.cu")),
            "algorithmic_flops": flops, "algorithmic_bytes": by,
            "per_unit": f"{flops_per_antenna_sample(L, M):.1f} FP32 flops and {esz} B per antenna-sample",
            "peak_source": "measured: gc_peak_probe FP32 FMA on this GPU",
            "hbm": {"achieved": by / dur / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": by / dur / 1e9 / hbm_peak}}
    if "fftcorr_tc_accumulate" in kern:
        ms, n = kern["fftcorr_tc_accumulate"]
        dur = ms / n * 1e-3
        units = N * C * T
        by = float(esz) * units
        # column stage on the CUDA cores: the M column FFTs (radix-2 count),
        # |X|^2 (4 per bin) and the gain multiply (6 per antenna)
        lg = math.log2(M)
        col = (10.0 * M * (M / 2) * lg + 4.0 * M * M + 6.0 * N) / N
        col_flops = col * units
        # row stage on the tensor cores: per sample 3 split terms x (8 Re +
        # 8 Im K-steps) of 128 x 64 x 16 binary16 MMAs
        mma = float(C) * T * 48 * 2.0 * 128 * 64 * 16
        tc_peak = peaks.get("bf16_tflops") or 1900.0
        fft_equiv = flops_per_antenna_sample(L, M) * units
        rl["fftcorr_tc_accumulate"] = {
            "bound": "alu", "achieved": col_flops / dur / 1e12, "peak": probes["fp32"], "unit": "TFLOP/s",
            "frac": col_flops / dur / 1e12 / probes["fp32"],
            "traffic": recorded_traffic("fftcorr_tc_accumulate" + key,
                                        source_hash("paper_2005_03060_gb300/csrc/gc_fftcorr_tc.cu")),
            "algorithmic_flops": col_flops, "algorithmic_bytes": by,
            "per_unit": (f"{col:.1f} FP32 flops (column stage) and {esz} B per antenna-sample on the CUDA "
                         f"cores; {48 * 2.0 * 128 * 64 * 16 / N:.0f} binary16 MMA flops per antenna-sample "
                         "(row stage) on the tensor cores"),
            "peak_source": "measured: gc_peak_probe FP32 FMA on this GPU",
            "tensor": {"achieved": mma / dur / 1e12, "peak": tc_peak, "unit": "TFLOP/s (f16 MMA executed)",
                       "frac": mma / dur / 1e12 / tc_peak, "executed_flops": mma,
                       "peak_source": ("measured: MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16 burst; f16 "
                                       "runs at the bf16 rate)" if peaks.get("bf16_tflops") else
                                       "fallback 1.9 PFLOP/s")},
            "radix2_equivalent": {"achieved": fft_equiv / dur / 1e12, "unit": "TFLOP/s",
                                  "per_unit": f"{flops_per_antenna_sample(L, M):.1f} flops per antenna-sample "
                                              "(the CUDA-core kernel's whole-FFT count)",
                                  "frac_of_fp32_peak": fft_equiv / dur / 1e12 / probes["fp32"]},
            "hbm": {"achieved": by / dur / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": by / dur / 1e9 / hbm_peak}}
    if "xeng_accumulate" in kern:
        ms, n = kern["xeng_accumulate"]
        dur = ms / n * 1e-3
        by = float(esz) * N * C * T
        ops = 8.0 * sel.P * C * T          # complex multiply-accumulate = 8 ops per pair-sample
        traffic = recorded_traffic("xeng_accumulate" + key,
                                   source_hash("paper_2005_03060_gb300/csrc/gc_xengine.cu"))
        hbm = {"achieved": by / dur / 1e9, "peak": hbm_peak, "unit": "GB/s", "frac": by / dur / 1e9 / hbm_peak}
        if w.wl["vfmt"] == "i4c":
            rl["xeng_accumulate"] = {
                "bound": "alu", "achieved": ops / dur / 1e12, "peak": probes["dp4a"], "unit": "TOPS (int8 dp4a)",
                "frac": ops / dur / 1e12 / probes["dp4a"], "traffic": traffic, "algorithmic_ops": ops,
                "algorithmic_bytes": by, "per_unit": f"{8.0 * sel.P / N:.1f} int ops and 1 B per antenna-sample",
                "peak_source": "measured: gc_peak_probe dp4a on this GPU", "hbm": hbm}
        else:
            rl["xeng_accumulate"] = {
                "bound": "hbm", **hbm, "traffic": traffic, "algorithmic_bytes": by, "useful_flops": ops,
                "per_unit": "8 B per antenna-sample", "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    if "xeng_tc_accumulate" in kern:
        ms, n = kern["xeng_tc_accumulate"]
        dur = ms / n * 1e-3
        by = float(esz) * N * C * T
        ops = 8.0 * sel.P * C * T          # useful: 8 integer ops per pair-sample
        # executed: per 32-sample stage of each 128-antenna block, four dense
        # e4m3 MMAs of 128 x 256 x 32 (D1 = RE.RE + IM.IM, D2 = IM.RE - RE.IM)
        stages = C * (N // 128) * math.ceil(T / 32)
        mma = stages * 4 * 2.0 * 128 * 256 * 32
        rl["xeng_tc_accumulate"] = {
            "bound": "tensor", "achieved": mma / dur / 1e12, "peak": probes["tc_f8"],
            "unit": "TFLOP/s (e4m3 MMA executed)", "frac": mma / dur / 1e12 / probes["tc_f8"],
            "traffic": recorded_traffic("xeng_tc_accumulate" + key,
                                        source_hash("paper_2005_03060_gb300/csrc/gc_xengine_tc.cu")),
            "executed_flops": mma, "useful_ops": ops, "useful_fraction": ops / mma,
            "useful_tops": ops / dur / 1e12, "algorithmic_bytes": by,
            "per_unit": (f"1 B and {8.0 * sel.P / N:.1f} useful integer ops per antenna-sample; "
                         f"{4 * 2.0 * 128 * 256 * 32 / (128 * 32):.0f} executed MMA flops per antenna-sample "
                         "(128 own antennas x 256-antenna halo per 32-sample stage)"),
            "peak_source": "measured: gc_peak_probe dense e4m3 tcgen05 MMA on this GPU",
            "hbm": {"achieved": by / dur / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": by / dur / 1e9 / hbm_peak}}
    if "lincal_cg" in kern:
        ms, n = kern["lincal_cg"]
        dur = ms / n * 1e-3
        cg_it = float(np.sum(st_last["inner"]))
        gn_it = float(np.sum(st_last["iters"]))
        ne = N + sel.n_ubl
        # algorithmic FP32 flops of the matrix-free Gauss-Newton in relative
        # coordinates (each pair once, in its cheapest form): per CG iteration
        # the operator (s_p = q_i + conj(q_j) + w_k, weight |m_p|^2, three row
        # updates: ~14 per pair) and the vector updates (~20 per complex
        # unknown); per Gauss-Newton iteration the residual pass (model,
        # residual, right-hand side, diagonal: ~50 per pair), the projection,
        # line search and update (~60 per unknown)
        flops = cg_it * (14.0 * sel.P + 20.0 * ne) + gn_it * (50.0 * sel.P + 60.0 * ne)
        rl["lincal_cg"] = {"bound": "alu", "achieved": flops / dur / 1e12, "peak": probes["fp32"],
                           "unit": "TFLOP/s", "frac": flops / dur / 1e12 / probes["fp32"], "traffic": None,
                           "algorithmic_flops": flops, "cg_iterations": cg_it, "gn_iterations": gn_it,
                           "chans_per_s": C / dur,
                           "note": ("one 256-thread CTA per channel, two per SM, channels taken from a device "
                                    "counter; each pair is evaluated by both of its antennas (no atomics); "
                                    "bound by latency (L2-resident CG vectors) and block barriers"),
                           "peak_source": "measured: gc_peak_probe FP32 FMA on this GPU"}
    return rl


def tune_workload(ctx, w) -> dict:
    """Run the project's autotuner (paper_2005_03060_gb300/autotune.py) over
    the correlator and X-engine knobs of workload w; returns the choices and
    the timings behind them."""
    from paper_2005_03060_gb300 import autotune
    out = {"correlator": autotune.tune_correlator(ctx, w.volt, w.gains, w.L, reps=1)}
    out["xengine"] = autotune.tune_xengine(ctx, w.volt, w.sel, reps=1)
    return out


def calibration_variants(w: Workload, Cs: int, reps_fast: int):
    """The other solvers on the first Cs channels of the same V^reduced,
    compared with the banded FP64 solve (gain difference after the output
    convention, which every solver applies)."""
    import numpy as np
    import torch

    from paper_2005_03060_gb300 import gridcorr
    ctx, sel = w.ctx, w.sel
    vr, au = w.vr[:Cs].contiguous(), w.au[:Cs].contiguous()
    out, g64 = {}, None
    # op: the matrix-free operator ("cal.operator": 0 gather over the grid, 1 pair-list scatter)
    # lincal_cg_plain_fp32: the same matrix-free solver with every reduction
    # in FP32 (the like-for-like plain-FP32 form of the mixed one)
    for name, solver, prec, allc, op, r32 in [("lincal_fp64", "lincal", "fp64", False, 0, False),
                                              ("lincal_fp32", "lincal", "fp32", False, 0, False),
                                              ("omnical_fp32", "omnical", "fp32", False, 0, False),
                                              ("lincal_cg_mixed", "lincal_cg", "fp32", True, 0, False),
                                              ("lincal_cg_plain_fp32", "lincal_cg", "fp32", True, 0, True),
                                              ("lincal_cg_mixed_pair_scatter", "lincal_cg", "fp32", True, 1, False)]:
        ctx.set_tuning("cal.operator", op)
        v_in, a_in = (w.vr, w.au) if allc else (vr, au)
        Cn = w.C if allc else Cs
        reps = reps_fast if allc else 1
        g, V, st = ctx.calibrate(v_in, sel, a_in, solver=solver, precision=prec, fp32_reductions=r32)
        torch.cuda.synchronize(w.dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            ctx.calibrate(v_in, sel, a_in, solver=solver, precision=prec, gains=g, vmodel=V, stats=st,
                          fp32_reductions=r32)
        b.record()
        torch.cuda.synchronize(w.dev)
        ms = a.elapsed_time(b) / reps
        sv = gridcorr.decode_stats(st)
        if g64 is None:
            g64 = g[:Cs].clone()
        diff = ((g[:Cs] - g64).abs() / g64.abs()).max().item()
        out[name] = {"ms": ms, "channels": Cn, "chans_per_s": Cn / (ms * 1e-3),
                     "max_rel_gain_diff_vs_lincal_fp64": diff,
                     "mean_iters": float(np.mean(sv["iters"])), "mean_cg_iters": float(np.mean(sv["inner"])),
                     "converged": int(np.sum(sv["status"] == 0))}
    ctx.set_tuning("cal.operator", 0)
    return out


# ----------------------------------------------------------------------------- batching and differentiation forms
BATCH_GRIDS = (8, 12, 16, 24, 32, 40, 48, 64, 80, 96, 112, 128)
BATCH_T = 2048
DIFF_L, DIFF_C, DIFF_T = 128, 512, 4096


def _batch_channels():
    """Channels per array of the batching form, drawn U{64..512} (seeded)."""
    import numpy as np
    return [int(c) for c in np.random.default_rng(2048).integers(64, 513, size=len(BATCH_GRIDS))]


def _forms_timed(fn, stream, reps):
    """Mean CUDA-event time of fn on `stream` after one untimed call."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_batching(ctx, dev, stream):
    """Batching form: twelve square arrays of 8x8 .. 128x128 with U{64..512}
    channels each (T = 2048, subset selections), calibrated by the
    matrix-free lincal in one persistent gc_calibrate_batched launch, against
    one gc_calibrate launch per array.  V^reduced comes from the paper's own
    visibility-level simulation (Sec. 3) at SNR 10 per sample."""
    import numpy as np
    import torch

    from paper_2005_03060_gb300 import gridcorr, synth

    chans = _batch_channels()
    arrays, per = [], []
    for k, (L, C) in enumerate(zip(BATCH_GRIDS, chans)):
        sel = gridcorr.Selection("subset", L, BATCH_T)
        pt = sel.pair_type()
        tp = (sel.win_t1 - sel.win_t0)[pt]
        sums, _, _ = synth.make_visibilities(300 + k, L, C, sel.pair_i, sel.pair_j, pt, sel.n_ubl, tp,
                                             snr=10.0, device=dev)
        arrays.append({"vred": sums.contiguous(), "sel": sel})
        per.append((torch.empty(C, L * L, dtype=torch.complex64, device=dev),
                    torch.empty(C, sel.n_ubl, dtype=torch.complex64, device=dev),
                    torch.empty(C, 32, dtype=torch.uint8, device=dev)))

    def one_launch_per_array():
        for a, (g, v, st) in zip(arrays, per):
            ctx.calibrate(a["vred"], a["sel"], solver="lincal_cg", precision="fp32", gains=g, vmodel=v, stats=st)

    from paper_2005_03060_gb300 import autotune
    tuned = autotune.tune_calibration(ctx, arrays, reps=1)   # "cal.order", "cal.ctas_per_sm"
    ms_per = _forms_timed(one_launch_per_array, stream, 3)
    for a, (g, v, st) in zip(arrays, ctx.calibrate_batched(arrays)):
        a["gains"], a["vmodel"], a["stats"] = g, v, st
    ms_b = _forms_timed(lambda: ctx.calibrate_batched(arrays), stream, 3)
    ctx.device_status()
    # the same persistent launch captured once into a CUDA graph and replayed
    torch.cuda.synchronize()
    side = torch.cuda.Stream(device=stream.device)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        ctx.calibrate_batched(arrays)
    graph.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps_g = 3
    # replay() launches on the current stream: time it there
    e0.record(stream)
    for _ in range(reps_g):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_g = e0.elapsed_time(e1) / reps_g
    ctx.device_status()
    ok = all(bool(np.all(gridcorr.decode_stats(a["stats"])["status"] == 0)) for a in arrays)
    diff = max(((a["gains"] - g).abs() / g.abs()).max().item() for a, (g, _, _) in zip(arrays, per))
    total = sum(chans)
    return {"arrays": [[L, C] for L, C in zip(BATCH_GRIDS, chans)], "channels": total,
            "antennas": sum(L * L for L in BATCH_GRIDS), "T": BATCH_T,
            "batched_ms": ms_b, "batched_chans_per_s": total / (ms_b * 1e-3),
            "per_array_ms": ms_per, "per_array_chans_per_s": total / (ms_per * 1e-3),
            "graph_ms": ms_g, "graph_chans_per_s": total / (ms_g * 1e-3),
            "autotuned": {k: {"knob": v["knob"], "best": v["best"], "ms": v["ms"]} for k, v in tuned.items()},
            "all_converged": ok, "max_gain_diff_batched_vs_per_array": diff,
            "l2": f"V^reduced of all arrays {sum(a['vred'].numel() * 8 for a in arrays) / 1e9:.2f} GB, larger than L2",
            "input": "V^reduced from the paper's visibility-level simulation (Sec. 3), SNR 10 per sample; "
                     "subset selections (p = 1, log2); batched_ms: eager launch, graph_ms: the same "
                     "launch captured in a CUDA graph and replayed; knobs from the autotuner"}


def measure_differentiation(ctx, dev, stream, hbm_peak, channels=None):
    """Differentiation form: the chi^2 of the redundant model (numerator of
    Eq. redchi) and its adjoint on the 128x128 array (16 384 antennas, 512
    channels, T = 4096, subset selection), residuals recomputed in the
    backward pass or checkpointed by the forward pass.  Exact int32 pair sums
    (the visibility-level simulation rounded to integers) stand where the
    X-engine output of 4+4-bit voltages would; the evaluation point is the
    true gains and visibilities.  chi^2 is bandwidth-bound: algorithmic bytes
    are 8 per pair per pass over V^reduced or the residuals, plus the gains
    and model visibilities once."""
    import torch

    from paper_2005_03060_gb300 import gridcorr, synth

    L, C, T = DIFF_L, channels or DIFF_C, DIFF_T
    sel = gridcorr.Selection("subset", L, T)
    pt = sel.pair_type()
    tp = (sel.win_t1 - sel.win_t0)[pt]
    sums, g, v = synth.make_visibilities(500, L, C, sel.pair_i, sel.pair_j, pt, sel.n_ubl, tp,
                                         snr=10.0, device=dev)
    vr = torch.stack([sums.real.round(), sums.imag.round()], dim=-1).to(torch.int32).contiguous()
    del sums
    g, v = g.contiguous(), v.contiguous()
    res = torch.empty(C, sel.P, dtype=torch.complex64, device=dev)
    out = torch.empty(C, dtype=torch.float64, device=dev)
    ms = {"chi2_fwd": _forms_timed(lambda: ctx.chi2(vr, sel, g, v, out=out), stream, 5),
          "chi2_bwd": _forms_timed(lambda: ctx.chi2_backward(vr, sel, g, v), stream, 5),
          "chi2_fwd_ckpt": _forms_timed(lambda: ctx.chi2(vr, sel, g, v, out=out, residuals=res), stream, 5),
          "chi2_bwd_ckpt": _forms_timed(lambda: ctx.chi2_backward_ckpt(res, sel, g, v), stream, 5)}
    ctx.device_status()
    pairs = C * sel.P * 8
    par = C * (L * L + sel.n_ubl) * 8
    algo = {"chi2_fwd": pairs + par, "chi2_bwd": pairs + 2 * par,
            "chi2_fwd_ckpt": 2 * pairs + par, "chi2_bwd_ckpt": pairs + 2 * par}
    kern = {}
    for k, t in ms.items():
        gbs = algo[k] / (t * 1e6)
        kern[k] = {"ms": t, "algorithmic_bytes": algo[k], "gb_s": gbs, "hbm_frac": gbs / hbm_peak}
    return {"L": L, "antennas": L * L, "channels": C, "pairs": sel.P, "kernels": kern,
            "fwd_bwd_chans_per_s": C / ((ms["chi2_fwd"] + ms["chi2_bwd"]) * 1e-3),
            "hbm_peak_gbs": hbm_peak,
            "l2": f"V^reduced {vr.numel() * 4 / 1e9:.2f} GB, larger than L2",
            "input": "int32 pair sums rounded from the paper's visibility-level simulation (Sec. 3), SNR 10 "
                     "per sample; evaluation at the true gains and visibilities"}


def measure_forms(ctx, dev, stream, hbm_peak, diff_channels=None):
    """Both forms; a failure is recorded in the result instead of ending the run."""
    import torch
    out = {}
    for name, fn in (("batching", lambda: measure_batching(ctx, dev, stream)),
                     ("differentiation", lambda: measure_differentiation(ctx, dev, stream, hbm_peak,
                                                                         diff_channels))):
        try:
            out[name] = fn()
        except Exception as e:                      # noqa: BLE001 -- reported, not hidden
            out[name] = {"error": f"{type(e).__name__}: {e}"[:400]}
        torch.cuda.empty_cache()
    return out


def cpu_forms_baseline():
    """The oracle on one channel of each form (context only): the chi^2 and
    its gradient at 16 384 antennas, and one FP64 lincal of a 16x16 array of
    the batching form."""
    import numpy as np

    from oracle import calib as oc
    from oracle import select as osel
    from paper_2005_03060_gb300 import synth

    out = {}
    sel = osel.subset(DIFF_L, DIFF_T)
    pt = sel.pair_type()
    tp = (sel.win_t1 - sel.win_t0)[pt]
    sums, g, v = synth.make_visibilities(500, DIFF_L, 1, sel.pair_i, sel.pair_j, pt, sel.n_ubl, tp, snr=10.0)
    vobs = sums[0].numpy().astype(np.complex128) / tp
    gg, vv = g[0].numpy().astype(np.complex128), v[0].numpy().astype(np.complex128)
    t0 = time.perf_counter()
    oc.chi2(vobs, gg, vv, sel.pair_i, sel.pair_j, pt)
    oc.chi2_grad(vobs, gg, vv, sel.pair_i, sel.pair_j, pt)
    dt = time.perf_counter() - t0
    out["differentiation"] = {"value": 1.0 / dt, "unit": "channels/s", "cores": 1, "kind": "oracle",
                              "sample": f"chi^2 and its gradient (numpy, FP64) of one channel of the "
                                        f"{DIFF_L}x{DIFF_L} array ({sel.P} pairs)"}
    L = 16
    sel = osel.subset(L, BATCH_T)
    pt = sel.pair_type()
    tp = (sel.win_t1 - sel.win_t0)[pt]
    sums, _, _ = synth.make_visibilities(302, L, 1, sel.pair_i, sel.pair_j, pt, sel.n_ubl, tp, snr=10.0)
    vobs = sums[0].numpy().astype(np.complex128) / tp
    t0 = time.perf_counter()
    oc.calibrate(vobs, sel.pair_i, sel.pair_j, pt, sel.types, L, "lincal")
    dt = time.perf_counter() - t0
    out["batching"] = {"value": 1.0 / dt, "unit": "channels/s", "cores": _host_cores(), "kind": "oracle",
                       "sample": f"one FP64 lincal (dense normal equations, numpy; its BLAS may use every "
                                 f"core) of one channel of the {L}x{L} array of the batching form"}
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2005_03060_gb300 import gridcorr, shard

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]
    C = args.channels or wl["C"]
    ctx = gridcorr.Context(local_rank)
    w = Workload(wl, C, dev, ctx, rank)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # launch shapes from the autotuner, on this workload's own data (knobs
    # only change how the work is split, never the arithmetic's definition)
    autotuned = None if args.no_autotune else tune_workload(ctx, w)
    for _ in range(args.warmup):
        w.step()
    ctx.device_status()

    props = torch.cuda.get_device_properties(dev)
    pci = getattr(props, "pci_bus_id", None)
    sampler = ClockSampler(f"{pci}" if pci else str(local_rank))
    ctx.profile(True)
    ctx.profile_read()
    barrier()
    sampler.start()
    time.sleep(0.3)
    ms_total = _timed(w.step, args.steps, stream, barrier)
    clocks = sampler.stop()
    kern = ctx.profile_read()
    ctx.profile(False)
    ctx.device_status()
    st_last = gridcorr.decode_stats(w.stats)
    ms_step = shard.max_over_ranks(ms_total, dev) / args.steps
    value = shard.job_rate(w.units, world, ms_step)

    # ---- calibration variants on the same V^reduced (equal-error comparison)
    variants = calibration_variants(w, min(C, 16 if wl["L"] > 32 else C), max(1, min(5, args.steps // 4)))
    # the oracle's calibration of one channel of this workload's own
    # V^reduced (the full integration the GPU calibrates), timed once for
    # the CPU baseline
    cal_cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            cal_cpu = oracle_calibration_time(w)
        except Exception as e:                          # noqa: BLE001 -- reported, not hidden
            cal_cpu = {"error": f"{type(e).__name__}: {e}"[:400]}

    # ---- end to end through the public API with host buffers (pinned): the
    # voltages stream from host memory chunk by chunk (gc_integrate_host),
    # the copies overlapping the kernels; gains in, V^unique and gains out
    h_volt = torch.empty(w.volt.shape, dtype=w.volt.dtype, pin_memory=True)
    h_volt.copy_(w.volt)
    h_gains = torch.empty(w.gains.shape, dtype=w.gains.dtype, pin_memory=True)
    h_gains.copy_(w.gains)
    h_vu = torch.empty(w.vu.shape, dtype=w.vu.dtype, pin_memory=True)
    h_g = torch.empty(w.gains.shape, dtype=w.gains.dtype, pin_memory=True)
    e2e_steps = max(3, min(args.steps, 5))

    def e2e_step():
        # the gains go in from pinned host memory: the library copies them on
        # its copy stream ahead of the voltage chunks
        g_out = w.gbuf[(w.k + 1) % 2]
        ctx.integrate_host(h_volt, w.sel, h_gains, w.vu, w.vr, w.au, g_out, w.vmod, w.stats)
        w.k += 1
        h_vu.copy_(w.vu, non_blocking=True)
        h_g.copy_(g_out, non_blocking=True)

    for _ in range(2):
        e2e_step()
    # this box's pinned host-to-device rate (one plain copy of the voltages):
    # the streamed step cannot beat bytes / rate however well it overlaps
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    w.volt.copy_(h_volt, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    link_gbs = h_volt.numel() * h_volt.element_size() / (e0.elapsed_time(e1) * 1e6)
    ctx.profile(True)
    ctx.profile_read()
    e2e_ms = _timed(e2e_step, e2e_steps, stream, barrier) / e2e_steps
    e2e_kern = ctx.profile_read()
    ctx.profile(False)
    e2e_ms = shard.max_over_ranks(e2e_ms, dev)
    chunk_copy = e2e_kern.get("h2d_chunk", (0.0, 0))
    e2e = {"value": shard.job_rate(w.units, world, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": h_volt.numel() * h_volt.element_size() + h_gains.numel() * 8,
           "d2h_bytes_per_step": h_vu.numel() * 8 + h_g.numel() * 8,
           "h2d_link_gbs": link_gbs,
           "link_floor_ms": h_volt.numel() * h_volt.element_size() / (link_gbs * 1e6),
           "h2d_chunk_copies": {"count_per_step": chunk_copy[1] / e2e_steps,
                                "ms_per_step": chunk_copy[0] / e2e_steps,
                                "note": "sum of the chunk copies' own durations (events on the copy stream)"},
           "path": ("gc_integrate_host: pinned host voltages streamed in channel chunks through three "
                    "staging buffers, copies up to two chunks ahead of the kernels; pinned host gains "
                    "copied by the library on its copy stream; V^unique and gains D2H")}
    del h_volt

    peaks = load_peaks() or {}
    probes = {k: ctx.peak_probe(k) for k in ("fp32", "fp64", "dp4a", "tc_f8", "mma_s8")}
    rl = rooflines(w, kern, st_last, peaks, probes)
    if "lincal_fp64" in variants:
        v64 = variants["lincal_fp64"]
        D = max(abs(int(dy) * w.L + int(dx)) for dx, dy in w.sel.types.tolist())
        flops = v64["channels"] * v64["mean_iters"] * lincal_flops_per_iter(w.N, w.sel.n_ubl, w.sel.P, 2 * D + 1)
        v64["fp64_frac"] = flops / (v64["ms"] * 1e-3) / 1e12 / probes["fp64"]
    dom = max(kern.items(), key=lambda kv: kv[1][0])[0]
    roofline = dict(rl.get(dom, {"bound": "unknown"}))
    roofline["kernel"] = dom
    launches = sum(n for _, n in kern.values())
    units_note = (f"inputs ({ESZ[wl['vfmt']] * w.units / 1e9:.1f} GB per GPU) larger than L2; no flush needed")
    sel_desc = f"subset p=1 log2: {w.sel.P} pairs, {w.sel.n_ubl} types"

    # ---- secondary workload (context): the paper-scale complex64 array
    secondary = None
    if not args.no_secondary and world == 1 and args.workload != "paper32" and args.channels is None:
        del w
        torch.cuda.empty_cache()
        w2 = Workload(WORKLOADS["paper32"], WORKLOADS["paper32"]["C"], dev, ctx, rank)
        tuned2 = tune_workload(ctx, w2)
        for _ in range(3):
            w2.step()
        ctx.profile(True)
        ctx.profile_read()
        steps2 = max(5, min(args.steps, 20))
        ms2 = _timed(w2.step, steps2, stream, barrier) / steps2
        kern2 = ctx.profile_read()
        ctx.profile(False)
        ctx.device_status()
        st2 = gridcorr.decode_stats(w2.stats)
        rl2 = rooflines(w2, kern2, st2, peaks, probes)
        secondary = {"workload": WORKLOADS["paper32"]["name"], "value": w2.units / (ms2 * 1e-3), "unit": UNIT,
                     "ms_per_step": ms2, "steps": steps2, "calibrated_chans_per_s": w2.C / (ms2 * 1e-3),
                     "kernels": {k: {"ms_per_step": v[0] / steps2, "launches": v[1]} for k, v in kern2.items()},
                     "rooflines": rl2, "autotuned": tuned2}
    forms = None
    if not args.no_forms and world == 1 and args.channels is None:
        forms = measure_forms(ctx, dev, stream, peaks.get("hbm_gbs", 6800.0))
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("i4c (exact X-engine; FFT row stage f16x3 tensor MMA with FP32 accumulation, column "
                      "stage FP32; FP32 solver)") if wl["vfmt"] == "i4c" else "c64",
            "data": "synthetic",
            "calibrated_chans_per_s": C * world / (ms_step * 1e-3),
            "config": {"workload": wl["name"] if C == wl["C"] else
                       f"profiling case: {C} channels of the {args.workload} workload",
                       "L": wl["L"], "channels_per_gpu": C, "T": wl["T"], "fft": max(16, gridcorr.fft_size(wl["L"])),
                       "selection": sel_desc,
                       "calibration": "lincal (Gauss-Newton, matrix-free PCG step, FP32 products, FP64 "
                                      "reductions), step tol 1e-6",
                       "l2": units_note,
                       "parallelism": f"channels split over {world} GPU(s), no collective"},
            "roofline": roofline, "rooflines": rl,
            "kernels": {k: {"ms_per_step": v[0] / args.steps, "launches": v[1]} for k, v in kern.items()},
            "calibration_variants": variants,
            "autotuned": autotuned,
            "measured_peaks": {"fp32_tflops": probes["fp32"], "fp64_tflops": probes["fp64"],
                               "dp4a_tops": probes["dp4a"], "tc_f8_tflops": probes["tc_f8"],
                               "mma_sync_s8_tops": probes["mma_s8"]},
            "gpu_launches": launches,
            "e2e": e2e, "clocks": clocks}
    if secondary:
        line["secondary"] = secondary
    if forms:
        line["forms"] = forms
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
        line["cpu_baseline"]["calibration"] = cal_cpu
        if forms:
            try:
                line["cpu_baseline"]["forms"] = cpu_forms_baseline()
            except Exception as e:                  # noqa: BLE001 -- reported, not hidden
                line["cpu_baseline"]["forms"] = {"error": f"{type(e).__name__}: {e}"[:400]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="precision64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batching and differentiation forms (timed after the cycle)")
    ap.add_argument("--channels", type=int, default=None,
                    help="channels per GPU (default: the workload's); smaller values are for "
                         "profiling captures only")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (for profiling captures of them)")
    ap.add_argument("--only-forms", action="store_true",
                    help="time only the batching and differentiation forms (the differentiation form "
                         "with --channels channels when given); for profiling captures")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.only_forms:
        import torch
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        from paper_2005_03060_gb300 import gridcorr
        ctx = gridcorr.Context(local_rank)
        peaks = load_peaks() or {}
        print(json.dumps(measure_forms(ctx, dev, torch.cuda.current_stream(dev), peaks.get("hbm_gbs", 6800.0),
                                       args.channels)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
