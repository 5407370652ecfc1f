#!/usr/bin/env python
"""Benchmark of the FFT-correlator system hot path on GB300.

Workload (one step = one integration of the paper-scale array):
  32 x 32 regular grid (1024 antennas), 256 channels, 4096 time samples per
  integration, complex64 voltages from 200 point sources at SNR 10 with
  ~5 % gain-amplitude scatter and random phases, 64 x 64 FFT.
  One step is one cycle of the paper's Fig. 1 system: the FFT-correlator
  with the current gains (V^unique), the reduced X-engine over the subset
  selection (V^reduced, 10446 pairs), and the per-channel calibration
  (Gauss-Newton lincal, matrix-free CG step, FP32 products with FP64
  reductions) whose gains the next step's correlator applies.  The banded
  FP64 and FP32 normal-equation solvers and omnical are timed on the same
  V^reduced and reported with their gain difference.

Prints one JSON line (rank 0).  `value` is antenna-samples per second over
the whole job (sum over ranks / max rank time); each rank processes its own
channels (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
WORKLOAD = dict(L=32, C=256, T=4096, n_src=200, snr=10.0, vfmt="c64")
WORKLOAD_NAME = ("paper-scale: 32x32 grid (1024 antennas), 256 channels, 4096 samples, "
                 "complex64, 200 sources, SNR 10, 64x64 FFT")


def flops_per_antenna_sample(L: int, M: int) -> float:
    """Algorithmic FP32 flops of the pruned radix-2 FFT-correlator per
    antenna-sample: row FFTs over the L non-zero rows (first stage free),
    M column FFTs, |X|^2 accumulation (4 per bin) and the gain multiply
    (6 per antenna); 10 flops per radix-2 butterfly."""
    lg = math.log2(M)
    bfly = L * (M / 2) * (lg - 1) + M * (M / 2) * lg
    return (10.0 * bfly + 4.0 * M * M + 6.0 * L * L) / (L * L)


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


def recorded_traffic(kernel: str, src_hash: str):
    """DRAM bytes per launch from a committed ncu capture, if the kernel's
    source has not changed since."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = d.get(kernel)
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle arm
def _oracle_pipeline(Cs: int, Ts: int, with_cal: bool):
    """The oracle's per-channel pipeline on Cs channels x Ts samples of the
    workload: FX correlator + Eq. modelvis (OpenMP over channels), X-engine
    over the subset selection, and lincal (numpy) for every channel."""
    import numpy as np

    import oracle
    from oracle import calib as oc
    from oracle import select as osel
    from paper_2005_03060_gb300 import synth

    L = WORKLOAD["L"]
    volt, gains, _ = synth.make_voltages(2, L, Cs, Ts, n_src=WORKLOAD["n_src"])
    v = volt.numpy()
    g = gains.numpy()
    sel = osel.subset(L, Ts)
    pt = sel.pair_type()

    def run():
        _, nt = oracle.fx_multi(v, g, L)
        for c in range(Cs):
            vc = v[c].astype(np.complex128)
            s = oracle.xengine_c64(vc, sel.pair_i, sel.pair_j, sel.win_t0[pt], sel.win_t1[pt])
            if with_cal:
                oc.calibrate(s / Ts, sel.pair_i, sel.pair_j, pt, sel.types, L, "lincal")
        return nt

    return run


def cpu_baseline():
    """One channel x 256 samples of the workload through the whole oracle
    pipeline (about 10-30 s of host CPU work)."""
    L = WORKLOAD["L"]
    Ts = 256
    run = _oracle_pipeline(1, Ts, True)
    t0 = time.perf_counter()
    run()
    dt = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    return {"value": L * L * Ts / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"1 channel x {Ts} samples of the {L * L}-antenna workload through the FP64 "
                       "oracle: FX correlator (all N^2 pairs, Eq. modelvis), X-engine over the subset "
                       "selection, lincal to 1e-10 (numpy/BLAS on all host cores)"),
            "seconds": round(dt, 2)}


def run_reference(args, rank):
    if rank != 0:
        return
    L = WORKLOAD["L"]
    budget = 150.0 / (args.steps + args.warmup)     # seconds per step
    Ts = 256
    probe = _oracle_pipeline(1, Ts, True)
    t0 = time.perf_counter()
    probe()
    t_full = time.perf_counter() - t0
    if t_full <= budget:
        Cs, with_cal = 1, True
    else:
        # calibration alone exceeds the per-step budget: time the O(N^2)
        # correlation part on a sample sized for the budget
        t0 = time.perf_counter()
        _oracle_pipeline(1, 16, False)()
        t16 = time.perf_counter() - t0
        Ts = int(max(8, min(WORKLOAD["T"], 16 * budget / max(t16, 1e-3))))
        Cs, with_cal = 1, False
    run = _oracle_pipeline(Cs, Ts, with_cal)
    desc = (f"{Cs} channel x {Ts} samples of the {L * L}-antenna workload per step through the FP64 "
            f"oracle: FX correlator (Eq. modelvis) and X-engine"
            + (", lincal to 1e-10" if with_cal else
               f"; lincal omitted (one channel alone takes {t_full:.1f} s, over the {budget:.1f} s "
               "per-step budget of this run)"))
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    dt = (time.perf_counter() - t0) / args.steps
    value = L * L * Cs * Ts / dt
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- rooflines
def lincal_flops_per_iter(N: int, n_ubl: int, P: int, bw: int) -> float:
    """FP64 flops of one Gauss-Newton iteration of the banded solver:
    band Cholesky (n bw^2), forward solve of the border and rhs
    (2 (m+1) n bw), Schur complement (m^2 n), back substitution (2 n bw),
    assembly (~150 per pair-visit, two visits per pair)."""
    n, m = 2 * N, 2 * n_ubl
    return n * bw * bw + 2.0 * (m + 1) * n * bw + m * m * n + 2.0 * n * bw + 300.0 * P


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2005_03060_gb300 import gridcorr, synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    L, C, T = WORKLOAD["L"], args.channels or WORKLOAD["C"], WORKLOAD["T"]
    N = L * L
    M = max(16, gridcorr.fft_size(L))

    volt = torch.empty(C, T, N, dtype=torch.complex64, device=dev)
    volt, gains, _ = synth.make_voltages(2 + 1000 * rank, L, C, T, n_src=WORKLOAD["n_src"],
                                         snr=WORKLOAD["snr"], device=dev, out=volt)
    ctx = gridcorr.Context(local_rank)
    sel = gridcorr.Selection("subset", L, T)
    stream = torch.cuda.current_stream(dev)
    W = 2 * L - 1
    vu = torch.empty(C, W, W, dtype=torch.complex64, device=dev)
    vr = torch.empty(C, sel.P, dtype=torch.complex64, device=dev)
    au = torch.empty(C, N, dtype=torch.float32, device=dev)
    gbuf = [gains.clone(), torch.empty_like(gains)]
    vmod = torch.zeros(C, sel.n_ubl, dtype=torch.complex64, device=dev)
    stats = torch.empty(C, 32, dtype=torch.uint8, device=dev)
    state = {"k": 0}

    def step(solver="lincal_cg", precision="fp32"):
        g_in = gbuf[state["k"] % 2]
        g_out = gbuf[(state["k"] + 1) % 2]
        ctx.correlate(volt, g_in, L, out=vu)
        ctx.reduce(volt, sel, out=vr, out_autos=au)
        ctx.calibrate(vr, sel, au, solver=solver, precision=precision, gains=g_out, vmodel=vmod,
                      stats=stats)
        state["k"] += 1

    for _ in range(args.warmup):
        step()
    ctx.device_status()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    props = torch.cuda.get_device_properties(dev)
    pci = getattr(props, "pci_bus_id", None)
    sampler = ClockSampler(f"{pci}" if pci else str(local_rank))
    ctx.profile(True)
    ctx.profile_read()
    barrier()
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms_total = e0.elapsed_time(e1)
    kern = ctx.profile_read()
    ctx.profile(False)
    ctx.device_status()
    st_last = gridcorr.decode_stats(stats)
    t = torch.tensor([ms_total], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_step = float(t.item()) / args.steps
    units_per_rank = N * C * T
    value = units_per_rank * world / (ms_step * 1e-3)

    # ---- calibration variants on the same V^reduced (equal-error comparison)
    g_ref = gbuf[state["k"] % 2].clone()
    variants = {}
    reps = max(3, min(20, args.steps // 10))
    for name, solver, prec in [("lincal_fp64", "lincal", "fp64"), ("lincal_fp32", "lincal", "fp32"),
                               ("lincal_cg_mixed", "lincal_cg", "fp32"), ("omnical_fp32", "omnical", "fp32")]:
        gv = torch.empty_like(gains)
        ctx.calibrate(vr, sel, au, solver=solver, precision=prec, gains=gv, vmodel=vmod, stats=stats)
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            ctx.calibrate(vr, sel, au, solver=solver, precision=prec, gains=gv, vmodel=vmod, stats=stats)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / reps
        sv = gridcorr.decode_stats(stats)
        diff = ((gv - g_ref).abs() / g_ref.abs()).max().item()
        variants[name] = {"ms": ms, "chans_per_s": C / (ms * 1e-3),
                          "max_rel_gain_diff_vs_lincal_fp64": diff,
                          "mean_iters": float(np.mean(sv["iters"])),
                          "mean_cg_iters": float(np.mean(sv["inner"])),
                          "converged": int(np.sum(sv["status"] == 0))}

    # ---- end to end through the public API with host buffers (pinned)
    h_volt = torch.empty(volt.shape, dtype=volt.dtype, pin_memory=True)
    h_volt.copy_(volt)
    h_gains = torch.empty(gains.shape, dtype=gains.dtype, pin_memory=True)
    h_gains.copy_(gains)
    h_vu = torch.empty(vu.shape, dtype=vu.dtype, pin_memory=True)
    h_g = torch.empty(gains.shape, dtype=gains.dtype, pin_memory=True)
    e2e_steps = max(3, min(args.steps, 10))

    def e2e_step():
        volt.copy_(h_volt, non_blocking=True)
        gbuf[state["k"] % 2].copy_(h_gains, non_blocking=True)
        step()
        h_vu.copy_(vu, non_blocking=True)
        h_g.copy_(gbuf[state["k"] % 2], non_blocking=True)

    for _ in range(2):
        e2e_step()
    barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    barrier()
    t = torch.tensor([e0.elapsed_time(e1) / e2e_steps], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_ms = float(t.item())
    e2e = {"value": units_per_rank * world / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": h_volt.numel() * 8 + h_gains.numel() * 8,
           "d2h_bytes_per_step": h_vu.numel() * 8 + h_g.numel() * 8}
    del h_volt

    peaks = load_peaks() or {}
    fp32_peak = ctx.peak_probe("fp32")
    fp64_peak = ctx.peak_probe("fp64")
    if rank != 0:
        return

    # ---- rooflines
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    rl = {}
    if "fftcorr_accumulate" in kern:
        ms, n = kern["fftcorr_accumulate"]
        dur = ms / n * 1e-3
        flops = flops_per_antenna_sample(L, M) * N * C * T
        by = 8.0 * N * C * T
        rl["fftcorr_accumulate"] = {
            "bound": "alu", "achieved": flops / dur / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": flops / dur / 1e12 / fp32_peak,
            "traffic": recorded_traffic("fftcorr_accumulate",
                                        source_hash("paper_2005_03060_gb300/csrc/gc_fftcorr.cu")),
            "algorithmic_flops": flops, "algorithmic_bytes": by,
            "peak_source": "measured: gc_peak_probe FP32 FMA on this GPU",
            "hbm": {"achieved": by / dur / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": by / dur / 1e9 / hbm_peak}}
    if "xeng_accumulate" in kern:
        ms, n = kern["xeng_accumulate"]
        dur = ms / n * 1e-3
        by = 8.0 * N * C * T
        rl["xeng_accumulate"] = {
            "bound": "hbm", "achieved": by / dur / 1e9, "peak": hbm_peak, "unit": "GB/s",
            "frac": by / dur / 1e9 / hbm_peak, "traffic": None, "algorithmic_bytes": by,
            "useful_flops": 8.0 * sel.P * C * T,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    lname = "lincal_fp64"
    if "lincal_cg" in kern:
        ms, n = kern["lincal_cg"]
        dur = ms / n * 1e-3
        cg_it = float(np.sum(st_last["inner"]))
        gn_it = float(np.sum(st_last["iters"]))
        nm = 2 * N + 2 * sel.n_ubl
        # algorithmic FP32 flops: operator pass (~70 per pair) and vector updates (~12 per
        # unknown) per CG iteration; residual/gradient pass, projection and line search
        # (~90 per pair, ~40 per unknown) per Gauss-Newton iteration
        flops = cg_it * (70.0 * sel.P + 12.0 * nm) + gn_it * (90.0 * sel.P + 40.0 * nm)
        rl["lincal_cg"] = {"bound": "alu", "achieved": flops / dur / 1e12, "peak": fp32_peak,
                           "unit": "TFLOP/s", "frac": flops / dur / 1e12 / fp32_peak, "traffic": None,
                           "algorithmic_flops": flops, "cg_iterations": cg_it, "gn_iterations": gn_it,
                           "chans_per_s": C / dur,
                           "note": "one CTA per channel; latency bound at 2 channels per SM",
                           "peak_source": "measured: gc_peak_probe FP32 FMA on this GPU"}
    if lname in kern:
        ms, n = kern[lname]
        dur = ms / n * 1e-3
        it_total = float(np.sum(st_last["iters"]))
        D = max(abs(int(dy) * L + int(dx)) for dx, dy in sel.types.tolist())
        flops = it_total * lincal_flops_per_iter(N, sel.n_ubl, sel.P, 2 * D + 1)
        rl[lname] = {"bound": "fp64", "achieved": flops / dur / 1e12, "peak": fp64_peak,
                     "unit": "TFLOP/s", "frac": flops / dur / 1e12 / fp64_peak, "traffic": None,
                     "algorithmic_flops": flops, "iterations": it_total,
                     "peak_source": "measured: gc_peak_probe FP64 FMA on this GPU"}
    dom = max(kern.items(), key=lambda kv: kv[1][0])[0]
    roofline = dict(rl.get(dom, {"bound": "unknown"}))
    roofline["kernel"] = dom
    launches = sum(n for _, n in kern.values())
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic",
            "calibrated_chans_per_s": C * world / (ms_step * 1e-3),
            "config": {"workload": WORKLOAD_NAME if C == WORKLOAD["C"] else
                       f"profiling case: {C} channels of the paper-scale workload",
                       "L": L, "channels_per_gpu": C, "T": T, "fft": M,
                       "selection": f"subset p=1 log2: {sel.P} pairs, {sel.n_ubl} types",
                       "calibration": "lincal (Gauss-Newton, matrix-free PCG step, FP32 products, FP64 "
                                      "reductions), step tol 1e-6",
                       "l2": f"inputs ({8 * N * C * T / 1e9:.2f} GB per GPU) larger than L2",
                       "parallelism": f"channels split over {world} GPU(s), no collective"},
            "roofline": roofline, "rooflines": rl,
            "kernels": {k: {"ms_per_step": v[0] / args.steps, "launches": v[1]} for k, v in kern.items()},
            "calibration_variants": variants,
            "measured_peaks": {"fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak},
            "gpu_launches": launches,
            "e2e": e2e, "clocks": clocks}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--channels", type=int, default=None,
                    help="channels per GPU (default: the workload's 256); smaller values are "
                         "for profiling captures only")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
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
