#!/usr/bin/env python
"""Benchmark of the FFT-correlator system hot path on GB300.

Workload (one step = one integration of the paper-scale array):
  32 x 32 regular grid (1024 antennas), 256 channels, 4096 time samples per
  integration, complex64 voltages from 200 point sources at SNR 10 with
  ~5 % gain-amplitude scatter and random phases, 64 x 64 FFT.
  The step runs the FFT-correlator (calibrated voltages -> V^unique).

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
def oracle_sample_fn(target_s: float):
    """Oracle FX correlator on a bounded sample of the workload (host cores).
    Returns (callable, description, antenna-samples per call)."""
    import numpy as np
    import torch

    import oracle
    from paper_2005_03060_gb300 import synth

    L, C = WORKLOAD["L"], WORKLOAD["C"]
    N = L * L
    cores = os.cpu_count() or 1
    Cs = min(C, max(1, cores))
    volt, gains, _ = synth.make_voltages(2, L, Cs, 64, n_src=WORKLOAD["n_src"])
    v = volt.numpy()
    g = gains.numpy()

    t0 = time.perf_counter()
    _, used = oracle.fx_multi(v[:, :8], g, L)
    probe = time.perf_counter() - t0
    Ts = int(max(8, min(WORKLOAD["T"], 8 * target_s / max(probe, 1e-3))))
    volt, gains, _ = synth.make_voltages(2, L, Cs, Ts, n_src=WORKLOAD["n_src"])
    v = volt.numpy()

    def run():
        _, nt = oracle.fx_multi(v, g, L)
        return nt

    desc = (f"FP64 FX oracle (all N^2 pairs, then Eq. modelvis averaging) on {Cs} channels x "
            f"{Ts} samples of the {N}-antenna workload, OpenMP over channels")
    return run, desc, N * Cs * Ts, used


def cpu_baseline(target_s=12.0):
    run, desc, units, _ = oracle_sample_fn(target_s)
    t0 = time.perf_counter()
    nt = run()
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": desc,
            "seconds": round(dt, 2)}


def run_reference(args, rank):
    if rank != 0:
        return
    run, desc, units, _ = oracle_sample_fn(1.0)
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    nt = 1
    for _ in range(args.steps):
        nt = run()
    dt = (time.perf_counter() - t0) / args.steps
    value = units / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, local_rank):
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
    vu = torch.empty(C, 2 * L - 1, 2 * L - 1, dtype=torch.complex64, device=dev)
    ctx = gridcorr.Context(local_rank)
    stream = torch.cuda.current_stream(dev)

    def step():
        ctx.correlate(volt, gains, L, out=vu)

    for _ in range(args.warmup):
        step()
    ctx.device_status()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    props = torch.cuda.get_device_properties(dev)
    pci = getattr(props, "pci_bus_id", None)
    gpu_id = f"{pci}" if pci else str(local_rank)
    sampler = ClockSampler(gpu_id)
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
    t = torch.tensor([ms_total], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_step = float(t.item()) / args.steps
    units_per_rank = N * C * T
    value = units_per_rank * world / (ms_step * 1e-3)

    # ---- end to end through the public API with host buffers (pinned)
    h_volt = torch.empty(volt.shape, dtype=volt.dtype, pin_memory=True)
    h_volt.copy_(volt)
    h_gains = torch.empty(gains.shape, dtype=gains.dtype, pin_memory=True)
    h_gains.copy_(gains)
    h_out = torch.empty(vu.shape, dtype=vu.dtype, pin_memory=True)
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(2):
        volt.copy_(h_volt, non_blocking=True)
        gains.copy_(h_gains, non_blocking=True)
        step()
        h_out.copy_(vu, non_blocking=True)
    barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        volt.copy_(h_volt, non_blocking=True)
        gains.copy_(h_gains, non_blocking=True)
        step()
        h_out.copy_(vu, non_blocking=True)
    e1.record(stream)
    barrier()
    t = torch.tensor([e0.elapsed_time(e1) / e2e_steps], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_ms = float(t.item())
    e2e = {"value": units_per_rank * world / (e2e_ms * 1e-3), "unit": UNIT,
           "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": h_volt.numel() * 8 + h_gains.numel() * 8,
           "d2h_bytes_per_step": h_out.numel() * 8}
    del h_volt

    if rank != 0:
        return

    # ---- roofline of the dominant kernel
    peaks = load_peaks() or {}
    dom = max(kern.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    dom_avg_s = dom_ms / dom_n * 1e-3
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    n_sm = props.multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FMA = 2
    flops = flops_per_antenna_sample(L, M) * N * C * T
    achieved = flops / dom_avg_s / 1e12
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    bytes_launch = 8.0 * N * C * T
    src_h = source_hash("paper_2005_03060_gb300/csrc/gc_fftcorr.cu")
    roofline = {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "traffic": recorded_traffic(dom_name, src_h),
                "algorithmic_bytes": bytes_launch,
                "algorithmic_flops": flops,
                "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz",
                "hbm": {"achieved": bytes_launch / dom_avg_s / 1e9, "peak": hbm_peak,
                        "unit": "GB/s", "frac": bytes_launch / dom_avg_s / 1e9 / hbm_peak,
                        "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"}}
    launches = sum(n for _, n in kern.values())
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME if C == WORKLOAD["C"] else
                       f"profiling case: {C} channels of the paper-scale workload",
                       "L": L, "channels_per_gpu": C, "T": T,
                       "fft": M, "l2": f"inputs ({8 * N * C * T / 1e9:.2f} GB per GPU) larger than L2",
                       "parallelism": f"channels split over {world} GPU(s), no collective"},
            "roofline": roofline,
            "kernels": {k: {"ms_per_step": v[0] / args.steps, "launches": v[1]} for k, v in kern.items()},
            "gpu_launches": launches,
            "e2e": e2e, "clocks": clocks}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
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
