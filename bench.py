#!/usr/bin/env python
"""Throughput of the explicit shallow-water step (cell-updates/s) on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp64|fp32]

Workload: the single-floodplain configuration -- 5 km x 2 km, 1600 x 625 jittered
quads = 2,000,000 triangles, seeded sinusoid + noise bed 400 m above datum,
64-patch Manning map, a 2 m deep meandering main channel (the rest dry), inflow
hydrograph 0 -> 500 m^3/s over 600 s on the upstream side, transmissive outlet,
walls.  Synthetic inputs from paper_2102_12862_b300.workloads (seed 2).

A step is one pass of the whole hot path over all cells (edge fluxes, update,
friction, dt reduction, time advance).  W untimed warm-up steps run from t = 0,
then K steps are timed with CUDA events on the stream the kernels run on.  The
working set (about 0.5 GB in FP64) is larger than the 126 MB L2, so no flush is
needed between steps.  Under torchrun every rank steps its own replica of the
workload (the path has no exchange between independent runs: replicas only,
weak scaling); value = all ranks' cell-updates / the slowest rank's time.

--impl reference times the FP64 CPU oracle (the serial edge-loop program the
CUDA path is checked against) on the host cores, one oracle step of the same
workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s"
# Algorithmic cost per cell-update (one cell, one step); derivation in the design notes.
BYTES_PER_CELL_UPDATE = {"fp64": 156.0, "fp32": 84.0}
FP64_FLOPS_PER_CELL_UPDATE = 213.0
# FP64 peak: ncu's sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained = 296 DFMA/cycle
# on this B300 (2 per SM), x 2 FLOP x the 2.032 GHz maximum SM clock.
FP64_PEAK_TFLOPS = 296 * 2 * 2.032e9 / 1e12
HBM_FALLBACK_GBS = 6400.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--e2e-steps", type=int, default=50, help="steps per end-to-end call")
    ap.add_argument("--e2e-iters", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("bm_kernels.cuh", "bm_api.cu", "bm_internal.h"):
        with open(os.path.join(ROOT, "paper_2102_12862_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(precision: str):
    """DRAM bytes per step-kernel launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"step_{precision}_floodplain_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_hash") == kernel_source_hash():
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline_sample(seconds: float, rank: int):
    """Time the FP64 oracle, as it stands, on the floodplain workload from t = 0."""
    import oracle
    from paper_2102_12862_b300 import workloads as W
    s = W.floodplain()
    o = oracle.Oracle(s)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    n = max(1, min(200, int(seconds / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return {"value": s.n_cells * n / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"serial FP64 oracle (gcc -O2 -ffp-contract=off), {n} steps of the 2,000,000-cell "
                      f"floodplain from t = 0 after 1 untimed step, {dt:.1f} s wall"}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle on the host cores."""
    if rank != 0:
        return 0
    import oracle
    from paper_2102_12862_b300 import workloads as W
    s = W.floodplain()
    o = oracle.Oracle(s)
    t0 = time.perf_counter()
    o.step(max(1, args.warmup))
    one = (time.perf_counter() - t0) / max(1, args.warmup)
    k = max(1, min(args.steps, int(120.0 / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    v = s.n_cells * k / dt
    line = {"metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus, "steps": k,
            "requested_steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / k,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "floodplain 2,000,000 triangles, FP64, oracle from t = 0", "cells": s.n_cells},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{k} oracle steps of the full workload from t = 0 (bounded to about 2 min)"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    from paper_2102_12862_b300 import bm
    from paper_2102_12862_b300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")

    def barrier():
        if dist is not None:
            dist.barrier()

    def allmax(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    s = W.floodplain()
    mesh = bm.Mesh.from_scenario(s)
    st = bm.State.from_scenario(s, mesh=mesh, precision=args.precision)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    st.set_stream(stream.cuda_stream)
    st.step(args.warmup)
    wet_before = None

    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.step_async(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    st.sync()
    ms = e0.elapsed_time(e1)
    ms_max = allmax(ms)
    n = s.n_cells
    value = n * args.steps * ws / (ms_max / 1e3)
    stats = st.stats()

    # dominant kernel: average duration of the step kernel, events around each launch
    nk = min(args.steps, 200)
    k_ms, tot_ms = st.step_timed(nk)
    kern_s = k_ms / nk / 1e3
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)
    prec = args.precision
    bytes_launch = BYTES_PER_CELL_UPDATE[prec] * n
    traffic = ncu_traffic(prec)
    hbm_gbs = bytes_launch / kern_s / 1e9
    if prec == "fp64":
        flops = FP64_FLOPS_PER_CELL_UPDATE * n
        achieved = flops / kern_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "ncu peak_sustained 296 DFMA/cycle x 2 x 2.032 GHz (no FP64 figure in MEASURED_PEAKS.json)",
                "kernel": "step_batch<double,true>", "kernel_ms": kern_s * 1e3,
                "hbm": {"achieved": hbm_gbs, "peak": hbm, "unit": "GB/s", "frac": hbm_gbs / hbm,
                        "algorithmic_bytes_per_launch": bytes_launch}}
    else:
        roof = {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm, "unit": "GB/s", "frac": hbm_gbs / hbm,
                "traffic": traffic, "kernel": "step_batch<float,false>", "kernel_ms": kern_s * 1e3,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback"}

    # end to end through the C ABI with pinned host buffers: upload, E steps, download
    E = args.e2e_steps
    pin = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(6)]
    Hh, qxh, qyh, Ho, qxo, qyo = [p.numpy() for p in pin]
    Hh[:], qxh[:], qyh[:] = s.H, s.qx, s.qy
    times = []
    for it in range(args.e2e_iters + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st.upload(Hh, qxh, qyh, 0.0)
        st.step(E)
        bm.bm_state_download(st.handle, n, Ho, qxo, qyo)
        t1 = time.perf_counter()
        if it > 0:
            times.append(t1 - t0)
    e2e_t = max(allmax(statistics.median(times)), 1e-12)
    e2e = {"value": n * E * ws / e2e_t, "unit": METRIC, "h2d_bytes_per_step": 3 * 8 * n / E,
           "d2h_bytes_per_step": 3 * 8 * n / E,
           "call": f"bm_state_upload + bm_step({E}) + bm_state_download, pinned host arrays"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(args.cpu_seconds, rank)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32+f64",
                "data": "synthetic",
                "config": {"workload": f"floodplain 2,000,000 triangles, {prec.upper()}, steps from t = 0 "
                                       f"after {args.warmup} warm-up steps", "cells": n,
                           "edges": mesh.info["n_edges"], "precision": prec,
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                           "l2": "working set > 126 MB L2, no flush",
                           "sim_time_s": stats["t"], "e2e_steps_per_call": E},
                "roofline": roof, "e2e": e2e, "gpu_launches": 2 * args.steps, "clocks": clk,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
