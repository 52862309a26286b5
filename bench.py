#!/usr/bin/env python
"""Throughput of the explicit shallow-water step (cell-updates/s) on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the single-floodplain configuration -- 5 km x 2 km, 1600 x 625 jittered
quads = 2,000,000 triangles, seeded sinusoid + noise bed 400 m above datum,
64-patch Manning map, a 2 m deep meandering main channel (the rest dry), inflow
hydrograph 0 -> 500 m^3/s over 600 s on the upstream side, walls, positivity time
step -- run for 3,600 simulated seconds with moving wet/dry fronts.  Synthetic
inputs from paper_2102_12862_b300.workloads (seed 2).

A step is one pass of the whole hot path over all cells (edge fluxes, update,
friction, dt reduction, time advance: one kernel launch).  The cost of a step grows
as the flood spreads, so the run is sampled: states at t = 0, 600, 1,800 and 3,600 s
(made by a GPU run of the workload in the same precision, downloaded) are each
uploaded, stepped W untimed warm-up steps and then K timed steps (CUDA events on the
stream the kernels run on); `value` is the whole run's rate, the run's step count over
the step-weighted time (trapezoids between the windows).  `e2e` is the user's call for the whole
configuration through the C ABI: upload of the initial state from pinned host memory,
bm_run_until(3,600 s), download, wall-clock.  The line's `value` is plain FP64;
`fp32_bulk` repeats every measurement for the FP32-bulk precision mode.  The working
set (0.3-0.5 GB) is larger than the 126 MB L2, so no flush is needed.  Under torchrun
every rank steps its own replica (no exchange between independent runs: replicas only,
weak scaling); value = all ranks' cell-updates / the slowest rank's time.

Also in the line: the 1,000,000-cell wet lake (the HBM / FP64-arithmetic bound
context), a batched ensemble (FP32-bulk, one launch per step for all members) against
FP64 plain, a bounded serving trace with p50 / p99 time-to-result, and the optional
features' cost.  Accuracy: the first 50 steps through the C ABI against the FP64 CPU
oracle run for the same steps, which is also the timed CPU baseline.

--impl reference times that oracle alone (serial C on the host cores) on the same
workload and metric.
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
# Algorithmic DRAM bytes per cell-update (the hot-path scope table's per-unit figure):
# the state read and written, bed, Manning coefficient, three neighbour indices, three
# edges' geometry and the area -- FP64 156 B, FP32-bulk 84 B.
BYTES_PER_CELL_UPDATE = {"fp64": 156, "fp32": 84}
# The tighter count of what the tile layout moves (each mesh edge read once): per cell
# the state read and written (FP64: H, qx, qy; FP32-bulk: H hi/lo, qx, qy), z, g n^2,
# 1/|Omega| and the slot word; per mesh edge the code word and nx, ny, l.
LAYOUT_BYTES_PER_CELL = {"fp64": 2 * 24 + 3 * 8 + 4, "fp32": 2 * 16 + 3 * 4 + 4}
LAYOUT_BYTES_PER_EDGE = {"fp64": 4 + 3 * 8, "fp32": 4 + 3 * 4}
# FP64 arithmetic per wet cell-update of the step kernel (DADD + DMUL + 2 DFMA thread
# instructions executed, ncu counters on the 1,000,000-cell wet lake: 3.187e8 FLOP per
# launch over 991,485 wet cells); dry cells take no FP64 instruction.
FP64_FLOP_PER_WET_CELL = 321.4
FP64_PEAK_TFLOPS = 1.2023  # 296 DFMA lanes per cycle (ncu peak) x 2 FLOP x 2.031 GHz
HBM_FALLBACK_GBS = 6400.0
T_WINDOWS = (0.0, 600.0, 1800.0, 3600.0)  # the floodplain run's sampled times [s]
L2_FLUSH_STEPS = 50  # steps of the L2-flushed cross-check
KERNEL_NAME = {"fp64": "step_pipe<double, 0, 2>", "fp32": "step_pipe<float, 0, 2>"}  # plain level, 2 slots


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200, help="timed steps of each floodplain window")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=50, help="steps of the oracle accuracy check")
    ap.add_argument("--t-end", type=float, default=3600.0, help="simulated seconds of the floodplain run")
    ap.add_argument("--ensemble-members", type=int, default=64, help="members of the ensemble leg (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=50, help="requests of the serving leg (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle (and the accuracy check)")
    ap.add_argument("--precisions", default="fp64,fp32")
    ap.add_argument("--lake-steps", type=int, default=500,
                    help="steps of the mostly wet lake-at-rest line (0: skip it)")
    ap.add_argument("--track-steps", type=int, default=200,
                    help="steps of the flood-tracking and passive-species cost line (0: skip it)")
    ap.add_argument("--stress-steps", type=int, default=100000, help="stress: lake-at-rest steps")
    ap.add_argument("--workload", choices=["floodplain", "ensemble", "serve", "stress", "lake", "window"],
                    default="floodplain",
                    help="floodplain: the default line; ensemble: batched uneven meshes; serve: request loop; "
                         "lake: the wet-lake leg alone; window: a few floodplain steps from the run's state at "
                         "--t-start (for profilers)")
    ap.add_argument("--t-start", type=float, default=0.0, help="window: simulated time of the state stepped")
    ap.add_argument("--state-file", default="",
                    help="window: the state at --t-start is read from this .npz if it exists, else made by a "
                         "GPU run from t = 0 and saved there")
    ap.add_argument("--instances", type=int, default=256, help="ensemble members")
    ap.add_argument("--requests", type=int, default=200, help="serving trace length")
    ap.add_argument("--rate", type=float, default=20.0, help="serving arrivals per second (Poisson)")
    ap.add_argument("--time-scale", type=float, default=0.1,
                    help="serving: requested simulated durations U[600, 7200] s are scaled by this")
    ap.add_argument("--mesh-pool", type=int, default=16, help="serving: distinct meshes reused by requests")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp32", help="ensemble / serve precision")
    return ap.parse_args()


def len_tiles(mesh) -> int:
    """The mesh's tiles of 256 cells."""
    return int(mesh.info["n_tiles"])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def kernel_source_hash() -> str:
    """Hash of the step kernel's sources with comments and blank lines removed, so that
    a profile stays attached to the code it was taken on across comment edits."""
    h = hashlib.sha256()
    for f in ("bm_kernels.cuh", "bm_step.cuh", "bm_internal.h"):
        with open(os.path.join(ROOT, "paper_2102_12862_b300", "csrc", f), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def ncu_profile(precision: str):
    """The committed ncu summary of the step kernel on the floodplain (DRAM bytes per
    tile a launch takes, FP64-pipe activity), if it was taken on the current kernel
    source (else None)."""
    path = os.path.join(ROOT, "profiles", f"step_{precision}_floodplain_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_hash") == kernel_source_hash():
            return d
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


def replica_aggregate(dist, n_cells_local: float, steps: int, ms_local: float, device=None) -> tuple[float, float]:
    """Replicas only: each rank stepped its own copy of the workload.  Returns the
    slowest rank's time and the whole-job rate (all ranks' cell-updates / that time)."""
    if dist is None:
        return ms_local, n_cells_local * steps / (ms_local / 1e3)
    import torch
    t = torch.tensor([ms_local, n_cells_local], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    tot = t.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms_max = float(mx[0].item())
    return ms_max, float(tot[1].item()) * steps / (ms_max / 1e3)


def errors_vs_oracle(s, H, qx, qy, o) -> dict:
    """L1 / L-inf of depth and velocity, relative mass defect of the GPU state vs the oracle."""
    area = o.area()
    h, ho = H - s.z, o.H - s.z
    wet = (ho > 1e-3) & (h > 1e-3)
    du = np.abs(qx[wet] / h[wet] - o.qx[wet] / ho[wet]) if wet.any() else np.zeros(1)
    dv = np.abs(qy[wet] / h[wet] - o.qy[wet] / ho[wet]) if wet.any() else np.zeros(1)
    vo = float(np.sum(area * ho))
    return {"l1_h_m": float(np.sum(area * np.abs(h - ho)) / area.sum()),
            "linf_h_m": float(np.max(np.abs(h - ho))),
            "rel_linf_h": float(np.max(np.abs(h - ho)) / max(np.max(np.abs(ho)), 1e-300)),
            "rel_linf_hu": float(np.max(np.abs(qx - o.qx)) / max(np.max(np.abs(o.qx)), 1e-300)),
            "rel_linf_hv": float(np.max(np.abs(qy - o.qy)) / max(np.max(np.abs(o.qy)), 1e-300)),
            "l1_vel_ms": float(np.mean(np.hypot(du, dv))),
            "linf_vel_ms": float(max(du.max(), dv.max())),
            "rel_mass_vs_oracle": abs(float(np.sum(area * h)) - vo) / max(abs(vo), 1e-300)}


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
            "config": {"workload": "floodplain 2,000,000 triangles, FP64 oracle, steps from t = 0",
                       "cells": s.n_cells},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{k} oracle steps of the full workload after {args.warmup} warm-up steps "
                                       f"(bounded to about 2 min)"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def floodplain_snapshots(s, st, t_end: float) -> list:
    """States of the floodplain run at the sampled times (T_WINDOWS up to t_end): the
    state st (fresh, at t = 0) runs from t = 0 and is downloaded at each, with the run's
    step count and wet fraction.  Each precision samples its own run (the other
    precision's state differs by its rounding: an FP32-bulk dry cell's surface lies up
    to half an FP32 ulp of the bed offset above the FP64 bed, a film the FP64 step would
    have to flux)."""
    snaps = []
    for tw in [t for t in T_WINDOWS if t <= t_end]:
        if tw > 0:
            st.run_until(tw)
        H, qx, qy, t = st.download()
        snaps.append({"t": t, "H": H, "qx": qx, "qy": qy, "steps": st.stats(volume=False)["steps"],
                      "wet": float(np.mean(H - s.z > s.params["h_min"]))})
    return snaps


def step_weighted(snaps: list, ms: list) -> tuple[int, float]:
    """The run's steps and its time from the windows' times per step: trapezoids
    between consecutive windows, weighted by the steps the run took between them."""
    total_ms = 0.0
    for a in range(len(snaps) - 1):
        total_ms += (snaps[a + 1]["steps"] - snaps[a]["steps"]) * 0.5 * (ms[a] + ms[a + 1])
    steps = snaps[-1]["steps"] - snaps[0]["steps"]
    if steps <= 0:  # a single window
        return 1, ms[0]
    return steps, total_ms


def measure(args, prec, s, mesh, torch, bm, dist, ws, rank):
    """The floodplain windows, the whole-run rate, the rooflines and the end-to-end run of
    one precision."""
    def barrier():
        if dist is not None:
            dist.barrier()

    def allmax(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    n = s.n_cells
    st = bm.State.from_scenario(s, mesh=mesh, precision=prec)
    snaps = floodplain_snapshots(s, st, args.t_end)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    st.set_stream(stream.cuda_stream)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    windows, ms_list = [], []
    for sn in snaps:
        st.upload(sn["H"], sn["qx"], sn["qy"], sn["t"])
        st.step(args.warmup)
        taken0, n_tiles = st.work()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.step_async(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        st.sync()
        ms = allmax(e0.elapsed_time(e1)) / args.steps
        ms_list.append(ms)
        # the share of the tiles the launches take (mean of the window's first and last)
        sn["taken"] = 0.5 * (taken0 + st.work()[0]) / n_tiles
        w = {"t_s": sn["t"], "wet_fraction": sn["wet"], "tiles_taken": sn["taken"], "ms_per_step": ms,
             "value": n * ws / (ms / 1e3),
             "hbm_frac": BYTES_PER_CELL_UPDATE[prec] * n * sn["taken"] / (ms / 1e3) / 1e9 / hbm}
        if prec == "fp64":
            w["fp64_frac"] = FP64_FLOP_PER_WET_CELL * sn["wet"] * n / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS
        windows.append(w)
    steps, total_ms = step_weighted(snaps, ms_list)
    ms_run = total_ms / steps  # the run's mean time per step (= mean launch duration: one launch a step)

    # cross-check of the cache state: the first and last windows again with L2 flushed
    # (a 256 MiB buffer written) before every timed step, each step timed alone
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flushed = []
    for sn in (snaps[0], snaps[-1]) if len(snaps) > 1 else (snaps[0],):
        st.upload(sn["H"], sn["qx"], sn["qy"], sn["t"])
        st.step(args.warmup)
        tot = 0.0
        for _ in range(L2_FLUSH_STEPS):
            flush_buf.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st.step_async(1)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        st.sync()
        flushed.append({"t_s": sn["t"], "ms_per_step": tot / L2_FLUSH_STEPS, "steps": L2_FLUSH_STEPS})
    del flush_buf
    value = n * ws / (ms_run / 1e3)

    # dominant kernel (the step kernel, the only one in the timed windows): algorithmic
    # bytes per launch over the run's mean launch duration.  A launch moves the bytes of
    # the tiles it takes; a skipped tile (dry, at rest, no changed neighbour: its step is
    # a copy-through) moves none, so the units of a launch are the cells of its tiles
    taken = sum((snaps[a + 1]["steps"] - snaps[a]["steps"]) * 0.5 * (snaps[a]["taken"] + snaps[a + 1]["taken"])
                for a in range(len(snaps) - 1)) / max(steps, 1) if len(snaps) > 1 else snaps[0]["taken"]
    bytes_launch = BYTES_PER_CELL_UPDATE[prec] * n * taken
    layout_bytes = (LAYOUT_BYTES_PER_CELL[prec] * n + LAYOUT_BYTES_PER_EDGE[prec] * mesh.info["n_edges"]) * taken
    prof = ncu_profile(prec)
    # DRAM traffic per launch: ncu's bytes per tile taken (windows at t = 0 and the run's
    # end, their mean) times the run's mean tiles per launch
    traffic = (prof["dram_bytes_per_tile"] * taken * len_tiles(mesh)) if prof else None
    roof = {"bound": "hbm", "achieved": bytes_launch / (ms_run / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": bytes_launch / (ms_run / 1e3) / 1e9 / hbm, "traffic": traffic,
            "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {prof['dram_bytes_per_tile']:.0f} B "
                               f"per tile taken (profiles/{prof['summary']}), x the run's mean tiles per launch")
                              if prof else "no ncu summary of the current kernel source",
            "kernel": KERNEL_NAME[prec], "kernel_ms": ms_run,
            "algorithmic_bytes_per_launch": bytes_launch,
            "tiles_taken": taken,
            "bytes": f"{BYTES_PER_CELL_UPDATE[prec]} B per cell-update of the tiles a launch takes (the run's "
                     f"step-weighted share {taken:.3f} of the tiles; the others are dry, at rest and unchanged)",
            "layout_bytes_per_launch": layout_bytes,
            "layout_frac": layout_bytes / (ms_run / 1e3) / 1e9 / hbm,
            # the same bytes per cell-update over every cell of the mesh (as if each
            # launch streamed all tiles): the step's rate in the metric's own units,
            # against the copy bandwidth
            "frac_all_cells": BYTES_PER_CELL_UPDATE[prec] * n / (ms_run / 1e3) / 1e9 / hbm,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback"}
    if prec == "fp64":
        wet_steps = sum((snaps[a + 1]["steps"] - snaps[a]["steps"]) * 0.5 * (snaps[a]["wet"] + snaps[a + 1]["wet"])
                        for a in range(len(snaps) - 1)) or snaps[0]["wet"]
        flop = FP64_FLOP_PER_WET_CELL * n * wet_steps / max(steps, 1)  # per launch, run mean
        roof_fp64 = {"bound": "alu", "achieved": flop / (ms_run / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": flop / (ms_run / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                     "traffic": traffic,
                     "kernel": KERNEL_NAME[prec], "kernel_ms": ms_run,
                     "flop_per_launch": flop,
                     "flops": f"{FP64_FLOP_PER_WET_CELL} FP64 FLOP (DADD + DMUL + 2 DFMA, counted by ncu) per wet "
                              f"cell-update x the run's step-weighted wet cells",
                     "fp64_pipe_active": prof.get("fp64_pipe_active") if prof else None,
                     "peak_source": "296 DFMA lanes per cycle (ncu peak) x 2 FLOP x 2.031 GHz (max SM clock)"}
    else:
        roof_fp64 = None

    # end to end, the configuration as a user runs it through the C ABI: the initial
    # state from pinned host memory, bm_run_until(t_end), the final state back
    pin = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(6)]
    Hh, qxh, qyh, Ho, qxo, qyo = [p.numpy() for p in pin]
    Hh[:], qxh[:], qyh[:] = s.H, s.qx, s.qy
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st.upload(Hh, qxh, qyh, 0.0)
    st.run_until(args.t_end)
    bm.bm_state_download(st.handle, n, Ho, qxo, qyo)
    wall = allmax(time.perf_counter() - t0)
    clk = clocks.stop()
    e2e_steps = st.stats(volume=False)["steps"]
    e2e = {"value": n * e2e_steps * ws / wall, "unit": METRIC, "wall_s": wall, "steps": e2e_steps,
           "h2d_bytes_per_step": 3 * 8 * n / max(e2e_steps, 1), "d2h_bytes_per_step": 3 * 8 * n / max(e2e_steps, 1),
           "call": f"bm_state_upload + bm_run_until({args.t_end:g} s) + bm_state_download, pinned host arrays"}

    # accuracy leg: the first steps from t = 0 (compared with the oracle by the caller)
    st.upload(s.H, s.qx, s.qy, 0.0)
    st.step(args.e2e_steps)
    Hf, qxf, qyf, _ = st.download()
    out = {"value": value, "ms_per_step": ms_run, "steps_run": steps, "windows": windows, "roofline": roof,
           "l2_flushed": flushed,
           "windows_desc": ", ".join(f"{sn['t']:g}" for sn in snaps),
           "roofline_fp64": roof_fp64, "e2e": e2e, "clocks": clk,
           "gpu_launches": args.steps * len(snaps)}
    st.close()
    return out, (Hf, qxf, qyf)


def measure_lake(args, torch, bm, W):
    """The same step on a mostly wet mesh, as context for the floodplain numbers: the
    1,000,000-triangle lake at rest on 5 m fractal relief (partially dry islands).  Its
    wet tiles run the full flux and friction arithmetic every step.  Also reports the
    largest velocity and the relative volume change after the timed steps (the lake
    must stay at rest)."""
    s = W.fractal_lake()
    mesh = bm.Mesh.from_scenario(s)
    n_wet = int(np.count_nonzero(s.H - s.z > s.params["h_min"]))
    hbm = measured_peaks().get("hbm_gbs", HBM_FALLBACK_GBS)
    out = {"workload": "lake at rest, 1,000,000 triangles, z = 400 m + fractal relief (5 m), surface 403 m",
           "cells": s.n_cells, "wet_fraction": n_wet / s.n_cells, "steps": args.lake_steps}
    for prec in [p for p in args.precisions.split(",") if p]:
        st = bm.State.from_scenario(s, mesh=mesh, precision=prec)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        st.set_stream(stream.cuda_stream)
        st.step(args.warmup)
        v0 = st.stats()["volume"]
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.step_async(args.lake_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        st.sync()
        ms = e0.elapsed_time(e1)
        H, qx, qy, _ = st.download()
        h = H - s.z
        wet = h > 1e-3
        speed = float(np.max(np.hypot(qx[wet], qy[wet]) / h[wet])) if wet.any() else 0.0
        v1 = st.stats()["volume"]
        r = {"value": s.n_cells * args.lake_steps / (ms / 1e3), "unit": METRIC, "ms_per_step": ms / args.lake_steps,
             "max_speed_ms": speed, "rel_volume_change": abs(v1 - v0) / abs(v0),
             "hbm_frac": BYTES_PER_CELL_UPDATE[prec] * s.n_cells / (ms / args.lake_steps / 1e3) / 1e9 / hbm}
        if prec == "fp64":
            flop = FP64_FLOP_PER_WET_CELL * n_wet
            achieved = flop / (ms / args.lake_steps / 1e3) / 1e12
            r["roofline_fp64_arith"] = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                                        "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                                        "flop_per_launch": flop,
                                        "flops": f"{FP64_FLOP_PER_WET_CELL} FP64 FLOP per wet cell-update x "
                                                 f"{n_wet} wet cells"}
        out["fp32_bulk" if prec == "fp32" else prec] = r
        st.close()
    return out


def run_lake(args, ws, rank, torch, bm, W):
    """The wet-lake leg alone (its own line)."""
    print(json.dumps(measure_lake(args, torch, bm, W)), flush=True)
    return 0


def measure_tracking(args, torch, bm, W):
    """The optional features' cost on the floodplain: the same args.track_steps steps
    from t = 0 plain, with flood tracking (arrival time of 0.05 m, maxima of depth,
    velocity, discharge and bed shear stress, updated in the step kernel) and with two
    passive species (one entering with the inflow at c = 1, one filling the initially
    wet river at c = 0.5; the step kernel exports its edge mass fluxes, the species
    kernel advects them after each step), with rain on a disk (a source region: the
    rate kernel before each step, the S term in the step kernel) and, in FP64, with bed
    evolution (sand: d = 1 mm, MPM-like closure; the bed-flux and update kernels)."""
    s = W.floodplain()
    mesh = bm.Mesh.from_scenario(s)
    h0 = np.maximum(s.H - s.z, 0.0)
    rain_region = W.disk_region(s, 2500.0, 1000.0, 500.0)
    out = {"workload": "floodplain 2,000,000 triangles, steps from t = 0, arrival threshold 0.05 m; "
                       "2 passive species (inflow c = 1; river c = 0.5); bed evolution (sand d = 1 mm, MPM-like, FP64); "
                       "rain 50 mm/h on a 500 m disk "
                       f"({int((rain_region >= 0).sum())} cells, 9 % wet at t = 0)",
           "steps": args.track_steps}
    for prec in [p for p in args.precisions.split(",") if p]:
        res = {}
        for mode in ("plain", "tracked", "species", "sources") + (("morpho",) if prec == "fp64" else ()):
            st = bm.State.from_scenario(s, mesh=mesh, precision=prec)
            stream = torch.cuda.Stream()
            torch.cuda.set_stream(stream)
            st.set_stream(stream.cuda_stream)
            if mode == "tracked":
                st.track(0.05)
            elif mode == "species":
                st.set_scalars(np.stack([np.zeros_like(h0), 0.5 * h0]), c_in=[1.0, 0.0])
            elif mode == "morpho":
                st.set_morpho(porosity=0.4, s=2.65, d=0.001, alpha=8.0, m=1.5, theta_cr=0.047)
            elif mode == "sources":
                st.set_sources(rain_region, [bm.SOURCE_INTENSITY], [bm.SINK_EXACT],
                               [(np.array([0.0]), np.array([50.0]))])
            st.step(args.warmup)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st.step_async(args.track_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            st.sync()
            res[mode] = e0.elapsed_time(e1) / args.track_steps
            if mode == "tracked":
                rec = st.download_track()
                res["arrived"] = int(np.sum(~np.isnan(rec["t_arrival"])))
            elif mode == "species":
                hc = st.download_scalars()
                res["inflow_species_volume"] = float(hc[0] @ tri_areas(s))
            st.close()
        out["fp32_bulk" if prec == "fp32" else prec] = {
            "ms_per_step": res["plain"], "ms_per_step_tracked": res["tracked"],
            "overhead": res["tracked"] / res["plain"] - 1.0, "cells_arrived": res["arrived"],
            "ms_per_step_2_species": res["species"], "overhead_2_species": res["species"] / res["plain"] - 1.0,
            "inflow_species_volume_m3": res["inflow_species_volume"],
            "ms_per_step_rain": res["sources"], "overhead_rain": res["sources"] / res["plain"] - 1.0}
        if "morpho" in res:
            out["fp64"].update({"ms_per_step_morpho": res["morpho"],
                                "overhead_morpho": res["morpho"] / res["plain"] - 1.0})
    return out


def tri_areas(s):
    a, b, c = s.xy[s.tri[:, 0]], s.xy[s.tri[:, 1]], s.xy[s.tri[:, 2]]
    return 0.5 * np.abs((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))


def run_stress(args, ws, rank, torch, bm, W):
    """Precision stress: (1) the 1,000,000-triangle lake at rest on fractal relief
    (surface 403 m over a 400 m datum, partially dry) for args.stress_steps steps in
    FP32-bulk and FP64 -- largest velocity, surface drift and relative mass defect; (2) Thacker's
    planar sloshing in a paraboloid on 250k cells for one period, FP64 and FP32-bulk --
    errors against the closed form, between the two precisions, and mass defects."""
    out = {"metric": "precision stress", "n_gpus": ws, "data": "synthetic"}
    s = W.fractal_lake()
    for prec in ("fp32", "fp64"):
        st = bm.State.from_scenario(s, precision=prec)
        v0 = st.stats()["volume"]
        t0 = time.perf_counter()
        st.step(args.stress_steps)
        wall = time.perf_counter() - t0
        H, qx, qy, _ = st.download()
        h = H - s.z
        wet = h > 1e-3
        v1 = st.stats()["volume"]
        out[f"lake_{prec}"] = {"workload": "lake at rest, 1,000,000 triangles, z = 400 m + fractal relief (5 m), "
                                           "surface 403 m", "steps": args.stress_steps, "wall_s": wall,
                               "max_speed_ms": float(np.max(np.hypot(qx[wet], qy[wet]) / h[wet])),
                               "max_surface_drift_m": float(np.max(np.abs(H - s.H))),
                               "rel_mass_defect": abs(v1 - v0) / abs(v0)}
        st.close()
    s = W.thacker()
    area = tri_areas(s)
    c = s.xy[s.tri].mean(axis=1)
    om = np.sqrt(2 * 9.81 * 10.0) / 3000.0
    T = 2 * np.pi / om
    he, ue, ve = W.thacker_exact(c[:, 0], c[:, 1], T)
    res = {}
    for prec in ("fp64", "fp32"):
        st = bm.State.from_scenario(s, precision=prec)
        v0 = st.stats()["volume"]
        st.run_until(T)
        H, qx, qy, _ = st.download()
        v1 = st.stats()["volume"]
        res[prec] = (H - s.z, qx, qy)
        h = H - s.z
        out[f"thacker_{prec}"] = {"cells": s.n_cells, "t_s": T, "steps": st.stats(volume=False)["steps"],
                                  "l1_depth_vs_exact_m": float(np.sum(area * np.abs(h - he)) / area.sum()),
                                  "rel_mass_defect": abs(v1 - v0) / abs(v0)}
        st.close()
    (h64, qx64, qy64), (h32, qx32, qy32) = res["fp64"], res["fp32"]
    wet = (h64 > 1e-3) & (h32 > 1e-3)
    out["thacker_fp32_vs_fp64"] = {
        "l1_depth_m": float(np.sum(area * np.abs(h32 - h64)) / area.sum()),
        "linf_depth_m": float(np.max(np.abs(h32 - h64))),
        "l1_speed_ms": float(np.mean(np.hypot(qx32[wet] / h32[wet] - qx64[wet] / h64[wet],
                                              qy32[wet] / h32[wet] - qy64[wet] / h64[wet])))}
    print(json.dumps(out), flush=True)
    return 0


def ensemble_leg(args, torch, bm, W, n_members: int, steps: int) -> dict:
    """Batched FP32-bulk ensemble: n_members floodplain-recipe meshes, log-uniform sizes in
    [5k, 500k] triangles (member k seeded 5000 + k), stepped together by one launch per
    step (each member with its own dt), launch shape from the autotuner; steps timed
    with CUDA events after warm-up."""
    scs = [W.ensemble_instance(k) for k in range(n_members)]
    meshes = [bm.Mesh.from_scenario(x) for x in scs]
    sts = [bm.State.from_scenario(x, mesh=m, precision="fp32") for x, m in zip(scs, meshes)]
    b = bm.Batch(sts)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    b.set_stream(stream.cuda_stream)
    best, _ = b.autotune(5)
    b.step(args.warmup)
    cells = sum(x.n_cells for x in scs)
    clocks = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step_async(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    b.sync()
    ms = e0.elapsed_time(e1)
    b.close()
    for x in sts:
        x.close()
    return {"workload": f"{n_members} floodplain-recipe meshes, log-uniform 5k-500k triangles ({cells} cells), "
                        f"FP32-bulk, one launch per step, per-member dt", "members": n_members, "cells": cells,
            "steps": steps, "value": cells * steps / (ms / 1e3), "unit": METRIC, "ms_per_step": ms / steps,
            "ctas_per_sm": best, "clocks": clk, "gpu_launches": steps}


def serving_leg(args, torch, bm, W, n_requests: int, rate: float = 20.0, pool: int = 6,
                time_scale: float = 0.1, precision: str = "fp32") -> dict:
    """Request loop: Poisson arrivals at `rate` per second of flood scenarios on a pool of
    meshes (sizes log-uniform in [10k, 2M] triangles), each run for a duration drawn
    from U[600, 7200] s x time_scale; a bounded trace of n_requests arrivals, then
    drained.  p50 / p99 time-to-result (submission to result) and the throughput."""
    rng = np.random.default_rng(6)
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(2e6), pool)).astype(int)
    scs = [W.ensemble_instance(1000 + k, size_override=int(n)) for k, n in enumerate(sizes)]
    meshes = [bm.Mesh.from_scenario(x) for x in scs]
    sv = bm.Server(precision=precision, steps_per_round=32)
    gaps = rng.exponential(1.0 / rate, n_requests)
    picks = rng.integers(0, pool, n_requests)
    t_ends = rng.uniform(600.0, 7200.0, n_requests) * time_scale
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    tickets = []
    t_start = time.perf_counter()
    next_t = t_start
    for k in range(n_requests):
        next_t += gaps[k]
        while time.perf_counter() < next_t:
            time.sleep(min(0.001, max(0.0, next_t - time.perf_counter())))
        x = scs[picks[k]]
        tickets.append(sv.submit(meshes[picks[k]], x.H, x.qx, x.qy, t_end=float(t_ends[k]), **x.params))
    lat = [sv.wait(tk, 3600.0)[3] for tk in tickets]
    wall = time.perf_counter() - t_start
    clk = clocks.stop()
    stt = sv.stats()
    sv.close()
    return {"workload": f"{n_requests} Poisson arrivals at {rate:g}/s, {pool}-mesh pool log-uniform 10k-2M "
                        f"triangles ({', '.join(str(int(n)) for n in sizes)}), durations U[600, 7200] s x {time_scale:g}, "
                        f"{precision.upper()}", "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "throughput": stt["cell_updates"] / wall, "unit": METRIC,
            "wall_s": wall, "completed": stt["completed"], "clocks": clk}


def run_ensemble(args, ws, rank, torch, bm, W):
    """Batched ensemble: args.instances floodplain-recipe meshes, log-uniform sizes in
    [5k, 500k] triangles (member k seeded 5000 + k), stepped together by one launch
    per step, each with its own dt."""
    scs = [W.ensemble_instance(k) for k in range(args.instances)]
    meshes = [bm.Mesh.from_scenario(s) for s in scs]
    sts = [bm.State.from_scenario(s, mesh=m, precision=args.precision) for s, m in zip(scs, meshes)]
    b = bm.Batch(sts)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    b.set_stream(stream.cuda_stream)
    best, _ = b.autotune(5)
    b.step(args.warmup)
    cells = sum(s.n_cells for s in scs)
    clocks = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step_async(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    b.sync()
    ms = e0.elapsed_time(e1)
    value = cells * args.steps / (ms / 1e3)
    # every member to 600 s of simulated time (per-member dt), timed as one job
    t0 = time.perf_counter()
    b.run_until(600.0)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    upd = sum(st.stats(volume=False)["steps"] * sc.n_cells for st, sc in zip(sts, scs)) - cells * (args.steps + args.warmup)
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": f"batched ensemble, {args.instances} floodplain-recipe meshes, log-uniform "
                                   f"5k-500k triangles, one launch per step, per-member dt",
                       "members": args.instances, "cells": cells, "precision": args.precision,
                       "ctas_per_sm": best, "l2": "working set > L2, no flush"},
            "run_until_600s": {"wall_s": wall, "cell_updates_per_s": upd / wall},
            "gpu_launches": args.steps, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args, ws, rank, torch, bm, W):
    """Request loop: Poisson arrivals at args.rate per second of flood scenarios on a
    pool of meshes (sizes log-uniform in [10k, 2M] triangles), each run for a
    duration drawn from U[600, 7200] s x time_scale; bounded trace of args.requests
    arrivals, then drained.  Reports p50 / p99 time-to-result and the throughput."""
    rng = np.random.default_rng(6)
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(2e6), args.mesh_pool)).astype(int)
    pool = [W.ensemble_instance(1000 + k, size_override=int(n)) for k, n in enumerate(sizes)]
    meshes = [bm.Mesh.from_scenario(s) for s in pool]
    sv = bm.Server(precision=args.precision, steps_per_round=32)
    gaps = rng.exponential(1.0 / args.rate, args.requests)
    picks = rng.integers(0, args.mesh_pool, args.requests)
    t_ends = rng.uniform(600.0, 7200.0, args.requests) * args.time_scale
    tickets = []
    t_start = time.perf_counter()
    next_t = t_start
    for k in range(args.requests):
        next_t += gaps[k]
        while time.perf_counter() < next_t:
            time.sleep(min(0.001, max(0.0, next_t - time.perf_counter())))
        sc = pool[picks[k]]
        tickets.append(sv.submit(meshes[picks[k]], sc.H, sc.qx, sc.qy, t_end=float(t_ends[k]), **sc.params))
    lat = []
    for tk in tickets:
        r = sv.wait(tk, 3600.0)
        lat.append(r[3])
    wall = time.perf_counter() - t_start
    st = sv.stats()
    sv.close()
    line = {"metric": "p50/p99 time-to-result", "value": float(np.percentile(lat, 50)), "unit": "s",
            "p99_s": float(np.percentile(lat, 99)), "n_gpus": ws, "steps": None, "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": f"serving: {args.requests} Poisson arrivals at {args.rate}/s, {args.mesh_pool}-mesh "
                                   f"pool log-uniform 10k-2M triangles, durations U[600, 7200] s x {args.time_scale}",
                       "precision": args.precision},
            "throughput": {"value": st["cell_updates"] / wall, "unit": METRIC, "wall_s": wall,
                           "completed": st["completed"]},
            "gpu_launches": None}
    print(json.dumps(line), flush=True)
    return 0


def run_window(args, ws, rank, torch, bm, W):
    """A few steps of the floodplain run from its state at --t-start, in --precision:
    the command profilers capture (a short process, few launches before the captured
    ones).  The state comes from --state-file when that exists (written by an earlier
    run of this command), else from a run from t = 0 on the GPU (saved there if a path
    is given).  Prints the window's time per step and the tiles its launches take."""
    s = W.floodplain()
    st = bm.State.from_scenario(s, precision=args.precision)
    if args.t_start > 0:
        if args.state_file and os.path.exists(args.state_file):
            d = np.load(args.state_file)
            st.upload(d["H"], d["qx"], d["qy"], float(d["t"]))
        else:
            st.run_until(args.t_start)
            if args.state_file:
                H, qx, qy, t = st.download()
                np.savez(args.state_file, H=H, qx=qx, qy=qy, t=t)
    stream = torch.cuda.Stream()
    st.set_stream(stream.cuda_stream)
    st.step(args.warmup)
    st.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.step_async(args.steps)
    e1.record(stream)
    e1.synchronize()
    st.sync()
    taken, total = st.work()
    print(json.dumps({"workload": f"floodplain 2,000,000 triangles, {args.precision}, {args.steps} steps from the "
                                  f"run's state at t = {st.stats(volume=False)['t']:.1f} s",
                      "ms_per_step": e0.elapsed_time(e1) / max(args.steps, 1), "tiles_taken": taken,
                      "tiles": total}))
    return 0


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload != "floodplain":
        import torch
        from paper_2102_12862_b300 import bm
        from paper_2102_12862_b300 import workloads as W
        torch.cuda.set_device(local)
        fn = {"ensemble": run_ensemble, "serve": run_serve, "stress": run_stress, "lake": run_lake,
              "window": run_window}[args.workload]
        return fn(args, ws, rank, torch, bm, W) if rank == 0 or ws == 1 else 0

    import torch
    from paper_2102_12862_b300 import bm
    from paper_2102_12862_b300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")

    s = W.floodplain()
    mesh = bm.Mesh.from_scenario(s)
    precs = [p for p in args.precisions.split(",") if p]
    res, finals = {}, {}
    for p in precs:
        res[p], finals[p] = measure(args, p, s, mesh, torch, bm, dist, ws, rank)

    lake = measure_lake(args, torch, bm, W) if (rank == 0 and args.lake_steps > 0) else None
    ens = (ensemble_leg(args, torch, bm, W, args.ensemble_members, args.steps)
           if (rank == 0 and args.ensemble_members > 0) else None)
    serve = serving_leg(args, torch, bm, W, args.serve_requests) if (rank == 0 and args.serve_requests > 0) else None
    tracking = measure_tracking(args, torch, bm, W) if (rank == 0 and args.track_steps > 0) else None

    cpu, acc = None, {}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        o = oracle.Oracle(s)
        t0 = time.perf_counter()
        o.step(args.e2e_steps)
        dt = time.perf_counter() - t0
        cpu = {"value": s.n_cells * args.e2e_steps / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
               "sample": f"serial FP64 oracle (gcc -O2 -ffp-contract=off), the first {args.e2e_steps} steps of "
                         f"the 2,000,000-cell floodplain from t = 0, {dt:.1f} s wall"}
        for p in precs:
            acc[p] = errors_vs_oracle(s, *finals[p], o)
            acc[p]["steps"] = args.e2e_steps

    if rank == 0:
        main_p = precs[0]
        r = res[main_p]
        windows_desc = r["windows_desc"]
        line = {"metric": METRIC, "value": r["value"], "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if main_p == "fp64" else "f32+f64",
                "data": "synthetic",
                "config": {"workload": f"floodplain 2,000,000 triangles, {main_p.upper()}, the {args.t_end:g} s run: "
                                       f"windows of K steps after {args.warmup} warm-up steps from its states at "
                                       f"t = {windows_desc} s (a GPU run of the same precision made them), value = the run's "
                                       f"{r['steps_run']} steps over their step-weighted time",
                           "cells": s.n_cells, "edges": mesh.info["n_edges"], "precision": main_p,
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                           "l2": "inputs larger than L2 (state and tile records > 126 MB), no flush; the tiles a "
                                 "launch takes stay partly in L2 between steps as in the run itself (l2_flushed: "
                                 "the first and last windows with L2 flushed before every step)",
                           "sim_time_s": args.t_end,
                           "oracle_check_steps": args.e2e_steps},
                "windows": r["windows"], "at_t0": r["windows"][0],
                # FP64 is bound by its FP64 arithmetic (B300: 2 lanes per SM and cycle), FP32-bulk
                # by latency inside tiles; the HBM figure of both is reported beside
                "roofline": r["roofline_fp64"] if main_p == "fp64" else r["roofline"],
                "roofline_hbm": r["roofline"], "l2_flushed": r["l2_flushed"],
                "e2e": r["e2e"], "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "cpu_baseline": cpu,
                "accuracy_vs_oracle": acc.get(main_p)}
        for p in precs[1:]:
            q = res[p]
            key = "fp32_bulk" if p == "fp32" else p
            line[key] = {"value": q["value"], "unit": METRIC, "ms_per_step": q["ms_per_step"],
                         "dtype": "f32+f64" if p == "fp32" else "f64", "windows": q["windows"],
                         "roofline": q["roofline"], "l2_flushed": q["l2_flushed"], "e2e": q["e2e"], "clocks": q["clocks"],
                         "gpu_launches": q["gpu_launches"], "accuracy_vs_oracle": acc.get(p)}
        if ens is not None:
            ens["vs_fp64_plain"] = ens["value"] / r["value"] if main_p == "fp64" else None
            line["ensemble_fp32_bulk"] = ens
        if serve is not None:
            line["serving"] = serve
        if lake is not None:
            line["wet_lake"] = lake
        if tracking is not None:
            line["optional_features"] = tracking
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
