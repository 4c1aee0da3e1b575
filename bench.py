#!/usr/bin/env python3
"""Benchmark of the PP Active Flux MHD stage (arXiv:2506.04857) on GB300.

Metric: FP64 cell-stage updates per second (one cell-stage = one cell's 32
unknowns -- its average and its x-face, y-face and corner point values --
advanced through one SSP-RK3 stage with all limiters), whole job.

Default workload: the low-beta blast on a 2048 x 2048 outflow grid
(gamma = 1.4, p = 1000 inside r < 0.1 else 0.1, |B| = 100/sqrt(4 pi) along
the diagonal, kappa = 1, CFL 0.2), synthetic initial data (af_inputs).  A step
is one SSP-RK3 step: dt reduction plus three limited stages.  One state is
1.07 GB, far larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--workload blast2048|ot512|vortex64]
  python bench.py --impl reference ...   (the CPU oracle on the host cores)

Under torchrun (N > 1) each rank advances its own copy of the workload (the
path has no exchange between independent runs): weak scaling, max-over-ranks
time.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import af_inputs as ai  # noqa: E402

WORKLOADS = {
    "blast2048": ("low-beta blast 2048x2048 outflow, kappa=1", lambda: ai.blast(2048)),
    "blast512": ("low-beta blast 512x512 outflow, kappa=1 (profiling size)", lambda: ai.blast(512)),
    "blast1024": ("low-beta blast 1024x1024 outflow, kappa=1 (profiling size)", lambda: ai.blast(1024)),
    "ot512": ("Orszag-Tang 512x512 periodic, kappa=1", lambda: ai.orszag_tang(512)),
    "vortex64": ("smooth vortex 64x64 periodic, kappa=0", lambda: ai.vortex(64)),
    "ensemble256": ("256 seeded Orszag-Tang runs, nx, ny drawn from {64,128,256,512}, kappa=1, one batch",
                    lambda: ai.orszag_tang(64)),
    "adjoint256": ("discrete adjoint: 256x256 perturbed vortex, kappa=0, 200 steps, checkpoints every 20",
                   lambda: ai.perturbed_vortex(256, seed=0)),
    "jets1024": ("MHD jets (Example 4.8) 1024x3072: left half, reflective at x=0, Mach-800 inflow jet at the "
                 "bottom, B_a=sqrt(20000), kappa=2", lambda: ai.jets(1024)),
    "jets512": ("MHD jets 512x1536 (profiling size of the jets)", lambda: ai.jets(512)),
    "blast1d": ("1D strong blast (p = 1000 / 0.1, B = (100/sqrt(4pi))(1,1,0)/sqrt(2)) on 4,194,304 cells, "
                "outflow, kappa=1", lambda: ai.blast1d(1 << 22)),
    "divb2048": ("divergence measures (Example 4.4) of the 2048x2048 low-beta blast after 3 steps",
                 lambda: ai.blast(2048)),
    "divb512": ("divergence measures (Example 4.4) of the 512x512 low-beta blast after 3 steps (profiling size)",
                lambda: ai.blast(512)),
    "lattice2048": ("rarefaction lattice 2048x2048 periodic (v = 6 (sgn sin 128 pi x, sgn sin 128 pi y), rho = 1, "
                    "p = 0.4, B = (0, 0.5, 0), gamma = 1.4), kappa=1: every positivity limiter and the Newton "
                    "solve act in each stage", lambda: ai.rarefaction_lattice(2048, periods=64)),
    "lattice512": ("rarefaction lattice 512x512, 16 periods (profiling size)",
                   lambda: ai.rarefaction_lattice(512, periods=16)),
}

# Algorithmic FP64 flops per cell-stage of each kernel: the arithmetic of the
# scheme as the paper writes it, with the PP limiters off (their tests and
# occasional blends are extra work, not counted), counted by the counting
# build of the oracle: python -m oracle.count_flops (64x64 grids, the jets on
# 256x768, the 1D blast on 4096 cells; +, -, *, /, sqrt, exp, min/max, |.| one
# flop each).
ALGO_FLOPS = {
    "blast_low_beta": {"k_pointdata": 714.9, "k_points": 1294.8, "k_faces": 253.9, "k_cells": 628.0, "k_final": 16.3},
    "orszag_tang": {"k_pointdata": 708.0, "k_points": 1267.0, "k_faces": 250.0, "k_cells": 628.0, "k_final": 16.0},
    "vortex": {"k_pointdata": 708.0, "k_points": 1267.0, "k_faces": 234.0, "k_cells": 468.0, "k_final": 16.0},
    "rarefaction_lattice": {"k_pointdata": 708.5, "k_points": 1267.0, "k_faces": 250.0, "k_cells": 628.0,
                            "k_final": 16.0},
    "jets": {"k_pointdata": 720.7, "k_points": 1271.6, "k_faces": 250.7, "k_cells": 628.0, "k_final": 16.1},
    "blast1d": {"k1_pointdata": 432.4, "k1_points": 332.1, "k1_faces": 93.0, "k1_cells": 96.0, "k1_final": 16.0},
}
# Flops per cell of the two divergence measures (af_divb), same counter.
ALGO_FLOPS_DIVB = {"blast_low_beta": 414.0}
# Executed FP64 arithmetic per cell of one af_divb call (k_divb; the one-block sum is
# negligible), from the capture named in "source"; filled in below EXEC_FP64.
EXEC_FP64_DIVB = {}
# Executed FP64 arithmetic per cell-stage of each stage kernel: DADD, DMUL and DFMA
# thread instructions (ncu sm__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on.sum)
# of one captured step, divided by the cell-stages of that step.  Flops = DADD + DMUL +
# 2 DFMA: the arithmetic the FP64 pipe executes, which is what the FP64 peak bounds.
# The kernels run part of their binary64 products and sums on the integer pipes
# (mul_i, sub_i: bitwise the IEEE results, no FP64 instruction); int_mul and int_add
# count them per cell-stage, as the DMUL and DADD counts of the same captures on the
# build that ran every product on the FP64 pipe (kernel digest e1110cc7...) minus those
# of the build that first moved them (before the FP32 certificates, which remove FP64
# work outright): a lower bound, since later changes moved a few more operations.  The literal count of the paper's formulas (ALGO_FLOPS) is larger where a
# kernel uses a cheaper algebraic form (the LLF-FVS line as one expression, products
# by 1/h), so it is reported beside the roofline, never divided by the peak.  Each
# table names the capture it comes from and a digest of the kernel sources it was
# taken on: once the kernels change, the line says so ("counts_stale") until the
# capture is retaken.  The work-list kernels of the limiter slow paths are summed as
# k_points_slow and k_cells_slow (the box and the Newton pass), the names af_timing
# reports them under.
EXEC_FP64 = {
    "blast_low_beta": {"source": "profiles/fp64ops_stage_kernels.md", "digest": "7013560c17a537ed1abec9766d30c1192bfdcd19", "kernels": {
        "k_pointdata": {"dadd": 93.04, "dmul": 0.01, "dfma": 183.15, "pipe": 276.19, "dram_bytes": 1119.0, "int_mul": 124.09, "int_add": 0.00},
        "k_points": {"dadd": 155.22, "dmul": 8.01, "dfma": 222.38, "pipe": 385.60, "dram_bytes": 1946.1, "int_mul": 40.06, "int_add": 0.00},
        "k_points_slow": {"dadd": 0.14, "dmul": 0.19, "dfma": 0.39, "pipe": 0.74, "dram_bytes": 1.9, "int_mul": 0.02, "int_add": 0.00},
        "k_faces": {"dadd": 74.11, "dmul": 5.95, "dfma": 52.36, "pipe": 134.39, "dram_bytes": 744.0, "int_mul": 44.08, "int_add": 0.00},
        "k_cells": {"dadd": 58.01, "dmul": 3.00, "dfma": 122.02, "pipe": 183.03, "dram_bytes": 1224.2, "int_mul": 51.00, "int_add": 0.00},
        "k_cells_slow": {"dadd": 0.06, "dmul": 0.18, "dfma": 0.20, "pipe": 0.54, "dram_bytes": 0.8, "int_mul": 0.00, "int_add": 0.00},
        "k_final": {"dadd": 0.00, "dmul": 0.00, "dfma": 21.33, "pipe": 21.33, "dram_bytes": 329.5, "int_mul": 8.33, "int_add": 16.00},
    }},
    "orszag_tang": {"source": "profiles/fp64ops_stage_kernels.md", "digest": "7013560c17a537ed1abec9766d30c1192bfdcd19", "kernels": {
        "k_pointdata": {"dadd": 93.00, "dmul": 0.00, "dfma": 183.00, "pipe": 276.00, "dram_bytes": 948.2, "int_mul": 124.00, "int_add": 0.00},
        "k_points": {"dadd": 156.00, "dmul": 8.00, "dfma": 228.00, "pipe": 392.00, "dram_bytes": 1803.4, "int_mul": 42.00, "int_add": 0.00},
        "k_points_slow": {"dadd": 0.00, "dmul": 0.00, "dfma": 0.00, "pipe": 0.00, "dram_bytes": 0.2, "int_mul": 0.00, "int_add": 0.00},
        "k_faces": {"dadd": 74.00, "dmul": 0.00, "dfma": 74.00, "pipe": 148.00, "dram_bytes": 637.8, "int_mul": 46.00, "int_add": 0.00},
        "k_cells": {"dadd": 58.00, "dmul": 3.00, "dfma": 122.00, "pipe": 183.00, "dram_bytes": 1073.7, "int_mul": 51.00, "int_add": 0.00},
        "k_cells_slow": {"dadd": 0.00, "dmul": 0.00, "dfma": 0.00, "pipe": 0.00, "dram_bytes": 0.3, "int_mul": 0.00, "int_add": 0.00},
        "k_final": {"dadd": 0.00, "dmul": 0.00, "dfma": 21.33, "pipe": 21.33, "dram_bytes": 277.4, "int_mul": 8.33, "int_add": 16.00},
    }},
    "jets": {"source": "profiles/fp64ops_stage_kernels.md", "digest": "7013560c17a537ed1abec9766d30c1192bfdcd19", "kernels": {
        "k_pointdata": {"dadd": 93.05, "dmul": 0.00, "dfma": 183.17, "pipe": 276.21, "dram_bytes": 1098.4, "int_mul": 124.13, "int_add": 0.00},
        "k_points": {"dadd": 189.44, "dmul": 8.27, "dfma": 222.40, "pipe": 420.13, "dram_bytes": 2399.5, "int_mul": 39.14, "int_add": 0.00},
        "k_points_slow": {"dadd": 0.02, "dmul": 0.02, "dfma": 0.05, "pipe": 0.10, "dram_bytes": 0.2, "int_mul": 0.00, "int_add": 0.00},
        "k_faces": {"dadd": 83.13, "dmul": 6.02, "dfma": 52.13, "pipe": 143.30, "dram_bytes": 723.8, "int_mul": 44.08, "int_add": 0.00},
        "k_cells": {"dadd": 58.52, "dmul": 3.00, "dfma": 122.01, "pipe": 183.54, "dram_bytes": 1212.2, "int_mul": 51.00, "int_add": 0.00},
        "k_cells_slow": {"dadd": 0.03, "dmul": 0.09, "dfma": 0.10, "pipe": 0.27, "dram_bytes": 0.2, "int_mul": 0.00, "int_add": 0.00},
        "k_final": {"dadd": 0.00, "dmul": 0.00, "dfma": 21.33, "pipe": 21.33, "dram_bytes": 322.2, "int_mul": 8.33, "int_add": 16.00},
    }},
    "rarefaction_lattice": {"source": "profiles/fp64ops_stage_kernels.md", "digest": "7013560c17a537ed1abec9766d30c1192bfdcd19", "kernels": {
        "k_pointdata": {"dadd": 93.50, "dmul": 1.87, "dfma": 187.23, "pipe": 283.05, "dram_bytes": 942.7, "int_mul": 124.00, "int_add": 0.00},
        "k_points": {"dadd": 156.00, "dmul": 8.00, "dfma": 228.80, "pipe": 392.77, "dram_bytes": 1865.1, "int_mul": 39.81, "int_add": 0.00},
        "k_points_slow": {"dadd": 49.23, "dmul": 68.69, "dfma": 141.61, "pipe": 271.05, "dram_bytes": 529.2, "int_mul": 6.84, "int_add": 0.00},
        "k_faces": {"dadd": 74.00, "dmul": 0.57, "dfma": 75.13, "pipe": 149.66, "dram_bytes": 637.8, "int_mul": 46.00, "int_add": 0.00},
        "k_cells": {"dadd": 64.34, "dmul": 4.36, "dfma": 136.73, "pipe": 206.08, "dram_bytes": 1092.5, "int_mul": 51.00, "int_add": 0.00},
        "k_cells_slow": {"dadd": 44.31, "dmul": 54.71, "dfma": 233.66, "pipe": 347.47, "dram_bytes": 321.6, "int_mul": 0.00, "int_add": 0.00},
        "k_final": {"dadd": 0.00, "dmul": 2.86, "dfma": 24.20, "pipe": 27.05, "dram_bytes": 277.8, "int_mul": 8.33, "int_add": 13.14},
    }},
    "blast1d": {"source": "profiles/fp64ops_stage_kernels.md", "digest": "8915d37b6cf721a281ba9d891fc8e24ab5bd1867", "kernels": {
        "k1_pointdata": {"dadd": 31.00, "dmul": 8.00, "dfma": 106.00, "pipe": 145.00, "dram_bytes": 667.8, "int_mul": 76.00, "int_add": 0.00},
        "k1_points": {"dadd": 41.00, "dmul": 9.33, "dfma": 55.33, "pipe": 107.67, "dram_bytes": 430.6, "int_mul": 9.00, "int_add": 0.00},
        "k1_faces": {"dadd": 30.00, "dmul": 20.00, "dfma": 19.00, "pipe": 72.00, "dram_bytes": 358.9, "int_mul": 4.00, "int_add": 0.00},
        "k1_cells": {"dadd": 9.00, "dmul": 19.00, "dfma": 8.00, "pipe": 37.00, "dram_bytes": 289.9, "int_mul": 10.00, "int_add": 0.00},
        "k1_final": {"dadd": 0.00, "dmul": 14.33, "dfma": 28.33, "pipe": 45.67, "dram_bytes": 252.5, "int_mul": 3.00, "int_add": 0.00},
    }},
}
EXEC_FP64_DIVB["blast_low_beta"] = {"source": "profiles/divb_blast512.md", "digest": "7013560c17a537ed1abec9766d30c1192bfdcd19",
                                     "dadd": 67.99, "dmul": 19.01, "dfma": 57.03, "pipe": 143.98}
# FP64 roofline from unit counts and clock: the GB300 SM retires 2 DFMA thread
# instructions per cycle (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
# peak_sustained = 2 / SM / cycle), i.e. 4 flops per SM-cycle.
FP64_FLOPS_PER_SM_CYCLE = 4.0
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one k_points
# launch per cell, from one ncu capture of the 1024x1024 low-beta blast
# (1.031 GB read + 0.255 GB written for 1,048,576 cells); the 2048x2048 launch
# is taken as 4x that (the kernel's traffic is per cell: its own and its
# neighbours' point data).
DRAM_BYTES_PER_CELL = {"k_points": 1226.0}
# Stage work arrays of a 2D context per index point (point data of the four
# classes and the centres, centre values, sensor, face data, Lambda, Lim1, face theta).
WORK_DOUBLES_PER_CELL = 163
# Algorithmic bytes per cell-stage: read U^(s) (32 doubles), read U^n on stages
# 2 and 3, write U^(s+1): (512 + 768 + 768)/3 B.
ALGO_BYTES_PER_CS = (512.0 + 768.0 + 768.0) / 3.0


# Kernels launched on the library's second stream, concurrently with the main stream's.
SIDE_STREAM_KERNELS = ("k_points_slow",)

KERNEL_FILES_2D = ("af_kernels.cu", "af_math.cuh", "af_device.cuh", "af_internal.h")
KERNEL_FILES_1D = ("af_kernels1d.cuh", "af_math.cuh", "af_device.cuh", "af_internal.h")


def kernel_digest(files=KERNEL_FILES_2D) -> str:
    """sha1 of the CUDA sources that define a workload's stage kernels, in the given order."""
    import hashlib
    d = os.path.join(ROOT, "paper_2506_04857_gb300", "csrc")
    h = hashlib.sha1()
    for name in files:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def exec_flops(name: str):
    """{kernel: FP64-pipe flops per cell-stage}, {kernel: integer-pipe flops per
    cell-stage}, the capture's source, and whether the kernels changed since the
    capture (None, None, None when no capture covers the workload)."""
    t = EXEC_FP64.get(name)
    if t is None:
        return None, None, None, None
    fl = {k: v["dadd"] + v["dmul"] + 2.0 * v["dfma"] for k, v in t["kernels"].items()}
    fi = {k: v.get("int_mul", 0.0) + v.get("int_add", 0.0) for k, v in t["kernels"].items()}
    files = KERNEL_FILES_1D if name == "blast1d" else KERNEL_FILES_2D
    return fl, fi, t["source"], kernel_digest(files) != t["digest"]


def fp64_roofline(name, ktimes, cells_per_launch, units_timed, ms_timed, peak, peak_src, probe, world=1):
    """Roofline of the dominant stage kernel and of the whole step on executed FP64 flops
    (bound: the FP64 ALU pipe).  ktimes: {kernel: (total ms, launches)} of the timed region.
    achieved / frac count the flops the FP64 pipe executed; work_* add the binary64
    products and sums the kernels ran on the integer pipes (the same arithmetic, other
    hardware), so work_frac may exceed the FP64 pipe's share of the peak."""
    lit = ALGO_FLOPS.get(name, {})
    fl, fi, src, stale = exec_flops(name)
    known = fl if fl is not None else lit
    dom = max((k for k in ktimes if k in known and k not in SIDE_STREAM_KERNELS), key=lambda k: ktimes[k][0])
    dom_ms, dom_n = ktimes[dom]
    avg_s = dom_ms / max(dom_n, 1) * 1e-3
    # shares of the library stream's serial time; a kernel on the second stream runs beside
    # the face and cell passes, so its event time is wall time shared with them
    tot = sum(v[0] for k, v in ktimes.items() if k not in SIDE_STREAM_KERNELS)
    r = {"bound": "alu", "kernel": dom, "unit": "TFLOP/s", "peak": peak, "peak_source": peak_src,
         "probe_fp64_tflops": probe,
         "kernel_time_share": {k: round(v[0] / tot, 4) for k, v in ktimes.items()
                               if v[1] and k not in SIDE_STREAM_KERNELS},
         "overlapped_kernel_time": {k: round(v[0] / tot, 4) for k, v in ktimes.items()
                                    if v[1] and k in SIDE_STREAM_KERNELS},
         "literal_flops_per_cell_stage": lit.get(dom), "literal_flops_per_cell_stage_all_kernels": sum(lit.values()),
         "literal_note": "the paper's formulas counted as written (oracle counting build, PP limiters off); "
                         "context only, not divided by the peak"}
    if fl is None:
        r.update({"achieved": None, "frac": None, "executed_counts": None})
        return r
    achieved = fl[dom] * cells_per_launch / avg_s * 1e-12
    work = (fl[dom] + fi[dom]) * cells_per_launch / avg_s * 1e-12
    step_tf = sum(fl.values()) * units_timed / (ms_timed * 1e-3) * 1e-12 / world
    step_work = (sum(fl.values()) + sum(fi.values())) * units_timed / (ms_timed * 1e-3) * 1e-12 / world
    pipe = EXEC_FP64[name]["kernels"][dom].get("pipe")
    if pipe is not None:   # FP64-pipe thread instructions per second against 2 per SM per cycle (= peak / 2 flops)
        r["fp64_pipe_busy"] = pipe * cells_per_launch / avg_s / (peak * 1e12 / 2.0)
    r.update({"achieved": achieved, "frac": achieved / peak, "frac_of_probe": achieved / probe if probe else None,
              "executed_flops_per_cell_stage": fl[dom], "executed_flops_per_cell_stage_all_kernels": sum(fl.values()),
              "int_pipe_flops_per_cell_stage": fi[dom], "int_pipe_flops_per_cell_stage_all_kernels": sum(fi.values()),
              "work_achieved": work, "work_frac": work / peak,
              "executed_counts": src, "counts_stale": stale,
              "step_achieved_tflops": step_tf, "step_frac": step_tf / peak,
              "step_frac_of_probe": step_tf / probe if probe else None,
              "step_work_tflops": step_work, "step_work_frac": step_work / peak})
    return r


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of the ranks' values of x (a job's time is that of its
    slowest rank); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_runs(cells, rank: int, world: int):
    """Indices of the ensemble runs that `rank` advances: a greedy
    longest-processing-time partition by cell count (largest run first, to
    the least loaded rank; ties by index), the same on every rank."""
    order = sorted(range(len(cells)), key=lambda r: (-cells[r], r))
    load = [0] * world
    owner = [0] * len(cells)
    for r in order:
        k = min(range(world), key=lambda q: (load[q], q))
        owner[r] = k
        load[k] += cells[r]
    return [r for r in range(len(cells)) if owner[r] == rank]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def window_problem(pb, i0, j0, w):
    """A w x w window of cells of pb as an outflow sub-problem (for the CPU oracle)."""
    import dataclasses
    return dataclasses.replace(pb, nx=w, ny=w, x0=pb.x0 + i0 * pb.dx, x1=pb.x0 + (i0 + w) * pb.dx,
                               y0=pb.y0 + j0 * pb.dy, y1=pb.y0 + (j0 + w) * pb.dy, bc=ai.OUTFLOW)


def cpu_sample_problem(key, pb, w):
    """The bounded CPU sample of a workload: a w x w window on its most active region."""
    if key.startswith("jets"):
        sub = ai.jets(128)
        return sub, "the jets problem at %dx%d with its own sides" % (sub.nx, sub.ny)
    if key.startswith("blast"):
        # window straddling the blast front (radius 0.1 = 204.8 cells from the centre)
        c = pb.nx // 2
        w = min(w, pb.nx)
        r = int(round(0.1 / pb.dx))
        i0, j0 = min(pb.nx - w, c + r - w // 2), c - w // 2
    else:
        i0 = j0 = 0
        w = min(w, pb.nx)
    if w >= pb.nx and w >= pb.ny and pb.bc != ai.OUTFLOW:
        return pb, "the whole %dx%d workload" % (pb.nx, pb.ny)
    sub = window_problem(pb, i0, j0, w)
    desc = "%dx%d window [%d:%d, %d:%d] of the %dx%d workload as an outflow sub-problem" % (
        w, w, i0, i0 + w, j0, j0 + w, pb.nx, pb.ny)
    return sub, desc


def threads_used():
    try:
        n = int(os.environ.get("OMP_NUM_THREADS", "0"))
    except ValueError:
        n = 0
    return n if n > 0 else len(os.sched_getaffinity(0))


def run_oracle_steps(sub, steps, budget_s=None):
    import oracle
    U = ai.dofs(sub)
    t0 = time.perf_counter()
    done = 0
    for _ in range(steps):
        U, _ = oracle.step(sub, U)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    return done, time.perf_counter() - t0


def cpu_unit(key, pb, w):
    """The oracle's bounded sample of a workload: (one call, units per call,
    metric, unit, description)."""
    import oracle
    oracle.build()
    if key == "blast1d":
        sub = ai.blast1d(1 << 16, kappa=pb.kappa)
        st = [ai.dofs1(sub)]

        def run():
            st[0], _ = oracle.step1(sub, st[0])
        return (run, sub.n * 3, "FP64 AF-MHD 1D cell-stage updates/s", "cell-stage updates/s",
                "the same blast on %d cells, one SSP-RK3 step per call" % sub.n)
    if key.startswith("divb"):
        sub, d = cpu_sample_problem("blast", pb, w)
        V = ai.dofs(sub)
        return (lambda: oracle.divb(sub, V), sub.nx * sub.ny, "FP64 divergence-measure cell evaluations/s",
                "cell evaluations/s", d + " (initial state), both measures per call")
    sub, d = cpu_sample_problem(key, pb, w)
    st = [ai.dofs(sub)]

    def run():
        st[0], _ = oracle.step(sub, st[0])
    return run, sub.nx * sub.ny * 3, "FP64 AF-MHD cell-stage updates/s", "cell-stage updates/s", \
        d + ", one SSP-RK3 step per call"


def cpu_rate(key, pb, budget_s, w):
    run, units, _, unit, desc = cpu_unit(key, pb, w)
    run()   # warm-up (first-touch, thread pool)
    t0, n = time.perf_counter(), 0
    while n < 1000 and time.perf_counter() - t0 < budget_s:
        run()
        n += 1
    t = time.perf_counter() - t0
    return {"value": units * n / t, "unit": unit, "cores": threads_used(), "kind": "oracle",
            "sample": "%s: %d calls in %.1f s" % (desc, n, t)}


def cpu_baseline(key, pb, budget_s=12.0, w=512):
    """The oracle, as it stands, timed on the host cores on a bounded sample,
    and on one core (a child process with OMP_NUM_THREADS=1, a 128-cell-wide
    sample for about 8 s)."""
    res = cpu_rate(key, pb, budget_s, w)
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--workload", key, "--cpu-rate-only"],
                             env=env, capture_output=True, text=True, timeout=120)
        res["single_thread"] = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:   # the multi-core figure stands alone
        res["single_thread"] = {"unavailable": str(e)[:200]}
    return res


def reference_arm(args, key, desc, pb):
    """--impl reference: the CPU oracle on the host cores (the paper ships no code)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if key == "adjoint256":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no backward pass to time (its "
                          "complex-step build differentiates the forward step), so no adjoint/forward ratio"}),
              flush=True)
        return 0
    run, units, metric, unit, sdesc = cpu_unit(key, pb, 128)
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    t = time.perf_counter() - t0
    value = units * args.steps / t
    cells = pb.n if hasattr(pb, "n") else pb.nx * pb.ny
    line = {"metric": metric, "value": value, "unit": unit,
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "cells": cells, "sample": sdesc},
            "cpu_baseline": {"value": value, "unit": unit, "cores": threads_used(),
                             "kind": "oracle", "sample": "%s, one call per timed step" % sdesc},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if hasattr(pb, "nx"):
        line["config"]["nx"], line["config"]["ny"] = pb.nx, pb.ny
    print(json.dumps(line), flush=True)
    return 0


def ensemble_cost(stream, steps=3, warm=3):
    """The batched ensemble (256 seeded Orszag-Tang runs, nx, ny drawn from {64, 128, 256,
    512}) against the plain per-run loop on the same GPU, one rank: aggregate cell-stage
    updates/s of each, after the autotuner; the batch replays a 3-step CUDA graph."""
    import torch
    import paper_2506_04857_gb300 as af
    every = ai.ot_ensemble(256, seed=0)
    cells = sum(p.nx * p.ny for p in every)
    states = [ai.dofs(p) for p in every]
    with torch.cuda.stream(stream):
        b = af.af_batch_create([p.nx for p in every], [p.ny for p in every], [p.gamma for p in every],
                               [p.bc for p in every])
        af.af_batch_set_stream(b, stream)
        for r, (p, U) in enumerate(zip(every, states)):
            af.af_batch_set_domain(b, r, p.x0, p.x1, p.y0, p.y1)
            af.af_batch_set_params(b, r, cfl=p.cfl, kappa=p.kappa)
            af.af_batch_set_state(b, r, U)
        choice = af.af_batch_autotune(b, reps=2)
        af.af_batch_graph(b, True)
        af.af_batch_step(b, warm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        af.af_batch_step(b, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_batch = e0.elapsed_time(e1)
        rc, cnt = af.af_batch_status(b, reset=True)
        if rc != af.AF_OK:
            raise SystemExit("batch: " + af.af_batch_last_error(b))
        af.af_batch_destroy(b)
        solvers = []
        for p, U in zip(every, states):
            sv = af.Solver(p.nx, p.ny, p.gamma, p.bc, domain=(p.x0, p.x1, p.y0, p.y1), cfl=p.cfl, kappa=p.kappa,
                           stream=stream)
            sv.set_state(U)
            solvers.append(sv)
        for _ in range(warm):
            for sv in solvers:
                sv.step(dt_out=False)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            for sv in solvers:
                sv.step(dt_out=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_loop = e0.elapsed_time(e1)
        for sv in solvers:
            sv.close()
    v_batch = cells * 3 * steps / (ms_batch * 1e-3)
    v_loop = cells * 3 * steps / (ms_loop * 1e-3)
    return {"workload": WORKLOADS["ensemble256"][0], "runs": len(every), "cells": cells, "steps": steps,
            "warmup": warm, "batched": v_batch, "plain_loop": v_loop, "batched_over_loop": v_batch / v_loop,
            "unit": "cell-stage updates/s", "autotune": choice, "graph": True,
            "launches_per_step": {"batched": 19, "plain_loop": 19 * len(every)}}


def ensemble_bench(args, desc):
    """The batched ensemble against the plain per-run loop on the same GPU.
    Under torchrun the runs are sharded over the ranks (shard_runs; no data
    exchange) and the job's time is that of the slowest rank."""
    import torch
    import paper_2506_04857_gb300 as af

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    every = ai.ot_ensemble(256, seed=0)
    total_cells = sum(p.nx * p.ny for p in every)
    pbs = [every[r] for r in shard_runs([p.nx * p.ny for p in every], rank, world)]
    states = [ai.dofs(p) for p in pbs]
    cells = sum(p.nx * p.ny for p in pbs)
    steps = max(3, (args.steps + 2) // 3 * 3)
    warm = max(3, (args.warmup + 2) // 3 * 3)
    with torch.cuda.stream(stream):
        # batched: one persistent launch per pass for all runs, 3-step graph, autotuned tiles
        b = af.af_batch_create([p.nx for p in pbs], [p.ny for p in pbs], [p.gamma for p in pbs],
                               [p.bc for p in pbs])
        af.af_batch_set_stream(b, stream)
        for r, (p, U) in enumerate(zip(pbs, states)):
            af.af_batch_set_domain(b, r, p.x0, p.x1, p.y0, p.y1)
            af.af_batch_set_params(b, r, cfl=p.cfl, kappa=p.kappa)
            af.af_batch_set_state(b, r, U)
        choice = af.af_batch_autotune(b, reps=2)
        af.af_batch_graph(b, True)
        af.af_batch_step(b, warm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        af.af_batch_step(b, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_batch = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        rc, cnt = af.af_batch_status(b, reset=True)
        if rc != af.AF_OK:
            raise SystemExit("batch: " + af.af_batch_last_error(b))
        af.af_batch_destroy(b)
        # plain loop: one af_ctx per run, stepped one after the other on the same stream
        solvers = []
        for p, U in zip(pbs, states):
            sv = af.Solver(p.nx, p.ny, p.gamma, p.bc, domain=(p.x0, p.x1, p.y0, p.y1), cfl=p.cfl, kappa=p.kappa,
                           stream=stream)
            sv.set_state(U)
            solvers.append(sv)
        for _ in range(warm):
            for sv in solvers:
                sv.step(dt_out=False)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            for sv in solvers:
                sv.step(dt_out=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_loop = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        for sv in solvers:
            sv.close()
    v_batch = total_cells * 3 * steps / (ms_batch * 1e-3)
    v_loop = total_cells * 3 * steps / (ms_loop * 1e-3)
    line = {"metric": "FP64 AF-MHD cell-stage updates/s", "value": v_batch, "unit": "cell-stage updates/s",
            "n_gpus": world, "steps": steps, "warmup": warm, "ms_per_step": ms_batch / steps,
            "higher_is_better": True, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "runs": len(every), "cells": total_cells, "seed": 0,
                       "runs_per_rank": len(pbs), "sharding": "runs over ranks, greedy by cells"},
            "batched": {"value": v_batch, "autotune": choice, "graph": True, "launches_per_step": 19},
            "plain_loop": {"value": v_loop, "ms_per_step": ms_loop / steps, "launches_per_step": 19 * len(pbs)},
            "batched_over_loop": v_batch / v_loop, "limiter_counters": cnt}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def limiter_cost(s, pb, stream, cnt, steps, reps=6):
    """What the positivity limiters cost while they act: the first stage of the current
    state (the state the timed region ended with) run `reps` times with the PP limiters on
    and `reps` times with them off (same input, same dt), per-kernel times from af_timing.
    The difference is the limiter work (the point LLF states and scaling limiter in
    k_points, the LLF update, source limiter, 16-vertex box and Newton solves in k_cells,
    the face theta and admissibility test in k_final).  Per limited cell: the k_cells
    difference over the cells with some Lambda_I < 1 in one such stage."""
    import paper_2506_04857_gb300 as af
    U = s.get_state()
    dt = s.dt()
    res = {}
    for pp in (True, False):
        af.af_set_params(s.ctx, pb.cfl, pb.kappa, pp)
        s.set_state(U)
        s.stage(0, dt)            # warm-up
        s.status(reset=True)
        s.timing(True)
        for _ in range(reps):
            s.set_state(U)
            s.stage(0, dt)
        kt = s.timing(False)
        rc, c = s.status(reset=True)
        res[pp] = ({k: v[0] / max(v[1], 1) for k, v in kt.items() if v[1]}, c)
    af.af_set_params(s.ctx, pb.cfl, pb.kappa, True)
    s.set_state(U)
    on, c_on = res[True]
    off, _ = res[False]
    lam_cells = c_on["lambda_lt1"] / reps
    out = {"stage_input": "the state after the timed region, first stage, %d repetitions each way" % reps,
           "ms_per_launch_pp_on": {k: round(v, 4) for k, v in on.items()},
           "ms_per_launch_pp_off": {k: round(v, 4) for k, v in off.items()},
           "cells_lambda_lt1_per_stage": lam_cells,
           "newton_solves_per_stage": c_on["newton_solves"] / reps,
           "points_limited_per_stage": c_on["point_limited"] / reps,
           "faces_theta_lt1_per_stage": c_on["face_theta_lt1"] / reps,
           "timed_region_counters_per_stage": {k: v / (3 * steps) for k, v in cnt.items()
                                               if k not in ("newton_maxit",)}}
    stage_on = sum(v for k, v in on.items() if k not in ("k_dt",))
    stage_off = sum(v for k, v in off.items() if k not in ("k_dt",))
    out["limiter_share_of_stage"] = (stage_on - stage_off) / stage_on
    # the cell limiter: k_cells and its list passes (box, Newton, count), over the cells
    # with some Lambda_I < 1; the point limiter: k_points and its list pass, over the
    # points the scaling limiter changed
    cell_extra = on.get("k_cells", 0.0) + on.get("k_cells_slow", 0.0) - off.get("k_cells", 0.0)
    point_extra = on.get("k_points", 0.0) + on.get("k_points_slow", 0.0) - off.get("k_points", 0.0)
    out["cell_limiter_ms_per_stage"] = cell_extra
    out["point_limiter_ms_per_stage"] = point_extra
    if lam_cells > 0:
        out["cell_limiter_ns_per_cell_lambda_lt1"] = cell_extra * 1e6 / lam_cells
    if out["points_limited_per_stage"] > 0:
        out["point_limiter_ns_per_limited_point"] = point_extra * 1e6 / out["points_limited_per_stage"]
    return out


def adjoint_cost(stream, nsteps=200, every=20):
    """Wall-time ratio backward / forward of the differentiable solve on the
    adjoint workload: 256x256 perturbed vortex (kappa = 0), 200 SSP-RK3 steps,
    checkpoints every 20 steps, objective the total magnetic energy.  The
    backward pass includes the recomputation of every segment from its
    checkpoint and the stage recomputation inside each adjoint step."""
    import torch
    import paper_2506_04857_gb300 as af
    from paper_2506_04857_gb300.adjoint import af_steps, magnetic_energy
    pb = ai.perturbed_vortex(256, seed=0)
    s = af.Solver(pb.nx, pb.ny, pb.gamma, pb.bc, domain=(pb.x0, pb.x1, pb.y0, pb.y1), cfl=pb.cfl, kappa=0.0,
                  stream=stream)
    U0 = [torch.from_numpy(u).cuda() for u in ai.dofs(pb)]

    def once(n, sens=False):
        X0 = [t.clone().requires_grad_(True) for t in U0]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        out = af_steps(s, X0, n, checkpoint_every=every, dt_sensitivity=sens)
        ev[1].record(stream)
        J = magnetic_energy(out, pb.dx, pb.dy, pb.bc)
        ev[2].record(stream)
        J.backward()
        ev[3].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])

    once(2 * every)                   # warm-up (first adjoint call allocates its workspace)
    fwd, bwd = once(nsteps)
    fwd_s, bwd_s = once(nsteps, sens=True)   # dt differentiated through its formula
    s.close()
    return {"workload": "256x256 perturbed MHD vortex (random Fourier |k|<=4, amplitude 1e-3 of rho and B), "
                        "kappa=0, %d steps, checkpoints every %d steps, objective total magnetic energy" % (nsteps, every),
            "forward_ms": fwd, "backward_ms": bwd, "forward_ms_per_step": fwd / nsteps,
            "adjoint_ms_per_step": bwd / nsteps, "ratio": bwd / fwd,
            "target": "<= 4", "includes": "segment recompute from checkpoints (stage states kept) + point data of 3 stage states + 3 VJPs",
            "dt_sensitivity": {"forward_ms": fwd_s, "backward_ms": bwd_s, "ratio": bwd_s / fwd_s,
                               "includes": "as above + U3 kept + the mu dt reduction and the argmax gradient"}}


def adjoint_limited_cost(stream, nsteps=40, every=20):
    """The same ratio on a limited run: the low-beta blast 256x256 (kappa = 1; the point,
    centre and flux limiters act at the front), 40 steps, checkpoints every 20.  The
    backward pass records every step's limiter coefficients while it recomputes a segment
    and applies af_adjoint_step_frozen (the gradient along the branch the forward pass took)."""
    import torch
    import paper_2506_04857_gb300 as af
    from paper_2506_04857_gb300.adjoint import af_steps, magnetic_energy
    pb = ai.blast(256)
    s = af.Solver(pb.nx, pb.ny, pb.gamma, pb.bc, domain=(pb.x0, pb.x1, pb.y0, pb.y1), cfl=pb.cfl, kappa=pb.kappa,
                  stream=stream)
    U0 = [torch.from_numpy(u).cuda() for u in ai.dofs(pb)]

    def once(n):
        X0 = [t.clone().requires_grad_(True) for t in U0]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        out = af_steps(s, X0, n, checkpoint_every=every)
        ev[1].record(stream)
        J = magnetic_energy(out, pb.dx, pb.dy, pb.bc)
        ev[2].record(stream)
        J.backward()
        ev[3].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])

    once(every)   # warm-up
    s.status(reset=True)
    fwd, bwd = once(nsteps)
    rc, cnt = s.status(reset=True)
    s.close()
    return {"workload": "256x256 low-beta blast, kappa=1, %d steps, checkpoints every %d steps, objective total "
                        "magnetic energy, limiters active" % (nsteps, every),
            "forward_ms": fwd, "backward_ms": bwd, "forward_ms_per_step": fwd / nsteps,
            "adjoint_ms_per_step": bwd / nsteps, "ratio": bwd / fwd,
            "includes": "segment recompute recording the limiter coefficients + point data of 3 stage states + "
                        "3 frozen-branch VJPs",
            "limiter_counters_forward_and_recompute": cnt}


def adjoint_bench(args, desc):
    """The adjoint workload alone: its backward / forward wall-time ratio."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    r = adjoint_cost(stream, nsteps=args.adjoint_steps)
    cells = 256 * 256
    line = {"metric": "adjoint/forward wall-time ratio", "value": r["ratio"], "unit": "x", "n_gpus": 1,
            "steps": args.adjoint_steps, "warmup": 1, "ms_per_step": r["adjoint_ms_per_step"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "cells": cells, "checkpoint_every": 20},
            "adjoint": r,
            "backward_cell_steps_per_s": cells * args.adjoint_steps / (r["backward_ms"] * 1e-3)}
    print(json.dumps(line), flush=True)
    return 0


def l2_note(state_bytes, work_bytes=0):
    """How the timed iterations avoid a warm L2: the state, or the working set
    of a stage (three state buffers and the work arrays), exceeds the 129 MB L2."""
    if state_bytes > 129e6:
        return "state %.2f GB per buffer > 129 MB L2 (no flush needed)" % (state_bytes * 1e-9)
    ws = 3 * state_bytes + work_bytes
    if ws > 129e6:
        return ("state %.0f MB, but a stage's working set (3 states + work arrays) is %.2f GB > 129 MB L2 "
                "(no flush needed)" % (state_bytes * 1e-6, ws * 1e-9))
    return "no L2 flush; working set (%.0f MB) smaller than L2" % (ws * 1e-6)


def fp64_peak(torch, local, clk):
    props = torch.cuda.get_device_properties(local)
    max_mhz = (clk or {}).get("sm_max_mhz") or measured_peaks().get("sm_max_mhz", 2070.0)
    peak = FP64_FLOPS_PER_SM_CYCLE * props.multi_processor_count * max_mhz * 1e6 * 1e-12
    return peak, "derived: 2 DFMA/SM/cycle x %d SMs x %.0f MHz x 2 flops" % (props.multi_processor_count, max_mhz)


def setup_ranks(torch):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return world, rank, local, dist


def oned_bench(args, desc):
    """The 1D scheme (af1d_*) on one long grid: every rank runs its own replica
    (weak scaling); per-kernel times from af1d_timing."""
    import torch
    import paper_2506_04857_gb300 as af

    world, rank, local, dist = setup_ranks(torch)
    stream = torch.cuda.current_stream()
    pb = WORKLOADS[args.workload][1]()
    U0 = ai.dofs1(pb)
    s = af.Solver1D(pb.n, pb.gamma, pb.bc, domain=(pb.x0, pb.x1), cfl=pb.cfl, kappa=pb.kappa, stream=stream)
    s.set_state([torch.from_numpy(u).cuda() for u in U0])
    probe = af.af_probe_fp64(stream)
    for _ in range(args.warmup):
        s.step(dt_out=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    s.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.step(dt_out=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ktimes = s.timing(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    clk = clocks.stop()
    rc, cnt = s.status(reset=True)
    if rc != af.AF_OK:
        raise SystemExit("libaf reported %s after the timed region" % af.af1d_last_error(s.ctx))
    value = pb.n * 3 * args.steps * world / (ms * 1e-3)
    peak, peak_src = fp64_peak(torch, local, clk)
    roofline = fp64_roofline(pb.name, ktimes, pb.n, pb.n * 3 * args.steps * world, ms, peak, peak_src, probe, world)
    roofline["traffic"] = None
    # end to end through the C ABI with host buffers (blocking copies)
    host = [np.ascontiguousarray(u) for u in U0]
    out = [np.empty_like(u) for u in host]
    nbytes = sum(u.nbytes for u in host)
    t0 = time.perf_counter()
    for _ in range(3):
        s.set_state(host)
        s.step(dt_out=False)
        s.get_state(out=out, device=False)
    te = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": pb.n * 3 * 3 * world / te, "unit": "cell-stage updates/s", "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "steps": 3, "api": "af1d_set_state + af1d_step + af1d_get_state"}
    if rank == 0:
        line = {"metric": "FP64 AF-MHD 1D cell-stage updates/s", "value": value, "unit": "cell-stage updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (analytic initial condition, af_inputs)",
                "config": {"workload": desc, "cells": pb.n, "gamma": pb.gamma, "cfl": pb.cfl, "kappa": pb.kappa,
                           "bc": "outflow", "per_rank_replica": world > 1, "l2": l2_note(nbytes)},
                "gpu_launches": sum(n for _, n in ktimes.values()), "roofline": roofline, "e2e": e2e,
                "clocks": clk, "limiter_counters": cnt}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload, pb, budget_s=10.0)
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def divb_bench(args, desc):
    """The divergence measures (af_divb) of one state, repeatedly: the state after
    3 steps of the 2048x2048 low-beta blast; one call = k_divb + k_divb_sum."""
    import torch
    import paper_2506_04857_gb300 as af

    world, rank, local, dist = setup_ranks(torch)
    stream = torch.cuda.current_stream()
    pb = WORKLOADS[args.workload][1]()
    s = af.Solver(pb.nx, pb.ny, pb.gamma, pb.bc, domain=(pb.x0, pb.x1, pb.y0, pb.y1), cfl=pb.cfl, kappa=pb.kappa,
                  stream=stream)
    s.set_state([torch.from_numpy(u).cuda() for u in ai.dofs(pb)])
    for _ in range(3):
        s.step(dt_out=False)
    res = torch.empty(2, dtype=torch.float64, device="cuda")
    calls = max(args.steps, 10)
    warm = max(args.warmup, 3)
    for _ in range(warm):
        s.divb(out=res)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(calls):
        s.divb(out=res)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    clk = clocks.stop()
    cells = pb.nx * pb.ny
    value = cells * calls * world / (ms * 1e-3)
    peak, peak_src = fp64_peak(torch, local, clk)
    state_bytes = cells * 32 * 8   # the four classes, read once per call
    lit = ALGO_FLOPS_DIVB[pb.name]
    ex = EXEC_FP64_DIVB.get(pb.name)
    roofline = {"bound": "alu", "kernel": "k_divb + k_divb_sum (one call)", "peak": peak, "unit": "TFLOP/s",
                "traffic": None, "peak_source": peak_src, "literal_flops_per_cell": lit,
                "literal_note": "the formulas counted as written (oracle counting build); context only, "
                                "not divided by the peak",
                "hbm_bound_cells_per_s": measured_peaks().get("hbm_gbs", 6775.6) * 1e9 / (32 * 8)}
    if ex is not None:   # executed FP64-pipe flops per cell, as for the stage kernels
        fl = ex["dadd"] + ex["dmul"] + 2.0 * ex["dfma"]
        achieved = fl * cells / (ms / calls * 1e-3) * 1e-12
        stale = kernel_digest(KERNEL_FILES_2D) != ex["digest"]
        roofline.update({"achieved": achieved, "frac": achieved / peak, "executed_flops_per_cell": fl,
                         "int_pipe_flops_per_cell": ex.get("int_mul", 0.0), "executed_counts": ex["source"],
                         "counts_stale": stale})
    else:
        roofline.update({"achieved": None, "frac": None})
    # end to end: host state in, the two measures out
    host = [torch.from_numpy(u).pin_memory() for u in s.get_state(device=False)]
    t0 = time.perf_counter()
    for _ in range(3):
        s.set_state(host)
        s.divb()
    te = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": cells * 3 * world / te, "unit": "cell evaluations/s", "h2d_bytes_per_step": state_bytes,
           "d2h_bytes_per_step": 16, "steps": 3, "api": "af_set_state (pinned host) + af_divb (host result)"}
    if rank == 0:
        line = {"metric": "FP64 divergence-measure cell evaluations/s", "value": value,
                "unit": "cell evaluations/s", "n_gpus": world, "steps": calls, "warmup": warm,
                "ms_per_step": ms / calls, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic (analytic initial condition, af_inputs, 3 steps)",
                "config": {"workload": desc, "nx": pb.nx, "ny": pb.ny, "cells": cells,
                           "per_rank_replica": world > 1, "l2": l2_note(state_bytes)},
                "gpu_launches": 2 * calls, "roofline": roofline, "e2e": e2e, "clocks": clk,
                "measures": [float(v) for v in res.cpu()]}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload, pb, budget_s=10.0)
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="blast2048", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--cpu-rate-only", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    key = args.workload
    desc, make = WORKLOADS[key]
    if args.cpu_rate_only:   # child of cpu_baseline: the oracle on the cores it was given
        print(json.dumps(cpu_rate(key, make(), 8.0, 128)), flush=True)
        return 0
    if key == "ensemble256" and args.impl == "ours":
        return ensemble_bench(args, desc)
    if key == "adjoint256" and args.impl == "ours":
        return adjoint_bench(args, desc)
    if key == "blast1d" and args.impl == "ours":
        return oned_bench(args, desc)
    if key.startswith("divb") and args.impl == "ours":
        return divb_bench(args, desc)
    pb = make()
    if args.impl == "reference":
        return reference_arm(args, key, desc, pb)

    import torch
    import paper_2506_04857_gb300 as af

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()

    U0 = ai.dofs(pb)
    sides = {}
    if any(pb.sides):   # reflective / inflow sides (the jets)
        sides = dict(sides=pb.sides, inflow=(pb.inflow_lo, pb.inflow_hi, pb.inflow_U))
    s = af.Solver(pb.nx, pb.ny, pb.gamma, pb.bc, domain=(pb.x0, pb.x1, pb.y0, pb.y1), cfl=pb.cfl, kappa=pb.kappa,
                  stream=stream, **sides)
    dev_state = [torch.from_numpy(u).cuda() for u in U0]
    s.set_state(dev_state)
    peak_fp64 = af.af_probe_fp64(stream)
    for _ in range(args.warmup):
        s.step(dt_out=False)
    torch.cuda.synchronize()

    # ---------------- timed region: K steps, inputs resident in HBM --------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    s.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.step(dt_out=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ktimes = s.timing(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    rc, cnt = s.status(reset=True)
    if rc != af.AF_OK:
        raise SystemExit("libaf reported %s after the timed region" % af.af_last_error(s.ctx))
    cells = pb.nx * pb.ny
    units = cells * 3 * args.steps * world
    value = units / (ms * 1e-3)
    launches = sum(n for _, n in ktimes.values())

    # ---------------- roofline of the dominant kernel -----------------------
    peak, peak_src = fp64_peak(torch, local, clk)
    roofline = fp64_roofline(pb.name, ktimes, cells, units, ms, peak, peak_src, peak_fp64, world)
    _, _, src, stale = exec_flops(pb.name)
    dram = EXEC_FP64.get(pb.name, {}).get("kernels", {}).get(roofline["kernel"], {}).get("dram_bytes")
    roofline["traffic"] = dram * cells if dram is not None and not stale else None
    roofline["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per cell of the capture, "
                                  "times the cells of one launch") if roofline["traffic"] else None
    roofline["hbm_bound_cell_stages_per_s"] = measured_peaks().get("hbm_gbs", 6775.6) * 1e9 / ALGO_BYTES_PER_CS

    limiter = limiter_cost(s, pb, stream, cnt, args.steps) if key.startswith("lattice") else None

    # ---------------- end to end through the C ABI with host buffers --------
    # af_step_host: every step copies its input state from pinned host memory and
    # its result back; the copies of neighbouring steps overlap the step itself.
    # The input is the state the timed region ended with (the same flow regime).
    host_in = [torch.from_numpy(u).pin_memory() for u in s.get_state(device=False)]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    bytes_state = sum(u.nbytes for u in U0)
    s.step_host(host_in, host_out)
    s.sync()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        s.step_host(host_in, host_out)
    s.sync()
    te = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    # the same steps with blocking copies (af_set_state / af_step / af_get_state), for context
    t0 = time.perf_counter()
    for _ in range(2):
        s.set_state(host_in)
        s.step(dt_out=False)
        s.get_state(out=[h.numpy() for h in host_out], device=False)
    torch.cuda.synchronize()
    ts = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    rc, _ = s.status(reset=True)
    if rc != af.AF_OK:
        raise SystemExit("libaf reported %s in the end-to-end steps" % af.af_last_error(s.ctx))
    e2e = {"value": cells * 3 * args.e2e_steps * world / te, "unit": "cell-stage updates/s",
           "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state, "steps": args.e2e_steps,
           "api": "af_step_host (pinned host buffers, copies overlapped with neighbouring steps)",
           "serial_value": cells * 3 * 2 * world / ts,
           "serial_api": "af_set_state + af_step + af_get_state, blocking copies"}

    if rank == 0:
        line = {"metric": "FP64 AF-MHD cell-stage updates/s", "value": value, "unit": "cell-stage updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (analytic initial condition, af_inputs)",
                "config": {"workload": desc, "nx": pb.nx, "ny": pb.ny, "cells": cells, "gamma": pb.gamma,
                           "cfl": pb.cfl, "kappa": pb.kappa, "bc": "outflow" if pb.bc == ai.OUTFLOW else "periodic",
                           "per_rank_replica": world > 1,
                           "l2": l2_note(sum(u.nbytes for u in U0), WORK_DOUBLES_PER_CELL * 8 * cells)},
                "gpu_launches": launches, "roofline": roofline, "e2e": e2e, "clocks": clk,
                "limiter_counters": cnt}
        if limiter is not None:
            line["limiter_cost"] = limiter
        if not args.no_adjoint and world == 1:
            line["adjoint"] = adjoint_cost(stream)
            line["adjoint_limited"] = adjoint_limited_cost(stream)
        if not args.no_ensemble and world == 1 and key == "blast2048":
            s.close()
            line["ensemble"] = ensemble_cost(torch.cuda.Stream())   # graph capture needs a non-default stream
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(key, pb)
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
