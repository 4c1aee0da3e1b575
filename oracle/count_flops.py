"""Count the algorithmic FP64 operations of one cell-stage with the counting
build of the oracle (af_oracle.cpp compiled with -DAF_ORACLE_COUNT).

The count is taken with the positivity-preserving limiters off (pp_on = 0):
what remains is the scheme's arithmetic (point data, cell-centre values,
LLF-FVS point updates, shock sensor, Simpson and LLF face fluxes, Powell
source, sensor-blended cell update, SSP-RK3 combination).  The PP limiters'
tests and their occasional blends are extra work that is not counted, so a
throughput measured against this count is a lower bound on the work done.

Convention: +, -, *, /, sqrt, exp, min/max and |.| each count one flop (the
oracle uses no fused multiply-add); comparisons that only steer branches are
listed but not counted.

Usage: python -m oracle.count_flops [--out FILE]   (writes a JSON summary; 2D
workloads, the jets with their reflective and inflow sides, the 1D scheme and
the divergence measures)
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import af_inputs as ai  # noqa: E402
import oracle  # noqa: E402

# GPU kernels of libaf and the oracle phases whose arithmetic each performs
KERNELS = {
    "k_pointdata": ["pointdata", "center"],
    "k_points": ["point_ho", "sensor_phi", "rk_points"],
    "k_faces": ["face", "sensor_theta"],
    "k_cells": ["cell_src", "cell_update"],
    "k_final": ["cell_final", "rk_avg"],
}


def count(pb, stages: int = 3) -> dict:
    U = ai.dofs(pb)
    oracle.counts(reset=True)
    dt = oracle.dt(pb, U, count=True)
    cnt_dt = oracle.counts(reset=True)
    coef = [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)]
    Us = U
    tot = np.zeros_like(cnt_dt)
    for s in range(stages):
        a, b = coef[s]
        Us = oracle.stage(pb, U, Us, dt, a, b, count=True, pp_on=False)
        tot += oracle.counts(reset=True)
    cells = pb.nx * pb.ny * stages
    fl = oracle.flops(tot) / cells
    fl_dt = oracle.flops(cnt_dt).sum() / cells       # dt once per step, amortised over its stages
    per_phase = {name: float(fl[i]) for i, name in enumerate(oracle.PHASES)}
    # The oracle's dt pass recomputes the point data of all DoFs; on the GPU the
    # maximum is a by-product of the point-data pass, so it is not counted.
    per_phase.pop("dt")
    # SSP-RK3 combination: 24 of the 32 values per cell are point values
    per_phase["rk_points"] = 0.75 * per_phase["rk"]
    per_phase["rk_avg"] = 0.25 * per_phase.pop("rk")
    kinds = {k: float(tot[:, q].sum() / cells) for q, k in enumerate(oracle.KINDS)}
    per_kernel = {k: sum(per_phase[p] for p in ph) for k, ph in KERNELS.items()}
    return {"workload": pb.name, "nx": pb.nx, "ny": pb.ny, "kappa": pb.kappa, "stages": stages,
            "flops_per_cell_stage": sum(per_phase.values()), "dt_pass_flops_per_cell_stage_not_counted": float(fl_dt),
            "per_phase": per_phase, "per_kernel": per_kernel, "ops_per_cell_stage_by_kind": kinds}


# 1D kernels of libaf (k1_*) and the oracle phases whose arithmetic each performs
KERNELS_1D = {
    "k1_pointdata": ["pointdata", "center"],
    "k1_points": ["point_ho", "sensor_phi", "rk_points"],
    "k1_faces": ["face", "sensor_theta"],
    "k1_cells": ["cell_src", "cell_update"],
    "k1_final": ["cell_final", "rk_avg"],
}


def count1(pb, stages: int = 3) -> dict:
    """The same count for the 1D scheme (16 unknowns per cell: average and point value)."""
    U = ai.dofs1(pb)
    oracle.counts(reset=True)
    dt = oracle.dt1(pb, U, count=True)
    oracle.counts(reset=True)
    coef = [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)]
    Us, tot = U, None
    for s in range(stages):
        a, b = coef[s]
        Us = oracle.stage1(pb, U, Us, dt, a, b, count=True, pp_on=False)
        c = oracle.counts(reset=True)
        tot = c if tot is None else tot + c
    cells = pb.n * stages
    fl = oracle.flops(tot) / cells
    per_phase = {name: float(fl[i]) for i, name in enumerate(oracle.PHASES)}
    per_phase.pop("dt")
    # SSP-RK3 combination: 8 of the 16 values per cell are point values
    per_phase["rk_points"] = 0.5 * per_phase["rk"]
    per_phase["rk_avg"] = 0.5 * per_phase.pop("rk")
    per_kernel = {k: sum(per_phase[p] for p in ph) for k, ph in KERNELS_1D.items()}
    return {"workload": pb.name, "n": pb.n, "kappa": pb.kappa, "stages": stages,
            "flops_per_cell_stage": sum(per_phase.values()), "per_phase": per_phase, "per_kernel": per_kernel}


def count_divb(pb) -> dict:
    """Flops per cell of the two divergence measures of Example 4.4 (af_divb)."""
    U = ai.dofs(pb)
    oracle.counts(reset=True)
    oracle.divb(pb, U, count=True)
    tot = oracle.counts(reset=True)
    fl = float(oracle.flops(tot).sum()) / (pb.nx * pb.ny)
    return {"workload": pb.name, "nx": pb.nx, "ny": pb.ny, "flops_per_cell": fl}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--n", type=int, default=64)
    args = ap.parse_args()
    res = {"blast_low_beta": count(ai.blast(args.n)), "orszag_tang": count(ai.orszag_tang(args.n)),
           "vortex": count(ai.vortex(args.n)),
           # 32 cells per period, as in the 2048x2048, 64-period workload
           "rarefaction_lattice": count(ai.rarefaction_lattice(args.n, periods=max(1, args.n // 32))),
           # the jets' ghost point data (reflective and inflow sides) is formed per
           # ghost, so a wider grid keeps that overhead small
           "jets": count(ai.jets(4 * args.n)),
           "blast1d": count1(ai.blast1d(64 * args.n)),
           "divb_blast_low_beta": count_divb(ai.blast(args.n))}
    txt = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt + "\n")
    print(txt)


if __name__ == "__main__":
    main()
