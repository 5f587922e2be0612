"""Count the algorithmic flops of one cell-step with the instrumented oracle.

Runs the flop-counting build of the oracle (``liborc_count.so``: add, sub,
mul, div, sqrt = 1 flop each; min, max, compare, abs = 0) on the ensemble
workload's first cloud (20 bubbles, 64^3) for the first STEPS steps,
including each step's reductions (max signal speed, max pressure), and
writes flops per cell-step and per cell-stage to
paper_1705_04374_gb300/data/flops_per_cell_step.json.  The benchmark reads
that file to express kernel throughput in FLOP/s.

Usage: python oracle/count_flops.py
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import cloud, solver  # noqa: E402

N = 64
STEPS = 20


def main() -> None:
    w = W.cfg2("fp64")
    sp = w.solver
    bub = cloud.sample_cloud(w.cloud, W.BASE_SEED, 0)
    Q = solver.init_cloud(sp, N, bub)
    g = solver.grid_from_params(sp, N)
    solver.flop_reset()
    for _ in range(STEPS):
        dt = sp.cfl * g.h / solver.max_speed(g, Q)
        Q = solver.rk3_step(g, Q, dt, count=True)
    # rk3_step(count=True) counted the stages; add one reduction pass per step
    stage_flops = solver.flop_count()
    solver.flop_reset()
    lib = solver._lib(True)
    lib.orc_max_speed(g, solver._p(Q))
    reduce_flops = solver.flop_count()
    cells = N ** 3
    per_step = (stage_flops / STEPS + reduce_flops) / cells
    out = {
        "_what": "algorithmic flops per cell and full RK3 step (3 stages + one reduction pass), "
                 "counted by the oracle (add/sub/mul/div/sqrt = 1, min/max/compare = 0)",
        "_workload": f"first cloud of the ensemble workload, 20 bubbles, {N}^3, first {STEPS} steps",
        "_script": "oracle/count_flops.py",
        "flops_per_cell_step": per_step,
        "flops_per_cell_stage": stage_flops / STEPS / cells / 3.0,
        "reduction_flops_per_cell": reduce_flops / cells,
    }
    dst = os.path.join(ROOT, "paper_1705_04374_gb300", "data", "flops_per_cell_step.json")
    with open(dst, "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")
    print(json.dumps(out, indent=2))


if __name__ == "__main__":
    main()
