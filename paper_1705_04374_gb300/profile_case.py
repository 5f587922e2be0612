"""A small, fixed solver workload for profiler captures.

    python -m paper_1705_04374_gb300.profile_case [--samples 64] [--steps 2]
                                                   [--precision fp32|fp64] [--N 64] [--variant 0|1]

Runs the ensemble workload's clouds (20 bubbles) on a reduced number of
samples: initial condition, then `steps` RK3 steps in profiling mode (one
kernel launch per stage, no graphs).  With 64 samples on 64^3 each state
buffer holds 470 MB (FP32), larger than the 129 MB L2, so DRAM counters keep
their meaning, while the device holds about 1.4 GB.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main() -> None:
    import torch

    import workloads as W
    from paper_1705_04374_gb300 import api

    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=64)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--variant", type=int, default=0, help="0: one block per tile, 1: persistent")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    w = W.cfg2(a.precision)
    s = api.Solver(w.solver, a.precision)
    g = api.make_group(w.solver, a.N, list(range(a.samples)), W.BASE_SEED)
    b = api.Batch(s, w.cloud, [g])
    b.init()
    b.set_variant(a.variant)
    b.set_profiling(True)
    b.run(a.steps)
    torch.cuda.synchronize()
    ms, n = b.stage_time()
    print(f"profile_case: {a.samples} x {a.N}^3 {a.precision}, variant {a.variant}, {a.steps} steps, "
          f"stage kernel avg {ms / max(n, 1):.3f} ms over {n} launches")
    b.close()


if __name__ == "__main__":
    main()
