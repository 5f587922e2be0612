"""Build the oracle's C solver into two shared libraries (test infrastructure).

``liborc.so`` is the plain FP64 solver; ``liborc_count.so`` is the same source
with the flop counter compiled in.  Both use ``-O2 -ffp-contract=off`` so that
x86 and Arm builds round identically (gcc contracts a*b+c into an FMA on Arm
unless told not to).  The solver shares no source with the CUDA library.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "solver.c")
LIBS = {
    "liborc.so": [],
    "liborc_count.so": ["-DORC_COUNT_FLOPS"],
}


def lib_path(name: str = "liborc.so") -> str:
    return os.path.join(HERE, name)


def build(force: bool = False) -> None:
    procs = []
    for name, extra in LIBS.items():
        out = lib_path(name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            continue
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
               *extra, SRC, "-o", out + ".tmp", "-lm"]
        procs.append((out, subprocess.Popen(cmd)))
    for out, p in procs:
        if p.wait() != 0:
            raise RuntimeError(f"oracle build failed: {out}")
        os.replace(out + ".tmp", out)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
