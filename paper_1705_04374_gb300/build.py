"""Build the CUDA library ``libofmlmc.so`` in-tree for sm_103a.

Translation units compiled in parallel: the solver kernels once per
precision (``kernels_fp64.cu`` without FMA contraction, ``kernels_fp32.cu``),
the device-facing C ABI (``solver.cu``, ``solver_static.cu``, ``probe.cu``) with nvcc, and
``host.cpp`` (sampler, estimator, errors) with g++ -ffp-contract=off.  The CUDA runtime is linked
statically so the library has no run-time dependency beyond the driver.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libofmlmc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")

_NV = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
SOURCES = {
    # FP64 kernels round exactly like the FP64 reference: no FMA contraction
    "kernels_fp64.o": _NV + ["-fmad=false", "-c", os.path.join(CSRC, "kernels_fp64.cu")],
    # FP32 stencil: approximate division / square root (2 ulp), flush-to-zero
    "kernels_fp32.o": _NV + ["-use_fast_math", "-c", os.path.join(CSRC, "kernels_fp32.cu")],
    "solver.o": _NV + ["-c", os.path.join(CSRC, "solver.cu")],
    "solver_static.o": _NV + ["-c", os.path.join(CSRC, "solver_static.cu")],
    "mlp.o": _NV + ["-c", os.path.join(CSRC, "mlp.cu")],
    "run.o": _NV + ["-c", os.path.join(CSRC, "run.cu")],
    "probe.o": _NV + ["-c", os.path.join(CSRC, "probe.cu")],
    "host.o": ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I", INCLUDE,
               "-c", os.path.join(CSRC, "host.cpp")],
}


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "ofmlmc.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    for obj, cmd in SOURCES.items():
        out = os.path.join(BUILD, obj)
        procs.append((obj, subprocess.Popen(cmd + ["-o", out], stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
    for obj, p in procs:
        log, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"compiling {obj} failed:\n{log}")
        if verbose and log:
            print(log)
    link = [NVCC, *ARCH, "-shared", "-o", LIB + ".tmp"] + [os.path.join(BUILD, o) for o in SOURCES]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking failed:\n{r.stdout}{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
