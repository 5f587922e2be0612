"""Benchmark: cell-updates/s of the batched cloud-collapse ensemble on GB300.

Workload (one "step" = one full pass of the hot path over the batch): 512
seeded clouds of 20 bubbles on 64^3 grids, sampled on the host, initial
condition, CFL-stepped low-storage RK3 (WENO5 + HLLC) to t_end (~120 steps),
on-device QoI reductions (peak pressure, its location, 8 sensor histories).
A cell-update is one cell advanced by one full 3-stage RK step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
                    [--impl ours|reference]
    python bench.py --profile-case [--samples 64] [--steps 2] [--precision ..] [--variant 0|1]

value: cell-updates/s over K full solves with the clouds already resident in
HBM (CUDA events on the launching stream; barrier + synchronize around the
timed region; max over ranks).  e2e: the same metric through the C ABI call
ofm_solve_batch with host arrays (cloud upload and QoI download inside the
timed region).  --impl reference times the FP64 CPU oracle on the host cores
on a bounded sample of the same workload.  --profile-case runs a small fixed
case for profiler captures (initial condition, then --steps RK3 steps with one
launch per stage and CUDA events around each stage kernel; with 64 clouds each
FP32 state buffer holds 470 MB, larger than the 129 MB L2, and the device
holds about 1.4 GB) and prints the average stage-kernel time.
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "cell-updates/s/GPU"
UNIT = "cell-updates/s"
N_GRID = 64
M_SAMPLES = 512
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FLOPS_FILE = os.path.join(ROOT, "paper_1705_04374_gb300", "data", "flops_per_cell_step.json")
TRAFFIC_FILE = os.path.join(ROOT, "paper_1705_04374_gb300", "data", "ncu_traffic.json")
KERNEL_SRC = [os.path.join(ROOT, "paper_1705_04374_gb300", "csrc", f) for f in ("kernels.cuh", "types.cuh")]

# FP32 non-tensor peak from unit counts: the device's SM count (queried) x 128
# FP32 lanes x 2 flops per multiply-add x the maximum SM clock (measured
# peaks file, else nvidia-smi's clocks.max.sm, else 2070 MHz).  Packed
# two-lane FP32 instructions (FFMA2) do not raise it: a register FFMA2 chain
# probe runs at the scalar rate.  FP64 at the nominal 1.25 TFLOP/s of the part.
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_FALLBACK = 2070.0
FP64_PEAK_TFLOPS = 1.25
HBM_FALLBACK_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--samples", type=int, default=None)
    p.add_argument("--profile-case", action="store_true")
    p.add_argument("--variant", type=int, default=0, help="--profile-case: 0 one block per tile, 1 persistent")
    a = p.parse_args()
    if a.samples is None:
        a.samples = 64 if a.profile_case else M_SAMPLES
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(precision):
    w = W.cfg2(precision)
    return w, w.solver


# --------------------------------------------------------------------------- CPU oracle

def oracle_cell_steps(sp, cloud, ids, steps_each):
    """Time the FP64 oracle: each id one 64^3 cloud advanced steps_each steps."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import cloud as ocloud
    from oracle import solver as osolver

    def one(sid):
        bub = ocloud.sample_cloud(cloud, W.BASE_SEED, sid)
        Q = osolver.init_cloud(sp, N_GRID, bub)
        g = osolver.grid_from_params(sp, N_GRID)
        for _ in range(steps_each):
            Q = osolver.rk3_step(g, Q, sp.cfl * g.h / osolver.max_speed(g, Q))
        return N_GRID ** 3 * steps_each

    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        total = sum(ex.map(one, ids))
    return total, time.perf_counter() - t0, threads


def cpu_baseline(sp, cloud):
    cores = os.cpu_count() or 1
    ids = list(range(cores))
    steps_each = 2
    cells, secs, threads = oracle_cell_steps(sp, cloud, ids, steps_each)
    return {"value": cells / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(ids)} of the 512 clouds, {steps_each} RK3 steps each from the initial "
                      f"condition on 64^3 (plain FP64 C oracle, one thread per cloud), "
                      f"{cells:.3e} cell-updates in {secs:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w, sp = workload("fp64")
    from oracle import build as obuild
    obuild.build()
    cores = os.cpu_count() or 1
    vals = []
    for k in range(args.warmup + args.steps):
        ids = list(range(k * cores, (k + 1) * cores))
        cells, secs, threads = oracle_cell_steps(sp, w.cloud, ids, 1)
        if k >= args.warmup:
            vals.append((cells, secs))
    cells = sum(c for c, _ in vals)
    secs = sum(s for _, s in vals)
    v = cells / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded random clouds", "config": reference_config(cores),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: {cores} of the 512 clouds (one per host thread), one RK3 "
                                   "step from the initial condition on 64^3, plain FP64 C oracle"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- GPU arm

def config_dict(precision, world, samples=M_SAMPLES):
    es = 4 if precision == "fp32" else 8
    buf_gb = samples * 7 * N_GRID ** 3 * es / 1e9
    return {"workload": f"ensemble: {samples} seeded clouds x 20 bubbles, 64^3, to t_end (~120 RK3 steps), "
                        "QoIs: peak pressure + location, 8 sensor histories",
            "grid": N_GRID, "samples_per_gpu": samples, "bubbles": 20,
            "stencil_precision": precision, "reductions": "f64",
            "graphs": "8-step CUDA-graph chunks",
            "parallelism": f"replicas x{max(world, 1)} (independent samples per GPU)",
            "l2": f"inputs {'larger' if buf_gb > 0.129 else 'smaller'} than L2: 3 state buffers of "
                  f"{buf_gb:.2f} GB ({precision}) per GPU"}


def reference_config(cores):
    """The reference arm's workload: the ensemble's clouds, timed on the CPU
    as a bounded sample (one RK3 step per cloud from the initial condition)."""
    return {"workload": "ensemble: seeded clouds x 20 bubbles, 64^3 (the same clouds as the GPU arm)",
            "grid": N_GRID, "bubbles": 20, "stencil_precision": "fp64", "reductions": "f64",
            "timed": f"each step: {cores} clouds (one per host thread), one RK3 step from the initial "
                     "condition, plain FP64 C oracle on the host cores",
            "parallelism": "host threads, one cloud each"}


def fp32_peak_tflops(device_index, peaks, clk):
    """SMs x 128 lanes x 2 x max SM clock, with where each factor came from."""
    import torch
    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz, src = SM_MAX_MHZ_FALLBACK, "default 2070 MHz"
    if peaks and peaks.get("sm_max_mhz"):
        mhz, src = float(peaks["sm_max_mhz"]), "measured peaks file"
    elif clk and clk.get("sm_max_mhz"):
        mhz, src = float(clk["sm_max_mhz"]), "nvidia-smi clocks.max.sm"
    tf = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return tf, f"derived: {sms} SMs (device query) x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz ({src})"


def load_json(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def kernel_hash():
    """Hash of the stage-kernel sources without comments and blank lines: a
    recorded ncu traffic figure stays valid across comment edits only."""
    h = hashlib.sha256()
    for path in KERNEL_SRC:
        with open(path) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(text.encode())
    return h.hexdigest()[:16]


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1705_04374_gb300 import api
    from paper_1705_04374_gb300 import native as nv
    from paper_1705_04374_gb300 import sharding

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    w, sp = workload(args.precision)
    M = args.samples
    ids = sharding.rank_sample_ids(rank, M)
    solver = api.Solver(sp, args.precision)
    group = api.make_group(sp, N_GRID, ids, W.BASE_SEED)
    batch = api.Batch(solver, w.cloud, [group])

    def solve_resident():
        batch.init()
        while batch.run(1 << 20) > 0:
            pass

    for _ in range(args.warmup):
        solve_resident()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    launches0 = batch.launches()
    cells = 0.0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        solve_resident()
        cells += batch.cell_steps()
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = batch.launches() - launches0
    batch.qoi(allow_bad=True)
    statuses = [q.status for q in group.qoi]
    ms_all, cells_all = sharding.aggregate(ms, cells, world, device="cuda")
    value = sharding.job_rate(ms_all / 1e3, cells_all)

    # kernel timing: one more solve with CUDA events around every stage kernel
    batch.set_profiling(True)
    solve_resident()
    stage_ms, stage_n = batch.stage_time()
    batch.set_profiling(False)
    avg_stage_ms = stage_ms / max(stage_n, 1)
    batch.close()
    del batch
    torch.cuda.empty_cache()

    # end to end through the C ABI with host arrays (clouds from pinned memory)
    cp = w.cloud
    bub_host = torch.empty((M * cp.n_bubbles * 4,), dtype=torch.float64).pin_memory()
    bub_np = bub_host.numpy().reshape(M * cp.n_bubbles, 4)
    for i, sid in enumerate(ids):
        bub_np[i * cp.n_bubbles:(i + 1) * cp.n_bubbles] = api.sample_cloud(cp, W.BASE_SEED, sid)
    e2e_group = api.Group(N_GRID, ids, W.BASE_SEED, len(sp.sensors), sp.n_out_times)
    e2e_group.c.bubbles = C.cast(C.c_void_p(bub_host.data_ptr()), C.POINTER(nv.ofm_bubble))
    garr = (nv.ofm_group * 1)(e2e_group.c)
    cpar = api.cloud_params(cp)
    nbytes = C.c_size_t()
    nv.check(nv.lib().ofm_batch_workspace_bytes(solver.h, C.byref(cpar), garr, 1, C.byref(nbytes)), "ws")
    ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
    ws_ptr = (ws.data_ptr() + 255) // 256 * 256
    sptr = C.c_void_p(stream.cuda_stream)

    def solve_e2e():
        rc = nv.lib().ofm_solve_batch(solver.h, C.byref(cpar), garr, 1, C.c_void_p(ws_ptr), nbytes.value, sptr)
        if rc not in (nv.OFM_OK, nv.OFM_ENUMERIC):
            nv.check(rc, "ofm_solve_batch")
        return sum(q.n_steps for q in e2e_group.qoi) * float(N_GRID ** 3)

    # bytes one e2e step moves, from the library's own accounting of an identical solve
    probe = api.Batch(solver, cp, [e2e_group])
    probe.init()
    while probe.run(1 << 20) > 0:
        pass
    probe.qoi(allow_bad=True)
    h2d, d2h = probe.transfer_bytes()
    probe.close()
    del probe
    torch.cuda.empty_cache()

    solve_e2e()
    barrier()
    t0 = time.perf_counter()
    e2e_cells = 0.0
    for _ in range(args.steps):
        e2e_cells += solve_e2e()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s_all, e2e_cells_all = sharding.aggregate(e2e_s, e2e_cells, world, device="cuda")
    e2e_value = sharding.job_rate(e2e_s_all, e2e_cells_all)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # the FP pipes' multiply-add rate measured now, at the clocks this GPU runs at
    probe_tflops = api.probe_fma_tflops(args.precision)
    try:
        rmse = rmse_compare(api)
    except Exception as exc:  # reported, never silently replaced
        rmse = {"failed": str(exc)}

    # roofline of the dominant kernel (the RK-stage kernel)
    flops = load_json(FLOPS_FILE) or {}
    f_stage = flops.get("flops_per_cell_stage")
    cells_per_launch = M * N_GRID ** 3
    peaks = load_json(PEAKS_FILE)
    hbm_peak = None
    hbm_src = "fallback"
    if peaks:
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in peaks:
                hbm_peak = float(peaks[k]) if not isinstance(peaks[k], dict) else float(peaks[k].get("value"))
                hbm_src = "measured"
                break
    if hbm_peak is None:
        hbm_peak = HBM_FALLBACK_GBS
    es = 4 if args.precision == "fp32" else 8
    # words per cell: stage 1 Q in, Q' and dQ out; stage 2 Q, dQ in, Q', dQ out; stage 3 Q, dQ in, Q' out
    bytes_per_cell_stage = (21 + 28 + 21) / 3.0 * es
    # DRAM bytes per cell of each of the three stage launches (one ncu capture
    # each), averaged like the CUDA-event time: traffic of the average launch
    traffic_rec = load_json(TRAFFIC_FILE) or {}
    traffic = None
    if traffic_rec.get("kernel_hash") == kernel_hash() and traffic_rec.get("precision") == args.precision:
        per_stage = traffic_rec.get("dram_bytes_per_cell_stage_by_stage")
        if per_stage and len(per_stage) == 3:
            traffic = float(np.mean(per_stage)) * cells_per_launch
    if args.precision == "fp32":
        alu_peak, alu_peak_src = fp32_peak_tflops(local, peaks, clk)
    else:
        alu_peak, alu_peak_src = FP64_PEAK_TFLOPS, "nominal FP64 of the part"
    achieved_tflops = f_stage * cells_per_launch / (avg_stage_ms / 1e3) / 1e12 if f_stage else None
    achieved_gbs = bytes_per_cell_stage * cells_per_launch / (avg_stage_ms / 1e3) / 1e9
    alu_ceiling = alu_peak * 1e12 / f_stage if f_stage else float("inf")   # cell-stages/s
    hbm_ceiling = hbm_peak * 1e9 / bytes_per_cell_stage
    if alu_ceiling <= hbm_ceiling and achieved_tflops is not None:
        roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved_tflops / alu_peak, "traffic": traffic,
                    "traffic_per_stage_B_per_cell": traffic_rec.get("dram_bytes_per_cell_stage_by_stage")
                    if traffic is not None else None,
                    "peak_source": alu_peak_src,
                    "kernel": "stage_kernel (fused WENO5 + HLLC + 2N update)",
                    "per_launch": {"cells": cells_per_launch, "flops_per_cell": f_stage,
                                   "avg_ms": avg_stage_ms, "launches_timed": stage_n},
                    "fma_probe": {"tflops": probe_tflops, "frac": achieved_tflops / probe_tflops,
                                  "what": "ofm_probe_fma_tflops: register multiply-add chains, measured in this run"}}
    else:
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                    "kernel": "stage_kernel", "avg_ms": avg_stage_ms}
    roofline_hbm = {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_gbs / hbm_peak, "peak_source": hbm_src,
                    "algorithmic_bytes_per_cell_stage": bytes_per_cell_stage}

    cpu = None
    try:
        from oracle import build as obuild
        obuild.build()
        cpu = cpu_baseline(W.cfg2("fp64").solver, w.cloud)
    except Exception as exc:  # reported, never silently replaced
        cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"failed: {exc}"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic: seeded random clouds (no dataset exists for this workload)",
        "config": config_dict(args.precision, world, args.samples),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "api": "ofm_solve_batch (host clouds in pinned memory, "
                                                 "QoIs and sensor histories back to the host)"},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roofline,
        "roofline_hbm": roofline_hbm,
        "cpu_baseline": cpu,
        "samples_failed": int(sum(1 for s in statuses if s)),
        "rmse_compare": rmse,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def rmse_compare(api):
    """GPU-seconds to a fixed OF-MLMC RMSE on a bounded configuration: 3 levels
    16^3/32^3/64^3, 20-bubble clouds, the centre sensor's peak pressure, tau =
    8e4 Pa (about 1 % of its mean).  FP32 to tau; FP32 with the learned
    surrogate of the top level term to tau; FP64: its warm-up iteration
    measured (the same sample ids as the FP32 runs' first pairs), the run to
    tau extrapolated as the FP32 run's final sample numbers times the pair
    costs W_l at FP64's measured seconds per cell-step (same variances up to
    the FP32 bias, which the common warm-up samples measure and the FP32 RMSE
    includes: sqrt(eps^2 + bias^2))."""
    cloud = W.cloud_uniform(20)
    sp = W.tiny(16, 20).solver
    levels, tau, qoi = [16, 32, 64], 8.0e4, 1
    common = dict(target=tau, qoi=qoi, max_iterations=8, min_samples=16, max_cell_steps=4e11)
    s32 = api.Solver(sp, "fp32")
    r32, p32, _ = api.run_ofmlmc(s32, cloud, levels, **common)
    rs, _, _ = api.run_ofmlmc(s32, cloud, levels, surrogate=True, surrogate_min_pairs=64, surrogate_nearest=1,
                              **common)
    s64 = api.Solver(sp, "fp64")
    w64, p64, _ = api.run_ofmlmc(s64, cloud, levels, **dict(common, max_iterations=1))
    sec_per_cell64 = w64["gpu_seconds"] / w64["cell_steps"]
    fp64_gpu_s = float(sum(m * w for m, w in zip(r32["M"], r32["W"]))) * sec_per_cell64
    # FP32 bias on the common warm-up samples, with FP64's coefficients
    alpha = w64["est"]["alpha"]
    m0 = [len(p) for p in p64]
    mean32 = sum(float(np.mean(alpha[l] * p32[l][:m0[l], 0] - (alpha[l - 1] * p32[l][:m0[l], 1] if l else 0.0)))
                 for l in range(len(levels)))
    bias = abs(mean32 - w64["est"]["mean"])

    def arm(r):
        return {"gpu_seconds": r["gpu_seconds"], "eps": float(np.sqrt(r["est"]["eps2"])),
                "rmse": float(np.sqrt(r["est"]["eps2"] + bias ** 2)), "M": r["M"], "mean": r["est"]["mean"]}
    sur = arm(rs)
    sur.update(surrogate_used=rs["surrogate_used"], beta=rs["beta"], surrogate_seconds=rs["surrogate_seconds"])
    return {"config": "3 levels 16^3/32^3/64^3, 20-bubble clouds, centre-sensor peak pressure, tau 8e4 Pa "
                      "(~1 % of the mean)", "tau": tau, "fp32_bias": bias,
            "fp32": arm(r32), "fp32_surrogate": sur,
            "fp64": {"gpu_seconds": fp64_gpu_s, "method": "warm-up measured (gpu_seconds %.2f, M %s), extrapolated "
                     "to the FP32 run's sample numbers at %.3g s per cell-step" % (w64["gpu_seconds"], w64["M"],
                                                                                   sec_per_cell64)},
            "fp64_over_fp32": fp64_gpu_s / r32["gpu_seconds"],
            "fp64_over_fp32_surrogate": fp64_gpu_s / rs["gpu_seconds"]}


def run_profile_case(args):
    """Small fixed case for profiler captures (see the module docstring)."""
    import torch

    from paper_1705_04374_gb300 import api
    torch.cuda.set_device(0)
    w, sp = workload(args.precision)
    s = api.Solver(sp, args.precision)
    g = api.make_group(sp, N_GRID, list(range(args.samples)), W.BASE_SEED)
    b = api.Batch(s, w.cloud, [g])
    b.init()
    b.set_variant(args.variant)
    b.set_profiling(True)
    b.run(args.steps)
    torch.cuda.synchronize()
    ms, n = b.stage_time()
    print(f"profile case: {args.samples} x {N_GRID}^3 {args.precision}, variant {args.variant}, {args.steps} steps, "
          f"stage kernel avg {ms / max(n, 1):.3f} ms over {n} launches")
    b.close()


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
