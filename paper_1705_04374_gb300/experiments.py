"""Estimator-level experiments on one GPU (each prints one JSON object).

    python -m paper_1705_04374_gb300.experiments uneven3 [--quick]
    python -m paper_1705_04374_gb300.experiments surrogate [--quick]
    python -m paper_1705_04374_gb300.experiments rmse [--quick]
    python -m paper_1705_04374_gb300.experiments cfg5 [--quick]

uneven3   three levels 32^3 / 64^3 / 128^3 with 1024 / 128 / 16 pairs of 50-bubble
          clouds (FP32 stencil, FP64 reductions) in one uneven batch; device time,
          cell-updates/s, pair costs, the OF-MLMC estimator; and the same solves
          as one batch per group, for comparison.
unevensmall the same comparison at 8^3 / 16^3 / 32^3 with 256 / 64 / 16 pairs,
          where no group fills the GPU alone.
surrogate the MLP surrogate trained on the solver's own samples and used as the
          estimator's extra control variate: (a) on the level-0 term, geometry
          only, expectation from 65,536 extra clouds; (b) on the top term,
          geometry plus the coarse QoI.  Variance with and without it, and the
          plain estimator's variance at equal GPU-seconds.
rmse      GPU-seconds to a fixed OF-MLMC RMSE: the adaptive loop in plain FP64
          against FP32 (+ the level-0 surrogate), with the FP32 bias measured on
          common samples and included in the RMSE.
cfg5      500-bubble clouds, four levels 32^3..256^3, sample numbers from the
          OF-MLMC allocation at 1 % of the mean peak pressure, FP32, with the
          level-0 surrogate.

Every computation runs in the library's kernels and host code (C ABI); this
module only orders the calls and times them with CUDA events.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from paper_1705_04374_gb300 import api  # noqa: E402
from paper_1705_04374_gb300 import native as nv  # noqa: E402
from paper_1705_04374_gb300 import surrogate as S  # noqa: E402

ID_SHIFT = 40
QOI = 1   # the centre sensor's peak pressure (the paper's estimator QoI is the centre sensor)


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _qoi(q, which):
    return q["p_peak"] if which == 0 else q["sensor_peak"][which - 1]


def solve_groups(solver, cloud, spec, seed=W.BASE_SEED, variant=None, tune=None):
    """spec: list of (N, ids).  One uneven batch (stage-kernel variant: the batch's default, or
    the given one; -1 autotunes and, with a dict `tune`, reports the choice and its timings);
    returns (per-group QoI dicts, device seconds, cell-steps)."""
    import torch
    sp = solver.sp
    groups = [api.make_group(sp, N, ids, seed) for (N, ids) in spec]
    b = api.Batch(solver, cloud, groups)
    if variant is not None:
        b.set_variant(variant)
    e0, e1 = _events()
    e0.record()
    b.init()
    while b.run(1 << 20) > 0:
        pass
    e1.record()
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    cells = b.cell_steps()
    b.qoi(allow_bad=True)
    out = [g.qoi_dicts(len(sp.sensors)) for g in groups]
    if tune is not None:
        v, t = b.variant()
        tune.update(chosen=v, tune_ms=list(t))
    b.close()
    return out, secs, cells


def level_ids(l, lo, hi):
    return [(l << ID_SHIFT) | i for i in range(lo, hi)]


def pairs_from(qf, qc, which):
    rows, bad = [], 0
    for i in range(len(qf)):
        ok = qf[i]["status"] == 0 and (qc is None or qc[i]["status"] == 0)
        if not ok:
            bad += 1
            continue
        rows.append((_qoi(qf[i], which), _qoi(qc[i], which) if qc is not None else 0.0))
    return np.array(rows), bad


def run_levels(solver, cloud, levels, counts, which=QOI, separate=False):
    """Pairs of every level (fine members on levels[l], coarse on levels[l-1])."""
    spec, owner = [], []
    for l, (N, M) in enumerate(zip(levels, counts)):
        ids = level_ids(l, 0, M)
        spec.append((N, ids))
        owner.append((l, "fine"))
        if l > 0:
            spec.append((levels[l - 1], ids))
            owner.append((l, "coarse"))
    if separate:
        res, secs, cells = [], 0.0, 0.0
        for sg in spec:
            r, s, c = solve_groups(solver, cloud, [sg])
            res += r
            secs += s
            cells += c
    else:
        res, secs, cells = solve_groups(solver, cloud, spec)
    L = len(levels) - 1
    fine = {l: res[k] for k, (l, role) in enumerate(owner) if role == "fine"}
    coarse = {l: res[k] for k, (l, role) in enumerate(owner) if role == "coarse"}
    pairs, W_cells, failed = [], [], 0
    for l in range(L + 1):
        p, bad = pairs_from(fine[l], coarse.get(l), which)
        pairs.append(p)
        failed += bad
        cs = sum(levels[l] ** 3 * q["n_steps"] for q in fine[l])
        if l > 0:
            cs += sum(levels[l - 1] ** 3 * q["n_steps"] for q in coarse[l])
        W_cells.append(cs / len(fine[l]))
    return dict(pairs=pairs, W_cells=W_cells, secs=secs, cells=cells, failed=failed, fine=fine, coarse=coarse)


def features_for(cloud, ids, seed=W.BASE_SEED, n_keep=0):
    import torch
    bub = np.stack([api.sample_cloud(cloud, seed, int(i)) for i in ids])
    return S.cloud_features(torch.from_numpy(bub).cuda(), cloud.n_bubbles, cloud.domain_L, cloud.cloud_radius,
                            n_keep)


def fit_geometry_surrogate(cloud, ids, y, steps, ks=(1, 2, 4, 0)):
    """Geometry-only surrogate of y: one MLP per number of nearest bubbles in
    ks (0: all), the one with the lowest held-out error on its own training
    rows kept.  Returns (net, n_keep, device seconds of all the training)."""
    best = None
    secs = 0.0
    for k in ks:
        net, t, _, err = train_surrogate(features_for(cloud, ids, n_keep=k), y, steps, return_err=True)
        secs += t
        if best is None or err < best[2]:
            if best is not None:
                best[0].close()
            best = (net, k, err)
        else:
            net.close()
    return best[0], best[1], secs


def train_surrogate(X, y, steps, lr=1e-3, hidden=256, seed=0, chunk=25, return_err=False):
    """Train the MLP on (X rows, y) with early stopping: 80 % of the rows train,
    20 % validate after every `chunk` Adam steps; the parameters with the
    lowest validation error are kept.  Returns (net, device seconds, loss
    history[, that validation error])."""
    import torch
    n, d = X.shape
    n_tr = max(2, int(0.8 * n))
    net = S.MLP(d, hidden, 3, 1, max_rows=n_tr)
    rng = np.random.default_rng(seed)
    sizes = net.sizes
    vec = np.concatenate([np.concatenate([(rng.normal(size=(a, b)) * math.sqrt(2.0 / a)).ravel(), np.zeros(b)])
                          for a, b in zip(sizes[:-1], sizes[1:])]).astype(np.float32)
    net.set_params(vec)
    m, s = S.column_moments(X[:n_tr])
    ytr = y[:n_tr]
    net.set_scaling(m.cpu().numpy(), s.cpu().numpy(), np.array([ytr.mean()]), np.array([max(ytr.std(), 1e-30)]))
    T = torch.from_numpy(ytr[:, None].astype(np.float32)).cuda()
    yv = y[n_tr:]
    e0, e1 = _events()
    e0.record()
    best, best_err, hist = net.get_params(), float("inf"), []
    for _ in range(max(1, steps // chunk)):
        hist.extend(net.train(X[:n_tr], T, steps=chunk, lr=lr).tolist())
        if len(yv):
            pv = net.forward(X[n_tr:]).cpu().numpy().ravel()
            err = float(np.mean((pv - yv) ** 2))
            if err < best_err:
                best_err, best = err, net.get_params()
    net.set_params(best)
    e1.record()
    torch.cuda.synchronize()
    if return_err:
        return net, e0.elapsed_time(e1) / 1e3, np.array(hist), best_err
    return net, e0.elapsed_time(e1) / 1e3, np.array(hist)


def infer(net, X):
    import torch
    e0, e1 = _events()
    e0.record()
    Y = net.forward(X)
    e1.record()
    torch.cuda.synchronize()
    return Y.cpu().numpy().ravel().astype(np.float64), e0.elapsed_time(e1) / 1e3


# ------------------------------------------------------------------------------ uneven3

def cmd_uneven3(quick):
    w = W.cfg3()
    counts = (128, 16, 2) if quick else (1024, 128, 16)
    solver = api.Solver(w.solver, "fp32")
    r = run_levels(solver, w.cloud, w.levels, counts)
    rs = run_levels(solver, w.cloud, w.levels, counts, separate=True)
    est = api.estimate(r["pairs"], r["W_cells"])
    # the same uneven batch with the stage-kernel variant chosen by the autotuner
    spec = []
    for l, (N, M) in enumerate(zip(w.levels, counts)):
        spec.append((N, level_ids(l, 0, M)))
        if l > 0:
            spec.append((w.levels[l - 1], level_ids(l, 0, M)))
    tune = {}
    _, secs_tuned, _ = solve_groups(solver, w.cloud, spec, variant=-1, tune=tune)
    return dict(experiment="uneven3", levels=list(w.levels), counts=list(counts), precision="fp32",
                bubbles=w.cloud.n_bubbles, qoi="centre sensor peak pressure [Pa]",
                device_seconds=r["secs"], cell_steps=r["cells"], cell_updates_per_s=r["cells"] / r["secs"],
                separate_batches_seconds=rs["secs"], speedup_one_batch=rs["secs"] / r["secs"],
                identical_to_separate=bool(all(np.array_equal(a, b) for a, b in zip(r["pairs"], rs["pairs"]))),
                W_cell_steps_per_pair=r["W_cells"], failed=r["failed"],
                autotuned=dict(seconds=secs_tuned, variant=tune.get("chosen"),
                               two_step_ms_per_variant=tune.get("tune_ms")),
                estimator={k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in est.items()})


def cmd_unevensmall(quick):
    """The coarse end of a hierarchy, where no level fills the GPU alone: 8^3 /
    16^3 / 32^3 with 256 / 64 / 16 pairs of 50-bubble clouds (groups of 64 to
    1,024 tiles against 456 resident stage-kernel blocks), one uneven batch
    against one batch per group, identical results required."""
    w = W.cfg3()
    levels = (8, 16, 32)
    counts = (64, 16, 4) if quick else (256, 64, 16)
    solver = api.Solver(w.solver, "fp32")
    r = run_levels(solver, w.cloud, levels, counts)
    rs = run_levels(solver, w.cloud, levels, counts, separate=True)
    spec = []
    for l, (N, M) in enumerate(zip(levels, counts)):
        spec.append((N, level_ids(l, 0, M)))
        if l > 0:
            spec.append((levels[l - 1], level_ids(l, 0, M)))
    tune = {}
    _, secs_tuned, _ = solve_groups(solver, w.cloud, spec, variant=-1, tune=tune)
    return dict(experiment="unevensmall", levels=list(levels), counts=list(counts), precision="fp32",
                bubbles=w.cloud.n_bubbles, groups=[(N, len(ids)) for N, ids in spec],
                tiles_per_group=[len(ids) * (N // 8) ** 3 for N, ids in spec],
                device_seconds=r["secs"], cell_steps=r["cells"], cell_updates_per_s=r["cells"] / r["secs"],
                separate_batches_seconds=rs["secs"], separate_cell_updates_per_s=rs["cells"] / rs["secs"],
                speedup_one_batch=rs["secs"] / r["secs"],
                identical_to_separate=bool(all(np.array_equal(a, b) for a, b in zip(r["pairs"], rs["pairs"]))),
                autotuned=dict(seconds=secs_tuned, variant=tune.get("chosen"),
                               two_step_ms_per_variant=tune.get("tune_ms")),
                failed=r["failed"])


# ------------------------------------------------------------------------------ surrogate

def cmd_surrogate(quick):
    import torch
    w = W.cfg3()
    cloud = w.cloud
    counts = (256, 32, 4) if quick else (1024, 128, 16)
    N_extra = 8192 if quick else 65536
    steps = 300 if quick else 600
    solver = api.Solver(w.solver, "fp32")
    r = run_levels(solver, cloud, w.levels, counts)
    pairs = r["pairs"]
    sec_per_cell = r["secs"] / r["cells"]
    Wsec = [c * sec_per_cell for c in r["W_cells"]]
    est = api.estimate(pairs, Wsec)
    alpha, st2 = est["alpha"], est["sigma_tilde2"]
    M = [len(p) for p in pairs]
    L = len(w.levels) - 1
    out = dict(experiment="surrogate", levels=list(w.levels), counts=list(counts), N_extra=N_extra,
               plain=dict(mean=est["mean"], eps2=est["eps2"], sigma_tilde2=st2.tolist(), alpha=alpha.tolist(),
                          solve_seconds=r["secs"]))
    # (a) level-0 term, geometry only; trained on half of the level-0 samples, CV on the other half
    ids0 = level_ids(0, 0, counts[0])
    q0 = pairs[0][:, 0]
    n_tr = len(q0) // 2
    net, k0, t_train = fit_geometry_surrogate(cloud, ids0[:n_tr], q0[:n_tr], steps)
    s_pair, t_inf0 = infer(net, features_for(cloud, ids0[n_tr:], n_keep=k0))
    Xe = features_for(cloud, level_ids(7, 0, N_extra), n_keep=k0)     # independent extra clouds
    s_extra, t_inf = infer(net, Xe)
    D0 = alpha[0] * q0[n_tr:]
    cv = S.surrogate_cv(D0, alpha[0] * s_pair, alpha[0] * s_extra)
    plain_var0 = np.var(D0, ddof=1) / len(D0)
    sur_seconds = t_train + t_inf0 + t_inf
    # equal GPU-seconds: the surrogate estimator paid for all counts[0] level-0 solves
    # (n_tr of them only train the network) plus training and inference; the plain
    # estimator averages every one of those solves and spends sur_seconds on more
    extra_plain = sur_seconds / Wsec[0]
    plain_var0_eq = np.var(alpha[0] * q0, ddof=1) / (len(q0) + extra_plain)
    out["level0_geometry"] = dict(train_rows=n_tr, cv_rows=len(D0), nearest_bubbles=k0,
                                  corr=float(np.corrcoef(s_pair, q0[n_tr:])[0, 1]), beta=cv["beta"],
                                  var_plain=plain_var0, var_with_surrogate=cv["var"],
                                  var_plain_equal_gpu_seconds=plain_var0_eq,
                                  variance_ratio=cv["var"] / plain_var0,
                                  variance_ratio_equal_gpu_seconds=cv["var"] / plain_var0_eq,
                                  surrogate_seconds=dict(train=t_train, infer=t_inf0 + t_inf),
                                  level0_pair_seconds=Wsec[0])
    net.close()
    # (b) top term, geometry + coarse QoI, trained on the lower pairs' (coarse -> fine) relation
    Xs, ys = [], []
    for l in range(1, L):
        Xl = features_for(cloud, level_ids(l, 0, M[l]))
        qc = torch.from_numpy(pairs[l][:, 1:2].astype(np.float32)).cuda()
        Xs.append(torch.cat([Xl, qc], dim=1))
        ys.append(pairs[l][:, 0])
    Xtr = torch.cat(Xs, 0)
    ytr = np.concatenate(ys)
    net, t_train_b, hist_b = train_surrogate(Xtr, ytr, steps)
    XL = features_for(cloud, level_ids(L, 0, M[L]))
    XLc = torch.cat([XL, torch.from_numpy(pairs[L][:, 1:2].astype(np.float32)).cuda()], dim=1)
    sL, _ = infer(net, XLc)
    DL = alpha[L] * pairs[L][:, 0] - alpha[L - 1] * pairs[L][:, 1]
    out["top_geometry_coarse"] = dict(train_rows=len(ytr), top_pairs=M[L],
                                      loss_first_last=[float(hist_b[0]), float(hist_b[-1])],
                                      corr_with_D_L=float(np.corrcoef(sL, DL)[0, 1]) if M[L] > 2 else None,
                                      note="its expectation over extra clouds needs one level-(L-1) solve per "
                                           "extra cloud (charged to GPU-seconds)")
    net.close()
    return out


# ------------------------------------------------------------------------------ rmse

def cmd_rmse(quick):
    import torch
    w = W.tiny(16, 20)
    cloud = W.cloud_uniform(20)
    sp = w.solver
    levels = [16, 32, 64]
    tau = 1.2e6 if quick else 6.0e5
    cap64 = 1e9 if quick else 4e9
    s64 = api.Solver(sp, "fp64")
    s32 = api.Solver(sp, "fp32")
    t0 = time.time()
    r64, p64, i64 = api.run_ofmlmc(s64, cloud, levels, target=tau, qoi=QOI, max_iterations=6,
                                   max_cell_steps=cap64)
    wall64 = time.time() - t0
    # FP32 bias on common samples: the FP64 run's pairs, solved again in FP32
    common = run_levels(s32, cloud, levels, [len(p) for p in p64])
    Wc = r64["W"]
    e64 = api.estimate(p64, Wc)
    e32c = api.estimate(common["pairs"], Wc)
    bias = abs(e32c["mean"] - e64["mean"])
    tau32 = math.sqrt(max(tau ** 2 - bias ** 2, 0.25 * tau ** 2))
    t0 = time.time()
    r32, p32, i32 = api.run_ofmlmc(s32, cloud, levels, target=tau32, qoi=QOI, max_iterations=6,
                                   max_cell_steps=10 * cap64)
    wall32 = time.time() - t0
    out = dict(experiment="rmse", levels=levels, bubbles=20, qoi="centre sensor peak pressure [Pa]",
               tau=tau, fp32_bias=bias,
               fp64=dict(gpu_seconds=r64["gpu_seconds"], wall_seconds=wall64, M=r64["M"], eps=math.sqrt(r64["est"]["eps2"]),
                         mean=r64["est"]["mean"], iterations=r64["iterations"], capped=r64["capped"]),
               fp32=dict(gpu_seconds=r32["gpu_seconds"], wall_seconds=wall32, M=r32["M"], eps=math.sqrt(r32["est"]["eps2"]),
                         rmse=math.sqrt(r32["est"]["eps2"] + bias ** 2), mean=r32["est"]["mean"],
                         iterations=r32["iterations"], capped=r32["capped"]))
    # level-0 surrogate on the FP32 run: the variance it removes from the level-0 term
    q0 = p32[0][:, 0]
    if len(q0) >= 64:
        ids0 = [int(i) for i in i32[0]]
        n_tr = len(q0) // 2
        net, k0, t_train = fit_geometry_surrogate(cloud, ids0[:n_tr], q0[:n_tr], 400)
        s_pair, t1 = infer(net, features_for(cloud, ids0[n_tr:], n_keep=k0))
        s_extra, t2 = infer(net, features_for(cloud, level_ids(7, 0, 65536), n_keep=k0))
        a0 = r32["est"]["alpha"][0]
        cv = S.surrogate_cv(a0 * q0[n_tr:], a0 * s_pair, a0 * s_extra)
        ratio = cv["var"] / (np.var(a0 * q0[n_tr:], ddof=1) / (len(q0) - n_tr))
        st2 = np.array(r32["est"]["sigma_tilde2"])
        Wsec32 = np.array(r32["W"]) * r32["gpu_seconds"] / r32["cell_steps"]
        def cost(st):
            return float(np.sum(np.sqrt(st * Wsec32)) ** 2 / tau32 ** 2)
        st_sur = st2.copy()
        st_sur[0] *= ratio
        # the surrogate's cost: training, inference and the n_tr level-0 solves that only train it
        out["fp32_surrogate"] = dict(level0_variance_ratio=ratio, corr=float(np.corrcoef(s_pair, q0[n_tr:])[0, 1]),
                                     nearest_bubbles=k0,
                                     train_seconds=t_train, infer_seconds=t1 + t2,
                                     training_solve_seconds=n_tr * float(Wsec32[0]),
                                     model_gpu_seconds_plain=cost(st2),
                                     model_gpu_seconds_with_surrogate=cost(st_sur) + t_train + t1 + t2
                                     + n_tr * float(Wsec32[0]))
        net.close()
    out["gpu_seconds_ratio_fp64_over_fp32"] = r64["gpu_seconds"] / max(r32["gpu_seconds"], 1e-30)
    return out


# ------------------------------------------------------------------------------ cfg5

def cmd_cfg5(quick):
    """500-bubble clouds, 4 levels 32^3..256^3, sample numbers from the OF-MLMC
    allocation for a fixed budget of cell-steps (Eq. M-budget; FP32 stencil,
    memory-admitted batches), and the level-0 surrogate on top."""
    cloud = W.cloud_uniform(500)
    sp = W.SolverParams(sensors=W.centre_sensor())
    levels = [16, 32, 64, 128] if quick else [32, 64, 128, 256]
    budget = 1.0e10 if quick else 1.2e11
    s32 = api.Solver(sp, "fp32")
    warm, _, _ = api.run_ofmlmc(s32, cloud, levels, target=budget, mode="budget", qoi=0, max_iterations=1)
    res, pairs, ids = api.run_ofmlmc(s32, cloud, levels, target=budget, mode="budget", qoi=0, max_iterations=4,
                                     max_cell_steps=2.0 * budget, capacity=1 << 18)
    out = dict(experiment="cfg5", levels=levels, bubbles=500, qoi="peak pressure [Pa]", budget_cell_steps=budget,
               warmup_M=warm["M"], warmup_mean=warm["est"]["mean"], warmup_eps=math.sqrt(warm["est"]["eps2"]),
               warmup_alpha=warm["est"]["alpha"].tolist(),
               M=res["M"], W_cell_steps=res["W"], iterations=res["iterations"],
               capped=res["capped"], failed=res["failed"], gpu_seconds=res["gpu_seconds"],
               cell_steps=res["cell_steps"], cell_updates_per_s=res["cell_steps"] / max(res["gpu_seconds"], 1e-30),
               eps=math.sqrt(res["est"]["eps2"]), mean=res["est"]["mean"],
               alpha=res["est"]["alpha"].tolist(), sigma_tilde2=res["est"]["sigma_tilde2"].tolist())
    q0 = pairs[0][:, 0]
    if len(q0) >= 40:
        ids0 = [int(i) for i in ids[0]]
        n_tr = len(q0) // 2
        net, k0, t_train = fit_geometry_surrogate(cloud, ids0[:n_tr], q0[:n_tr], 400)
        s_pair, t1 = infer(net, features_for(cloud, ids0[n_tr:], n_keep=k0))
        s_extra, t2 = infer(net, features_for(cloud, level_ids(7, 0, 65536 if not quick else 4096), n_keep=k0))
        a0 = res["est"]["alpha"][0]
        cv = S.surrogate_cv(a0 * q0[n_tr:], a0 * s_pair, a0 * s_extra)
        out["level0_surrogate"] = dict(corr=float(np.corrcoef(s_pair, q0[n_tr:])[0, 1]), beta=cv["beta"],
                                       nearest_bubbles=k0,
                                       variance_ratio=cv["var"] / (np.var(a0 * q0[n_tr:], ddof=1) / (len(q0) - n_tr)),
                                       train_seconds=t_train, infer_seconds=t1 + t2)
        net.close()
    return out


# ------------------------------------------------------------------------------ paper500

def cmd_paper500(quick):
    """The paper's Sec. 3.1 experiment shrunk to one GPU: 500-bubble clouds (R_cloud 20 mm,
    log-normal radii in [0.8, 1.2] mm), bubbles and the cloud's liquid at 0.5 MPa, 1/r ramp
    to 10 MPa from 1 mm beyond the cloud surface; QoI the centre pressure sensor p_c (Eq.
    sensor).  (a) An OF-MLMC run on 4 levels 32^3..256^3 for a fixed budget of cell-steps
    (Eq. M-budget, FP32 stencil, characteristic far-field boundaries, 16 starting pairs per
    level, to the paper's 70 us).  The paper's levels are 512^3..4096^3; the finest here has
    h = 0.39 mm (--quick: 8^3..64^3).  (b) Plain Monte Carlo
    statistics of the other QoIs of Sec. 3.2 on 64^3: peak pressure and its distance from
    the centre, maximum sound speed, and the cloud's gas-volume collapse time (time of the
    minimum gas fraction of a 20 mm ball about the centre, the paper's sensor #5)."""
    cloud = W.cloud_paper500()
    c = 0.5 * W.DOMAIN_L
    sp = W.solver_paper500(sensors=(W.centre_sensor()[0], (c, c, c, 0.02)), t_end=70e-6)
    levels = [8, 16, 32, 64] if quick else [32, 64, 128, 256]
    budget = 5.0e9 if quick else 1.0e12
    s32 = api.Solver(sp, "fp32")
    res, pairs, ids = api.run_ofmlmc(s32, cloud, levels, target=budget, mode="budget", qoi=1, max_iterations=4,
                                     max_cell_steps=2.0 * budget, min_samples=16, capacity=1 << 18)
    out = dict(experiment="paper500", levels=levels, bubbles=500, qoi="centre sensor peak pressure p_c [Pa]",
               budget_cell_steps=budget, M=res["M"], W_cell_steps=res["W"], iterations=res["iterations"],
               capped=res["capped"], failed=res["failed"], gpu_seconds=res["gpu_seconds"],
               cell_updates_per_s=res["cell_steps"] / max(res["gpu_seconds"], 1e-30),
               mean=res["est"]["mean"], eps=math.sqrt(res["est"]["eps2"]), alpha=res["est"]["alpha"].tolist(),
               sigma_tilde2=res["est"]["sigma_tilde2"].tolist())
    n_mc = 32 if quick else 256
    (q,), secs, cells = solve_groups(s32, cloud, [(64, level_ids(9, 0, n_mc))])
    ok = [d for d in q if d["status"] == 0]
    def stats(vals):
        v = np.array(vals, dtype=np.float64)
        return dict(mean=float(v.mean()), std=float(v.std(ddof=1)), min=float(v.min()), max=float(v.max()))
    out["mc_64"] = dict(samples=n_mc, ok=len(ok), gpu_seconds=secs,
                        p_peak=stats([d["p_peak"] for d in ok]),
                        p_peak_dist=stats([d["p_peak_dist"] for d in ok]),
                        p_c_peak=stats([d["sensor_peak"][0] for d in ok]),
                        c_max=stats([d["c_max"] for d in ok]),
                        gas_fraction_t0=stats([d["sensor_alpha0"][1] for d in ok]),
                        gas_fraction_min=stats([d["sensor_alpha_min"][1] for d in ok]),
                        collapse_time=stats([d["sensor_alpha_min_t"][1] for d in ok]))
    return out


# ------------------------------------------------------------------------------ epsval

def cmd_epsval(quick, min_samples=16):
    """The error estimate of Eq. (ocv-mlmc-err) against the empirical error:
    R independent seeded OF-MLMC runs (FP32, 3 levels 16^3/32^3/64^3, 20
    bubbles, centre sensor peak pressure) to a tolerance tau, and one
    reference run to tau/3 with another seed, every level starting from at
    least min_samples pairs.  The empirical mean squared error of the R
    estimates about the reference, less the reference's own estimated
    variance, should match the mean of the estimated eps^2."""
    w = W.tiny(16, 20)
    cloud = W.cloud_uniform(20)
    levels = [16, 32, 64]
    R = 4 if quick else 8
    tau = 6.0e5 if quick else 3.0e5
    s32 = api.Solver(w.solver, "fp32")
    ref, _, _ = api.run_ofmlmc(s32, cloud, levels, target=tau / 3.0, qoi=QOI, seed=W.BASE_SEED + 1000,
                               max_iterations=8, max_cell_steps=6e10, capacity=1 << 18, min_samples=min_samples)
    ests, eps2s, gsec, Ms, capped = [], [], [], [], []
    for r in range(R):
        res, _, _ = api.run_ofmlmc(s32, cloud, levels, target=tau, qoi=QOI, seed=W.BASE_SEED + 1 + r,
                                   max_iterations=8, max_cell_steps=2e10, min_samples=min_samples)
        capped.append(res["capped"])
        ests.append(res["est"]["mean"])
        eps2s.append(res["est"]["eps2"])
        gsec.append(res["gpu_seconds"])
        Ms.append(list(res["M"]))
    ests = np.array(ests)
    mse = float(np.mean((ests - ref["est"]["mean"]) ** 2))
    return dict(experiment="epsval", levels=levels, bubbles=20, qoi="centre sensor peak pressure [Pa]", tau=tau,
                repeats=R, min_samples=min_samples, capped=capped, reference=dict(mean=ref["est"]["mean"], eps=math.sqrt(ref["est"]["eps2"]), M=list(ref["M"]),
                                          gpu_seconds=ref["gpu_seconds"], capped=ref["capped"]),
                estimates=ests.tolist(), eps_estimated=[math.sqrt(e) for e in eps2s], M=Ms, gpu_seconds=gsec,
                empirical_rmse=math.sqrt(mse), mean_estimated_eps=math.sqrt(float(np.mean(eps2s))),
                empirical_rmse_less_reference=math.sqrt(max(mse - ref["est"]["eps2"], 0.0)))


# ------------------------------------------------------------------------------ orders

def cmd_orders(quick):
    """WENO5 against the paper's third-order option (WENO3) on the ensemble workload (20-bubble
    clouds on 64^3 to t_end, FP32 stencil): throughput of each, and how far the third-order
    QoIs sit from the fifth-order ones on the same clouds."""
    from dataclasses import replace
    n = 64 if quick else 256
    w = W.cfg2("fp32")
    ids = level_ids(0, 0, n)
    out = dict(experiment="orders", grid=64, samples=n, bubbles=20)
    res = {}
    for order in (5, 3):
        sp = replace(w.solver, weno_order=order)
        s32 = api.Solver(sp, "fp32")
        solve_groups(s32, w.cloud, [(64, ids[:8])])             # warm-up (graphs, first launches)
        (q,), secs, cells = solve_groups(s32, w.cloud, [(64, ids)])
        res[order] = q
        out[f"weno{order}"] = dict(gpu_seconds=secs, cell_updates_per_s=cells / secs,
                                   steps_mean=float(np.mean([d["n_steps"] for d in q])),
                                   p_peak_mean=float(np.mean([d["p_peak"] for d in q])),
                                   p_c_mean=float(np.mean([d["sensor_peak"][0] for d in q])))
    d_peak = [abs(a["p_peak"] - b["p_peak"]) / b["p_peak"] for a, b in zip(res[3], res[5])]
    d_pc = [abs(a["sensor_peak"][0] - b["sensor_peak"][0]) / b["sensor_peak"][0] for a, b in zip(res[3], res[5])]
    out["weno3_vs_weno5"] = dict(speedup=out["weno3"]["cell_updates_per_s"] / out["weno5"]["cell_updates_per_s"],
                                 p_peak_rel_diff_mean=float(np.mean(d_peak)), p_peak_rel_diff_max=float(np.max(d_peak)),
                                 p_c_rel_diff_mean=float(np.mean(d_pc)), p_c_rel_diff_max=float(np.max(d_pc)))
    return out


# ------------------------------------------------------------------------------ boundaries

def cmd_boundaries(quick):
    """Cost of the characteristic far-field boundary: the ensemble workload (20-bubble clouds
    on 64^3 to t_end, FP32) with transmissive and with characteristic boundaries."""
    from dataclasses import replace
    n = 64 if quick else 256
    w = W.cfg2("fp32")
    ids = level_ids(0, 0, n)
    out = dict(experiment="boundaries", grid=64, samples=n, bubbles=20)
    for name, bc in (("transmissive", nv.OFM_BC_TRANSMISSIVE), ("characteristic", nv.OFM_BC_CHARACTERISTIC)):
        s32 = api.Solver(replace(w.solver, bc=bc), "fp32")
        solve_groups(s32, w.cloud, [(64, ids[:8])])             # warm-up (graphs, first launches)
        (q,), secs, cells = solve_groups(s32, w.cloud, [(64, ids)])
        out[name] = dict(gpu_seconds=secs, cell_updates_per_s=cells / secs,
                         p_peak_mean=float(np.mean([d["p_peak"] for d in q])))
    out["ratio"] = out["characteristic"]["cell_updates_per_s"] / out["transmissive"]["cell_updates_per_s"]
    return out


# ------------------------------------------------------------------------------ fitwarm

def cmd_fitwarm(quick):
    """Step 3's variance fit with the finest level started from one pair (the appendix on
    M_L = 1) against the plain warm-up of two pairs per level: 4 levels 8^3..64^3, 20-bubble
    clouds, centre-sensor peak pressure, FP32, tolerance mode; R seeded runs each.  Reports
    the warm-up cost, the total cost, the final error estimate and the estimates."""
    w = W.tiny(16, 20)
    cloud = W.cloud_uniform(20)
    levels = [8, 16, 32, 64]
    R = 3 if quick else 16
    tau = 6.0e5
    s32 = api.Solver(w.solver, "fp32")
    out = dict(experiment="fitwarm", levels=levels, bubbles=20, tau=tau, repeats=R)
    for name, fit in (("plain", False), ("fit", True)):
        runs = []
        for r in range(R):
            warm, _, _ = api.run_ofmlmc(s32, cloud, levels, target=tau, qoi=QOI, seed=W.BASE_SEED + 500 + r,
                                        max_iterations=1, max_cell_steps=4e10, fit_variances=fit)
            res, _, _ = api.run_ofmlmc(s32, cloud, levels, target=tau, qoi=QOI, seed=W.BASE_SEED + 500 + r,
                                       max_iterations=6, max_cell_steps=4e10, fit_variances=fit)
            runs.append(dict(warmup_M=warm["M"], warmup_cell_steps=warm["cell_steps"], M=res["M"],
                             iterations=res["iterations"], cell_steps=res["cell_steps"],
                             gpu_seconds=res["gpu_seconds"], eps=math.sqrt(res["est"]["eps2"]),
                             mean=res["est"]["mean"], capped=res["capped"]))
        out[name] = dict(runs=runs,
                         warmup_cell_steps_mean=float(np.mean([x["warmup_cell_steps"] for x in runs])),
                         cell_steps_mean=float(np.mean([x["cell_steps"] for x in runs])),
                         gpu_seconds_mean=float(np.mean([x["gpu_seconds"] for x in runs])),
                         eps_mean=float(np.mean([x["eps"] for x in runs])),
                         mean_of_estimates=float(np.mean([x["mean"] for x in runs])),
                         spread_of_estimates=float(np.std([x["mean"] for x in runs], ddof=1)))
    return out


# ------------------------------------------------------------------------------ surrogate inside the loop

def cmd_surloop(quick, nearest=(1, 2, 4), levels=None, tau=None, min_pairs=64, steps=600, hidden=256):
    """Plain OF-MLMC against OF-MLMC with the learned surrogate of the top level
    term inside ofm_run, to the same tolerance and with the same seed (FP32,
    20-bubble clouds, centre-sensor peak pressure).  For each number of
    nearest bubbles in the surrogate's input: GPU-seconds to reach tau (the
    surrogate's training and inference included), the final eps, beta, and
    eps^2 x GPU-seconds (at equal GPU-seconds eps^2 scales as 1/cost, so
    this product compares the two at equal GPU-seconds)."""
    cloud = W.cloud_uniform(20)
    sp = W.tiny(16, 20).solver
    levels = levels or ([16, 32] if quick else [16, 32, 64])
    tau = tau or (6.0e5 if quick else 2.5e5)
    s32 = api.Solver(sp, "fp32")
    common = dict(target=tau, qoi=QOI, max_iterations=8, min_samples=16, max_cell_steps=4e11)

    def summary(r):
        e2 = r["est"]["eps2"]
        return dict(gpu_seconds=r["gpu_seconds"], M=r["M"], eps=math.sqrt(e2), mean=r["est"]["mean"],
                    iterations=r["iterations"], capped=r["capped"], eps2_times_gpu_seconds=e2 * r["gpu_seconds"],
                    surrogate_used=r["surrogate_used"], beta=r["beta"], surrogate_seconds=r["surrogate_seconds"],
                    eps_plain_same_pairs=math.sqrt(r["eps2_plain"]),
                    sigma_tilde2=r["est"]["sigma_tilde2"].tolist(),
                    sigma_tilde2_plain=r["sigma_tilde2_plain"].tolist())
    plain, _, _ = api.run_ofmlmc(s32, cloud, levels, **common)
    out = dict(experiment="surloop", levels=levels, tau=tau, bubbles=20, qoi="centre sensor peak pressure [Pa]",
               min_pairs=min_pairs, steps=steps, hidden=hidden, plain=summary(plain), surrogate={})
    for k in nearest:
        r, _, _ = api.run_ofmlmc(s32, cloud, levels, surrogate=True, surrogate_min_pairs=min_pairs,
                                 surrogate_nearest=k, surrogate_steps=steps, surrogate_hidden=hidden, **common)
        out["surrogate"][str(k)] = summary(r)
    return out


# ------------------------------------------------------------------------------ cfg5 to a tolerance

def cmd_cfg5tol(quick, tau_rel=0.01, mean_guess=8.97e6):
    """500-bubble clouds, 4 levels 32^3..256^3 (--quick: 16^3..128^3), peak
    pressure, to tau = 1 % of its mean (mean from the earlier budget run of
    this configuration, 8.97e6 Pa), FP32 stencil with the learned surrogate of
    the top level term enabled (it enters once the finest level has 64 pairs),
    memory-admitted batches.  The plain FP32 estimator on the same final pairs
    is reported beside it.  FP64: its throughput measured per level on the
    same clouds (2 samples, 6 steps each) and the run's cell-steps divided by
    it; the FP32 bias from 3 common clouds solved to t_end in both precisions
    on the two coarsest levels."""
    import torch
    cloud = W.cloud_uniform(500)
    sp = W.SolverParams(sensors=W.centre_sensor())
    levels = [16, 32, 64, 128] if quick else [32, 64, 128, 256]
    tau = tau_rel * mean_guess
    s32 = api.Solver(sp, "fp32")
    res, pairs, ids = api.run_ofmlmc(s32, cloud, levels, target=tau, mode="tol", qoi=0, max_iterations=6,
                                     min_samples=16, max_cell_steps=8e12, capacity=1 << 18, surrogate=True,
                                     surrogate_min_pairs=64, surrogate_nearest=1)
    out = dict(experiment="cfg5tol", levels=levels, bubbles=500, qoi="peak pressure [Pa]", tau=tau,
               M=res["M"], W_cell_steps=res["W"], iterations=res["iterations"], capped=res["capped"],
               failed=res["failed"], gpu_seconds=res["gpu_seconds"], cell_steps=res["cell_steps"],
               eps=math.sqrt(res["est"]["eps2"]), eps_plain_same_pairs=math.sqrt(res["eps2_plain"]),
               mean=res["est"]["mean"], alpha=res["est"]["alpha"].tolist(),
               sigma_tilde2=res["est"]["sigma_tilde2"].tolist(), surrogate_used=res["surrogate_used"],
               beta=res["beta"], surrogate_seconds=res["surrogate_seconds"])
    # FP64 throughput per level on the same clouds
    s64 = api.Solver(sp, "fp64")
    rate64 = []
    for N in levels:
        g = api.make_group(sp, N, level_ids(8, 0, 2), W.BASE_SEED)
        b = api.Batch(s64, cloud, [g])
        b.init()
        b.run(2)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        b.run(6)
        e1.record()
        torch.cuda.synchronize()
        rate64.append(2.0 * N ** 3 * 6 / (e0.elapsed_time(e1) / 1e3))
        b.close()
    fp64_s = float(sum(m * w / r for m, w, r in zip(res["M"], res["W"], rate64)))
    # FP32 bias on common clouds (two coarsest levels, t_end, both precisions)
    bias = []
    for N in levels[:2]:
        sid = level_ids(9, 0, 3)
        (q32,), _, _ = solve_groups(s32, cloud, [(N, sid)])
        (q64,), _, _ = solve_groups(s64, cloud, [(N, sid)])
        bias.append(float(np.mean([a["p_peak"] - b["p_peak"] for a, b in zip(q32, q64)])))
    out.update(fp64_rate_cell_updates_per_s=rate64, fp64_gpu_seconds_extrapolated=fp64_s,
               fp64_over_fp32=fp64_s / max(res["gpu_seconds"], 1e-30), fp32_bias_by_level=bias,
               rmse_fp32=math.sqrt(res["est"]["eps2"] + max(abs(b) for b in bias) ** 2))
    return out


# ------------------------------------------------------------------------------ MLP timing

def cmd_mlptime(quick):
    """The surrogate MLP (3 hidden layers of 256, GELU, BF16 operands, FP32
    accumulation) at the shapes of the surrogate configurations: inference on
    65,536 rows with 4 x 50 + 1 and 4 x 500 + 1 inputs, and training steps on
    512 rows; CUDA events, algorithmic flops 2 rows sum(fan_in fan_out)
    (forward; training 3 times that)."""
    import torch
    out = {}
    for d_in in (201, 2001):
        sizes = [d_in, 256, 256, 256, 1]
        gemm = sum(a * b for a, b in zip(sizes[:-1], sizes[1:]))
        rows = 65536
        net = S.MLP(d_in, 256, 3, 1, max_rows=rows)
        rng = np.random.default_rng(0)
        net.set_params(np.concatenate([np.concatenate([(rng.normal(size=(a, b)) * math.sqrt(2.0 / a)).ravel(),
                                                       np.zeros(b)]) for a, b in zip(sizes[:-1], sizes[1:])])
                       .astype(np.float32))
        X = torch.randn(rows, d_in, device="cuda")
        net.forward(X)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for _ in range(10):
            net.forward(X)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        res = dict(forward_rows=rows, forward_ms=ms, forward_tflops=2.0 * rows * gemm / (ms * 1e-3) / 1e12)
        net.close()
        n_tr = 512
        net = S.MLP(d_in, 256, 3, 1, max_rows=n_tr)
        net.set_params(np.zeros(sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:])), dtype=np.float32) + 0.01)
        Xt = torch.randn(n_tr, d_in, device="cuda")
        Tt = torch.randn(n_tr, 1, device="cuda")
        net.train(Xt, Tt, steps=5)
        torch.cuda.synchronize()
        e0.record()
        net.train(Xt, Tt, steps=100)
        e1.record()
        torch.cuda.synchronize()
        ms_t = e0.elapsed_time(e1) / 100
        res.update(train_rows=n_tr, train_step_ms=ms_t,
                   train_tflops=3 * 2.0 * n_tr * gemm / (ms_t * 1e-3) / 1e12)
        net.close()
        out[f"d_in_{d_in}"] = res
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["uneven3", "unevensmall", "surrogate", "rmse", "cfg5", "epsval", "paper500",
                                     "orders", "fitwarm", "boundaries", "surloop", "cfg5tol", "mlptime"])
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--min-samples", type=int, default=16, help="epsval: pairs every level starts with")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    fn = {"uneven3": cmd_uneven3, "unevensmall": cmd_unevensmall, "surrogate": cmd_surrogate, "rmse": cmd_rmse, "cfg5": cmd_cfg5,
          "epsval": cmd_epsval, "paper500": cmd_paper500, "orders": cmd_orders, "fitwarm": cmd_fitwarm,
          "boundaries": cmd_boundaries, "surloop": cmd_surloop, "cfg5tol": cmd_cfg5tol,
          "mlptime": cmd_mlptime}[a.what]
    print(json.dumps(fn(a.quick, a.min_samples) if a.what == "epsval" else fn(a.quick)), flush=True)


if __name__ == "__main__":
    main()
