"""Python front end of the C ABI: configuration marshalling and a Batch object.

Device memory for a batch's workspace comes from PyTorch (a uint8 CUDA
tensor); its raw pointer and the current torch stream are passed to the
library, which does all of the work.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np

from . import native as nv


def solver_config(sp, precision: str = "fp64") -> nv.ofm_solver_config:
    c = nv.ofm_solver_config()
    c.gamma[0], c.gamma[1] = sp.gamma
    c.pc[0], c.pc[1] = sp.pc
    c.rho0[0], c.rho0[1] = sp.rho0
    c.p_gas = sp.p_gas
    c.p_liq = sp.p_liq
    c.p_cloud = getattr(sp, "p_cloud", 0.0)
    c.ramp_radius = getattr(sp, "ramp_radius", 0.0)
    c.bc_penalty = getattr(sp, "bc_penalty", 1.0)
    c.weno_order = getattr(sp, "weno_order", 5)
    c.cfl = sp.cfl
    c.t_end = sp.t_end
    c.weno_eps = sp.weno_eps
    c.domain_L = sp.domain_L
    c.precision = {"fp64": nv.OFM_FP64, "fp32": nv.OFM_FP32}[precision]
    c.bc = sp.bc
    c.max_steps = sp.max_steps
    c.n_sensors = len(sp.sensors)
    for i, s in enumerate(sp.sensors):
        for k in range(4):
            c.sensors[i][k] = s[k]
    c.n_out_times = sp.n_out_times
    return c


def cloud_params(cp) -> nv.ofm_cloud_params:
    c = nv.ofm_cloud_params()
    c.n_bubbles = cp.n_bubbles
    c.radius_law = cp.radius_law
    c.cloud_radius = cp.cloud_radius
    c.r_min = cp.r_min
    c.r_max = cp.r_max
    c.ln_mu = cp.ln_mu
    c.ln_sigma = cp.ln_sigma
    c.domain_L = cp.domain_L
    return c


def sample_cloud(cp, seed: int, sample_id: int) -> np.ndarray:
    out = (nv.ofm_bubble * max(cp.n_bubbles, 1))()
    p = cloud_params(cp)
    nv.check(nv.lib().ofm_sample_cloud(C.byref(p), seed, sample_id, out), "ofm_sample_cloud")
    return np.array([[b.x, b.y, b.z, b.r] for b in out[: cp.n_bubbles]]).reshape(-1, 4)


class Solver:
    def __init__(self, sp, precision: str = "fp64"):
        self.sp = sp
        self.precision = precision
        self.cfg = solver_config(sp, precision)
        h = C.c_void_p()
        nv.check(nv.lib().ofm_solver_create(C.byref(h), C.byref(self.cfg)), "ofm_solver_create")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            nv.lib().ofm_solver_destroy(self.h)
            self.h = None


class Group:
    """Host-side arrays of one group (kept alive for the C side)."""

    def __init__(self, N: int, sample_ids: Sequence[int], seed: int, n_sensors: int, n_out: int,
                 bubbles: Optional[np.ndarray] = None, n_bubbles: int = 0, alpha_hist: bool = False):
        self.N = N
        self.M = len(sample_ids)
        self.ids = np.ascontiguousarray(np.asarray(sample_ids, dtype=np.uint64))
        self.seed = seed
        self.qoi = (nv.ofm_qoi * self.M)()
        self.hist = np.zeros((self.M, max(n_sensors, 0), n_out)) if n_sensors and n_out else None
        # gas-fraction sensor histories on the same output times (opt-in: one more device-to-host copy)
        self.alpha_hist = np.zeros_like(self.hist) if alpha_hist and self.hist is not None else None
        self.bub = None
        if bubbles is not None:
            b = np.ascontiguousarray(np.asarray(bubbles, dtype=np.float64).reshape(self.M * n_bubbles, 4))
            self.bub = b
        self.c = nv.ofm_group()
        self.c.N = N
        self.c.n_samples = self.M
        self.c.sample_ids = self.ids.ctypes.data_as(C.POINTER(C.c_uint64))
        self.c.seed = seed
        self.c.bubbles = self.bub.ctypes.data_as(C.POINTER(nv.ofm_bubble)) if self.bub is not None else None
        self.c.qoi_out = C.cast(self.qoi, C.POINTER(nv.ofm_qoi))
        self.c.sensor_hist = (self.hist.ctypes.data_as(C.POINTER(C.c_double))
                              if self.hist is not None else None)
        self.c.alpha_hist = (self.alpha_hist.ctypes.data_as(C.POINTER(C.c_double))
                             if self.alpha_hist is not None else None)

    def qoi_dicts(self, n_sensors: int) -> List[dict]:
        out = []
        for q in self.qoi:
            out.append(dict(p_peak=q.p_peak, peak_index=q.peak_index, p_peak_xyz=np.array(q.p_peak_xyz[:]),
                            p_peak_t=q.p_peak_t, p_peak_dist=q.p_peak_dist,
                            sensor_peak=np.array(q.sensor_peak[:n_sensors]),
                            totals0=np.array(q.totals0[:]), totals_end=np.array(q.totals_end[:]),
                            t_final=q.t_final, n_steps=q.n_steps, status=q.status, c_max=q.c_max,
                            sensor_alpha0=np.array(q.sensor_alpha0[:n_sensors]),
                            sensor_alpha_min=np.array(q.sensor_alpha_min[:n_sensors]),
                            sensor_alpha_min_t=np.array(q.sensor_alpha_min_t[:n_sensors])))
        return out


def _torch_stream_ptr():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Batch:
    """One ofm_batch: groups of samples on their grids, device workspace from torch."""

    def __init__(self, solver: Solver, cloud, groups: List[Group], device: str = "cuda"):
        import torch
        self.solver = solver
        self.cloud = cloud
        self.cp = cloud_params(cloud)
        self.groups = groups
        self.garr = (nv.ofm_group * len(groups))(*[g.c for g in groups])
        nbytes = C.c_size_t()
        L = nv.lib()
        nv.check(L.ofm_batch_workspace_bytes(solver.h, C.byref(self.cp), self.garr, len(groups),
                                             C.byref(nbytes)), "ofm_batch_workspace_bytes")
        self.ws_bytes = nbytes.value
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        h = C.c_void_p()
        nv.check(L.ofm_batch_create(C.byref(h), solver.h, C.byref(self.cp), self.garr, len(groups),
                                    C.c_void_p(aligned), self.ws_bytes, _torch_stream_ptr()),
                 "ofm_batch_create")
        self.h = h

    def init(self):
        nv.check(nv.lib().ofm_batch_init(self.h), "ofm_batch_init")

    def run(self, max_steps: int = 1 << 30) -> int:
        a = C.c_int()
        nv.check(nv.lib().ofm_batch_run(self.h, max_steps, C.byref(a)), "ofm_batch_run")
        return a.value

    def qoi(self, allow_bad: bool = False) -> int:
        rc = nv.lib().ofm_batch_qoi(self.h)
        if rc == nv.OFM_ENUMERIC and allow_bad:
            return rc
        nv.check(rc, "ofm_batch_qoi")
        return rc

    def _elem(self):
        return np.float64 if self.solver.precision == "fp64" else np.float32

    def state(self, group: int, sample: int) -> np.ndarray:
        N = self.groups[group].N
        buf = np.empty((7, N, N, N), dtype=self._elem())
        nv.check(nv.lib().ofm_batch_copy_state(self.h, group, sample, buf.ctypes.data_as(C.c_void_p),
                                               buf.nbytes), "ofm_batch_copy_state")
        return buf

    def set_state(self, group: int, sample: int, Q: np.ndarray):
        buf = np.ascontiguousarray(Q, dtype=self._elem())
        nv.check(nv.lib().ofm_batch_set_state(self.h, group, sample, buf.ctypes.data_as(C.c_void_p),
                                              buf.nbytes), "ofm_batch_set_state")

    def cell_steps(self) -> float:
        v = C.c_double()
        nv.check(nv.lib().ofm_batch_cell_steps(self.h, C.byref(v)), "ofm_batch_cell_steps")
        return v.value

    def launches(self) -> int:
        v = C.c_int64()
        nv.check(nv.lib().ofm_batch_kernel_launches(self.h, C.byref(v)), "ofm_batch_kernel_launches")
        return v.value

    def set_profiling(self, on: bool):
        nv.check(nv.lib().ofm_batch_set_profiling(self.h, int(on)), "ofm_batch_set_profiling")

    def set_variant(self, variant: int):
        nv.check(nv.lib().ofm_batch_set_variant(self.h, variant), "ofm_batch_set_variant")

    def variant(self):
        v = C.c_int()
        t = (C.c_float * 2)()
        nv.check(nv.lib().ofm_batch_get_variant(self.h, C.byref(v), t), "ofm_batch_get_variant")
        return v.value, tuple(t)

    def stage_time(self):
        ms = C.c_double()
        n = C.c_int64()
        nv.check(nv.lib().ofm_batch_stage_time(self.h, C.byref(ms), C.byref(n)), "ofm_batch_stage_time")
        return ms.value, n.value

    def transfer_bytes(self):
        a = C.c_int64()
        d = C.c_int64()
        nv.check(nv.lib().ofm_batch_transfer_bytes(self.h, C.byref(a), C.byref(d)), "ofm_batch_transfer_bytes")
        return a.value, d.value

    def close(self):
        if getattr(self, "h", None):
            nv.lib().ofm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def make_group(sp, N: int, ids: Sequence[int], seed: int, bubbles=None, n_bubbles: int = 0,
               alpha_hist: bool = False) -> Group:
    return Group(N, ids, seed, len(sp.sensors), sp.n_out_times, bubbles=bubbles, n_bubbles=n_bubbles,
                 alpha_hist=alpha_hist)


def solve_batch_host(solver: Solver, cloud, groups: List[Group], workspace=None) -> int:
    """ofm_solve_batch with host arrays (library-allocated workspace unless given)."""
    cp = cloud_params(cloud)
    garr = (nv.ofm_group * len(groups))(*[g.c for g in groups])
    ws_ptr = C.c_void_p(0)
    ws_bytes = 0
    if workspace is not None:
        ws_ptr = C.c_void_p(workspace[0])
        ws_bytes = workspace[1]
    stream = _torch_stream_ptr()
    return nv.lib().ofm_solve_batch(solver.h, C.byref(cp), garr, len(groups), ws_ptr, ws_bytes, stream)


def estimate(pairs: Sequence[np.ndarray], W: Sequence[float], fit: bool = False) -> dict:
    """ofm_estimate (or, with fit, ofm_estimate_fitted) on per-level (M_l, 2)
    arrays of (q_l, q_{l-1})."""
    L = len(pairs) - 1
    arrs = [np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(-1, 2)) for p in pairs]
    M = (C.c_int64 * (L + 1))(*[a.shape[0] for a in arrs])
    ptrs = (C.POINTER(C.c_double) * (L + 1))(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs])
    Wc = (C.c_double * (L + 1))(*W)
    out = nv.ofm_estimate_out()
    n = L + 1
    res = {}
    if fit:
        vf = (C.c_double * n)()
        nv.check(nv.lib().ofm_estimate_fitted(L, M, ptrs, Wc, C.byref(out), vf), "ofm_estimate_fitted")
        res["V_fit"] = np.array(vf[:n])
    else:
        nv.check(nv.lib().ofm_estimate(L, M, ptrs, Wc, C.byref(out)), "ofm_estimate")
    res.update(alpha=np.array(out.alpha[:n]), sigma2=np.array(out.sigma2[:n]), cov=np.array(out.cov[:n]),
               sigma_tilde2=np.array(out.sigma_tilde2[:n]), mean=out.mean, eps2=out.eps2)
    return res


def estimate_surrogate(pairs: Sequence[np.ndarray], W: Sequence[float], h_top, h_extra, beta=None) -> dict:
    """ofm_estimate_surrogate: OF-MLMC with the surrogate's prediction of the top
    level term as an extra control variate (beta None: the optimal one)."""
    L = len(pairs) - 1
    arrs = [np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(-1, 2)) for p in pairs]
    M = (C.c_int64 * (L + 1))(*[a.shape[0] for a in arrs])
    ptrs = (C.POINTER(C.c_double) * (L + 1))(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs])
    Wc = (C.c_double * (L + 1))(*W)
    ht = np.ascontiguousarray(h_top, dtype=np.float64)
    he = np.ascontiguousarray(h_extra, dtype=np.float64)
    out = nv.ofm_estimate_out()
    b = C.c_double()
    plain = (C.c_double * (L + 1))()
    nv.check(nv.lib().ofm_estimate_surrogate(L, M, ptrs, Wc, ht.ctypes.data_as(C.POINTER(C.c_double)),
                                             he.ctypes.data_as(C.POINTER(C.c_double)),
                                             float("nan") if beta is None else float(beta), C.byref(out),
                                             C.byref(b), plain), "ofm_estimate_surrogate")
    n = L + 1
    return dict(alpha=np.array(out.alpha[:n]), sigma2=np.array(out.sigma2[:n]), cov=np.array(out.cov[:n]),
                sigma_tilde2=np.array(out.sigma_tilde2[:n]), sigma_tilde2_plain=np.array(plain[:n]),
                mean=out.mean, eps2=out.eps2, beta=b.value)


def sj_bandwidth(x) -> float:
    """ofm_sj_bandwidth: the solve-the-equation bandwidth of a Gaussian-kernel KDE."""
    xs = np.ascontiguousarray(x, dtype=np.float64)
    h = C.c_double()
    nv.check(nv.lib().ofm_sj_bandwidth(xs.ctypes.data_as(C.POINTER(C.c_double)), xs.size, C.byref(h)),
             "ofm_sj_bandwidth")
    return h.value


def level_kde(pairs: Sequence[np.ndarray], alpha, x):
    """ofm_level_kde: the level-wise density of Sec. 3.2 on the points x; returns (density, bandwidths)."""
    L = len(pairs) - 1
    arrs = [np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(-1, 2)) for p in pairs]
    M = (C.c_int64 * (L + 1))(*[a.shape[0] for a in arrs])
    ptrs = (C.POINTER(C.c_double) * (L + 1))(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs])
    al = (C.c_double * (L + 1))(*alpha)
    xs = np.ascontiguousarray(x, dtype=np.float64)
    f = np.zeros_like(xs)
    bw = (C.c_double * (L + 1))()
    nv.check(nv.lib().ofm_level_kde(L, M, ptrs, al, xs.ctypes.data_as(C.POINTER(C.c_double)), xs.size,
                                    f.ctypes.data_as(C.POINTER(C.c_double)), bw), "ofm_level_kde")
    return f, np.array(bw[:L + 1])


def fit_level_variances(V: Sequence[float], M: Sequence[int]):
    """ofm_fit_level_variances: (a, b, V_fit) of ln V_l = a + b l (V[0] ignored)."""
    L = len(V) - 1
    Vc = (C.c_double * (L + 1))(*[0.0 if not np.isfinite(v) else float(v) for v in V])
    Mc = (C.c_int64 * (L + 1))(*[int(m) for m in M])
    vf = (C.c_double * (L + 1))()
    coef = (C.c_double * 2)()
    nv.check(nv.lib().ofm_fit_level_variances(L, Mc, Vc, vf, coef), "ofm_fit_level_variances")
    return coef[0], coef[1], np.array(vf[:])


def level_moments(pairs: np.ndarray) -> tuple:
    """ofm_level_moments_of on one level's (M, 2) pairs: (n, mean_f, mean_c, m2_f, m2_c, c_fc)."""
    arr = np.ascontiguousarray(pairs, dtype=np.float64).reshape(-1, 2)
    out = nv.ofm_level_moments()
    nv.check(nv.lib().ofm_level_moments_of(arr.ctypes.data_as(C.POINTER(C.c_double)), arr.shape[0], C.byref(out)),
             "ofm_level_moments_of")
    return (out.n, out.mean_f, out.mean_c, out.m2_f, out.m2_c, out.c_fc)


def _moments_c(m) -> "nv.ofm_level_moments":
    return nv.ofm_level_moments(int(m[0]), *[float(x) for x in m[1:]])


def merge_moments(a, b) -> tuple:
    """ofm_merge_moments: summary of the union of two disjoint pair sets."""
    x, y, out = _moments_c(a), _moments_c(b), nv.ofm_level_moments()
    nv.check(nv.lib().ofm_merge_moments(C.byref(x), C.byref(y), C.byref(out)), "ofm_merge_moments")
    return (out.n, out.mean_f, out.mean_c, out.m2_f, out.m2_c, out.c_fc)


def estimate_moments(moments, W, fit: bool = False) -> dict:
    """ofm_estimate_moments (or, with fit, ofm_estimate_moments_fitted) on per-level summaries."""
    L = len(moments) - 1
    arr = (nv.ofm_level_moments * (L + 1))(*[_moments_c(m) for m in moments])
    Wc = (C.c_double * (L + 1))(*W)
    out = nv.ofm_estimate_out()
    n = L + 1
    res = {}
    if fit:
        vf = (C.c_double * n)()
        nv.check(nv.lib().ofm_estimate_moments_fitted(L, arr, Wc, C.byref(out), vf), "ofm_estimate_moments_fitted")
        res["V_fit"] = np.array(vf[:n])
    else:
        nv.check(nv.lib().ofm_estimate_moments(L, arr, Wc, C.byref(out)), "ofm_estimate_moments")
    res.update(alpha=np.array(out.alpha[:n]), sigma2=np.array(out.sigma2[:n]), cov=np.array(out.cov[:n]),
               sigma_tilde2=np.array(out.sigma_tilde2[:n]), mean=out.mean, eps2=out.eps2)
    return res


def optimal_samples(sigma_tilde2, W, target: float, mode: str = "tol", M_done=None) -> np.ndarray:
    L = len(W) - 1
    s = (C.c_double * (L + 1))(*sigma_tilde2)
    Wc = (C.c_double * (L + 1))(*W)
    Md = (C.c_int64 * (L + 1))(*M_done) if M_done is not None else None
    out = (C.c_int64 * (L + 1))()
    m = nv.OFM_MODE_TOL if mode == "tol" else nv.OFM_MODE_BUDGET
    nv.check(nv.lib().ofm_optimal_samples(L, s, Wc, Md, target, m, out), "ofm_optimal_samples")
    return np.array(out[:])


def probe_fma_tflops(precision: str = "fp32") -> float:
    """ofm_probe_fma_tflops on the current device and torch stream."""
    out = C.c_double()
    prec = nv.OFM_FP32 if precision == "fp32" else nv.OFM_FP64
    nv.check(nv.lib().ofm_probe_fma_tflops(prec, C.byref(out), _torch_stream_ptr()), "ofm_probe_fma_tflops")
    return out.value


def warmup_samples(W) -> np.ndarray:
    L = len(W) - 1
    Wc = (C.c_double * (L + 1))(*W)
    out = (C.c_int64 * (L + 1))()
    nv.check(nv.lib().ofm_warmup_samples(L, Wc, out), "ofm_warmup_samples")
    return np.array(out[:])


def run_ofmlmc(solver: Solver, cloud, levels, target: float, mode: str = "tol", qoi: int = 0,
               seed: int = 20170509, max_iterations: int = 10, min_samples: int = 2,
               max_batch_bytes: int = 0, capacity: int = 1 << 16, max_cell_steps: float = 0.0,
               fit_variances: bool = False, surrogate: bool = False, surrogate_min_pairs: int = 0,
               surrogate_nearest: int = 0, surrogate_steps: int = 0, surrogate_hidden: int = 0,
               surrogate_lr: float = 0.0):
    """ofm_run: the adaptive OF-MLMC loop over GPU solves.  Returns (result dict, pairs per level, ids per level).
    fit_variances: step 3's variance fit, and one warm-up pair on the finest of L >= 3 levels.
    surrogate: the learned surrogate of q_L as an extra control variate of the top level term
    (the result then holds its predictions per pair under "h", NaN where none)."""
    cfg = nv.ofm_run_config()
    cfg.L = len(levels) - 1
    for i, n in enumerate(levels):
        cfg.N[i] = n
    cfg.mode = nv.OFM_MODE_TOL if mode == "tol" else nv.OFM_MODE_BUDGET
    cfg.target = target
    cfg.qoi = qoi
    cfg.seed = seed
    cfg.max_iterations = max_iterations
    cfg.min_samples = min_samples
    cfg.max_batch_bytes = max_batch_bytes
    cfg.max_cell_steps = max_cell_steps
    cfg.fit_variances = 1 if fit_variances else 0
    cfg.surrogate = 1 if surrogate else 0
    cfg.surrogate_min_pairs = surrogate_min_pairs
    cfg.surrogate_nearest = surrogate_nearest
    cfg.surrogate_steps = surrogate_steps
    cfg.surrogate_hidden = surrogate_hidden
    cfg.surrogate_lr = surrogate_lr
    h = np.full(capacity, np.nan)
    cfg.surrogate_h_out = h.ctypes.data_as(C.POINTER(C.c_double))
    cp = cloud_params(cloud)
    pairs = np.zeros((capacity, 2))
    ids = np.zeros(capacity, dtype=np.uint64)
    res = nv.ofm_run_result()
    nv.check(nv.lib().ofm_run(solver.h, C.byref(cp), C.byref(cfg), pairs.ctypes.data_as(C.POINTER(C.c_double)),
                              ids.ctypes.data_as(C.POINTER(C.c_uint64)), capacity, C.byref(res),
                              _torch_stream_ptr()), "ofm_run")
    L = cfg.L
    M = [res.M[l] for l in range(L + 1)]
    per_pairs, per_ids, per_h, at = [], [], [], 0
    for l in range(L + 1):
        per_pairs.append(pairs[at:at + M[l]].copy())
        per_ids.append(ids[at:at + M[l]].copy())
        per_h.append(h[at:at + M[l]].copy())
        at += M[l]
    n = L + 1
    est = dict(alpha=np.array(res.est.alpha[:n]), sigma2=np.array(res.est.sigma2[:n]),
               cov=np.array(res.est.cov[:n]), sigma_tilde2=np.array(res.est.sigma_tilde2[:n]),
               mean=res.est.mean, eps2=res.est.eps2)
    out = dict(iterations=res.iterations, M=M, W=[res.W[l] for l in range(n)], gpu_seconds=res.gpu_seconds,
               cell_steps=res.cell_steps, failed=res.failed, capped=res.capped, est=est,
               surrogate_used=bool(res.surrogate_used), beta=res.beta, surrogate_seconds=res.surrogate_seconds,
               eps2_plain=res.eps2_plain, sigma_tilde2_plain=np.array(res.sigma_tilde2_plain[:n]), h=per_h)
    return out, per_pairs, per_ids
