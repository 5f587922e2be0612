"""Workload definitions and seeded input generators.

This module is shared by the tests, the benchmark and the CUDA library's
Python binding.  It holds parameters (material constants, grid sizes, sample
counts, sensor positions, end times) and seeded random inputs for tests.  It
contains none of the method's arithmetic: no closure, no flux, no estimator.

Units are SI.  The domain is the cube [0, L]^3 with L = 0.1 m (Section 3.1 of
the paper uses [0, 100 mm]^3).
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import List, Tuple

import numpy as np

DOMAIN_L = 0.1            # m
BASE_SEED = 20170509      # fixed base seed of every synthetic workload

# Material constants.  Phase 1 is the liquid, phase 2 the gas.
EOS_CONFIG = dict(gamma=(6.12, 1.4), pc=(3.43e8, 0.0), rho0=(1000.0, 5.0))
# Section 2.1 gives water gamma = 6.59, pc = 4.049e8 Pa and air 1.4, 0;
# Section 3.1 gives densities 1000 and 5 kg/m^3.
EOS_PAPER = dict(gamma=(6.59, 1.4), pc=(4.049e8, 0.0), rho0=(1000.0, 5.0))

# End time: 60 steps of the 32^3 grid at CFL 0.3 in water at rest at 1e7 Pa
# (c = 1469.8 m/s for the configuration's water), 60 * 0.3 * (0.1/32) / 1469.8.
T_END_CONFIG = 3.827e-5   # s

SENSOR_RADIUS = 5e-4      # m, Eq. (sensor-params)


@dataclass(frozen=True)
class CloudParams:
    n_bubbles: int
    cloud_radius: float            # m, radius of the ball holding the centres
    r_min: float                   # m
    r_max: float                   # m
    radius_law: int = 0            # 0 uniform, 1 log-normal truncated to [r_min, r_max]
    ln_mu: float = float(np.log(1e-3))
    ln_sigma: float = 0.1
    domain_L: float = DOMAIN_L


@dataclass(frozen=True)
class SolverParams:
    gamma: Tuple[float, float] = EOS_CONFIG["gamma"]
    pc: Tuple[float, float] = EOS_CONFIG["pc"]
    rho0: Tuple[float, float] = EOS_CONFIG["rho0"]
    p_gas: float = 2.34e3
    p_liq: float = 1.0e7
    cfl: float = 0.3
    t_end: float = T_END_CONFIG
    bc: int = 0                    # 0 transmissive, 1 periodic, 2 characteristic far field at p_liq
    bc_penalty: float = 1.0        # kappa of the characteristic boundary (0 = transmissive)
    weno_eps: float = 1e-6
    weno_order: int = 5            # 5: WENO5, 3: WENO3 (Jiang & Shu)
    max_steps: int = 100000
    domain_L: float = DOMAIN_L
    sensors: Tuple[Tuple[float, float, float, float], ...] = ()   # (x, y, z, r) in m
    n_out_times: int = 65
    # Cloud pressure ramp (Sec. 3.1; off when ramp_radius == 0): the liquid is at
    # p_cloud within ramp_radius of the domain centre and rises as 1/r towards
    # p_liq beyond it.
    p_cloud: float = 0.0
    ramp_radius: float = 0.0


def centre_sensor() -> Tuple[Tuple[float, float, float, float], ...]:
    c = 0.5 * DOMAIN_L
    return ((c, c, c, SENSOR_RADIUS),)


def eight_sensors(cloud_radius: float) -> Tuple[Tuple[float, float, float, float], ...]:
    """Centre, +-R_cloud/2 on each axis, and 0.45 L from the centre along x."""
    c = 0.5 * DOMAIN_L
    h = 0.5 * cloud_radius
    pts = [(c, c, c),
           (c + h, c, c), (c - h, c, c),
           (c, c + h, c), (c, c - h, c),
           (c, c, c + h), (c, c, c - h),
           (c + 0.45 * DOMAIN_L, c, c)]
    return tuple((x, y, z, SENSOR_RADIUS) for (x, y, z) in pts)


def cloud_uniform(n_bubbles: int) -> CloudParams:
    """Centres uniform in a ball of radius 0.3 L, radii uniform in [0.05, 0.1] L."""
    return CloudParams(n_bubbles=n_bubbles, cloud_radius=0.3 * DOMAIN_L,
                       r_min=0.05 * DOMAIN_L, r_max=0.1 * DOMAIN_L)


def cloud_paper500() -> CloudParams:
    """Section 3.1: 500 bubbles, cloud radius 20 mm, log-normal radii in [0.8, 1.2] mm."""
    return CloudParams(n_bubbles=500, cloud_radius=0.02, r_min=0.8e-3, r_max=1.2e-3,
                       radius_law=1)


@dataclass(frozen=True)
class Workload:
    name: str
    cloud: CloudParams
    solver: SolverParams
    levels: Tuple[int, ...]               # grid N per level, coarse to fine
    samples: Tuple[int, ...]              # M per level
    precision: str = "fp64"


def cfg1() -> Workload:
    """Plain 2-level OF-MLMC, FP64: 4 bubbles, 16 x 16^3 and 4 x 32^3 (pairs with 16^3)."""
    return Workload("cfg1-2level-4bubbles", cloud_uniform(4),
                    SolverParams(sensors=centre_sensor()), (16, 32), (16, 4), "fp64")


def cfg2(precision: str = "fp32") -> Workload:
    """Single-level ensemble: 512 clouds of 20 bubbles on 64^3, 8 sensors."""
    cl = cloud_uniform(20)
    return Workload("cfg2-512x64^3-20bubbles", cl,
                    SolverParams(sensors=eight_sensors(cl.cloud_radius)), (64,), (512,),
                    precision)


def cfg3() -> Workload:
    """3-level OF-MLMC 32^3/64^3/128^3, M = 1024/128/16, 50 bubbles, FP32 stencil."""
    return Workload("cfg3-3level-50bubbles", cloud_uniform(50),
                    SolverParams(sensors=centre_sensor()), (32, 64, 128), (1024, 128, 16), "fp32")


def solver_paper500(**kw) -> SolverParams:
    """Section 3.1 pressures: bubbles and the liquid around them at 0.5 MPa, rising
    from 1 mm beyond the 20 mm cloud surface towards p_inf = 10 MPa; characteristic
    far-field boundaries at p_inf."""
    kw.setdefault("sensors", centre_sensor())
    kw.setdefault("bc", 2)
    return SolverParams(p_gas=0.5e6, p_liq=1.0e7, p_cloud=0.5e6, ramp_radius=0.021, **kw)


def tiny(n: int = 16, n_bubbles: int = 4, samples: int = 2) -> Workload:
    return Workload(f"tiny-{n}", cloud_uniform(n_bubbles),
                    SolverParams(sensors=centre_sensor()), (n,), (samples,), "fp64")


# ---------------------------------------------------------------------------
# Seeded random inputs for tests (no method arithmetic).
# ---------------------------------------------------------------------------

def smooth_periodic_primitives(n: int, seed: int, amp: float = 0.05) -> np.ndarray:
    """Random smooth periodic primitive field W[7][n][n][n] (non-dimensional).

    Variables: a1r1, a2r2, u, v, w, p, a2.  Low Fourier modes only, so the
    field is smooth and periodic on the unit cube with cell centres (i+1/2)/n.
    """
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")

    def field_(scale: float) -> np.ndarray:
        f = np.zeros_like(X)
        for _ in range(3):
            kx, ky, kz = rng.integers(1, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            f += (np.sin(2 * np.pi * kx * X + ph[0]) * np.cos(2 * np.pi * ky * Y + ph[1])
                  * np.sin(2 * np.pi * kz * Z + ph[2]))
        return scale * f / 3.0

    a2 = 0.5 + 0.4 * field_(1.0)
    W = np.empty((7, n, n, n))
    W[0] = (1.0 - a2) * (1.0 + field_(amp))
    W[1] = a2 * 0.005 * (1.0 + field_(amp))
    W[2] = field_(amp)
    W[3] = field_(amp)
    W[4] = field_(amp)
    W[5] = 1.0 + field_(amp)
    W[6] = a2
    return W


def toy_levels(M, L: int, a: float, b: float, seed: int, mu: float = 1.0,
               c: float = 0.5) -> List[np.ndarray]:
    """Draws for the toy hierarchy q_l = mu + c 2^-l + Z + 2^-l (a Z + b Y), Z, Y ~ N(0,1).

    Each sample of pair l draws one Z shared by its two members and an
    independent Y for each member.  Returns, per level l, an array (M_l, 2)
    of (q_l, q_{l-1}) (column 1 is zero for l = 0).  M is an int or a
    per-level sequence.  The hierarchy's means, variances and covariances
    are known in closed form, which pins the estimator oracle.
    """
    rng = np.random.default_rng(seed)
    Ms = [int(M)] * (L + 1) if np.isscalar(M) else [int(m) for m in M]
    out = []
    for l in range(L + 1):
        m = Ms[l]
        Z = rng.standard_normal(m)
        Yf = rng.standard_normal(m)
        Yc = rng.standard_normal(m)
        qf = mu + c * 2.0 ** (-l) + Z + 2.0 ** (-l) * (a * Z + b * Yf)
        if l > 0:
            qc = mu + c * 2.0 ** (-(l - 1)) + Z + 2.0 ** (-(l - 1)) * (a * Z + b * Yc)
        else:
            qc = np.zeros(m)
        out.append(np.stack([qf, qc], axis=1))
    return out


def with_solver(w: Workload, **kw) -> Workload:
    return replace(w, solver=replace(w.solver, **kw))
