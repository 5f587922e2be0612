"""ctypes front end of the oracle's plain FP64 C solver (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  It loads ``liborc.so`` built from ``oracle/solver.c`` and does the
SI <-> non-dimensional conversion of the configuration.

Non-dimensional units (reading: the paper gives no scaling): length L,
density rho_ref = 1000 kg/m^3, pressure p_ref = p_liq, velocity
u_ref = sqrt(p_ref/rho_ref), time L/u_ref.  QoIs are returned in SI.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

NV = 7
RHO_REF = 1000.0


class OrcGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("bc", C.c_int),
                ("h", C.c_double), ("gamma1", C.c_double), ("gamma2", C.c_double),
                ("pc1", C.c_double), ("pc2", C.c_double), ("cfl", C.c_double),
                ("weno_eps", C.c_double), ("p_inf", C.c_double), ("bc_penalty", C.c_double),
                ("weno_order", C.c_int)]


class OrcQoi(C.Structure):
    _fields_ = [("p_peak", C.c_double), ("peak_index", C.c_long), ("p_peak_t", C.c_double),
                ("sensor_peak", C.c_double * 8), ("totals0", C.c_double * 6),
                ("totals_end", C.c_double * 6), ("n_steps", C.c_int), ("status", C.c_int),
                ("t_final", C.c_double), ("c_max", C.c_double), ("sensor_alpha0", C.c_double * 8),
                ("sensor_alpha_min", C.c_double * 8), ("sensor_alpha_min_t", C.c_double * 8)]


_LIBS = {}
_D = C.POINTER(C.c_double)


def _lib(count: bool = False) -> C.CDLL:
    name = "liborc_count.so" if count else "liborc.so"
    if name not in _LIBS:
        _build.build()
        lib = C.CDLL(_build.lib_path(name))
        G = C.POINTER(OrcGrid)
        lib.orc_prim_from_cons.argtypes = [G, _D, _D]
        lib.orc_cons_from_prim.argtypes = [G, _D, _D]
        lib.orc_prim_to_cons_array.argtypes = [G, _D, _D, C.c_long]
        lib.orc_cons_to_prim_array.argtypes = [G, _D, _D, C.c_long]
        lib.orc_weno5.argtypes = [C.c_double] * 6
        lib.orc_weno5.restype = C.c_double
        lib.orc_weno3.argtypes = [C.c_double] * 4
        lib.orc_weno3.restype = C.c_double
        lib.orc_hllc.argtypes = [G, _D, _D, C.c_int, _D, _D]
        lib.orc_rhs.argtypes = [G, _D, _D]
        lib.orc_rhs.restype = C.c_int
        lib.orc_rk3_step.argtypes = [G, _D, C.c_double]
        lib.orc_rk3_step.restype = C.c_int
        lib.orc_rk_coefficients.argtypes = [_D, _D]
        lib.orc_max_speed.argtypes = [G, _D]
        lib.orc_max_speed.restype = C.c_double
        lib.orc_totals.argtypes = [G, _D, _D]
        lib.orc_init_cloud.argtypes = [G, _D, C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_double, _D]
        lib.orc_sensor_cell_count.argtypes = [G, _D]
        lib.orc_sensor_cell_count.restype = C.c_int
        lib.orc_solve.argtypes = [G, _D, C.c_double, C.c_int, C.c_int, _D, C.c_int, _D, _D,
                                  C.POINTER(OrcQoi)]
        lib.orc_solve.restype = C.c_int
        lib.orc_advance.argtypes = [G, _D, C.c_double, C.c_int, C.POINTER(C.c_int)]
        lib.orc_advance.restype = C.c_int
        lib.orc_flop_count.restype = C.c_double
        lib.orc_admissible.argtypes = [G, _D]
        lib.orc_admissible.restype = C.c_int
        lib.orc_fallback_count.restype = C.c_long
        _LIBS[name] = lib
    return _LIBS[name]


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


@dataclass
class Units:
    L: float
    p_ref: float

    @property
    def u_ref(self) -> float:
        return math.sqrt(self.p_ref / RHO_REF)

    @property
    def t_ref(self) -> float:
        return self.L / self.u_ref


def make_grid(nx: int, ny: Optional[int] = None, nz: Optional[int] = None, *, gamma=(6.12, 1.4),
              pc_nd=(34.3, 0.0), bc: int = 0, h: Optional[float] = None, cfl: float = 0.3,
              weno_eps: float = 1e-6, p_inf: float = 1.0, bc_penalty: float = 1.0,
              weno_order: int = 5) -> OrcGrid:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    g = OrcGrid()
    g.nx, g.ny, g.nz, g.bc = nx, ny, nz, bc
    g.h = 1.0 / nx if h is None else h
    g.gamma1, g.gamma2 = gamma
    g.pc1, g.pc2 = pc_nd
    g.cfl = cfl
    g.weno_eps = weno_eps
    g.p_inf = p_inf
    g.bc_penalty = bc_penalty
    g.weno_order = weno_order
    return g


def grid_from_params(sp, N: int) -> OrcGrid:
    u = Units(sp.domain_L, sp.p_liq)
    # the far field of the characteristic boundary is the liquid pressure p_liq = p_ref
    return make_grid(N, gamma=tuple(sp.gamma), pc_nd=(sp.pc[0] / u.p_ref, sp.pc[1] / u.p_ref),
                     bc=sp.bc, cfl=sp.cfl, weno_eps=sp.weno_eps, p_inf=1.0,
                     bc_penalty=getattr(sp, "bc_penalty", 1.0), weno_order=getattr(sp, "weno_order", 5))


def cells(g: OrcGrid) -> int:
    return g.nx * g.ny * g.nz


def prim_to_cons(g: OrcGrid, W: np.ndarray) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    n = W.size // NV
    Q = np.empty_like(W)
    _lib().orc_prim_to_cons_array(C.byref(g), _p(W), _p(Q), n)
    return Q


def cons_to_prim(g: OrcGrid, Q: np.ndarray) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    n = Q.size // NV
    W = np.empty_like(Q)
    _lib().orc_cons_to_prim_array(C.byref(g), _p(Q), _p(W), n)
    return W


def weno5(a, b, c, d, e, eps=1e-6) -> float:
    return _lib().orc_weno5(a, b, c, d, e, eps)


def weno3(a, b, c, eps=1e-6) -> float:
    return _lib().orc_weno3(a, b, c, eps)


def hllc(g: OrcGrid, wl, wr, direction: int):
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    F = np.zeros(NV)
    uf = C.c_double(0.0)
    _lib().orc_hllc(C.byref(g), _p(wl), _p(wr), direction, _p(F), C.byref(uf))
    return F, uf.value


def rhs(g: OrcGrid, Q: np.ndarray) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    R = np.empty_like(Q)
    if _lib().orc_rhs(C.byref(g), _p(Q), _p(R)) != 0:
        raise MemoryError("orc_rhs")
    return R


def rk3_step(g: OrcGrid, Q: np.ndarray, dt: float, count: bool = False) -> np.ndarray:
    Q = np.array(Q, dtype=np.float64, order="C", copy=True)
    if _lib(count).orc_rk3_step(C.byref(g), _p(Q), dt) != 0:
        raise MemoryError("orc_rk3_step")
    return Q


def rk_coefficients():
    A = np.zeros(3)
    B = np.zeros(3)
    _lib().orc_rk_coefficients(_p(A), _p(B))
    return A, B


def max_speed(g: OrcGrid, Q: np.ndarray) -> float:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    return _lib().orc_max_speed(C.byref(g), _p(Q))


def totals(g: OrcGrid, Q: np.ndarray) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    t = np.zeros(6)
    _lib().orc_totals(C.byref(g), _p(Q), _p(t))
    return t


def advance(g: OrcGrid, Q: np.ndarray, t_end: float, max_steps: int = 100000):
    Q = np.array(Q, dtype=np.float64, order="C", copy=True)
    n = C.c_int(0)
    rc = _lib().orc_advance(C.byref(g), _p(Q), t_end, max_steps, C.byref(n))
    if rc != 0:
        raise RuntimeError(f"orc_advance rc={rc}")
    return Q, n.value


def admissible(g: OrcGrid, w) -> bool:
    """The face-state test of the positivity fallback (reading of Sec. 2.2)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    return bool(_lib().orc_admissible(C.byref(g), _p(w)))


def fallback_count() -> int:
    """Face states that fell back to their cell's primitives in this thread
    since the last fallback_reset() (test hook)."""
    return int(_lib().orc_fallback_count())


def fallback_reset() -> None:
    _lib().orc_fallback_reset()


def flop_count() -> float:
    return _lib(True).orc_flop_count()


def flop_reset() -> None:
    _lib(True).orc_flop_reset()


def bubbles_nd(bubbles_si: np.ndarray, L: float) -> np.ndarray:
    """(nb, 4) metres -> (nb, 4) in units of L."""
    return np.ascontiguousarray(np.asarray(bubbles_si, dtype=np.float64) / L)


def init_cloud(sp, N: int, bubbles_si: np.ndarray) -> np.ndarray:
    """Initial state Q[7][N][N][N] (non-dimensional) for one cloud."""
    g = grid_from_params(sp, N)
    u = Units(sp.domain_L, sp.p_liq)
    b = bubbles_nd(bubbles_si, sp.domain_L).reshape(-1)
    nb = b.size // 4
    Q = np.zeros((NV, N, N, N))
    _lib().orc_init_cloud(C.byref(g), _p(b) if nb else None, nb, sp.rho0[0] / RHO_REF,
                          sp.rho0[1] / RHO_REF, sp.p_gas / u.p_ref, sp.p_liq / u.p_ref,
                          sp.p_cloud / u.p_ref, sp.ramp_radius / sp.domain_L, _p(Q))
    return Q


QOI_FIELDS = ("p_peak", "p_peak_x", "p_peak_y", "p_peak_z", "p_peak_t", "p_peak_dist",
              "n_steps", "status")


def solve(sp, N: int, bubbles_si: np.ndarray, count_flops: bool = False,
          Q0: Optional[np.ndarray] = None):
    """Solve one cloud to t_end on N^3 and return (qoi dict, sensor histories, final Q).

    QoIs in SI: p_peak [Pa], its cell-centre location [m] and time [s], its
    distance from the domain centre [m], sensor peaks [Pa], conserved totals
    (non-dimensional), step count and status bits; c_max [m/s], the maximum
    over time of the maximum mixture sound speed; per sensor the gas fraction
    (mean alpha2 over the sensor's cells) at t = 0, its minimum over time and
    the first time of that minimum [s].
    """
    g = grid_from_params(sp, N)
    u = Units(sp.domain_L, sp.p_liq)
    Q = init_cloud(sp, N, bubbles_si) if Q0 is None else np.array(Q0, dtype=np.float64)
    ns = len(sp.sensors)
    sens = np.ascontiguousarray(np.asarray(sp.sensors, dtype=np.float64).reshape(-1) / sp.domain_L) \
        if ns else np.zeros(4)
    n_out = sp.n_out_times
    hist = np.zeros(max(ns, 1) * n_out)
    ahist = np.zeros(max(ns, 1) * n_out)
    out = OrcQoi()
    rc = _lib(count_flops).orc_solve(C.byref(g), _p(Q), sp.t_end / u.t_ref, sp.max_steps, ns,
                                     _p(sens), n_out, _p(hist), _p(ahist), C.byref(out))
    if rc != 0:
        raise RuntimeError(f"orc_solve rc={rc}")
    idx = out.peak_index
    i, j, k = idx % N, (idx // N) % N, idx // (N * N)
    h = 1.0 / N
    xyz = np.array([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h]) * sp.domain_L
    centre = 0.5 * sp.domain_L
    q = dict(
        p_peak=out.p_peak * u.p_ref,
        peak_index=idx,
        p_peak_xyz=xyz,
        p_peak_t=out.p_peak_t * u.t_ref,
        p_peak_dist=float(np.sqrt(np.sum((xyz - centre) ** 2))),
        sensor_peak=np.array(out.sensor_peak[:ns]) * u.p_ref,
        totals0=np.array(out.totals0[:]),
        totals_end=np.array(out.totals_end[:]),
        n_steps=out.n_steps,
        status=out.status,
        t_final=out.t_final * u.t_ref,
        c_max=out.c_max * u.u_ref,
        sensor_alpha0=np.array(out.sensor_alpha0[:ns]),
        sensor_alpha_min=np.array(out.sensor_alpha_min[:ns]),
        sensor_alpha_min_t=np.array(out.sensor_alpha_min_t[:ns]) * u.t_ref,
        alpha_hist=ahist[: ns * n_out].reshape(ns, n_out).copy(),
    )
    return q, hist[: ns * n_out].reshape(ns, n_out) * u.p_ref, Q
