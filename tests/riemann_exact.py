"""Exact solution of the 1-D Riemann problem for two stiffened gases.

Independent pin for the oracle solver (Section 2.2's scheme must converge to
it).  Follows the classical exact Riemann solver for the Euler equations
(Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4)
with each side's pressure shifted by its stiffening constant, p -> p + pc,
which maps a stiffened gas onto an ideal gas with the same gamma.  The
material interface moves with the contact.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Side:
    rho: float
    u: float
    p: float
    gamma: float
    pc: float

    @property
    def c(self) -> float:
        return math.sqrt(self.gamma * (self.p + self.pc) / self.rho)


def _f(s: Side, pstar: float):
    """Toro's pressure function and its derivative for one side."""
    g = s.gamma
    P = pstar + s.pc
    Pk = s.p + s.pc
    if P > Pk:  # shock
        A = 2.0 / ((g + 1.0) * s.rho)
        B = (g - 1.0) / (g + 1.0) * Pk
        sq = math.sqrt(A / (P + B))
        f = (P - Pk) * sq
        df = sq * (1.0 - 0.5 * (P - Pk) / (P + B))
    else:  # rarefaction
        f = 2.0 * s.c / (g - 1.0) * ((P / Pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (s.rho * s.c) * (P / Pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(L: Side, R: Side):
    """(p*, u*) by Newton iteration on f_L + f_R + du = 0, bracketed."""
    du = R.u - L.u
    lo = max(-L.pc, -R.pc) + 1e-14 * max(1.0, L.p + L.pc, R.p + R.pc)
    hi = 10.0 * max(L.p + L.pc, R.p + R.pc) + 1.0
    while _f(L, hi)[0] + _f(R, hi)[0] + du < 0.0:
        hi *= 2.0
    p = 0.5 * (L.p + R.p)
    p = min(max(p, lo), hi)
    for _ in range(200):
        fl, dl = _f(L, p)
        fr, dr = _f(R, p)
        g = fl + fr + du
        if g > 0:
            hi = p
        else:
            lo = p
        pn = p - g / (dl + dr)
        if not (lo < pn < hi):
            pn = 0.5 * (lo + hi)
        if abs(pn - p) <= 1e-15 * abs(p + max(L.pc, R.pc)) + 1e-300:
            p = pn
            break
        p = pn
    fl, _ = _f(L, p)
    fr, _ = _f(R, p)
    u = 0.5 * (L.u + R.u) + 0.5 * (fr - fl)
    return p, u


def sample(L: Side, R: Side, xi: np.ndarray):
    """Return (rho, u, p, left_material) at similarity coordinates xi = (x - x0)/t."""
    ps, us = star_state(L, R)
    rho = np.zeros_like(xi)
    u = np.zeros_like(xi)
    p = np.zeros_like(xi)
    left = np.zeros(xi.shape, dtype=bool)
    for n, S in enumerate(xi):
        if S <= us:
            K, sgn = L, 1.0
            left[n] = True
        else:
            K, sgn = R, -1.0
        g = K.gamma
        Pk = K.p + K.pc
        P = ps + K.pc
        if P > Pk:  # shock on side K
            Ssh = K.u - sgn * K.c * math.sqrt((g + 1.0) / (2.0 * g) * P / Pk + (g - 1.0) / (2.0 * g))
            behind = (S >= Ssh) if sgn > 0 else (S <= Ssh)
            if behind:
                r = (g - 1.0) / (g + 1.0)
                rho[n] = K.rho * (P / Pk + r) / (r * P / Pk + 1.0)
                u[n], p[n] = us, ps
            else:
                rho[n], u[n], p[n] = K.rho, K.u, K.p
        else:  # rarefaction on side K
            cs = K.c * (P / Pk) ** ((g - 1.0) / (2.0 * g))
            head = K.u - sgn * K.c
            tail = us - sgn * cs
            if (sgn > 0 and S <= head) or (sgn < 0 and S >= head):
                rho[n], u[n], p[n] = K.rho, K.u, K.p
            elif (sgn > 0 and S >= tail) or (sgn < 0 and S <= tail):
                rho[n] = K.rho * (P / Pk) ** (1.0 / g)
                u[n], p[n] = us, ps
            else:  # inside the fan
                uu = 2.0 / (g + 1.0) * (sgn * K.c + 0.5 * (g - 1.0) * K.u + S)
                cc = 2.0 / (g + 1.0) * (K.c + sgn * 0.5 * (g - 1.0) * (K.u - S))
                rho[n] = K.rho * (cc / K.c) ** (2.0 / (g - 1.0))
                u[n] = uu
                p[n] = Pk * (cc / K.c) ** (2.0 * g / (g - 1.0)) - K.pc
    return rho, u, p, left
