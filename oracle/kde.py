"""Oracle for the level-wise kernel density estimate of Sec. 3.2 (test infrastructure).

Plain numpy in FP64.  Sec. 3.2 estimates the PDF of a QoI with level-dependent
kernel density estimators whose bandwidth comes from the "solve-the-equation"
method of Sheather and Jones (1991).  Readings (the paper gives no formula):

  - the density is the OF-MLMC estimator (Eq. ocv-mlmc) of E[K_b(x - q)]:
        f(x) = sum_l (1/M_l) sum_i [alpha_l K_{b_l}(x - q_l^i) - alpha_{l-1} K_{b_l}(x - q_{l-1}^i)]
    (alpha_{-1} = 0), with the Gaussian kernel K_b(u) = exp(-u^2/(2 b^2))/(b sqrt(2 pi));
    it integrates to alpha_L = 1 for any coefficients;
  - level l uses one bandwidth for both members of its pairs, the larger of
    the two members' solve-the-equation bandwidths ("maximum bandwidth").

Solve-the-equation bandwidth for the Gaussian kernel (R(K) = 1/(2 sqrt pi),
mu_2(K) = 1): h solves h = [R(K) / (n psi_4(g(h)))]^(1/5) with the density
functional psi_r = int f^(r) f estimated as
    psi_r(g) = sum_{i != j} phi^(r)((x_i - x_j)/g) / (n (n - 1) g^(r+1)),
and the pilot bandwidth g(h) = [2 K^(4)(0) mu_2 / R(K)]^(1/7) [psi_4(a) / -psi_6(b)]^(1/7) h^(5/7),
where a and b are the pilot bandwidths for psi_4 and psi_6 under a normal
reference with scale s = min(sd, IQR/1.349):
    a = [-2 K^(4)(0) / (mu_2 psi_6^N n)]^(1/7),  b = [-2 K^(6)(0) / (mu_2 psi_8^N n)]^(1/9),
    psi_6^N = -15 / (16 sqrt(pi) s^7),  psi_8^N = 105 / (32 sqrt(pi) s^9).
A pilot estimate with the wrong sign (psi_4 > 0 > psi_6 for any smooth
density; a small sample can break it) takes its normal-reference value,
psi_4^N = 3/(8 sqrt(pi) s^5) or psi_6^N.  The root is bracketed (from the normal-reference bandwidth (4/(3n))^(1/5) s,
doubling or halving; a trial h whose pilot estimate of psi_4 is not positive
counts as too small) and found by bisection.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

SQRT2PI = math.sqrt(2.0 * math.pi)
RK = 1.0 / (2.0 * math.sqrt(math.pi))          # R(K) of the Gaussian kernel
K4_0 = 3.0 / SQRT2PI                            # K''''(0)
K6_0 = -15.0 / SQRT2PI                          # K^(6)(0)


def phi_deriv(u: np.ndarray, r: int) -> np.ndarray:
    """r-th derivative of the standard normal density (r = 4 or 6):
    phi(u) He_r(u) with the probabilists' Hermite polynomials."""
    phi = np.exp(-0.5 * u * u) / SQRT2PI
    if r == 4:
        return phi * (u ** 4 - 6.0 * u ** 2 + 3.0)
    if r == 6:
        return phi * (u ** 6 - 15.0 * u ** 4 + 45.0 * u ** 2 - 15.0)
    raise ValueError(r)


def psi_hat(x: np.ndarray, r: int, g: float) -> float:
    """psi_r estimated with bandwidth g, the diagonal i = j left out."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    iu = np.triu_indices(n, 1)
    d = (x[iu[0]] - x[iu[1]]) / g           # phi^(r) is even: each unordered pair twice
    return float(2.0 * phi_deriv(d, r).sum() / (n * (n - 1) * g ** (r + 1)))


def normal_scale(x: np.ndarray) -> float:
    x = np.asarray(x, dtype=np.float64)
    sd = float(np.std(x, ddof=1))
    q75, q25 = np.percentile(x, [75.0, 25.0])
    iqr = float(q75 - q25) / 1.349
    return min(sd, iqr) if iqr > 0.0 else sd


def sj_bandwidth(x: Sequence[float], iters: int = 200) -> float:
    """Sheather-Jones solve-the-equation bandwidth of a Gaussian-kernel KDE."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 2:
        raise ValueError("needs two samples")
    s = normal_scale(x)
    if not s > 0.0:
        return 0.0
    psi6_n = -15.0 / (16.0 * math.sqrt(math.pi) * s ** 7)
    psi8_n = 105.0 / (32.0 * math.sqrt(math.pi) * s ** 9)
    a = (-2.0 * K4_0 / (psi6_n * n)) ** (1.0 / 7.0)
    b = (-2.0 * K6_0 / (psi8_n * n)) ** (1.0 / 9.0)
    # psi_4 > 0 > psi_6 for any smooth density; a small sample can give a pilot
    # estimate of the wrong sign, which then takes its normal-reference value
    p4 = psi_hat(x, 4, a)
    p6 = psi_hat(x, 6, b)
    if not p4 > 0.0:
        p4 = 3.0 / (8.0 * math.sqrt(math.pi) * s ** 5)
    if not p6 < 0.0:
        p6 = psi6_n
    ratio = p4 / -p6
    c_g = (2.0 * K4_0 / RK * ratio) ** (1.0 / 7.0)

    def f(h):
        p4 = psi_hat(x, 4, c_g * h ** (5.0 / 7.0))
        if not p4 > 0.0:            # a pilot bandwidth this small resolves no curvature: h is too small
            return math.inf
        return (RK / (n * p4)) ** 0.2 - h

    # bracket around the normal-reference bandwidth (4/(3n))^(1/5) s
    h0 = (4.0 / (3.0 * n)) ** 0.2 * s
    lo, hi = h0, h0
    while f(hi) > 0.0:
        hi *= 2.0
    while f(lo) < 0.0:
        lo *= 0.5
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-10 * hi:
            break
    return 0.5 * (lo + hi)


def gauss_kde(samples: np.ndarray, b: float, x: np.ndarray) -> np.ndarray:
    """(1/n) sum_i K_b(x - samples_i)."""
    u = (np.asarray(x, dtype=np.float64)[:, None] - np.asarray(samples, dtype=np.float64)[None, :]) / b
    return np.exp(-0.5 * u * u).sum(axis=1) / (samples.size * b * SQRT2PI)


def level_kde(pairs, alpha, x):
    """The level-wise density and the bandwidth of every level (reading above)."""
    L = len(pairs) - 1
    x = np.asarray(x, dtype=np.float64)
    f = np.zeros_like(x)
    bw = np.zeros(L + 1)
    for l in range(L + 1):
        fine = pairs[l][:, 0]
        b = sj_bandwidth(fine)
        if l > 0:
            b = max(b, sj_bandwidth(pairs[l][:, 1]))
        bw[l] = b
        f += alpha[l] * gauss_kde(fine, b, x)
        if l > 0:
            f -= alpha[l - 1] * gauss_kde(pairs[l][:, 1], b, x)
    return f, bw
