"""Pins of the level-wise kernel density oracle (Sec. 3.2): the Gaussian
derivatives against finite differences, the density functionals against
their closed forms for a normal density, the solve-the-equation bandwidth
against the AMISE-optimal bandwidth of a normal density, the single-level
estimate against SciPy's Gaussian KDE, and the unit mass of the level-wise
estimate for any coefficients."""
import math

import numpy as np
import pytest

from oracle import kde

import workloads as W


def test_gaussian_derivatives_match_finite_differences():
    u = np.linspace(-5, 5, 41)
    h = 1e-2
    phi = lambda t: np.exp(-0.5 * t * t) / math.sqrt(2 * math.pi)
    # 4th and 6th derivatives by repeated central differences of the density
    d2 = lambda f: (lambda t: (f(t + h) - 2 * f(t) + f(t - h)) / (h * h))
    d4 = d2(d2(phi))
    d6 = d2(d4)
    assert np.allclose(kde.phi_deriv(u, 4), d4(u), atol=2e-3)
    assert np.allclose(kde.phi_deriv(u, 6), d6(u), atol=3e-2)


def test_density_functionals_of_a_normal_sample():
    """psi_r = int f^(r) f; for N(0, s^2) psi_4 = 3/(8 sqrt(pi) s^5).  With a
    Gaussian pilot g the estimate's expectation is the r-th derivative at 0 of
    the density of X - Y + g Z, i.e. of N(0, 2 s^2 + g^2):
    3/(sqrt(2 pi) v^(5/2)) for r = 4 and -15/(sqrt(2 pi) v^(7/2)) for r = 6."""
    rng = np.random.default_rng(3)
    s = 2.0
    x = s * rng.standard_normal(2000)
    # (pilots well above the sample spacing: the pair term of the U-statistic scales with 1/g^(r+1))
    for g in (2.5, 4.0):
        v = 2 * s * s + g * g
        assert kde.psi_hat(x, 4, g) == pytest.approx(3.0 / (math.sqrt(2 * math.pi) * v ** 2.5), rel=0.05)
        assert kde.psi_hat(x, 6, g) == pytest.approx(-15.0 / (math.sqrt(2 * math.pi) * v ** 3.5), rel=0.08)
    # and the pilot-free limit is the functional itself
    assert 3.0 / (math.sqrt(2 * math.pi) * (2 * s * s) ** 2.5) == pytest.approx(3.0 / (8 * math.sqrt(math.pi) * s ** 5))


@pytest.mark.parametrize("n", [400, 1500])
def test_solve_the_equation_bandwidth_of_a_normal_sample(n):
    """For a normal density the AMISE-optimal Gaussian-kernel bandwidth is
    (4/(3n))^(1/5) s; the solve-the-equation bandwidth estimates it."""
    rng = np.random.default_rng(n)
    s = 0.7
    x = 5.0 + s * rng.standard_normal(n)
    assert kde.sj_bandwidth(x) == pytest.approx((4.0 / (3.0 * n)) ** 0.2 * s, rel=0.15)


def test_bandwidth_is_narrower_for_a_bimodal_sample():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(600) - 3.0, rng.standard_normal(600) + 3.0])
    assert kde.sj_bandwidth(x) < 0.6 * (4.0 / (3.0 * x.size)) ** 0.2 * np.std(x, ddof=1)
    assert kde.sj_bandwidth(x) > 0.5 * (4.0 / (3.0 * 600)) ** 0.2   # about the width for one mode


def test_single_level_estimate_is_scipys_gaussian_kde():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(5)
    q = rng.gamma(3.0, 2.0, size=400)
    pairs = [np.stack([q, np.zeros_like(q)], axis=1)]
    x = np.linspace(-2, 25, 301)
    f, bw = kde.level_kde(pairs, [1.0], x)
    ref = stats.gaussian_kde(q, bw_method=bw[0] / np.std(q, ddof=1))(x)
    assert np.allclose(f, ref, rtol=1e-10, atol=1e-14)


def test_level_wise_density_has_unit_mass_and_the_ofmlmc_mean():
    """For any coefficients the level-wise density has mass alpha_L = 1 and,
    the Gaussian kernel being symmetric, first moment equal to the OF-MLMC
    mean estimate of Eq. (ocv-mlmc) on the same pairs and coefficients."""
    from oracle import estimator as E
    pairs = W.toy_levels([600, 200, 80], 2, 0.5, 0.6, seed=11)
    x = np.linspace(-12, 14, 26001)
    for alpha in ([1.0, 1.0, 1.0], [0.8, 1.3, 1.0]):
        f, _ = kde.level_kde(pairs, alpha, x)
        assert np.trapezoid(f, x) == pytest.approx(1.0, abs=1e-9)
        assert np.trapezoid(x * f, x) == pytest.approx(E.ofmlmc_mean(pairs, np.array(alpha)), abs=1e-8)


def test_small_sample_with_a_wrong_signed_pilot_still_gets_a_bandwidth():
    """A 120-point sample whose pilot estimate of psi_6 comes out positive
    (psi_6 < 0 for any smooth density): the normal-reference psi_6 replaces it
    and the bandwidth stays near the normal-reference one."""
    x = W.toy_levels([300, 120, 40], 2, 0.5, 0.6, seed=12)[1][:, 0]
    s = kde.normal_scale(x)
    b = (-2.0 * kde.K6_0 / (105.0 / (32.0 * math.sqrt(math.pi) * s ** 9) * x.size)) ** (1.0 / 9.0)
    assert kde.psi_hat(x, 6, b) > 0.0           # the case this test is about
    h = kde.sj_bandwidth(x)
    assert np.isfinite(h) and 0.5 < h / ((4.0 / (3.0 * x.size)) ** 0.2 * s) < 2.0
