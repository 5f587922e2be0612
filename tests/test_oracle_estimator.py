"""Pins of the estimator oracle: closed forms, special cases, brute force,
the paper's printed numbers, and a toy hierarchy with known moments."""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize

import workloads as Wk
from oracle import estimator as E

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ofmlmc_paper_numbers.json")))


def toy_moments(L, a, b, mu=1.0, c=0.5):
    """Closed forms for q_l = mu + c 2^-l + (1 + a 2^-l) Z + b 2^-l Y."""
    s = lambda l: 1.0 + a * 2.0 ** (-l)
    mean = [mu + c * 2.0 ** (-l) for l in range(L + 1)]
    var = [s(l) ** 2 + b ** 2 * 4.0 ** (-l) for l in range(L + 1)]
    cov = [0.0] + [s(l) * s(l - 1) for l in range(1, L + 1)]
    return np.array(mean), np.array(var), np.array(cov)


def test_two_level_closed_form():
    """L = 1: alpha_0 = W_1/(W_1 + W_0) Cov/V[q_0], Eq. (alpha-opt-works)."""
    s2 = np.array([2.0, 3.0])
    cov = np.array([0.0, 1.7])
    W = np.array([1.0, 17.0])
    a = E.alpha_optimal(s2, cov, W)
    assert a[1] == 1.0
    assert abs(a[0] - 17.0 / 18.0 * 1.7 / 2.0) < 1e-15


def test_alpha_minimises_cost_brute_force():
    rng = np.random.default_rng(0)
    for L in (2, 3, 4):
        s2 = rng.uniform(0.5, 2.0, L + 1)
        cov = np.concatenate([[0.0], rng.uniform(0.2, 0.9, L) * np.sqrt(s2[1:] * s2[:-1])])
        W = 16.0 ** np.arange(L + 1)
        a = E.alpha_optimal(s2, cov, W)
        f = lambda x: E.cost_functional(np.append(x, 1.0), s2, cov, W)
        res = minimize(f, np.ones(L), method="Nelder-Mead",
                       options=dict(xatol=1e-10, fatol=1e-12, maxiter=20000, maxfev=40000))
        assert np.allclose(a[:L], res.x, rtol=1e-4, atol=1e-6)
        assert f(a[:L]) <= f(np.ones(L)) + 1e-12
        assert f(a[:L]) <= res.fun * (1 + 1e-12)
        for _ in range(200):   # no nearby point does better
            d = rng.normal(size=L) * 10.0 ** rng.uniform(-6, -1)
            assert f(a[:L] + d) >= f(a[:L]) * (1 - 1e-14)


def test_alpha_one_reduces_to_classical_mlmc():
    pairs = Wk.toy_levels(50, 3, 0.3, 0.4, seed=1)
    assert abs(E.ofmlmc_mean(pairs, np.ones(4)) - E.mlmc_mean(pairs)) == 0.0
    manual = pairs[0][:, 0].mean() + sum((p[:, 0] - p[:, 1]).mean() for p in pairs[1:])
    assert abs(E.mlmc_mean(pairs) - manual) < 1e-14


def test_indicators_converge_to_closed_forms():
    L, a, b = 3, 0.5, 0.8
    pairs = Wk.toy_levels(200000, L, a, b, seed=2)
    _, var, cov = toy_moments(L, a, b)
    s2, c = E.indicators(pairs)
    assert np.allclose(s2, var, rtol=0.01)
    assert np.allclose(c[1:], cov[1:], rtol=0.01)
    W = 16.0 ** np.arange(L + 1)
    assert np.allclose(E.alpha_optimal(s2, c, W), E.alpha_optimal(var, cov, W), rtol=0.02)


def test_estimator_unbiased_and_error_estimate_matches_rmse():
    L, a, b = 2, 0.5, 1.0
    mean, var, cov = toy_moments(L, a, b)
    W = np.array([1.0, 17.0, 272.0])
    alpha = E.alpha_optimal(var, cov, W)    # fixed coefficients: exactly unbiased
    M = [400, 60, 12]
    R = 600
    ests, e2 = [], []
    for r in range(R):
        pairs = Wk.toy_levels(M, L, a, b, seed=1000 + r)
        ests.append(E.ofmlmc_mean(pairs, alpha))
        e2.append(E.eps2(E.sigma_tilde2(pairs, alpha), M))
    ests = np.array(ests)
    mse = np.mean((ests - mean[L]) ** 2)
    # closed-form variance of the estimator with these coefficients
    st2 = [alpha[0] ** 2 * var[0]] + [alpha[l] ** 2 * var[l] + alpha[l - 1] ** 2 * var[l - 1]
                                      - 2 * alpha[l] * alpha[l - 1] * cov[l] for l in range(1, L + 1)]
    v_exact = sum(s / m for s, m in zip(st2, M))
    assert abs(ests.mean() - mean[L]) < 4 * math.sqrt(v_exact / R)
    assert abs(mse / v_exact - 1) < 0.15
    assert abs(np.mean(e2) / v_exact - 1) < 0.05


def test_optimal_M_tol_and_budget():
    st2 = np.array([1.0, 0.2, 0.04, 0.01])
    W = 16.0 ** np.arange(4)
    tau = 0.01
    M = E.optimal_M(st2, W, tau, "tol")
    assert E.eps2(st2, M) <= tau ** 2
    # one fewer sample on every level violates the tolerance only through rounding slack
    raw = (1 / tau ** 2) * np.sqrt(st2 / W) * np.sum(np.sqrt(st2 * W))
    assert abs(np.sum(st2 / raw) - tau ** 2) < 1e-12 * tau ** 2
    B = 1e6
    Mb = E.optimal_M(st2, W, B, "budget")
    assert E.total_work(Mb, W) >= B * (1 - 1e-12)
    assert E.total_work(Mb - 1, W) < B
    # Lagrange optimality: M_l proportional to sqrt(sigma~^2_l / W_l)
    r = raw / np.sqrt(st2 / W)
    assert np.allclose(r, r[0])


def test_keep_samples_reoptimisation():
    st2 = np.array([1.0, 0.2, 0.04, 0.01])
    W = 16.0 ** np.arange(4)
    tau = 0.01
    M_done = np.array([200000, 10, 1, 1])   # level 0 is over-sampled already (optimum 123889)
    M = E.optimal_M_keep(st2, W, M_done, tau, "tol")
    assert np.all(M >= M_done)
    assert M[0] == 200000
    assert E.eps2(st2, M) <= tau ** 2 * (1 + 1e-12)
    plain = E.optimal_M(st2, W, tau, "tol")
    assert np.all(M[1:] <= plain[1:])      # the kept samples relax the other levels


def test_warmup_sequence_printed_in_paper():
    W = 16.0 ** np.arange(4)
    M = E.warmup_M(W)
    assert list(M) == GOLD["warmup_L3_W_16pow"]["M_l0_to_lL"]
    assert E.total_work(M, W) <= 2 * W[-1]


def test_work_model_reproduces_budget_ratio_of_table():
    """Pair costs W_l = (16^l + 16^(l-1)) w: the printed OF-MLMC sample numbers
    cost ~8 finest solves, as the text states."""
    M = GOLD["table"]["OF-MLMC"]["M"]
    W = np.array([1.0] + [16.0 ** l + 16.0 ** (l - 1) for l in range(1, 4)])
    ratio = E.total_work(M, W) / 16.0 ** 3
    assert abs(ratio - GOLD["budget_over_finest_solve"]["value"]) < 0.1


def test_mc_equivalent_squared_ratio():
    M, Wmc = E.mc_equivalent(4.0, 0.1, 3.0)
    assert M == 400 and Wmc == 1200.0


def test_adaptive_loop_reaches_tolerance_on_toy():
    L, a, b = 3, 0.4, 0.6
    mean, _, _ = toy_moments(L, a, b)
    W = np.array([1.0] + [16.0 ** l + 16.0 ** (l - 1) for l in range(1, L + 1)])
    rng_seed = [10]

    def draw(l, m):
        rng_seed[0] += 1
        Ms = [0] * (L + 1)
        Ms[l] = m
        return Wk.toy_levels(Ms, L, a, b, seed=rng_seed[0])[l]

    est = E.adaptive(draw, W, tau=0.02)
    assert math.sqrt(est["eps2"]) <= 0.02
    assert len(est["history"]) <= 4
    assert abs(est["mean"] - mean[L]) < 5 * 0.02
    assert est["history"][0] == list(np.maximum(E.warmup_M(W), 2))


def test_zero_variance_needs_no_samples():
    assert list(E.optimal_M([0.0, 0.0], [1.0, 16.0], 0.1, "tol")) == [0, 0]
    assert list(E.optimal_M([0.0, 0.0], [1.0, 16.0], 1e3, "budget")) == [0, 0]


def test_merged_summaries_equal_the_summary_of_the_union():
    """Pairwise combination of per-process summaries is exact: any split of a
    sample set, merged in any order, gives the two-pass summary of the whole
    (including empty parts and single samples)."""
    rng = np.random.default_rng(7)
    p = rng.normal(3.0e6, 4.0e5, (37, 2))
    p[:, 1] = 0.8 * p[:, 0] + rng.normal(0, 1e5, 37)
    whole = E.level_moments(p)
    for cuts in ([0, 37], [1, 36], [5, 20, 12], [0, 0, 37], [13, 1, 1, 22]):
        parts, at = [], 0
        for c in cuts:
            parts.append(E.level_moments(p[at:at + c]))
            at += c
        for order in (parts, parts[::-1]):
            acc = (0, 0.0, 0.0, 0.0, 0.0, 0.0)
            for q in order:
                acc = E.merge_moments(acc, q)
            assert acc[0] == whole[0]
            assert np.allclose(acc[1:], whole[1:], rtol=1e-12, atol=0.0)
    # two single samples: m2 = (x1 - x2)^2 / 2, the textbook two-point variance
    m = E.merge_moments(E.level_moments(np.array([[1.0, 4.0]])), E.level_moments(np.array([[3.0, 1.0]])))
    assert m == (2, 2.0, 2.5, 2.0, 4.5, -3.0)


def test_estimate_from_summaries_equals_estimate_from_pairs():
    """The summary path is the pair path re-associated: same alpha, indicators,
    mean and error to round-off on a three-level toy."""
    L, a, b = 2, 0.5, 1.0
    pairs = Wk.toy_levels([300, 40, 9], L, a, b, seed=11)
    W = np.array([1.0, 17.0, 272.0])
    ref = E.estimate(pairs, W)
    got = E.estimate_from_moments([E.level_moments(p) for p in pairs], W)
    for k in ("alpha", "sigma2", "cov", "sigma_tilde2"):
        assert np.allclose(got[k], ref[k], rtol=1e-11, atol=1e-14), k
    assert abs(got["mean"] - ref["mean"]) <= 1e-12 * abs(ref["mean"])
    assert abs(got["eps2"] - ref["eps2"]) <= 1e-11 * ref["eps2"]


# ----------------------------------------------------------------- step 3's optional variance fit

def test_fit_recovers_an_exact_exponential():
    V = np.array([np.nan] + [3.0 * 0.25 ** l for l in range(1, 4)])
    a, b, V_fit = E.fit_diff_variances(V, [9, 7, 5, 3])
    assert abs(a - math.log(3.0)) < 1e-13 and abs(b - math.log(0.25)) < 1e-13
    assert np.allclose(V_fit[1:], V[1:], rtol=1e-13, atol=0)


def test_fit_is_the_weighted_least_squares_line():
    """Against numpy's weighted polynomial fit (it minimises sum (w (y - p))^2,
    so w = sqrt of the inverse log-variance 2/(M - 1))."""
    rng = np.random.default_rng(5)
    M = [50, 40, 9, 3]
    V = np.array([np.nan, 0.8, 0.15, 0.05])
    V[1:] *= np.exp(rng.normal(0.0, 0.3, 3))
    a, b, _ = E.fit_diff_variances(V, M)
    x = np.array([1.0, 2.0, 3.0])
    w = np.sqrt((np.array(M[1:]) - 1) / 2.0)
    slope, icpt = np.polyfit(x, np.log(V[1:]), 1, w=w)
    assert abs(b - slope) < 1e-12 and abs(a - icpt) < 1e-12
    # levels with fewer than two pairs carry no empirical variance and are left out
    a2, b2, V2 = E.fit_diff_variances(np.array([np.nan, 0.8, 0.15, np.nan]), [50, 40, 9, 1])
    slope2, icpt2 = np.polyfit([1.0, 2.0], np.log([0.8, 0.15]), 1)
    assert abs(b2 - slope2) < 1e-12 and abs(a2 - icpt2) < 1e-12
    assert abs(V2[3] - math.exp(a2 + 3 * b2)) < 1e-15


def test_fit_is_the_posterior_mean_under_flat_priors():
    """Bayesian inference (Sec. 2.4.3, step 3) with Gaussian errors of ln V_l
    and flat priors: the posterior mean of (a, b), integrated on a grid."""
    M = [0, 12, 6, 4]
    V = np.array([np.nan, 0.5, 0.2, 0.03])
    a, b, _ = E.fit_diff_variances(V, M)
    x = np.array([1.0, 2.0, 3.0])
    y = np.log(V[1:])
    s2 = 2.0 / (np.array(M[1:]) - 1)
    A = np.linspace(a - 8, a + 8, 801)
    B = np.linspace(b - 5, b + 5, 801)
    AA, BB = np.meshgrid(A, B, indexing="ij")
    logp = np.zeros_like(AA)
    for xi, yi, si in zip(x, y, s2):
        logp -= (yi - AA - BB * xi) ** 2 / (2.0 * si)
    p = np.exp(logp - logp.max())
    assert abs((p * AA).sum() / p.sum() - a) < 1e-6
    assert abs((p * BB).sum() / p.sum() - b) < 1e-6


def test_log_sample_variance_error_model():
    """Var[ln V^] ~ 2/(M - 1) for Gaussian level differences (the error bars
    the fit's weights stand for), by Monte Carlo."""
    rng = np.random.default_rng(7)
    M = 101
    x = rng.standard_normal((20000, M)) * 0.3
    lv = np.log(x.var(axis=1, ddof=1))
    assert abs(lv.var() / (2.0 / (M - 1)) - 1.0) < 0.05


def test_fit_needs_two_levels():
    with pytest.raises(ValueError):
        E.fit_diff_variances(np.array([np.nan, 0.5, np.nan]), [4, 4, 1])


def _toy_alpha_and_diffvar(L, a, b, W):
    _, var, cov = toy_moments(L, a, b)
    V = np.array([np.nan] + [4.0 ** (-l) * (a * a + 5.0 * b * b) for l in range(1, L + 1)])
    return E.alpha_optimal(var, cov, W), var, cov, V


def test_fitted_estimator_converges_to_closed_forms():
    """Toy hierarchy: V[q_l - q_{l-1}] = 4^-l (a^2 + 5 b^2) is an exact
    exponential, so the fit and alpha approach the closed forms."""
    L, a, b = 3, 0.4, 0.6
    W = np.array([1.0] + [16.0 ** l + 16.0 ** (l - 1) for l in range(1, L + 1)])
    alpha_true, var, cov, V = _toy_alpha_and_diffvar(L, a, b, W)
    pairs = Wk.toy_levels([40000, 20000, 20000, 20000], L, a, b, seed=3)
    est = E.estimate_fitted(pairs, W)
    assert np.allclose(est["V_fit"][1:], V[1:], rtol=0.03)
    assert abs(est["fit"][1] - math.log(0.25)) < 0.03
    assert np.allclose(est["alpha"], alpha_true, atol=0.02)
    assert np.allclose(est["cov"][1:], cov[1:], rtol=0.03)


def test_fitted_estimator_with_one_finest_pair():
    """M_L = 1 (the appendix's warm-up): V_L is extrapolated from levels
    1..L-1, sigma^2_L = sigma^2_{L-1}, sigma~^2_L from the fitted moments.
    Against the closed forms under that reading; the reading itself moves
    Cov[q_L, q_{L-1}] by (sigma^2_L - sigma^2_{L-1})/2, which on this toy
    (variance falling 10 % from level 2 to 3) shifts alpha by about 0.05."""
    L, a, b = 3, 0.4, 0.6
    W = np.array([1.0] + [16.0 ** l + 16.0 ** (l - 1) for l in range(1, L + 1)])
    alpha_true, var, cov, V = _toy_alpha_and_diffvar(L, a, b, W)
    var_r = var.copy()
    var_r[L] = var[L - 1]
    cov_r = cov.copy()
    cov_r[L] = 0.5 * (var_r[L] + var_r[L - 1] - V[L])
    alpha_r = E.alpha_optimal(var_r, cov_r, W)
    pairs = Wk.toy_levels([40000, 20000, 20000, 1], L, a, b, seed=4)
    est = E.estimate_fitted(pairs, W)
    assert est["M"][L] == 1
    assert est["sigma2"][L] == est["sigma2"][L - 1]
    assert abs(est["V_fit"][L] / V[L] - 1.0) < 0.1
    assert np.allclose(est["alpha"], alpha_r, atol=0.02)
    assert np.max(np.abs(est["alpha"] - alpha_true)) < 0.08
    al = est["alpha"]
    st2_r = al[L] ** 2 * var_r[L] + al[L - 1] ** 2 * var_r[L - 1] - 2 * al[L] * al[L - 1] * cov_r[L]
    assert abs(est["sigma_tilde2"][L] / st2_r - 1.0) < 0.2
    with pytest.raises(ValueError):
        E.estimate_fitted(Wk.toy_levels([100, 100, 1], 2, a, b, seed=4), W[:3])


def test_fitted_moments_stay_positive_semi_definite_with_few_pairs():
    """With two or three pairs a level's fitted V_l can leave the range a
    covariance allows; clamped, |Cov_l| <= sigma_l sigma_{l-1} and every
    sigma~^2 is a variance (>= 0), including the modelled finest one."""
    Wc = [4096.0, 69632.0, 397312.0, 1380352.0]
    clamped = 0
    for seed in range(300):
        pairs = Wk.toy_levels([43, 5, 2, 1], 3, 0.4, 0.7, seed=seed)
        est = E.estimate_fitted(pairs, Wc)
        s2, cov = est["sigma2"], est["cov"]
        for l in range(1, 4):
            assert abs(cov[l]) <= math.sqrt(s2[l] * s2[l - 1]) * (1 + 1e-12)
        assert np.all(est["sigma_tilde2"] >= -1e-12 * np.max(s2))
        free = E.fit_diff_variances(E.diff_variances(pairs), [43, 5, 2, 1])[2]
        clamped += int(not np.allclose(free[1:], est["V_fit"][1:], rtol=1e-14))
    assert clamped > 0        # the clamp was exercised


def test_adaptive_loop_with_fit_starts_the_finest_level_from_one_pair():
    L, a, b = 3, 0.4, 0.6
    mean, _, _ = toy_moments(L, a, b)
    W = np.array([1.0] + [16.0 ** l + 16.0 ** (l - 1) for l in range(1, L + 1)])
    seed = [40]

    def draw(l, m):
        seed[0] += 1
        Ms = [0] * (L + 1)
        Ms[l] = m
        return Wk.toy_levels(Ms, L, a, b, seed=seed[0])[l]

    est = E.adaptive(draw, W, tau=0.02, fit=True)
    assert est["history"][0][L] == 1
    assert est["history"][0][:L] == list(np.maximum(E.warmup_M(W), 2))[:L]
    assert math.sqrt(est["eps2"]) <= 0.02
    assert abs(est["mean"] - mean[L]) < 5 * 0.02


# ---------------------------------------------------------------- surrogate control variate (not in the paper)

def _toy_with_inputs(M, L, a, b, seed, mu=1.0, c=0.5):
    """The toy hierarchy of workloads.toy_levels, also returning each pair's
    shared input Z (the "cloud") so that a surrogate can be evaluated."""
    rng = np.random.default_rng(seed)
    pairs, Zs = [], []
    for l in range(L + 1):
        m = M[l]
        Z = rng.standard_normal(m)
        Yf, Yc = rng.standard_normal(m), rng.standard_normal(m)
        qf = mu + c * 2.0 ** (-l) + Z + 2.0 ** (-l) * (a * Z + b * Yf)
        qc = (mu + c * 2.0 ** (-(l - 1)) + Z + 2.0 ** (-(l - 1)) * (a * Z + b * Yc)) if l > 0 else np.zeros(m)
        pairs.append(np.stack([qf, qc], axis=1))
        Zs.append(Z)
    return pairs, Zs


def _h(Z, q_coarse):
    """A fixed, nonlinear, imperfect surrogate of q_L from (input, q_{L-1})."""
    return 0.8 * q_coarse + 0.3 * np.tanh(Z) + 0.05 * Z ** 2


def test_surrogate_estimator_with_zero_beta_is_plain_ofmlmc():
    pairs, Zs = _toy_with_inputs([200, 60, 20], 2, 0.5, 0.6, seed=1)
    W = [1.0, 5.0, 25.0]
    ref = E.estimate(pairs, W)
    got = E.estimate_surrogate(pairs, W, _h(Zs[2], pairs[2][:, 1]), _h(Zs[1], pairs[1][:, 0]), beta=0.0)
    assert got["mean"] == pytest.approx(ref["mean"], rel=1e-14, abs=1e-14)
    assert np.allclose(got["sigma_tilde2"], ref["sigma_tilde2"], rtol=1e-13)
    assert got["eps2"] == pytest.approx(ref["eps2"], rel=1e-13)
    # a surrogate that only repeats alpha_{L-1} q_{L-1} leaves nothing to correct: beta = 0
    flat = E.estimate_surrogate(pairs, W, ref["alpha"][1] * pairs[2][:, 1], ref["alpha"][1] * pairs[1][:, 0])
    assert flat["beta"] == 0.0 and flat["mean"] == pytest.approx(ref["mean"], rel=1e-14)


def test_surrogate_beta_minimises_the_error_estimate():
    pairs, Zs = _toy_with_inputs([300, 80, 25], 2, 0.5, 0.6, seed=2)
    W = [1.0, 5.0, 25.0]
    ht, he = _h(Zs[2], pairs[2][:, 1]), _h(Zs[1], pairs[1][:, 0])
    best = E.estimate_surrogate(pairs, W, ht, he)
    grid = np.linspace(best["beta"] - 1.0, best["beta"] + 1.0, 2001)
    e2 = [E.estimate_surrogate(pairs, W, ht, he, beta=b)["eps2"] for b in grid]
    assert best["eps2"] <= min(e2) * (1 + 1e-12)
    assert abs(grid[int(np.argmin(e2))] - best["beta"]) <= 1e-3
    assert best["eps2"] < best["eps2_plain"]


def test_surrogate_estimator_unbiased_and_error_formula_for_fixed_coefficients():
    """Over independent repeats with fixed alpha and beta: the mean of the
    estimates is E[q_L] = mu + c 2^-L (any surrogate, even a biased one), and
    their variance is the mean of eps^2 = sum_l sigma~^2_l / M_l."""
    L, M, W = 2, [120, 40, 12], [1.0, 5.0, 25.0]
    alpha, beta = np.array([0.9, 0.95, 1.0]), 0.7
    R = 4000
    est, e2 = [], []
    for r in range(R):
        pairs, Zs = _toy_with_inputs(M, L, 0.5, 0.6, seed=1000 + r)
        ht = _h(Zs[2], pairs[2][:, 1]) + 3.0            # biased on purpose
        he = _h(Zs[1], pairs[1][:, 0]) + 3.0
        out = E.estimate_surrogate(pairs, W, ht, he, alpha=alpha, beta=beta)
        est.append(out["mean"])
        e2.append(out["eps2"])
    est = np.array(est)
    truth = 1.0 + 0.5 * 2.0 ** (-L)
    assert abs(est.mean() - truth) < 4.0 * est.std() / math.sqrt(R)
    assert est.var(ddof=1) == pytest.approx(np.mean(e2), rel=0.08)


def test_a_good_surrogate_lowers_the_top_level_variance():
    """In the toy q_L = mu + c 2^-L + Z + 2^-L (a Z + b Y_f); the coarse member's
    own Y is independent, so the best prediction of q_L from the input Z is
    E[q_L | Z] = mu + c 2^-L + (1 + a 2^-L) Z.  As the surrogate it leaves the
    top level term only q_L - E[q_L | Z] = 2^-L b Y_f: variance (2^-L b)^2
    against ~0.13 for the plain term (a = 0.5, b = 0.6, L = 2, alpha ~ 1)."""
    a, b, L = 0.5, 0.6, 2
    pairs, Zs = _toy_with_inputs([4000, 800, 400], L, a, b, seed=5)
    W = [1.0, 5.0, 25.0]
    good = lambda Z: 1.0 + 0.5 * 2.0 ** (-L) + (1.0 + a * 2.0 ** (-L)) * Z
    out = E.estimate_surrogate(pairs, W, good(Zs[2]), good(Zs[1]))
    assert 0.8 < out["beta"] < 1.2
    assert out["sigma_tilde2"][2] < 0.3 * out["sigma_tilde2_plain"][2]
    assert out["sigma_tilde2"][2] == pytest.approx((2.0 ** (-L) * b) ** 2, rel=0.25)
    assert out["eps2"] < out["eps2_plain"]
