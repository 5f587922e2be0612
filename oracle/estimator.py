"""Oracle for the MLMC / OF-MLMC estimator (test infrastructure).

Plain numpy in FP64, following Section 2.4 of the paper:
  - classical MLMC telescoping estimator, Eq. (mlmc), and its MSE, Eq. (mlmc-err);
  - OF-MLMC control-variate coefficients from the tridiagonal system,
    Eq. (alpha-matvec), which minimises the cost-weighted variance of
    Eq. (cv-mlmc-var);
  - the OF-MLMC estimator, Eq. (ocv-mlmc), and its MSE, Eq. (ocv-mlmc-err);
  - optimal sample numbers for a tolerance, Eq. (M-tol), or a budget,
    Eq. (M-budget), with the keep-computed-samples re-optimisation of step 7;
  - warm-up sample numbers, Eq. (warmup);
  - the MC-equivalent cost, Eq. (speedup);
  - the same estimator from per-level summaries (counts, means, squared
    deviations, fine/coarse co-deviation) that combine across processes;
  - (not in the paper) a learned surrogate as an extra control variate of the
    top level term with its own coefficient (estimate_surrogate).

Input convention: ``pairs[l]`` is an (M_l, 2) array; column 0 holds q_l and
column 1 holds q_{l-1} evaluated on the same random input (column 1 unused
for l = 0).  W[l] is the cost of one sample at l = 0 and of one pair
(levels l and l-1) for l > 0.

Readings of points the paper leaves open:
  - sigma^2_l is the unbiased sample variance pooled over every computed
    q_l (fine members of pair l and coarse members of pair l+1);
    sigma^2_{l,l-1} is the unbiased sample covariance of pair l;
  - sigma~^2_l is the unbiased sample variance of alpha_l q_l - alpha_{l-1} q_{l-1}
    over pair l (of alpha_0 q_0 for l = 0);
  - the tolerance constraint is eps_OF <= tau, i.e. sum sigma~^2_l/M_l <= tau^2;
  - the MC-equivalent sample number is ceil((sigma_L/eps)^2) (the printed
    formula omits the square);
  - the optional fit of step 3 (Sec. 2.4.3, Sec. 3.2 and the appendix on
    M_L = 1) is applied to the variances of the level differences
    V_l = V[q_l - q_{l-1}] (the quantity the results section fits), not to
    the covariances: ln V_l = a + b l by least squares over the levels l >= 1
    with at least two pairs, each weighted by the inverse of the Gaussian
    error of ln V_l, Var[ln V_l] ~ 2/(M_l - 1) (the posterior mean under
    flat priors); the fitted V_l, clamped to [(sigma_l - sigma_{l-1})^2,
    (sigma_l + sigma_{l-1})^2] (the range in which the second moments of
    (q_l, q_{l-1}) stay positive semi-definite), give the covariances of
    Eq. (alpha-matvec) as (sigma^2_l + sigma^2_{l-1} - V_l)/2; a level with one pair takes
    sigma^2_l = sigma^2_{l-1} (no sample variance exists) and its sigma~^2_l
    from the fitted second moments.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np


def _var(x: np.ndarray) -> float:
    x = np.asarray(x, dtype=np.float64)
    m = x.size
    if m < 2:
        return float("nan")
    mu = x.sum() / m
    return float(((x - mu) ** 2).sum() / (m - 1))


def _cov(x: np.ndarray, y: np.ndarray) -> float:
    m = x.size
    if m < 2:
        return float("nan")
    return float(((x - x.sum() / m) * (y - y.sum() / m)).sum() / (m - 1))


def indicators(pairs: Sequence[np.ndarray]):
    """(sigma2[0..L], cov[0..L]) with cov[0] = 0 (Step 3)."""
    L = len(pairs) - 1
    sigma2 = np.zeros(L + 1)
    cov = np.zeros(L + 1)
    for l in range(L + 1):
        members = [pairs[l][:, 0]]
        if l < L:
            members.append(pairs[l + 1][:, 1])
        sigma2[l] = _var(np.concatenate(members))
        if l > 0:
            cov[l] = _cov(pairs[l][:, 0], pairs[l][:, 1])
    return sigma2, cov


def alpha_matrix(sigma2: np.ndarray, cov: np.ndarray, W: np.ndarray):
    """Matrix and right-hand side of Eq. (alpha-matvec) for alpha_0..alpha_{L-1}."""
    L = len(sigma2) - 1
    A = np.zeros((L, L))
    rhs = np.zeros(L)
    for l in range(L):
        A[l, l] = sigma2[l] * (W[l + 1] + W[l])
        if l > 0:
            A[l, l - 1] = -cov[l] * W[l]
        if l + 1 < L:
            A[l, l + 1] = -cov[l + 1] * W[l + 1]
    rhs[L - 1] = cov[L] * W[L]
    return A, rhs


def alpha_optimal(sigma2, cov, W) -> np.ndarray:
    """alpha[0..L] with alpha_L = 1 (Step 4)."""
    L = len(sigma2) - 1
    alpha = np.ones(L + 1)
    if L > 0:
        A, rhs = alpha_matrix(np.asarray(sigma2), np.asarray(cov), np.asarray(W, dtype=np.float64))
        alpha[:L] = np.linalg.solve(A, rhs)
    return alpha


def cost_functional(alpha, sigma2, cov, W) -> float:
    """C[q_L^*] of Eq. (cv-mlmc-var) for given coefficients (alpha_L = 1)."""
    L = len(sigma2) - 1
    C = alpha[0] ** 2 * sigma2[0] * W[0]
    for l in range(1, L + 1):
        C += (alpha[l] ** 2 * sigma2[l] + alpha[l - 1] ** 2 * sigma2[l - 1]
              - 2.0 * alpha[l] * alpha[l - 1] * cov[l]) * W[l]
    return float(C)


def sigma_tilde2(pairs, alpha) -> np.ndarray:
    """Variances of the alpha-weighted level differences (Step 5)."""
    L = len(pairs) - 1
    out = np.zeros(L + 1)
    out[0] = _var(alpha[0] * pairs[0][:, 0])
    for l in range(1, L + 1):
        out[l] = _var(alpha[l] * pairs[l][:, 0] - alpha[l - 1] * pairs[l][:, 1])
    return out


def ofmlmc_mean(pairs, alpha) -> float:
    """Eq. (ocv-mlmc)."""
    L = len(pairs) - 1
    e = alpha[0] * pairs[0][:, 0].sum() / pairs[0].shape[0]
    for l in range(1, L + 1):
        d = alpha[l] * pairs[l][:, 0] - alpha[l - 1] * pairs[l][:, 1]
        e += d.sum() / pairs[l].shape[0]
    return float(e)


def mlmc_mean(pairs) -> float:
    """Eq. (mlmc): the alpha = 1 special case."""
    return ofmlmc_mean(pairs, np.ones(len(pairs)))


def eps2(sig_t2, M) -> float:
    """Eq. (ocv-mlmc-err): sum sigma~^2_l / M_l."""
    return float(sum(s / m for s, m in zip(sig_t2, M)))


def estimate(pairs, W):
    """Steps 3-5 and the estimator of step 6: a dict of everything the paper names."""
    sigma2, cov = indicators(pairs)
    alpha = alpha_optimal(sigma2, cov, W)
    st2 = sigma_tilde2(pairs, alpha)
    M = [p.shape[0] for p in pairs]
    return dict(alpha=alpha, sigma2=sigma2, cov=cov, sigma_tilde2=st2,
                mean=ofmlmc_mean(pairs, alpha), eps2=eps2(st2, M), M=M)


# ---------------------------------------------------------------------------
# Step 3's optional fit: an exponential decay of the level-difference
# variances, so that the finest level can start from one warm-up pair.

def diff_variances(pairs) -> np.ndarray:
    """V[q_l - q_{l-1}] of pair l (nan for l = 0 and for fewer than two pairs)."""
    out = np.full(len(pairs), np.nan)
    for l in range(1, len(pairs)):
        out[l] = _var(pairs[l][:, 0] - pairs[l][:, 1])
    return out


def fit_diff_variances(V, M):
    """Weighted least-squares line through ln V_l over l >= 1 with M_l >= 2 and
    V_l > 0, weights (M_l - 1)/2.  Returns (a, b, V_fit) with
    V_fit[l] = exp(a + b l) for l >= 1 (V_fit[0] = nan)."""
    L = len(V) - 1
    used = [l for l in range(1, L + 1) if M[l] >= 2 and V[l] > 0.0]
    if len(used) < 2:
        raise ValueError("the fit needs two levels l >= 1 with at least two pairs")
    w = np.array([(M[l] - 1) / 2.0 for l in used])
    x = np.array(used, dtype=np.float64)
    y = np.array([math.log(V[l]) for l in used])
    # normal equations of min sum w (y - a - b x)^2
    Sw, Sx, Sy = w.sum(), (w * x).sum(), (w * y).sum()
    Sxx, Sxy = (w * x * x).sum(), (w * x * y).sum()
    det = Sw * Sxx - Sx * Sx
    b = (Sw * Sxy - Sx * Sy) / det
    a = (Sy - b * Sx) / Sw
    V_fit = np.full(L + 1, np.nan)
    for l in range(1, L + 1):
        V_fit[l] = math.exp(a + b * l)
    return a, b, V_fit


def estimate_fitted(pairs, W):
    """estimate() with the fitted level-difference variances in Eq. (alpha-matvec).
    Level 0 needs two samples; a level l >= 1 may have one pair."""
    L = len(pairs) - 1
    M = [p.shape[0] for p in pairs]
    if M[0] < 2 or min(M) < 1:
        raise ValueError("level 0 needs two samples and every level one pair")
    sigma2 = np.zeros(L + 1)
    for l in range(L + 1):
        members = [pairs[l][:, 0]]
        if l < L:
            members.append(pairs[l + 1][:, 1])
        pooled = np.concatenate(members)
        sigma2[l] = _var(pooled) if pooled.size >= 2 else sigma2[l - 1]
    a, b, V_fit = fit_diff_variances(diff_variances(pairs), M)
    cov = np.zeros(L + 1)
    for l in range(1, L + 1):
        # Cauchy-Schwarz: |Cov| <= sigma_l sigma_{l-1}
        lo = (math.sqrt(sigma2[l]) - math.sqrt(sigma2[l - 1])) ** 2
        hi = (math.sqrt(sigma2[l]) + math.sqrt(sigma2[l - 1])) ** 2
        V_fit[l] = min(max(V_fit[l], lo), hi)
        cov[l] = 0.5 * (sigma2[l] + sigma2[l - 1] - V_fit[l])
    alpha = alpha_optimal(sigma2, cov, W)
    st2 = np.zeros(L + 1)
    for l in range(L + 1):
        if M[l] >= 2:
            d = alpha[l] * pairs[l][:, 0] - (alpha[l - 1] * pairs[l][:, 1] if l > 0 else 0.0)
            st2[l] = _var(d)
        else:
            st2[l] = (alpha[l] ** 2 * sigma2[l] + alpha[l - 1] ** 2 * sigma2[l - 1]
                      - 2.0 * alpha[l] * alpha[l - 1] * cov[l])
    return dict(alpha=alpha, sigma2=sigma2, cov=cov, sigma_tilde2=st2, mean=ofmlmc_mean(pairs, alpha),
                eps2=eps2(st2, M), M=M, fit=(a, b), V_fit=V_fit)


# ---------------------------------------------------------------------------
# The same estimator from per-level summaries, for samples spread over several
# processes (Sec. 2.4: the estimator needs only per-level means, variances and
# the fine/coarse covariance).  A summary is (n, mean_f, mean_c, m2_f, m2_c,
# c_fc): pair count, means of the fine and coarse members, their sums of
# squared deviations and the sum of products of deviations.  Two summaries of
# disjoint sample sets combine exactly (pairwise update of Chan, Golub and
# LeVeque, 1979).

def level_moments(p: np.ndarray) -> tuple:
    """Summary of one level's (M, 2) pairs, two passes."""
    p = np.asarray(p, dtype=np.float64)
    n = p.shape[0]
    if n == 0:
        return (0, 0.0, 0.0, 0.0, 0.0, 0.0)
    mf, mc = float(np.mean(p[:, 0])), float(np.mean(p[:, 1]))
    df, dc = p[:, 0] - mf, p[:, 1] - mc
    return (n, mf, mc, float(np.sum(df * df)), float(np.sum(dc * dc)), float(np.sum(df * dc)))


def merge_moments(a: tuple, b: tuple) -> tuple:
    """Summary of the union of two disjoint sample sets."""
    na, nb = a[0], b[0]
    if na == 0:
        return tuple(b)
    if nb == 0:
        return tuple(a)
    n = na + nb
    dfm, dcm = b[1] - a[1], b[2] - a[2]
    w = na * nb / n
    return (n, a[1] + dfm * nb / n, a[2] + dcm * nb / n,
            a[3] + b[3] + dfm * dfm * w, a[4] + b[4] + dcm * dcm * w, a[5] + b[5] + dfm * dcm * w)


def estimate_from_moments(moms, W):
    """estimate() from per-level summaries: the pooled variances of step 3
    (fine members of pair l with coarse members of pair l+1), the covariances,
    alpha, sigma~^2 = V[alpha_l q_l - alpha_{l-1} q_{l-1}], the mean and eps^2."""
    L = len(moms) - 1
    sigma2 = np.zeros(L + 1)
    cov = np.zeros(L + 1)
    for l in range(L + 1):
        n, mf, _, m2f = moms[l][0], moms[l][1], moms[l][2], moms[l][3]
        pooled = (n, mf, 0.0, m2f, 0.0, 0.0)
        if l < L:
            nx = moms[l + 1]
            pooled = merge_moments(pooled, (nx[0], nx[2], 0.0, nx[4], 0.0, 0.0))
        sigma2[l] = pooled[3] / (pooled[0] - 1)
        cov[l] = moms[l][5] / (n - 1) if l > 0 else 0.0
    alpha = alpha_optimal(sigma2, cov, W)
    st2 = np.zeros(L + 1)
    mean = 0.0
    for l in range(L + 1):
        n, mf, mc, m2f, m2c, cfc = moms[l]
        if l == 0:
            st2[0] = alpha[0] ** 2 * m2f / (n - 1)
            mean += alpha[0] * mf
        else:
            st2[l] = (alpha[l] ** 2 * m2f + alpha[l - 1] ** 2 * m2c - 2.0 * alpha[l] * alpha[l - 1] * cfc) / (n - 1)
            mean += alpha[l] * mf - alpha[l - 1] * mc
    M = [m[0] for m in moms]
    return dict(alpha=alpha, sigma2=sigma2, cov=cov, sigma_tilde2=st2, mean=mean, eps2=eps2(st2, M), M=M)


def optimal_M(sig_t2, W, target: float, mode: str) -> np.ndarray:
    """Eq. (M-tol) (mode 'tol', target = tau) or Eq. (M-budget) (mode 'budget', target = B).

    Both formulas divide by sum_k sqrt(sigma~^2_k W_k); when every sigma~^2 is
    zero (a QoI without sampling variance) no sample is needed: zeros.
    """
    s = np.asarray(sig_t2, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    total = float(np.sum(np.sqrt(s * W)))
    if total == 0.0:
        return np.zeros(len(s), dtype=np.int64)
    if mode == "tol":
        raw = (1.0 / target ** 2) * np.sqrt(s / W) * total
    elif mode == "budget":
        raw = target * np.sqrt(s / W) / total
    else:
        raise ValueError(mode)
    return np.array([math.ceil(x) for x in raw], dtype=np.int64)


def optimal_M_keep(sig_t2, W, M_done, target: float, mode: str) -> np.ndarray:
    """Step 7 with the keep-samples remark.

    Levels whose optimum falls below the samples already computed keep them;
    their share (sigma~^2_l/M_l of tau^2, or M_l W_l of the budget) is taken
    off the target and the remaining levels are re-optimised, until no
    optimum falls below what is computed.
    """
    s = np.asarray(sig_t2, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    M_done = np.asarray(M_done, dtype=np.int64)
    n = len(s)
    fixed = np.zeros(n, dtype=bool)
    while True:
        free = ~fixed
        if mode == "tol":
            rem = target ** 2 - float(np.sum(s[fixed] / M_done[fixed]))
            if rem <= 0.0:
                raise ValueError("tolerance already consumed by the kept levels")
            Mf = optimal_M(s[free], W[free], math.sqrt(rem), "tol")
        else:
            rem = target - float(np.sum(M_done[fixed] * W[fixed]))
            if rem <= 0.0:
                raise ValueError("budget already consumed by the kept levels")
            Mf = optimal_M(s[free], W[free], rem, "budget")
        M = M_done.copy()
        M[free] = Mf
        newly = free & (M < M_done)
        if not newly.any():
            M[fixed] = M_done[fixed]
            return M
        fixed |= newly


def warmup_M(W) -> np.ndarray:
    """Eq. (warmup): M_l = ceil(W_L/W_l / 2^(L-l))."""
    W = np.asarray(W, dtype=np.float64)
    L = len(W) - 1
    return np.array([math.ceil(W[L] / W[l] / 2.0 ** (L - l)) for l in range(L + 1)],
                    dtype=np.int64)


def mc_equivalent(sigma2_L: float, eps: float, W_finest_sample: float):
    """Eq. (speedup) with the squared ratio: (M_MC, W_MC)."""
    M = math.ceil(sigma2_L / eps ** 2)
    return M, M * W_finest_sample


def total_work(M, W) -> float:
    return float(np.sum(np.asarray(M, dtype=np.float64) * np.asarray(W, dtype=np.float64)))


def adaptive(draw, W, tau: float, max_iter: int = 10, mode: str = "tol",
             budget: Optional[float] = None, min_samples: int = 2, fit: bool = False):
    """Steps 1-8 of the adaptive OF-MLMC algorithm.

    ``draw(l, m)`` returns m new pairs for level l (an (m, 2) array).  Returns
    the final estimate dict plus the per-iteration sample numbers.  Reading:
    without the optional Bayesian fit of step 3, a sample variance needs two
    samples, so every level starts with at least ``min_samples``.  With the
    fit (``fit=True``) and L >= 3 the finest level keeps Eq. (warmup)'s single
    pair (the appendix on M_L = 1): levels 1..L-1 carry the fit.
    """
    L = len(W) - 1
    M_target = np.maximum(warmup_M(W), min_samples)                # step 1
    if fit and L >= 3:
        M_target[L] = warmup_M(W)[L]
    pairs: List[np.ndarray] = [np.zeros((0, 2)) for _ in range(L + 1)]
    history = []
    est = None
    for it in range(max_iter):
        for l in range(L + 1):                                       # step 2
            need = int(M_target[l]) - pairs[l].shape[0]
            if need > 0:
                pairs[l] = np.concatenate([pairs[l], draw(l, need)])
        history.append([p.shape[0] for p in pairs])
        est = estimate_fitted(pairs, W) if fit else estimate(pairs, W)  # steps 3-5
        spent = total_work([p.shape[0] for p in pairs], W)
        if math.sqrt(est["eps2"]) <= tau or (mode == "budget" and spent >= budget):
            break                                                    # step 6
        M_done = np.array([p.shape[0] for p in pairs])
        target = tau if mode == "tol" else budget
        M_target = optimal_M_keep(est["sigma_tilde2"], W, M_done, target, mode)  # step 7
    est = dict(est)
    est["history"] = history
    return est


def surrogate_cv(D_top: np.ndarray, s_paired: np.ndarray, s_extra: np.ndarray):
    """Extra control variate for the top-level term of the estimator.

    D_top[i] = q_L^i - alpha_{L-1} q_{L-1}^i on the M finest-pair inputs,
    s_paired[i] the surrogate on the same inputs, s_extra the surrogate on N
    independent extra inputs.  The corrected estimate of E[D_top] is
        mean(D) + beta (mean(s_extra) - mean(s_paired)),
    unbiased for any fixed beta; the variance-minimising coefficient is
        beta = Cov(D, s) / (V[s] (1 + M/N)),
    giving variance (V[D] - Cov(D, s)^2 / (V[s] (1 + M/N))) / M.
    (Not in the paper: a standard control variate with an estimated mean.)
    """
    M = D_top.size
    N = s_extra.size
    vs = _var(s_paired)
    c = _cov(D_top, s_paired)
    beta = c / (vs * (1.0 + M / N)) if vs > 0 else 0.0
    corr = beta * (s_extra.sum() / N - s_paired.sum() / M)
    var = (_var(D_top) - c * c / (vs * (1.0 + M / N))) / M if vs > 0 else _var(D_top) / M
    return dict(beta=beta, correction=float(corr), var=float(var),
                mean=float(D_top.sum() / M + corr))


def estimate_surrogate(pairs, W, h_top, h_extra, alpha=None, beta=None):
    """OF-MLMC with a surrogate of q_L as an extra control variate (not in the paper).

    h_top[i]: the surrogate's prediction of q_L on the input of level-L pair
    i (its cloud and its coarse member q_{L-1}), from a network that was not
    trained on pair i; h_extra[j]: the surrogate on the input of the fine
    member of level-(L-1) pair j (its cloud and that q_{L-1}), with the
    networks weighted so that h_extra and h_top have the same expectation
    (both inputs are a random cloud and its q_{L-1}).  The control variate is
    the surrogate's prediction of the top level term,
        g = h - alpha_{L-1} q_{L-1},
    and with the coefficients alpha of Eq. (alpha-matvec) (unless given) the
    two top level terms become

        level L-1:  alpha_{L-1} q_{L-1} - alpha_{L-2} q_{L-2} + beta g  (over the level-(L-1) pairs)
        level L:    q_L - alpha_{L-1} q_{L-1} - beta g                  (over the level-L pairs)

    Their expectations move by +beta E[g] and -beta E[g], so the estimator of
    Eq. (ocv-mlmc) stays unbiased for any fixed alpha and beta; each level is
    still a mean over its own independent pairs, so Eq. (ocv-mlmc-err) and
    the sample numbers of step 7 apply to the modified sigma~^2_l.  Unless
    given, beta minimises eps^2 = sum_l sigma~^2_l / M_l at the current M_l:

        beta = (Cov_L(D_L, g)/M_L - Cov_{L-1}(D_{L-1}, g)/M_{L-1})
               / (V_{L-1}[g]/M_{L-1} + V_L[g]/M_L)

    (D_l the plain level terms; beta = 0 when g does not vary).  Needs L >= 1.
    """
    L = len(pairs) - 1
    if L < 1:
        raise ValueError("the surrogate control variate needs L >= 1")
    base = estimate(pairs, W)
    alpha = base["alpha"] if alpha is None else np.asarray(alpha, dtype=np.float64)
    h_top = np.asarray(h_top, dtype=np.float64)
    h_extra = np.asarray(h_extra, dtype=np.float64)
    M = [p.shape[0] for p in pairs]
    if h_top.size != M[L] or h_extra.size != M[L - 1]:
        raise ValueError("h_top needs one value per level-L pair, h_extra one per level-(L-1) pair")
    D = [alpha[0] * pairs[0][:, 0]]
    for l in range(1, L + 1):
        D.append(alpha[l] * pairs[l][:, 0] - alpha[l - 1] * pairs[l][:, 1])
    g_top = h_top - alpha[L - 1] * pairs[L][:, 1]
    g_extra = h_extra - alpha[L - 1] * pairs[L - 1][:, 0]
    if beta is None:
        den = _var(g_extra) / M[L - 1] + _var(g_top) / M[L]
        num = _cov(D[L], g_top) / M[L] - _cov(D[L - 1], g_extra) / M[L - 1]
        beta = num / den if den > 0.0 else 0.0
    Dm = list(D)
    Dm[L - 1] = D[L - 1] + beta * g_extra
    Dm[L] = D[L] - beta * g_top
    st2 = np.array([_var(d) for d in Dm])
    mean = float(sum(d.sum() / d.size for d in Dm))
    st2_plain = sigma_tilde2(pairs, alpha)
    return dict(alpha=alpha, beta=float(beta), sigma2=base["sigma2"], cov=base["cov"], sigma_tilde2=st2,
                sigma_tilde2_plain=st2_plain, mean=mean, eps2=eps2(st2, M), eps2_plain=eps2(st2_plain, M), M=M)
