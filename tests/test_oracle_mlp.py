"""Pins of the MLP oracle (finite differences, textbook Adam) and of the
surrogate control variate (unbiasedness with a bad surrogate, variance)."""
import math

import numpy as np

from oracle import estimator as E
from oracle import mlp


def _params(rng, sizes):
    return [(rng.normal(size=(a, b)) * math.sqrt(2.0 / a), rng.normal(size=b) * 0.1)
            for a, b in zip(sizes[:-1], sizes[1:])]


def test_gelu_matches_its_definition_and_derivative():
    x = np.linspace(-6, 6, 101)
    ref = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in x])
    assert np.allclose(mlp.gelu(x), ref, rtol=1e-15, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = _params(rng, [7, 5, 6, 4, 2])
    X = rng.normal(size=(9, 7))
    T = rng.normal(size=(9, 2))
    y, cache = mlp.forward(P, X)
    G = mlp.backward(P, cache, y, T)
    h = 1e-6
    for li, (W, b) in enumerate(P):
        for arr, g in ((W, G[li][0]), (b, G[li][1])):
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(5)]:
                old = arr[idx]
                arr[idx] = old + h
                fp = mlp.mse_loss(mlp.forward(P, X)[0], T)
                arr[idx] = old - h
                fm = mlp.mse_loss(mlp.forward(P, X)[0], T)
                arr[idx] = old
                assert abs((fp - fm) / (2 * h) - g[idx]) < 1e-7 * max(1.0, abs(g[idx]))


def test_adam_first_step_is_sign_times_lr():
    """With bias correction the first Adam step is lr * g/(|g| + eps')."""
    P = [(np.array([[1.0, -2.0]]), np.array([0.5, 0.0]))]
    G = [(np.array([[0.3, -4.0]]), np.array([1e-3, 0.0]))]
    opt = mlp.Adam(P, lr=0.01)
    new = opt.step(P, G)
    assert np.allclose(new[0][0], [[1.0 - 0.01, -2.0 + 0.01]], atol=1e-9)
    assert abs(new[0][1][0] - (0.5 - 0.01 * 1e-3 / (1e-3 + 1e-8))) < 1e-12
    assert new[0][1][1] == 0.0


def test_training_reduces_loss_on_a_smooth_target():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(256, 4))
    T = (np.sin(X[:, :1]) + 0.5 * X[:, 1:2] * X[:, 2:3])
    P = _params(rng, [4, 32, 32, 32, 1])
    P, losses = mlp.train(P, X, T, epochs=30, batch=64, lr=3e-3)
    assert losses[-1] < 0.2 * losses[0]


def test_surrogate_cv_unbiased_even_when_bad():
    rng = np.random.default_rng(2)
    M, N, R = 40, 400, 3000
    means, vars_ = [], []
    for r in range(R):
        Z = rng.normal(size=M + N)
        D = 3.0 + Z[:M] + 0.3 * rng.normal(size=M)
        bad = 5.0 * np.cos(Z) + 10.0          # biased, poorly correlated surrogate
        out = E.surrogate_cv(D, bad[:M], bad[M:])
        means.append(out["mean"])
    assert abs(np.mean(means) - 3.0) < 4 * np.std(means) / math.sqrt(R)


def test_surrogate_cv_variance_formula():
    """s = 0.9 Z, D = Z + 0.5 eps: V[D] = 1.25, V[s] = 0.81, Cov(D, s) = 0.9."""
    rng = np.random.default_rng(3)
    M, N, R = 50, 500, 4000
    beta = 0.9 / (0.81 * (1 + M / N))
    est, formula = [], []
    for r in range(R):
        Z = rng.normal(size=M + N)
        D = Z[:M] + 0.5 * rng.normal(size=M)
        s = 0.9 * Z
        est.append(D.mean() + beta * (s[M:].mean() - s[:M].mean()))
        formula.append(E.surrogate_cv(D, s[:M], s[M:])["var"])
    v_formula = (1.25 - 0.9 ** 2 / (0.81 * (1 + M / N))) / M
    assert abs(np.var(est) / v_formula - 1) < 0.1
    assert abs(np.mean(formula) / v_formula - 1) < 0.1


def test_cloud_features_order_and_nearest_subset():
    """Hand-made cloud in a 0.1 m box: the bubble containing the centre has a
    negative surface gap and comes first, then the others by |x_b - c| - r_b;
    n_keep keeps that many nearest bubbles."""
    from oracle import mlp as M
    b = np.array([[0.05, 0.05, 0.06, 0.001],    # gap 0.010 - 0.001 = 0.009
                  [0.02, 0.05, 0.05, 0.002],    # gap 0.030 - 0.002 = 0.028
                  [0.05, 0.05, 0.05, 0.0005],   # gap -0.0005 (contains the centre)
                  [0.05, 0.07, 0.05, 0.012]])   # gap 0.020 - 0.012 = 0.008
    f = M.cloud_features(b, 0.1, 0.02).reshape(-1, 4)
    assert np.allclose(f[:, 3] * 0.02, [0.0005, 0.012, 0.001, 0.002])
    assert np.allclose(f[1, :3] * 0.02, [0.0, 0.02, 0.0])
    assert np.array_equal(M.cloud_features(b, 0.1, 0.02, 2), f[:2].ravel())
    assert np.array_equal(M.cloud_features(b, 0.1, 0.02, 9), f.ravel())
