"""Pins of the MLP oracle (finite differences, textbook Adam) and of the
surrogate control variate (unbiasedness with a bad surrogate, variance)."""
import math

import numpy as np
import pytest

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


def test_forward_of_a_network_with_identity_or_off_hidden_units():
    """Every hidden pre-activation here is >= 47 or <= -59, where exact-erf
    GELU is the identity or zero in FP64 (erf(x/sqrt 2) rounds to +-1), and
    the output layer is linear, so the output is integer arithmetic done by
    hand:
      layer 1, rows (1, 2) and (-1, 3): z = (67, -61, 70), (68, -59, 65) -> h = (67, 0, 70), (68, 0, 65)
      layer 2: z = (47, -160), (53, -170) -> h = (47, 0), (53, 0)
      output:  2*47 - 100 = -6,  2*53 - 100 = 6.
    A dropped bias, GELU on the output layer (GELU(-6) ~ -6e-9), a missing
    GELU on a hidden layer or a transposed operand changes the result.  All
    numbers are exact in BF16, so the BF16-operand forward gives the same."""
    P = [(np.array([[1.0, -1.0, 2.0], [3.0, 0.0, -1.0]]), np.array([60.0, -60.0, 70.0])),
         (np.array([[1.0, 0.0], [5.0, 1.0], [-1.0, 2.0]]), np.array([50.0, -300.0])),
         (np.array([[2.0], [7.0]]), np.array([-100.0]))]
    X = np.array([[1.0, 2.0], [-1.0, 3.0]])
    for lowp in (False, True):
        y, (acts, pres) = mlp.forward(P, X, lowp=lowp)
        assert np.array_equal(y, [[-6.0], [6.0]])
        assert np.array_equal(acts[1], [[67.0, 0.0, 70.0], [68.0, 0.0, 65.0]])
        assert np.array_equal(pres[1], [[47.0, -160.0], [53.0, -170.0]])


def test_forward_gelu_at_one_is_the_normal_cdf():
    """A hidden unit with pre-activation +-1: GELU(x) = x Phi(x), with the
    tabulated standard normal CDF Phi(1) = 0.8413447460685429."""
    P = [(np.array([[1.0, -1.0]]), np.zeros(2)), (np.array([[1.0], [1.0]]), np.array([0.25]))]
    y, _ = mlp.forward(P, np.array([[1.0]]))
    phi1 = 0.8413447460685429
    assert abs(y[0, 0] - (phi1 - (1.0 - phi1) + 0.25)) < 1e-15


def test_bf16_rounding_of_listed_bit_patterns():
    """Round to nearest, ties to even, on FP32 bit patterns (IEEE 754
    roundTiesToEven onto the 8-bit-significand format)."""
    cases = {
        0x3F800000: 0x3F80,   # 1.0
        0x3F807FFF: 0x3F80,   # just below the midpoint of 1.0 and 1 + 2^-7
        0x3F808000: 0x3F80,   # midpoint, lower neighbour even
        0x3F808001: 0x3F81,   # just above the midpoint
        0x3F818000: 0x3F82,   # midpoint, upper neighbour even
        0xBF818000: 0xBF82,   # the same, negative
        0x7F7F7FFF: 0x7F7F,   # largest finite BF16
        0x7F7F8000: 0x7F80,   # midpoint of the largest finite and infinity: to infinity (even)
        0x00008000: 0x0000,   # subnormal midpoint, lower neighbour (zero) even
        0x00018000: 0x0002,   # subnormal midpoint, upper neighbour even
        0x80000000: 0x8000,   # -0
    }
    bits = np.array(list(cases), dtype=np.uint32)
    got = mlp.bf16(bits.view(np.float32)).astype(np.float32).view(np.uint32)
    want = np.array(list(cases.values()), dtype=np.uint32) << 16
    assert np.array_equal(got, want), [hex(v) for v in got]


def test_bf16_matches_torch_conversion():
    """Against PyTorch's own FP32 -> BF16 conversion on normal, subnormal and
    near-overflow values (NaN excluded)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    u = rng.integers(0, 2 ** 32, size=200000, dtype=np.uint64).astype(np.uint32)
    u = np.concatenate([u, rng.integers(0, 2 ** 24, size=5000).astype(np.uint32),
                        0x7F7F0000 + rng.integers(0, 2 ** 16, size=5000).astype(np.uint32)])
    f = u.view(np.float32)
    f = f[~np.isnan(f)]
    ref = torch.from_numpy(f.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    got = mlp.bf16(f).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


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
