"""Oracle for the MLP surrogate (test infrastructure).

Plain numpy FP64.  Architecture: d_in -> H -> H -> H -> d_out, exact-erf GELU
after each hidden layer, linear output, mean-squared-error loss, Adam
(Kingma & Ba 2015) with bias correction.  Weights are stored (fan_in, fan_out)
so a layer is y = x @ W + b.  Initial weights are inputs (drawn by the
caller's seeded generator), so both implementations start from the same
numbers.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np
from scipy.special import erf

SQRT1_2 = 1.0 / math.sqrt(2.0)


def gelu(x: np.ndarray) -> np.ndarray:
    return 0.5 * x * (1.0 + erf(x * SQRT1_2))


def gelu_grad(x: np.ndarray) -> np.ndarray:
    return 0.5 * (1.0 + erf(x * SQRT1_2)) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(params: List[Tuple[np.ndarray, np.ndarray]], X: np.ndarray):
    """Returns (output, cache of pre-activations and activations)."""
    acts = [X]
    pres = []
    h = X
    for i, (Wt, b) in enumerate(params):
        z = h @ Wt + b
        pres.append(z)
        h = gelu(z) if i + 1 < len(params) else z
        acts.append(h)
    return h, (acts, pres)


def mse_loss(y: np.ndarray, t: np.ndarray) -> float:
    return float(np.mean((y - t) ** 2))


def backward(params, cache, y: np.ndarray, t: np.ndarray):
    """Gradients of the MSE loss w.r.t. every (W, b)."""
    acts, pres = cache
    g = 2.0 * (y - t) / y.size
    grads = [None] * len(params)
    for i in reversed(range(len(params))):
        Wt, _ = params[i]
        if i + 1 < len(params):
            g = g * gelu_grad(pres[i])
        grads[i] = (acts[i].T @ g, g.sum(axis=0))
        g = g @ Wt.T
    return grads


class Adam:
    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.t = 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        out = []
        for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[i][j] + (1.0 - self.b1) * g
                v = self.b2 * self.v[i][j] + (1.0 - self.b2) * g * g
                self.m[i] = (m, self.m[i][1]) if j == 0 else (self.m[i][0], m)
                self.v[i] = (v, self.v[i][1]) if j == 0 else (self.v[i][0], v)
                new.append(p - self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps))
            out.append((new[0], new[1]))
        return out


def train(params, X, T, epochs: int, batch: int, lr: float = 1e-3):
    """Full-batch-order minibatch training (rows taken in order, no shuffle)."""
    opt = Adam(params, lr=lr)
    losses = []
    n = X.shape[0]
    for _ in range(epochs):
        for s in range(0, n, batch):
            xb, tb = X[s:s + batch], T[s:s + batch]
            y, cache = forward(params, xb)
            losses.append(mse_loss(y, tb))
            params = opt.step(params, backward(params, cache, y, tb))
    return params, losses
