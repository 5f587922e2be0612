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
from typing import List, Tuple

import numpy as np
from scipy.special import erf

SQRT1_2 = 1.0 / math.sqrt(2.0)


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), via the FP32 value.

    BF16 keeps the top 16 bits of an IEEE single; rounding adds 0x7FFF plus
    the lowest kept bit before truncating (finite inputs).
    """
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x: np.ndarray) -> np.ndarray:
    return 0.5 * x * (1.0 + erf(x * SQRT1_2))


def gelu_grad(x: np.ndarray) -> np.ndarray:
    return 0.5 * (1.0 + erf(x * SQRT1_2)) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def _op(a, lowp: bool):
    return bf16(a) if lowp else a


def forward(params: List[Tuple[np.ndarray, np.ndarray]], X: np.ndarray, lowp: bool = False):
    """Returns (output, cache of pre-activations and activations).

    lowp: round every GEMM operand to BF16 (the network's specified operand
    precision); products and sums stay FP64.
    """
    acts = [X]
    pres = []
    h = X
    for i, (Wt, b) in enumerate(params):
        z = _op(h, lowp) @ _op(Wt, lowp) + b
        pres.append(z)
        h = gelu(z) if i + 1 < len(params) else z
        acts.append(h)
    return h, (acts, pres)


def mse_loss(y: np.ndarray, t: np.ndarray) -> float:
    return float(np.mean((y - t) ** 2))


def backward(params, cache, y: np.ndarray, t: np.ndarray, lowp: bool = False):
    """Gradients of the MSE loss w.r.t. every (W, b); lowp as in forward."""
    acts, pres = cache
    g = 2.0 * (y - t) / y.size
    grads = [None] * len(params)
    for i in reversed(range(len(params))):
        Wt, _ = params[i]
        if i + 1 < len(params):
            g = g * gelu_grad(pres[i])
        grads[i] = (_op(acts[i], lowp).T @ _op(g, lowp), g.sum(axis=0))
        g = _op(g, lowp) @ _op(Wt, lowp).T
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


def flatten(params) -> np.ndarray:
    """Parameter vector: for each layer W (fan_in x fan_out, row-major) then b."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(vec: np.ndarray, sizes) -> list:
    out, at = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = vec[at:at + a * b].reshape(a, b)
        at += a * b
        bb = vec[at:at + b]
        at += b
        out.append((W.copy(), bb.copy()))
    return out


def cloud_features(bubbles: np.ndarray, domain_L: float, scale: float, n_keep: int = 0) -> np.ndarray:
    """Bubbles (nb, 4) in metres -> features ordered by the gap between each
    bubble's surface and the domain centre, |x_b - c| - r_b (ties by index):
    ((x-c)/s, (y-c)/s, (z-c)/s, r/s), for the n_keep bubbles nearest the
    centre in that order (0: all)."""
    c = 0.5 * domain_L
    inv = 1.0 / scale
    d = bubbles[:, :3] - c
    key = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]) - bubbles[:, 3]
    order = np.lexsort((np.arange(len(key)), key))
    f = np.empty((len(key), 4))
    f[:, :3] = (bubbles[order, :3] - c) * inv
    f[:, 3] = bubbles[order, 3] * inv
    k = len(key) if n_keep <= 0 else min(n_keep, len(key))
    return f[:k].ravel()
