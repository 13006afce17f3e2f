"""CPU ORACLE for the learned cost model (TEST INFRASTRUCTURE ONLY).

A multilayer perceptron 20 -> 64 -> 64 -> 2 with ReLU hidden units, trained on
the squared error of predicted per-variant log costs, with Adam (Kingma & Ba,
"Adam: A Method for Stochastic Optimization", ICLR 2015, Algorithm 1). This is
the scheduler's analogue of the paper's performance-aware task scheduling
(Sec. IV, PATS: estimated per-task speedups pick the device), here picking the
per-tile variant and the packing order; it never touches pixel values.

fp64 NumPy, written from the definitions (matrix products are the only
library primitive); shares nothing with the CUDA kernels.

Layout (matches the C ABI's flat parameter blob, row-major):
    W1 (64, 20), b1 (64), W2 (64, 64), b2 (64), W3 (2, 64), b3 (2)
Loss over a batch of N samples with targets T (N, 2):
    L = 1 / (2 N) * sum_n sum_k (Y[n, k] - T[n, k])^2
"""
from __future__ import annotations

import numpy as np

SIZES = (20, 64, 64, 2)
NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes():
    d0, d1, d2, d3 = SIZES
    return [(d1, d0), (d1,), (d2, d1), (d2,), (d3, d2), (d3,)]


def n_params() -> int:
    return sum(int(np.prod(s)) for s in shapes())


def unflatten(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, s in zip(NAMES, shapes()):
        n = int(np.prod(s))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[n], np.float64).ravel() for n in NAMES])


def init(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, s in zip(NAMES, shapes()):
        if name.startswith("W"):
            bound = np.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-bound, bound, size=s).ravel())
        else:
            parts.append(np.zeros(s).ravel())
    return np.concatenate(parts)


def forward(theta: np.ndarray, X: np.ndarray):
    """Returns (Y, cache); Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 per row."""
    p = unflatten(theta)
    X = np.asarray(X, np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ p["W2"].T + p["b2"]
    A2 = np.maximum(Z2, 0.0)
    Y = A2 @ p["W3"].T + p["b3"]
    return Y, (X, Z1, A1, Z2, A2)


def loss(Y: np.ndarray, T: np.ndarray) -> float:
    N = Y.shape[0]
    return float(0.5 * np.sum((Y - T) ** 2) / N)


def backward(theta: np.ndarray, cache, Y: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Gradient of the loss with respect to the flat parameters (chain rule)."""
    p = unflatten(theta)
    X, Z1, A1, Z2, A2 = cache
    N = Y.shape[0]
    dY = (Y - T) / N
    g = {"W3": dY.T @ A2, "b3": dY.sum(axis=0)}
    dZ2 = (dY @ p["W3"]) * (Z2 > 0)
    g["W2"] = dZ2.T @ A1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * (Z1 > 0)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return flatten(g)


def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1). Returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(theta, X, T, epochs, lr=1e-3, batch=256, seed=0):
    """Mini-batch Adam over shuffled epochs (shuffle order from `seed`)."""
    rng = np.random.default_rng(seed)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    t = 0
    N = X.shape[0]
    for _ in range(epochs):
        perm = rng.permutation(N)
        for s in range(0, N, batch):
            idx = perm[s:s + batch]
            Y, cache = forward(theta, X[idx])
            g = backward(theta, cache, Y, T[idx])
            t += 1
            theta, m, v = adam_step(theta, g, m, v, t, lr)
    return theta
