"""ORACLE — test infrastructure only (see the package docstring).

fp64 NumPy statement of the kernel selector's network and its training step:

* network: x (F=5 features) -> ReLU(x W1 + b1) (64) -> ReLU(h1 W2 + b2) (64)
  -> y = h2 W3 + b3 (C outputs, one predicted log-time per candidate kernel
  configuration);
* loss: mean squared error over all B x C outputs,
  L = sum((y - t)^2) / (B C), so dL/dy = 2 (y - t) / (B C);
* update: Adam (Kingma and Ba, "Adam: A Method for Stochastic Optimization",
  2015, Algorithm 1) with bias-corrected moments.

Weights are stored [in, out] row-major; parameter order is
W1, b1, W2, b2, W3, b3.  Plain matrix products, no fusion.
"""
from __future__ import annotations

import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes(F: int = 5, H: int = 64, C: int = 4):
    return [(F, H), (H,), (H, H), (H,), (H, C), (C,)]


def forward(P, X):
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in P]
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    return y, (X, z1, h1, z2, h2)


def loss(Y, T):
    Y = np.asarray(Y, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    return float(np.sum((Y - T) ** 2) / Y.size)


def backward(P, cache, Y, T):
    """Gradients of the MSE loss with respect to W1, b1, W2, b2, W3, b3."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in P]
    X, z1, h1, z2, h2 = cache
    dy = 2.0 * (np.asarray(Y, np.float64) - np.asarray(T, np.float64)) / Y.size
    dW3 = h2.T @ dy
    db3 = dy.sum(axis=0)
    dh2 = dy @ W3.T
    dz2 = dh2 * (z2 > 0)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (z1 > 0)
    dW1 = X.T @ dz1
    db1 = dz1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def loss_and_grad(P, X, T):
    Y, cache = forward(P, X)
    return loss(Y, T), backward(P, cache, Y, T)


def adam_step(P, G, M, V, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam step (t is the 1-based step number); returns new (P, M, V)."""
    newP, newM, newV = [], [], []
    for p, g, m, v in zip(P, G, M, V):
        p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        newP.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        newM.append(m)
        newV.append(v)
    return newP, newM, newV
