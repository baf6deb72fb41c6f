"""Pins for the fp64 selector-network oracle (no GPU): central finite
differences for the backward pass, the affine closed form of the forward pass
when every ReLU is active, and Adam's closed-form steps."""
from __future__ import annotations

import numpy as np

from oracle import mlp


def _params(dg, C=4, stream=0, scale=0.5):
    out = []
    for i, s in enumerate(mlp.shapes(C=C)):
        n = int(np.prod(s))
        u = dg.uniform(dg.STREAM_TESTS + 9000 + 10 * stream + i, n)
        out.append(((u - 0.5) * 2 * scale).reshape(s))
    return out


def test_forward_affine_when_relus_active(dg):
    # positive inputs and weights keep every pre-activation positive, so the
    # network is the affine map X W1 W2 W3 + (b1 W2 W3 + b2 W3 + b3)
    P = [np.abs(p) + 0.01 for p in _params(dg, stream=1)]
    X = dg.uniform(dg.STREAM_TESTS + 9100, 7 * 5).reshape(7, 5) + 0.1
    W1, b1, W2, b2, W3, b3 = P
    want = X @ (W1 @ W2 @ W3) + (b1 @ W2 @ W3 + b2 @ W3 + b3)
    got, _ = mlp.forward(P, X)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_forward_relu_zeroes_negative_layer(dg):
    P = _params(dg, stream=2)
    P[0] = -np.abs(P[0])
    P[1] = -np.abs(P[1]) - 0.1
    X = dg.uniform(dg.STREAM_TESTS + 9101, 4 * 5).reshape(4, 5)
    # h1 == 0, so y = relu(b2) W3 + b3 for every sample
    want = np.maximum(P[3], 0) @ P[4] + P[5]
    got, _ = mlp.forward(P, X)
    assert np.allclose(got, np.tile(want, (4, 1)), rtol=1e-12)


def test_backward_matches_central_differences(dg):
    P = _params(dg, stream=3)
    X = (dg.uniform(dg.STREAM_TESTS + 9102, 6 * 5).reshape(6, 5) - 0.5) * 3
    T = dg.uniform(dg.STREAM_TESTS + 9103, 6 * 4).reshape(6, 4)
    _, G = mlp.loss_and_grad(P, X, T)
    h = 1e-6
    for pi, p in enumerate(P):
        flat = p.reshape(-1)
        for j in range(0, flat.size, max(1, flat.size // 40)):
            old = flat[j]
            flat[j] = old + h
            lp = mlp.loss(mlp.forward(P, X)[0], T)
            flat[j] = old - h
            lm = mlp.loss(mlp.forward(P, X)[0], T)
            flat[j] = old
            num = (lp - lm) / (2 * h)
            assert abs(num - G[pi].reshape(-1)[j]) < 1e-7 + 1e-5 * abs(num), (mlp.NAMES[pi], j)


def test_adam_closed_form(dg):
    # with bias correction the first step is -lr * g / (|g| + eps), and a
    # constant gradient keeps giving the same step
    P = _params(dg, stream=4)
    G = [np.full_like(p, 0.37) if i % 2 else np.full_like(p, -2.5) for i, p in enumerate(P)]
    M = [np.zeros_like(p) for p in P]
    V = [np.zeros_like(p) for p in P]
    lr, eps = 1e-2, 1e-8
    cur = P
    for t in range(1, 6):
        nxt, M, V = mlp.adam_step(cur, G, M, V, t, lr, eps=eps)
        for a, b, g in zip(cur, nxt, G):
            assert np.allclose(b - a, -lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-15)
        cur = nxt


def test_adam_descends_quadratic(dg):
    # minimising sum((p - 3)^2) from 0 converges to 3
    p = [np.zeros(3)]
    M, V = [np.zeros(3)], [np.zeros(3)]
    for t in range(1, 3001):
        g = [2 * (p[0] - 3.0)]
        p, M, V = mlp.adam_step(p, g, M, V, t, 0.05)
    assert np.allclose(p[0], 3.0, atol=1e-3)
