"""The selector network's GPU kernels against the fp64 oracle: forward
outputs, every gradient (relative per-tensor L2 error <= 1e-4, the bound set
for fp32 sums of at most a few thousand terms), and Adam steps."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import mlp

pytestmark = pytest.mark.gpu
F, H, C = 5, 64, 4


@pytest.fixture(scope="module")
def bm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1402_4073_gb300 as bm
    return bm


def _params(dg, stream):
    out = []
    for i, s in enumerate(mlp.shapes(F, H, C)):
        n = int(np.prod(s))
        u = dg.uniform(dg.STREAM_TESTS + 13000 + 10 * stream + i, n)
        out.append(((u - 0.5) * (2.0 / np.sqrt(s[0]))).reshape(s))
    return out


def _flat(P):
    return torch.from_numpy(np.concatenate([p.reshape(-1) for p in P]).astype(np.float32)).cuda()


def _split(t):
    a = t.detach().cpu().numpy().astype(np.float64)
    out, o = [], 0
    for s in mlp.shapes(F, H, C):
        n = int(np.prod(s))
        out.append(a[o:o + n].reshape(s))
        o += n
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("B", [1, 7, 256, 3000])
def test_forward_backward_match_oracle(bm, dg, B):
    P = _params(dg, B)
    X = (dg.uniform(dg.STREAM_TESTS + 13100 + B, B * F).reshape(B, F) - 0.5) * 4
    T = dg.uniform(dg.STREAM_TESTS + 13200 + B, B * C).reshape(B, C) * 3
    # run the oracle on the fp32-rounded values the GPU sees
    P32 = [p.astype(np.float32).astype(np.float64) for p in P]
    X32, T32 = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    want_y, cache = mlp.forward(P32, X32)
    want_g = mlp.backward(P32, cache, want_y, T32)
    want_l = mlp.loss(want_y, T32)

    params = _flat(P)
    x = torch.from_numpy(X.astype(np.float32)).cuda()
    t = torch.from_numpy(T.astype(np.float32)).cuda()
    y, h1, h2 = bm.mlp_forward(params, x, H, C)
    grads, loss = bm.mlp_backward(params, x, h1, h2, y, t)
    torch.cuda.synchronize()
    assert _rel(y.cpu().numpy().astype(np.float64), want_y) < 1e-5
    assert abs(float(loss.item()) - want_l) <= 1e-4 * abs(want_l) + 1e-7
    for name, g, w in zip(mlp.NAMES, _split(grads), want_g):
        assert _rel(g, w) < 1e-4, name


def test_adam_matches_oracle(bm, dg):
    P = _params(dg, 99)
    params = _flat(P)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    M = [np.zeros_like(p) for p in P]
    V = [np.zeros_like(p) for p in P]
    cur = [p.astype(np.float32).astype(np.float64) for p in P]
    for step in range(1, 6):
        G = [np.sin(np.arange(p.size).reshape(p.shape) * (0.1 * step) + i) * 0.01
             for i, p in enumerate(P)]
        g = _flat(G)
        bm.mlp_adam(params, g, m, v, step, 1e-3)
        cur, M, V = mlp.adam_step(cur, [gg.astype(np.float32).astype(np.float64) for gg in G],
                                  M, V, step, 1e-3)
    torch.cuda.synchronize()
    for a, b in zip(_split(params), cur):
        assert np.allclose(a, b, rtol=1e-5, atol=1e-6)


def test_training_reduces_loss(bm, dg):
    """A few hundred GPU Adam steps fit a smooth target far better than the
    initial network."""
    B = 512
    X = (dg.uniform(dg.STREAM_TESTS + 13300, B * F).reshape(B, F) - 0.5) * 2
    T = np.stack([X[:, 0] * 2 + X[:, 1] ** 2, np.sin(X[:, 2]), X[:, 3] - X[:, 4], X[:, 0] * X[:, 1]],
                 axis=1)
    params = _flat(_params(dg, 7))
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    x = torch.from_numpy(X.astype(np.float32)).cuda()
    t = torch.from_numpy(T.astype(np.float32)).cuda()
    first = None
    for step in range(1, 401):
        y, h1, h2 = bm.mlp_forward(params, x, H, C)
        grads, loss = bm.mlp_backward(params, x, h1, h2, y, t)
        if first is None:
            first = float(loss.item())
        bm.mlp_adam(params, grads, m, v, step, 3e-3)
    y, h1, h2 = bm.mlp_forward(params, x, H, C)
    _, loss = bm.mlp_backward(params, x, h1, h2, y, t)
    assert float(loss.item()) < 0.05 * first
