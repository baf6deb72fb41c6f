"""GPU parity of weighted thresholds with an optional AND / OR / AND NOT of
one more bitmap, against the oracle (bit-exact): small and large weights,
weight 0, repeated ids, theta at 0, 1, the sum and above it, every combining
operation, ragged r, and enough weight-1 inputs to fill sixteen-input blocks."""
from __future__ import annotations

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1402_4073_gb300 as bm
    return bm


def _run(bm, pool, ids, weights, theta, post_op=0, post_id=0):
    out = pool.empty_words()
    out.fill_(-1)
    card = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    bm.weighted_threshold(pool, ids, weights, theta, out, card, post_op, post_id)
    torch.cuda.synchronize()
    pool.status()
    return bm.to_numpy_words(out), int(card.item())


@pytest.mark.parametrize("r_bits", [64, 1000, 16384 * 3 + 17])
def test_weighted_small(bm, oracle_lib, dg, r_bits):
    words = dg.bernoulli(dg.STREAM_TESTS + 21000, r_bits, np.linspace(0.05, 0.8, 24))
    ids = np.array(list(range(20)) + [3, 3, 7], dtype=np.uint32)
    weights = np.array([1, 2, 3, 1, 0, 5, 1, 1, 4, 1, 1, 1, 2, 1, 1, 7, 1, 1, 1, 1, 2, 1, 3],
                       dtype=np.uint32)
    s = int(weights.sum())
    with bm.Pool(r_bits, words.shape[0]) as pool:
        pool.put_dense(words)
        for theta in (0, 1, 2, 7, s // 2, s - 1, s, s + 1):
            got = _run(bm, pool, ids, weights, theta)
            want = oracle_lib.weighted(words, ids, weights, r_bits, theta)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], theta
        for op in (1, 2, 3):
            for theta in (0, s // 3, s + 1):
                got = _run(bm, pool, ids, weights, theta, op, 23)
                want = oracle_lib.weighted(words, ids, weights, r_bits, theta, op, words[23])
                assert np.array_equal(got[0], want[0]) and got[1] == want[1], (op, theta)
        # all weights 1: the plain threshold
        ones = np.ones(20, dtype=np.uint32)
        for theta in (1, 5, 20):
            got = _run(bm, pool, ids[:20], ones, theta)
            want = oracle_lib.threshold(words, ids[:20], r_bits, theta)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], theta


@pytest.mark.parametrize("wmax", [25, 300, 2000, 70000, 500000, (1 << 24) - 1])
def test_weighted_large(bm, oracle_lib, dg, wmax):
    """Sums of about 2^12, 2^16, 2^18, 2^23, 2^26 and 2^31: every compiled
    plane count from 12 to 32 (weights too large to run as copies)."""
    r_bits = 20000
    n = 300
    words = dg.bernoulli(dg.STREAM_TESTS + 21100, r_bits, np.linspace(0.02, 0.9, 50))
    ids = (np.arange(n) * 7 % 50).astype(np.uint32)
    u = dg.uniform(dg.STREAM_TESTS + 21101, n)
    weights = np.maximum(1, (u * wmax).astype(np.uint64)).astype(np.uint32)
    weights[::5] = 1  # some weight-1 inputs, enough for full sixteen-input blocks
    s = int(weights.astype(np.uint64).sum())
    assert s < (1 << 32)
    with bm.Pool(r_bits, 50) as pool:
        pool.put_dense(words)
        for theta in (1, s // 4, s // 2, (3 * s) // 4, s, s + 1):
            got = _run(bm, pool, ids, weights, theta)
            want = oracle_lib.weighted(words, ids, weights, r_bits, theta)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], theta
        got = _run(bm, pool, ids, weights, s // 2, 3, 49)
        want = oracle_lib.weighted(words, ids, weights, r_bits, s // 2, 3, words[49])
        assert np.array_equal(got[0], want[0]) and got[1] == want[1]


def test_weighted_eight_planes(bm, oracle_lib, dg):
    """A sum of 8 planes above 8 per input (no copies): the smallest
    carry-save form, with weight-1 inputs beside it."""
    r_bits = 64 * 300 + 9
    words = dg.bernoulli(dg.STREAM_TESTS + 21300, r_bits, np.linspace(0.05, 0.95, 20))
    ids = np.arange(20, dtype=np.uint32)
    weights = np.full(20, 12, dtype=np.uint32)
    weights[:3] = 1
    s = int(weights.sum())
    assert 8 * 20 < s < 256
    with bm.Pool(r_bits, 20) as pool:
        pool.put_dense(words)
        for theta in (1, 12, 13, 100, s - 1, s):
            got = _run(bm, pool, ids, weights, theta)
            want = oracle_lib.weighted(words, ids, weights, r_bits, theta)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], theta


def test_weighted_errors(bm, dg):
    r_bits = 5000
    words = dg.bernoulli(dg.STREAM_TESTS + 21200, r_bits, np.array([0.1, 0.2, 0.3]))
    with bm.Pool(r_bits, 4) as pool:
        pool.put_dense(words)
        out = pool.empty_words()
        with pytest.raises(bm.BMError) as e:
            bm.weighted_threshold(pool, [0, 1], [1, bm.BM_WEIGHT_MAX + 1], 1, out)
        assert e.value.code == bm.BM_EINVAL
        with pytest.raises(bm.BMError) as e:
            bm.weighted_threshold(pool, [0] * 300, [bm.BM_WEIGHT_MAX] * 300, 1, out)  # sum >= 2^32
        assert e.value.code == bm.BM_EINVAL
        with pytest.raises(bm.BMError) as e:
            bm.weighted_threshold(pool, [0, 1], [1, 1], 1, out, post_op=1, post_id=3)  # no bitmap 3
        assert e.value.code == bm.BM_ERANGE
        with pytest.raises(bm.BMError) as e:
            bm.weighted_threshold(pool, [0, 1], [1, 1], 1, out, post_op=4)
        assert e.value.code == bm.BM_EINVAL
        with pytest.raises(bm.BMError) as e:
            bm.weighted_threshold(pool, [0, 3], [1, 1], 1, out)
        assert e.value.code == bm.BM_ERANGE
