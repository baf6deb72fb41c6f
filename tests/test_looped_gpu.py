"""GPU parity of the Looped recurrence (Sec. 4.4) for small thresholds and,
through the corrected complement identity (Sec. 2.3), for thresholds near N,
against the CPU oracle, bit-exact: T = 1, 2, 3 and N - T + 1 = 1, 2, 3, the
negated predicate "count < T", repeated ids, all-zero and all-one inputs,
n mod 16 remainders, ragged r; and the same answers with Looped turned off."""
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


def _words(dg, r_bits, stream):
    nw = (r_bits + 63) // 64
    w = dg.bernoulli(stream, r_bits, np.linspace(0.03, 0.97, 38))
    zero = np.zeros((1, nw), np.uint64)
    one = np.full((1, nw), np.uint64(0xFFFFFFFFFFFFFFFF))
    if r_bits % 64:
        one[0, -1] &= np.uint64((1 << (r_bits % 64)) - 1)
    return np.concatenate([w, zero, one])  # ids 38 (zeros) and 39 (ones)


def _check(bm, pool, oracle_lib, dg, words, r_bits, ids, theta):
    n = len(ids)
    out = pool.empty_words()
    card = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    out.fill_(-1)
    bm.threshold(pool, ids, theta, out, card)
    torch.cuda.synchronize()
    pool.status()
    want = oracle_lib.threshold(words, ids, r_bits, theta)
    assert np.array_equal(bm.to_numpy_words(out), want[0]), (n, theta)
    assert int(card.item()) == want[1], (n, theta)
    # "count < theta": the threshold negated
    table = dg.table_from_bools([c < theta for c in range(n + 1)])
    out.fill_(-1)
    bm.symmetric(pool, ids, table, out, card)
    torch.cuda.synchronize()
    pool.status()
    want = oracle_lib.symmetric(words, ids, r_bits, table)
    assert np.array_equal(bm.to_numpy_words(out), want[0]), (n, theta, "<")
    assert int(card.item()) == want[1], (n, theta, "<")


@pytest.mark.parametrize("r_bits", [320, 64 * 777 + 5, 16384 * 3 + 17, 1 << 20])
def test_looped_matches_oracle(bm, oracle_lib, dg, r_bits):
    words = _words(dg, r_bits, dg.STREAM_TESTS + 22000)
    rng = np.random.default_rng(22001)
    with bm.Pool(r_bits, words.shape[0]) as pool:
        pool.put_dense(words)
        for max_t in (3, 0):
            pool.set_looped(max_t)
            assert pool.configs()["looped"] == max_t
            for n in (1, 2, 3, 4, 5, 15, 16, 17, 33, 40, 100):
                ids = rng.integers(0, words.shape[0], n).astype(np.uint32)
                if n >= 5:
                    ids[:2] = [38, 39]  # an all-zero and an all-one input
                    ids[4] = ids[3]     # a repeated id
                for theta in sorted({1, 2, 3, 4, n - 3, n - 2, n - 1, n}):
                    if 1 <= theta <= n:
                        _check(bm, pool, oracle_lib, dg, words, r_bits, ids, theta)


def test_looped_large_dense_workload_subset(bm, oracle_lib, dg):
    """Clustered inputs as in the large dense workload (densities
    max(0.5/k, 1e-4), runs of mean 8 rows), 256 inputs over r = 2^20:
    T = 2 directly and T = 255 through the complement, with rows planted
    where exactly 254, 255 and 256 inputs are set."""
    r_bits = 1 << 20
    words = dg.runs(dg.STREAM_TESTS + 22100, r_bits, dg.config2_density(256), 8.0)
    for row, k in ((1000, 254), (5000, 255), (9001, 256)):
        words[:k, row // 64] |= np.uint64(1 << (row % 64))
    ids = np.arange(256, dtype=np.uint32)
    with bm.Pool(r_bits, 256) as pool:
        pool.put_dense(words)
        pool.set_looped(3)
        for theta in (1, 2, 3, 254, 255, 256):
            _check(bm, pool, oracle_lib, dg, words, r_bits, ids, theta)


def test_looped_errors(bm):
    with bm.Pool(6400, 2) as pool:
        with pytest.raises(bm.BMError) as e:
            pool.set_looped(4)
        assert e.value.code == bm.BM_EINVAL
        assert pool.configs()["looped"] == 0
