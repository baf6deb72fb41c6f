"""bm_threshold_noalloc: the threshold query for callers that cannot call
cudaMalloc (for example a plugin whose host program owns all device memory,
or a service that must not allocate once running).  It keeps its ids in a
fixed device array inside the library instead of pool-allocated buffers.

Checked through the C ABI against bm_threshold (the pool entry point) and
against the oracle, on calls in a row: the second with fewer ids, so that
stale ids left in the shared array by the first call would show; theta = 0
and theta = n + 1 (the constant predicates); and the largest accepted n,
16384 ids with repeats.  Integer outputs: bit-exact."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

NOALLOC_MAX_N = 16384


def _noalloc(bm, pool, ids, theta, r_bits, nbm, stream):
    info = pool.info()
    got = pool.empty_words()
    got.fill_(-1)
    got_card = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    rc = bm.lib.bm_threshold_noalloc(
        ctypes.c_void_p(info["dense_base"]), info["stride_words"], nbm, r_bits, ids.ctypes.data,
        len(ids), theta, got.data_ptr(), got_card.data_ptr(), stream)
    assert rc == 0, bm.lib.bm_strerror(rc)
    return got, got_card


def _check_calls(bm, oracle_lib, words, r_bits, calls):
    nbm = words.shape[0]
    with bm.Pool(r_bits, nbm) as pool:
        pool.put_dense(words)
        stream = torch.cuda.current_stream().cuda_stream
        for ids, theta in calls:
            want = pool.empty_words()
            want_card = torch.zeros(1, dtype=torch.int64, device="cuda")
            bm.threshold(pool, ids, theta, want, want_card)
            got, got_card = _noalloc(bm, pool, ids, theta, r_bits, nbm, stream)
            torch.cuda.synchronize()
            what = f"n={len(ids)} theta={theta}"
            # the pool entry point
            assert torch.equal(got, want), what
            assert int(got_card.item()) == int(want_card.item()), what
            # the oracle
            o_words, o_card = oracle_lib.threshold(words, ids, r_bits, theta)
            assert np.array_equal(bm.to_numpy_words(got), o_words), what
            assert int(got_card.item()) == o_card, what
        return pool.info()


def test_noalloc_matches_pool_entry_point_and_oracle(dg, oracle_lib):
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    import paper_1402_4073_gb300 as bm

    r_bits = 64 * 20000 + 29
    nbm = 48
    words = dg.bernoulli(dg.STREAM_TESTS + 9500, r_bits, np.linspace(0.02, 0.7, nbm))
    first = dg.floyd(dg.STREAM_TESTS + 9501, nbm, 40).astype(np.uint32)
    few = np.array([3, 3, 17, 5, 40], dtype=np.uint32)  # fewer ids, a repeat
    calls = [(first, 9), (few, 2), (few, 0), (few, len(few) + 1), (first, 1), (first, 40)]
    _check_calls(bm, oracle_lib, words, r_bits, calls)

    # sizes beyond the fixed scratch array are refused
    with bm.Pool(r_bits, nbm) as pool:
        pool.put_dense(words)
        info = pool.info()
        too_many = np.zeros(NOALLOC_MAX_N + 1, dtype=np.uint32)
        out = pool.empty_words()
        rc = bm.lib.bm_threshold_noalloc(ctypes.c_void_p(info["dense_base"]), info["stride_words"],
                                         nbm, r_bits, too_many.ctypes.data, len(too_many), 1,
                                         out.data_ptr(), None,
                                         torch.cuda.current_stream().cuda_stream)
        assert rc == bm.BM_EINVAL


def test_noalloc_largest_n(dg, oracle_lib):
    """n = 16384 ids drawn with repeats from 48 bitmaps (the whole scratch
    array), theta at the median count, then a short call after it."""
    import paper_1402_4073_gb300 as bm

    r_bits = 64 * 600 + 13
    nbm = 48
    words = dg.bernoulli(dg.STREAM_TESTS + 9510, r_bits, np.linspace(0.05, 0.6, nbm))
    u = dg.uniform(dg.STREAM_TESTS + 9511, NOALLOC_MAX_N)
    ids = np.minimum((u * nbm).astype(np.int64), nbm - 1).astype(np.uint32)
    theta = int(np.median(oracle_lib.counts(words, ids, r_bits)))
    calls = [(ids, theta), (ids[:7].copy(), 3)]
    _check_calls(bm, oracle_lib, words, r_bits, calls)
