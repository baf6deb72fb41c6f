"""How a single query reaches its kernel: queries of at most 256 ids (and no
truth table) carry their ids in the kernel's parameter block, larger ones and
table queries stage them in device memory; the cardinality is completed by
the kernel through the staging slot's header, with no memset before it.
Both sides of the 256-id boundary, on every single-query path, against the
oracle bit-exactly; the header must come back to zero after every launch,
which a long run of calls cycling through the slots (and two streams, and
calls without a cardinality) would expose."""
from __future__ import annotations

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

R_BITS = 64 * 3000 + 41
NBM = 300


@pytest.fixture(scope="module")
def bm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1402_4073_gb300 as bm
    return bm


@pytest.fixture(scope="module")
def served(bm, dg):
    d = dg.pool_densities(dg.STREAM_TESTS + 19000, NBM, 1e-3, 0.3)
    words = dg.runs(dg.STREAM_TESTS + 19001, R_BITS, d, 64.0)
    flat, offs = dg.positions(words, R_BITS)
    pool = bm.Pool(R_BITS, NBM)
    pool.put_dense(words)
    pool.put_positions(flat, offs)
    pool.put_rle()
    yield pool, words
    pool.close()


def _ids(dg, n, k):
    u = dg.uniform(dg.STREAM_TESTS + 19100 + 7 * n + k, n)
    return np.minimum((u * NBM).astype(np.int64), NBM - 1).astype(np.uint32)  # repeats allowed


@pytest.mark.parametrize("n", [1, 255, 256, 257, 600])
def test_every_path_both_sides_of_the_inline_limit(bm, oracle_lib, dg, served, n):
    pool, words = served
    ids = _ids(dg, n, 0)
    queries = [dg.Query(ids, 0, theta=max(1, n // 4)),
               dg.Query(ids, 1, lo=1, hi=max(1, n // 3)),
               dg.Query(ids, 2, table=dg.table_from_bools(np.arange(n + 1) % 3 == 1))]
    for q in queries:
        want = oracle_lib.query(words, q, R_BITS)
        for path in (bm.PATH_DENSE, bm.PATH_SPARSE, bm.PATH_RLE):
            out = pool.empty_words().fill_(-1)
            card = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            assert bm.query_run(pool, q, out, card, path=path) == path
            torch.cuda.synchronize()
            pool.status()
            what = f"n={n} kind={q.kind} path={path}"
            assert np.array_equal(bm.to_numpy_words(out), want[0]), what
            assert int(card.item()) == want[1], what
    pool.set_looped(3)  # theta = 2 and theta = n - 1 through the Looped kernel
    try:
        for theta in (2, max(2, n - 1)):
            want = oracle_lib.threshold(words, ids, R_BITS, theta)
            out = pool.empty_words().fill_(-1)
            card = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            bm.threshold(pool, ids, theta, out, card)
            torch.cuda.synchronize()
            assert np.array_equal(bm.to_numpy_words(out), want[0]), f"looped n={n} theta={theta}"
            assert int(card.item()) == want[1]
    finally:
        pool.set_looped(0)


def test_many_calls_two_streams_and_no_cardinality(bm, oracle_lib, dg, served):
    """40 calls alternating between two streams (the 8 staging slots cycle
    five times), every fifth without a cardinality; each result and
    cardinality against the oracle."""
    pool, words = served
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs, cards, wants = [], [], []
    for i in range(40):
        n = (3, 40, 256, 257, 700)[i % 5]
        ids = _ids(dg, n, i)
        theta = 1 + i % max(1, n // 2)
        path = (bm.PATH_DENSE, bm.PATH_SPARSE, bm.PATH_RLE)[i % 3]
        stream = s1 if i % 2 else s2
        q = dg.Query(ids, 0, theta=theta)
        o = pool.empty_words()
        c = None if i % 5 == 4 else torch.full((1,), -1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()  # the buffers exist before the other stream uses them
        bm.query_run(pool, q, o, c, path=path, stream=stream)
        outs.append(o)
        cards.append(c)
        wants.append(oracle_lib.query(words, q, R_BITS))
    torch.cuda.synchronize()
    pool.status()
    for i, (o, c, w) in enumerate(zip(outs, cards, wants)):
        assert np.array_equal(bm.to_numpy_words(o), w[0]), i
        if c is not None:
            assert int(c.item()) == w[1], i
