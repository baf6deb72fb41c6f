"""Parity at the full workload sizes, in the configurations bench.py times:
the mixed batch (2000 x 2^24, 4096 queries), the sparse + selector pool
(5000 x 2^24, dense and lists), the serving pool (10000 x 2^22), the
clustered run-length pools (256 x 2^26) and the co-sparse pool with lists of
zeros (1500 x 2^24).  The
oracle checks sampled output word ranges of sampled queries (it computes any
word range on its own); every cardinality is checked against the popcount of
the whole returned bitmap."""
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


def _ranges(dg, stream, words, k=6, width=48):
    """k random word ranges plus the first and the last range."""
    u = dg.uniform(stream, k)
    starts = sorted({0, max(0, words - width)} | {int(x * (words - width)) for x in u})
    return [(s, min(words, s + width)) for s in starts]


def _popcount(words_u64: np.ndarray) -> int:
    return int(np.unpackbits(words_u64.view(np.uint8)).sum())


def _check_sampled(oracle_lib, dg, pool_words, q, r_bits, got_words, got_card, stream):
    assert _popcount(got_words) == got_card
    for w0, w1 in _ranges(dg, stream, len(got_words)):
        want, _ = oracle_lib.query(pool_words, q, r_bits, w0, w1)
        assert np.array_equal(got_words[w0:w1], want), (q.n, q.kind, w0)


def test_mixed_batch_full_size(bm, oracle_lib, dg):
    r_bits = 1 << 24
    words, _ = dg.mixed_pool(2000, r_bits)
    queries = dg.mixed_queries(4096, 2000)
    with bm.Pool(r_bits, 2000) as pool:
        pool.put_dense(words)
        outs = [pool.empty_words() for _ in queries]
        cards = torch.zeros(len(queries), dtype=torch.int64, device="cuda")
        bm.threshold_batch(pool, queries, outs, cards, paths=[bm.PATH_DENSE] * len(queries))
        torch.cuda.synchronize()
        pool.status()
        cards = cards.cpu().numpy()
        pick = dg.floyd(dg.STREAM_TESTS + 18000, len(queries), 96)
        for i in pick:
            _check_sampled(oracle_lib, dg, words, queries[i], r_bits, bm.to_numpy_words(outs[i]),
                           int(cards[i]), dg.STREAM_TESTS + 18001 + int(i))
        # one query of the batch alone: identical
        o = pool.empty_words()
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        bm.query_run(pool, queries[int(pick[0])], o, c, path=bm.PATH_DENSE)
        torch.cuda.synchronize()
        assert torch.equal(o, outs[int(pick[0])]) and int(c.item()) == int(cards[int(pick[0])])


def test_sparse_pool_full_size(bm, oracle_lib, dg):
    r_bits = 1 << 24
    words, flat, offs, _ = dg.sparse_pool(5000, r_bits)
    queries = dg.sparse_queries(2000, 5000)
    pick = [queries[int(i)] for i in dg.floyd(dg.STREAM_TESTS + 18100, len(queries), 48)]
    with bm.Pool(r_bits, 5000) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        for k, q in enumerate(pick):
            outs = {}
            for path in (bm.PATH_DENSE, bm.PATH_SPARSE):
                o = pool.empty_words()
                c = torch.zeros(1, dtype=torch.int64, device="cuda")
                bm.query_run(pool, q, o, c, path=path)
                torch.cuda.synchronize()
                outs[path] = (bm.to_numpy_words(o), int(c.item()))
            assert np.array_equal(outs[bm.PATH_DENSE][0], outs[bm.PATH_SPARSE][0])
            assert outs[bm.PATH_DENSE][1] == outs[bm.PATH_SPARSE][1]
            _check_sampled(oracle_lib, dg, words, q, r_bits, *outs[bm.PATH_SPARSE],
                           dg.STREAM_TESTS + 18101 + k)
        # the batched form with the density rule routing each query
        o = [pool.empty_words() for _ in pick]
        c = torch.zeros(len(pick), dtype=torch.int64, device="cuda")
        chosen = bm.threshold_batch(pool, pick, o, c)
        torch.cuda.synchronize()
        pool.status()
        c = c.cpu().numpy()
        for k, q in enumerate(pick):
            _check_sampled(oracle_lib, dg, words, q, r_bits, bm.to_numpy_words(o[k]), int(c[k]),
                           dg.STREAM_TESTS + 18201 + k)
        assert set(chosen.tolist()) <= {bm.PATH_DENSE, bm.PATH_SPARSE}


def test_serving_pool_full_size(bm, oracle_lib, dg):
    from paper_1402_4073_gb300.serve import Server
    r_bits = 1 << 22
    words, _ = dg.serving_pool(10000, r_bits)
    queries = dg.serving_queries(64, 20000.0)
    with bm.Pool(r_bits, 10000) as pool:
        pool.put_dense(words)
        slot = (pool.words * 8 + 255) // 256 * 256
        with Server(pool, mem_budget=128 * slot, max_batch=64, max_inflight=2) as srv:
            tickets = [srv.submit(q) for q in queries]
            for k, (q, t) in enumerate(zip(queries, tickets)):
                assert srv.wait(t, 30000) == 0
                got, card, lat, qu, path = srv.result(t)
                srv.release(t)
                _check_sampled(oracle_lib, dg, words, q, r_bits, got, card,
                               dg.STREAM_TESTS + 18301 + k)


def test_rle_clustered_full_size(bm, oracle_lib, dg):
    """The run-length path on the bench's clustered pool (256 x 2^26, runs of
    mean 4096 and 8 rows): every word equals the dense path's, sampled ranges
    equal the oracle's."""
    r_bits, n = 1 << 26, 256
    ids = np.arange(n, dtype=np.uint32)
    queries = [dg.Query(ids, 0, theta=2), dg.Query(ids, 0, theta=128), dg.Query(ids, 1, lo=2, hi=10)]
    for mean_run in (4096.0, 8.0):
        words = dg.runs(dg.STREAM_CONFIG2, r_bits, dg.config2_density(n), mean_run)
        with bm.Pool(r_bits, n) as pool:
            pool.put_dense(words)
            pool.put_rle()
            out_d, out_r = pool.empty_words(), pool.empty_words()
            cd = torch.zeros(1, dtype=torch.int64, device="cuda")
            cr = torch.zeros(1, dtype=torch.int64, device="cuda")
            for k, q in enumerate(queries):
                bm.query_run(pool, q, out_d, cd, path=bm.PATH_DENSE)
                bm.query_run(pool, q, out_r, cr, path=bm.PATH_RLE)
                torch.cuda.synchronize()
                pool.status()
                assert torch.equal(out_d, out_r), (mean_run, k)
                assert int(cd.item()) == int(cr.item())
                _check_sampled(oracle_lib, dg, words, q, r_bits, bm.to_numpy_words(out_r),
                               int(cr.item()), dg.STREAM_TESTS + 18600 + k)


def test_lists_of_zeros_full_size(bm, oracle_lib, dg):
    """Co-sparse pool of the bench (1500 x 2^24, half the bitmaps given by
    their zeros): ScanCount equals the dense path on every word."""
    r_bits, nbm = 1 << 24, 1500
    half = nbm // 2
    d = dg.pool_densities(dg.STREAM_SPARSE + (11 << 32), nbm, 1e-5, 1e-2)
    d[half:] = 1.0 - d[half:]
    words = dg.bernoulli(dg.STREAM_SPARSE + (12 << 32), r_bits, d)
    flat1, offs1 = dg.positions(words[:half], r_bits)
    flat0, offs0 = dg.positions(~words[half:], r_bits)
    with bm.Pool(r_bits, nbm) as pool:
        pool.put_dense(words)
        pool.put_positions(flat1, offs1)
        pool.put_positions(flat0, offs0, first_id=half, zeros=True)
        out_d, out_s = pool.empty_words(), pool.empty_words()
        cd = torch.zeros(1, dtype=torch.int64, device="cuda")
        cs = torch.zeros(1, dtype=torch.int64, device="cuda")
        for n in (1500, 300, 16):
            ids = dg.floyd(dg.STREAM_SPARSE + (13 << 32) + n, nbm, n)
            q = dg.Query(ids, 0, theta=n // 2 + 1)
            bm.query_run(pool, q, out_d, cd, path=bm.PATH_DENSE)
            bm.query_run(pool, q, out_s, cs, path=bm.PATH_SPARSE)
            torch.cuda.synchronize()
            pool.status()
            assert torch.equal(out_d, out_s), n
            assert int(cd.item()) == int(cs.item())
            _check_sampled(oracle_lib, dg, words, q, r_bits, bm.to_numpy_words(out_s),
                           int(cs.item()), dg.STREAM_TESTS + 18700 + n)
