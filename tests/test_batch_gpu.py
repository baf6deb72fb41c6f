"""Batched queries: every result of a batch equals the same query run alone
and the CPU oracle, bit-exactly, whatever path each query takes."""
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


@pytest.fixture(scope="module")
def mixed(dg):
    """Scaled mixed workload: 200 bitmaps of r = 2^18 + 77 rows, densities
    log-uniform in [1e-4, 0.5]; 96 queries, N log-uniform in [3, 200]."""
    r_bits = (1 << 18) + 77
    d = dg.pool_densities(dg.STREAM_TESTS + 12000, 200, 1e-4, 0.5)
    words = dg.bernoulli(dg.STREAM_TESTS + 12001, r_bits, d)
    flat, offs = dg.positions(words, r_bits)
    queries = dg._queries(dg.STREAM_TESTS + 12002, 96, 200, 3, 200, None, 0.1)
    # a few truth-table queries with many transitions, and repeated ids
    for j in range(0, 96, 16):
        n = queries[j].n
        f = (np.arange(n + 1) % 3 == 1)
        queries[j] = dg.Query(np.concatenate([queries[j].ids, queries[j].ids[:2]]), 2,
                              table=dg.table_from_bools(np.append(f, [True, False])))
    return r_bits, words, flat, offs, queries


def _batch(bm, pool, queries, paths=None):
    outs = [pool.empty_words().fill_(-1) for _ in queries]
    cards = torch.full((len(queries),), -1, dtype=torch.int64, device="cuda")
    chosen = bm.threshold_batch(pool, queries, outs, cards, paths)
    torch.cuda.synchronize()
    pool.status()
    return [bm.to_numpy_words(o) for o in outs], cards.cpu().numpy(), chosen


@pytest.mark.parametrize("batch_cfg", [(2, 0, 2), (1, 0, 2), (2, 1, 2), (2, 0, 1), (1, 1, 1),
                                       (2, 2, 2), (2, 2, 1), (3, 0, 1)])
def test_batch_matches_oracle(bm, oracle_lib, dg, mixed, batch_cfg):
    r_bits, words, flat, offs, queries = mixed
    with bm.Pool(r_bits, words.shape[0]) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        pool.set_batch_config(*batch_cfg)
        # alternate forced paths, plus AUTO (density rule)
        paths = [(bm.PATH_AUTO, bm.PATH_DENSE, bm.PATH_SPARSE)[i % 3] for i in range(len(queries))]
        outs, cards, chosen = _batch(bm, pool, queries, paths)
        for i, q in enumerate(queries):
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(outs[i], want[0]), f"query {i} (n={q.n}, path {chosen[i]})"
            assert cards[i] == want[1], f"query {i} card"
            if paths[i] != bm.PATH_AUTO:
                assert chosen[i] == paths[i]


def test_batch_equals_alone_and_repeats(bm, dg, mixed):
    r_bits, words, flat, offs, queries = mixed
    with bm.Pool(r_bits, words.shape[0]) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        outs, cards, chosen = _batch(bm, pool, queries)
        for i, q in enumerate(queries):
            o = pool.empty_words()
            c = torch.zeros(1, dtype=torch.int64, device="cuda")
            bm.query_run(pool, q, o, c, path=int(chosen[i]))
            torch.cuda.synchronize()
            assert np.array_equal(bm.to_numpy_words(o), outs[i])
            assert int(c.item()) == cards[i]
        # the same batch again (graph replay) and several batches in flight
        s = torch.cuda.Stream()
        runs = []
        for k in range(4):
            sub = queries[k * 20:(k + 1) * 20]
            o = [pool.empty_words() for _ in sub]
            c = torch.zeros(len(sub), dtype=torch.int64, device="cuda")
            bm.threshold_batch(pool, sub, o, c, stream=s)
            runs.append((k, o, c))
        torch.cuda.synchronize()
        for k, o, c in runs:
            for j in range(len(o)):
                assert np.array_equal(bm.to_numpy_words(o[j]), outs[k * 20 + j])
                assert int(c[j].item()) == cards[k * 20 + j]


@pytest.mark.parametrize("tile", [8192, 16384, 32768, 65536])
def test_batch_sparse_counter_widths_interleaved(bm, oracle_lib, dg, tile):
    """One batch of ScanCount items with 8-bit (n <= 255) and 16-bit (n > 255)
    counters interleaved, so CTAs go from one width to the other: counters
    and spare words left by one item never leak into the next.  Run twice."""
    r_bits = (1 << 18) + 77
    n_bm = 1300
    d = dg.pool_densities(dg.STREAM_TESTS + 12200, n_bm, 1e-4, 2e-2)
    words = dg.bernoulli(dg.STREAM_TESTS + 12201, r_bits, d)
    words[:, 7] |= np.uint64(0xFF00)  # rows where every input is set
    flat, offs = dg.positions(words, r_bits)
    small = dg._queries(dg.STREAM_TESTS + 12202, 20, n_bm, 2, 255, 40, 0.2)
    large = dg._queries(dg.STREAM_TESTS + 12203, 20, n_bm, 256, n_bm, 300, 0.2)
    queries = [q for pair in zip(small, large) for q in pair]
    with bm.Pool(r_bits, n_bm) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        pool.set_sparse_config(tile, 512, 2)
        want = [oracle_lib.query(words, q, r_bits) for q in queries]
        for rep in range(2):
            outs, cards, chosen = _batch(bm, pool, queries, [bm.PATH_SPARSE] * len(queries))
            assert all(c == bm.PATH_SPARSE for c in chosen)
            for i, q in enumerate(queries):
                assert np.array_equal(outs[i], want[i][0]), f"rep {rep} query {i} (n={q.n})"
                assert cards[i] == want[i][1], f"rep {rep} query {i} card"


def test_batch_single_query_and_errors(bm, oracle_lib, dg):
    r_bits = 70000
    words = dg.bernoulli(dg.STREAM_TESTS + 12100, r_bits, np.full(10, 0.3))
    with bm.Pool(r_bits, 10) as pool:
        pool.put_dense(words)
        q = dg.Query(np.arange(10), 0, theta=4)
        outs, cards, chosen = _batch(bm, pool, [q])
        want = oracle_lib.query(words, q, r_bits)
        assert np.array_equal(outs[0], want[0]) and cards[0] == want[1]
        assert chosen[0] == bm.PATH_DENSE  # no lists: the rule must pick dense
        o = [pool.empty_words()]
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        with pytest.raises(bm.BMError):
            bm.threshold_batch(pool, [dg.Query(np.array([0, 11]), 0, theta=1)], o, c)
        with pytest.raises(bm.BMError):
            bm.threshold_batch(pool, [q], o, c, paths=[bm.PATH_SPARSE])  # no lists loaded
