"""Autotuner: picks a shape for each kernel by measurement, caches it per
GPU model and pool shape, and never changes a result."""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_autotune_installs_and_caches(oracle_lib, dg, tmp_path):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1402_4073_gb300 as bm
    r_bits = (1 << 20) + 3
    d = dg.pool_densities(dg.STREAM_TESTS + 16000, 300, 1e-4, 0.3)
    words = dg.bernoulli(dg.STREAM_TESTS + 16001, r_bits, d)
    flat, offs = dg.positions(words, r_bits)
    cache = str(tmp_path / "tune.txt")
    queries = dg._queries(dg.STREAM_TESTS + 16002, 12, 300, 3, 300, None, 0.2)
    with bm.Pool(r_bits, 300) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        rep = pool.autotune(cache)
        assert "dense=" in rep and "sparse=" in rep and "batch=" in rep, rep
        assert os.path.exists(cache) and open(cache).read().count("dense=") == 1
        cfg = pool.configs()
        # a second pool of the same shape reuses the cached choice
        with bm.Pool(r_bits, 300) as p2:
            p2.put_dense(words[:5])
            p2.put_positions(flat, offs)
            rep2 = p2.autotune(cache)
            assert rep2.startswith("cached"), rep2
            assert p2.configs() == cfg
        for q in queries:
            want = oracle_lib.query(words, q, r_bits)
            for path in (bm.PATH_DENSE, bm.PATH_SPARSE):
                o = pool.empty_words()
                c = torch.zeros(1, dtype=torch.int64, device="cuda")
                bm.query_run(pool, q, o, c, path=path)
                torch.cuda.synchronize()
                assert np.array_equal(bm.to_numpy_words(o), want[0]) and int(c.item()) == want[1]
        outs = [pool.empty_words() for _ in queries]
        cards = torch.zeros(len(queries), dtype=torch.int64, device="cuda")
        bm.threshold_batch(pool, queries, outs, cards)
        torch.cuda.synchronize()
        for i, q in enumerate(queries):
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(bm.to_numpy_words(outs[i]), want[0])
            assert int(cards[i].item()) == want[1]
