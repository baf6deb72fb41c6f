"""Learned selector: trained on the GPU by the library's own kernels from
timings of the library's own kernels; results stay bit-exact whatever it
picks; its time lost is compared with the fixed density rule's."""
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


def test_selector_trains_routes_and_stays_exact(bm, oracle_lib, dg):
    from paper_1402_4073_gb300 import selector
    r_bits = 1 << 21
    n_bm = 600
    d = dg.pool_densities(dg.STREAM_TESTS + 14000, n_bm, 1e-5, 3e-2)
    words = dg.bernoulli(dg.STREAM_TESTS + 14001, r_bits, d)
    flat, offs = dg.positions(words, r_bits)
    train_q = dg.sparse_queries(160, pool=n_bm, nmax=600, stream=dg.STREAM_TESTS + 14002)
    test_q = dg.sparse_queries(80, pool=n_bm, nmax=600, stream=dg.STREAM_TESTS + 14003)
    with bm.Pool(r_bits, n_bm) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        ftr, ttr = selector.collect(pool, train_q, reps=3)
        fte, tte = selector.collect(pool, test_q, reps=3)
        model = selector.train(ftr, ttr, steps=1500)
        res = selector.evaluate(pool, model, test_q, fte, tte)
        print("selector:", res)
        assert np.isfinite(model.final_loss)
        assert res["time_lost_mlp"] <= res["time_lost_always_dense"] + 1e-9
        assert res["time_lost_mlp"] <= res["time_lost_rule"] + 0.05
        # with the network installed, AUTO results are exact, single and batched
        selector.install(pool, model)
        outs = [pool.empty_words() for _ in test_q[:24]]
        cards = torch.zeros(24, dtype=torch.int64, device="cuda")
        chosen = bm.threshold_batch(pool, test_q[:24], outs, cards)
        torch.cuda.synchronize()
        for i, q in enumerate(test_q[:24]):
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(bm.to_numpy_words(outs[i]), want[0])
            assert int(cards[i].item()) == want[1]
            o = pool.empty_words()
            c = torch.zeros(1, dtype=torch.int64, device="cuda")
            path = bm.query_run(pool, q, o, c)
            torch.cuda.synchronize()
            assert np.array_equal(bm.to_numpy_words(o), want[0]) and int(c.item()) == want[1]
            assert path in (bm.PATH_DENSE, bm.PATH_SPARSE)
        assert set(chosen.tolist()) <= {bm.PATH_DENSE, bm.PATH_SPARSE}
