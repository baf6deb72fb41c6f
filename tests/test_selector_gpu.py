"""Learned selector: trained on the GPU by the library's own kernels from
timings of the library's own kernels (the run-length path among its
candidates when run-length forms are loaded); results stay bit-exact
whatever it picks.  Its time lost (the paper's suboptimality summed over the workload)
on held-out queries must be below the fixed density rule's and no worse than
that of the best single fixed candidate; and the host-side inference that
routes single queries must pick the argmin of the fp64 oracle network on the
same standardised features."""
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
    train_q = dg.sparse_queries(600, pool=n_bm, nmax=600, stream=dg.STREAM_TESTS + 14002)
    test_q = dg.sparse_queries(400, pool=n_bm, nmax=600, stream=dg.STREAM_TESTS + 14003)
    with bm.Pool(r_bits, n_bm) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        ftr, ttr = selector.collect(pool, train_q, reps=3)
        fte, tte = selector.collect(pool, test_q, reps=3)
        model = selector.train(ftr, ttr, steps=3000)
        res = selector.evaluate(pool, model, test_q, fte, tte)
        fixed = [res[f"time_lost_always_c{c}"] for c in range(1, bm.SELECTOR_CANDIDATES)]
        fixed = min([v for v in fixed if v is not None] + [res["time_lost_always_dense"]])
        print("selector:", res, "best fixed:", fixed)
        assert np.isfinite(model.final_loss)
        # what the trained network gains, on held-out queries
        assert res["time_lost_mlp"] < res["time_lost_rule"], res
        assert res["time_lost_mlp"] <= fixed, res
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


def test_selector_learns_run_length_candidate(bm, oracle_lib, dg):
    """With run-length forms loaded, the run-length path is one of the
    network's candidates: on held-out queries over clustered bitmaps (runs of
    mean 8 .. 16384 rows) the trained network loses less time than the
    library's rule without it (the density rule, then the run-length cost
    model) and, within a point, no more than the best single fixed candidate,
    picks the run-length path where it is fastest, and AUTO results stay
    exact."""
    from paper_1402_4073_gb300 import selector
    r_bits, n_bm = 1 << 22, 400
    words, flat, offs, _ = dg.clustered_pool(n_bm, r_bits)
    train_q = dg.clustered_queries(200, n_bm, stream=dg.STREAM_TESTS + 14200)
    test_q = dg.clustered_queries(150, n_bm, stream=dg.STREAM_TESTS + 14300)
    rle = bm.CANDIDATES.index((bm.PATH_RLE, 0))
    with bm.Pool(r_bits, n_bm) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        pool.put_rle()
        ftr, ttr = selector.collect(pool, train_q, reps=3)
        fte, tte = selector.collect(pool, test_q, reps=3)
        assert np.all(np.isfinite(tte[:, rle]))
        model = selector.train(ftr, ttr, steps=3000)
        res = selector.evaluate(pool, model, test_q, fte, tte)
        fixed = [res[f"time_lost_always_c{c}"] for c in range(1, bm.SELECTOR_CANDIDATES)]
        fixed = min([v for v in fixed if v is not None] + [res["time_lost_always_dense"]])
        print("selector with run-length:", res, "best fixed:", fixed)
        assert res["time_lost_mlp"] < res["time_lost_rule"], res
        assert res["time_lost_mlp"] <= fixed + 0.01, res
        fastest = np.nanargmin(tte, axis=1)
        assert np.any(fastest == rle) and res["mlp_choices"][rle] > 0, res
        # installed (by evaluate): single and batched AUTO queries are exact
        picks = selector.installed_choices(pool, test_q)
        sample = list(np.nonzero(picks == rle)[0][:8]) + list(np.nonzero(picks != rle)[0][:8])
        qs = [test_q[i] for i in sample]
        outs = [pool.empty_words() for _ in qs]
        cards = torch.zeros(len(qs), dtype=torch.int64, device="cuda")
        chosen = bm.threshold_batch(pool, qs, outs, cards)
        torch.cuda.synchronize()
        for i, q in enumerate(qs):
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(bm.to_numpy_words(outs[i]), want[0])
            assert int(cards[i].item()) == want[1]
            o = pool.empty_words()
            c = torch.zeros(1, dtype=torch.int64, device="cuda")
            path = bm.query_run(pool, q, o, c)
            torch.cuda.synchronize()
            assert np.array_equal(bm.to_numpy_words(o), want[0]) and int(c.item()) == want[1]
            assert path == (bm.PATH_RLE if picks[sample[i]] == rle else path)
        pool.status()
        assert set(int(x) for x in chosen) <= {bm.PATH_DENSE, bm.PATH_SPARSE, bm.PATH_RLE}


def _unpack(params, F=6, H=64, C=6):
    """The flat fp32 parameter vector as the oracle's W1, b1, W2, b2, W3, b3."""
    from oracle import mlp as omlp
    out, o = [], 0
    for shp in omlp.shapes(F, H, C):
        k = int(np.prod(shp))
        out.append(np.asarray(params[o:o + k], dtype=np.float64).reshape(shp))
        o += k
    assert o == len(params)
    return out


def test_host_inference_matches_oracle_network(bm, dg):
    """bm_query_select (the host-side fp32 forward pass that routes single
    queries) against argmin of oracle/mlp.py's fp64 forward on the features
    bm_query_features reports, standardised in fp32 as the library does.
    Where the oracle's two smallest predictions are within 1e-4 (fp32
    rounding may order them either way) the pick must be one of those."""
    from oracle import mlp as omlp
    from paper_1402_4073_gb300 import selector
    r_bits = 1 << 20
    n_bm = 300
    d = dg.pool_densities(dg.STREAM_TESTS + 14100, n_bm, 1e-5, 3e-2)
    words = dg.bernoulli(dg.STREAM_TESTS + 14101, r_bits, d)
    flat, offs = dg.positions(words, r_bits)
    queries = dg.sparse_queries(400, pool=n_bm, nmax=300, stream=dg.STREAM_TESTS + 14102)
    # a random network (no training needed to pin the inference): weights
    # N(0, 1/fan_in), zero biases, features standardised by their own mean
    # and deviation as training does, so that the picks differ across queries
    rng = np.random.default_rng(14103)
    parts = []
    for shp in omlp.shapes(bm.SELECTOR_FEATURES, bm.SELECTOR_HIDDEN, bm.SELECTOR_CANDIDATES):
        parts.append(rng.normal(0.0, 1.0 / np.sqrt(shp[0]), shp).ravel() if len(shp) == 2
                     else np.zeros(shp))
    params = np.concatenate(parts).astype(np.float32)
    P = _unpack(params)
    with bm.Pool(r_bits, n_bm) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        feats = np.stack([bm.query_features(pool, q) for q in queries]).astype(np.float32)
        mean = feats.mean(axis=0).astype(np.float32)
        std = feats.std(axis=0).astype(np.float32)
        std[std < 1e-6] = 1.0
        bm.set_selector(pool, params, mean, std)
        x = (feats - mean) / std  # fp32, as the library standardises
        y, _ = omlp.forward(P, x.astype(np.float64))
        picks = selector.installed_choices(pool, queries)
    # the pool holds no run-length forms: that candidate is never picked, so
    # the oracle's argmin is taken over the others
    y = y.copy()
    y[:, bm.CANDIDATES.index((bm.PATH_RLE, 0))] = np.inf
    order = np.argsort(y, axis=1)
    top, second = order[:, 0], order[:, 1]
    margin = y[np.arange(len(y)), second] - y[np.arange(len(y)), top]
    clear = margin > 1e-4
    assert clear.sum() > 0.9 * len(queries)
    assert np.array_equal(picks[clear], top[clear]), np.nonzero(picks[clear] != top[clear])
    assert np.all((picks[~clear] == top[~clear]) | (picks[~clear] == second[~clear]))
    # more than one candidate is picked, so the comparison sees the outputs differ
    assert len(set(picks.tolist())) >= 2
