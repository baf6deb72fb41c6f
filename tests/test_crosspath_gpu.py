"""Seeded randomized parity across every path, bit-exact against the oracle.

Random pools (ragged r; clustered and scattered inputs, densities
log-uniform in [1e-4, 0.6]; the last third given to ScanCount by their
zeros) and random queries (thresholds including theta = 0 and theta > N,
intervals including count 0, truth tables; repeated ids).  Each query runs
on the dense counter in three kernel shapes, the Looped recurrence,
ScanCount, the run-length form and BM_PATH_AUTO, and all of them once more
as one batch with automatic and explicit paths (run-length ones included)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

N_BITMAPS = 24
ZEROS_FROM = 16  # ids from here on are listed by their zeros


@pytest.fixture(scope="module")
def bm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1402_4073_gb300 as bm
    return bm


def _words(dg, rng, stream, r_bits):
    d = np.exp(np.log(1e-4) + rng.random(N_BITMAPS) * (np.log(0.6) - np.log(1e-4)))
    half = N_BITMAPS // 2
    clustered = dg.runs(stream, r_bits, d[:half], float(rng.choice([8.0, 256.0, 4096.0])))
    scattered = dg.bernoulli(stream + 1, r_bits, d[half:])
    return np.concatenate([clustered, scattered])


def _zeros_of(words, r_bits):
    comp = ~words
    if r_bits % 64:
        comp[:, -1] &= np.uint64((1 << (r_bits % 64)) - 1)
    return comp


def _query(dg, rng):
    n = int(rng.integers(1, 80))
    ids = rng.integers(0, N_BITMAPS, n).astype(np.uint32)
    kind = int(rng.choice([0, 0, 0, 1, 2]))
    if kind == 0:
        return dg.Query(ids, 0, theta=int(rng.integers(0, n + 2)))
    if kind == 1:
        lo, hi = sorted(int(x) for x in rng.integers(0, n + 2, 2))
        return dg.Query(ids, 1, lo=lo, hi=hi)
    return dg.Query(ids, 2, table=dg.table_from_bools(rng.random(n + 1) < 0.4))


def _check(bm, got_out, got_card, want, what):
    assert np.array_equal(bm.to_numpy_words(got_out), want[0]), what
    assert int(got_card.item()) == want[1], what


@pytest.mark.parametrize("case", range(6))
def test_cross_path_random(bm, oracle_lib, dg, case):
    rng = np.random.default_rng(7000 + case)
    r_bits = [64, 1000, 64 * 1500 + 7, 16384 * 5 + 33, (1 << 20) + 5, 3 * 65536][case]
    words = _words(dg, rng, dg.STREAM_TESTS + 30000 + 10 * case, r_bits)
    queries = [_query(dg, rng) for _ in range(10)]
    wants = [oracle_lib.query(words, q, r_bits) for q in queries]
    flat1, offs1 = dg.positions(words[:ZEROS_FROM], r_bits)
    flat0, offs0 = dg.positions(_zeros_of(words[ZEROS_FROM:], r_bits), r_bits)
    with bm.Pool(r_bits, N_BITMAPS) as pool:
        pool.put_dense(words)
        pool.put_positions(flat1, offs1)
        pool.put_positions(flat0, offs0, first_id=ZEROS_FROM, zeros=True)
        pool.put_rle()
        out = pool.empty_words()
        card = torch.full((1,), -1, dtype=torch.int64, device="cuda")

        def run(q, path):
            out.fill_(-1)
            card.fill_(-1)
            bm.query_run(pool, q, out, card, path=path)
            torch.cuda.synchronize()
            pool.status()

        for i, (q, want) in enumerate(zip(queries, wants)):
            for path in (bm.PATH_SPARSE, bm.PATH_RLE, bm.PATH_AUTO):
                run(q, path)
                _check(bm, out, card, want, (case, i, "path", path))
            for shape in ((0, 256, 4, 2, 0, 2), (0, 256, 4, 2, 1, 1), (1, 128, 4, 1, 0, 2)):
                pool.set_dense_config(*shape)
                run(q, bm.PATH_DENSE)
                _check(bm, out, card, want, (case, i, "dense", shape))
            pool.set_looped(3)
            run(q, bm.PATH_DENSE)
            _check(bm, out, card, want, (case, i, "looped"))
            pool.set_looped(0)

        outs = [pool.empty_words() for _ in queries]
        for o in outs:
            o.fill_(-1)
        cards = torch.full((len(queries),), -1, dtype=torch.int64, device="cuda")
        paths = [(bm.PATH_AUTO, bm.PATH_DENSE, bm.PATH_SPARSE, bm.PATH_RLE)[i % 4]
                 for i in range(len(queries))]
        bm.threshold_batch(pool, queries, outs, cards, paths=paths)
        torch.cuda.synchronize()
        pool.status()
        for i, want in enumerate(wants):
            _check(bm, outs[i], cards[i], want, (case, i, "batch"))
