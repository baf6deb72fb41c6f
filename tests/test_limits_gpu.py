"""Edge sizes of the C ABI: the largest row count (r = 2^32, including the
very last row) and the largest query (n = BM_N_MAX = 65535 inputs, 17
counter planes, 16-bit ScanCount counters holding the full count), both
paths, against the oracle; n = BM_N_MAX + 1 is refused."""
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


_POP8 = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)


def _popcount(words: np.ndarray) -> int:
    b = words.view(np.uint8)
    return sum(int(_POP8[b[i:i + (1 << 24)]].sum(dtype=np.uint64)) for i in range(0, b.size, 1 << 24))


def _run(bm, pool, q, path):
    o = pool.empty_words()
    o.fill_(-1)
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    bm.query_run(pool, q, o, c, path=path)
    torch.cuda.synchronize()
    pool.status()
    return bm.to_numpy_words(o), int(c.item())


def test_max_rows(bm, oracle_lib, dg):
    r_bits = 1 << 32
    words = dg.bernoulli(dg.STREAM_TESTS + 19000, r_bits, np.array([2e-4, 1e-4, 3e-4]))
    last = np.uint64(1) << np.uint64(63)
    words[:, -1] |= last          # row 2^32 - 1 set in every bitmap
    words[0, 0] |= np.uint64(1)   # row 0 in one
    flat, offs = dg.positions(words, r_bits)
    assert flat[offs[1] - 1] == r_bits - 1
    nw = words.shape[1]
    with bm.Pool(r_bits, 3) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        for theta in (1, 2, 3):
            q = dg.Query(np.array([0, 1, 2]), 0, theta=theta)
            got = {p: _run(bm, pool, q, p) for p in (bm.PATH_DENSE, bm.PATH_SPARSE)}
            assert np.array_equal(got[bm.PATH_DENSE][0], got[bm.PATH_SPARSE][0])
            assert got[bm.PATH_DENSE][1] == got[bm.PATH_SPARSE][1]
            w, c = got[bm.PATH_DENSE]
            assert c == _popcount(w)
            assert (int(w[-1]) >> 63) & 1 == 1  # the last row is set everywhere
            for w0 in (0, nw // 3, nw - 64):
                want, _ = oracle_lib.query(words, q, r_bits, w0, w0 + 64)
                assert np.array_equal(w[w0:w0 + 64], want), (theta, w0)


def test_max_inputs(bm, oracle_lib, dg):
    r_bits = 4096 + 13
    n_pool = 40
    words = dg.bernoulli(dg.STREAM_TESTS + 19100, r_bits, np.linspace(0.02, 0.98, n_pool))
    words[:, 3] = np.uint64(0xFFFFFFFFFFFFFFFF)  # rows whose count reaches n
    flat, offs = dg.positions(words, r_bits)
    n = bm.BM_N_MAX
    ids = (np.arange(n) % n_pool).astype(np.uint32)
    with bm.Pool(r_bits, n_pool) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        for theta in (1, n // 2, n - 1, n):
            q = dg.Query(ids, 0, theta=theta)
            want = oracle_lib.query(words, q, r_bits)
            assert want[1] > 0
            for path in (bm.PATH_DENSE, bm.PATH_SPARSE):
                got = _run(bm, pool, q, path)
                assert np.array_equal(got[0], want[0]) and got[1] == want[1], (theta, path)
        f = np.zeros(n + 1, bool)
        f[n // 3:n // 3 + 5000] = True
        f[n] = True
        q = dg.Query(ids, 2, table=dg.table_from_bools(f))
        want = oracle_lib.query(words, q, r_bits)
        for path in (bm.PATH_DENSE, bm.PATH_SPARSE):
            got = _run(bm, pool, q, path)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], path
        out = pool.empty_words()
        with pytest.raises(bm.BMError) as e:
            bm.threshold(pool, np.zeros(n + 1, np.uint32), 1, out)
        assert e.value.code == bm.BM_EINVAL
