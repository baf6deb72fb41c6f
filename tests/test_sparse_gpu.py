"""GPU parity of the ScanCount kernel over sorted position lists, and of the
single-query path choice, against the CPU oracle (bit-exact)."""
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


def _run(bm, pool, q, path):
    out = pool.empty_words()
    out.fill_(-1)
    card = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    chosen = bm.query_run(pool, q, out, card, path=path)
    torch.cuda.synchronize()
    pool.status()
    return (bm.to_numpy_words(out), int(card.item())), chosen


def _eq(got, want, what=""):
    assert np.array_equal(got[0], want[0]), f"{what}: words differ"
    assert got[1] == want[1], f"{what}: card {got[1]} != {want[1]}"


def _pool(bm, dg, r_bits, dens, stream, lists=True):
    words = dg.bernoulli(stream, r_bits, dens)
    flat, offs = dg.positions(words, r_bits)
    pool = bm.Pool(r_bits, words.shape[0])
    pool.put_dense(words)
    if lists:
        pool.put_positions(flat, offs)
    return pool, words, flat, offs


@pytest.mark.parametrize("tile", [8192, 16384, 32768, 65536])
@pytest.mark.parametrize("r_bits", [1, 100, 8192, 8193, 65536 * 3 + 77, 1 << 20])
def test_scancount_tiles_and_ragged_rows(bm, oracle_lib, dg, tile, r_bits):
    dens = np.array([1e-3, 1e-2, 0.05, 0.3, 0.0, 1.0, 2e-3, 0.5])
    pool, words, flat, offs = _pool(bm, dg, r_bits, dens, dg.STREAM_TESTS + 11000)
    with pool:
        pool.set_sparse_config(tile, 512, 2)
        ids = np.array([0, 1, 2, 3, 4, 5, 6, 7, 2, 2], dtype=np.uint32)  # repeats
        for theta in (0, 1, 2, 3, 5, 10, 11):
            q = dg.Query(ids, 0, theta=theta)
            got, path = _run(bm, pool, q, bm.PATH_SPARSE)
            assert path == bm.PATH_SPARSE
            _eq(got, oracle_lib.scancount(flat, offs, ids, r_bits, theta), f"theta={theta}")
            _eq(got, oracle_lib.query(words, q, r_bits), f"dense view theta={theta}")
        q = dg.Query(ids, 1, lo=2, hi=4)
        got, _ = _run(bm, pool, q, bm.PATH_SPARSE)
        _eq(got, oracle_lib.query(words, q, r_bits), "interval")


@pytest.mark.parametrize("shape", [(32768, 512, 2, 2), (32768, 256, 2, 4), (16384, 256, 4, 2),
                                   (65536, 512, 1, 2), (8192, 64, 8, 4), (65536, 96, 1, 4)])
def test_scancount_kernel_shapes(bm, oracle_lib, dg, shape):
    """Every shape the autotuner may pick (tile rows, threads, CTAs/SM,
    pieces per load batch) gives the same exact result, for both counter
    widths and a table predicate, with groups that leave warps idle
    (n < 32 per warp) and groups that span several pieces."""
    r_bits = 3 * 65536 + 4099
    pool_n = 400
    dens = dg.log_uniform(dg.uniform(dg.STREAM_TESTS + 11150, pool_n), 1e-4, 5e-2)
    words = dg.bernoulli(dg.STREAM_TESTS + 11151, r_bits, dens)
    flat, offs = dg.positions(words, r_bits)
    with bm.Pool(r_bits, pool_n) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        pool.set_sparse_config(*shape)
        for n in (3, 40, 255, 256, 400, 1000):
            ids = (np.arange(n) * 7 % pool_n).astype(np.uint32)
            for q in (dg.Query(ids, 0, theta=max(1, n // 50)),
                      dg.Query(ids, 1, lo=2, hi=max(2, n // 20))):
                got, _ = _run(bm, pool, q, bm.PATH_SPARSE)
                _eq(got, oracle_lib.query(words, q, r_bits), f"shape={shape} n={n} kind={q.kind}")


@pytest.mark.parametrize("N", [2, 255, 256, 300, 4096])
def test_scancount_counter_width(bm, oracle_lib, dg, N):
    """8-bit counters up to N = 255, 16-bit above; planted rows reach count N."""
    r_bits = 1 << 17
    pool_n = min(N, 600)
    dens = dg.log_uniform(dg.uniform(dg.STREAM_TESTS + 11100, pool_n), 1e-4, 2e-2)
    words = dg.bernoulli(dg.STREAM_TESTS + 11101, r_bits, dens)
    words[:, 5] |= np.uint64(0xF0F0)  # rows where every input is set
    ids = (np.arange(N) % pool_n).astype(np.uint32)
    flat, offs = dg.positions(words, r_bits)
    with bm.Pool(r_bits, pool_n) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        for theta in (1, 2, N // 2, N - 1, N, N + 1):
            q = dg.Query(ids, 0, theta=max(theta, 0))
            got, _ = _run(bm, pool, q, bm.PATH_SPARSE)
            want = oracle_lib.query(words, q, r_bits)
            _eq(got, want, f"N={N} theta={theta}")
        f = np.zeros(N + 1, bool)
        f[::3] = True
        f[N] = True
        q = dg.Query(ids, 2, table=dg.table_from_bools(f))
        got, _ = _run(bm, pool, q, bm.PATH_SPARSE)
        _eq(got, oracle_lib.query(words, q, r_bits), "table")


def test_sparse_workload_subset(bm, oracle_lib, dg):
    """Scaled sparse workload: 300 bitmaps, r = 2^20, densities log-uniform in
    [1e-5, 1e-2], queries with N log-uniform in [2, 300], theta <= min(N, 64),
    on every path, against the oracle."""
    r_bits = 1 << 20
    d = dg.pool_densities(dg.STREAM_TESTS + 11200, 300, 1e-5, 1e-2)
    words = dg.bernoulli(dg.STREAM_TESTS + 11201, r_bits, d)
    flat, offs = dg.positions(words, r_bits)
    queries = dg.sparse_queries(12, pool=300, nmax=300, stream=dg.STREAM_TESTS + 11202)
    with bm.Pool(r_bits, 300) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        for q in queries:
            want = oracle_lib.query(words, q, r_bits)
            for path in (bm.PATH_DENSE, bm.PATH_SPARSE, bm.PATH_AUTO):
                got, chosen = _run(bm, pool, q, path)
                _eq(got, want, f"n={q.n} path={path}")
                assert chosen in (bm.PATH_DENSE, bm.PATH_SPARSE)


def _lists_to_words(lists, r_bits):
    words = np.zeros((len(lists), (r_bits + 63) // 64), dtype=np.uint64)
    for k, l in enumerate(lists):
        for x in l:
            words[k, x // 64] |= np.uint64(1) << np.uint64(x % 64)
    return words


def _flat(lists):
    offs = np.zeros(len(lists) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(l) for l in lists])
    flat = np.concatenate([np.asarray(l, dtype=np.uint32) for l in lists]) if offs[-1] else \
        np.zeros(0, np.uint32)
    return flat, offs


@pytest.mark.parametrize("tile", [8192, 16384, 32768, 65536])
def test_list_padding_and_alignment(bm, oracle_lib, dg, tile):
    """Lists of every length mod 4, last positions just below and above 65536,
    slices that cross tile and index boundaries, an empty list, the last row;
    loaded in several calls (host and device, one list replaced): the pool's
    16-byte alignment and padding never add or drop a count."""
    r_bits = 3 * 65536 + 5000
    rng = dg.uniform(dg.STREAM_TESTS + 11050, 4000)
    rand = np.unique((rng * r_bits).astype(np.uint64)).astype(np.uint32)
    lists = [
        [65535],
        [65536],
        [0, 1, 2, 3, 4],
        [65533, 65534, 65535, 65536, 65537, 65538],
        [],
        [r_bits - 1],
        list(rand[: 4 * (len(rand) // 4) - 1]),
        [8191, 8192, 16383, 16384, 32767, 32768],
        [65532, 65533, 65534],
        [131071, 131072, 131073],
    ]
    replaced = [7, 65535, 65536, 131072, r_bits - 2]
    with bm.Pool(r_bits, len(lists)) as pool:
        f0, o0 = _flat(lists[:4])
        pool.put_positions(f0, o0)
        f1, o1 = _flat(lists[4:8])
        pool.put_positions(torch.from_numpy(f1.view(np.int32).copy()).cuda(), o1, first_id=4)
        f2, o2 = _flat(lists[8:])
        pool.put_positions(f2, o2, first_id=8)
        f3, o3 = _flat([replaced])
        pool.put_positions(f3, o3, first_id=2)  # appended; the old copy stays unused
        lists[2] = replaced
        flat, offs = _flat(lists)
        words = _lists_to_words(lists, r_bits)
        pool.put_dense(words)
        pool.set_sparse_config(tile, 512, 2)
        ids = np.array(list(range(len(lists))) + [0, 3, 3, 9], dtype=np.uint32)
        for theta in (1, 2, 3, 4):
            q = dg.Query(ids, 0, theta=theta)
            got, _ = _run(bm, pool, q, bm.PATH_SPARSE)
            _eq(got, oracle_lib.scancount(flat, offs, ids, r_bits, theta), f"theta={theta}")
            _eq(got, oracle_lib.query(words, q, r_bits), f"dense view theta={theta}")
        for k in range(len(lists)):  # each list alone reproduces its bitmap
            q = dg.Query(np.array([k]), 0, theta=1)
            got, _ = _run(bm, pool, q, bm.PATH_SPARSE)
            assert np.array_equal(got[0], words[k]) and got[1] == len(lists[k]), k


def _zeros_of(words: np.ndarray, r_bits: int) -> np.ndarray:
    comp = ~words
    if r_bits % 64:
        comp[:, -1] &= np.uint64((1 << (r_bits % 64)) - 1)
    return comp


@pytest.mark.parametrize("tile", [8192, 32768, 65536])
@pytest.mark.parametrize("r_bits", [70001, (1 << 18) + 3])
def test_lists_of_zeros(bm, oracle_lib, dg, tile, r_bits):
    """Dense inputs given to ScanCount by their zeros (the complement
    identity, input by input), mixed with inputs given by their ones, in
    single and batched queries, with 8- and 16-bit counters: every result
    equals the oracle on the dense view."""
    lo_d = dg.log_uniform(dg.uniform(dg.STREAM_TESTS + 11500, 30), 1e-4, 0.1)
    hi_d = 1.0 - dg.log_uniform(dg.uniform(dg.STREAM_TESTS + 11501, 30), 1e-4, 0.1)
    words = dg.bernoulli(dg.STREAM_TESTS + 11502, r_bits, np.concatenate([lo_d, hi_d]))
    nw = words.shape[1]
    ones = np.full((1, nw), np.uint64(0xFFFFFFFFFFFFFFFF))
    ones[0, -1] = np.uint64((1 << (r_bits % 64)) - 1) if r_bits % 64 else ones[0, -1]
    words = np.concatenate([words, ones])  # id 60: all ones (an empty list of zeros)
    words[:, 17] |= np.uint64(0xF0)        # rows every input holds
    flat1, offs1 = dg.positions(words[:30], r_bits)
    flat0, offs0 = dg.positions(_zeros_of(words[30:], r_bits), r_bits)
    n_bm = words.shape[0]
    with bm.Pool(r_bits, n_bm) as pool:
        pool.put_dense(words)
        pool.put_positions(flat1, offs1)
        pool.put_positions(flat0, offs0, first_id=30, zeros=True)
        pool.set_sparse_config(tile, 512, 2)
        for k in (0, 29, 30, 59, 60):
            assert pool.bitmap_cardinality(k) == oracle_lib.cardinality(words[k], r_bits)
        small = np.array([0, 31, 5, 60, 45, 45, 12, 59, 2, 33], dtype=np.uint32)
        big = (np.arange(400) * 7 % n_bm).astype(np.uint32)  # 16-bit counters, repeats
        queries = []
        for ids in (small, big):
            n = len(ids)
            for theta in (1, 2, n // 3, n // 2, n - 1, n):
                queries.append(dg.Query(ids, 0, theta=theta))
            queries.append(dg.Query(ids, 1, lo=n // 4, hi=n // 2))
            f = (np.arange(n + 1) % 3 == 0)
            queries.append(dg.Query(ids, 2, table=dg.table_from_bools(f)))
        wants = [oracle_lib.query(words, q, r_bits) for q in queries]
        for q, want in zip(queries, wants):
            got, _ = _run(bm, pool, q, bm.PATH_SPARSE)
            _eq(got, want, f"n={q.n} kind={q.kind} theta={q.theta}")
        outs = [pool.empty_words().fill_(-1) for _ in queries]
        cards = torch.full((len(queries),), -1, dtype=torch.int64, device="cuda")
        bm.threshold_batch(pool, queries, outs, cards, paths=[bm.PATH_SPARSE] * len(queries))
        torch.cuda.synchronize()
        pool.status()
        for i, want in enumerate(wants):
            _eq((bm.to_numpy_words(outs[i]), int(cards[i].item())), want, f"batch query {i}")


def test_lists_from_device_and_validation(bm, dg):
    r_bits = 50000
    words = dg.bernoulli(dg.STREAM_TESTS + 11300, r_bits, np.array([0.01, 0.02, 0.03]))
    flat, offs = dg.positions(words, r_bits)
    with bm.Pool(r_bits, 4) as pool:
        pool.put_dense(words)
        pool.put_positions(torch.from_numpy(flat.view(np.int32)).cuda(), offs)
        assert pool.info()["lists_loaded"] == 3
        q = dg.Query(np.array([0, 1, 2]), 0, theta=1)
        out = pool.empty_words()
        bm.query_run(pool, q, out, path=bm.PATH_SPARSE)
        a = bm.to_numpy_words(out)
        assert np.array_equal(a, words[0] | words[1] | words[2])
        # id 3 has no list: the sparse path is refused, AUTO uses dense (absent too -> error)
        with pytest.raises(bm.BMError) as e:
            bm.query_run(pool, dg.Query(np.array([0, 3]), 0, theta=1), out, path=bm.PATH_SPARSE)
        assert e.value.code == bm.BM_ERANGE
        # unsorted or out-of-range lists are refused (host and device input)
        bad = np.array([5, 3], dtype=np.uint32)
        with pytest.raises(bm.BMError):
            pool.put_positions(bad, np.array([0, 2]), first_id=3)
        with pytest.raises(bm.BMError):
            pool.put_positions(torch.tensor([1, r_bits], dtype=torch.int32, device="cuda"),
                               np.array([0, 2]), first_id=3)
        with pytest.raises(bm.BMError):
            pool.set_sparse_config(10000, 512, 2)


def test_auto_rule_picks_sparse_for_sparse_inputs(bm, dg):
    r_bits = 1 << 20
    words = dg.bernoulli(dg.STREAM_TESTS + 11400, r_bits, np.array([1e-4] * 8 + [0.4] * 8))
    flat, offs = dg.positions(words, r_bits)
    with bm.Pool(r_bits, 16) as pool:
        pool.put_dense(words)
        pool.put_positions(flat, offs)
        assert bm.query_select(pool, dg.Query(np.arange(8), 0, theta=2))[0] == bm.PATH_SPARSE
        assert bm.query_select(pool, dg.Query(np.arange(8, 16), 0, theta=2))[0] == bm.PATH_DENSE
