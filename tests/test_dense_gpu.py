"""GPU parity of the dense bit-sliced counter against the CPU oracle, through
the C ABI.  Integer results: every output word and every cardinality must be
bit-exact."""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

# every feeding variant of the dense kernel: (variant, threads, stages, ctas_per_sm)
# (variant, threads, stages, ctas_per_sm, adder, words_per_thread)
VARIANTS = [(0, 256, 4, 2, 0, 2), (1, 256, 3, 1, 0, 2), (0, 256, 4, 2, 1, 1), (1, 64, 3, 2, 0, 2),
            (1, 128, 2, 1, 0, 2), (0, 256, 4, 3, 1, 2), (0, 256, 4, 2, 0, 1), (1, 128, 4, 1, 0, 2),
            (0, 256, 4, 2, 2, 2)]


@pytest.fixture(scope="module")
def bm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1402_4073_gb300 as bm
    return bm


def _mask(r_bits):
    w = (r_bits + 63) // 64
    m = np.full(w, np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    if r_bits % 64:
        m[-1] = np.uint64((1 << (r_bits % 64)) - 1)
    return m


def run_query(bm, pool, q):
    out = pool.empty_words()
    out.fill_(-1)  # poison: every word must be rewritten
    card = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    if q.kind == 0:
        bm.threshold(pool, q.ids, q.theta, out, card)
    elif q.kind == 1:
        bm.interval(pool, q.ids, q.lo, q.hi, out, card)
    else:
        bm.symmetric(pool, q.ids, q.table, out, card)
    torch.cuda.synchronize()
    pool.status()
    return bm.to_numpy_words(out), int(card.item())


def check_equal(got, want, what=""):
    gw, gc = got
    ww, wc = want
    if not np.array_equal(gw, ww):
        bad = np.nonzero(gw != ww)[0]
        raise AssertionError(f"{what}: {len(bad)} words differ, first at {bad[:5]}")
    assert gc == wc, f"{what}: cardinality {gc} != {wc}"


def make_pool(bm, words, r_bits):
    pool = bm.Pool(r_bits, words.shape[0])
    pool.put_dense(words)
    return pool


@pytest.mark.parametrize("variant", VARIANTS)
def test_config1_all_queries(bm, oracle_lib, dg, variant):
    words, queries = dg.config1()
    r_bits = 1 << 20
    with make_pool(bm, words, r_bits) as pool:
        pool.set_dense_config(*variant)
        for q in queries:
            check_equal(run_query(bm, pool, q), oracle_lib.query(words, q, r_bits), str(q.kind))


@pytest.mark.parametrize("variant", VARIANTS[:2])
@pytest.mark.parametrize("N", [1, 2, 3, 7, 12])
def test_exhaustive_small_n(bm, oracle_lib, N, variant):
    # row i has bit k set iff bit k of i is set: counts are popcount(i)
    r_bits = 1 << N
    rows = np.arange(r_bits)
    bits = ((rows[None, :] >> np.arange(N)[:, None]) & 1).astype(bool)
    if r_bits < 64:
        bits = np.pad(bits, ((0, 0), (0, 64 - r_bits)))
    words = np.packbits(bits, axis=1, bitorder="little").view(np.uint64).copy()
    with make_pool(bm, words, r_bits) as pool:
        pool.set_dense_config(*variant)
        ids = np.arange(N)
        for theta in range(0, N + 2):
            out = pool.empty_words()
            card = torch.zeros(1, dtype=torch.int64, device="cuda")
            bm.threshold(pool, ids, theta, out, card)
            torch.cuda.synchronize()
            assert int(card.item()) == sum(math.comb(N, c) for c in range(theta, N + 1))
            check_equal((bm.to_numpy_words(out), int(card.item())),
                        oracle_lib.threshold(words, ids, r_bits, theta), f"theta={theta}")


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("r_bits", [1, 63, 64, 65, 127, 128, 129, 1000, 4096 + 17, 100003, 300000])
def test_ragged_rows(bm, oracle_lib, dg, r_bits, variant):
    N = 37
    words = dg.bernoulli(dg.STREAM_TESTS + 3000 + r_bits % 1000, r_bits, np.linspace(0.05, 0.9, N))
    words[:, -1] |= ~_mask(r_bits)[-1]  # garbage above r must be ignored
    with make_pool(bm, words, r_bits) as pool:
        pool.set_dense_config(*variant)
        ids = np.arange(N)
        for theta in (0, 1, 2, 18, 36, 37, 38):
            q = dg.Query(ids, 0, theta=theta)
            check_equal(run_query(bm, pool, q), oracle_lib.query(words, q, r_bits), f"theta={theta}")


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("N", [1, 2, 15, 16, 17, 31, 32, 33, 100, 511, 512])
def test_n_sweep_with_repeats(bm, oracle_lib, dg, N, variant):
    r_bits = 64 * 1000 + 40
    pool_n = 64
    words = dg.bernoulli(dg.STREAM_TESTS + 4000, r_bits,
                         dg.log_uniform(dg.uniform(dg.STREAM_TESTS + 4001, pool_n), 0.01, 0.9))
    ids = (dg.uniform(dg.STREAM_TESTS + 4002 + N, N) * pool_n).astype(np.uint32)  # repeats
    with make_pool(bm, words, r_bits) as pool:
        pool.set_dense_config(*variant)
        for theta in sorted({0, 1, 2, max(1, N // 3), max(1, N // 2), N, N + 1}):
            q = dg.Query(ids, 0, theta=theta)
            check_equal(run_query(bm, pool, q), oracle_lib.query(words, q, r_bits),
                        f"N={N} theta={theta}")
        lo, hi = max(0, N // 4), max(0, N // 2)
        q = dg.Query(ids, 1, lo=lo, hi=hi)
        check_equal(run_query(bm, pool, q), oracle_lib.query(words, q, r_bits), "interval")


@pytest.mark.parametrize("variant", VARIANTS[:2])
def test_symmetric_tables(bm, oracle_lib, dg, variant):
    r_bits = 64 * 2048 + 5
    N = 40
    words = dg.bernoulli(dg.STREAM_TESTS + 5000, r_bits, np.full(N, 0.5))
    ids = np.arange(N)
    u = dg.uniform(dg.STREAM_TESTS + 5001, 6 * (N + 1)).reshape(6, N + 1)
    tables = [u[0] < 0.5, u[1] < 0.1, u[2] < 0.9, np.arange(N + 1) % 2 == 1,
              np.arange(N + 1) % 3 == 0, np.zeros(N + 1, bool), np.ones(N + 1, bool),
              (np.arange(N + 1) >= 10) & (np.arange(N + 1) <= 30) | (np.arange(N + 1) == 3)]
    with make_pool(bm, words, r_bits) as pool:
        pool.set_dense_config(*variant)
        for i, f in enumerate(tables):
            q = dg.Query(ids, 2, table=dg.table_from_bools(f))
            check_equal(run_query(bm, pool, q), oracle_lib.query(words, q, r_bits), f"table {i}")


@pytest.mark.parametrize("variant", VARIANTS[:2])
@pytest.mark.parametrize("N", [4096, 9000])
def test_large_n(bm, oracle_lib, dg, N, variant):
    r_bits = 64 * 300 + 9
    pool_n = 600
    words = dg.bernoulli(dg.STREAM_TESTS + 6000, r_bits, np.full(pool_n, 0.3))
    ids = (dg.uniform(dg.STREAM_TESTS + 6001 + N, N) * pool_n).astype(np.uint32)
    with make_pool(bm, words, r_bits) as pool:
        pool.set_dense_config(*variant)
        for theta in (1, int(0.28 * N), int(0.3 * N), int(0.32 * N), N):
            q = dg.Query(ids, 0, theta=theta)
            check_equal(run_query(bm, pool, q), oracle_lib.query(words, q, r_bits), f"theta={theta}")
        f = np.zeros(N + 1, bool)
        f[int(0.29 * N):int(0.31 * N)] = True
        f[::97] = True
        q = dg.Query(ids, 2, table=dg.table_from_bools(f))
        check_equal(run_query(bm, pool, q), oracle_lib.query(words, q, r_bits), "table")


def test_cardinality_entry_point(bm, oracle_lib, dg):
    for r_bits in (1, 64, 65, 100003):
        w = dg.bernoulli(dg.STREAM_TESTS + 7000, r_bits, [0.4])[0]
        w[-1] |= ~_mask(r_bits)[-1]
        t = torch.from_numpy(w.view(np.int64)).cuda()
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        bm.cardinality(t, r_bits, c)
        assert int(c.item()) == oracle_lib.cardinality(w, r_bits)


def test_pool_put_and_errors(bm, dg):
    r_bits = 5000
    words = dg.bernoulli(dg.STREAM_TESTS + 7100, r_bits, np.full(4, 0.5))
    with bm.Pool(r_bits, 8) as pool:
        pool.put_dense(words)
        assert pool.info()["dense_loaded"] == 4
        assert pool.bitmap_cardinality(2) == sum(bin(int(x)).count("1") for x in words[2])
        out = pool.empty_words()
        with pytest.raises(bm.BMError) as e:
            bm.threshold(pool, [0, 5], 1, out)  # id 5 not loaded
        assert e.value.code == bm.BM_ERANGE
        with pytest.raises(bm.BMError) as e:
            bm.threshold(pool, [0, 9], 1, out)  # id >= capacity
        assert e.value.code == bm.BM_ERANGE
        with pytest.raises(bm.BMError) as e:
            bm.threshold(pool, [], 1, out)
        assert e.value.code == bm.BM_EINVAL
        with pytest.raises(bm.BMError):
            pool.set_dense_config(1, 96, 4, 1)
        # device-resident input load gives the same pool contents
        with bm.Pool(r_bits, 4) as p2:
            p2.put_dense(torch.from_numpy(words.view(np.int64)).cuda())
            a, b = pool.empty_words(), p2.empty_words()
            bm.threshold(pool, [0, 1, 2, 3], 2, a)
            bm.threshold(p2, [0, 1, 2, 3], 2, b)
            torch.cuda.synchronize()
            assert torch.equal(a, b)


def test_unaligned_output_buffer(bm, oracle_lib, dg):
    r_bits = 64 * 777 + 3
    words = dg.bernoulli(dg.STREAM_TESTS + 7200, r_bits, np.full(20, 0.3))
    with make_pool(bm, words, r_bits) as pool:
        for variant in VARIANTS:
            pool.set_dense_config(*variant)
            big = torch.zeros(pool.words + 1, dtype=torch.int64, device="cuda")
            out = big[1:]  # 8-byte aligned, not 16
            card = torch.zeros(1, dtype=torch.int64, device="cuda")
            bm.threshold(pool, np.arange(20), 5, out, card)
            torch.cuda.synchronize()
            check_equal((bm.to_numpy_words(out), int(card.item())),
                        oracle_lib.threshold(words, np.arange(20), r_bits, 5), str(variant))
            assert int(big[0].item()) == 0


def test_streams_and_back_to_back_calls(bm, oracle_lib, dg):
    """Many calls in flight on two streams reuse the staging ring safely."""
    r_bits = 64 * 4096
    words = dg.bernoulli(dg.STREAM_TESTS + 7300, r_bits, np.full(50, 0.2))
    with make_pool(bm, words, r_bits) as pool:
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        outs, cards, wants = [], [], []
        for i in range(24):
            n = 3 + i
            ids = np.arange(i, i + n) % 50
            theta = 1 + i % n
            o = pool.empty_words()
            c = torch.zeros(1, dtype=torch.int64, device="cuda")
            bm.threshold(pool, ids, theta, o, c, stream=s1 if i % 2 else s2)
            outs.append(o)
            cards.append(c)
            wants.append(oracle_lib.threshold(words, ids, r_bits, theta))
        torch.cuda.synchronize()
        for o, c, w in zip(outs, cards, wants):
            check_equal((bm.to_numpy_words(o), int(c.item())), w)


# --- full-size large dense workload ------------------------------------------------


@pytest.fixture(scope="module")
def config2(dg):
    words, queries = dg.config2()
    return words, queries


@pytest.fixture(scope="module")
def config2_answers(oracle_lib, config2):
    words, queries = config2
    return [oracle_lib.query(words, q, 1 << 26) for q in queries]


@pytest.mark.parametrize("variant", VARIANTS[:2] + [VARIANTS[8], "tuned"])
def test_config2_full_size(bm, config2, config2_answers, variant):
    """N=256, r=2^26: the whole output bitmap and its cardinality of every
    query, against the oracle run over every word.  "tuned" runs the shape the
    autotuner installs on this pool (the one the benchmark times); VARIANTS[8]
    is the 32-input adder shape, where each thread walks several columns of
    the grid-stride loop at this size."""
    words, queries = config2
    r_bits = 1 << 26
    with make_pool(bm, words, r_bits) as pool:
        if variant == "tuned":
            report = pool.autotune()
            what = f"tuned {pool.configs()['dense']} ({report})"
        else:
            pool.set_dense_config(*variant)
            what = str(variant)
        for q, want in zip(queries, config2_answers):
            got = run_query(bm, pool, q)
            check_equal(got, want, f"{what} kind={q.kind} theta={q.theta}")


def test_config2_full_size_looped(bm, config2, config2_answers):
    """The same queries with the Looped recurrence on (theta = 2 directly,
    theta = 255 through the complement identity; the others stay on the
    counter), against the oracle over every word."""
    words, queries = config2
    with make_pool(bm, words, 1 << 26) as pool:
        pool.set_looped(3)
        for q, want in zip(queries, config2_answers):
            got = run_query(bm, pool, q)
            check_equal(got, want, f"looped kind={q.kind} theta={q.theta}")


def test_config2_planted_rows(bm, oracle_lib, dg, config2):
    """theta = 128 and 255 select nothing on the pure workload; plant rows
    with 100..256 ones so that both thresholds have answers."""
    words, queries = config2
    words = words.copy()
    r_bits = 1 << 26
    u = dg.uniform(dg.STREAM_TESTS + 8000, 3 * 4000).reshape(3, 4000)
    rows = (u[0] * r_bits).astype(np.int64)
    ks = (100 + u[1] * 157).astype(np.int64)
    for row, k in zip(rows, ks):
        sel = dg.floyd(dg.STREAM_TESTS + 8001 + int(row) % 100000, 256, int(k))
        words[sel, row >> 6] |= np.uint64(1) << np.uint64(row & 63)
    ids = np.arange(256)
    with make_pool(bm, words, r_bits) as pool:
        pool.set_dense_config(1, 128, 4, 1)
        for theta in (128, 255, 256):
            q = dg.Query(ids, 0, theta=theta)
            want = oracle_lib.query(words, q, r_bits)
            assert want[1] > 0 or theta == 256
            for looped in (0, 3):  # 255 and 256 take the Looped form when on
                pool.set_looped(looped)
                got = run_query(bm, pool, q)
                check_equal(got, want, f"planted theta={theta} looped={looped}")
