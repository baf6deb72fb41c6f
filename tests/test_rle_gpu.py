"""GPU parity of the run-length path (word runs of zeros, ones and literals
with clean-run pruning) against the CPU oracle on the dense view, bit-exact:
clustered and scattered inputs, clean inputs of both kinds, ragged r, more
inputs than one classification pass, and predicates whose transitions fall
at or below the number of all-ones inputs of a tile."""
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
    assert chosen == path
    return bm.to_numpy_words(out), int(card.item())


def _runs_of(words: np.ndarray) -> tuple[int, int]:
    """(runs, literal words) of the word-run form, restated here: maximal runs
    of equal kind, kinds all-zero / all-one / other."""
    kind = np.where(words == 0, 0, np.where(words == np.uint64(0xFFFFFFFFFFFFFFFF), 1, 2))
    runs = 1 + int(np.count_nonzero(kind[1:] != kind[:-1])) if len(kind) else 0
    return runs, int(np.count_nonzero(kind == 2))


def _pool(bm, words, r_bits):
    pool = bm.Pool(r_bits, words.shape[0])
    pool.put_dense(words)
    pool.put_rle()
    return pool


def _mixed_words(dg, r_bits, stream):
    """Clustered (long runs), scattered, all-zero, all-one and word-alternating
    bitmaps side by side."""
    nw = (r_bits + 63) // 64
    clustered = dg.runs(stream, r_bits, np.array([0.3, 0.05, 0.6, 0.01]), 3000.0)
    scattered = dg.bernoulli(stream + 1, r_bits, np.array([0.01, 0.5]))
    zero = np.zeros((1, nw), np.uint64)
    one = np.full((1, nw), np.uint64(0xFFFFFFFFFFFFFFFF))
    alt = np.zeros((1, nw), np.uint64)
    alt[0, ::2] = np.uint64(0xFFFFFFFFFFFFFFFF)
    alt[0, 1::4] = np.uint64(0x00FF00FF00FF00FF)
    words = np.concatenate([clustered, scattered, zero, one, alt])
    tail = r_bits % 64
    if tail:
        words[:, -1] &= np.uint64((1 << tail) - 1)
    return words


@pytest.mark.parametrize("r_bits", [64, 100, 16384, 16384 * 3 + 4099, 1 << 20])
def test_rle_matches_oracle(bm, oracle_lib, dg, r_bits):
    words = _mixed_words(dg, r_bits, dg.STREAM_TESTS + 20000)
    n_bm = words.shape[0]
    with _pool(bm, words, r_bits) as pool:
        for k in range(n_bm):
            assert pool.rle_info(k) == _runs_of(words[k]), k
        ids = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 7, 7, 2], dtype=np.uint32)  # ones input thrice
        n = len(ids)
        for theta in (0, 1, 2, 3, 4, 5, 7, n, n + 1):
            q = dg.Query(ids, 0, theta=theta)
            got = _run(bm, pool, q, bm.PATH_RLE)
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], f"theta={theta}"
        for lo, hi in ((1, 3), (3, 5), (4, 12)):
            q = dg.Query(ids, 1, lo=lo, hi=hi)
            got = _run(bm, pool, q, bm.PATH_RLE)
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], f"[{lo},{hi}]"
        # many transitions (a table), with f(0) = 1 and odd counts
        f = (np.arange(n + 1) % 2 == 1)
        f[0] = True
        q = dg.Query(ids, 2, table=dg.table_from_bools(f))
        got = _run(bm, pool, q, bm.PATH_RLE)
        want = oracle_lib.query(words, q, r_bits)
        assert np.array_equal(got[0], want[0]) and got[1] == want[1], "table"


def test_rle_many_inputs_and_clean_ones(bm, oracle_lib, dg):
    """n = 2500 (three classification passes of 1024) with a third of the
    inputs all ones: thresholds below, at and above the clean-one count, an
    interval and a table predicate."""
    r_bits = 16384 * 5 + 77
    nw = (r_bits + 63) // 64
    base = dg.runs(dg.STREAM_TESTS + 20100, r_bits, np.linspace(0.001, 0.7, 60), 2000.0)
    one = np.full((1, nw), np.uint64(0xFFFFFFFFFFFFFFFF))
    one[0, -1] &= np.uint64((1 << (r_bits % 64)) - 1)
    words = np.concatenate([base, one])
    n = 2500
    ids = (np.arange(n) % words.shape[0]).astype(np.uint32)
    ids[::3] = 60  # the all-ones bitmap, 834 times
    with _pool(bm, words, r_bits) as pool:
        for theta in (1, 800, 834, 835, 900, 1300, n):
            q = dg.Query(ids, 0, theta=theta)
            got = _run(bm, pool, q, bm.PATH_RLE)
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], f"theta={theta}"
        q = dg.Query(ids, 1, lo=834, hi=860)
        got = _run(bm, pool, q, bm.PATH_RLE)
        want = oracle_lib.query(words, q, r_bits)
        assert np.array_equal(got[0], want[0]) and got[1] == want[1], "interval"
        # same answers on the dense path
        dense = _run(bm, pool, q, bm.PATH_DENSE)
        assert np.array_equal(dense[0], got[0]) and dense[1] == got[1]
        # a table predicate over the three passes (many transitions, f(0) = 1)
        f = (np.arange(n + 1) % 7) < 3
        q = dg.Query(ids, 2, table=dg.table_from_bools(f))
        got = _run(bm, pool, q, bm.PATH_RLE)
        want = oracle_lib.query(words, q, r_bits)
        assert np.array_equal(got[0], want[0]) and got[1] == want[1], "table"


def test_rle_clustered_workload_subset(bm, oracle_lib, dg):
    """Scaled clustered workload: 64 bitmaps of r = 2^22 rows, densities
    max(0.5/k, 1e-4) in runs of mean 4096 rows; the four bench queries."""
    r_bits = 1 << 22
    words = dg.runs(dg.STREAM_TESTS + 20200, r_bits, dg.config2_density(64), 4096.0)
    ids = np.arange(64, dtype=np.uint32)
    with _pool(bm, words, r_bits) as pool:
        for q in (dg.Query(ids, 0, theta=2), dg.Query(ids, 0, theta=32), dg.Query(ids, 0, theta=63),
                  dg.Query(ids, 1, lo=2, hi=10)):
            got = _run(bm, pool, q, bm.PATH_RLE)
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], q


def _rle_wins(pool, ids, dense_speedup):
    """The library's run-length cost model (GB300 fit, device time per query):
    12.5 us plus 1.3 us per round of 256-word tiles over three CTAs per SM
    plus 1.05 us per MB of summaries and containers, against 9 us plus
    0.14 us per MB of dense words, divided by dense_speedup."""
    info = pool.info()
    stored = sum(pool.rle_bytes(int(i)) for i in ids)
    tiles = (info["words"] + 255) // 256
    dense_mb = len(ids) * info["r_bits"] / 8.0 / 1e6
    rounds = -(-tiles // (3 * info["sm_count"]))
    return 12.5 + 1.3 * rounds + 1.05 * stored / 1e6 < (9.0 + 0.14 * dense_mb) / dense_speedup


def test_rle_auto_selection(bm, oracle_lib, dg):
    """BM_PATH_AUTO takes the run-length path for a query over clustered
    inputs (few runs) and the dense counter over incompressible ones, alone
    and in a batch, with the same answers as the oracle either way."""
    r_bits = 1 << 25
    clustered = dg.runs(dg.STREAM_TESTS + 20400, r_bits, np.linspace(0.01, 0.3, 48), 4096.0)
    scattered = dg.bernoulli(dg.STREAM_TESTS + 20401, r_bits, np.linspace(0.2, 0.5, 48))
    words = np.concatenate([clustered, scattered])
    with _pool(bm, words, r_bits) as pool:
        for ids, want_path in ((np.arange(48), bm.PATH_RLE), (np.arange(48, 96), bm.PATH_DENSE)):
            ids = ids.astype(np.uint32)
            for q in (dg.Query(ids, 0, theta=3), dg.Query(ids, 1, lo=2, hi=9)):
                assert bm.query_select(pool, q)[0] == want_path
                out = pool.empty_words()
                out.fill_(-1)
                card = torch.full((1,), -1, dtype=torch.int64, device="cuda")
                assert bm.query_run(pool, q, out, card) == want_path
                torch.cuda.synchronize()
                pool.status()
                want = oracle_lib.query(words, q, r_bits)
                assert np.array_equal(bm.to_numpy_words(out), want[0]) and int(card.item()) == want[1]
        # an input without a run-length form keeps the query on the dense counter
        words2 = words[:49].copy()
        with bm.Pool(r_bits, 49) as pool2:
            pool2.put_dense(words2)
            pool2.put_rle(0, 40)
            q = dg.Query(np.arange(48, dtype=np.uint32), 0, theta=3)
            assert bm.query_select(pool2, q)[0] == bm.PATH_DENSE
            q = dg.Query(np.arange(40, dtype=np.uint32), 0, theta=3)
            assert bm.query_select(pool2, q)[0] == bm.PATH_RLE
        # in a batch a query left dense shares the pool's slabs with the others,
        # so the run-length path must beat the dense estimate divided by the
        # batch's measured speed-up (2.5) instead
        want_auto = bm.PATH_RLE if _rle_wins(pool, np.arange(48), 2.5) else bm.PATH_DENSE
        assert _rle_wins(pool, np.arange(48), 1.0)
        qs = [dg.Query(np.arange(48, dtype=np.uint32), 0, theta=3),
              dg.Query(np.arange(48, 96, dtype=np.uint32), 0, theta=3),
              dg.Query(np.arange(0, 96, 2, dtype=np.uint32), 2,
                       table=dg.table_from_bools(np.arange(49) % 3 == 1))]
        outs = [pool.empty_words() for _ in qs]
        for o in outs:
            o.fill_(-1)
        cards = torch.full((len(qs),), -1, dtype=torch.int64, device="cuda")
        paths = bm.threshold_batch(pool, qs, outs, cards, paths=[bm.PATH_AUTO, bm.PATH_AUTO, bm.PATH_RLE])
        torch.cuda.synchronize()
        pool.status()
        assert list(paths) == [want_auto, bm.PATH_DENSE, bm.PATH_RLE]
        for i, q in enumerate(qs):
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(bm.to_numpy_words(outs[i]), want[0]), i
            assert int(cards[i].item()) == want[1], i


def test_rle_errors(bm, dg):
    r_bits = 5000
    words = dg.bernoulli(dg.STREAM_TESTS + 20300, r_bits, np.array([0.1, 0.2, 0.3]))
    with bm.Pool(r_bits, 4) as pool:
        pool.put_dense(words)
        with pytest.raises(bm.BMError) as e:
            pool.put_rle(0, 4)  # id 3 has no dense copy
        assert e.value.code == bm.BM_ERANGE
        pool.put_rle(0, 3)
        assert pool.info()["rle_loaded"] == 3
        out = pool.empty_words()
        with pytest.raises(bm.BMError) as e:  # id 3 has no run-length form
            bm.query_run(pool, dg.Query(np.array([0, 3]), 0, theta=1), out, path=bm.PATH_RLE)
        assert e.value.code == bm.BM_ERANGE
        with pytest.raises(bm.BMError) as e:  # in a batch as well
            bm.threshold_batch(pool, [dg.Query(np.array([0, 3]), 0, theta=1)], [out],
                               torch.zeros(1, dtype=torch.int64, device="cuda"), paths=[bm.PATH_RLE])
        assert e.value.code == bm.BM_ERANGE
        with pytest.raises(bm.BMError):
            pool.rle_info(3)


def _tiled_bytes(words: np.ndarray) -> int:
    """Device bytes of the tiled run-length form, restated here: an 8-byte
    summary per 256-word tile, and for a tile that is neither all clean-0 nor
    all clean-1 words a container of 80 header bytes plus 8 per literal word,
    padded to 16 bytes."""
    ones = np.uint64(0xFFFFFFFFFFFFFFFF)
    total = 0
    for t0 in range(0, len(words), 256):
        w = words[t0:t0 + 256]
        lit = int(np.count_nonzero((w != 0) & (w != ones)))
        total += 8
        if lit == 0 and (np.all(w == 0) or np.all(w == ones)):
            continue
        total += (80 + 8 * lit + 15) // 16 * 16
    return total


def test_rle_form_sizes_rebuild_and_growth(bm, oracle_lib, dg):
    """The form's size matches its definition word by word (ragged last tile,
    tiles that are one clean run, literal-only tiles); forms built by several
    calls over different id ranges (each call's summaries land in its own
    columns of the tile-major matrix), an id rebuilt after the others (its
    old form left behind), and queries across all of them keep the oracle's
    answers."""
    r_bits = 256 * 64 * 7 + 64 * 37 + 11  # seven full tiles and a ragged eighth
    nw = (r_bits + 63) // 64
    words = _mixed_words(dg, r_bits, dg.STREAM_TESTS + 20500)
    full = np.full(nw, np.uint64(0xFFFFFFFFFFFFFFFF))
    full[-1] = np.uint64((1 << (r_bits % 64)) - 1)
    blocky = np.zeros(nw, np.uint64)  # whole tiles of ones, zeros, literals
    blocky[0:256] = np.uint64(0xFFFFFFFFFFFFFFFF)
    blocky[512:768] = np.uint64(0x5555555555555555)
    blocky[1024:1100] = np.uint64(0xFFFFFFFFFFFFFFFF)
    words = np.concatenate([words, full[None, :], blocky[None, :]])
    n_bm = words.shape[0]
    with bm.Pool(r_bits, n_bm) as pool:
        pool.put_dense(words)
        pool.put_rle(0, 3)
        pool.put_rle(3, n_bm - 3)
        pool.put_rle(1, 1)  # rebuilt: appended after the others
        for k in range(n_bm):
            assert pool.rle_bytes(k) == _tiled_bytes(words[k]), k
            assert pool.rle_info(k) == _runs_of(words[k]), k
        ids = np.arange(n_bm, dtype=np.uint32)
        for q in (dg.Query(ids, 0, theta=1), dg.Query(ids, 0, theta=3), dg.Query(ids, 1, lo=2, hi=4),
                  dg.Query(np.array([1, 1, 7, 8, 8], dtype=np.uint32), 0, theta=3)):
            got = _run(bm, pool, q, bm.PATH_RLE)
            want = oracle_lib.query(words, q, r_bits)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1], q


def test_rle_constant_tiles_aligned_and_unaligned_output(bm, oracle_lib, dg):
    """Tiles that RBMrg's pruning settles (whole tiles of one value) are
    written whole by 16-byte stores into an aligned output and word by word
    into one that is only 8-byte aligned, and around a ragged last tile;
    both give the oracle's words and cardinality, with nothing written past
    the buffer."""
    r_bits = 256 * 64 * 6 + 64 * 5 + 9
    nw = (r_bits + 63) // 64
    ones = np.uint64(0xFFFFFFFFFFFFFFFF)
    words = np.zeros((6, nw), np.uint64)
    words[0:3, : 256 * 3] = ones  # three inputs all ones over the first three tiles
    words[3, 256 * 4:256 * 5] = np.uint64(0x00FF00FF00FF00FF)
    words[4:6] = dg.runs(dg.STREAM_TESTS + 20600, r_bits, np.array([0.02, 0.2]), 4096.0)
    words[:, -1] &= np.uint64((1 << (r_bits % 64)) - 1)
    ids = np.arange(6, dtype=np.uint32)
    with _pool(bm, words, r_bits) as pool:
        for q in (dg.Query(ids, 0, theta=3), dg.Query(ids, 0, theta=0), dg.Query(ids, 0, theta=1),
                  dg.Query(ids, 1, lo=0, hi=2)):
            want = oracle_lib.query(words, q, r_bits)
            for shift in (0, 1):
                big = torch.full((pool.words + 2,), -7, dtype=torch.int64, device="cuda")
                out = big[shift:shift + pool.words]
                card = torch.zeros(1, dtype=torch.int64, device="cuda")
                assert bm.query_run(pool, q, out, card, path=bm.PATH_RLE) == bm.PATH_RLE
                torch.cuda.synchronize()
                pool.status()
                assert np.array_equal(bm.to_numpy_words(out), want[0]), (q, shift)
                assert int(card.item()) == want[1], (q, shift)
                if shift:
                    assert int(big[0].item()) == -7
                assert int(big[shift + pool.words].item()) == -7
