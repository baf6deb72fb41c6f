"""Pins for the CPU oracle (no GPU).  Each test checks the oracle against
something other than itself: a value printed in the paper, a closed form, a
textbook identity, or an independent formulation of the same function."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

from paper_algos import carry_save_vertical, looped

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ALL = np.uint64(0xFFFFFFFFFFFFFFFF)


def _golden(name):
    d = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        d.setdefault(k, []).append(v)
    return d


def _mask(r_bits):
    w = (r_bits + 63) // 64
    m = np.full(w, ALL, dtype=np.uint64)
    if r_bits % 64:
        m[-1] = np.uint64((1 << (r_bits % 64)) - 1)
    return m


def _rand_pool(dg, n, r_bits, p=0.3, stream=0):
    return dg.bernoulli(dg.STREAM_TESTS + stream * 1000, r_bits, np.full(n, p))


def _rows(words, r_bits):
    """Set rows of a word array, via Python integers (independent of the oracle)."""
    out = []
    for j, w in enumerate(words.tolist()):
        for b in range(64):
            if (w >> b) & 1 and j * 64 + b < r_bits:
                out.append(j * 64 + b)
    return out


# --- paper worked examples -------------------------------------------------


def test_bit_layout_example(oracle_lib, dg):
    g = _golden("bit_layout.txt")
    W = int(g["W"][0][0])
    members = [int(x) for x in g["set"][0]]
    printed = g["words"][0]
    # rebuild the bitmap from the printed W-bit words (MSB on the left)
    value = 0
    for j, s in enumerate(printed):
        assert len(s) == W
        value |= int(s, 2) << (W * j)
    r_bits = W * len(printed)
    words = np.array([value], dtype=np.uint64)
    assert _rows(words, r_bits) == members
    # the one-input threshold T_1 reproduces the bitmap; its cardinality is |S|
    out, card = oracle_lib.threshold(words.reshape(1, -1), [0], r_bits, 1)
    assert out.tolist() == words.tolist() and card == len(members)
    assert oracle_lib.cardinality(words, r_bits) == len(members)
    flat, offs = dg.positions(words.reshape(1, -1), r_bits)
    assert flat.tolist() == members


def test_comparator_example_t167(oracle_lib):
    """1023 inputs where row i has exactly i ones (i < 1024): T_168 must equal
    the paper's reduced comparator for count > 0010100111 (binary)."""
    g = _golden("comparator_167.txt")
    n_bits = int(g["n"][0][0])
    t_minus_1 = int(g["t_minus_1"][0][0], 2)
    terms = [[int(x) for x in t] for t in g["term"]]
    assert t_minus_1 == 167
    N, r_bits = (1 << n_bits) - 1, 1 << n_bits
    rows = np.arange(r_bits)
    # bitmap k has row i set iff k < i
    bits = (np.arange(N)[:, None] < rows[None, :])
    pool = np.packbits(bits, axis=1, bitorder="little").view(np.uint64)
    cnt = oracle_lib.counts(pool, np.arange(N), r_bits)
    assert cnt.tolist() == rows.tolist()
    out, card = oracle_lib.threshold(pool, np.arange(N), r_bits, t_minus_1 + 1)
    got = np.unpackbits(out.view(np.uint8), bitorder="little").astype(bool)
    formula = np.zeros(r_bits, dtype=bool)
    for term in terms:
        acc = np.ones(r_bits, dtype=bool)
        for j in term:
            acc &= ((rows >> j) & 1).astype(bool)
        formula |= acc
    assert np.array_equal(got, formula)
    assert card == r_bits - (t_minus_1 + 1)


def test_padding_rule_example(oracle_lib, dg):
    g = _golden("padding_rule.txt")
    N, T = int(g["N"][0][0]), int(g["T"][0][0])
    Np, Tp = int(g["N_prime"][0][0]), int(g["T_prime"][0][0])
    z, o = int(g["zero_pads"][0][0]), int(g["one_pads"][0][0])
    assert Np + z + o == N
    r_bits = 5000
    pool = _rand_pool(dg, Np, r_bits, 0.5, stream=1)
    pad = np.vstack([pool, np.zeros((z, pool.shape[1]), np.uint64),
                     np.tile(_mask(r_bits), (o, 1))])
    want, cw = oracle_lib.threshold(pool, np.arange(Np), r_bits, Tp)
    got, cg = oracle_lib.threshold(pad, np.arange(N), r_bits, T)
    assert np.array_equal(want, got) and cw == cg


def test_padding_rule_general(oracle_lib, dg):
    """(N, T) covers (N', T') iff N' <= N and T - (N - N') <= T' <= T: pad with
    T - T' all-one and the rest all-zero bitmaps."""
    r_bits = 3000
    N = 9
    for Np in range(1, N + 1):
        pool = _rand_pool(dg, Np, r_bits, 0.4, stream=10 + Np)
        for T in range(1, N + 1):
            for Tp in range(max(1, T - (N - Np)), min(T, Np) + 1):
                ones = T - Tp
                zeros = N - Np - ones
                pad = np.vstack([pool, np.tile(_mask(r_bits), (ones, 1)),
                                 np.zeros((zeros, pool.shape[1]), np.uint64)])
                a = oracle_lib.threshold(pool, np.arange(Np), r_bits, Tp)
                b = oracle_lib.threshold(pad, np.arange(N), r_bits, T)
                assert np.array_equal(a[0], b[0]) and a[1] == b[1]


# --- exhaustive enumeration (closed form) ------------------------------------


def _exhaustive_pool(N):
    r_bits = 1 << N
    rows = np.arange(r_bits)
    bits = ((rows[None, :] >> np.arange(N)[:, None]) & 1).astype(bool)
    if r_bits < 64:
        bits = np.pad(bits, ((0, 0), (0, 64 - r_bits)))
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint64).copy(), r_bits


@pytest.mark.parametrize("N", list(range(1, 13)))
def test_exhaustive_threshold(oracle_lib, N):
    pool, r_bits = _exhaustive_pool(N)
    pc = np.array([bin(i).count("1") for i in range(r_bits)])
    for theta in range(0, N + 2):
        out, card = oracle_lib.threshold(pool, np.arange(N), r_bits, theta)
        assert card == sum(math.comb(N, c) for c in range(theta, N + 1))
        got = np.unpackbits(out.view(np.uint8), bitorder="little")[:r_bits].astype(bool)
        assert np.array_equal(got, pc >= theta)


def test_exhaustive_golden_n12(oracle_lib):
    g = _golden("exhaustive_binomial.txt")
    N = int(g["N"][0][0])
    cards = [int(x) for x in g["cards"][0]]
    pool, r_bits = _exhaustive_pool(N)
    got = [oracle_lib.threshold(pool, np.arange(N), r_bits, t)[1] for t in range(N + 2)]
    assert got == cards


@pytest.mark.parametrize("N", [1, 2, 5, 8, 12])
def test_exhaustive_symmetric(oracle_lib, dg, N):
    pool, r_bits = _exhaustive_pool(N)
    pc = np.array([bin(i).count("1") for i in range(r_bits)])
    u = dg.uniform(dg.STREAM_TESTS + 77 + N, 8 * (N + 1)).reshape(8, N + 1)
    for f in (u < 0.5):
        table = dg.table_from_bools(f)
        out, card = oracle_lib.symmetric(pool, np.arange(N), r_bits, table)
        assert card == sum(math.comb(N, c) for c in range(N + 1) if f[c])
        got = np.unpackbits(out.view(np.uint8), bitorder="little")[:r_bits].astype(bool)
        assert np.array_equal(got, f[pc])
    # XOR (parity) is the symmetric function "weight is odd" (Sec. 2.2)
    parity = dg.table_from_bools([c % 2 == 1 for c in range(N + 1)])
    out, _ = oracle_lib.symmetric(pool, np.arange(N), r_bits, parity)
    x = np.zeros_like(pool[0])
    for k in range(N):
        x ^= pool[k]
    assert np.array_equal(out, x & _mask(r_bits))


# --- definitions ---------------------------------------------------------------


@pytest.mark.parametrize("r_bits", [1, 63, 64, 65, 1000, 4096 + 17])
def test_definitions_or_and_all_none(oracle_lib, dg, r_bits):
    N = 7
    pool = _rand_pool(dg, N, r_bits, 0.35, stream=2 + r_bits)
    # inputs may carry garbage beyond r: it must be ignored
    pool[:, -1] |= ~_mask(r_bits)[-1]
    ids = np.arange(N)
    m = _mask(r_bits)
    o = np.zeros_like(pool[0])
    a = np.full_like(pool[0], ALL)
    for k in range(N):
        o |= pool[k]
        a &= pool[k]
    assert np.array_equal(oracle_lib.threshold(pool, ids, r_bits, 1)[0], o & m)
    assert np.array_equal(oracle_lib.threshold(pool, ids, r_bits, N)[0], a & m)
    out0, c0 = oracle_lib.threshold(pool, ids, r_bits, 0)
    assert np.array_equal(out0, m) and c0 == r_bits
    outz, cz = oracle_lib.threshold(pool, ids, r_bits, N + 1)
    assert not outz.any() and cz == 0


def test_majority_of_three(oracle_lib, dg):
    r_bits = 10000
    pool = _rand_pool(dg, 3, r_bits, 0.5, stream=3)
    a, b, c = pool
    want = ((a & b) | (b & c) | (a & c)) & _mask(r_bits)
    assert np.array_equal(oracle_lib.threshold(pool, [0, 1, 2], r_bits, 2)[0], want)


def test_interval_is_andnot_of_thresholds(oracle_lib, dg):
    """[L, U] = T_L AND NOT T_{U+1} (Sec. 4.3, "Sorting")."""
    r_bits, N = 7777, 11
    pool = _rand_pool(dg, N, r_bits, 0.4, stream=4)
    ids = np.arange(N)
    for L in range(0, N + 1):
        for U in range(L, N + 1):
            got = oracle_lib.symmetric(pool, ids, r_bits, oracle_lib.interval_table(N, L, U))[0]
            tl = oracle_lib.threshold(pool, ids, r_bits, L)[0]
            tu = oracle_lib.threshold(pool, ids, r_bits, U + 1)[0]
            assert np.array_equal(got, tl & ~tu)


def test_complement_identity_corrected(oracle_lib, dg):
    """NOT T(theta, b) = T(N - theta + 1, NOT b).  The identity as printed in
    Sec. 2.3, with N - theta, fails already for N = 1, theta = 1."""
    r_bits = 3000
    m = _mask(r_bits)
    for N in range(1, 8):
        pool = _rand_pool(dg, N, r_bits, 0.3, stream=5 + N)
        neg = (~pool) & m
        ids = np.arange(N)
        for theta in range(0, N + 2):
            lhs = (~oracle_lib.threshold(pool, ids, r_bits, theta)[0]) & m
            rhs = oracle_lib.threshold(neg, ids, r_bits, N - theta + 1)[0]
            assert np.array_equal(lhs, rhs)
    pool = _rand_pool(dg, 1, r_bits, 0.3, stream=99)
    printed = oracle_lib.threshold((~pool) & m, [0], r_bits, 0)[0]
    assert not np.array_equal((~oracle_lib.threshold(pool, [0], r_bits, 1)[0]) & m, printed)


def test_monotone_permutation_duplicates(oracle_lib, dg):
    r_bits, N = 5000, 12
    pool = _rand_pool(dg, N, r_bits, 0.45, stream=6)
    ids = np.arange(N)
    prev = None
    for theta in range(0, N + 2):
        cur = oracle_lib.threshold(pool, ids, r_bits, theta)[0]
        if prev is not None:
            assert not (cur & ~prev).any()  # T_{theta} subset of T_{theta-1}
        prev = cur
    perm = dg.floyd(dg.STREAM_TESTS + 7, N, N)
    for theta in (2, 5, 9):
        assert np.array_equal(oracle_lib.threshold(pool, ids, r_bits, theta)[0],
                              oracle_lib.threshold(pool, perm, r_bits, theta)[0])
    # a repeated id counts with multiplicity: ids [0, 0, 1] at theta 2 is
    # "bitmap 0, or bitmap 1 together with ... bitmap 0" = bitmap 0
    got = oracle_lib.threshold(pool, [0, 0, 1], r_bits, 2)[0]
    assert np.array_equal(got, pool[0] & _mask(r_bits))
    got = oracle_lib.threshold(pool, [0, 0, 1], r_bits, 3)[0]
    assert np.array_equal(got, pool[0] & pool[1] & _mask(r_bits))


# --- weighted thresholds and combining (Sec. 2.3) -------------------------------


def test_weighted_is_replication(oracle_lib, dg):
    """A weight is the number of copies of an input (Sec. 2.3)."""
    r_bits = 3000
    pool = _rand_pool(dg, 6, r_bits, 0.4, stream=30)
    ids = np.array([0, 1, 2, 3, 4, 5])
    weights = np.array([1, 3, 2, 5, 1, 4])
    rep = np.repeat(ids, weights)
    for theta in range(0, int(weights.sum()) + 2):
        a = oracle_lib.weighted(pool, ids, weights, r_bits, theta)
        b = oracle_lib.threshold(pool, rep, r_bits, theta)
        assert np.array_equal(a[0], b[0]) and a[1] == b[1], theta
    # weight 0 drops an input; all weights 1 is the plain threshold
    a = oracle_lib.weighted(pool, ids, [1, 0, 1, 0, 1, 0], r_bits, 2)
    assert np.array_equal(a[0], oracle_lib.threshold(pool, [0, 2, 4], r_bits, 2)[0])
    a = oracle_lib.weighted(pool, ids, np.ones(6), r_bits, 3)
    assert np.array_equal(a[0], oracle_lib.threshold(pool, ids, r_bits, 3)[0])


def test_weighted_binary_weights_exhaustive(oracle_lib):
    """Inputs k = 0..N-1 with bit(k, i) = bit k of i and weight 2^k: every row's
    weighted sum is i itself, so the output is [i >= theta] exactly."""
    N = 10
    pool, r_bits = _exhaustive_pool(N)
    weights = 1 << np.arange(N)
    for theta in (0, 1, 2, 3, 511, 512, 513, 1000, 1023, 1024):
        out, card = oracle_lib.weighted(pool, np.arange(N), weights, r_bits, theta)
        assert card == max(0, r_bits - theta)
        got = np.unpackbits(out.view(np.uint8), bitorder="little")[:r_bits].astype(bool)
        assert np.array_equal(got, np.arange(r_bits) >= theta)
    # large weights: one input of weight 2^31 decides alone
    out, _ = oracle_lib.weighted(pool, [3, 0, 1], [1 << 31, 1, 1], r_bits, 1 << 31)
    assert np.array_equal(out, pool[3] & _mask(r_bits))


def test_weighted_post_ops(oracle_lib, dg):
    r_bits = 777
    pool = _rand_pool(dg, 5, r_bits, 0.5, stream=31)
    ids, weights = [0, 1, 2, 3], [2, 1, 1, 3]
    t, _ = oracle_lib.weighted(pool, ids, weights, r_bits, 3)
    m = pool[4]
    mask = _mask(r_bits)
    for op, want in ((1, t & m), (2, (t | m) & mask), (3, t & ~m & mask)):
        got, card = oracle_lib.weighted(pool, ids, weights, r_bits, 3, op, m)
        assert np.array_equal(got, want), op
        assert card == int(sum(bin(int(x)).count("1") for x in want))


# --- independent formulations from the paper -----------------------------------


@pytest.mark.parametrize("N", [1, 2, 3, 4, 7, 16, 20])
def test_looped_matches_oracle(oracle_lib, dg, N):
    r_bits = 4000 + N
    pool = _rand_pool(dg, N, r_bits, 0.5, stream=20 + N)
    m = _mask(r_bits)
    for T in range(1, N + 1):
        want = looped(list(pool), T) & m
        assert np.array_equal(oracle_lib.threshold(pool, np.arange(N), r_bits, T)[0], want)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 8, 13, 33])
def test_carry_save_vertical_matches_oracle(oracle_lib, dg, N):
    r_bits = 3000 + N
    pool = _rand_pool(dg, N, r_bits, 0.5, stream=40 + N)
    m = _mask(r_bits)
    for T in range(1, N + 1):
        want = carry_save_vertical(list(pool), T) & m
        assert np.array_equal(oracle_lib.threshold(pool, np.arange(N), r_bits, T)[0], want)


def test_scancount_matches_dense(oracle_lib, dg):
    r_bits = 20000 + 37
    pool = dg.bernoulli(dg.STREAM_TESTS + 500, r_bits, np.array([1e-3, 0.01, 0.1, 0.5, 0.0, 1.0]))
    flat, offs = dg.positions(pool, r_bits)
    for k in range(pool.shape[0]):
        assert flat[offs[k]:offs[k + 1]].tolist() == _rows(pool[k], r_bits)
    ids = [0, 1, 2, 3, 4, 5, 2]
    for theta in range(0, 9):
        a = oracle_lib.threshold(pool, ids, r_bits, theta)
        b = oracle_lib.scancount(flat, offs, ids, r_bits, theta)
        assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    tab = oracle_lib.interval_table(len(ids), 2, 4)
    a = oracle_lib.symmetric(pool, ids, r_bits, tab)
    b = oracle_lib.scancount(flat, offs, ids, r_bits, table=tab)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    # a sub-range of words
    a = oracle_lib.threshold(pool, ids, r_bits, 2, 100, 250)
    b = oracle_lib.scancount(flat, offs, ids, r_bits, 2, None, 100, 250)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]


def test_word_range_matches_full(oracle_lib, dg):
    r_bits, N = 64 * 300 + 5, 9
    pool = _rand_pool(dg, N, r_bits, 0.4, stream=8)
    full, _ = oracle_lib.threshold(pool, np.arange(N), r_bits, 4)
    part, card = oracle_lib.threshold(pool, np.arange(N), r_bits, 4, 250, 301)
    assert np.array_equal(full[250:301], part)
    assert card == sum(bin(int(w)).count("1") for w in part.tolist())


def test_config1_statistics(oracle_lib, dg):
    """Config-1 inputs are i.i.d. Bernoulli(0.1): the answer sizes must sit
    within 6 sigma of 2^20 * P[Binomial(16, 0.1) in the selected set]."""
    words, queries = dg.config1()
    r_bits = 1 << 20

    def tail(lo, hi):
        return sum(math.comb(16, c) * 0.1 ** c * 0.9 ** (16 - c) for c in range(lo, hi + 1))

    for q, (lo, hi) in zip(queries, [(3, 16), (8, 16), (2, 5)]):
        _, card = oracle_lib.query(words, q, r_bits)
        p = tail(lo, hi)
        mean, sd = r_bits * p, math.sqrt(r_bits * p * (1 - p))
        assert abs(card - mean) < 6 * sd + 1, (q, card, mean)
