"""ORACLE — test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, loads or calls anything here, and nothing
here imports the product.

``oracle.c`` is the plain definition of a threshold / symmetric-function query
over bitmaps (per-row counters, then a comparison) and of a weighted threshold
with an optional AND / OR / AND NOT of one more bitmap, compiled with gcc.
``mlp.py`` is the fp64 NumPy statement of the selector network's forward pass,
backward pass and Adam step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over output words)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.oracle_cardinality.argtypes = [vp, u64]
        lib.oracle_cardinality.restype = u64
        lib.oracle_counts.argtypes = [vp, u64, vp, u32, u64, u64, u64, vp]
        lib.oracle_counts.restype = None
        lib.oracle_threshold.argtypes = [vp, u64, vp, u32, u64, u64, u64, u64, vp, vp]
        lib.oracle_threshold.restype = None
        lib.oracle_symmetric.argtypes = [vp, u64, vp, u32, u64, vp, u64, u64, vp, vp]
        lib.oracle_symmetric.restype = None
        lib.oracle_scancount.argtypes = [vp, vp, vp, u32, u64, u64, vp, u64, u64, vp, vp]
        lib.oracle_scancount.restype = None
        lib.oracle_weighted.argtypes = [vp, u64, vp, vp, u32, u64, u64, u32, vp, u64, u64, vp, vp]
        lib.oracle_weighted.restype = None
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        lib.oracle_get_threads.argtypes = []
        lib.oracle_get_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle inputs must be C-contiguous"
    return a.ctypes.data


def _words(r_bits: int) -> int:
    return (r_bits + 63) // 64


def _prep(pool: np.ndarray, ids):
    pool = np.ascontiguousarray(pool, dtype=np.uint64)
    if pool.ndim == 1:
        pool = pool.reshape(1, -1)
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
    if len(ids):
        assert int(ids.max()) < pool.shape[0], "id out of range"
    return pool, ids


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops."""
    _L().oracle_set_threads(int(n))


def threads() -> int:
    return int(_L().oracle_get_threads())


def cardinality(words: np.ndarray, r_bits: int) -> int:
    """Ones among the first r bits, counted one bit at a time."""
    words = np.ascontiguousarray(words, dtype=np.uint64)
    assert words.size >= _words(r_bits)
    return int(_L().oracle_cardinality(_p(words), r_bits))


def counts(pool: np.ndarray, ids, r_bits: int, w0: int = 0, w1: int | None = None) -> np.ndarray:
    """Per-row counts c_i for rows [64*w0, min(64*w1, r))."""
    pool, ids = _prep(pool, ids)
    w1 = _words(r_bits) if w1 is None else w1
    nrows = max(0, min(64 * w1, r_bits) - 64 * w0)
    out = np.zeros(max(nrows, 1), dtype=np.uint32)
    _L().oracle_counts(_p(pool), pool.shape[1], _p(ids), len(ids), r_bits, w0, w1, _p(out))
    return out[:nrows]


def threshold(pool: np.ndarray, ids, r_bits: int, theta: int, w0: int = 0,
              w1: int | None = None):
    """(output words w0..w1-1, number of ones among them) of T_theta over pool[ids]."""
    pool, ids = _prep(pool, ids)
    w1 = _words(r_bits) if w1 is None else w1
    out = np.zeros(max(w1 - w0, 1), dtype=np.uint64)
    card = np.zeros(1, dtype=np.uint64)
    _L().oracle_threshold(_p(pool), pool.shape[1], _p(ids), len(ids), r_bits, int(theta), w0, w1,
                          _p(out), _p(card))
    return out[: w1 - w0], int(card[0])


def symmetric(pool: np.ndarray, ids, r_bits: int, table: np.ndarray, w0: int = 0,
              w1: int | None = None):
    """(output words, ones) of the symmetric function whose bit c of `table` is f(c)."""
    pool, ids = _prep(pool, ids)
    table = np.ascontiguousarray(table, dtype=np.uint64)
    assert table.size * 64 >= len(ids) + 1, "table needs n+1 bits"
    w1 = _words(r_bits) if w1 is None else w1
    out = np.zeros(max(w1 - w0, 1), dtype=np.uint64)
    card = np.zeros(1, dtype=np.uint64)
    _L().oracle_symmetric(_p(pool), pool.shape[1], _p(ids), len(ids), r_bits, _p(table), w0, w1,
                          _p(out), _p(card))
    return out[: w1 - w0], int(card[0])


def scancount(flat: np.ndarray, offsets: np.ndarray, ids, r_bits: int, theta: int = 0,
              table: np.ndarray | None = None, w0: int = 0, w1: int | None = None):
    """ScanCount over sorted position lists (counter per row, then compare)."""
    flat = np.ascontiguousarray(flat, dtype=np.uint32)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
    if table is not None:
        table = np.ascontiguousarray(table, dtype=np.uint64)
        assert table.size * 64 >= len(ids) + 1
    w1 = _words(r_bits) if w1 is None else w1
    out = np.zeros(max(w1 - w0, 1), dtype=np.uint64)
    card = np.zeros(1, dtype=np.uint64)
    fp = flat if len(flat) else np.zeros(1, dtype=np.uint32)
    _L().oracle_scancount(_p(fp), _p(offsets), _p(ids), len(ids), r_bits, int(theta),
                          _p(table), w0, w1, _p(out), _p(card))
    return out[: w1 - w0], int(card[0])


def weighted(pool: np.ndarray, ids, weights, r_bits: int, theta: int, post_op: int = 0,
             post: np.ndarray | None = None, w0: int = 0, w1: int | None = None):
    """(output words, ones) of the weighted threshold [sum of weights of the
    inputs holding a row >= theta], combined with `post` by post_op (0 none,
    1 AND, 2 OR, 3 AND NOT)."""
    pool, ids = _prep(pool, ids)
    weights = np.ascontiguousarray(np.asarray(weights, dtype=np.uint32))
    assert len(weights) == len(ids)
    w1 = _words(r_bits) if w1 is None else w1
    if post is None:
        post = np.zeros(_words(r_bits), dtype=np.uint64)
    post = np.ascontiguousarray(post, dtype=np.uint64)
    out = np.zeros(max(w1 - w0, 1), dtype=np.uint64)
    card = np.zeros(1, dtype=np.uint64)
    _L().oracle_weighted(_p(pool), pool.shape[1], _p(ids), _p(weights), len(ids), r_bits,
                         int(theta), int(post_op), _p(post), w0, w1, _p(out), _p(card))
    return out[: w1 - w0], int(card[0])


def interval_table(n: int, lo: int, hi: int) -> np.ndarray:
    """Truth table of f(c) = [lo <= c <= hi] over c = 0..n, packed bit c = f(c)."""
    out = np.zeros((n + 1 + 63) // 64, dtype=np.uint64)
    for c in range(max(lo, 0), min(hi, n) + 1):
        out[c // 64] |= np.uint64(1) << np.uint64(c % 64)
    return out


def query(pool: np.ndarray, q, r_bits: int, w0: int = 0, w1: int | None = None):
    """Oracle answer for a datagen.Query (threshold, interval or table)."""
    if q.kind == 0:
        return threshold(pool, q.ids, r_bits, q.theta, w0, w1)
    if q.kind == 1:
        return symmetric(pool, q.ids, r_bits, interval_table(q.n, q.lo, q.hi), w0, w1)
    return symmetric(pool, q.ids, r_bits, q.table, w0, w1)
