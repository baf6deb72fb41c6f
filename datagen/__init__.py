"""Seeded synthetic inputs for threshold and symmetric-function queries.

This module only draws inputs: dense bitmaps, sorted position lists and query
parameters.  It holds none of the method's arithmetic (no counting, no
comparison with a threshold), so the oracle tests and the CUDA tests can both
take their inputs from it.

Every generator is deterministic in (seed, stream).  The paper seeded its
synthetic sets with 1111 (Sec. 5, "Synthetic data"); the workloads here reuse
that seed and separate workloads and purposes by stream number.

Workload recipes (bitmaps of r rows as ceil(r/64) little-endian uint64 words):

* ``config1``: N=16, r=2^20, every bit i.i.d. Bernoulli(0.1); queries theta=3,
  theta=8 and the interval count in [2, 5].
* ``config2``: N=256, r=2^26; bitmap k (1-based) has density max(0.5/k, 1e-4),
  its ones placed as runs of geometric length (mean 8) at uniform starts;
  queries theta in {2, 128, 255} and the interval [2, 10].
* ``mixed_pool`` / ``mixed_queries``: a resident pool (2000 x 2^24 at full
  size) with log-uniform densities in [1e-4, 0.5]; queries pick N log-uniform
  in [3, 1000] distinct bitmaps, theta uniform in [1, N], and with probability
  0.1 an interval [L, U] from two sorted uniform draws in [1, N].
* ``sparse_pool`` / ``sparse_queries``: 5000 x 2^24, densities log-uniform in
  [1e-5, 1e-2], each bitmap also as a sorted uint32 position list; N
  log-uniform in [2, 4096], theta uniform in [1, min(N, 64)].
* ``clustered_pool`` / ``clustered_queries``: five blocks of bitmaps whose ones
  come in runs of mean 8 .. 16384 rows, densities log-uniform in [1e-4, 0.5],
  with position lists; each query takes its ids from one block.
* ``serving_pool`` / ``serving_queries``: 10000 x 2^22, densities log-uniform in
  [1e-5, 0.5]; N log-uniform in [2, 4096], theta uniform in [1, N], Poisson
  arrival times at a given rate.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

SEED = 1111
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "datagen.c")
_SO = os.path.join(_HERE, "_datagen.so")
_lib = None

# stream bases: one disjoint range of 2^40 streams per workload and purpose
STREAM_CONFIG1 = 1 << 40
STREAM_CONFIG2 = 2 << 40
STREAM_MIXED = 3 << 40
STREAM_SPARSE = 4 << 40
STREAM_SERVING = 5 << 40
STREAM_CLUSTERED = 6 << 40
STREAM_TESTS = 9 << 40
_QUERY_OFFSET = 1 << 32  # query-parameter streams sit above the bitmap streams


def build(force: bool = False) -> str:
    """Compile the generator library with gcc (host code, any architecture)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.dg_uniform.argtypes = [u64, u64, u64, vp]
        lib.dg_raw.argtypes = [u64, u64, u64, vp]
        lib.dg_bernoulli.argtypes = [u64, u64, u32, u64, vp, vp, u64]
        lib.dg_runs.argtypes = [u64, u64, u32, u64, vp, ctypes.c_double, vp, u64]
        lib.dg_positions.argtypes = [vp, u32, u64, u64, vp, vp]
        lib.dg_floyd.argtypes = [u64, u64, u32, u32, vp, vp]
        for f in (lib.dg_uniform, lib.dg_raw, lib.dg_bernoulli, lib.dg_runs, lib.dg_positions, lib.dg_floyd):
            f.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def words_for(r_bits: int) -> int:
    return (r_bits + 63) // 64


def uniform(stream: int, n: int, seed: int = SEED) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    if n:
        _L().dg_uniform(seed, stream, n, _p(out))
    return out


def raw64(stream: int, n: int, seed: int = SEED) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    if n:
        _L().dg_raw(seed, stream, n, _p(out))
    return out


def bernoulli(stream0: int, r_bits: int, p, seed: int = SEED) -> np.ndarray:
    """Bitmaps with i.i.d. Bernoulli(p[k]) bits; returns (len(p), ceil(r/64)) uint64."""
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64))
    w = words_for(r_bits)
    out = np.empty((len(p), w), dtype=np.uint64)
    if len(p) and w:
        _L().dg_bernoulli(seed, stream0, len(p), r_bits, _p(p), _p(out), w)
    return out


def runs(stream0: int, r_bits: int, density, mean_len: float = 8.0, seed: int = SEED) -> np.ndarray:
    """Bitmaps whose ones are runs of geometric length at uniform starts."""
    d = np.ascontiguousarray(np.asarray(density, dtype=np.float64))
    w = words_for(r_bits)
    out = np.empty((len(d), w), dtype=np.uint64)
    if len(d):
        _L().dg_runs(seed, stream0, len(d), r_bits, _p(d), float(mean_len), _p(out), w)
    return out


def positions(words: np.ndarray, r_bits: int):
    """Sorted uint32 position lists of each row of `words`: (flat, offsets[nbm+1])."""
    words = np.ascontiguousarray(words)
    nbm, stride = words.shape
    offs = np.zeros(nbm + 1, dtype=np.uint64)
    _L().dg_positions(_p(words), nbm, stride, r_bits, _p(offs), None)
    flat = np.empty(int(offs[-1]), dtype=np.uint32)
    if len(flat):
        _L().dg_positions(_p(words), nbm, stride, r_bits, _p(offs), _p(flat))
    return flat, offs


def floyd(stream: int, n: int, k: int, seed: int = SEED) -> np.ndarray:
    """k distinct integers from [0, n), Floyd's algorithm."""
    assert 0 <= k <= n
    out = np.empty(k, dtype=np.uint32)
    seen = np.empty(max(n, 1), dtype=np.uint8)
    if k:
        _L().dg_floyd(seed, stream, n, k, _p(out), _p(seen))
    return out


def log_uniform(u: np.ndarray, a: float, b: float) -> np.ndarray:
    return np.exp(math.log(a) + u * (math.log(b) - math.log(a)))


def log_uniform_int(u: np.ndarray, a: int, b: int) -> np.ndarray:
    return np.clip(np.rint(log_uniform(u, a, b)), a, b).astype(np.int64)


def uniform_int(u: np.ndarray, lo: int, hi) -> np.ndarray:
    """Integers uniform in [lo, hi] (hi may be an array)."""
    hi = np.asarray(hi)
    x = lo + np.floor(u * (hi - lo + 1)).astype(np.int64)
    return np.minimum(x, hi)


# ---------------------------------------------------------------------------
# queries


KIND_THRESHOLD = 0
KIND_INTERVAL = 1
KIND_TABLE = 2


@dataclass
class Query:
    ids: np.ndarray            # uint32 bitmap ids (repeats allowed)
    kind: int = KIND_THRESHOLD
    theta: int = 0
    lo: int = 0
    hi: int = 0
    table: np.ndarray | None = None  # uint64 words, bit c = f(c), for KIND_TABLE
    arrival_s: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(len(self.ids))


def table_from_bools(f) -> np.ndarray:
    """Pack a truth table f[0..n] into uint64 words, bit c = f[c]."""
    f = np.asarray(f, dtype=bool)
    out = np.zeros((len(f) + 63) // 64, dtype=np.uint64)
    for c in np.nonzero(f)[0]:
        out[c // 64] |= np.uint64(1) << np.uint64(c % 64)
    return out


# ---------------------------------------------------------------------------
# workloads


def config1(r_bits: int = 1 << 20, n: int = 16, p: float = 0.1):
    """N=16 bitmaps of r=2^20 bits, i.i.d. Bernoulli(0.1)."""
    words = bernoulli(STREAM_CONFIG1, r_bits, np.full(n, p))
    ids = np.arange(n, dtype=np.uint32)
    queries = [Query(ids, KIND_THRESHOLD, theta=3), Query(ids, KIND_THRESHOLD, theta=8),
               Query(ids, KIND_INTERVAL, lo=2, hi=5)]
    return words, queries


def config2_density(n: int = 256) -> np.ndarray:
    k = np.arange(1, n + 1, dtype=np.float64)
    return np.maximum(0.5 / k, 1e-4)


def config2(r_bits: int = 1 << 26, n: int = 256):
    """N=256 run-structured bitmaps of r=2^26 bits, densities max(0.5/k, 1e-4)."""
    words = runs(STREAM_CONFIG2, r_bits, config2_density(n), 8.0)
    ids = np.arange(n, dtype=np.uint32)
    queries = [Query(ids, KIND_THRESHOLD, theta=2), Query(ids, KIND_THRESHOLD, theta=128),
               Query(ids, KIND_THRESHOLD, theta=255), Query(ids, KIND_INTERVAL, lo=2, hi=10)]
    return words, queries


def pool_densities(stream: int, n: int, dmin: float, dmax: float) -> np.ndarray:
    return log_uniform(uniform(stream, n), dmin, dmax)


def mixed_pool(n_bitmaps: int = 2000, r_bits: int = 1 << 24):
    d = pool_densities(STREAM_MIXED + _QUERY_OFFSET - 1, n_bitmaps, 1e-4, 0.5)
    return bernoulli(STREAM_MIXED, r_bits, d), d


def _queries(stream: int, n_queries: int, pool: int, nmin: int, nmax: int, theta_cap,
             p_interval: float):
    u = uniform(stream, 5 * n_queries).reshape(n_queries, 5)
    ns = log_uniform_int(u[:, 0], nmin, min(nmax, pool))
    out = []
    for q in range(n_queries):
        n = int(ns[q])
        ids = floyd(stream + 1 + q, pool, n)
        cap = n if theta_cap is None else min(n, theta_cap)
        if u[q, 2] < p_interval:
            a = int(uniform_int(u[q, 3], 1, n))
            b = int(uniform_int(u[q, 4], 1, n))
            out.append(Query(ids, KIND_INTERVAL, lo=min(a, b), hi=max(a, b)))
        else:
            out.append(Query(ids, KIND_THRESHOLD, theta=int(uniform_int(u[q, 1], 1, cap))))
    return out


def mixed_queries(n_queries: int = 4096, pool: int = 2000, nmin: int = 3, nmax: int = 1000):
    return _queries(STREAM_MIXED + _QUERY_OFFSET, n_queries, pool, nmin, nmax, None, 0.1)


def sparse_pool(n_bitmaps: int = 5000, r_bits: int = 1 << 24):
    d = pool_densities(STREAM_SPARSE + _QUERY_OFFSET - 1, n_bitmaps, 1e-5, 1e-2)
    words = bernoulli(STREAM_SPARSE, r_bits, d)
    flat, offs = positions(words, r_bits)
    return words, flat, offs, d


def sparse_queries(n_queries: int = 2000, pool: int = 5000, nmin: int = 2, nmax: int = 4096,
                   stream: int = STREAM_SPARSE + _QUERY_OFFSET):
    return _queries(stream, n_queries, pool, nmin, nmax, 64, 0.0)


CLUSTERED_RUNS = (8.0, 64.0, 512.0, 4096.0, 16384.0)


def clustered_pool(n_bitmaps: int = 400, r_bits: int = 1 << 22):
    """Bitmaps in five equal blocks of ids whose ones come in runs of mean
    length 8, 64, 512, 4096 and 16384 rows (geometric, at uniform starts),
    densities log-uniform in [1e-4, 0.5]; with their position lists."""
    d = pool_densities(STREAM_CLUSTERED + _QUERY_OFFSET - 1, n_bitmaps, 1e-4, 0.5)
    words = np.empty((n_bitmaps, words_for(r_bits)), dtype=np.uint64)
    per = n_bitmaps // len(CLUSTERED_RUNS)
    for g, mean in enumerate(CLUSTERED_RUNS):
        lo = g * per
        hi = n_bitmaps if g == len(CLUSTERED_RUNS) - 1 else lo + per
        words[lo:hi] = runs(STREAM_CLUSTERED + lo, r_bits, d[lo:hi], mean)
    flat, offs = positions(words, r_bits)
    return words, flat, offs, d


def clustered_queries(n_queries: int = 300, pool: int = 400, nmin: int = 2, nmax: int = 400,
                      stream: int = STREAM_CLUSTERED + _QUERY_OFFSET):
    """Queries over one block of clustered_pool each (blocks in turn): N
    log-uniform in [nmin, min(nmax, block)], theta uniform in [1, min(N, 64)],
    an interval with probability 0.1."""
    groups = len(CLUSTERED_RUNS)
    per = pool // groups
    by_group = [_queries(stream + (g << 32), (n_queries + groups - 1) // groups, per, nmin,
                         min(nmax, per), 64, 0.1) for g in range(groups)]
    out = []
    for i in range(n_queries):
        g = i % groups
        q = by_group[g][i // groups]
        q.ids = (q.ids + np.uint32(g * per)).astype(np.uint32)
        out.append(q)
    return out


def serving_pool(n_bitmaps: int = 10000, r_bits: int = 1 << 22):
    d = pool_densities(STREAM_SERVING + _QUERY_OFFSET - 1, n_bitmaps, 1e-5, 0.5)
    return bernoulli(STREAM_SERVING, r_bits, d), d


def serving_queries(n_queries: int, rate_qps: float, pool: int = 10000, nmin: int = 2,
                    nmax: int = 4096, stream: int = STREAM_SERVING + _QUERY_OFFSET):
    qs = _queries(stream, n_queries, pool, nmin, nmax, None, 0.0)
    gaps = -np.log1p(-uniform(stream - 2, n_queries)) / rate_qps
    t = np.cumsum(gaps)
    for q, a in zip(qs, t):
        q.arrival_s = float(a)
    return qs
