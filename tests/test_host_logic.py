"""Host-side logic that needs no GPU: input generators, the selector's
time-lost metric, the serving summary and bench.py's bookkeeping."""
from __future__ import annotations

import math

import numpy as np


def test_generators_deterministic_and_independent(dg):
    a = dg.raw64(dg.STREAM_TESTS + 1, 1000)
    b = dg.raw64(dg.STREAM_TESTS + 1, 1000)
    c = dg.raw64(dg.STREAM_TESTS + 2, 1000)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    u = dg.uniform(dg.STREAM_TESTS + 3, 200000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    # Bernoulli bitmaps: per-bitmap density within 6 sigma, rows >= r never set
    r = 100003
    p = np.array([0.0, 1e-3, 0.05, 0.5, 1.0])
    w = dg.bernoulli(dg.STREAM_TESTS + 4, r, p)
    ones = np.array([int(np.unpackbits(x.view(np.uint8)).sum()) for x in w])
    assert ones[0] == 0 and ones[-1] == r
    for k in (1, 2, 3):
        sd = math.sqrt(r * p[k] * (1 - p[k]))
        assert abs(ones[k] - r * p[k]) < 6 * sd + 1
    assert int(w[-1, -1]) == (1 << (r % 64)) - 1
    # runs: at least the target count of ones
    d = dg.config2_density(8)
    wr = dg.runs(dg.STREAM_TESTS + 5, 1 << 16, d)
    for k in range(8):
        assert int(np.unpackbits(wr[k].view(np.uint8)).sum()) >= round(d[k] * (1 << 16))


def test_floyd_and_queries(dg):
    s = dg.floyd(dg.STREAM_TESTS + 6, 1000, 999)
    assert len(set(s.tolist())) == 999 and s.max() < 1000
    qs = dg.mixed_queries(200, 300, nmax=300)
    for q in qs:
        assert 3 <= q.n <= 300 and len(set(q.ids.tolist())) == q.n
        if q.kind == dg.KIND_INTERVAL:
            assert 1 <= q.lo <= q.hi <= q.n
        else:
            assert 1 <= q.theta <= q.n
    sq = dg.sparse_queries(100, 500, nmax=500)
    assert all(1 <= q.theta <= min(q.n, 64) for q in sq)
    sv = dg.serving_queries(500, 1000.0, pool=600, nmax=600)
    t = np.array([q.arrival_s for q in sv])
    assert np.all(np.diff(t) > 0) and abs(len(sv) / t[-1] - 1000.0) < 200.0


def test_clustered_workload(dg):
    """Five blocks of ids with runs of growing mean length: the mean length
    of the runs of ones grows block by block; every query stays inside one
    block, blocks in turn, and its predicate is in range."""
    r, n = 1 << 18, 50
    words, flat, offs, d = dg.clustered_pool(n, r)
    assert words.shape == (n, (r + 63) // 64) and len(offs) == n + 1
    bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")[:, :r].astype(np.int8)
    ones = bits.sum(axis=1)
    starts = np.maximum(np.diff(bits, axis=1), 0).sum(axis=1) + bits[:, 0]
    assert np.array_equal(offs[1:] - offs[:-1], ones.astype(np.uint64))
    per = n // len(dg.CLUSTERED_RUNS)
    mean_run = [ones[g * per:(g + 1) * per].sum() / max(1, starts[g * per:(g + 1) * per].sum())
                for g in range(len(dg.CLUSTERED_RUNS))]
    assert all(a < b for a, b in zip(mean_run, mean_run[1:])), mean_run
    assert np.all((d >= 1e-4) & (d <= 0.5))
    qs = dg.clustered_queries(40, n, nmax=n)
    for i, q in enumerate(qs):
        g = i % len(dg.CLUSTERED_RUNS)
        assert np.all(q.ids // per == g) and len(set(q.ids.tolist())) == len(q.ids)
        if q.kind == dg.KIND_INTERVAL:
            assert 1 <= q.lo <= q.hi <= len(q.ids)
        else:
            assert 1 <= q.theta <= min(len(q.ids), 64)


def test_time_lost_metric():
    from paper_1402_4073_gb300 import selector
    times = np.array([[10.0, 5.0, 7.0, 9.0], [1.0, 2.0, 3.0, 4.0], [4.0, 4.0, 1.0, 8.0]])
    best = np.array([1, 0, 2])
    assert selector.time_lost(times, best) == 0.0
    worst = np.array([0, 3, 3])
    # (10-5) + (4-1) + (8-1) over 5+1+1
    assert abs(selector.time_lost(times, worst) - 15.0 / 7.0) < 1e-12
    # a NaN is a candidate the query cannot run: its row stays, its best is
    # among the others, and a policy choosing it has no time lost
    times[1, 0] = np.nan
    assert abs(selector.time_lost(times, worst) - 14.0 / 8.0) < 1e-12
    assert selector.time_lost(times, np.array([1, 0, 2])) is None


def test_serving_summary():
    from paper_1402_4073_gb300.serve import summarize
    res = {"latency_us": np.array([10.0, 20.0, 30.0, 40.0, 1000.0]),
           "queue_us": np.array([1.0, 2.0, 3.0, 4.0, 5.0]),
           "status": np.array([0, 0, 0, -6, 0], dtype=np.int32), "wall_s": 2.0}
    s = summarize(res, 3.0)
    assert s["completed"] == 4 and s["refused"] == 1 and s["errors"] == 0
    assert s["achieved_qps"] == 2.0 and s["p50_us"] == 25.0
    assert s["p99_us"] > 900.0


def test_bench_bookkeeping():
    import bench
    assert bench.query_bytes(256, 1 << 26) == 2155872256  # N*r/8 + r/8
    peak, src = bench.peaks()
    assert peak > 0 and src in ("measured", "fallback")
    assert len(bench.sources_sha()) == 16
