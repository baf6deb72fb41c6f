#!/usr/bin/env python
"""Threshold-query throughput on the large dense workload.

Workload: N = 256 bitmaps of r = 2^26 rows (2 GiB resident in HBM), bitmap k
of density max(0.5/k, 1e-4) with its ones in geometric runs (mean 8); one
step runs the four queries theta = 2, 128, 255 and the interval [2, 10].
Metric: input GB/s = sum over queries of (N * r/8 + r/8) bytes / step time.
Inputs (2.15 GB per query) exceed the 129 MB L2, so no flush is needed
between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs the same workload on its own GPU (independent
queries, weak scaling); the step time is the maximum over ranks.  The
``reference`` arm times the CPU oracle on the host cores on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

R_BITS = 1 << 26
N = 256
WORKLOAD = "large dense: N=256 bitmaps x r=2^26 rows, densities max(0.5/k,1e-4) in geometric runs; " \
           "queries theta=2,128,255 and interval [2,10]"
METRIC = "threshold-query input GB/s"
DENSE_SOURCES = ["paper_1402_4073_gb300/csrc/bm_dense.cu", "paper_1402_4073_gb300/csrc/bm_device.cuh",
                 "paper_1402_4073_gb300/csrc/bm_dense_common.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dense_csa_n256_r2e26.txt")


def query_bytes(n: int, r_bits: int) -> int:
    """Algorithmic bytes of one query: n inputs read plus one output written."""
    return n * r_bits // 8 + r_bits // 8


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def alu_peak_ops() -> float:
    """Integer lane-ops per second of one GB300: SMs x 64 int32 lanes per SM
    per clock x the maximum SM clock (2070 MHz)."""
    return 152 * 64 * 2.07e9


def sources_sha() -> str:
    h = hashlib.sha256()
    for s in DENSE_SOURCES:
        h.update(open(os.path.join(ROOT, s), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_launch():
    """dram bytes per dense launch from the committed ncu summary, if it was
    taken on the current kernel sources."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    kv = {}
    for line in open(TRAFFIC_FILE):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != sources_sha():
        return None
    try:
        return int(float(kv["dram_bytes_per_launch"]))
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.device), "-lms", "50", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup(backend: str):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return rank, world, local


def cpu_sample_time(words, queries, r_bits, budget_s: float):
    """Time the oracle on a bounded prefix of words, grown until it takes
    about budget_s seconds; returns (bytes per second, sample words, seconds,
    the oracle's answers over that prefix)."""
    import oracle
    nw = 256
    while True:
        t0 = time.perf_counter()
        answers = [oracle.query(words, q, r_bits, 0, nw) for q in queries]
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or nw >= words.shape[1]:
            break
        nw = min(words.shape[1], nw * 4)
    rows = 64 * nw
    nbytes = sum(query_bytes(q.n, rows) for q in queries)
    return nbytes / dt, nw, dt, answers


def oracle_check(bm, outs, cards, answers, nw, total_words):
    """Compare the timed run's outputs with the oracle's answers over the
    sampled prefix of nw words (and the cardinalities when the sample covers
    every word)."""
    cards_h = cards.cpu().numpy()
    words_ok = all(np_equal(bm.to_numpy_words(o)[:nw], a[0]) for o, a in zip(outs, answers))
    full = nw >= total_words
    cards_ok = (not full) or all(int(c) == a[1] for c, a in zip(cards_h, answers))
    return {"checked_vs_oracle": bool(words_ok and cards_ok and full),
            "oracle_check": f"output words 0..{nw} of {total_words} of every query "
                            f"{'equal' if words_ok else 'DIFFER'}; cardinalities "
                            f"{('equal' if cards_ok else 'DIFFER') if full else 'not compared (prefix)'}"}


def np_equal(a, b) -> bool:
    import numpy as np
    return bool(np.array_equal(a, b))


def bench_batched(bm, datagen, passes: int = 2, small: bool = False, config: str = ""):
    """Mixed batch (2000 x 2^24 pool, 4096 queries): plain one query per
    launch vs one batched graph replay; queries/s of each.  small: 400 x 2^22
    pool and 512 queries (for profiling only).  config: "ctas,adder,words"
    for the batch kernel instead of the autotuner (the only batch launches are
    then the warm-up replay and the timed ones)."""
    import torch
    r_bits, nbm, nq = (1 << 22, 400, 512) if small else (1 << 24, 2000, 4096)
    words, _ = datagen.mixed_pool(nbm, r_bits)
    queries = datagen.mixed_queries(nq, nbm, nmax=min(1000, nbm))
    pool = bm.Pool(r_bits, nbm)
    pool.put_dense(words)
    del words
    if config:
        pool.set_batch_config(*[int(x) for x in config.split(",")])
        tune = f"batch fixed by --batch-config {config}"
    else:
        tune = pool.autotune()
    outs = [pool.empty_words() for _ in queries]
    cards_plain = torch.zeros(len(queries), dtype=torch.int64, device="cuda")
    cards_batch = torch.zeros(len(queries), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    singles = [bm.PreparedQuery(pool, q, outs[i], bm.PATH_DENSE) for i, q in enumerate(queries)]
    card_views = [cards_plain[i:i + 1] for i in range(len(queries))]

    def plain():
        for sq, c in zip(singles, card_views):
            sq.run(c)

    prepared = bm.PreparedBatch(pool, queries, outs, paths=[bm.PATH_DENSE] * len(queries))

    def batched():
        prepared.run(cards_batch)

    def timed(fn):
        fn()  # warm-up (graph capture on first use)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(passes):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return best

    t_plain = timed(plain)
    t_batch = timed(batched)
    same = bool(torch.equal(cards_plain, cards_batch))
    pool.status()
    logical = sum(query_bytes(q.n, r_bits) for q in queries)
    # integer roofline: ~2 three-input logic ops per 32-bit input word (one
    # full adder per input in the sideways-sum tree, Sec. 4.3), against
    # SMs x 64 int32 lanes x the maximum SM clock
    ops = sum(2 * q.n * ((r_bits + 31) // 32) for q in queries)
    peak_ops = alu_peak_ops()
    pool.close()
    return {"alu_roofline": {"bound": "alu", "achieved_Tops": round(ops / t_batch / 1e12, 2),
                             "peak_Tops": round(peak_ops / 1e12, 2),
                             "frac": round(ops / t_batch / peak_ops, 4),
                             "ops": "2 LOP3 per 32-bit input word",
                             "peak_source": "152 SMs x 64 int32 lanes x 2070 MHz (recipe unit counts)"},
            "workload": f"mixed: {nbm} x 2^{r_bits.bit_length() - 1} pool (densities log-uniform "
                        f"[1e-4,0.5]), {nq} queries N log-uniform [3,{min(1000, nbm)}], 10% intervals",
            "plain_queries_per_s": round(len(queries) / t_plain, 1),
            "batched_queries_per_s": round(len(queries) / t_batch, 1),
            "speedup": round(t_plain / t_batch, 3),
            "plain_logical_GBps": round(logical / t_plain / 1e9, 1),
            "batched_logical_GBps": round(logical / t_batch / 1e9, 1),
            "cardinalities_equal": same, "timing": f"best of {passes} passes, CUDA events",
            "autotune": tune}


def bench_selector_clustered(bm, datagen, small: bool = False):
    """The selector with the run-length path among its candidates: a pool of
    five blocks of bitmaps whose ones come in runs of mean 8 .. 16384 rows
    (dense words, position lists and run-length forms of all), each query's
    ids from one block.  Trained on its own timings of separate training
    queries; time lost on the test queries for the network, for the library's
    rule without a network (density rule, then the run-length cost model)
    and for fixed candidates, and how often each candidate is the fastest and
    the network's pick."""
    import numpy as np
    from paper_1402_4073_gb300 import selector
    r_bits, nbm, nq = ((1 << 20), 200, 150) if small else ((1 << 22), 400, 300)
    words, flat, offs, _ = datagen.clustered_pool(nbm, r_bits)
    test_q = datagen.clustered_queries(nq, nbm)
    train_q = datagen.clustered_queries(nq, nbm, stream=datagen.STREAM_CLUSTERED + (7 << 36))
    pool = bm.Pool(r_bits, nbm)
    pool.put_dense(words)
    pool.put_positions(flat, offs)
    pool.put_rle()
    del words, flat
    tune = pool.autotune()
    ftr, ttr = selector.collect(pool, train_q, reps=3)
    fte, tte = selector.collect(pool, test_q, reps=3)
    model = selector.train(ftr, ttr, steps=3000)
    res = selector.evaluate(pool, model, test_q, fte, tte)
    pool.status()
    pool.close()
    out = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in res.items()}
    out.update({"workload": f"clustered: {nbm} x 2^{r_bits.bit_length() - 1} pool, five blocks "
                            "with runs of mean 8..16384 rows (densities log-uniform [1e-4,0.5]; "
                            f"dense + lists + run-length forms), {nq} queries from one block "
                            "each, N log-uniform [2,block], theta<=min(N,64), 10% intervals",
                "candidates": ["dense", "sparse16k", "sparse32k", "sparse64k", "dense1w", "rle"],
                "fastest_choices": np.bincount(np.nanargmin(tte, axis=1),
                                               minlength=bm.SELECTOR_CANDIDATES).tolist(),
                "train_queries": nq, "final_train_loss": round(model.final_loss, 5),
                "autotune": tune})
    return out


def bench_selector(bm, datagen, n_train: int = 600, small: bool = False):
    """Sparse workload (5000 x 2^24, dense + lists; 2000 queries): train the
    selector on its own timings of separate training queries, then report
    time lost on the 2000 workload queries for the network and the fixed
    rule, and queries/s of the batched+selected form vs plain dense."""
    import torch
    from paper_1402_4073_gb300 import selector
    r_bits, nbm, nq = (1 << 22, 800, 300) if small else (1 << 24, 5000, 2000)
    if small:
        n_train = 100
    words, flat, offs, _ = datagen.sparse_pool(nbm, r_bits)
    test_q = datagen.sparse_queries(nq, nbm, nmax=min(4096, nbm))
    train_q = datagen.sparse_queries(n_train, nbm, nmax=min(4096, nbm),
                                     stream=datagen.STREAM_SPARSE + (7 << 32))
    pool = bm.Pool(r_bits, nbm)
    pool.put_dense(words)
    pool.put_positions(flat, offs)
    del words, flat
    tune = pool.autotune()
    ftr, ttr = selector.collect(pool, train_q, reps=3)
    fte, tte = selector.collect(pool, test_q, reps=3)
    t0 = time.perf_counter()
    model = selector.train(ftr, ttr, steps=3000)
    train_s = time.perf_counter() - t0
    res = selector.evaluate(pool, model, test_q, fte, tte)
    selector.install(pool, model)
    outs = [pool.empty_words() for _ in test_q]
    cards_a = torch.zeros(len(test_q), dtype=torch.int64, device="cuda")
    cards_b = torch.zeros(len(test_q), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, passes=2):
        fn()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(passes):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return best

    singles = [bm.PreparedQuery(pool, q, outs[i], bm.PATH_DENSE) for i, q in enumerate(test_q)]
    card_views = [cards_a[i:i + 1] for i in range(len(test_q))]
    t_plain = timed(lambda: [sq.run(c) for sq, c in zip(singles, card_views)])
    chosen = []
    prepared = bm.PreparedBatch(pool, test_q, outs)  # PATH_AUTO: the installed selector routes
    t_sel = timed(lambda: chosen.append(prepared.run(cards_b).copy()))
    same = bool(torch.equal(cards_a, cards_b))
    pool.status()
    pool.close()
    out = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in res.items()}
    out.update({"workload": f"sparse: {nbm} x 2^{r_bits.bit_length() - 1} pool (densities log-uniform "
                            f"[1e-5,1e-2], dense + position lists), {nq} queries N log-uniform "
                            f"[2,{min(4096, nbm)}], theta<=min(N,64)",
                "train_queries": n_train, "train_steps": 3000, "train_s": round(train_s, 2),
                "final_train_loss": round(model.final_loss, 5),
                "plain_dense_queries_per_s": round(len(test_q) / t_plain, 1),
                "batched_selected_queries_per_s": round(len(test_q) / t_sel, 1),
                "speedup": round(t_plain / t_sel, 3),
                "sparse_share": round(float((chosen[-1] == bm.PATH_SPARSE).mean()), 3),
                "cardinalities_equal": same, "autotune": tune})
    return out


def bench_sparse(bm, datagen, reps: int = 20, small: bool = False, config: str = ""):
    """ScanCount alone (Sec. 4.2): single queries over the position lists of a
    1500 x 2^24 pool (densities log-uniform [1e-5,1e-2]); N = 1500, 537, 128
    and 16 random lists, theta = min(N, 8).  Per N: CUDA-event time per
    launch and its fraction of the HBM peak for the algorithmic bytes 4 B +
    r/8 (B = listed positions read, the output written).  small: 2^22 rows."""
    import numpy as np
    import torch
    r_bits, nbm = ((1 << 22) if small else (1 << 24)), 1500
    words, flat, offs, _ = datagen.sparse_pool(nbm, r_bits)
    pool = bm.Pool(r_bits, nbm)
    pool.put_dense(words)
    pool.put_positions(flat, offs)
    del words, flat
    if config:
        pool.set_sparse_config(*[int(x) for x in config.split(",")])
        tune = "fixed by --sparse-config"
    else:
        tune = pool.autotune()
    lens = offs[1:].astype(np.int64) - offs[:-1].astype(np.int64)
    peak, peak_src = peaks()
    out = pool.empty_words()
    card = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rows = []
    for n in (1500, 537, 128, 16):
        ids = datagen.floyd(datagen.STREAM_SPARSE + (9 << 32) + n, nbm, n)
        q = datagen.Query(ids, datagen.KIND_THRESHOLD, theta=min(n, 8))
        pq = bm.PreparedQuery(pool, q, out, bm.PATH_SPARSE)
        for _ in range(3):
            pq.run(card)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        torch.cuda.synchronize()
        for i in range(reps):
            ev[2 * i].record(stream)
            pq.run(card)
            ev[2 * i + 1].record(stream)
        torch.cuda.synchronize()
        us = statistics.median(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(reps)) * 1e3
        b = int(lens[ids].sum())
        alg = 4 * b + r_bits // 8
        # device time per call on each tile size the selector can pick
        tuned = pool.configs()["sparse"]
        by_tile = {}
        for tile in (16384, 32768, 65536):
            pool.set_sparse_config(tile, tuned["threads"], tuned["ctas_per_sm"], tuned["unroll"])
            by_tile[tile] = call_times(lambda: pq.run(card), reps, flush)
        pool.set_sparse_config(**tuned)
        best = min(by_tile, key=lambda t: by_tile[t][0])
        cold, hot = by_tile[best]
        rows.append({"N": n, "positions": b, "us_per_query": round(us, 1),
                     "achieved_GBps": round(alg / us / 1e3, 1),
                     "frac": round(alg / us / 1e3 / peak, 4),
                     "tile_rows": best, "cold_us": round(cold, 2),
                     "cold_frac": round(alg / cold / 1e3 / peak, 4), "hot_us": round(hot, 2),
                     "cold_us_by_tile": {str(t): round(v[0], 2) for t, v in by_tile.items()}})
    pool.status()
    pool.close()
    cos = bench_cosparse(bm, datagen, r_bits, nbm, reps, peak, config)
    return {"workload": f"sparse single queries: {nbm} x 2^{r_bits.bit_length() - 1} pool "
                        "(densities log-uniform [1e-5,1e-2], position lists), theta=min(N,8)",
            "kernel": "ScanCount (scancount_kernel)", "bytes": "4 * positions + r/8 per query",
            "peak": peak, "peak_source": f"hbm_gbs of {peak_src}",
            "timing": f"us_per_query / frac: median of {reps} launches of the tuned tile, CUDA "
                      "events around each bm_query_run (host time inside); cold/hot (as in the "
                      "small part) on the best of the selector's three tile sizes",
            "queries": rows, "autotune": tune, "co_sparse": cos}


def bench_cosparse(bm, datagen, r_bits, nbm, reps, peak, config=""):
    """Co-sparse pool: half the bitmaps of density d, half of density 1 - d
    (d log-uniform [1e-5,1e-2]); the dense half loaded as lists of their zeros
    (complement identity, Sec. 2.3).  Random queries of N = 1500, 537, 128,
    16 ids, theta = N/2 + 1, on ScanCount and on the dense path."""
    import numpy as np
    import torch
    half = nbm // 2
    d = datagen.pool_densities(datagen.STREAM_SPARSE + (11 << 32), nbm, 1e-5, 1e-2)
    d[half:] = 1.0 - d[half:]
    words = datagen.bernoulli(datagen.STREAM_SPARSE + (12 << 32), r_bits, d)
    flat1, offs1 = datagen.positions(words[:half], r_bits)
    comp = ~words[half:]
    if r_bits % 64:
        comp[:, -1] &= np.uint64((1 << (r_bits % 64)) - 1)
    flat0, offs0 = datagen.positions(comp, r_bits)
    del comp
    pool = bm.Pool(r_bits, nbm)
    pool.put_dense(words)
    del words
    pool.put_positions(flat1, offs1)
    pool.put_positions(flat0, offs0, first_id=half, zeros=True)
    if config:
        pool.set_sparse_config(*[int(x) for x in config.split(",")])
    else:
        pool.autotune()
    lens = np.concatenate([offs1[1:].astype(np.int64) - offs1[:-1].astype(np.int64),
                           offs0[1:].astype(np.int64) - offs0[:-1].astype(np.int64)])
    del flat1, flat0
    out = pool.empty_words()
    card = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rows = []
    for n in (1500, 537, 128, 16):
        ids = datagen.floyd(datagen.STREAM_SPARSE + (13 << 32) + n, nbm, n)
        q = datagen.Query(ids, datagen.KIND_THRESHOLD, theta=n // 2 + 1)
        t = {}
        for path in (bm.PATH_SPARSE, bm.PATH_DENSE):
            pq = bm.PreparedQuery(pool, q, out, path)
            for _ in range(3):
                pq.run(card)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
            torch.cuda.synchronize()
            for i in range(reps):
                ev[2 * i].record(stream)
                pq.run(card)
                ev[2 * i + 1].record(stream)
            torch.cuda.synchronize()
            t[path] = statistics.median(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(reps)) * 1e3
        b = int(lens[ids].sum())
        alg = 4 * b + r_bits // 8
        rows.append({"N": n, "inputs_by_zeros": int((ids >= half).sum()), "listed_positions": b,
                     "sparse_us": round(t[bm.PATH_SPARSE], 1), "dense_us": round(t[bm.PATH_DENSE], 1),
                     "sparse_frac": round(alg / t[bm.PATH_SPARSE] / 1e3 / peak, 4)})
    pool.status()
    pool.close()
    return {"workload": f"co-sparse: {nbm} x 2^{r_bits.bit_length() - 1} pool, half of density d, "
                        "half 1 - d (d log-uniform [1e-5,1e-2]) given by their zeros; theta = N/2 + 1",
            "queries": rows}


def bench_rle(bm, datagen, reps: int = 10, small: bool = False):
    """Run-length form with clean-run pruning (Sec. 2.1, 4.1) against the dense
    path on the same pools: N = 256 bitmaps of r = 2^26 rows, densities
    max(0.5/k, 1e-4), ones in runs of mean 4096, 256 and 8 rows; the four
    queries of the main benchmark.  Per pool and query: device time per call
    on each path (call_times: L2 flushed before each call; and back to back
    for the run-length path), logical input GB/s (N r/8 + r/8 per
    query), and for the run-length path its algorithmic bytes (the inputs'
    run-length forms: one 8-byte summary per input and tile and the
    containers of the mixed tiles; plus r/8 written) and their fraction of
    the HBM peak.
    small: r = 2^22."""
    import numpy as np
    import torch
    r_bits, n = ((1 << 22) if small else (1 << 26)), 256
    ids = np.arange(n, dtype=np.uint32)
    queries = [datagen.Query(ids, datagen.KIND_THRESHOLD, theta=2),
               datagen.Query(ids, datagen.KIND_THRESHOLD, theta=128),
               datagen.Query(ids, datagen.KIND_THRESHOLD, theta=255),
               datagen.Query(ids, datagen.KIND_INTERVAL, lo=2, hi=10)]
    peak, peak_src = peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2
    pools = []
    for mean_run in (4096.0, 256.0, 8.0):
        words = datagen.runs(datagen.STREAM_CONFIG2, r_bits, datagen.config2_density(n), mean_run)
        pool = bm.Pool(r_bits, n)
        pool.put_dense(words)
        del words
        pool.put_rle()
        runs = lits = stored = 0
        for k in range(n):
            a, b = pool.rle_info(k)
            runs, lits, stored = runs + a, lits + b, stored + pool.rle_bytes(k)
        # the inputs' run-length forms (summaries, containers) + the output
        alg = stored + r_bits // 8
        out = pool.empty_words()
        card = torch.zeros(1, dtype=torch.int64, device="cuda")
        rows = []
        for q in queries:
            t, hot = {}, {}
            for path in (bm.PATH_DENSE, bm.PATH_RLE):
                pq = bm.PreparedQuery(pool, q, out, path)
                t[path], hot[path] = call_times(lambda: pq.run(card), reps, flush)
            logical = query_bytes(n, r_bits)
            rows.append({"query": f"theta={q.theta}" if q.kind == 0 else f"[{q.lo},{q.hi}]",
                         "dense_us": round(t[bm.PATH_DENSE], 1), "rle_us": round(t[bm.PATH_RLE], 1),
                         "rle_hot_us": round(hot[bm.PATH_RLE], 1),
                         "dense_logical_GBps": round(logical / t[bm.PATH_DENSE] / 1e3, 1),
                         "rle_logical_GBps": round(logical / t[bm.PATH_RLE] / 1e3, 1),
                         "rle_achieved_GBps": round(alg / t[bm.PATH_RLE] / 1e3, 1),
                         "rle_frac": round(alg / t[bm.PATH_RLE] / 1e3 / peak, 4)})
        pool.status()
        # what BM_PATH_AUTO takes for these single queries (run-length or dense)
        auto = {bm.PATH_DENSE: "dense", bm.PATH_SPARSE: "sparse", bm.PATH_RLE: "rle"}
        pools.append({"mean_run_rows": mean_run, "runs": runs, "literal_words": lits,
                      "rle_bytes_per_query": alg, "dense_bytes_per_query": query_bytes(n, r_bits),
                      "auto_path": auto.get(bm.query_select(pool, queries[0])[0], "?"),
                      "queries": rows})
        pool.close()
    return {"workload": f"clustered dense: N={n} bitmaps x r=2^{r_bits.bit_length() - 1} rows, "
                        "densities max(0.5/k,1e-4), ones in runs of the given mean length",
            "kernel": "rle_kernel (run-length form, clean-run pruning)",
            "peak": peak, "peak_source": f"hbm_gbs of {peak_src}",
            "timing": f"device time per bm_query_run: median of {reps} calls, each behind a "
                      "256 MiB fill (L2 flushed, host submission hidden); rle_hot_us: calls back "
                      "to back",
            "pools": pools}


def call_times(call, reps: int, flush):
    """Device time per call of `call` (one query through the C ABI):
    cold = median over `reps` calls, each queued behind a write of `flush`
    (larger than L2), so the interval between its events holds its GPU work
    and no host gap; hot = mean over `reps` calls queued back to back behind
    a sleep kernel (the per-call cost of a stream of calls).  Microseconds."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(3):
        call()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    torch.cuda.synchronize()
    for i in range(reps):
        flush.fill_(i & 255)
        ev[2 * i].record(stream)
        call()
        ev[2 * i + 1].record(stream)
    torch.cuda.synchronize()
    cold = statistics.median(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(reps)) * 1e3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda._sleep(4_000_000)  # about 2 ms: the host queues the calls meanwhile
    e0.record(stream)
    for _ in range(reps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    return cold, e0.elapsed_time(e1) * 1e3 / reps


def bench_small(bm, datagen, reps: int = 40):
    """Launch-bound single queries: the plain dense workload (N = 16 bitmaps
    of r = 2^20 rows, Bernoulli(0.1); theta = 3, theta = 8 and the interval
    [2, 5]) and dense N = 16 and N = 64 over r = 2^24 rows (the same
    density).  Per query, device time per call:
      cold: L2 flushed before each call by writing a 256 MiB buffer (larger
            than the 129 MB L2); the call is queued behind the flush, so the
            interval between its events holds its GPU work and no host gap;
      hot:  `reps` calls queued back to back behind a sleep kernel (inputs
            stay in L2): the per-call cost of a stream of calls.
    GB/s = (N r/8 + r/8) per call; the fraction is of the HBM copy peak."""
    import numpy as np
    import torch
    peak, peak_src = peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    card = torch.zeros(1, dtype=torch.int64, device="cuda")
    cases = []
    words1, queries1 = datagen.config1()
    cases.append(("plain dense N=16 x r=2^20", 1 << 20, words1, queries1))
    for n in (16, 64):
        w = datagen.bernoulli(datagen.STREAM_CONFIG1 + (5 << 32) + n, 1 << 24, [0.1] * n)
        cases.append((f"dense N={n} x r=2^24", 1 << 24, w,
                      [datagen.Query(np.arange(n, dtype=np.uint32), 0, theta=3)]))
    rows = []
    for name, r_bits, words, queries in cases:
        pool = bm.Pool(r_bits, words.shape[0])
        pool.put_dense(words)
        pool.autotune()
        out = pool.empty_words()
        for q in queries:
            def call():
                if q.kind == 0:
                    bm.threshold(pool, q.ids, q.theta, out, card)
                else:
                    bm.interval(pool, q.ids, q.lo, q.hi, out, card)
            cold, hot = call_times(call, reps, flush)
            nbytes = query_bytes(q.n, r_bits)
            rows.append({"case": name,
                         "query": f"theta={q.theta}" if q.kind == 0 else f"[{q.lo},{q.hi}]",
                         "cold_us": round(cold, 2), "hot_us": round(hot, 2),
                         "cold_GBps": round(nbytes / cold / 1e3, 1),
                         "cold_frac": round(nbytes / cold / 1e3 / peak, 4),
                         "hot_GBps": round(nbytes / hot / 1e3, 1)})
        pool.status()
        pool.close()
    return {"workload": "plain dense N=16 x r=2^20 (theta=3, 8, [2,5]); dense N=16, 64 x r=2^24",
            "timing": f"cold: median of {reps} calls, each after a 256 MiB write (L2 flushed); "
                      f"hot: {reps} calls back to back after a sleep kernel, mean",
            "peak": peak, "peak_source": f"hbm_gbs of {peak_src}", "queries": rows}


def bench_looped(bm, pool, queries, launch, cards, reps: int = 20):
    """The main workload's plain thresholds with T or N - T + 1 at most 3
    (theta = 2 and theta = 255 of N = 256) on the Looped recurrence (Sec. 4.4;
    theta = 255 through the complement identity) and on the counter planes,
    median of reps launches each (CUDA events; inputs larger than L2)."""
    import torch
    stream = torch.cuda.current_stream()
    peak, peak_src = peaks()

    def timed(i, q):
        for _ in range(3):
            launch(i, q)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        torch.cuda.synchronize()
        for k in range(reps):
            ev[2 * k].record(stream)
            launch(i, q)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        return statistics.median(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps)) * 1e3

    rows = []
    for i, q in enumerate(queries):
        t = min(q.theta, q.n - q.theta + 1) if q.kind == 0 else 0
        if not 1 <= t <= 3:
            continue
        row = {"theta": q.theta, "n": q.n, "t": t}
        got = {}
        for max_t, name in ((0, "counter_us"), (3, "looped_us")):
            pool.set_looped(max_t)
            row[name] = round(timed(i, q), 1)
            torch.cuda.synchronize()
            got[max_t] = int(cards[i].item())
        row["cards_equal"] = got[0] == got[3]
        gbps = query_bytes(q.n, R_BITS) / row["looped_us"] / 1e3
        row["looped_GBps"] = round(gbps, 1)
        row["looped_frac"] = round(gbps / peak, 4)
        rows.append(row)
    pool.set_looped(0)
    pool.status()
    return {"workload": WORKLOAD, "kernel": "looped_kernel<t,neg> vs the counter's pick",
            "peak": f"hbm_gbs of {peak_src}", "timing": f"median of {reps} launches, CUDA events",
            "queries": rows}


def bench_weighted(bm, datagen, reps: int = 5, small: bool = False):
    """Weighted thresholds (Sec. 2.3) on the main benchmark's pool (N = 256 bitmaps of
    r = 2^26 rows): weights uniform in [1, wmax] for wmax = 4, 1000 and 2^20, theta =
    sum / 8, alone and ANDed with bitmap 0; for wmax = 4 also the same query as
    replicated ids through the dense threshold.  small: r = 2^22."""
    import numpy as np
    import torch
    r_bits, n = ((1 << 22) if small else (1 << 26)), 256
    words, _ = datagen.config2(r_bits, n)
    pool = bm.Pool(r_bits, n)
    pool.put_dense(words)
    del words
    pool.set_dense_config(0, 256, 4, 2, 2, 2)
    peak, _ = peaks()
    ids = np.arange(n, dtype=np.uint32)
    out = pool.empty_words()
    card = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        torch.cuda.synchronize()
        for i in range(reps):
            ev[2 * i].record(stream)
            fn()
            ev[2 * i + 1].record(stream)
        torch.cuda.synchronize()
        return statistics.median(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(reps)) * 1e3

    rows = []
    for wmax in (4, 1000, 1 << 20):
        u = datagen.uniform(datagen.STREAM_TESTS + 777, n)
        w = np.maximum(1, (u * wmax).astype(np.int64)).astype(np.uint32)
        total = int(w.astype(np.uint64).sum())
        theta = total // 8
        row = {"wmax": wmax, "sum": total, "theta": theta,
               "weighted_us": round(timed(lambda: bm.weighted_threshold(pool, ids, w, theta, out, card)), 1),
               "weighted_and_us": round(timed(lambda: bm.weighted_threshold(pool, ids, w, theta, out, card,
                                                                            bm.POST_AND, 0)), 1)}
        if total <= bm.BM_N_MAX:
            rep = np.repeat(ids, w)
            row["replicated_ids_us"] = round(timed(lambda: bm.threshold(pool, rep, theta, out, card)), 1)
        gbps = query_bytes(n, r_bits) / row["weighted_us"] / 1e3
        row["input_GBps"] = round(gbps, 1)
        row["hbm_frac"] = round(gbps / peak, 4)
        # integer work: small weights run as copies (2 logic ops per input word
        # through the sideways-sum blocks); otherwise weight-1 inputs cost 2 and
        # each other input 3 per plane of the sum (carry-save full adders)
        lanes = (r_bits + 31) // 32
        if total <= bm.BM_N_MAX and total <= 8 * n:
            ops = 2 * total * lanes
        else:
            n1 = int((w == 1).sum())
            ops = (2 * n1 + 3 * total.bit_length() * int((w > 1).sum())) * lanes
        row["alu_frac"] = round(ops / (row["weighted_us"] * 1e-6) / alu_peak_ops(), 4)
        rows.append(row)
    pool.status()
    pool.close()
    return {"workload": f"weighted: the main pool (N={n} x r=2^{r_bits.bit_length() - 1}), "
                        "weights uniform in [1, wmax], theta = sum/8",
            "kernel": "weighted_kernel (bit-sliced weighted add)",
            "timing": f"median of {reps} calls, CUDA events", "queries": rows}


def bench_serving(bm, datagen, rates=(1000, 5000, 10000, 20000, 50000), seconds: float = 0.8,
                  small: bool = False):
    """Serving loop on the 10,000 x 2^22 pool: Poisson arrivals at each
    offered rate; p50/p99 latency and achieved queries/s.  small: 1000
    bitmaps, two rates, 300 requests each (for profiling only)."""
    from paper_1402_4073_gb300.serve import Server, summarize
    r_bits, nbm = 1 << 22, (1000 if small else 10000)
    if small:
        rates, seconds = (1000, 10000), 0.03
    words, _ = datagen.serving_pool(nbm, r_bits)
    pool = bm.Pool(r_bits, nbm)
    pool.put_dense(words)
    del words
    tune = pool.autotune()
    out, results, slo = [], [], 0
    slot = (pool.words * 8 + 255) // 256 * 256
    # two batches of up to 2048 in flight: under overload, larger batches share each slab
    # of the pool among more queries (saturation 28.5k q/s at 512, 31.2k at 1024, 33.1k
    # at 2048, with the same latency below saturation)
    with Server(pool, mem_budget=4096 * slot, max_batch=2048, max_inflight=2) as srv:
        # warm-up: graph capture and caches
        warm = datagen.serving_queries(256, 50000.0, pool=nbm, nmax=min(4096, nbm),
                                       stream=datagen.STREAM_SERVING + (9 << 32))
        srv.replay(warm, [q.arrival_s for q in warm])
        for k, rate in enumerate(rates):
            n = int(min(40000, max(300 if small else 500, rate * seconds)))
            qs = datagen.serving_queries(n, float(rate), pool=nbm, nmax=min(4096, nbm),
                                         stream=datagen.STREAM_SERVING + ((10 + k) << 32))
            res = srv.replay(qs, [q.arrival_s for q in qs])
            summ = summarize(res, float(rate))
            summ["requests"] = n
            out.append(summ)
            if k == 0:
                # the latency objective: ten times the p99 at the lowest offered rate
                slo = int(10 * summ["p99_us"])
            results.append(res)
        st = srv.stats()
    for summ, res in zip(out, results):
        summ.update({k2: v for k2, v in summarize(res, summ["offered_qps"], slo).items()
                     if k2 in ("slo_us", "within_slo", "goodput_qps")})
    # the same arrivals with load shedding by the objective (overloaded rates)
    shed = []
    with Server(pool, mem_budget=4096 * slot, max_batch=2048, max_inflight=2, slo_us=slo) as srv:
        srv.replay(warm, [q.arrival_s for q in warm])
        for k, rate in enumerate(rates):
            if rate < 20000:
                continue
            n = int(min(40000, max(300 if small else 500, rate * seconds)))
            qs = datagen.serving_queries(n, float(rate), pool=nbm, nmax=min(4096, nbm),
                                         stream=datagen.STREAM_SERVING + ((10 + k) << 32))
            res = srv.replay(qs, [q.arrival_s for q in qs])
            summ = summarize(res, float(rate), slo)
            summ["requests"] = n
            shed.append(summ)
    pool.status()
    pool.close()
    return {"workload": f"serving: {nbm} x 2^22 pool (densities log-uniform [1e-5,0.5]), Poisson "
                        f"arrivals, N log-uniform [2,{min(4096, nbm)}], theta uniform [1,N]",
            "admission": "4096 result slots (2 GiB); max batch 2048; 2 batches in flight",
            "mean_batch": round(st["batched_queries"] / max(1, st["batches"]), 1),
            "autotune": tune, "rates": out,
            "slo": f"{slo} us = 10 x p99 at the lowest offered rate; goodput = requests "
                   "completed within it per second",
            "rates_with_shedding": shed}


def oracle_threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    import oracle
    return oracle.threads()


def run_reference(args):
    rank, world, _ = dist_setup("gloo")
    if rank != 0:
        return
    import datagen
    import oracle
    oracle.build()
    datagen.build()
    # a launcher may limit each rank to one thread; rank 0 alone runs, on every core
    oracle.set_threads(os.cpu_count() or 1)
    words, queries = datagen.config2(R_BITS, N)
    cores = oracle_threads()
    # one step = the four queries over a fixed prefix of words, sized so that
    # the whole run (warm-up + timed steps) takes about two minutes
    per_step_s = min(1.0, 120.0 / max(1, args.steps + args.warmup))
    _, nw, dt, _ = cpu_sample_time(words, queries, R_BITS, 2.0)
    nw = max(64, int(nw * min(8.0, per_step_s / max(dt, 1e-3))))
    nw = min(nw, words.shape[1])
    for _ in range(args.warmup):
        for q in queries:
            oracle.query(words, q, R_BITS, 0, nw)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for q in queries:
            oracle.query(words, q, R_BITS, 0, nw)
    el = time.perf_counter() - t0
    step_bytes = sum(query_bytes(q.n, 64 * nw) for q in queries)
    value = step_bytes * args.steps / el / 1e9
    sample = f"first {nw} of {words.shape[1]} words ({64 * nw} rows) of each of the 4 queries per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * el / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "r_bits": R_BITS, "queries_per_step": 4},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=10.0,
                    help="seconds of oracle work for the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--r-log2", type=int, default=26,
                    help="rows = 2^r_log2 (smaller cases are for profiling only)")
    ap.add_argument("--dense-config", default="",
                    help="variant,threads,stages,ctas_per_sm[,adder]: skip the variant search")
    ap.add_argument("--parts", default="dense,small,looped,sparse,rle,weighted,batch,selector,serving",
                    help="comma list of dense, small, looped, sparse, rle, weighted, batch, selector, "
                         "serving")
    ap.add_argument("--sparse-config", default="",
                    help="tile_rows,threads,ctas_per_sm,unroll for the sparse part: skip tuning")
    ap.add_argument("--batch-config", default="",
                    help="ctas_per_sm,adder,words_per_thread for the batch part: skip tuning")
    ap.add_argument("--small", action="store_true",
                    help="scaled-down batch/selector/serving workloads (profiling only)")
    ap.add_argument("--shard", default="none", choices=["none", "rows"],
                    help="rows: under torchrun, split the rows of every bitmap across the ranks "
                         "(strong scaling: one query's work shared by all GPUs, cardinalities "
                         "summed by one all-reduce per step); the other parts are skipped")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    global R_BITS, WORKLOAD
    if args.r_log2 != 26:
        R_BITS = 1 << args.r_log2
        WORKLOAD = WORKLOAD.replace("r=2^26", f"r=2^{args.r_log2}")
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    rank, world, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.cuda_build_module().build()
    import datagen
    import paper_1402_4073_gb300 as bm
    datagen.build()

    words, queries = datagen.config2(R_BITS, N)
    shard_rows = args.shard == "rows"
    if shard_rows:
        # this rank's word-aligned slice of the rows of every bitmap
        from paper_1402_4073_gb300.shard import ShardedPool, sum_cardinalities
        spool = ShardedPool(R_BITS, N, rank=rank, world=world, device=local)
        spool.put_dense(words)
        pool = spool.pool
        local_rows = spool.rows
        args.parts = "dense"
    else:
        pool = bm.Pool(R_BITS, N, device=local)
        pool.put_dense(words)
        local_rows = R_BITS

    def exchange(c):
        """Row shards: the whole queries' cardinalities (one all-reduce)."""
        if shard_rows and world > 1:
            sum_cardinalities(c)

    stream = torch.cuda.current_stream()
    outs = [pool.empty_words() for _ in queries]
    cards = torch.zeros(len(queries), dtype=torch.int64, device="cuda")

    def launch(i, q, out=None):
        o = outs[i] if out is None else out
        if q.kind == 0:
            bm.threshold(pool, q.ids, q.theta, o, cards[i:i + 1])
        else:  # BM_KIND_INTERVAL through bm_query_run
            bm.interval(pool, q.ids, q.lo, q.hi, o, cards[i:i + 1])

    # kernel shape: the library's autotuner (results are identical for every shape)
    if args.dense_config:
        pool.set_dense_config(*[int(x) for x in args.dense_config.split(",")])
        tune_report = "fixed by --dense-config"
    else:
        tune_report = pool.autotune()
        print(f"autotune: {tune_report}", file=sys.stderr)
    best = pool.configs()["dense"]
    pool.status()

    for _ in range(args.warmup):
        for i, q in enumerate(queries):
            launch(i, q)
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    # keep the GPU busy while the sampler starts
    for _ in range(20):
        for i, q in enumerate(queries):
            launch(i, q)
    nq = len(queries)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2 * nq)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start.record(stream)
    for s in range(args.steps):
        for i, q in enumerate(queries):
            ev[s][2 * i].record(stream)
            launch(i, q)
            ev[s][2 * i + 1].record(stream)
        exchange(cards)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    pool.status()
    el_ms = start.elapsed_time(end)
    if world > 1:
        t = torch.tensor([el_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        el_ms = float(t.item())
    step_bytes = sum(query_bytes(q.n, R_BITS) for q in queries)
    # replicas: every rank ran the whole workload; row shards: all ranks together ran it once
    units = 1 if shard_rows else world
    value = step_bytes * args.steps * units / (el_ms / 1e3) / 1e9
    launch_ms = [ev[s][2 * i].elapsed_time(ev[s][2 * i + 1]) for s in range(args.steps)
                 for i in range(nq)]
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    achieved = query_bytes(N, local_rows) / avg_launch_s / 1e9
    peak, peak_src = peaks()

    # end to end through the public API: host ids in, every
    # output bitmap and cardinality copied back to pinned host memory every
    # step.  Each copy runs on a second stream after its query's kernel (an
    # event), so a query's result travels while the next query computes.
    # Outputs are double-buffered on both sides: step s + 1 is queued before
    # the host waits for the copies of step s, and step s + 2, which reuses
    # step s's device buffers, waits on the device for those copies.
    nbuf = 2
    e_outs = [[pool.empty_words() for _ in queries] for _ in range(nbuf)]
    e_cards = [torch.zeros(nq, dtype=torch.int64, device="cuda") for _ in range(nbuf)]
    host_out = [[torch.empty(pool.words, dtype=torch.int64, pin_memory=True) for _ in queries]
                for _ in range(nbuf)]
    host_card = [torch.empty(nq, dtype=torch.int64, pin_memory=True) for _ in range(nbuf)]
    copied = [None] * nbuf
    copy_stream = torch.cuda.Stream()

    def e2e_launch(i, q, o, c):
        if q.kind == 0:
            bm.threshold(pool, q.ids, q.theta, o, c)
        else:
            bm.interval(pool, q.ids, q.lo, q.hi, o, c)

    e2e_steps = max(3, min(args.steps, 50))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        b = s % nbuf
        if copied[b] is not None:
            stream.wait_event(copied[b])  # step s - nbuf's results have left these buffers
        for i, q in enumerate(queries):
            e2e_launch(i, q, e_outs[b][i], e_cards[b][i:i + 1])
            done = torch.cuda.Event()
            done.record(stream)
            copy_stream.wait_event(done)
            with torch.cuda.stream(copy_stream):
                host_out[b][i].copy_(e_outs[b][i], non_blocking=True)
        if shard_rows and world > 1:
            exchange(e_cards[b])
            summed = torch.cuda.Event()
            summed.record(stream)
            copy_stream.wait_event(summed)
        with torch.cuda.stream(copy_stream):
            host_card[b].copy_(e_cards[b], non_blocking=True)
        copied[b] = torch.cuda.Event()
        copied[b].record(copy_stream)
        if s >= 1:
            copied[(s - 1) % nbuf].synchronize()  # the host holds step s - 1's results
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    last = (e2e_steps - 1) % nbuf
    assert torch.equal(host_card[last], cards.cpu()), "end-to-end cardinalities differ"
    assert torch.equal(host_out[last][0], outs[0].cpu()), "end-to-end output differs"
    h2d = sum(4 * q.n for q in queries)
    d2h = nq * pool.words * 8 + nq * 8
    e2e = step_bytes * units / e2e_s / 1e9

    cpu = None
    checked = {"checked_vs_oracle": False, "oracle_check": "not run"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        oracle.set_threads(os.cpu_count() or 1)
        bps, nw, dt, answers = cpu_sample_time(words, queries, R_BITS, args.cpu_budget)
        cpu = {"value": round(bps / 1e9, 4), "unit": "GB/s", "cores": oracle_threads(),
               "kind": "oracle",
               "sample": f"the 4 queries over the first {nw} of {words.shape[1]} words "
                         f"({64 * nw} rows), {dt:.1f} s"}
        # the oracle's answers of that sample against the timed run's outputs
        checked = oracle_check(bm, outs, cards, answers, nw, words.shape[1])
        # the same oracle on one host thread, over a smaller prefix
        oracle.set_threads(1)
        bps1, nw1, dt1, _ = cpu_sample_time(words, queries, R_BITS, min(4.0, args.cpu_budget))
        oracle.set_threads(os.cpu_count() or 1)
        cpu["one_thread"] = {"value": round(bps1 / 1e9, 4), "unit": "GB/s", "cores": 1,
                             "sample": f"the 4 queries over the first {nw1} words, {dt1:.1f} s"}

    extra = {}
    parts = args.parts.split(",")
    if "looped" in parts:
        extra["looped"] = bench_looped(bm, pool, queries, launch, cards)
    pool.close()
    if "small" in parts:
        extra["small"] = bench_small(bm, datagen)
    if "sparse" in parts:
        extra["sparse"] = bench_sparse(bm, datagen, small=args.small, config=args.sparse_config)
    if "rle" in parts:
        extra["rle"] = bench_rle(bm, datagen, small=args.small)
    if "weighted" in parts:
        extra["weighted"] = bench_weighted(bm, datagen, small=args.small)
    if "batch" in parts:
        extra["batched"] = bench_batched(bm, datagen, small=args.small, config=args.batch_config)
    if "selector" in parts:
        extra["selector"] = bench_selector(bm, datagen, small=args.small)
        extra["selector"]["clustered"] = bench_selector_clustered(bm, datagen, small=args.small)
    if "serving" in parts:
        extra["serving"] = bench_serving(bm, datagen, small=args.small)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "strong" if shard_rows else "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "r_bits": R_BITS, "queries_per_step": nq,
                       "parallelism": (f"row shards x{world} ({local_rows} rows on rank 0), "
                                       "cardinalities all-reduced every step") if shard_rows else
                                      f"replicas x{world} (independent queries)",
                       "queries_per_s": round(nq * args.steps * units / (el_ms / 1e3), 1),
                       "l2": "inputs (2.15 GB per query) larger than L2; no flush",
                       "dense_config": best, "autotune": tune_report},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "peak_source": f"hbm_gbs of {peak_src}",
                         "traffic": traffic_per_launch(),
                         "kernel": "csa dense (bit-sliced carry-save counter)",
                         "algorithmic_bytes_per_launch": query_bytes(N, local_rows)},
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e, 2), "unit": "GB/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": nq * args.steps,
            **checked,
            "clocks": clocks,
            **extra,
        }))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
