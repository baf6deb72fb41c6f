"""Learned kernel selector: timing collection, training and evaluation.

For every query the library can run one of six candidate kernels
(``CANDIDATES``: the dense bit-sliced counter in the pool's shape, ScanCount
with 16K, 32K or 64K-row tiles, the dense counter with one 64-bit word per
thread, or the run-length path); results are identical, only the time
differs.  The paper picks among its algorithms by measured time and scores
each by its suboptimality, (t - t_best) / t_best (App. C).  Here a small
network (6 -> 64 -> 64 -> 6, ReLU, fp32) predicts the log time of each
candidate from the query's features; the smallest prediction among the
candidates the query's loaded forms allow wins.

* ``collect``: time every candidate on every query with the library's own
  kernels (CUDA events around calls queued back to back) and read each
  query's features.
* ``train``: fit the network to the log times on the GPU with the library's
  forward, backward and Adam kernels.
* ``time_lost``: sum(t_chosen - t_best) / sum(t_best) over a query set, the
  paper's suboptimality aggregated over the workload.
* ``install``: hand the trained weights to the pool, which then routes
  ``PATH_AUTO`` queries (single and batched) by them.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import (BM_ERANGE, CANDIDATES, PATH_AUTO, PATH_DENSE, PATH_RLE, PATH_SPARSE,
               SELECTOR_CANDIDATES, SELECTOR_FEATURES, SELECTOR_HIDDEN, BMError, Pool,
               PreparedQuery, mlp_adam, mlp_backward, mlp_forward, mlp_param_count,
               query_features, query_select, set_selector)


@dataclass
class Model:
    params: np.ndarray  # fp32, bm_mlp_forward layout
    mean: np.ndarray    # feature standardisation
    std: np.ndarray
    final_loss: float = float("nan")


def collect(pool: Pool, queries, reps: int = 3, stream=None):
    """(features [n, F], times_us [n, C]) for every query and candidate: the
    device time per call, `reps` calls queued back to back behind a short
    sleep kernel (so that the host's own per-call time, the same for every
    candidate, is not measured), mean per call.  A candidate the query's
    loaded forms do not allow (no lists, no run-length forms) is NaN."""
    stream = stream or torch.cuda.current_stream()
    info = pool.info()
    feats = np.stack([query_features(pool, q) for q in queries]).astype(np.float32)
    times = np.full((len(queries), SELECTOR_CANDIDATES), np.nan, dtype=np.float64)
    out = pool.empty_words()
    card = torch.zeros(1, dtype=torch.int64, device=out.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    saved = pool.configs()["sparse"]
    saved_dense = pool.configs()["dense"]
    sleep = getattr(torch.cuda, "_sleep", None)
    for c, (path, tile) in enumerate(CANDIDATES):
        if path == PATH_SPARSE:
            if info["lists_loaded"] == 0:
                continue
            pool.set_sparse_config(tile, saved["threads"], saved["ctas_per_sm"], saved["unroll"])
        if path == PATH_DENSE:
            if info["dense_loaded"] == 0:
                continue
            d = dict(saved_dense)
            if tile == 1:  # the one-word-per-thread shape, as the library runs candidate 4
                d.update(variant=0, words_per_thread=1, adder=0 if d["adder"] == 2 else d["adder"])
            pool.set_dense_config(**d)
        if path == PATH_RLE and info["rle_loaded"] == 0:
            continue
        for i, q in enumerate(queries):
            pq = PreparedQuery(pool, q, out, path)
            try:
                pq.run(card, stream)  # warm-up
            except BMError as e:
                if e.code != BM_ERANGE:  # only a missing form leaves the candidate out
                    raise
                continue
            with torch.cuda.stream(stream):
                if sleep is not None:
                    sleep(100_000 * reps)  # about 50 us per call: the host queues the calls
                e0.record(stream)
                for _ in range(reps):
                    pq.run(card, stream)
                e1.record(stream)
            stream.synchronize()
            times[i, c] = e0.elapsed_time(e1) * 1e3 / reps
    pool.set_sparse_config(**saved)
    pool.set_dense_config(**saved_dense)
    return feats, times


def _init_params(seed: int) -> np.ndarray:
    """He-uniform initial weights, zero biases (seeded NumPy generator)."""
    rng = np.random.default_rng(seed)
    F, H, C = SELECTOR_FEATURES, SELECTOR_HIDDEN, SELECTOR_CANDIDATES
    parts = []
    for fan_in, fan_out in ((F, H), (H, H), (H, C)):
        lim = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, size=fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == mlp_param_count(F, H, C)
    return p


def train(feats: np.ndarray, times_us: np.ndarray, steps: int = 3000, lr: float = 3e-3,
          seed: int = 1111, device: str = "cuda") -> Model:
    """Fit log(time) per candidate with full-batch Adam on the GPU.  A
    candidate a query cannot run (NaN time) is labelled ten times slower
    than the query's slowest candidate that ran; it is never picked for such
    a query anyway, since the selection skips candidates whose forms are
    missing."""
    ok = np.any(np.isfinite(times_us), axis=1)
    X = feats[ok].astype(np.float64)
    T = np.log(np.maximum(times_us[ok], 1e-3))
    worst = np.nanmax(T, axis=1, keepdims=True) + np.log(10.0)
    T = np.where(np.isfinite(T), T, worst)
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std[std < 1e-6] = 1.0
    x = torch.from_numpy(((X - mean) / std).astype(np.float32)).to(device)
    t = torch.from_numpy(T.astype(np.float32)).to(device)
    params = torch.from_numpy(_init_params(seed)).to(device)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    H, C = SELECTOR_HIDDEN, SELECTOR_CANDIDATES
    loss = None
    for step in range(1, steps + 1):
        y, h1, h2 = mlp_forward(params, x, H, C)
        grads, loss = mlp_backward(params, x, h1, h2, y, t)
        mlp_adam(params, grads, m, v, step, lr)
    torch.cuda.synchronize()
    return Model(params.cpu().numpy(), mean.astype(np.float32), std.astype(np.float32),
                 float(loss.item()) if loss is not None else float("nan"))


def predict(model: Model, feats: np.ndarray, device: str = "cuda") -> np.ndarray:
    """Predicted log times [n, C] by the library's forward kernel."""
    x = torch.from_numpy(((feats - model.mean) / model.std).astype(np.float32)).to(device)
    p = torch.from_numpy(model.params).to(device)
    y, _, _ = mlp_forward(p, x, SELECTOR_HIDDEN, SELECTOR_CANDIDATES)
    return y.cpu().numpy()


def time_lost(times_us: np.ndarray, choice: np.ndarray):
    """sum(t_chosen - t_best) / sum(t_best) over the queries, t_best among the
    candidates each query can run; None if a choice is one the query cannot
    run (a fixed policy that some queries' forms do not allow)."""
    ok = np.any(np.isfinite(times_us), axis=1)
    t = times_us[ok]
    chosen = t[np.arange(len(t)), choice[ok]]
    if not np.all(np.isfinite(chosen)):
        return None
    best = np.nanmin(t, axis=1)
    return float((chosen - best).sum() / best.sum())


def rule_choices(pool: Pool, queries) -> np.ndarray:
    """Candidate index the fixed density rule picks for each query (with no
    selector installed on the pool)."""
    set_selector(pool, None)
    return installed_choices(pool, queries)


def install(pool: Pool, model: Model) -> None:
    set_selector(pool, model.params, model.mean, model.std)


def installed_choices(pool: Pool, queries) -> np.ndarray:
    """Candidate index the pool's installed selector picks for each query
    (the host-side inference that single queries use)."""
    tiles = {tile: c for c, (p, tile) in enumerate(CANDIDATES) if p == PATH_SPARSE}
    dense = {w: c for c, (p, w) in enumerate(CANDIDATES) if p == PATH_DENSE}
    rle = CANDIDATES.index((PATH_RLE, 0))
    out = []
    for q in queries:
        path, tile = query_select(pool, q)
        out.append(dense.get(tile, 0) if path == PATH_DENSE
                   else rle if path == PATH_RLE else tiles.get(tile, 2))
    return np.array(out, dtype=np.int64)


def evaluate(pool: Pool, model: Model, queries, feats, times_us) -> dict:
    """Time lost of the network (as installed on the pool), the fixed rule
    and single-kernel policies, from one table of measured times."""
    rule = rule_choices(pool, queries)
    install(pool, model)
    mlp_choice = installed_choices(pool, queries)
    ok = np.any(np.isfinite(times_us), axis=1)
    res = {"queries": int(ok.sum()),
           "time_lost_mlp": time_lost(times_us, mlp_choice),
           "time_lost_rule": time_lost(times_us, rule),
           "time_lost_always_dense": time_lost(times_us, np.zeros(len(times_us), np.int64))}
    for c in range(1, SELECTOR_CANDIDATES):
        res[f"time_lost_always_c{c}"] = time_lost(times_us, np.full(len(times_us), c))
    best_total = float(np.nanmin(times_us[ok], axis=1).sum())
    res["total_us_best"] = best_total
    res["total_us_mlp"] = best_total * (1 + res["time_lost_mlp"])
    res["total_us_rule"] = best_total * (1 + res["time_lost_rule"])
    res["mlp_choices"] = np.bincount(mlp_choice[ok], minlength=SELECTOR_CANDIDATES).tolist()
    return res


__all__ = ["Model", "collect", "train", "predict", "time_lost", "rule_choices", "install",
           "evaluate", "PATH_AUTO"]
