"""Python driver of the serving loop (``bm_server_*`` in the C ABI).

The loop itself (admission by device memory, continuous batching, batches
overlapping on several streams) runs in the library's scheduler thread.
This module wraps it for interactive use and for Poisson-load experiments
whose submissions are issued by the library's native load generator, so
Python overhead does not limit the offered rate.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native, _q_from, check, lib

BM_OK, BM_ETIMEOUT, BM_EBUSY = 0, -5, -6


class Server:
    """The native serving loop over `pool` (bm_server_*).  Under overload,
    larger batches share each slab of the pool among more queries, so the
    default allows two batches of up to 2048 requests in flight; below
    saturation batches stay small and latency does not depend on it."""

    def __init__(self, pool, mem_budget: int, max_batch: int = 2048, max_inflight: int = 2,
                 max_queue: int = 1 << 20, batch_window_us: int = 0, slo_us: int = 0):
        """slo_us > 0: load shedding by a latency objective (batches sized so
        that their oldest request can still finish within slo_us; requests
        that cannot are dropped as expired)."""
        cfg = _native.bm_server_config(mem_budget, max_batch, max_inflight, max_queue,
                                       batch_window_us, slo_us, 0)
        h = ctypes.c_void_p()
        check(lib.bm_server_create(pool.handle, ctypes.byref(cfg), ctypes.byref(h)),
              "bm_server_create")
        self.handle = h
        self.pool = pool

    def close(self):
        if self.handle:
            lib.bm_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, query, path: int | None = None, deadline_us: int = 0) -> int:
        q, keep = _q_from(query, None, path)
        t = ctypes.c_uint64()
        check(lib.bm_server_submit_deadline(self.handle, ctypes.byref(q), deadline_us,
                                            ctypes.byref(t)), "bm_server_submit")
        return int(t.value)

    def cancel(self, ticket: int) -> None:
        check(lib.bm_server_cancel(self.handle, ticket), "bm_server_cancel")

    def wait(self, ticket: int, timeout_ms: int = 10000) -> int:
        return lib.bm_server_wait(self.handle, ticket, timeout_ms)

    def result(self, ticket: int, words: bool = True):
        """(words or None, cardinality, latency_us, queue_us, path)."""
        out = np.zeros(self.pool.words, dtype=np.uint64) if words else None
        card = ctypes.c_uint64()
        lat, qu = ctypes.c_double(), ctypes.c_double()
        path = ctypes.c_int32()
        check(lib.bm_server_result(self.handle, ticket, out.ctypes.data if words else None,
                                   ctypes.byref(card), ctypes.byref(lat), ctypes.byref(qu),
                                   ctypes.byref(path)), "bm_server_result")
        return out, int(card.value), lat.value, qu.value, int(path.value)

    def release(self, ticket: int) -> None:
        check(lib.bm_server_release(self.handle, ticket), "bm_server_release")

    def stats(self) -> dict:
        st = _native.bm_server_stats_t()
        check(lib.bm_server_stats(self.handle, ctypes.byref(st)), "bm_server_stats")
        return {k: getattr(st, k) for k, _ in st._fields_}

    def replay(self, queries, arrival_s) -> dict:
        """Open-loop load: submit queries[i] at arrival_s[i]; returns per-request
        latency, queueing time, cardinality and status arrays plus wall time."""
        n = len(queries)
        arr = (_native.bm_query * n)()
        keep = []
        for i, qo in enumerate(queries):
            q, k = _q_from(qo)
            arr[i] = q
            keep.append(k)
        t = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(n)
        qu = np.zeros(n)
        cards = np.zeros(n, dtype=np.uint64)
        status = np.zeros(n, dtype=np.int32)
        wall = ctypes.c_double()
        check(lib.bm_server_replay(self.handle, arr, n, t.ctypes.data, lat.ctypes.data,
                                   qu.ctypes.data, cards.ctypes.data, status.ctypes.data,
                                   ctypes.byref(wall)), "bm_server_replay")
        return {"latency_us": lat, "queue_us": qu, "cards": cards, "status": status,
                "wall_s": wall.value}


def summarize(res: dict, offered_qps: float, slo_us: float | None = None) -> dict:
    """Counts, achieved rate and latency percentiles of a replay; with
    slo_us also the goodput (requests completed within slo_us per second)."""
    ok = res["status"] == BM_OK
    lat = res["latency_us"][ok]
    n_ok = int(ok.sum())
    out = {
        "offered_qps": offered_qps,
        "completed": n_ok,
        "refused": int((res["status"] == BM_EBUSY).sum()),
        "expired": int((res["status"] == BM_ETIMEOUT).sum()),
        "errors": int(((res["status"] != BM_OK) & (res["status"] != BM_EBUSY) &
                       (res["status"] != BM_ETIMEOUT)).sum()),
        "achieved_qps": round(n_ok / res["wall_s"], 1) if res["wall_s"] > 0 else 0.0,
        "p50_us": round(float(np.percentile(lat, 50)), 1) if n_ok else None,
        "p99_us": round(float(np.percentile(lat, 99)), 1) if n_ok else None,
        "mean_queue_us": round(float(res["queue_us"][ok].mean()), 1) if n_ok else None,
    }
    if slo_us:
        good = int((lat <= slo_us).sum())
        out["slo_us"] = round(float(slo_us), 1)
        out["within_slo"] = good
        out["goodput_qps"] = round(good / res["wall_s"], 1) if res["wall_s"] > 0 else 0.0
    return out
