"""GB300-native threshold and symmetric-function queries over bitmaps.

Python binding of ``libbm.so`` (C ABI in ``include/bm.h``).  The binding only
marshals arguments: host arrays become pointers, torch CUDA tensors become
device pointers, and the current torch stream becomes the launch stream.
Device memory for outputs comes from PyTorch's allocator.

Bit layout: row i of a bitmap is bit i % 64 of 64-bit word i // 64.  Word
arrays are numpy ``uint64`` on the host and torch ``int64`` tensors (same
bits) on the device.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch  # loads the CUDA runtime that libbm.so then shares

from . import _native

lib = _native.load()

BM_OK, BM_EINVAL, BM_ERANGE, BM_ENOMEM, BM_ECUDA, BM_ETIMEOUT, BM_EBUSY, BM_ENOTREADY = (
    0, -1, -2, -3, -4, -5, -6, -7)
BM_N_MAX = 65535
BM_WEIGHT_MAX = (1 << 24) - 1


class BMError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = lib.bm_strerror(code).decode()
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


def check(rc: int, what: str = "") -> None:
    if rc != BM_OK:
        raise BMError(rc, what)


# the current stream's raw handle without building a Stream object (a few
# microseconds per call otherwise, as much as a small query's kernel)
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream) -> int:
    if stream is None:
        if _raw_stream is not None:
            return int(_raw_stream(torch.cuda.current_device()))
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _host_u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _host_u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _dev_ptr(t: torch.Tensor | None, min_bytes: int = 0) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if t.numel() * t.element_size() < min_bytes:
        raise ValueError(f"device buffer too small: need {min_bytes} bytes")
    return t.data_ptr()


def words_for(r_bits: int) -> int:
    return (r_bits + 63) // 64


class Pool:
    """A device-resident pool of `capacity` bitmaps of `r_bits` rows."""

    def __init__(self, r_bits: int, capacity: int, device: int | None = None, mem_budget: int = 0):
        """device: a CUDA device index; by default the current torch device."""
        if device is None:
            device = torch.cuda.current_device()
        h = ctypes.c_void_p()
        check(lib.bm_pool_create(device, r_bits, capacity, mem_budget, ctypes.byref(h)),
              "bm_pool_create")
        self.handle = h
        self.r_bits = r_bits
        self.capacity = capacity
        self.device = device
        self.words = words_for(r_bits)

    def close(self):
        if self.handle:
            lib.bm_pool_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def put_dense(self, words, first_id: int = 0):
        """Load bitmaps (rows of a 2-D uint64 numpy array or int64 CUDA tensor)."""
        if isinstance(words, torch.Tensor):
            if words.dim() == 1:
                words = words.view(1, -1)
            if words.stride(1) != 1:
                raise ValueError("rows must be contiguous")
            check(lib.bm_pool_put_dense(self.handle, first_id, words.shape[0], words.data_ptr(),
                                        words.stride(0), 1 if words.is_cuda else 0),
                  "bm_pool_put_dense")
            return
        w = _host_u64(words)
        if w.ndim == 1:
            w = w.reshape(1, -1)
        check(lib.bm_pool_put_dense(self.handle, first_id, w.shape[0], w.ctypes.data, w.shape[1], 0),
              "bm_pool_put_dense")

    def put_positions(self, flat, offsets, first_id: int = 0, zeros: bool = False):
        """Load sorted position lists: list j is flat[offsets[j]:offsets[j+1]],
        the rows where bitmap first_id + j is 1 (zeros=True: where it is 0)."""
        offs = _host_u64(offsets)
        fn = lib.bm_pool_put_complement_positions if zeros else lib.bm_pool_put_positions
        if isinstance(flat, torch.Tensor):
            check(fn(self.handle, first_id, len(offs) - 1, flat.data_ptr(), offs.ctypes.data,
                     1 if flat.is_cuda else 0), "bm_pool_put_positions")
            return
        f = _host_u32(flat)
        fp = f.ctypes.data if len(f) else None
        check(fn(self.handle, first_id, len(offs) - 1, fp, offs.ctypes.data, 0),
              "bm_pool_put_positions")

    def put_rle(self, first_id: int = 0, count: int | None = None) -> None:
        """Build the run-length form (clean-0 / clean-1 / literal words, per
        256-word tile) of dense ids first_id .. first_id + count - 1 (all
        loaded dense ids from first_id by default) for BM_PATH_RLE queries."""
        if count is None:
            count = self.info()["capacity"] - first_id
        check(lib.bm_pool_put_rle(self.handle, first_id, count), "bm_pool_put_rle")

    def _rle_stats(self, id_: int) -> tuple[int, int, int]:
        r, l, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        check(lib.bm_pool_rle_info(self.handle, id_, ctypes.byref(r), ctypes.byref(l),
                                   ctypes.byref(b)), "bm_pool_rle_info")
        return int(r.value), int(l.value), int(b.value)

    def rle_info(self, id_: int) -> tuple[int, int]:
        """(runs, literal words) of id's run-length form: maximal runs of
        words of one kind, and the words that are neither all 0 nor all 1."""
        return self._rle_stats(id_)[:2]

    def rle_bytes(self, id_: int) -> int:
        """Device bytes of id's run-length form (containers and summaries)."""
        return self._rle_stats(id_)[2]

    def info(self) -> dict:
        i = _native.bm_pool_info_t()
        check(lib.bm_pool_info(self.handle, ctypes.byref(i)), "bm_pool_info")
        return {k: getattr(i, k) for k, _ in i._fields_}

    def bitmap_cardinality(self, id_: int) -> int:
        c = ctypes.c_uint64()
        check(lib.bm_pool_bitmap_cardinality(self.handle, id_, ctypes.byref(c)))
        return int(c.value)

    def status(self) -> None:
        """Synchronise; raise BMError(BM_ETIMEOUT) if a device wait expired."""
        check(lib.bm_pool_status(self.handle), "bm_pool_status")

    def set_dense_config(self, variant: int, threads: int = 128, stages: int = 4,
                         ctas_per_sm: int = 1, adder: int = 0, words_per_thread: int = 2) -> None:
        c = _native.bm_dense_config_t(variant, threads, stages, ctas_per_sm, adder, words_per_thread)
        check(lib.bm_pool_set_dense_config(self.handle, ctypes.byref(c)), "bm_pool_set_dense_config")

    def set_looped(self, max_t: int) -> None:
        """Plain thresholds with min(T, N - T + 1) <= max_t (1..3) run the
        Looped recurrence on the dense path; 0 turns it off."""
        check(lib.bm_pool_set_looped(self.handle, max_t), "bm_pool_set_looped")

    def set_sparse_config(self, tile_rows: int = 32768, threads: int = 512,
                          ctas_per_sm: int = 2, unroll: int = 4) -> None:
        c = _native.bm_sparse_config_t(tile_rows, threads, ctas_per_sm, unroll)
        check(lib.bm_pool_set_sparse_config(self.handle, ctypes.byref(c)),
              "bm_pool_set_sparse_config")

    def set_batch_config(self, ctas_per_sm: int = 2, adder: int = 0,
                         words_per_thread: int = 2) -> None:
        c = _native.bm_batch_config_t(ctas_per_sm, adder, words_per_thread)
        check(lib.bm_pool_set_batch_config(self.handle, ctypes.byref(c)), "bm_pool_set_batch_config")

    def configs(self) -> dict:
        d, s, b = _native.bm_dense_config_t(), _native.bm_sparse_config_t(), _native.bm_batch_config_t()
        check(lib.bm_pool_get_dense_config(self.handle, ctypes.byref(d)))
        check(lib.bm_pool_get_sparse_config(self.handle, ctypes.byref(s)))
        check(lib.bm_pool_get_batch_config(self.handle, ctypes.byref(b)))
        lp = ctypes.c_uint32()
        check(lib.bm_pool_get_looped(self.handle, ctypes.byref(lp)))
        as_dict = lambda x: {k: getattr(x, k) for k, _ in x._fields_}
        return {"dense": as_dict(d), "sparse": as_dict(s), "batch": as_dict(b), "looped": int(lp.value)}

    def autotune(self, cache_path: str | None = None) -> str:
        """Measure kernel shapes on this pool and install the fastest."""
        buf = ctypes.create_string_buffer(1024)
        check(lib.bm_pool_autotune(self.handle, cache_path.encode() if cache_path else None, buf,
                                   len(buf)), "bm_pool_autotune")
        return buf.value.decode()

    def empty_words(self, n: int | None = None) -> torch.Tensor:
        shape = (self.words,) if n is None else (n, self.words)
        return torch.empty(shape, dtype=torch.int64, device=f"cuda:{self.device}")


def threshold(pool: Pool, ids, theta: int, out_words: torch.Tensor,
              out_card: torch.Tensor | None = None, stream=None) -> None:
    """T(theta) over pool bitmaps `ids` into `out_words` (+ cardinality)."""
    i = _host_u32(ids)
    check(lib.bm_threshold(pool.handle, i.ctypes.data, len(i), int(theta),
                           _dev_ptr(out_words, 8 * pool.words), _dev_ptr(out_card, 8), _stream(stream)),
          "bm_threshold")


def symmetric(pool: Pool, ids, table, out_words: torch.Tensor,
              out_card: torch.Tensor | None = None, stream=None) -> None:
    """Symmetric function with truth table `table` (uint64 words, bit c = f(c))."""
    i = _host_u32(ids)
    t = _host_u64(table)
    if t.size * 64 < len(i) + 1:
        raise ValueError("truth table needs n + 1 bits")
    check(lib.bm_symmetric(pool.handle, i.ctypes.data, len(i), t.ctypes.data,
                           _dev_ptr(out_words, 8 * pool.words), _dev_ptr(out_card, 8), _stream(stream)),
          "bm_symmetric")


def cardinality(words: torch.Tensor, r_bits: int, out_card: torch.Tensor, stream=None) -> None:
    check(lib.bm_cardinality(_dev_ptr(words, 8 * words_for(r_bits)), r_bits, _dev_ptr(out_card, 8),
                             _stream(stream)), "bm_cardinality")


def interval(pool: Pool, ids, lo: int, hi: int, out_words: torch.Tensor,
             out_card: torch.Tensor | None = None, path: int | None = None, stream=None) -> int:
    """Interval query lo <= count <= hi (BM_KIND_INTERVAL: the library builds
    T_lo AND NOT T_{hi+1}) on `path` (dense by default); returns the path
    that ran."""
    i = _host_u32(ids)
    q = _native.bm_query()
    q.ids = i.ctypes.data
    q.n = len(i)
    q.kind = KIND_INTERVAL
    q.theta, q.lo, q.hi = 0, int(lo), int(hi)
    q.table = None
    q.out_words = _dev_ptr(out_words, 8 * pool.words)
    q.path = PATH_DENSE if path is None else int(path)
    q.reserved = 0
    chosen = ctypes.c_int32()
    check(lib.bm_query_run(pool.handle, ctypes.byref(q), _dev_ptr(out_card, 8),
                           ctypes.byref(chosen), _stream(stream)), "bm_query_run")
    return int(chosen.value)


def to_numpy_words(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


# ---------------------------------------------------------------------------
# query descriptors, path choice, batches

KIND_THRESHOLD, KIND_INTERVAL, KIND_TABLE = 0, 1, 2
PATH_AUTO, PATH_DENSE, PATH_SPARSE, PATH_RLE = 0, 1, 2, 3
SELECTOR_FEATURES, SELECTOR_HIDDEN, SELECTOR_CANDIDATES = 6, 64, 6
# candidate c of the selector: (path, sparse tile rows, or for the dense path
# the words per thread: 0 = the pool's shape, 1 = one 64-bit word per thread)
CANDIDATES = [(PATH_DENSE, 0), (PATH_SPARSE, 16384), (PATH_SPARSE, 32768), (PATH_SPARSE, 65536),
              (PATH_DENSE, 1), (PATH_RLE, 0)]


def make_query(ids, kind: int = KIND_THRESHOLD, theta: int = 0, lo: int = 0, hi: int = 0,
               table=None, out_words: torch.Tensor | None = None, path: int = PATH_AUTO):
    """A bm_query struct plus the host arrays it points into (keep both alive)."""
    i = _host_u32(ids)
    t = _host_u64(table) if table is not None else None
    q = _native.bm_query()
    q.ids = i.ctypes.data if len(i) else None
    q.n = len(i)
    q.kind = kind
    q.theta, q.lo, q.hi = int(theta), int(lo), int(hi)
    q.table = t.ctypes.data if t is not None else None
    q.out_words = _dev_ptr(out_words) if out_words is not None else None
    q.path = path
    q.reserved = 0
    return q, (i, t)


def _q_from(obj, out_words=None, path=None):
    return make_query(obj.ids, obj.kind, getattr(obj, "theta", 0), getattr(obj, "lo", 0),
                      getattr(obj, "hi", 0), getattr(obj, "table", None), out_words,
                      PATH_AUTO if path is None else path)


def query_run(pool: Pool, query, out_words: torch.Tensor, out_card: torch.Tensor | None = None,
              path: int = PATH_AUTO, stream=None) -> int:
    """Run one query (an object with ids, kind, theta, lo, hi, table) on a path;
    returns the path that ran."""
    if out_words.numel() * out_words.element_size() < 8 * pool.words:
        raise ValueError("output buffer too small")
    q, keep = _q_from(query, out_words, path)
    chosen = ctypes.c_int32()
    check(lib.bm_query_run(pool.handle, ctypes.byref(q), _dev_ptr(out_card, 8),
                           ctypes.byref(chosen), _stream(stream)), "bm_query_run")
    return int(chosen.value)


class PreparedQuery:
    """One query's bm_query struct, marshalled once: run() is then a single
    bm_query_run call."""

    def __init__(self, pool: Pool, query, out_words: torch.Tensor, path: int = PATH_AUTO):
        if out_words.numel() * out_words.element_size() < 8 * pool.words:
            raise ValueError("output buffer too small")
        self.pool = pool
        self.q, self._keep = _q_from(query, out_words, path)
        self.ref = ctypes.byref(self.q)
        self.chosen = ctypes.c_int32()

    def run(self, out_card: torch.Tensor | None = None, stream=None) -> int:
        check(lib.bm_query_run(self.pool.handle, self.ref, _dev_ptr(out_card, 8),
                               ctypes.byref(self.chosen), _stream(stream)), "bm_query_run")
        return int(self.chosen.value)


class PreparedBatch:
    """The bm_query array of a batch, marshalled once: run() is then a single
    bm_threshold_batch call (re-runnable while queries and outputs stay)."""

    def __init__(self, pool: Pool, queries, outs, paths=None):
        nq = len(queries)
        self.pool, self.nq = pool, nq
        self.arr = (_native.bm_query * nq)()
        self._keep = []
        for i, qo in enumerate(queries):
            if outs[i].numel() * outs[i].element_size() < 8 * pool.words:
                raise ValueError("output buffer too small")
            q, k = _q_from(qo, outs[i], None if paths is None else int(paths[i]))
            self.arr[i] = q
            self._keep.append(k)
        self.chosen = np.zeros(nq, dtype=np.int32)

    def run(self, out_cards: torch.Tensor, stream=None) -> np.ndarray:
        if out_cards.numel() < self.nq:
            raise ValueError("out_cards too small")
        check(lib.bm_threshold_batch(self.pool.handle, self.arr, self.nq,
                                     _dev_ptr(out_cards, 8 * self.nq), self.chosen.ctypes.data,
                                     _stream(stream)), "bm_threshold_batch")
        return self.chosen


def threshold_batch(pool: Pool, queries, outs, out_cards: torch.Tensor, paths=None,
                    stream=None) -> np.ndarray:
    """Run a batch of queries (objects with ids, kind, theta, lo, hi, table)
    into outs[i]; cardinalities into out_cards[i].  Returns the chosen paths."""
    return PreparedBatch(pool, queries, outs, paths).run(out_cards, stream).copy()


POST_NONE, POST_AND, POST_OR, POST_ANDNOT = 0, 1, 2, 3


def weighted_threshold(pool: Pool, ids, weights, theta: int, out_words: torch.Tensor,
                       out_card: torch.Tensor | None = None, post_op: int = POST_NONE,
                       post_id: int = 0, stream=None) -> None:
    """Rows where the sum of weights of the inputs holding them reaches theta,
    optionally ANDed / ORed / AND-NOTed with pool bitmap post_id."""
    if out_words.numel() * out_words.element_size() < 8 * pool.words:
        raise ValueError("output buffer too small")
    i = _host_u32(ids)
    w = _host_u32(weights)
    if len(i) != len(w):
        raise ValueError("ids and weights differ in length")
    q = _native.bm_weighted_query(i.ctypes.data if len(i) else None, w.ctypes.data if len(w) else None,
                                  len(i), post_op, theta, post_id, 0, out_words.data_ptr())
    check(lib.bm_weighted_threshold(pool.handle, ctypes.byref(q), _dev_ptr(out_card, 8),
                                    _stream(stream)), "bm_weighted_threshold")


def query_features(pool: Pool, query) -> np.ndarray:
    q, keep = _q_from(query)
    out = np.zeros(SELECTOR_FEATURES, dtype=np.float32)
    check(lib.bm_query_features(pool.handle, ctypes.byref(q), out.ctypes.data), "bm_query_features")
    return out


def query_select(pool: Pool, query) -> tuple[int, int]:
    q, keep = _q_from(query)
    path, tile = ctypes.c_int32(), ctypes.c_uint32()
    check(lib.bm_query_select(pool.handle, ctypes.byref(q), ctypes.byref(path), ctypes.byref(tile)),
          "bm_query_select")
    return int(path.value), int(tile.value)


def set_selector(pool: Pool, params: np.ndarray | None, mean=None, std=None) -> None:
    if params is None:
        check(lib.bm_pool_set_selector(pool.handle, None, 0, None, None, 0), "bm_pool_set_selector")
        return
    p = np.ascontiguousarray(params, dtype=np.float32)
    m = np.ascontiguousarray(mean, dtype=np.float32)
    s = np.ascontiguousarray(std, dtype=np.float32)
    check(lib.bm_pool_set_selector(pool.handle, p.ctypes.data, p.size, m.ctypes.data, s.ctypes.data,
                                   SELECTOR_CANDIDATES), "bm_pool_set_selector")


# ---------------------------------------------------------------------------
# selector network kernels (fp32, device tensors)

def mlp_param_count(F: int = 6, H: int = 64, C: int = 6) -> int:
    return F * H + H + H * H + H + H * C + C


def mlp_forward(params: torch.Tensor, x: torch.Tensor, H: int, C: int, stream=None):
    B, F = x.shape
    h1 = torch.empty(B, H, dtype=torch.float32, device=x.device)
    h2 = torch.empty(B, H, dtype=torch.float32, device=x.device)
    y = torch.empty(B, C, dtype=torch.float32, device=x.device)
    check(lib.bm_mlp_forward(_dev_ptr(params), F, H, C, _dev_ptr(x), B, _dev_ptr(h1), _dev_ptr(h2),
                             _dev_ptr(y), _stream(stream)), "bm_mlp_forward")
    return y, h1, h2


def mlp_backward(params: torch.Tensor, x, h1, h2, y, target, stream=None):
    B, F = x.shape
    H, C = h1.shape[1], y.shape[1]
    grads = torch.empty_like(params)
    ws = torch.empty(B * (C + 2 * H), dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    check(lib.bm_mlp_backward(_dev_ptr(params), F, H, C, _dev_ptr(x), _dev_ptr(h1), _dev_ptr(h2),
                              _dev_ptr(y), _dev_ptr(target), B, _dev_ptr(grads), _dev_ptr(ws),
                              _dev_ptr(loss), _stream(stream)), "bm_mlp_backward")
    return grads, loss


def mlp_adam(params, grads, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
             eps: float = 1e-8, stream=None) -> None:
    check(lib.bm_mlp_adam(_dev_ptr(params), _dev_ptr(grads), _dev_ptr(m), _dev_ptr(v), params.numel(),
                          step, lr, beta1, beta2, eps, _stream(stream)), "bm_mlp_adam")
