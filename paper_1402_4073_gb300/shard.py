"""Row sharding of threshold queries across ranks (one GPU each).

Rows are independent in every query (Sec. 1: output bit i depends on bit i
of the inputs only; the paper's horizontal and vertical evaluations of
Sec. 2 both rest on it), so a pool can be split by rows: rank g holds rows
[row0_g, row1_g) of every bitmap, each range a whole number of 64-bit words.
Every rank runs each query on its own rows with no exchange of data; the
output bitmap is the concatenation of the ranks' parts and the cardinality
the sum of theirs: one all-reduce of one integer per query (of nq integers
per batch).

``ShardedPool`` is the per-rank object: a ``Pool`` over this rank's rows,
the loaders that cut full-width bitmaps to them, the query calls of the
single-GPU library on the local rows, and the all-reduce of the
cardinalities.  Outputs stay sharded; ``gather_words`` assembles a whole
bitmap on request.  Each rank reads only its own HBM: there is no peer
access and no multicast.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def row_range(r_bits: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [row0, row1) of `rank`: an even split of the ceil(r/64) words."""
    words = (r_bits + 63) // 64
    w0 = words * rank // world
    w1 = words * (rank + 1) // world
    return min(64 * w0, r_bits), min(64 * w1, r_bits)


def shard_words(words: np.ndarray, r_bits: int, rank: int, world: int):
    """This rank's slice of every bitmap (rows of `words`) and its row count."""
    row0, row1 = row_range(r_bits, rank, world)
    return np.ascontiguousarray(words[:, row0 // 64:(row1 + 63) // 64]), row1 - row0


def shard_positions(flat, offsets, row0: int, row1: int):
    """The rows [row0, row1) of sorted position lists (list j is
    flat[offsets[j]:offsets[j+1]]), shifted to start at 0: (flat, offsets)
    of the rank's lists."""
    flat = np.asarray(flat, dtype=np.uint32)
    offsets = np.asarray(offsets, dtype=np.uint64)
    parts, offs = [], [0]
    for j in range(len(offsets) - 1):
        lst = flat[int(offsets[j]):int(offsets[j + 1])]
        a, b = np.searchsorted(lst, [row0, row1])
        parts.append(lst[a:b] - np.uint32(row0))
        offs.append(offs[-1] + int(b - a))
    local = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint32)
    return local, np.asarray(offs, dtype=np.uint64)


def _on_device(group) -> bool:
    """True when the group's collectives take CUDA tensors (NCCL)."""
    return dist.get_backend(group) == "nccl"


def sum_cardinality(card: int, group=None) -> int:
    """Whole-query cardinality from each rank's part (one all-reduce)."""
    dev = "cuda" if _on_device(group) else "cpu"
    t = torch.tensor([int(card)], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item())


def sum_cardinalities(cards: torch.Tensor, group=None) -> torch.Tensor:
    """All-reduce (sum) of per-query cardinalities, in place where the
    backend takes the tensor's device; returns the summed tensor."""
    if cards.is_cuda and not _on_device(group):
        host = cards.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
        cards.copy_(host)
        return cards
    dist.all_reduce(cards, op=dist.ReduceOp.SUM, group=group)
    return cards


def gather_words(local, r_bits: int, world: int, group=None) -> np.ndarray:
    """The whole output bitmap from each rank's words (all-gather, ranks in
    order; parts padded to the largest for the collective).  `local` is a
    host uint64 array or a device int64 tensor of this rank's words."""
    sizes = [(row_range(r_bits, g, world)[1] - row_range(r_bits, g, world)[0] + 63) // 64
             for g in range(world)]
    m = max(sizes)
    dev = "cuda" if _on_device(group) else "cpu"
    buf = torch.zeros(m, dtype=torch.int64, device=dev)
    if isinstance(local, torch.Tensor):
        src = local.reshape(-1).to(dev)
    else:
        src = torch.from_numpy(np.ascontiguousarray(local).view(np.int64)).to(dev)
    buf[:len(src)] = src[:m]
    parts = [torch.zeros(m, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return np.concatenate([p[:s].cpu().numpy().view(np.uint64) for p, s in zip(parts, sizes)])


class ShardedPool:
    """This rank's rows of a pool of `capacity` bitmaps of `r_bits` rows.

    rank / world default to the process group's; give them explicitly to
    hold one shard without a process group (the sums and the gather are then
    the caller's).  A rank whose range is empty (r below 64 rows per rank)
    holds no pool and contributes nothing."""

    def __init__(self, r_bits: int, capacity: int, rank: int | None = None,
                 world: int | None = None, device: int | None = None, mem_budget: int = 0,
                 group=None):
        from . import Pool
        if rank is None or world is None:
            rank = dist.get_rank(group) if dist.is_initialized() else 0
            world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.r_bits, self.capacity, self.rank, self.world = r_bits, capacity, rank, world
        self.group = group
        self.row0, self.row1 = row_range(r_bits, rank, world)
        self.rows = self.row1 - self.row0
        self.word0 = self.row0 // 64
        self.words = (self.rows + 63) // 64
        self.pool = Pool(self.rows, capacity, device, mem_budget) if self.rows else None
        self.device = self.pool.device if self.pool is not None else device

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- loading: full-width bitmaps are cut to this rank's words -----------

    def put_dense(self, words, first_id: int = 0, sliced: bool = False) -> None:
        """Load bitmaps given as rows of full-width words (host uint64 array
        or int64 tensor); sliced=True: `words` already holds only this rank's
        words of each bitmap."""
        if self.pool is None:
            return
        if not sliced:
            words = words[:, self.word0:self.word0 + self.words]
        self.pool.put_dense(words, first_id)

    def put_positions(self, flat, offsets, first_id: int = 0) -> None:
        """Load sorted position lists of whole bitmaps (host arrays; list j is
        flat[offsets[j]:offsets[j+1]]); this rank keeps the positions in its
        rows, shifted to local row numbers."""
        if self.pool is None:
            return
        local, offs = shard_positions(flat, offsets, self.row0, self.row1)
        self.pool.put_positions(local, offs, first_id)

    def empty_words(self, n: int | None = None) -> torch.Tensor:
        """Device buffer for this rank's part of n output bitmaps."""
        w = max(1, self.words)
        shape = (w,) if n is None else (n, w)
        dev = "cuda" if self.device is None else f"cuda:{self.device}"
        return torch.empty(shape, dtype=torch.int64, device=dev)

    # -- queries on the local rows -------------------------------------------

    def threshold(self, ids, theta: int, out_words: torch.Tensor, out_card: torch.Tensor,
                  stream=None) -> None:
        """T(theta) on this rank's rows; out_card receives this rank's part."""
        from . import threshold
        if self.pool is None:
            out_card.zero_()
            return
        threshold(self.pool, ids, theta, out_words, out_card, stream)

    def batch(self, queries, outs, out_cards: torch.Tensor, paths=None, stream=None):
        """A batch of queries (objects with ids, kind, theta, lo, hi, table)
        on this rank's rows, one bm_threshold_batch call; out_cards receives
        this rank's parts.  Returns the chosen paths (None without rows)."""
        from . import threshold_batch
        if self.pool is None:
            out_cards.zero_()
            return None
        return threshold_batch(self.pool, queries, outs, out_cards, paths, stream)

    def prepared_batch(self, queries, outs, paths=None):
        """The batch marshalled once (see PreparedBatch), on this rank's rows."""
        from . import PreparedBatch
        return PreparedBatch(self.pool, queries, outs, paths) if self.pool is not None else None

    # -- the exchange: one all-reduce of the cardinalities -------------------

    def total_cards(self, local_cards: torch.Tensor) -> torch.Tensor:
        """Whole-query cardinalities: the sum of every rank's parts."""
        if self.world == 1:
            return local_cards
        return sum_cardinalities(local_cards, self.group)

    def gather(self, local_words) -> np.ndarray:
        """The whole output bitmap of one query (all-gather; host array)."""
        if self.world == 1:
            src = local_words if not isinstance(local_words, torch.Tensor) else \
                local_words.cpu().numpy().view(np.uint64)
            return np.asarray(src)[: (self.r_bits + 63) // 64]
        return gather_words(local_words[: self.words] if self.words else local_words[:0],
                            self.r_bits, self.world, self.group)
