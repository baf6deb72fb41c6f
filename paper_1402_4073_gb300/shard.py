"""Row sharding of a threshold query across ranks (one GPU each).

Rows are independent in every query (Sec. 1: output bit i depends on bit i
of the inputs only), so a pool can be split by rows: rank g holds rows
[row0_g, row1_g) of every bitmap, with each range a whole number of 64-bit
words.  Every rank runs the query on its rows with no exchange of data;
the output bitmap is the concatenation of the ranks' parts and the
cardinality the sum of theirs (one all-reduce of one integer per query).
This module is the host-side logic; the per-rank work is the ordinary
single-GPU path.
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


def sum_cardinality(card: int, group=None) -> int:
    """Whole-query cardinality from each rank's part (one all-reduce)."""
    t = torch.tensor([int(card)], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item())


def gather_words(local: np.ndarray, r_bits: int, world: int, group=None) -> np.ndarray:
    """The whole output bitmap from each rank's words (all-gather, ranks in
    order; parts padded to the largest for the collective)."""
    sizes = [(row_range(r_bits, g, world)[1] - row_range(r_bits, g, world)[0] + 63) // 64
             for g in range(world)]
    m = max(sizes)
    buf = torch.zeros(m, dtype=torch.int64)
    buf[:len(local)] = torch.from_numpy(np.ascontiguousarray(local).view(np.int64))
    parts = [torch.zeros(m, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return np.concatenate([p[:s].numpy().view(np.uint64) for p, s in zip(parts, sizes)])
