"""Host logic of row sharding, on CPU with two gloo ranks: the row ranges,
the slicing of full-width bitmaps, the all-reduce of the cardinalities and
the all-gather of the output.  The per-rank compute here is the oracle on
the rank's slice, so that this runs without a GPU; tests/test_shard_gpu.py
runs the same exchange around the library's kernels on each rank's shard."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, r_bits, q):
    import torch.distributed as dist

    import datagen
    import oracle
    from paper_1402_4073_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        words = datagen.bernoulli(datagen.STREAM_TESTS + 17000, r_bits, np.linspace(0.05, 0.6, 12))
        ids = np.array([0, 3, 5, 7, 7, 11, 2], dtype=np.uint32)
        local, rows = shard.shard_words(words, r_bits, rank, world)
        part, card = oracle.threshold(local, ids, rows, 3)
        total = shard.sum_cardinality(card)
        full = shard.gather_words(part, r_bits, world)
        want, want_card = oracle.threshold(words, ids, r_bits, 3)
        q.put((rank, bool(np.array_equal(full, want)), total == want_card))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("r_bits", [64 * 1000, 64 * 1001 + 13, 70])
def test_two_rank_row_shards(r_bits):
    import __graft_entry__
    __graft_entry__.cuda_build_module().build()  # the package loads libbm.so on import
    from paper_1402_4073_gb300 import shard
    # ranges tile the rows exactly, on word boundaries
    for world in (1, 2, 3, 8):
        spans = [shard.row_range(r_bits, g, world) for g in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == r_bits
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 == b0 and a0 % 64 == 0
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(g, 2, port, r_bits, q)) for g in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(ok_words and ok_card for _, ok_words, ok_card in results), results


def test_shard_positions_match_shard_words(dg):
    """The rank's slice of position lists equals the set bits of the rank's
    slice of the dense words, for every rank of a ragged split."""
    import __graft_entry__
    __graft_entry__.cuda_build_module().build()
    from paper_1402_4073_gb300 import shard
    r_bits = 64 * 777 + 19
    words = dg.bernoulli(dg.STREAM_TESTS + 17100, r_bits, np.linspace(0.001, 0.4, 9))
    flat, offs = dg.positions(words, r_bits)
    for world in (1, 2, 3, 5):
        for rank in range(world):
            local_words, rows = shard.shard_words(words, r_bits, rank, world)
            lflat, loffs = shard.shard_positions(flat, offs, *shard.row_range(r_bits, rank, world))
            want_flat, want_offs = dg.positions(local_words, rows) if rows else (
                np.zeros(0, np.uint32), np.zeros(len(offs), np.uint64))
            assert np.array_equal(lflat, want_flat), (world, rank)
            assert np.array_equal(loffs, np.asarray(want_offs, np.uint64)), (world, rank)
