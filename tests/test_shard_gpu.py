"""Row-sharded pools on the GPU path: every rank holds a word-aligned slice of
the rows of every bitmap and runs the library's batch kernels on it; the
concatenated outputs and the summed cardinalities equal the whole-pool
oracle answer, bit-exactly.

Two forms: one process holding three shards in turn (no process group;
ragged row count, so the last shard ends inside a word), and two processes
sharing the one GPU, each with its own shard, whose cardinalities are summed
by an all-reduce and whose outputs are all-gathered over a gloo group.  The
ranks' kernels never wait on one another: the only exchange is on the host.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

R_BITS = 64 * 3001 + 13
NBM = 40


def _workload(dg):
    d = dg.pool_densities(dg.STREAM_TESTS + 18000, NBM, 1e-3, 0.5)
    words = dg.bernoulli(dg.STREAM_TESTS + 18001, R_BITS, d)
    flat, offs = dg.positions(words, R_BITS)
    queries = dg._queries(dg.STREAM_TESTS + 18002, 24, NBM, 2, NBM, None, 0.2)
    n = queries[5].n
    queries[5] = dg.Query(queries[5].ids, 2, table=dg.table_from_bools(np.arange(n + 1) % 3 == 1))
    queries[6] = dg.Query(queries[6].ids, 0, theta=0)
    queries[7] = dg.Query(queries[7].ids, 0, theta=queries[7].n + 1)
    return words, flat, offs, queries


def _run_shard(bm, shard_mod, words, flat, offs, queries, rank, world, paths):
    sp = shard_mod.ShardedPool(R_BITS, NBM, rank=rank, world=world)
    sp.put_dense(words)
    sp.put_positions(flat, offs)
    outs = [sp.empty_words().fill_(-1) for _ in queries]
    cards = torch.full((len(queries),), -1, dtype=torch.int64, device="cuda")
    sp.batch(queries, outs, cards, paths)
    torch.cuda.synchronize()
    if sp.pool is not None:
        sp.pool.status()
    return sp, outs, cards


def test_three_shards_one_process(dg, oracle_lib):
    import paper_1402_4073_gb300 as bm
    from paper_1402_4073_gb300 import shard
    words, flat, offs, queries = _workload(dg)
    paths = [(bm.PATH_DENSE, bm.PATH_SPARSE, bm.PATH_AUTO)[i % 3] for i in range(len(queries))]
    world = 3
    parts, card_sum = [], np.zeros(len(queries), dtype=np.int64)
    for rank in range(world):
        sp, outs, cards = _run_shard(bm, shard, words, flat, offs, queries, rank, world, paths)
        parts.append([bm.to_numpy_words(o)[:sp.words] for o in outs])
        card_sum += cards.cpu().numpy()
        sp.close()
    for i, q in enumerate(queries):
        want_words, want_card = oracle_lib.query(words, q, R_BITS)
        got = np.concatenate([parts[g][i] for g in range(world)])
        assert np.array_equal(got, want_words), f"query {i} (kind {q.kind}, n {q.n})"
        assert int(card_sum[i]) == want_card, f"query {i} cardinality"


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_proc(rank, world, port, q):
    import torch.distributed as dist

    import datagen
    import oracle
    import paper_1402_4073_gb300 as bm
    from paper_1402_4073_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        words, flat, offs, queries = _workload(datagen)
        paths = [(bm.PATH_DENSE, bm.PATH_SPARSE)[i % 2] for i in range(len(queries))]
        sp, outs, cards = _run_shard(bm, shard, words, flat, offs, queries, rank, world, paths)
        total = sp.total_cards(cards).cpu().numpy()
        ok_words, ok_cards = True, True
        for i, qq in enumerate(queries):
            full = sp.gather(outs[i])
            want_words, want_card = oracle.query(words, qq, R_BITS)
            ok_words &= bool(np.array_equal(full, want_words))
            ok_cards &= int(total[i]) == want_card
        sp.close()
        q.put((rank, ok_words, ok_cards))
    except Exception as e:  # reported to the parent
        q.put((rank, False, repr(e)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_the_gpu_gloo(dg, oracle_lib):
    import paper_1402_4073_gb300  # noqa: F401  (library built and loadable)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_proc, args=(g, 2, port, q)) for g in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
    assert all(r[1] is True and r[2] is True for r in results), results
