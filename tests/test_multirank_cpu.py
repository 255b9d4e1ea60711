"""Host logic of the multi-rank benchmark path on the CPU (gloo, world size 2): queries are
sharded round-robin with nothing shared on the data path, and the step time is the
maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_items, out):
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ids = bench.shard(n_items, rank, world)
    batches = bench.batches_for(ids, 7, 5)
    gathered = [None] * world
    dist.all_gather_object(gathered, ids.tolist())
    t = torch.tensor([10.0 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out[rank] = (gathered, float(t.item()), [b.tolist() for b in batches])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    world, n = 2, 1001
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, n, out), nprocs=world, join=True)
        res = dict(out)
    gathered, tmax, batches = res[0]
    a, b = gathered
    assert set(a).isdisjoint(b)
    assert sorted(a + b) == list(range(n))
    assert tmax == 11.0 and res[1][1] == 11.0
    for bl in batches:
        assert len(bl) == 7 and set(bl) <= set(a)


def test_shard_single_rank_is_everything():
    import bench
    np.testing.assert_array_equal(bench.shard(10, 0, 1), np.arange(10))


def _shard_worker(rank, world, port, out):
    import oracle
    import emd_synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = emd_synth.small_text(4242, 1500, 24, 301, 5, 3, 30)
    bounds = [0, 140, 301]  # uneven contiguous shards
    shard = w.db.subset(np.arange(bounds[rank], bounds[rank + 1]))
    K = 10
    res = []
    for qi in range(w.queries.n):
        tf, tr = oracle.lc_query(w.emb, None, shard, *w.queries.row(qi), "act", 3)
        sym = np.maximum(tf, tr).astype(np.float32)
        order = np.lexsort((np.arange(len(sym)), sym))[:K]
        res.append((order.astype(np.int64), sym[order]))
    gathered = [None] * world
    dist.all_gather_object(gathered, (bounds[rank], res))  # K (distance, id) pairs per shard
    if rank == 0:
        out["gathered"] = gathered
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_database_shards_merge_exactly():
    """Each rank holds a contiguous slice of the documents and computes its own top-K (the
    oracle stands in for the device); one gather of K pairs per shard and emd_topk_merge give
    the top-K of the whole database."""
    import emd_synth
    import oracle
    import paper_1812_02091_gb300 as emd
    emd.load()
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
        gathered = out["gathered"]
    w = emd_synth.small_text(4242, 1500, 24, 301, 5, 3, 30)
    K = 10
    offs = [g[0] for g in gathered]
    for qi in range(w.queries.n):
        shards = [(g[1][qi][0][None, :], g[1][qi][1][None, :]) for g in gathered]
        mi, md = emd.emd_topk_merge(shards, offs, K)
        tf, tr = oracle.lc_query(w.emb, None, w.db, *w.queries.row(qi), "act", 3)
        sym = np.maximum(tf, tr).astype(np.float32)
        order = np.lexsort((np.arange(len(sym)), sym))[:K]
        np.testing.assert_array_equal(mi[0], order)
        np.testing.assert_array_equal(md[0], sym[order])


def test_merge_argument_checks():
    import paper_1812_02091_gb300 as emd
    emd.load()
    a = (np.array([[0, 1]], np.int64), np.array([[0.1, 0.2]], np.float32))
    with pytest.raises(emd.EmdError, match="INVALID_ARG"):
        emd.emd_topk_merge([a], [0], 3)  # K above n_shards * K_shard
    b = (np.array([[0, -1]], np.int64), np.array([[0.05, 0.0]], np.float32))
    mi, md = emd.emd_topk_merge([a, b], [0, 100], 3)  # negative ids skipped, ties by global id
    np.testing.assert_array_equal(mi[0], [100, 0, 1])
    with pytest.raises(emd.EmdError, match="INVALID_ARG"):
        emd.emd_topk_merge([b], [0], 2)  # one result only
