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
