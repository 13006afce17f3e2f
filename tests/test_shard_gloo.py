"""Multi-rank host logic on CPU (gloo, world size 2): LPT sharding covers every
tile exactly once, loads balance, and the max-over-ranks timing reduction the
benchmark uses works."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1311_0378_gb300.shard import lpt_shards, my_tiles


def test_lpt_properties():
    costs = [5, 1, 1, 1, 1, 1, 4, 3, 3]
    sh = lpt_shards(costs, 2)
    assert sorted(i for s in sh for i in s) == list(range(len(costs)))
    loads = [sum(costs[i] for i in s) for s in sh]
    assert max(loads) - min(loads) <= max(costs)
    assert lpt_shards(costs, 1) == [sorted(range(9), key=lambda i: (-costs[i], i))]
    with pytest.raises(ValueError):
        lpt_shards(costs, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, costs, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = my_tiles(costs, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    t = torch.tensor([float(sum(costs[i] for i in mine))])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((got, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    costs = [float((i * 37) % 11 + 1) for i in range(40)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    allt = sorted(i for s in got for i in s)
    assert allt == list(range(40))
    assert tmax == max(sum(costs[i] for i in s) for s in got)
