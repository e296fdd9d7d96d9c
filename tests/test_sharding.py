"""Multi-rank host logic on CPU: world-size-2 gloo process groups.

Independent cavities are split across ranks without any exchange on the data
path; each rank derives the same assignment on its own, and only the timing is
reduced (max over ranks)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1601_04633_gb300 import inputs, sharding


def test_assignment_is_a_balanced_partition():
    cavs = inputs.batch_sweep()
    w = [c.nx * c.ny for c in cavs]
    for world in (1, 2, 3, 4, 8):
        owner = sharding.assign(w, world)
        loads = [sum(x for x, r in zip(w, owner) if r == q) for q in range(world)]
        assert sum(loads) == sum(w) and len(owner) == len(w)
        assert max(loads) - min(loads) <= max(w)  # greedy bound
        shards = [sharding.shard(cavs, q, world) for q in range(world)]
        assert sorted(id(c) for s in shards for c in s) == sorted(id(c) for c in cavs)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cavs = inputs.batch_sweep()
    mine = sharding.shard(cavs, rank, world)
    nodes = sum(c.nx * c.ny for c in mine)
    import torch

    # every rank sees every other rank's share: together they cover the sweep once
    allnodes = [None] * world
    dist.all_gather_object(allnodes, (rank, nodes, [c.seed for c in mine]))
    t = sharding.reduce_max_seconds(0.5 + rank, dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, allnodes, t))


@pytest.mark.parametrize("world", [2])
def test_two_rank_gloo_sharding(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cavs = inputs.batch_sweep()
    for rank, allnodes, t in out:
        assert t == 0.5 + (world - 1)  # max over ranks
        seeds = sorted(s for _, _, ss in allnodes for s in ss)
        assert seeds == sorted(c.seed for c in cavs)
        assert sum(n for _, n, _ in allnodes) == sum(c.nx * c.ny for c in cavs)
