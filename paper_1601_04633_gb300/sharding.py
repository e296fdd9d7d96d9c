"""Sharding of independent cavities across ranks (one GPU per rank).

The cavities of a sweep are independent, so N ranks split them with no
exchange on the data path: each rank steps its own share (a batch on its GPU)
and only the timing is combined (max over ranks). The split balances node
counts greedily (largest first onto the least-loaded rank, ties to the lower
rank), which is deterministic, so every rank computes the same assignment
without communicating.
"""
from __future__ import annotations


def assign(weights, world: int):
    """Rank of each item: largest-first greedy balance of the item weights."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0] * world
    owner = [0] * len(weights)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += weights[i]
    return owner


def shard(cavities, rank: int, world: int):
    """The cavities rank ``rank`` of ``world`` steps (in their original order)."""
    owner = assign([c.nx * c.ny for c in cavities], world)
    return [c for c, r in zip(cavities, owner) if r == rank]


def reduce_max_seconds(seconds: float, dist=None) -> float:
    """Max over ranks of a per-rank time (the job's time); identity without a group."""
    if dist is None or not dist.is_initialized():
        return seconds
    import torch

    t = torch.tensor([seconds], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
