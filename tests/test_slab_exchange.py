"""Host-side logic of the y-slab decomposition, on CPU: the row partition, and
the halo exchange protocol between ranks over world-size-2 and -3 gloo process
groups (the same function moves the device messages over NCCL)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1601_04633_gb300 import slabs


def test_partition_rows_covers_the_cavity_evenly():
    for ny in (2, 7, 301, 4096):
        for parts in range(1, min(ny, 9) + 1):
            pr = slabs.partition_rows(ny, parts)
            assert len(pr) == parts and pr[0][0] == 0
            assert all(a[0] + a[1] == b[0] for a, b in zip(pr, pr[1:]))
            assert pr[-1][0] + pr[-1][1] == ny
            rows = [r for _, r in pr]
            assert max(rows) - min(rows) <= 1 and min(rows) >= 1
    with pytest.raises(ValueError):
        slabs.partition_rows(3, 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 37
    # Messages tagged by sender and face: 100 r + 1 (downward face), 100 r + 2 (upward face).
    send_below = torch.full((n,), 100 * rank + 1, dtype=torch.uint8)
    send_above = torch.full((n,), 100 * rank + 2, dtype=torch.uint8)
    recv_below = torch.zeros(n, dtype=torch.uint8)
    recv_above = torch.zeros(n, dtype=torch.uint8)
    for _ in range(3):  # repeated exchanges, as between time steps
        slabs.halo_exchange(dist, rank, world, send_below, send_above, recv_below, recv_above)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, recv_below.tolist(), recv_above.tolist()))


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, below, above = q.get(timeout=120)
        out[rank] = (below, above)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (below, above) in out.items():
        # From the rank below: its upward face; from the rank above: its downward face.
        assert below == ([100 * (rank - 1) + 2] * 37 if rank > 0 else [0] * 37)
        assert above == ([100 * (rank + 1) + 1] * 37 if rank < world - 1 else [0] * 37)
