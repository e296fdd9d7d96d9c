"""One cavity split into y-slabs of whole rows: one slab per rank (one GPU per
rank), or several slabs on one GPU.

The streaming of the two lattices (Eqs. 25 and 36) moves populations by at
most one row, so one time step of a slab needs, besides its own rows, one row
of each neighbour: the populations moving up (e_y = +1) of the last row of the
slab below and those moving down (e_y = -1) of the first row of the slab
above. Each slab context holds these as halo rows (``dmrt_create_slab``), and
between steps every slab sends its two boundary messages and receives its
neighbours' (``halo_exchange``: point-to-point sends and receives, one pair
per face). The hot-wall Nusselt mean of the cavity (Eq. 19) is the sum of the
slabs' shares. Every slab's state is bit for bit that of the same rows of the
whole cavity stepped as one context.

The exchange runs on any ``torch.distributed`` backend: NCCL between GPUs, or
gloo on CPU tensors (the host-side protocol is tested that way).
"""
from __future__ import annotations

import numpy as np


def partition_rows(ny: int, parts: int):
    """(y0, rows) of each of ``parts`` contiguous slabs of ``ny`` rows, as even
    as possible (the first ny % parts slabs take one row more)."""
    if parts < 1 or parts > ny:
        raise ValueError("need 1 <= parts <= ny")
    base, extra = divmod(ny, parts)
    out, y0 = [], 0
    for k in range(parts):
        rows = base + (1 if k < extra else 0)
        out.append((y0, rows))
        y0 += rows
    return out


def halo_exchange(dist, rank: int, world: int, send_below, send_above, recv_below, recv_above, group=None):
    """Swap boundary messages with the neighbouring ranks: rank r sends
    ``send_below`` to r - 1 and ``send_above`` to r + 1, and receives into
    ``recv_below`` from r - 1 and into ``recv_above`` from r + 1 (the first and
    last ranks have one neighbour). Blocks until the transfers are done (for
    NCCL: until they are ordered before later work on the current stream)."""
    ops = []
    if rank > 0:
        ops.append(dist.P2POp(dist.isend, send_below, rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, recv_below, rank - 1, group))
    if rank < world - 1:
        ops.append(dist.P2POp(dist.isend, send_above, rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, recv_above, rank + 1, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class LocalSlabs:
    """Several slabs of one cavity on one GPU, stepped in turn on one stream;
    the messages are delivered by device copies."""

    def __init__(self, params, parts: int, theta0=None, device="cuda", theta_hot_profile=None):
        from . import dmrt as D

        self.parts = partition_rows(params.ny, parts)
        self.slabs = []
        for y0, rows in self.parts:
            th = None if theta0 is None else np.asarray(theta0)[y0:y0 + rows]
            prof = None if theta_hot_profile is None else np.asarray(theta_hot_profile)[y0:y0 + rows]
            self.slabs.append(D.Slab(params, y0, rows, theta0=th, device=device, theta_hot_profile=prof))
        self._exchange(pack=True)

    def _exchange(self, pack=False):
        s = self.slabs
        if pack:
            for sl in s:
                sl.pack()
        for k in range(len(s) - 1):
            s[k].from_above.copy_(s[k + 1].to_below)
            s[k + 1].from_below.copy_(s[k].to_above)
        for sl in s:
            sl.unpack()

    def step(self, n: int):
        for _ in range(int(n)):
            for sl in self.slabs:
                sl.step_one()
            self._exchange()
        for sl in self.slabs:
            sl.finish()

    def get_state(self) -> np.ndarray:
        return np.concatenate([sl.get_state() for sl in self.slabs], axis=1)

    def nusselt(self, series_cap: int = 0):
        """(mean, local [ny], series): the cavity's values from the slabs' shares."""
        parts = [sl.nusselt(series_cap) for sl in self.slabs]
        mean = sum(p[0] for p in parts)
        local = np.concatenate([p[1] for p in parts])
        series = np.sum([p[2] for p in parts], axis=0) if series_cap else np.zeros(0)
        return mean, local, series

    def check(self):
        for sl in self.slabs:
            sl.check()

    def close(self):
        for sl in self.slabs:
            sl.close()


class DistributedSlab:
    """This rank's slab of a cavity split over ``world`` ranks (one GPU each);
    ``dist`` is ``torch.distributed`` with an initialised process group."""

    def __init__(self, dist, params, rank: int, world: int, theta0=None, device="cuda", **kw):
        from . import dmrt as D

        self.dist, self.rank, self.world = dist, rank, world
        self.y0, self.rows = partition_rows(params.ny, world)[rank]
        th = None if theta0 is None else np.asarray(theta0)[self.y0:self.y0 + self.rows]
        self.slab = D.Slab(params, self.y0, self.rows, theta0=th, device=device, **kw)
        self.slab.pack()
        self._exchange()

    def _exchange(self):
        s = self.slab
        halo_exchange(self.dist, self.rank, self.world, s.to_below, s.to_above, s.from_below, s.from_above)
        s.unpack()

    def step(self, n: int):
        for _ in range(int(n)):
            self.slab.step_one()
            self._exchange()
        self.slab.finish()

    def nusselt_series(self, cap: int):
        """The cavity's mean-Nu history (the slabs' shares summed over ranks)."""
        import torch

        series = self.slab.nusselt(cap)[2]
        t = torch.from_numpy(np.ascontiguousarray(series)).to(self.slab.device)
        self.dist.all_reduce(t)
        return t.cpu().numpy()

    def close(self):
        self.slab.close()
