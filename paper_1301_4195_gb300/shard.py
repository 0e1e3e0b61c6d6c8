"""Domain decomposition of the 1-D wall problem (Sec. 4.2).

The collision step is local to each spatial cell, so the x-grid splits into
contiguous shards with no communication for it; the transport needs, per
Runge-Kutta stage, two ghost cells on each side of a shard, copied from the
neighbouring shards.  This module holds the host side of that scheme:

* ``partition`` splits the grid into contiguous shards (sizes differ by at most
  one cell, each at least two cells);
* ``HaloExchange`` fills the ghost cells of the shards one process owns, by
  device copies between its own consecutive shards and by point-to-point
  messages (torch.distributed: NCCL between GPUs, gloo between CPU ranks) with
  the processes that own the neighbouring shards;
* ``ShardedWall`` runs Strang steps of the wall problem over those shards:
  every stage of the method runs in libcs (``cs_transport_shard_stage`` and
  ``cs_relax``), the exchange sits between the stages.

A shard's state is a window of ncells + 4 cells, window cell i = grid cell
first - 2 + i, the shard's own cells at 2 .. ncells+1.  Because every face is
computed from the same data as on the unsharded grid, the sharded run
reproduces ``cs_step`` bit for bit.

The paper orders blocking sends and receives by the parity of the rank so
that they cannot deadlock; here every message is posted non-blocking at once
and then waited for, which cannot deadlock either.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch

from . import api

GHOST = 2  # ghost cells per side: a face flux reads cells c-2 .. c+1


def partition(total: int, parts: int) -> List[Tuple[int, int]]:
    """(first, ncells) of each of `parts` contiguous shards of `total` cells;
    the first total % parts shards get one cell more.  Every shard needs at
    least two cells (the wall flux reads cells 0 and 1)."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    if total < 2 * parts:
        raise ValueError(f"{total} cells cannot give {parts} shards of >= 2 cells")
    q, r = divmod(total, parts)
    out, first = [], 0
    for i in range(parts):
        n = q + (1 if i < r else 0)
        out.append((first, n))
        first += n
    return out


def window(cells: torch.Tensor) -> torch.Tensor:
    """A window [ncells + 4, ...] holding `cells` at 2 .. ncells+1 (ghosts zero)."""
    w = torch.zeros((cells.shape[0] + 2 * GHOST,) + tuple(cells.shape[1:]), dtype=cells.dtype, device=cells.device)
    w[GHOST:GHOST + cells.shape[0]].copy_(cells)
    return w


def interior(w: torch.Tensor) -> torch.Tensor:
    return w[GHOST:w.shape[0] - GHOST]


class HaloExchange:
    """Fills the ghost cells of this process's shards.

    shards: global indices (consecutive) of the shards this process owns, out
    of nshards; owner[s] is the rank that owns shard s (None: single process).
    exchange(windows) takes this process's windows in shard order.  Ghosts
    beyond the grid's ends are left as they are (never read)."""

    def __init__(self, shards: Sequence[int], nshards: int, owner: Optional[Sequence[int]] = None, group=None):
        self.shards = list(shards)
        if self.shards != list(range(self.shards[0], self.shards[0] + len(self.shards))):
            raise ValueError("a process must own consecutive shards")
        self.nshards = nshards
        self.owner = list(owner) if owner is not None else None
        self.group = group
        if self.owner is None and len(self.shards) != nshards:
            raise ValueError("without torch.distributed one process owns every shard")

    def exchange(self, windows: Sequence[torch.Tensor]):
        if len(windows) != len(self.shards):
            raise ValueError("one window per owned shard")
        G = GHOST
        # neighbours inside this process: device copies
        for i in range(len(windows) - 1):
            a, b = windows[i], windows[i + 1]
            na, nb = a.shape[0] - 2 * G, b.shape[0] - 2 * G
            a[na + G:na + 2 * G].copy_(b[G:2 * G])   # right ghosts of a <- first cells of b
            b[0:G].copy_(a[na:na + G])               # left ghosts of b <- last cells of a
        if self.owner is None:
            return
        import torch.distributed as dist
        first, last = self.shards[0], self.shards[-1]
        wl, wr = windows[0], windows[-1]
        nr = wr.shape[0] - 2 * G
        reqs = []
        # tag 1: cells moving right (into a left ghost), tag 2: moving left
        if first > 0:
            peer = self.owner[first - 1]
            reqs.append(dist.isend(wl[G:2 * G].contiguous(), peer, group=self.group, tag=2))
            reqs.append(dist.irecv(wl[0:G], peer, group=self.group, tag=1))
        if last < self.nshards - 1:
            peer = self.owner[last + 1]
            reqs.append(dist.isend(wr[nr:nr + G].contiguous(), peer, group=self.group, tag=1))
            reqs.append(dist.irecv(wr[nr + G:nr + 2 * G], peer, group=self.group, tag=2))
        for r in reqs:
            r.wait()


class ShardedWall:
    """Strang steps (Sec. 3.1) of the wall problem over the shards one process owns.

    handle: an api.Handle; cells: list of this process's shard states
    [ncells_s, N, N, N] (float64, on the handle's device); firsts: their first
    grid cells; total: cells of the whole grid; dx: all total widths (device);
    f_far: [N^3] far-field gas (device)."""

    def __init__(self, handle: "api.Handle", cells: Sequence[torch.Tensor], firsts: Sequence[int], total: int,
                 dx: torch.Tensor, f_far: torch.Tensor, wall_T: float, wall_V, halo: HaloExchange, stream=None):
        self.h = handle
        self.total = int(total)
        self.firsts = [int(x) for x in firsts]
        self.n = [int(c.shape[0]) for c in cells]
        self.f = [window(c) for c in cells]
        self.f1 = [torch.empty_like(w) for w in self.f]
        self.dom = api._domain(dx, f_far, wall_T, wall_V)
        self._keep = (dx, f_far)
        self.halo = halo
        self.stream = stream
        self._prepared = False

    def _prepare(self):
        # one handle holds the tables: they cover the whole grid, and the
        # workspace has room for the largest shard
        big = max(range(len(self.n)), key=lambda i: self.n[i])
        api.cs_transport_shard_prepare(self.h.ptr, self.n[big], self.firsts[big], self.total, self.dom, self.stream)
        self._prepared = True

    def _stage(self, i, fin, a, x, b, y, c, out):
        api.cs_transport_shard_stage(self.h.ptr, fin, self.n[i], self.firsts[i], self.total, self.dom,
                                     a, x, b, y, c, out, self.stream)

    def transport(self, dt: float):
        """One Heun step of the transport: exchange, stage, exchange, stage."""
        if not self._prepared:
            self._prepare()
        self.halo.exchange(self.f)
        for i in range(len(self.f)):
            self._stage(i, self.f[i], 1.0, interior(self.f[i]), 0.0, None, dt, interior(self.f1[i]))
        self.halo.exchange(self.f1)
        for i in range(len(self.f)):
            fi = interior(self.f[i])
            self._stage(i, self.f1[i], 0.5, fi, 0.5, interior(self.f1[i]), 0.5 * dt, fi)

    def collide(self, dt: float, eps: float = 1.0):
        """One Heun step of df/dt = P_N Qt(f) / eps on every cell (no communication)."""
        for i in range(len(self.f)):
            api.cs_relax(self.h.ptr, interior(self.f[i]), self.n[i], dt, eps, 1, stream=self.stream)

    def step(self, dt: float, eps: float = 1.0, nsteps: int = 1):
        for _ in range(nsteps):
            self.transport(0.5 * dt)
            self.collide(dt, eps)
            self.transport(0.5 * dt)

    def cells(self) -> List[torch.Tensor]:
        return [interior(w) for w in self.f]
