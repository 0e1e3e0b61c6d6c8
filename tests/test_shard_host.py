"""Domain decomposition on the host (Sec. 4.2), no GPU.

* partition: contiguous shards, sizes within one cell, each >= 2 cells;
* the halo exchange of the package moves exactly the neighbouring cells, in
  one process and across gloo ranks (world sizes 2 and 3, one or two shards
  per rank);
* the decomposition itself: Heun transport steps of the wall problem with the
  oracle's shard right-hand side and the package's exchange reproduce the
  unsharded oracle bit for bit.
"""
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1301_4195_gb300 import inputs, shard

import dist_workers
from dist_workers import free_port


@pytest.mark.parametrize("total,parts", [(2, 1), (7, 3), (40, 3), (128, 8), (9, 4)])
def test_partition(total, parts):
    p = shard.partition(total, parts)
    assert len(p) == parts
    assert p[0][0] == 0 and sum(n for _, n in p) == total
    for (f0, n0), (f1, _) in zip(p, p[1:]):
        assert f1 == f0 + n0
    sizes = [n for _, n in p]
    assert min(sizes) >= 2 and max(sizes) - min(sizes) <= 1


def test_partition_rejects_small_shards():
    with pytest.raises(ValueError):
        shard.partition(5, 3)


def _check_windows(total, parts, wins):
    """window cell i of shard s = grid cell first-2+i (value index + 0.25);
    ghosts outside the grid keep their fill (-1)."""
    for s, (first, n) in enumerate(parts):
        w = wins[s]
        assert w.shape[0] == n + 4
        for i in range(n + 4):
            j = first - 2 + i
            expect = j + 0.25 if 0 <= j < total else -1.0
            assert np.all(w[i] == expect), (s, i, w[i], expect)


def test_halo_exchange_in_one_process():
    total, nshards = 23, 4
    parts = shard.partition(total, nshards)
    wins = []
    for first, n in parts:
        cells = torch.arange(first, first + n, dtype=torch.float64).reshape(n, 1).repeat(1, 3) + 0.25
        w = shard.window(cells)
        w[:2] = -1.0
        w[-2:] = -1.0
        wins.append(w)
    shard.HaloExchange(range(nshards), nshards).exchange(wins)
    _check_windows(total, parts, [w.numpy() for w in wins])


@pytest.mark.parametrize("world,nshards", [(2, 2), (3, 3), (2, 4)])
def test_halo_exchange_gloo(world, nshards):
    total = 17
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(dist_workers.halo_body, args=(world, free_port(), total, nshards, d), nprocs=world, join=True)
        wins = [np.load(f"{d}/win{s}.npy") for s in range(nshards)]
    _check_windows(total, shard.partition(total, nshards), wins)


def _unsharded(N, L, total, dt, nsteps, oracle):
    dx = inputs.wall_grid(total)
    far = inputs.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)
    f = inputs.wall_profile(N, L, total)
    for _ in range(nsteps):
        f = oracle.transport_rk2(f, N, L, dx, 1.5, (0.0, 0.0, 0.0), far, dt)
    return f


@pytest.mark.parametrize("world,nshards,total", [(2, 2, 12), (3, 3, 11), (2, 3, 9)])
def test_sharded_transport_matches_unsharded_oracle(oracle_mod, world, nshards, total):
    N, L, dt, nsteps = 8, 6.0, 0.01, 3
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(dist_workers.transport_body, args=(world, free_port(), N, L, total, nshards, dt, nsteps, d),
                 nprocs=world, join=True)
        got = np.concatenate([np.load(f"{d}/cells{s}.npy") for s in range(nshards)])
    ref = _unsharded(N, L, total, dt, nsteps, oracle_mod)
    assert got.shape == ref.shape
    assert np.isfinite(got).all()
    assert np.array_equal(got, ref), np.abs(got - ref).max()


def test_shard_rhs_reads_only_its_window(oracle_mod):
    """The window's cells outside the grid are never read (NaN there stays out
    of the result); every shard's right-hand side equals the unsharded one's
    rows."""
    N, L, total = 8, 6.0, 10
    dx = inputs.wall_grid(total)
    far = inputs.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)
    f = inputs.wall_profile(N, L, total)
    full = np.full((total + 4, N, N, N), np.nan)
    full[2:-2] = f
    r_all = oracle_mod.transport_rhs_window(full, N, L, total, 0, dx, 1.5, (0, 0, 0), far)
    assert np.isfinite(r_all).all()
    for first, n in shard.partition(total, 4):
        w = np.full((n + 4, N, N, N), np.nan)
        lo, hi = max(first - 2, 0), min(first + n + 2, total)
        w[lo - (first - 2):hi - (first - 2)] = f[lo:hi]
        r = oracle_mod.transport_rhs_window(w, N, L, total, first, dx, 1.5, (0, 0, 0), far)
        assert np.array_equal(r, r_all[first:first + n])
