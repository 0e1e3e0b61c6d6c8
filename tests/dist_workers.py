"""Rank bodies of the multi-process (gloo, CPU) tests; kept in a module of
their own so spawned processes can import them by name."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def owned_shards(rank, world, nshards):
    """Consecutive shards per rank (the first ranks take one more)."""
    q, r = divmod(nshards, world)
    first = rank * q + min(rank, r)
    return list(range(first, first + q + (1 if rank < r else 0)))


def halo_body(rank, world, port, total, nshards, out_dir):
    """Each rank fills its windows with the global cell index and exchanges;
    writes its windows to out_dir for the parent to check."""
    from paper_1301_4195_gb300 import shard
    init(rank, world, port)
    parts = shard.partition(total, nshards)
    mine = owned_shards(rank, world, nshards)
    owner = [r for r in range(world) for _ in owned_shards(r, world, nshards)]
    wins = []
    for s in mine:
        first, n = parts[s]
        cells = torch.arange(first, first + n, dtype=torch.float64).reshape(n, 1).repeat(1, 3) + 0.25
        w = shard.window(cells)
        w[:shard.GHOST] = -1.0
        w[-shard.GHOST:] = -1.0
        wins.append(w)
    shard.HaloExchange(mine, nshards, owner).exchange(wins)
    for s, w in zip(mine, wins):
        np.save(os.path.join(out_dir, f"win{s}.npy"), w.numpy())
    dist.barrier()
    dist.destroy_process_group()


def transport_body(rank, world, port, N, L, total, nshards, dt, nsteps, out_dir):
    """Heun transport steps of the wall problem on this rank's shards: the
    oracle's shard right-hand side per stage, the package's halo exchange
    between stages.  Writes the rank's cells to out_dir."""
    import oracle
    from paper_1301_4195_gb300 import inputs, shard
    init(rank, world, port)
    parts = shard.partition(total, nshards)
    mine = owned_shards(rank, world, nshards)
    owner = [r for r in range(world) for _ in owned_shards(r, world, nshards)]
    dx = inputs.wall_grid(total)
    f0 = inputs.wall_profile(N, L, total)
    far = inputs.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)
    halo = shard.HaloExchange(mine, nshards, owner)
    f = [shard.window(torch.from_numpy(f0[parts[s][0]:parts[s][0] + parts[s][1]].copy())) for s in mine]
    f1 = [torch.zeros_like(w) for w in f]
    G = shard.GHOST

    def rhs(i, w):
        s = mine[i]
        return oracle.transport_rhs_window(w.numpy(), N, L, total, parts[s][0], dx, 1.5, (0.0, 0.0, 0.0), far)

    for _ in range(nsteps):
        halo.exchange(f)
        for i in range(len(f)):
            n = parts[mine[i]][1]
            x = f[i][G:G + n].numpy()
            f1[i][G:G + n] = torch.from_numpy(x + dt * rhs(i, f[i]))
        halo.exchange(f1)
        for i in range(len(f)):
            n = parts[mine[i]][1]
            x, y = f[i][G:G + n].numpy(), f1[i][G:G + n].numpy()
            f[i][G:G + n] = torch.from_numpy(0.5 * (x + y + dt * rhs(i, f1[i])))
    for s, w in zip(mine, f):
        np.save(os.path.join(out_dir, f"cells{s}.npy"), w[G:w.shape[0] - G].numpy())
    dist.barrier()
    dist.destroy_process_group()



def bench_max_body(rank, world, port, out_dir):
    """bench.py's max over ranks on gloo: every rank must get the largest value."""
    import bench
    init(rank, world, port)
    got = bench.max_over_ranks(1.5 * (rank + 1), "cpu")
    np.save(os.path.join(out_dir, f"max{rank}.npy"), np.array([got]))
    dist.barrier()
    dist.destroy_process_group()
