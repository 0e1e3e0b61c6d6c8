"""Sharded wall problem on one GPU (Sec. 4.2): several shards in one process,
ghosts filled by device copies between stages.

* one shard stage against the oracle's shard right-hand side (FP64, 1e-13);
* Strang steps over 2-4 shards reproduce the unsharded cs_step bit for bit
  (every face and every cell sees the same data and the same arithmetic);
* the stage refuses tables that were not prepared for its grid.
"""
import numpy as np
import pytest
import torch

from paper_1301_4195_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 6.0


@pytest.fixture(scope="module")
def cs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_4195_gb300 import build
    build.build()
    from paper_1301_4195_gb300 import api
    return api


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def wall(N, total):
    return I.wall_grid(total), I.wall_profile(N, L, total), I.maxwellian(N, L, 1.0, (0, 0, 0), 1.0)


@pytest.mark.parametrize("first,n,total", [(0, 5, 12), (4, 4, 12), (7, 5, 12), (0, 12, 12)])
def test_shard_stage_matches_oracle(cs, orc, first, n, total):
    N = 8
    dx, f, far = wall(N, total)
    h = cs.Handle(N, L, 1.0, "fp64")
    w = np.zeros((n + 4, N, N, N))
    lo, hi = max(first - 2, 0), min(first + n + 2, total)
    w[lo - (first - 2):hi - (first - 2)] = f[lo:hi]
    dxd, fard = dev(dx), dev(far)
    dom = cs._domain(dxd, fard, 1.5, (0.0, 0.1, 0.0))
    cs.cs_transport_shard_prepare(h.ptr, n, first, total, dom)
    wd = dev(w)
    out = torch.empty((n, N, N, N), dtype=torch.float64, device="cuda")
    cs.cs_transport_shard_stage(h.ptr, wd, n, first, total, dom, 0.0, None, 0.0, None, 1.0, out)
    ref = orc.transport_rhs_window(w, N, L, total, first, dx, 1.5, (0.0, 0.1, 0.0), far)
    got = host(out)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    h.close()


@pytest.mark.parametrize("prec,N,total,nshards", [("fp64", 8, 20, 3), ("fp32", 16, 40, 4), ("fp32", 8, 9, 2)])
def test_sharded_steps_match_cs_step(cs, prec, N, total, nshards):
    from paper_1301_4195_gb300 import shard
    dx, f, far = wall(N, total)
    dxd, fard = dev(dx), dev(far)
    h_ref = cs.Handle(N, L, 1.0, prec)
    fr = dev(f)
    h_ref.step(fr, dxd, fard, 1.5, (0.0, 0.0, 0.0), 0.01, nsteps=3)
    ref = host(fr)

    h = cs.Handle(N, L, 1.0, prec)
    parts = shard.partition(total, nshards)
    cells = [dev(f[a:a + n]) for a, n in parts]
    sw = shard.ShardedWall(h, cells, [a for a, _ in parts], total, dxd, fard, 1.5, (0.0, 0.0, 0.0),
                           shard.HaloExchange(range(nshards), nshards))
    sw.step(0.01, nsteps=3)
    got = np.concatenate([host(c) for c in sw.cells()])
    assert np.isfinite(got).all()
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    cs.cs_status(h.ptr)
    h.close()
    h_ref.close()


def test_stage_needs_prepared_tables(cs):
    N, total, n = 8, 10, 5
    dx, f, far = wall(N, total)
    dxd, fard = dev(dx), dev(far)
    h = cs.Handle(N, L, 1.0, "fp64")
    dom = cs._domain(dxd, fard, 1.5, (0.0, 0.0, 0.0))
    w = torch.zeros((n + 4, N, N, N), dtype=torch.float64, device="cuda")
    out = torch.empty((n, N, N, N), dtype=torch.float64, device="cuda")
    with pytest.raises(cs.CSError) as e:
        cs.cs_transport_shard_stage(h.ptr, w, n, 0, total, dom, 0.0, None, 0.0, None, 1.0, out)
    assert e.value.code == cs.CS_EINVAL
    cs.cs_transport_shard_prepare(h.ptr, n, 0, total, dom)
    cs.cs_transport_shard_stage(h.ptr, w, n, 5, total, dom, 0.0, None, 0.0, None, 1.0, out)
    # a different wall, or tables overwritten by an unsharded call, are refused
    dom2 = cs._domain(dxd, fard, 1.6, (0.0, 0.0, 0.0))
    with pytest.raises(cs.CSError):
        cs.cs_transport_shard_stage(h.ptr, w, n, 0, total, dom2, 0.0, None, 0.0, None, 1.0, out)
    fa = dev(f)
    h.transport(fa, dxd, fard, 1.5, (0.0, 0.0, 0.0), 0.01)
    with pytest.raises(cs.CSError):
        cs.cs_transport_shard_stage(h.ptr, w, n, 0, total, dom, 0.0, None, 0.0, None, 1.0, out)
    # out inside the window it reads
    cs.cs_transport_shard_prepare(h.ptr, n, 0, total, dom)
    with pytest.raises(cs.CSError):
        cs.cs_transport_shard_stage(h.ptr, w, n, 0, total, dom, 0.0, None, 0.0, None, 1.0, w[2:2 + n])
    # shards outside the grid
    for first, nn in ((-1, 5), (6, 5), (0, 1)):
        with pytest.raises(cs.CSError):
            cs.cs_transport_shard_stage(h.ptr, w, nn, first, total, dom, 0.0, None, 0.0, None, 1.0, out)
    torch.cuda.synchronize()
    h.close()
