"""Transport in two space dimensions on the GPU against the oracle.

x: the wall problem's direction (non-uniform cells, wall at x = 0, far field
at the end); y: periodic, uniform cells.  FP64 transport 1e-13; Strang steps
1e-12 (FP64 handle) and 1e-7 (FP32 handle); a state uniform in y follows the
1-D transport; graph replay equals direct launches bit for bit.
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


def rel(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def problem(N, nx, ny, Y=3.0, seed=0):
    """Wall profile in x times a smooth periodic modulation in y, plus noise."""
    dx = I.wall_grid(nx)
    fx = I.wall_profile(N, L, nx)
    y = (np.arange(ny) + 0.5) * Y / ny
    mod = 1.0 + 0.3 * np.sin(2 * np.pi * y / Y)
    f = fx[:, None] * mod[None, :, None, None, None]
    f = f * (1 + 0.02 * np.random.default_rng(seed).standard_normal(f.shape))
    far = I.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)
    return dx, f, far, Y / ny


@pytest.mark.parametrize("N,nx,ny", [(8, 10, 6), (8, 7, 1), (4, 9, 5)])
def test_transport2d_matches_oracle(cs, orc, N, nx, ny):
    dx, f, far, dy = problem(N, nx, ny)
    h = cs.Handle(N, L, 1.0, "fp64")
    fd = dev(f)
    ref = f
    for _ in range(3):
        h.transport2d(fd, dev(dx), dev(far), 1.5, (0.0, 0.1, 0.0), ny, dy, 0.005)
        ref = orc.transport2d_rk2(ref, N, L, nx, ny, dx, dy, 1.5, (0.0, 0.1, 0.0), far, 0.005)
    assert rel(host(fd).reshape(ref.shape), ref) < 1e-13
    h.close()


def test_uniform_in_y_follows_the_1d_transport(cs):
    N, nx, ny = 8, 12, 4
    dx = I.wall_grid(nx)
    f1 = I.wall_profile(N, L, nx)
    far = I.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)
    h = cs.Handle(N, L, 1.0, "fp64")
    a = dev(f1)
    h.transport(a, dev(dx), dev(far), 1.5, (0.0, 0.0, 0.0), 0.01)
    b = dev(np.repeat(f1[:, None], ny, axis=1))
    h.transport2d(b, dev(dx), dev(far), 1.5, (0.0, 0.0, 0.0), ny, 0.4, 0.01)
    ra, rb = host(a), host(b)
    for j in range(ny):
        assert rel(rb[:, j], ra) < 1e-14
    h.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-7)])
def test_strang_step2d_matches_oracle(cs, orc, prec, tol):
    N, nx, ny = 8, 6, 4
    dx, f, far, dy = problem(N, nx, ny, seed=1)
    h = cs.Handle(N, L, 1.0, prec)
    fd = dev(f)
    h.step2d(fd, dev(dx), dev(far), 1.5, (0.0, 0.0, 0.0), ny, dy, 0.01, nsteps=2)
    ref = f
    for _ in range(2):
        ref = orc.strang_step2d(ref, N, L, 1.0, nx, ny, dx, dy, 1.5, (0.0, 0.0, 0.0), far, 0.01)
    assert rel(host(fd).reshape(ref.shape), ref) < tol
    h.close()


def test_step2d_graph_replay_matches_direct_launches(cs):
    N, nx, ny = 16, 12, 4
    dx, f, far, dy = problem(N, nx, ny, seed=2)
    h = cs.Handle(N, L, 1.0, "fp32")
    dxd, fard = dev(dx), dev(far)
    fa, fb = dev(f), dev(f)
    cs.cs_launch_count(reset=True)
    h.step2d(fa, dxd, fard, 1.5, (0.0, 0.0, 0.0), ny, dy, 0.01, nsteps=3)
    replayed = cs.cs_launch_count(reset=True)
    cs.cs_profile(h.ptr, True)
    h.step2d(fb, dxd, fard, 1.5, (0.0, 0.0, 0.0), ny, dy, 0.01, nsteps=3)
    direct = cs.cs_launch_count(reset=True)
    cs.cs_profile(h.ptr, False)
    cs.cs_profile_read(h.ptr, reset=True)
    assert np.array_equal(host(fa), host(fb))
    assert replayed == direct == 3 * 10
    cs.cs_status(h.ptr)
    h.close()


def test_domain2d_errors(cs):
    N, nx = 8, 6
    h = cs.Handle(N, L, 1.0, "fp64")
    dx, f, far, dy = problem(N, nx, 2)
    fd, dxd, fard = dev(f), dev(dx), dev(far)
    for ny, dyy in ((0, 0.5), (2, 0.0), (2, float("nan"))):
        with pytest.raises(cs.CSError) as e:
            cs.cs_transport2d(h.ptr, fd, nx, cs._domain2d(dxd, fard, 1.5, (0, 0, 0), ny, dyy), 0.01)
        assert e.value.code == cs.CS_EINVAL
    with pytest.raises(cs.CSError):
        cs.cs_transport2d(h.ptr, fd, 1, cs._domain2d(dxd, fard, 1.5, (0, 0, 0), 2, 0.5), 0.01)
    torch.cuda.synchronize()
    h.close()
