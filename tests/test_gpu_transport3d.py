"""Transport in three space dimensions on the GPU against the oracle.

x: the wall problem's direction (non-uniform cells, wall at x = 0, far field
at the end); y and z: periodic, uniform cells.  FP64 transport 1e-13;
Strang steps 1e-12 (FP64 handle) and 1e-7 (FP32 handle); one z-layer equals
the GPU's 2-D transport bit for bit; graph replay equals direct launches bit
for bit.
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


def problem(N, nx, ny, nz, Y=3.0, Z=2.0, seed=0):
    """Wall profile in x times smooth periodic modulations in y and z, plus noise."""
    dx = I.wall_grid(nx)
    fx = I.wall_profile(N, L, nx)
    y = (np.arange(ny) + 0.5) * Y / ny
    z = (np.arange(nz) + 0.5) * Z / nz
    my = 1.0 + 0.3 * np.sin(2 * np.pi * y / Y)
    mz = 1.0 + 0.2 * np.cos(2 * np.pi * z / Z)
    f = fx[:, None, None] * (my[:, None] * mz[None, :])[None, :, :, None, None, None]
    f = f * (1 + 0.02 * np.random.default_rng(seed).standard_normal(f.shape))
    far = I.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)
    return dx, f, far, Y / ny, Z / nz


@pytest.mark.parametrize("N,nx,ny,nz", [(8, 6, 3, 4), (8, 9, 1, 5), (4, 5, 4, 1)])
def test_transport3d_matches_oracle(cs, orc, N, nx, ny, nz):
    dx, f, far, dy, dz = problem(N, nx, ny, nz)
    h = cs.Handle(N, L, 1.0, "fp64")
    fd = dev(f)
    ref = f
    for _ in range(3):
        h.transport3d(fd, dev(dx), dev(far), 1.5, (0.0, 0.1, -0.1), ny, dy, nz, dz, 0.004)
        ref = orc.transport3d_rk2(ref, N, L, nx, ny, nz, dx, dy, dz, 1.5, (0.0, 0.1, -0.1), far, 0.004)
    assert rel(host(fd), ref) < 1e-13
    h.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-7)])
def test_strang3d_matches_oracle(cs, orc, prec, tol):
    N, nx, ny, nz = 8, 5, 3, 3
    dx, f, far, dy, dz = problem(N, nx, ny, nz, seed=1)
    h = cs.Handle(N, L, 1.0, prec)
    fd = dev(f)
    h.step3d(fd, dev(dx), dev(far), 1.5, (0, 0, 0), ny, dy, nz, dz, 0.01, nsteps=2)
    ref = orc.strang_step3d(f, N, L, 1.0, nx, ny, nz, dx, dy, dz, 1.5, (0, 0, 0), far, 0.01)
    ref = orc.strang_step3d(ref, N, L, 1.0, nx, ny, nz, dx, dy, dz, 1.5, (0, 0, 0), far, 0.01)
    assert rel(host(fd), ref) < tol
    cs.cs_status(h.ptr)
    h.close()


def test_single_z_layer_equals_the_2d_transport(cs):
    N, nx, ny = 16, 12, 5
    dx, f, far, dy, dz = problem(N, nx, ny, 1, seed=2)
    h = cs.Handle(N, L, 1.0, "fp32")
    a, b = dev(f), dev(f[:, :, 0])
    for _ in range(2):
        h.transport3d(a, dev(dx), dev(far), 1.5, (0.0, 0.2, 0.0), ny, dy, 1, 0.7, 0.01)
        h.transport2d(b, dev(dx), dev(far), 1.5, (0.0, 0.2, 0.0), ny, dy, 0.01)
    assert np.array_equal(host(a)[:, :, 0], host(b))
    h.close()


def test_step3d_replay_equals_direct_launches(cs):
    N, nx, ny, nz = 16, 8, 2, 3
    dx, f, far, dy, dz = problem(N, nx, ny, nz, seed=3)
    h = cs.Handle(N, L, 1.0, "fp32")
    a, b = dev(f), dev(f)
    h.step3d(a, dev(dx), dev(far), 1.5, (0, 0, 0), ny, dy, nz, dz, 0.01, nsteps=3)
    cs.cs_profile(h.ptr, True)
    h.step3d(b, dev(dx), dev(far), 1.5, (0, 0, 0), ny, dy, nz, dz, 0.01, nsteps=3)
    cs.cs_profile(h.ptr, False)
    cs.cs_profile_read(h.ptr, reset=True)
    assert np.array_equal(host(a), host(b))
    with pytest.raises(cs.CSError):  # ny * nz above the launch limit
        cs.cs_transport3d(h.ptr, a, nx, cs._domain3d(dev(dx), dev(far), 1.5, (0, 0, 0), 300, 0.1, 300, 0.1), 0.01)
    h.close()
