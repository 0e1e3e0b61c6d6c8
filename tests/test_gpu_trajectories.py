"""Whole runs of the wall problem, float path against the plain double path
on the GPU (both checked against the oracle step by step elsewhere): the
float convolution's error must not grow into the solution.

* The 128-cell N = 16 wall problem (unit Maxwellian, wall at T_w = 1.5),
  200 Strang steps of dt = 0.01: float and double states agree to 1e-5 of
  the largest value.
* N = 32 (32 cells of the same grid), 20 steps: the same on the wall cell,
  its neighbour, an interior and the last cell.
"""
import numpy as np
import pytest
import torch

from paper_1301_4195_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L, DT, TW = 6.0, 0.01, 1.5


@pytest.fixture(scope="module")
def cs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_4195_gb300 import build
    build.build()
    from paper_1301_4195_gb300 import api
    return api


def run(cs, N, ncells, prec, nsteps):
    h = cs.Handle(N, L, 1.0, prec)
    f = torch.from_numpy(I.wall_initial(N, L, ncells)).cuda()
    dx = torch.from_numpy(I.wall_grid(ncells)).cuda()
    far = torch.from_numpy(I.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)).cuda()
    h.step(f, dx, far, TW, (0.0, 0.0, 0.0), DT, nsteps=nsteps)
    torch.cuda.synchronize()
    cs.cs_status(h.ptr)
    out = f.cpu().numpy()
    h.close()
    return out


def test_wall16_200_steps_float_follows_double(cs):
    a = run(cs, 16, 128, "fp32", 200)
    b = run(cs, 16, 128, "fp64", 200)
    assert np.isfinite(a).all()
    assert np.abs(a - b).max() / np.abs(b).max() < 1e-5
    # the wall heats the gas: the state has left the initial Maxwellian near the wall
    m0 = I.wall_initial(16, L, 1)[0]
    assert np.abs(b[0] - m0).max() > 1e-3 * np.abs(m0).max()


def test_wall32_20_steps_float_follows_double_on_sampled_cells(cs):
    a = run(cs, 32, 32, "fp32", 20)
    b = run(cs, 32, 32, "fp64", 20)
    for c in (0, 1, 16, 31):
        assert np.abs(a[c] - b[c]).max() / np.abs(b[c]).max() < 1e-5, c

