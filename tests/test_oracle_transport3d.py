"""Pins of the oracle's transport in three space dimensions (no GPU).

x is the wall problem's direction (non-uniform cells, wall at x = 0, far
field at the end), y and z are periodic with uniform cells; the scheme adds
the three directions' flux differences (Sec. 3.4: the ideas carry over to
higher dimensions).
* nz = 1 is the 2-D problem, bit for bit; a state uniform in z gives every
  z-slab the 2-D right-hand side bit for bit; uniform in y and z is 1-D.
* The z-fluxes telescope: summed over a periodic line they vanish.
* z enters with v3 exactly as y enters with v2: exchanging the roles of y
  and z together with the velocity axes 2 and 3 maps one problem onto the
  other.
* The z-part is a second-order approximation of -v3 df/dz for a smooth
  periodic profile.
"""
import numpy as np
import pytest

from paper_1301_4195_gb300 import inputs

L = 6.0


def far(N):
    return inputs.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)


def test_single_z_layer_is_the_2d_problem(oracle_mod):
    N, nx, ny = 8, 6, 5
    dx = inputs.wall_grid(nx)
    rng = np.random.default_rng(1)
    f2 = inputs.wall2d_initial(N, L, nx, ny, 2.0) * (1 + 0.1 * rng.random((nx, ny, 1, 1, 1)))
    Vw = (0.0, 0.2, 0.1)
    r2 = oracle_mod.transport2d_rhs(f2, N, L, nx, ny, dx, 0.4, 1.5, Vw, far(N))
    r3 = oracle_mod.transport3d_rhs(f2[:, :, None], N, L, nx, ny, 1, dx, 0.4, 0.7, 1.5, Vw, far(N))
    assert np.array_equal(r3[:, :, 0], r2)
    s2 = oracle_mod.transport2d_rk2(f2, N, L, nx, ny, dx, 0.4, 1.5, Vw, far(N), 0.01)
    s3 = oracle_mod.transport3d_rk2(f2[:, :, None], N, L, nx, ny, 1, dx, 0.4, 0.7, 1.5, Vw, far(N), 0.01)
    assert np.array_equal(s3[:, :, 0], s2)


def test_uniform_in_z_gives_every_slab_the_2d_rhs(oracle_mod):
    N, nx, ny, nz = 8, 5, 4, 3
    dx = inputs.wall_grid(nx)
    rng = np.random.default_rng(2)
    f2 = inputs.wall2d_initial(N, L, nx, ny, 2.0) * (1 + 0.1 * rng.random((nx, ny, 1, 1, 1)))
    f3 = np.repeat(f2[:, :, None], nz, axis=2)
    r2 = oracle_mod.transport2d_rhs(f2, N, L, nx, ny, dx, 0.4, 1.5, (0, 0, 0), far(N))
    r3 = oracle_mod.transport3d_rhs(f3, N, L, nx, ny, nz, dx, 0.4, 0.3, 1.5, (0, 0, 0), far(N))
    for l in range(nz):
        assert np.array_equal(r3[:, :, l], r2)


def test_uniform_in_y_and_z_is_the_1d_transport(oracle_mod):
    N, nx, ny, nz = 8, 7, 3, 2
    dx = inputs.wall_grid(nx)
    f1 = inputs.wall_profile(N, L, nx)
    f3 = np.broadcast_to(f1[:, None, None], (nx, ny, nz, N, N, N)).copy()
    s1 = oracle_mod.transport_rk2(f1, N, L, dx, 1.5, (0.0, 0.2, 0.0), far(N), 0.01)
    s3 = oracle_mod.transport3d_rk2(f3, N, L, nx, ny, nz, dx, 0.3, 0.5, 1.5, (0.0, 0.2, 0.0), far(N), 0.01)
    for j in range(ny):
        for l in range(nz):
            assert np.array_equal(s3[:, j, l], s1)


def _z_profile(N, nx, ny, nz, Z):
    z = (np.arange(nz) + 0.5) * Z / nz
    m = far(N)
    prof = np.stack([m * (1.0 + 0.3 * np.sin(2 * np.pi * zz / Z)) for zz in z])  # [nz, N, N, N]
    return np.broadcast_to(prof[None, None], (nx, ny, nz, N, N, N)).copy(), z


def test_z_fluxes_telescope(oracle_mod):
    N, nx, ny, nz, Z = 8, 4, 3, 7, 2.0
    dx = inputs.wall_grid(nx)
    rng = np.random.default_rng(3)
    f = inputs.wall2d_initial(N, L, nx, ny, 2.0)[:, :, None] * (1 + 0.2 * rng.random((nx, ny, nz, 1, 1, 1)))
    r3 = oracle_mod.transport3d_rhs(f, N, L, nx, ny, nz, dx, 0.4, Z / nz, 1.5, (0, 0, 0), far(N))
    zpart = np.stack([r3[:, :, l] - oracle_mod.transport2d_rhs(np.ascontiguousarray(f[:, :, l]), N, L, nx, ny, dx,
                                                                0.4, 1.5, (0, 0, 0), far(N))
                      for l in range(nz)], axis=2)
    assert np.abs(zpart).max() > 1e-3
    assert np.abs(zpart.sum(axis=2)).max() < 1e-13 * np.abs(zpart).max() * nz


def test_z_enters_as_y_with_v3_for_v2(oracle_mod):
    """f depending on (x, z) only, ny = 1: its right-hand side is the 2-D one of
    the problem with z renamed y and the velocity axes 2, 3 exchanged."""
    N, nx, nz = 8, 5, 6
    dx = inputs.wall_grid(nx)
    rng = np.random.default_rng(4)
    g = inputs.wall2d_initial(N, L, nx, nz, 1.5) * (1 + 0.2 * rng.random((nx, nz, N, N, N)))  # [nx][nz][v]
    f3 = np.ascontiguousarray(np.swapaxes(g, 3, 4)[:, None])  # [nx][1][nz][v1][v3<->v2]
    r3 = oracle_mod.transport3d_rhs(f3, N, L, nx, 1, nz, dx, 0.9, 0.25, 1.5, (0, 0, 0), far(N))
    r2 = oracle_mod.transport2d_rhs(g, N, L, nx, nz, dx, 0.25, 1.5, (0, 0, 0), far(N))
    back = np.swapaxes(r3[:, 0], 3, 4)
    assert np.abs(back - r2).max() < 1e-14 * np.abs(r2).max()


def test_z_part_is_second_order(oracle_mod):
    N, nx, ny, Z = 8, 3, 1, 2.0
    dx = inputs.wall_grid(nx)
    v = inputs.velocity_grid(N, L)
    errs = []
    for nz in (16, 32, 64):
        f, z = _z_profile(N, nx, ny, nz, Z)
        r3 = oracle_mod.transport3d_rhs(f, N, L, nx, ny, nz, dx, 1.0, Z / nz, 1.5, (0, 0, 0), far(N))
        r2 = np.stack([oracle_mod.transport2d_rhs(np.ascontiguousarray(f[:, :, l]), N, L, nx, ny, dx, 1.0, 1.5,
                                                  (0, 0, 0), far(N)) for l in range(nz)], axis=2)
        zpart = r3 - r2
        exact = -v[2][None] * far(N)[None] * (0.3 * 2 * np.pi / Z * np.cos(2 * np.pi * z / Z))[:, None, None, None]
        # mean error: the limiter clips the slope at the profile's extrema, so
        # the maximum error is first order there (as in 2-D)
        errs.append(np.abs(zpart[1, 0] - exact).mean() / np.abs(exact).mean())
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5, errs
