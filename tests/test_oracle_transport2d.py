"""Pins of the oracle's transport in two space dimensions (no GPU).

x is the wall problem's direction (non-uniform cells, wall at x = 0, far
field at the end), y is periodic with uniform cells; the scheme adds the two
directions' flux differences.
* A state uniform in y has no y-flux: every row equals the 1-D transport.
* ny = 1 is the 1-D problem.
* The y-fluxes telescope: summed over a periodic row they vanish.
* Away from the x-boundaries the y-part is a second-order approximation of
  -v2 df/dy for a smooth periodic profile (errors fall about fourfold when
  dy halves).
"""
import numpy as np
import pytest

from paper_1301_4195_gb300 import inputs

L = 6.0


def far(N):
    return inputs.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)


def test_uniform_in_y_is_the_1d_transport(oracle_mod):
    N, nx, ny = 8, 10, 5
    dx = inputs.wall_grid(nx)
    f1 = inputs.wall_profile(N, L, nx)
    f2 = np.repeat(f1[:, None], ny, axis=1)
    r2 = oracle_mod.transport2d_rhs(f2, N, L, nx, ny, dx, 0.3, 1.5, (0.0, 0.2, 0.0), far(N))
    s1 = oracle_mod.transport_rk2(f1, N, L, dx, 1.5, (0.0, 0.2, 0.0), far(N), 0.01)
    s2 = oracle_mod.transport2d_rk2(f2, N, L, nx, ny, dx, 0.3, 1.5, (0.0, 0.2, 0.0), far(N), 0.01)
    full = np.full((nx + 4, N, N, N), np.nan)
    full[2:-2] = f1
    r1 = oracle_mod.transport_rhs_window(full, N, L, nx, 0, dx, 1.5, (0.0, 0.2, 0.0), far(N))
    for j in range(ny):
        assert np.array_equal(r2[:, j], r1)
        assert np.array_equal(s2[:, j], s1)


def test_single_row_is_the_1d_problem(oracle_mod):
    N, nx = 8, 9
    dx = inputs.wall_grid(nx)
    f1 = inputs.wall_profile(N, L, nx)
    s1 = oracle_mod.transport_rk2(f1, N, L, dx, 1.5, (0, 0, 0), far(N), 0.01)
    s2 = oracle_mod.transport2d_rk2(f1[:, None], N, L, nx, 1, dx, 0.5, 1.5, (0, 0, 0), far(N), 0.01)
    assert np.array_equal(s2[:, 0], s1)


def _y_profile(N, nx, ny, Y):
    y = (np.arange(ny) + 0.5) * Y / ny
    m = far(N)
    return np.stack([np.stack([m * (1.0 + 0.3 * np.sin(2 * np.pi * yy / Y)) for yy in y])] * nx), y


def test_y_fluxes_telescope(oracle_mod):
    N, nx, ny, Y = 8, 6, 7, 2.0
    dx = inputs.wall_grid(nx)
    f, _ = _y_profile(N, nx, ny, Y)
    rng = np.random.default_rng(5)
    f = f * (1 + 0.05 * rng.standard_normal(f.shape))
    r2 = oracle_mod.transport2d_rhs(f, N, L, nx, ny, dx, Y / ny, 1.5, (0, 0, 0), far(N))
    # the x-part of every row, from the 1-D routine
    rx = np.stack([oracle_mod.transport2d_rhs(f[:, j:j + 1], N, L, nx, 1, dx, Y / ny, 1.5, (0, 0, 0), far(N))[:, 0]
                   for j in range(ny)], axis=1)
    ry = r2 - rx
    scale = np.abs(ry).max()
    assert scale > 0
    assert np.abs(ry.sum(axis=1)).max() <= 1e-13 * scale * ny


def test_y_part_is_second_order(oracle_mod):
    N, nx, Y = 8, 12, 4.0
    dx = np.full(nx, 0.25)
    dv = 2 * L / N
    v2 = dv * (np.arange(N) - N // 2)
    errs = []
    for ny in (16, 32, 64):
        f, y = _y_profile(N, nx, ny, Y)
        r2 = oracle_mod.transport2d_rhs(f, N, L, nx, ny, dx, Y / ny, 1.0, (0, 0, 0), far(N))
        rx = np.stack([oracle_mod.transport2d_rhs(f[:, j:j + 1], N, L, nx, 1, dx, Y / ny, 1.0, (0, 0, 0),
                                                  far(N))[:, 0] for j in range(ny)], axis=1)
        ry = (r2 - rx)[nx // 2]  # one interior x-cell: [ny][N][N][N]
        m = far(N)
        # exact -v2 d/dy of m (1 + 0.3 sin(2 pi y / Y)) at the cell centres
        dfdy = m[None] * (0.3 * 2 * np.pi / Y * np.cos(2 * np.pi * y / Y))[:, None, None, None]
        exact = -v2[None, None, :, None] * dfdy
        errs.append(np.abs(ry - exact).mean() / np.abs(exact).mean())
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5, errs


def test_strang_2d_conserves_mass_up_to_boundary_fluxes(oracle_mod):
    """With x-uniform data equal to the far field and the wall in equilibrium
    with it (T_w = 1, V_w = 0), only the y-modulation evolves; periodic y and
    a balanced wall keep the total mass to rounding."""
    N, nx, ny, Y = 8, 6, 6, 3.0
    dx = inputs.wall_grid(nx)
    f, _ = _y_profile(N, nx, ny, Y)
    m0 = (f.sum(axis=(2, 3, 4)) * dx[:, None]).sum()
    g = oracle_mod.strang_step2d(f, N, L, 1.0, nx, ny, dx, Y / ny, 1.0, (0, 0, 0), far(N), 0.01)
    assert np.isfinite(g).all()
    m1 = (g.sum(axis=(2, 3, 4)) * dx[:, None]).sum()
    # the far end exchanges mass with the unmodulated far field: bounded by the
    # modulation's flux through one face over dt
    assert abs(m1 - m0) / m0 < 1e-3
