"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle tests.

This module holds no arithmetic of the method itself: it only tabulates
distribution functions on the velocity grid of Sec. 3.1 (v_k = dv (k - N/2),
dv = 2L/N) and draws the random parameters of the workloads.

Workload recipes (synthetic stand-ins for the paper's runs, Sec. 4-5):

* two-stream: 0.5 M(V=(+1.5,0,0), T=0.5) + 0.5 M(V=(-1.5,0,0), T=0.5).
* random mixture (per cell): 2-3 Maxwellians, rho ~ U[0.2, 1],
  V_i ~ U[-1, 1], T ~ U[0.3, 1.5], drawn from
  ``numpy.random.default_rng(13014195 + cell_id)``.
* wall problem: cells of width dx_j = min(dx0 * 1.05**j, 0.5), dx0 = 1/8,
  initial unit Maxwellian everywhere (Sec. 5, sudden heating).
* BKW (Maxwell molecules): the Bobylev-Krook-Wu closed form.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 13014195


def velocity_axis(N: int, L: float) -> np.ndarray:
    return (2.0 * L / N) * (np.arange(N) - N // 2)


def velocity_grid(N: int, L: float):
    a = velocity_axis(N, L)
    return np.meshgrid(a, a, a, indexing="ij")


def maxwellian(N: int, L: float, rho: float, V, T: float) -> np.ndarray:
    """rho (2 pi T)^{-3/2} exp(-|v - V|^2 / (2T)) on the grid, shape [N, N, N]."""
    v1, v2, v3 = velocity_grid(N, L)
    e = (v1 - V[0]) ** 2 + (v2 - V[1]) ** 2 + (v3 - V[2]) ** 2
    return rho * (2.0 * np.pi * T) ** -1.5 * np.exp(-e / (2.0 * T))


def mixture(N: int, L: float, params) -> np.ndarray:
    """Sum of Maxwellians, params rows (rho, V1, V2, V3, T)."""
    out = np.zeros((N, N, N))
    for rho, a, b, c, T in np.asarray(params, dtype=np.float64).reshape(-1, 5):
        out += maxwellian(N, L, rho, (a, b, c), T)
    return out


TWO_STREAM = ((0.5, 1.5, 0.0, 0.0, 0.5), (0.5, -1.5, 0.0, 0.0, 0.5))


def two_stream(N: int, L: float) -> np.ndarray:
    return mixture(N, L, TWO_STREAM)


def random_mixture_params(cell_id: int, nmin: int = 2, nmax: int = 3, seed_base: int = SEED_BASE):
    rng = np.random.default_rng(seed_base + int(cell_id))
    n = int(rng.integers(nmin, nmax + 1))
    rows = []
    for _ in range(n):
        rho = rng.uniform(0.2, 1.0)
        V = rng.uniform(-1.0, 1.0, size=3)
        T = rng.uniform(0.3, 1.5)
        rows.append((rho, V[0], V[1], V[2], T))
    return np.array(rows)


def random_mixture_cells(N: int, L: float, ncells: int, first_id: int = 0, nmin: int = 2,
                         nmax: int = 3, seed_base: int = SEED_BASE) -> np.ndarray:
    """[ncells, N, N, N] float64, cell c drawn from seed seed_base + first_id + c."""
    out = np.empty((ncells, N, N, N))
    for c in range(ncells):
        out[c] = mixture(N, L, random_mixture_params(first_id + c, nmin, nmax, seed_base))
    return out


def random_lambdas(ncells: int, first_id: int = 0, seed_base: int = SEED_BASE) -> np.ndarray:
    """lambda in {0, 1} per cell, half each in expectation."""
    rng = np.random.default_rng(seed_base + 7 + int(first_id))
    return rng.integers(0, 2, size=ncells).astype(np.float64)


def bkw(N: int, L: float, K: float) -> np.ndarray:
    """BKW solution of the Maxwell-molecule equation at shape parameter K
    (K = 1 - exp(-t/6), K >= 3/5): exp(-|v|^2/(2K)) / (2 (2 pi K)^{3/2})
    * ((5K - 3)/K + (1 - K)/K^2 |v|^2)."""
    v1, v2, v3 = velocity_grid(N, L)
    v2s = v1 * v1 + v2 * v2 + v3 * v3
    return (np.exp(-v2s / (2.0 * K)) / (2.0 * (2.0 * np.pi * K) ** 1.5)
            * ((5.0 * K - 3.0) / K + (1.0 - K) / K ** 2 * v2s))


def wall_grid(ncells: int, dx0: float = 0.125, ratio: float = 1.05, dxmax: float = 0.5) -> np.ndarray:
    """Cell widths clustered at the wall x = 0: dx_j = min(dx0 ratio^j, dxmax)."""
    j = np.arange(ncells, dtype=np.float64)
    return np.minimum(dx0 * ratio ** j, dxmax)


def wall_initial(N: int, L: float, ncells: int) -> np.ndarray:
    """Unit Maxwellian (rho = 1, V = 0, T = 1) in every cell, [ncells, N, N, N]."""
    m = maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)
    return np.broadcast_to(m, (ncells, N, N, N)).copy()


def wall_profile(N: int, L: float, ncells: int) -> np.ndarray:
    """A wall-problem state with structure in x, [ncells, N, N, N]: Maxwellians
    whose density, drift and temperature vary smoothly with the cell index,
    so every face of the grid carries a non-trivial flux and slope."""
    out = np.empty((ncells, N, N, N))
    for j in range(ncells):
        s = j / max(ncells - 1, 1)
        out[j] = maxwellian(N, L, 1.0 + 0.3 * np.sin(3.0 * s), (0.4 * np.cos(5.0 * s), 0.1, 0.0), 1.0 + 0.2 * s)
    return out


def wall2d_initial(N: int, L: float, nx: int, ny: int, Y: float) -> np.ndarray:
    """The wall problem in two space dimensions, [nx][ny][N, N, N]: the unit
    Maxwellian with density 1 + 0.2 sin(2 pi y / Y) across the periodic
    direction y (cell centres (j + 1/2) Y / ny), uniform across x."""
    m = maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)
    y = (np.arange(ny) + 0.5) * Y / ny
    rho = 1.0 + 0.2 * np.sin(2.0 * np.pi * y / Y)
    return np.broadcast_to(rho[None, :, None, None, None] * m[None, None], (nx, ny, N, N, N)).copy()
