"""Plain FP64 CPU oracle of the conservative spectral collision operator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  It shares no code with the CUDA library under
``paper_1301_4195_gb300/`` and neither side imports the other.

The arithmetic lives in ``cs_oracle.c`` (plain C, FP64, OpenMP over the
zeta_k outputs as in Sec. 4.1 of the paper); this module compiles it with gcc
and marshals numpy arrays.  Each wrapper names the passage of the paper it
follows.  Array conventions:

* ``f``: float64 ``[ncells, N, N, N]`` (or ``[ncells, N**3]``), velocity index
  ``(k1, k2, k3)`` in C order, ``v_k = dv (k - N/2)``.
* ``fhat`` / ``qhat``: complex128 of the same shape, ``zeta_k = dzeta (k - N/2)``.
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess
import threading

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SRC = _HERE / "cs_oracle.c"
_BUILD = _HERE / "_build"
_SO = _BUILD / "libcs_oracle.so"
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> pathlib.Path:
    """Compile cs_oracle.c into a shared library (gcc -O2, IEEE, OpenMP)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _SO.exists() or _SO.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"libcs_oracle.{os.getpid()}.so"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
               "-fno-fast-math", str(_SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(str(_SO))
            sigs = {
                "or_dv": (ctypes.c_double, [ctypes.c_int, ctypes.c_double]),
                "or_dzeta": (ctypes.c_double, [ctypes.c_double]),
                "or_gauss_legendre": (None, [ctypes.c_int, _dp, _dp]),
                "or_dft_forward": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]),
                "or_dft_inverse": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp,
                                                  ctypes.c_double, _dp, _dp]),
                "or_ghat": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _ip, _ip]),
                "or_ghat_quad": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                   _ip, _ip, ctypes.c_int]),
                "or_ghat_radial_quad": (ctypes.c_double, [ctypes.c_double] * 5 + [ctypes.c_int] * 2),
                "or_ghat_table": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]),
                "or_convolve": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, _dp, _dp, ctypes.c_int]),
                "or_convolve_at": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_int, _dp, ctypes.c_int, _ip, _dp, ctypes.c_int]),
                "or_moments": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]),
                "or_cct": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, _dp]),
                "or_conserve": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp]),
                "or_collide": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, _dp, ctypes.c_double, _dp,
                                              ctypes.c_int, ctypes.c_int]),
                "or_rk2_homogeneous": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                      ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int,
                                                      ctypes.c_double, ctypes.c_int, ctypes.c_int]),
                "or_transport_rk2": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp,
                                                    ctypes.c_double, _dp, _dp, ctypes.c_double]),
                "or_transport2d_rhs": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                      _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                                      _dp]),
                "or_transport2d_rk2": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                      _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                                      ctypes.c_double]),
                "or_strang_step2d": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                    ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                                    _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int]),
                "or_transport_rhs_window": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                           ctypes.c_int, ctypes.c_int, _dp, _dp,
                                                           ctypes.c_double, _dp, _dp, _dp]),
                "or_wall_flux": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp,
                                                ctypes.c_double, _dp, _dp]),
                "or_strang_step": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_int]),
                "or_q_bruteforce": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp,
                                                   ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int]),
                "or_rounding_scale": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_int, _dp, ctypes.c_double, _dp, ctypes.c_int]),
                "or_ghat_aniso": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                    _dp, _ip, _ip]),
                "or_convolve_b": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp,
                                                 ctypes.c_int, _dp, _dp, ctypes.c_int]),
                "or_collide_b": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp,
                                                ctypes.c_int, _dp, ctypes.c_double, _dp, ctypes.c_int, ctypes.c_int]),
                "or_q_bruteforce_b": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp,
                                                     ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int]),
                "or_transport3d_rhs": (ctypes.c_int, [ctypes.c_int, ctypes.c_double] + [ctypes.c_int] * 3 +
                                       [_dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                        _dp]),
                "or_transport3d_rk2": (ctypes.c_int, [ctypes.c_int, ctypes.c_double] + [ctypes.c_int] * 3 +
                                       [_dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                        ctypes.c_double]),
                "or_strang_step3d": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double] +
                                     [ctypes.c_int] * 3 + [_dp, _dp, ctypes.c_double, ctypes.c_double,
                                                           ctypes.c_double, _dp, _dp, ctypes.c_double,
                                                           ctypes.c_double, ctypes.c_int]),
                "or_max_threads": (ctypes.c_int, []),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_ip)


def _cells(f: np.ndarray, N: int) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return f.reshape(-1, N ** 3)


def max_threads() -> int:
    return _load().or_max_threads()


# ---------------------------------------------------------------- grids (Sec. 3.1)
def grid(N: int, L: float):
    """Velocity and Fourier mesh points, Sec. 3.1 ("meshpoints")."""
    lib = _load()
    dv, dz = lib.or_dv(N, L), lib.or_dzeta(L)
    k = np.arange(N) - N // 2
    return dv * k, dz * k, dv, dz


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _load().or_gauss_legendre(n, _d(x), _d(w))
    return x, w


# ---------------------------------------------------------- transforms (Sec. 3.2)
def dft_forward(f: np.ndarray, N: int, L: float) -> np.ndarray:
    """fhat(zeta_k) = (2 pi)^{-3/2} dv^3 sum_j f(v_j) exp(-i zeta_k . v_j)."""
    fc = _cells(f, N)
    out = np.zeros((fc.shape[0], N ** 3, 2))
    _load().or_dft_forward(N, L, fc.shape[0], _d(fc), _d(out))
    return (out[..., 0] + 1j * out[..., 1]).reshape(fc.shape[0], N, N, N)


def dft_inverse(qhat: np.ndarray, N: int, L: float, eps: float = 1.0, imag: bool = False):
    """Qt(v_j) = Re[(2 pi)^{-3/2} dzeta^3 sum_k Qhat(zeta_k) exp(i zeta_k . v_j)] / eps."""
    q = np.ascontiguousarray(qhat, dtype=np.complex128).reshape(-1, N ** 3)
    qi = np.ascontiguousarray(np.stack([q.real, q.imag], axis=-1))
    re = np.zeros((q.shape[0], N ** 3))
    im = np.zeros((q.shape[0], N ** 3))
    _load().or_dft_inverse(N, L, q.shape[0], _d(qi), eps, _d(re), _d(im))
    re = re.reshape(q.shape[0], N, N, N)
    if imag:
        return re, im.reshape(q.shape[0], N, N, N)
    return re


# ------------------------------------------------------------- weights (Sec. 2.2)
def ghat(N: int, L: float, lam: float, k, m) -> float:
    """Ghat(xi_m, zeta_k): closed form (lambda = 0, 1) or radial quadrature."""
    kk = np.ascontiguousarray(k, dtype=np.int32)
    mm = np.ascontiguousarray(m, dtype=np.int32)
    return _load().or_ghat(N, L, lam, _i(kk), _i(mm))


def ghat_quad(N: int, L: float, lam: float, k, m, nodes: int = 24) -> float:
    """Ghat(xi_m, zeta_k) by composite Gauss-Legendre of the radial integral."""
    kk = np.ascontiguousarray(k, dtype=np.int32)
    mm = np.ascontiguousarray(m, dtype=np.int32)
    return _load().or_ghat_quad(N, L, lam, _i(kk), _i(mm), nodes)


def ghat_radial_quad(a: float, b: float, c: float, r0: float, lam: float,
                     npanel: int = 40, nodes: int = 24) -> float:
    """int_0^r0 r^{lam+2} [sinc(a r) sinc(b r) - sinc(c r)] dr (no prefactor)."""
    return _load().or_ghat_radial_quad(a, b, c, r0, lam, npanel, nodes)


def ghat_table(N: int, L: float, lam: float) -> np.ndarray:
    """Full table Ghat[k, m], k, m flattened velocity indices (small N only)."""
    M = N ** 3
    out = np.zeros((M, M))
    _load().or_ghat_table(N, L, lam, _d(out))
    return out


# --------------------------------------------------------- convolution (Sec. 3.2)
def convolve(fhat: np.ndarray, N: int, L: float, lam: float, nthreads: int = 0) -> np.ndarray:
    """Qhat(zeta_k) = sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m) dzeta^3."""
    fh = np.ascontiguousarray(fhat, dtype=np.complex128).reshape(-1, N ** 3)
    fi = np.ascontiguousarray(np.stack([fh.real, fh.imag], axis=-1))
    out = np.zeros_like(fi)
    _load().or_convolve(N, L, lam, fh.shape[0], _d(fi), _d(out), nthreads)
    return (out[..., 0] + 1j * out[..., 1]).reshape(fh.shape[0], N, N, N)


def convolve_at(fhat: np.ndarray, N: int, L: float, lam: float, kflat, nthreads: int = 0) -> np.ndarray:
    """The convolution at the flat output indices kflat only: [ncells, len(kflat)]
    complex, each entry the same sum as convolve() computes there."""
    fh = np.ascontiguousarray(fhat, dtype=np.complex128).reshape(-1, N ** 3)
    fi = np.ascontiguousarray(np.stack([fh.real, fh.imag], axis=-1))
    ks = np.ascontiguousarray(kflat, dtype=np.int32)
    out = np.zeros((fh.shape[0], ks.shape[0], 2))
    _load().or_convolve_at(N, L, lam, fh.shape[0], _d(fi), ks.shape[0], _i(ks), _d(out), nthreads)
    return out[..., 0] + 1j * out[..., 1]


def rounding_scale(f: np.ndarray, N: int, L: float, lam: float, eps: float = 1.0, nthreads: int = 0) -> np.ndarray:
    """Per cell S = (2 pi)^{-3/2} dzeta^3 sum_k Shat_k / eps with Shat the
    convolution of Sec. 3.2 taken over the terms' magnitudes: a bound on
    max_j |Qt(v_j)| and the scale of a float evaluation's rounding error."""
    fc = _cells(f, N)
    out = np.zeros(fc.shape[0])
    _load().or_rounding_scale(N, L, lam, fc.shape[0], _d(fc), eps, _d(out), nthreads)
    return out


# --------------------------------------------- anisotropic scattering (Sec. 2, 2.2)
def _moments(beta) -> np.ndarray:
    b = np.ascontiguousarray(beta, dtype=np.float64).reshape(-1)
    assert 1 <= b.shape[0] <= 16
    return b


def ghat_aniso(N: int, L: float, lam: float, beta, k, m) -> float:
    """Ghat(xi_m, zeta_k) for B = |u|^lam b(cos theta), b given by its Legendre
    moments beta_l = int_{S^2} b(sigma . u^) P_l(sigma . u^) dsigma (Funk-Hecke
    reduction of the sphere integral, radial integrals of products of
    spherical Bessel functions by quadrature)."""
    b = _moments(beta)
    kk = np.ascontiguousarray(k, dtype=np.int32)
    mm = np.ascontiguousarray(m, dtype=np.int32)
    return _load().or_ghat_aniso(N, L, lam, b.shape[0], _d(b), _i(kk), _i(mm))


def convolve_b(fhat: np.ndarray, N: int, L: float, lam: float, beta, nthreads: int = 0) -> np.ndarray:
    """The convolution of Sec. 3.2 with the anisotropic weights."""
    b = _moments(beta)
    fh = np.ascontiguousarray(fhat, dtype=np.complex128).reshape(-1, N ** 3)
    fi = np.ascontiguousarray(np.stack([fh.real, fh.imag], axis=-1))
    out = np.zeros_like(fi)
    _load().or_convolve_b(N, L, lam, b.shape[0], _d(b), fh.shape[0], _d(fi), _d(out), nthreads)
    return (out[..., 0] + 1j * out[..., 1]).reshape(fh.shape[0], N, N, N)


def collide_b(f: np.ndarray, N: int, L: float, lam: float, beta, eps: float = 1.0,
              conserve: bool = True, nthreads: int = 0) -> np.ndarray:
    """P_N Qt(f) / eps with B = |u|^lam b(cos theta) (b by its Legendre moments)."""
    b = _moments(beta)
    fc = _cells(f, N)
    out = np.zeros_like(fc)
    _load().or_collide_b(N, L, lam, b.shape[0], _d(b), fc.shape[0], _d(fc), eps, _d(out), int(bool(conserve)),
                         nthreads)
    return out.reshape(-1, N, N, N)


# ------------------------------------------------------ conservation (Sec. 3.3)
def moments(f: np.ndarray, N: int, L: float) -> np.ndarray:
    """C f: dv^3 sums of (1, v1, v2, v3, |v|^2) f, per cell -> [ncells, 5]."""
    fc = _cells(f, N)
    out = np.zeros((fc.shape[0], 5))
    _load().or_moments(N, L, fc.shape[0], _d(fc), _d(out))
    return out


def cct(N: int, L: float) -> np.ndarray:
    A = np.zeros((5, 5))
    _load().or_cct(N, L, _d(A))
    return A


def conserve(Q: np.ndarray, N: int, L: float) -> np.ndarray:
    """P_N Qt = Qt - C^T (C C^T)^{-1} C Qt (returns a new array)."""
    q = _cells(Q, N).copy()
    _load().or_conserve(N, L, q.shape[0], _d(q))
    return q.reshape(-1, N, N, N)


# --------------------------------------------------------- collision (Sec. 3.2-3.3)
def collide(f: np.ndarray, N: int, L: float, lam: float, eps: float = 1.0,
            conserve: bool = True, nthreads: int = 0) -> np.ndarray:
    """P_N Qt(f) / eps for every cell (forward transform, convolution, inverse, projection)."""
    fc = _cells(f, N)
    out = np.zeros_like(fc)
    _load().or_collide(N, L, lam, fc.shape[0], _d(fc), eps, _d(out), int(bool(conserve)), nthreads)
    return out.reshape(-1, N, N, N)


def rk2_homogeneous(f: np.ndarray, N: int, L: float, lam: float, dt: float, nsteps: int,
                    eps: float = 1.0, conserve: bool = True, nthreads: int = 0) -> np.ndarray:
    """Heun's second-order Runge-Kutta on df/dt = P_N Qt(f) / eps (Sec. 3.1)."""
    fc = _cells(f, N).copy()
    _load().or_rk2_homogeneous(N, L, lam, fc.shape[0], _d(fc), dt, nsteps, eps,
                               int(bool(conserve)), nthreads)
    return fc.reshape(-1, N, N, N)


# ------------------------------------------------------------ transport (Sec. 3.4)
def transport_rk2(f: np.ndarray, N: int, L: float, dx: np.ndarray, Tw: float, Vw,
                  ffar: np.ndarray, dt: float) -> np.ndarray:
    """One Heun step of the finite-volume transport with the wall and far-field boundaries."""
    fc = _cells(f, N).copy()
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    ff = np.ascontiguousarray(ffar, dtype=np.float64).reshape(-1)
    assert fc.shape[0] == dxa.shape[0] >= 2
    _load().or_transport_rk2(N, L, fc.shape[0], _d(fc), _d(dxa), Tw, _d(vw), _d(ff), dt)
    return fc.reshape(-1, N, N, N)


def transport_rhs_window(fw: np.ndarray, N: int, L: float, nc: int, first: int, dx: np.ndarray, Tw: float,
                         Vw, ffar: np.ndarray) -> np.ndarray:
    """Transport right-hand side -(F_{j+1/2} - F_{j-1/2}) / dx_j (Sec. 3.4) of the
    cells first .. first+ncl-1 of an nc-cell grid, from the window fw of
    ncl + 4 cells (grid cells first-2 .. first+ncl+1; those outside the grid
    are not read).  dx holds all nc widths."""
    fwc = _cells(fw, N)
    ncl = fwc.shape[0] - 4
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    ff = np.ascontiguousarray(ffar, dtype=np.float64).reshape(-1)
    assert dxa.shape[0] == nc and ncl >= 1
    rhs = np.empty((ncl, N ** 3))
    rc = _load().or_transport_rhs_window(N, L, nc, first, ncl, _d(fwc), _d(dxa), Tw, _d(vw), _d(ff), _d(rhs))
    if rc != 0:
        raise ValueError("bad shard bounds")
    return rhs.reshape(-1, N, N, N)


def wall_flux(f: np.ndarray, N: int, L: float, dx: np.ndarray, Tw: float, Vw):
    """(outgoing wall flux, sigma_w) for the reconstructed face values of cell 0."""
    fc = _cells(f, N)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    out = np.zeros(2)
    _load().or_wall_flux(N, L, fc.shape[0], _d(fc), _d(dxa), Tw, _d(vw), _d(out))
    return float(out[0]), float(out[1])


def strang_step(f: np.ndarray, N: int, L: float, lam: float, dx: np.ndarray, Tw: float, Vw,
                ffar: np.ndarray, dt: float, eps: float = 1.0, nthreads: int = 0) -> np.ndarray:
    """Strang splitting T(dt/2) C(dt) T(dt/2), Sec. 3.1."""
    fc = _cells(f, N).copy()
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    ff = np.ascontiguousarray(ffar, dtype=np.float64).reshape(-1)
    _load().or_strang_step(N, L, lam, fc.shape[0], _d(fc), _d(dxa), Tw, _d(vw), _d(ff), dt, eps,
                           nthreads)
    return fc.reshape(-1, N, N, N)


# ---------------------------------------------- two space dimensions
def _grid2d(f, N, nx, ny):
    fc = np.ascontiguousarray(f, dtype=np.float64).reshape(nx * ny, N ** 3).copy()
    return fc


def transport2d_rhs(f: np.ndarray, N: int, L: float, nx: int, ny: int, dx: np.ndarray, dy: float, Tw: float,
                    Vw, ffar: np.ndarray) -> np.ndarray:
    """Right-hand side of the 2-D transport, f [nx][ny][N,N,N] (x: the wall
    problem's grid and boundaries, y: periodic, uniform dy)."""
    fc = _grid2d(f, N, nx, ny)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    ff = np.ascontiguousarray(ffar, dtype=np.float64).reshape(-1)
    out = np.empty_like(fc)
    rc = _load().or_transport2d_rhs(N, L, nx, ny, _d(fc), _d(dxa), dy, Tw, _d(vw), _d(ff), _d(out))
    if rc != 0:
        raise ValueError("bad 2-D grid")
    return out.reshape(nx, ny, N, N, N)


def transport2d_rk2(f: np.ndarray, N: int, L: float, nx: int, ny: int, dx: np.ndarray, dy: float, Tw: float,
                    Vw, ffar: np.ndarray, dt: float) -> np.ndarray:
    """One Heun step of the 2-D transport."""
    fc = _grid2d(f, N, nx, ny)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    ff = np.ascontiguousarray(ffar, dtype=np.float64).reshape(-1)
    _load().or_transport2d_rk2(N, L, nx, ny, _d(fc), _d(dxa), dy, Tw, _d(vw), _d(ff), dt)
    return fc.reshape(nx, ny, N, N, N)


def strang_step2d(f: np.ndarray, N: int, L: float, lam: float, nx: int, ny: int, dx: np.ndarray, dy: float,
                  Tw: float, Vw, ffar: np.ndarray, dt: float, eps: float = 1.0, nthreads: int = 0) -> np.ndarray:
    """Strang step T(dt/2) C(dt) T(dt/2) with the 2-D transport."""
    fc = _grid2d(f, N, nx, ny)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    ff = np.ascontiguousarray(ffar, dtype=np.float64).reshape(-1)
    _load().or_strang_step2d(N, L, lam, nx, ny, _d(fc), _d(dxa), dy, Tw, _d(vw), _d(ff), dt, eps, nthreads)
    return fc.reshape(nx, ny, N, N, N)


# ---------------------------------------------- three space dimensions
def transport3d_rhs(f: np.ndarray, N: int, L: float, nx: int, ny: int, nz: int, dx: np.ndarray, dy: float,
                    dz: float, Tw: float, Vw, ffar: np.ndarray) -> np.ndarray:
    """Right-hand side of the 3-D transport, f [nx][ny][nz][N,N,N] (x: the wall
    problem's grid and boundaries; y, z: periodic, uniform dy, dz)."""
    fc = np.ascontiguousarray(f, dtype=np.float64).reshape(nx * ny * nz, N ** 3).copy()
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    ff = np.ascontiguousarray(ffar, dtype=np.float64).reshape(-1)
    out = np.empty_like(fc)
    rc = _load().or_transport3d_rhs(N, L, nx, ny, nz, _d(fc), _d(dxa), dy, dz, Tw, _d(vw), _d(ff), _d(out))
    if rc != 0:
        raise ValueError("bad 3-D grid")
    return out.reshape(nx, ny, nz, N, N, N)


def transport3d_rk2(f: np.ndarray, N: int, L: float, nx: int, ny: int, nz: int, dx: np.ndarray, dy: float,
                    dz: float, Tw: float, Vw, ffar: np.ndarray, dt: float) -> np.ndarray:
    """One Heun step of the 3-D transport."""
    fc = np.ascontiguousarray(f, dtype=np.float64).reshape(nx * ny * nz, N ** 3).copy()
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    ff = np.ascontiguousarray(ffar, dtype=np.float64).reshape(-1)
    if _load().or_transport3d_rk2(N, L, nx, ny, nz, _d(fc), _d(dxa), dy, dz, Tw, _d(vw), _d(ff), dt) != 0:
        raise ValueError("bad 3-D grid")
    return fc.reshape(nx, ny, nz, N, N, N)


def strang_step3d(f: np.ndarray, N: int, L: float, lam: float, nx: int, ny: int, nz: int, dx: np.ndarray,
                  dy: float, dz: float, Tw: float, Vw, ffar: np.ndarray, dt: float, eps: float = 1.0,
                  nthreads: int = 0) -> np.ndarray:
    """Strang step T(dt/2) C(dt) T(dt/2) with the 3-D transport."""
    fc = np.ascontiguousarray(f, dtype=np.float64).reshape(nx * ny * nz, N ** 3).copy()
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    vw = np.ascontiguousarray(Vw, dtype=np.float64)
    ff = np.ascontiguousarray(ffar, dtype=np.float64).reshape(-1)
    if _load().or_strang_step3d(N, L, lam, nx, ny, nz, _d(fc), _d(dxa), dy, dz, Tw, _d(vw), _d(ff), dt, eps,
                                nthreads) != 0:
        raise ValueError("bad 3-D grid")
    return fc.reshape(nx, ny, nz, N, N, N)


# ---------------------------------------------- direct collision integral (Sec. 2)
def q_bruteforce_b(lam: float, r0: float, beta, mix, vpts, npan: int = 6, nr: int = 12,
                   nth: int = 16, nph: int = 32, nthreads: int = 0) -> np.ndarray:
    """q_bruteforce with B = |u|^lam b(cos theta), b(t) = sum_l (2l+1) beta_l P_l(t) / 4 pi."""
    b = _moments(beta)
    mx = np.ascontiguousarray(mix, dtype=np.float64).reshape(-1, 5)
    vp = np.ascontiguousarray(vpts, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(vp.shape[0])
    _load().or_q_bruteforce_b(lam, r0, b.shape[0], _d(b), mx.shape[0], _d(mx), vp.shape[0], _d(vp), npan, nr,
                              nth, nph, _d(out), nthreads)
    return out


def q_bruteforce(lam: float, r0: float, mix, vpts, npan: int = 6, nr: int = 12,
                 nth: int = 16, nph: int = 32, nthreads: int = 0) -> np.ndarray:
    """Quadrature of eq. (Q_general) with B = |u|^lam / 4 pi cut at |u| <= r0, for f a
    Maxwellian mixture mix[i] = (rho, V1, V2, V3, T), at the points vpts[n, 3]."""
    mx = np.ascontiguousarray(mix, dtype=np.float64).reshape(-1, 5)
    vp = np.ascontiguousarray(vpts, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(vp.shape[0])
    _load().or_q_bruteforce(lam, r0, mx.shape[0], _d(mx), vp.shape[0], _d(vp), npan, nr, nth,
                            nph, _d(out), nthreads)
    return out
