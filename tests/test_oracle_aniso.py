"""Pins of the oracle's anisotropic-scattering weights (Sec. 2: B = |u|^lambda
b(cos theta); Sec. 2.2 leaves the weights as integrals and computes only
b = 1/4pi; Sec. 4.2 notes the same convolution serves anisotropic b).

b is given by its Legendre moments beta_l = int_{S^2} b(sigma.u^) P_l(sigma.u^)
dsigma, i.e. b(t) = sum_l (2l+1) beta_l P_l(t) / 4pi.  None of these checks
compares the oracle with itself:

* beta = (1) is the isotropic b = 1/4pi: the series route equals the closed
  forms of Sec. 2.2 (lambda = 0, 1) and the isotropic quadrature (other lambda);
* the weights equal a direct numerical quadrature of their defining
  integrals (the sphere integral over sigma in G(u, zeta), then the Fourier
  integral over u), which uses no Legendre or Bessel function;
* odd moments of b drop out of Q (for identical particles only b(t) + b(-t)
  enters the convolution);
* Maxwell molecules: the traceless pressure tensor relaxes at the rate
  (3/4) rho int b sin^2 theta dsigma = (rho/2)(beta_0 - beta_2) (weak form,
  Sec. 2);
* the discrete operator against a direct 5-D quadrature of the collision
  integral with the same b.
"""
import math

import numpy as np
import pytest

from paper_1301_4195_gb300 import inputs as I

L = 6.0


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def b_of(beta, t):
    """b(t) = sum_l (2l+1) beta_l P_l(t) / 4pi (numpy's Legendre series)."""
    c = np.array([(2 * l + 1) * bl for l, bl in enumerate(beta)]) / (4 * math.pi)
    return np.polynomial.legendre.legval(t, c)


@pytest.mark.parametrize("lam", [0.0, 1.0, 0.5, -1.0])
def test_isotropic_moments_reproduce_the_isotropic_weights(oracle_mod, lam):
    N = 8
    rng = np.random.default_rng(11)
    km = rng.integers(0, N, size=(60, 6))
    km[0] = [4, 4, 4, 1, 2, 3]  # zeta = 0
    km[1] = [5, 4, 4, 4, 4, 4]  # xi = 0
    km[2] = [6, 4, 4, 5, 4, 4]  # xi = zeta / 2
    for beta in ([1.0], [1.0, 0.0, 0.0]):
        got = np.array([oracle_mod.ghat_aniso(N, L, lam, beta, r[:3], r[3:]) for r in km])
        ref = np.array([oracle_mod.ghat(N, L, lam, r[:3], r[3:]) for r in km])
        assert np.all(np.abs(got - ref) <= 1e-12 * np.maximum(np.abs(ref), 1e-3))


def direct_ghat(N, lam, beta, k, m, nr=8, nq=16, nmu=48, nang=64):
    """Ghat(xi, zeta) = (2 pi)^{-3/2} int_{|u|<r0} |u|^lam [I(u, zeta) e^{-i (xi - zeta/2).u}
    - beta_0 e^{-i xi.u}] du with I(u, zeta) = int_{S^2} b(sigma.u^) e^{-i |u| zeta.sigma / 2} dsigma,
    both integrals by plain product quadrature (lambda >= 0)."""
    dz = math.pi / L
    zeta = dz * (np.array(k) - N // 2)
    xi = dz * (np.array(m) - N // 2)
    w = xi - zeta / 2
    az = np.linalg.norm(zeta)
    if az == 0:
        return 0.0
    e3 = zeta / az
    e1 = np.cross(e3, [1.0, 0.0, 0.0] if abs(e3[0]) < 0.9 else [0.0, 1.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(e3, e1)
    # radial nodes: nr panels of nq Gauss-Legendre nodes on [0, r0]
    xg, wg = np.polynomial.legendre.leggauss(nq)
    h = L / nr
    r = np.concatenate([p * h + h * (xg + 1) / 2 for p in range(nr)])
    wr = np.concatenate([wg * h / 2 for _ in range(nr)])
    mu, wmu = np.polynomial.legendre.leggauss(nmu)   # cos of the angle between u and zeta
    ta, wta = np.polynomial.legendre.leggauss(nmu)   # cos of the angle between sigma and u
    ph = 2 * math.pi * np.arange(nang) / nang
    # I(r, mu): sigma in the frame of u^, whose first transverse axis lies in the (u^, zeta) plane
    A = r[:, None, None, None] * az / 2
    MU = mu[None, :, None, None]
    TA = ta[None, None, :, None]
    PH = ph[None, None, None, :]
    arg = A * (MU * TA + np.sqrt(1 - MU ** 2) * np.sqrt(1 - TA ** 2) * np.cos(PH))
    Iphi = np.exp(-1j * arg).sum(axis=3) * (2 * math.pi / nang)       # [r, mu, t]
    Irm = (Iphi * (b_of(beta, ta) * wta)[None, None, :]).sum(axis=2)  # [r, mu]
    # the u integral: u = r (sqrt(1-mu^2) (cos psi e1 + sin psi e2) + mu e3)
    s = np.sqrt(1 - mu ** 2)
    dirs = (s[:, None, None] * (np.cos(ph)[None, :, None] * e1 + np.sin(ph)[None, :, None] * e2)
            + mu[:, None, None] * e3)                                  # [mu, psi, 3]
    wdot = dirs @ w
    xdot = dirs @ xi
    R = r[:, None, None]
    integrand = (Irm[:, :, None] * np.exp(-1j * R * wdot[None]) - beta[0] * np.exp(-1j * R * xdot[None]))
    val = (integrand * (wr * r ** (lam + 2))[:, None, None] * wmu[None, :, None]).sum() * (2 * math.pi / nang)
    return (2 * math.pi) ** -1.5 * val


@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_aniso_weights_equal_direct_quadrature_of_their_definition(oracle_mod, lam):
    N = 8
    beta = [1.0, 0.4, 0.3, -0.15]
    pairs = [([5, 4, 4], [6, 4, 4]), ([6, 5, 3], [4, 3, 2]), ([2, 6, 5], [1, 4, 6]), ([7, 7, 7], [7, 6, 5]),
             ([4, 4, 6], [2, 4, 4]), ([3, 5, 4], [4, 4, 4])]
    for k, m in pairs:
        ref = direct_ghat(N, lam, beta, k, m)
        assert abs(ref.imag) < 1e-9 * max(abs(ref.real), 1e-3)  # the weights are real
        got = oracle_mod.ghat_aniso(N, L, lam, beta, k, m)
        assert abs(got - ref.real) < 1e-7 * max(abs(ref.real), 1e-2), (k, m, got, ref)


def test_convolution_equals_brute_force_over_the_pairwise_weights(oracle_mod):
    """N = 6: the oracle's convolution (which evaluates each distinct radial
    integral once) against the plain sum over every (k, m) of the weight
    evaluated pair by pair, written here with numpy."""
    N, lam, beta = 6, 1.0, [1.0, 0.3, 0.25]
    h = N // 2
    f = I.random_mixture_cells(N, L, 2, first_id=45)
    fh = oracle_mod.dft_forward(f, N, L).reshape(2, N, N, N)
    want = np.zeros((2, N, N, N), dtype=complex)
    rng = range(N)
    for k in np.ndindex(N, N, N):
        for m in np.ndindex(N, N, N):
            s = tuple(k[d] - m[d] + h for d in range(3))
            if min(s) < 0 or max(s) > N - 1:
                continue
            g = oracle_mod.ghat_aniso(N, L, lam, beta, k, m)
            want[(slice(None),) + k] += g * fh[(slice(None),) + m] * fh[(slice(None),) + s]
    want *= (math.pi / L) ** 3
    got = oracle_mod.convolve_b(fh, N, L, lam, beta)
    assert _rel(got, want) < 1e-13


def test_odd_moments_of_b_drop_out(oracle_mod):
    N = 8
    f = I.random_mixture_cells(N, L, 2, first_id=41)
    a = oracle_mod.collide_b(f, N, L, 1.0, [1.0, 0.5, 0.3, 0.2])
    b = oracle_mod.collide_b(f, N, L, 1.0, [1.0, 0.0, 0.3, 0.0])
    c = oracle_mod.collide(f, N, L, 1.0)
    assert _rel(a, b) < 1e-13
    assert _rel(b, c) > 1e-3  # the even moment beta_2 does change Q


@pytest.mark.parametrize("beta2", [0.3, -0.2])
def test_maxwell_molecules_pressure_law_with_anisotropic_b(oracle_mod, beta2):
    """lambda = 0: d/dt P'_ij = -(3/4) rho int b sin^2 theta dsigma P'_ij, and
    int b sin^2 theta dsigma = (2/3)(beta_0 - beta_2)."""
    N = 16
    beta = [1.0, 0.0, beta2]
    f = I.mixture(N, L, ((0.5, 1.0, 0, 0, 0.6), (0.5, -1.0, 0.2, 0, 0.6)))[None]
    Q = oracle_mod.collide_b(f, N, L, 0.0, beta)[0]
    v = I.velocity_grid(N, L)
    w = (2 * L / N) ** 3

    def second(g):
        return np.array([[np.sum(v[i] * v[j] * g) * w for j in range(3)] for i in range(3)])

    mom = oracle_mod.moments(f, N, L)[0]
    rho, J = mom[0], mom[1:4]
    P = second(f[0]) - np.outer(J, J) / rho
    Pd = P - np.eye(3) * np.trace(P) / 3
    dM = second(Q)
    dMd = dM - np.eye(3) * np.trace(dM) / 3
    nu = 0.5 * rho * (beta[0] - beta2)
    assert _rel(dMd, -nu * Pd) < 2e-2


def test_aniso_operator_matches_direct_quadrature_of_collision_integral(oracle_mod):
    N, LL = 16, 6.0
    beta = [1.0, 0.0, 0.4]
    mix = ((0.5, 1.0, 0.0, 0.0, 0.6), (0.5, -1.0, 0.2, 0.0, 0.6))
    f = I.mixture(N, LL, mix)[None]
    Qt = oracle_mod.collide_b(f, N, LL, 1.0, beta, conserve=False)[0]
    ax = I.velocity_axis(N, LL)
    idx = np.argsort(-np.abs(Qt).ravel())[:6:2]
    pts = np.array([[ax[i // (N * N)], ax[(i // N) % N], ax[i % N]] for i in idx])
    bf = oracle_mod.q_bruteforce_b(1.0, LL, beta, mix, pts, 6, 12, 12, 24)
    err = np.abs(bf - Qt.ravel()[idx]).max() / np.abs(Qt).max()
    iso = oracle_mod.q_bruteforce(1.0, LL, mix, pts, 6, 12, 12, 24)
    # the discretisation error (the isotropic operator at this N and L is 1.6 %
    # off its integral), far below the effect of b: the anisotropic operator
    # follows its own integral, not the isotropic one (50 % apart here)
    assert err < 3e-2
    assert err < 0.1 * np.abs(bf - iso).max() / np.abs(Qt).max()
