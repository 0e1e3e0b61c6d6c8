"""The convolution with weight tiles rebuilt from the radius tables (the
store-versus-recompute choice of the weights) against the oracle.

Ghat(xi_m, zeta_k) = A(|k'|^2, |2m'-k'|^2) - B(|m'|^2) (Sec. 2.2, eq.
GHat_calc with a = |zeta|/2, b = |xi - zeta/2|, c = |xi|): the tables hold A
and B in float, the kernel forms 2A - B(|m'|^2) - B(|k'-m'|^2) per entry.
The float tolerance of the convolution (1e-5 of the largest value) holds for
closed-form and quadrature lambda; a handle built with CS_WEIGHTS_RADIUS has
no table of every pair and runs the whole operator (conservation to 1e-12);
the autotuner times both weight modes; N = 64 runs without its 58 GB table.
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


def cplx(a):
    return a[..., 0] + 1j * a[..., 1]


def rinterleave(z):
    return np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1))


def rel(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def drift(Q, N):
    v = I.velocity_grid(N, L)
    rows = np.stack([np.ones_like(v[0]), v[0], v[1], v[2], v[0] ** 2 + v[1] ** 2 + v[2] ** 2]).reshape(5, -1)
    q = Q.reshape(Q.shape[0], -1)
    return float((np.abs(q @ rows.T) / (np.abs(q) @ np.abs(rows).T)).max())


@pytest.mark.parametrize("N,ncells,lam", [(8, 33, 1.0), (16, 3, 0.0), (16, 2, -1.0), (24, 2, 1.0), (32, 1, 1.0)])
def test_radius_convolution_matches_oracle(cs, orc, N, ncells, lam):
    f = I.random_mixture_cells(N, L, ncells, first_id=1700)
    fh = orc.dft_forward(f, N, L)
    h = cs.Handle(N, L, lam, "fp32")
    cs.cs_tune(h.ptr, cs.CS_TUNE_WEIGHTS, 2)
    assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_WEIGHTS) == 2
    got = cplx(host(h.convolve(dev(rinterleave(fh)))))
    ref = orc.convolve(fh, N, L, lam)
    for c in range(ncells):
        assert rel(got[c], ref[c]) < 1e-5, c
    # the stored tiles give the same sums up to the float rounding of the weights
    cs.cs_tune(h.ptr, cs.CS_TUNE_WEIGHTS, 1)
    stored = cplx(host(h.convolve(dev(rinterleave(fh)))))
    assert rel(got, stored) < 2e-6
    cs.cs_status(h.ptr)
    h.close()


def test_radius_tiles_with_the_tile_split_at_n32(cs, orc):
    """At N = 32 a handle may split each pencil's tiles into 2 or 4 ranges,
    also when it rebuilds the weight tiles from the radius tables: the
    ranges' sums agree with the stored tiles' to the weights' float rounding,
    with the whole-pencil sums to the sums' rounding, and with the oracle.
    40 cells: two 32-cell groups, the two-group launch."""
    N, nc = 32, 40
    f = I.random_mixture_cells(N, L, nc, first_id=1750)
    fh = orc.dft_forward(f, N, L)
    fd = dev(rinterleave(fh))
    ref = orc.convolve(fh[:2], N, L, 1.0)
    h = cs.Handle(N, L, 1.0, "fp32")
    cs.cs_tune(h.ptr, cs.CS_TUNE_WEIGHTS, 2)
    whole = cplx(host(h.convolve(fd)))
    for split in (2, 4):
        cs.cs_tune(h.ptr, cs.CS_TUNE_SPLIT, split)
        cs.cs_tune(h.ptr, cs.CS_TUNE_WEIGHTS, 2)
        got = cplx(host(h.convolve(fd)))
        cs.cs_tune(h.ptr, cs.CS_TUNE_WEIGHTS, 1)
        stored = cplx(host(h.convolve(fd)))
        assert rel(got, stored) < 2e-6, split
        assert rel(got, whole) < 1e-6, split
        for c in range(2):
            assert rel(got[c], ref[c]) < 1e-5, (split, c)
    cs.cs_status(h.ptr)
    h.close()


def test_radius_only_handle_runs_the_operator(cs, orc):
    N = 16
    f = I.random_mixture_cells(N, L, 5, first_id=1800)
    h = cs.Handle(N, L, 1.0, "fp32-radius")
    assert cs.cs_handle_info(h.ptr)[4] < 1e6  # no table of every pair
    with pytest.raises(cs.CSError) as e:
        cs.cs_tune(h.ptr, cs.CS_TUNE_WEIGHTS, 1)
    assert e.value.code == cs.CS_ENOTSUP
    got = host(h.collide(dev(f)))
    ref = orc.collide(f, N, L, 1.0)
    for c in range(f.shape[0]):
        assert rel(got[c], ref[c]) < 1e-5, c
    assert drift(got, N) < 1e-12
    # a Strang step replays as a graph like the stored form
    dx = I.wall_grid(8)
    fw = dev(I.wall_profile(N, L, 8))
    far = dev(I.maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0))
    h.step(fw, dev(dx), far, 1.5, (0.0, 0.0, 0.0), 0.01, nsteps=2)
    assert np.isfinite(host(fw)).all()
    cs.cs_status(h.ptr)
    h.close()


def test_autotune_times_both_weight_modes(cs):
    N, nc = 16, 64
    h = cs.Handle(N, L, 1.0, "fp32")
    ms = cs.cs_autotune(h.ptr, nc)
    assert ms > 0
    assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_WEIGHTS) in (1, 2)
    f = dev(I.random_mixture_cells(N, L, nc, first_id=1900))
    q = host(h.collide(f))
    assert np.isfinite(q).all() and drift(q, N) < 1e-12
    h.close()


def test_n64_without_the_table(cs, orc):
    N = 64
    f = I.random_mixture_cells(N, L, 2, first_id=2000)
    fh = orc.dft_forward(f, N, L)
    h = cs.Handle(N, L, 1.0, "fp32-radius")
    got = cplx(host(h.convolve(dev(rinterleave(fh))))).reshape(2, -1)
    rng = np.random.default_rng(64)
    ks = np.unique(np.concatenate([[0, N ** 3 - 1, (32 * N + 32) * N + 32], rng.integers(0, N ** 3, 30)])).astype(np.int32)
    ref = orc.convolve_at(fh, N, L, 1.0, ks)
    for c in range(2):
        assert np.abs(got[c, ks] - ref[c]).max() / np.abs(ref[c]).max() < 1e-5, c
    cs.cs_status(h.ptr)
    h.close()
