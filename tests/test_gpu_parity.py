"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative to the largest reference magnitude of the compared array):
  FP64 path: 1e-12 (operator), 1e-13 (transforms, projection, transport).
  FP32 path: 1e-5 on Q (the stated target), 2e-6 on the transforms.
Inputs are seeded synthetic distributions from paper_1301_4195_gb300.inputs.
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


_handles = {}


def handle(cs, N, lam, prec, LL=L):
    key = (N, lam, prec, LL)
    if key not in _handles:
        _handles[key] = cs.Handle(N, LL, lam, prec)
    return _handles[key]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(got, ref):
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / np.abs(np.asarray(ref)).max())


def cplx(a):  # [..., 2] -> complex
    return a[..., 0] + 1j * a[..., 1]


def rinterleave(z):
    return np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1))


# ------------------------------------------------------------------ a0: weights
@pytest.mark.parametrize("N", [4, 8, 16, 32])
@pytest.mark.parametrize("lam", [0.0, 1.0, 0.5, -1.0, -2.5])
def test_weights_match_oracle(cs, orc, N, lam):
    if lam not in (0.0, 1.0) and N == 32:
        pytest.skip("general-lambda quadrature is checked at N <= 16")
    h = handle(cs, N, lam, "fp64")
    rng = np.random.default_rng(N)
    km = rng.integers(0, N, size=(300, 6))
    hh = N // 2
    km = np.vstack([km, [[hh + 2, hh, hh, hh + 1, hh, hh], [hh + 1, hh + 1, hh - 1, hh, hh, hh],
                         [hh + 1, hh, hh, hh + 1, hh, hh], [hh, hh, hh, 1, 2, 3]]])
    km = np.clip(km, 0, N - 1)
    got = np.array(h.sample_weights(km.tolist()))
    ref = np.array([orc.ghat(N, L, lam, r[:3], r[3:]) for r in km])
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3)
    # closed forms: rounding level; general lambda: two implementations of the same
    # composite Gauss-Legendre sum over ~50 panels
    assert err.max() < (1e-12 if lam in (0.0, 1.0) else 1e-11)


# ------------------------------------------------------------------ a1: forward transform
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("N,ncells", [(4, 1), (8, 33), (12, 5), (16, 2), (24, 3), (32, 1)])
def test_transform_matches_oracle(cs, orc, prec, tol, N, ncells):
    f = I.random_mixture_cells(N, L, ncells)
    h = handle(cs, N, 1.0, prec)
    got = cplx(host(h.transform(dev(f))))
    ref = orc.dft_forward(f, N, L)
    assert rel(got, ref) < tol


# ------------------------------------------------------------------ a2: convolution
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("N,ncells,lam", [(4, 2, 1.0), (8, 33, 1.0), (8, 3, 0.0), (12, 4, 1.0), (16, 2, 0.0)])
def test_convolution_matches_oracle(cs, orc, prec, tol, N, ncells, lam):
    f = I.random_mixture_cells(N, L, ncells, first_id=100)
    fh = orc.dft_forward(f, N, L)
    h = handle(cs, N, lam, prec)
    got = cplx(host(h.convolve(dev(rinterleave(fh)))))
    ref = orc.convolve(fh, N, L, lam)
    for c in range(ncells):
        assert rel(got[c], ref[c]) < tol, c


# ------------------------------------------------------------------ a3: inverse transform
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("N,ncells", [(8, 3), (12, 33), (24, 3), (32, 1)])
def test_inverse_matches_oracle(cs, orc, prec, tol, N, ncells):
    f = I.random_mixture_cells(N, L, ncells, first_id=200)
    qh = orc.convolve(orc.dft_forward(f, N, L), N, L, 1.0) if N <= 12 else orc.dft_forward(f, N, L)
    h = handle(cs, N, 1.0, prec)
    got = host(h.inverse(dev(rinterleave(qh)), eps=0.7))
    ref = orc.dft_inverse(qh, N, L, eps=0.7)
    assert rel(got, ref) < tol


# ------------------------------------------------------------------ a4: projection
@pytest.mark.parametrize("N,ncells", [(4, 3), (8, 40), (32, 2)])
def test_projection_matches_oracle(cs, orc, N, ncells):
    rng = np.random.default_rng(N)
    q = rng.standard_normal((ncells, N, N, N))
    h = handle(cs, N, 1.0, "fp64")
    qd = dev(q)
    mom = host(h.conserve(qd, want_moments=True))
    got = host(qd)
    assert rel(got, orc.conserve(q, N, L)) < 1e-13
    assert rel(mom, orc.moments(q, N, L)) < 1e-13


def test_moments_match_oracle(cs, orc):
    N = 16
    f = I.random_mixture_cells(N, L, 7)
    h = handle(cs, N, 1.0, "fp64")
    assert rel(host(h.moments(dev(f))), orc.moments(f, N, L)) < 1e-13


# ------------------------------------------------------------------ a1-a4: the operator
def drift(orc, Q, N):
    """max over cells and rows of |C Q| / sum |C| |Q| (rounding-relative moment drift)."""
    v = I.velocity_grid(N, L)
    w = (2 * L / N) ** 3
    rows = np.stack([np.ones_like(v[0]), v[0], v[1], v[2], v[0] ** 2 + v[1] ** 2 + v[2] ** 2]).reshape(5, -1) * w
    q = Q.reshape(Q.shape[0], -1)
    return float((np.abs(q @ rows.T) / (np.abs(q) @ np.abs(rows).T)).max())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("N,ncells,lam,kind", [(8, 1, 1.0, "two_stream"), (8, 1, 0.0, "two_stream"),
                                               (12, 37, 1.0, "mix"), (16, 5, 0.0, "mix"), (16, 5, 1.0, "mix"),
                                               (4, 3, 1.0, "mix"), (8, 3, -1.0, "mix"), (16, 2, -2.5, "mix"),
                                               (24, 2, 1.0, "mix")])
def test_collide_matches_oracle(cs, orc, prec, tol, N, ncells, lam, kind):
    f = I.two_stream(N, L)[None] if kind == "two_stream" else I.random_mixture_cells(N, L, ncells, first_id=300)
    h = handle(cs, N, lam, prec)
    got = host(h.collide(dev(f)))
    ref = orc.collide(f, N, L, lam)
    for c in range(f.shape[0]):
        assert rel(got[c], ref[c]) < tol, c
    assert drift(orc, got, N) < 1e-12
    raw = host(h.collide(dev(f), conserve=False))
    refr = orc.collide(f, N, L, lam, conserve=False)
    assert rel(raw, refr) < tol


def test_collide_host_buffers(cs, orc):
    """The public call with host (pinned) tensors copies in and out around the C-ABI call."""
    N = 8
    f = torch.from_numpy(I.random_mixture_cells(N, L, 3, first_id=400)).pin_memory()
    h = handle(cs, N, 1.0, "fp64")
    got = h.collide(f).numpy()
    assert rel(got, orc.collide(f.numpy(), N, L, 1.0)) < 1e-12


def test_empty_and_error_cases(cs):
    N = 8
    h = handle(cs, N, 1.0, "fp64")
    empty = torch.empty((0, N, N, N), dtype=torch.float64, device="cuda")
    cs.cs_collide(h.ptr, empty, 0, 1.0, empty, 1)
    f = dev(I.random_mixture_cells(N, L, 2))
    with pytest.raises(cs.CSError) as e:
        cs.cs_collide(h.ptr, f, 2, 1.0, f, 1)  # f and Q overlap
    assert e.value.code == cs.CS_EINVAL
    with pytest.raises(cs.CSError) as e:
        cs.cs_collide(h.ptr, f, 2, 0.0, torch.empty_like(f), 1)  # eps must be > 0
    assert e.value.code == cs.CS_EINVAL
    rc = cs.lib().cs_collide(h.ptr, f.data_ptr() + 4, 1, 1.0, torch.empty_like(f).data_ptr(), 1, None)
    assert rc == cs.CS_EINVAL  # misaligned: rejected on the host before any launch
    hostbuf = torch.zeros((1, N, N, N), dtype=torch.float64)
    rc = cs.lib().cs_collide(h.ptr, hostbuf.data_ptr(), 1, 1.0, torch.empty_like(f).data_ptr(), 1, None)
    assert rc == cs.CS_EINVAL  # pageable host memory is not device memory


# ------------------------------------------------------------------ a5: Heun relaxation
def test_relax_two_stream_100_steps(cs, orc):
    """The N = 8, L = 6, lambda = 1 two-stream relaxation: 100 Heun steps of dt = 0.01."""
    N = 8
    f = I.two_stream(N, L)[None]
    h = handle(cs, N, 1.0, "fp64")
    fd = dev(f)
    h.relax(fd, 0.01, 100)
    got = host(fd)
    ref = orc.rk2_homogeneous(f, N, L, 1.0, 0.01, 100)
    assert rel(got, ref) < 1e-12
    m0, m1 = orc.moments(f, N, L), orc.moments(got, N, L)
    assert np.abs(m1 - m0).max() / np.abs(m0).max() < 1e-13


# ------------------------------------------------------------------ a6: transport and Strang
def _wall(N, nc):
    dx = I.wall_grid(nc)
    f = I.wall_initial(N, L, nc)
    x = np.cumsum(dx) - dx / 2
    f = f * (1 + 0.3 * np.exp(-x / 0.5))[:, None, None, None]  # non-trivial profile near the wall
    far = I.maxwellian(N, L, 1.0, (0, 0, 0), 1.0)
    return dx, f, far


@pytest.mark.parametrize("N,nc", [(4, 3), (8, 24)])
def test_transport_matches_oracle(cs, orc, N, nc):
    dx, f, far = _wall(N, nc)
    h = handle(cs, N, 1.0, "fp64")
    fd = dev(f)
    ref = f
    for _ in range(3):
        h.transport(fd, dev(dx), dev(far), 1.5, (0.0, 0.1, 0.0), 0.005)
        ref = orc.transport_rk2(ref, N, L, dx, 1.5, (0.0, 0.1, 0.0), far, 0.005)
    assert rel(host(fd), ref) < 1e-13


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-7)])
def test_strang_step_matches_oracle(cs, orc, prec, tol):
    N, nc = 8, 6
    dx, f, far = _wall(N, nc)
    h = handle(cs, N, 1.0, prec)
    fd = dev(f)
    h.step(fd, dev(dx), dev(far), 1.5, (0, 0, 0), 0.01, nsteps=2)
    ref = orc.strang_step(orc.strang_step(f, N, L, 1.0, dx, 1.5, (0, 0, 0), far, 0.01),
                          N, L, 1.0, dx, 1.5, (0, 0, 0), far, 0.01)
    assert rel(host(fd), ref) < tol


# ------------------------------------------------------------------ full-size sampled checks
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_n32_256_cells_sampled(cs, orc, prec, tol):
    """N = 32, 256 cells (the large-grid launch configuration): cells 0, 1, 64, 255
    against the oracle; conservation of every cell."""
    N, nc = 32, 256
    f = I.random_mixture_cells(N, L, nc, first_id=1000)
    h = handle(cs, N, 1.0, prec)
    got = host(h.collide(dev(f)))
    idx = [0, 1, 64, 255]
    ref = orc.collide(f[idx], N, L, 1.0)
    for i, c in enumerate(idx):
        assert rel(got[c], ref[i]) < tol, c
    assert drift(orc, got, N) < 1e-12


# ------------------------------------------------------------------ replay and status
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replay_matches_direct_launches(cs, prec):
    """cs_step replays a captured CUDA graph; with stage timing on it launches the
    kernels directly.  Both must give bit-identical states (same kernels, same order)."""
    N, nc = 16, 40
    dx, f, far = _wall(N, nc)
    h = handle(cs, N, 1.0, prec)
    fa, fb = dev(f), dev(f)
    dxd, fard = dev(dx), dev(far)
    cs.cs_launch_count(reset=True)
    h.step(fa, dxd, fard, 1.5, (0, 0, 0), 0.01, nsteps=3)
    replayed = cs.cs_launch_count(reset=True)
    cs.cs_profile(h.ptr, True)
    h.step(fb, dxd, fard, 1.5, (0, 0, 0), 0.01, nsteps=3)
    direct = cs.cs_launch_count(reset=True)
    cs.cs_profile(h.ptr, False)
    cs.cs_profile_read(h.ptr, reset=True)
    assert np.array_equal(host(fa), host(fb))
    # a replay counts the graph's kernel nodes: the same kernels as the direct launches
    assert replayed == direct and direct % 3 == 0
    if prec == "fp32":
        # per step: transport tables 1, four transport stages x 1, two collision
        # evaluations x (forward, convolution, inverse + projection), the second
        # forward transform inside the first inverse launch
        assert direct == 3 * 10
    ga, gb = dev(f), dev(f)
    h.relax(ga, 0.01, 4)
    cs.cs_profile(h.ptr, True)
    h.relax(gb, 0.01, 4)
    cs.cs_profile(h.ptr, False)
    cs.cs_profile_read(h.ptr, reset=True)
    assert np.array_equal(host(ga), host(gb))
    cs.cs_status(h.ptr)  # no bounded device wait expired


def test_collide_batched_matches_individual_calls(cs):
    """Uneven N and lambda in one replayed graph: every entry equals cs_collide
    bit for bit.  The float strip entries (N = 8, 16, 24, 32; group counts odd
    and even) share one persistent convolution launch; the N = 12, the double
    and the four-way split N = 16 entries run whole on their own branches."""
    specs = [(16, 0.0, 40, "fp32"), (16, 1.0, 24, "fp32"), (24, 0.0, 8, "fp32"), (24, 1.0, 33, "fp32"),
             (8, 1.0, 1, "fp32"), (32, 1.0, 3, "fp32"), (12, 1.0, 5, "fp32"), (8, 0.0, 7, "fp64")]
    hs = [cs.Handle(N, L, lam, prec) for N, lam, _, prec in specs]
    cs.cs_tune(hs[1].ptr, cs.CS_TUNE_SPLIT, 4)  # split four ways: runs outside the shared launch
    fs = [dev(I.random_mixture_cells(N, L, n, first_id=600 + 50 * i)) for i, (N, _, n, _) in enumerate(specs)]
    qs = [torch.empty_like(f) for f in fs]
    refs, alone = [], 0
    for h, f, (N, lam, n, _) in zip(hs, fs, specs):
        q = torch.empty_like(f)
        cs.cs_launch_count(reset=True)
        cs.cs_collide(h.ptr, f, n, 1.0, q, 1)
        alone += cs.cs_launch_count(reset=True)
        refs.append(host(q))
    entries = [(h.ptr, f, q, n) for h, f, q, (_, _, n, _) in zip(hs, fs, qs, specs)]
    for _ in range(2):  # capture, then replay
        for q in qs:
            q.fill_(float("nan"))
        cs.cs_launch_count(reset=True)
        cs.cs_collide_batched(entries)
        # five strip convolutions became one launch; alone, the entries of a
        # few cells at N = 24 and 32 took the few-cell kernel (two launches:
        # the transpose of f-hat and the convolution)
        few = sum(1 for N, _, n, prec in specs if prec == "fp32" and n <= {24: 9, 32: 6}.get(N, 0))
        assert few == 2
        assert cs.cs_launch_count(reset=True) == alone - 4 - few
        for q, r in zip(qs, refs):
            assert np.array_equal(host(q), r)
    # a launch choice changed after the capture holds at the next call: entry 0
    # rebuilds its weights from the radius tables and leaves the shared launch
    cs.cs_tune(hs[0].ptr, cs.CS_TUNE_WEIGHTS, 2)
    q0 = torch.empty_like(fs[0])
    cs.cs_collide(hs[0].ptr, fs[0], specs[0][2], 1.0, q0, 1)
    cs.cs_launch_count(reset=True)
    cs.cs_collide_batched(entries)
    assert cs.cs_launch_count(reset=True) == alone - 3 - few
    assert np.array_equal(host(qs[0]), host(q0))
    for q, r in zip(qs[1:], refs[1:]):
        assert np.array_equal(host(q), r)
    cs.cs_status(hs[0].ptr)  # no bounded device wait expired
    with pytest.raises(cs.CSError):
        cs.cs_collide_batched([(hs[0].ptr, fs[0], qs[0], 40), (hs[0].ptr, fs[0], qs[1], 24)])  # same handle twice
    for h in hs:
        h.close()


def test_relax_batched_matches_individual_calls(cs):
    """Heun steps of uneven entries in one replayed graph per step: each entry
    equals cs_relax on it bit for bit, and each of a step's two evaluations
    runs the four float strip entries' convolutions as one launch."""
    specs = [(16, 0.0, 40, "fp32"), (24, 1.0, 9, "fp32"), (8, 1.0, 3, "fp32"), (32, 0.0, 2, "fp32"),
             (12, 1.0, 5, "fp32"), (8, 0.0, 4, "fp64")]
    hs = [cs.Handle(N, L, lam, prec) for N, lam, _, prec in specs]
    f0 = [I.random_mixture_cells(N, L, n, first_id=700 + 40 * i) for i, (N, _, n, _) in enumerate(specs)]
    refs, alone = [], 0
    for h, f, (N, lam, n, _) in zip(hs, f0, specs):
        fd = dev(f)
        cs.cs_launch_count(reset=True)
        cs.cs_relax(h.ptr, fd, n, 0.01, 1.0, 3)
        alone += cs.cs_launch_count(reset=True)
        refs.append(host(fd))
    for _ in range(2):  # capture, then replay
        fs = [dev(f) for f in f0]
        cs.cs_launch_count(reset=True)
        cs.cs_relax_batched([(h.ptr, f, n) for h, f, (_, _, n, _) in zip(hs, fs, specs)], 0.01, nsteps=3)
        # four convolutions per evaluation became one; alone, the N = 24 (9
        # cells) and N = 32 (2 cells) entries took the few-cell kernel, two
        # launches per evaluation
        assert cs.cs_launch_count(reset=True) == alone - 3 * 2 * 3 - 2 * 2 * 3
        for f, r in zip(fs, refs):
            assert np.array_equal(host(f), r)
    with pytest.raises(cs.CSError):  # the same state twice
        cs.cs_relax_batched([(hs[0].ptr, fs[0], 40), (hs[1].ptr, fs[0], 9)], 0.01)
    cs.cs_status(hs[0].ptr)
    for h in hs:
        h.close()


def test_tile_split_choices_agree(cs, orc):
    """N = 16 in float: 2 or 4 tile ranges per pencil add the same terms in
    a different grouping; both match the oracle and each other to float
    rounding, and each is the same for any number of cells in the call."""
    N = 16
    f = I.random_mixture_cells(N, L, 40, first_id=950)
    h = cs.Handle(N, L, 1.0, "fp32")
    got = {}
    for split in (2, 4):
        cs.cs_tune(h.ptr, cs.CS_TUNE_SPLIT, split)
        assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_SPLIT) == split
        got[split] = host(h.collide(dev(f)))
        assert np.array_equal(host(h.collide(dev(f[:3]))), got[split][:3])  # fewer cells, same sums
    ref = orc.collide(f[:4], N, L, 1.0)
    for split in (2, 4):
        assert rel(got[split][:4], ref) < 1e-5
    assert rel(got[2], got[4]) < 1e-6
    with pytest.raises(cs.CSError):
        cs.cs_tune(h.ptr, cs.CS_TUNE_SPLIT, 3)
    h.close()


def test_launch_choices_give_identical_results(cs):
    """The convolution's launch shape (groups per CTA, resident CTAs) changes
    only scheduling: every cell's sum runs in the same order."""
    N, nc = 16, 128
    h = cs.Handle(N, L, 1.0, "fp32")
    f = dev(I.random_mixture_cells(N, L, nc, first_id=900))
    outs = []
    for gpc, ctas in ((1, 2), (2, 4), (1, 8), (0, 0)):
        cs.cs_tune(h.ptr, cs.CS_TUNE_GROUPS_PER_CTA, gpc)
        cs.cs_tune(h.ptr, cs.CS_TUNE_CTAS_PER_SM, ctas)
        assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_GROUPS_PER_CTA) == gpc
        assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_CTAS_PER_SM) == ctas
        q = torch.empty_like(f)
        cs.cs_collide(h.ptr, f, nc, 1.0, q, 1)
        outs.append(host(q))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    best = cs.cs_autotune(h.ptr, nc)
    assert best > 0
    with pytest.raises(cs.CSError):
        cs.cs_tune(h.ptr, 99, 1)
    with pytest.raises(cs.CSError):
        cs.cs_tune_get(h.ptr, 99)
    h.close()


def test_launch_choices_at_n32_give_identical_results(cs):
    """At N = 32 one, two or four 32-cell groups share a CTA (each group's
    strips rotated differently among the warps): only scheduling and shared
    weight tiles change, never a sum's order; four groups need a group count
    divisible by four and fall back to two otherwise."""
    N, nc = 32, 128
    h = cs.Handle(N, L, 1.0, "fp32")
    f = dev(I.random_mixture_cells(N, L, nc, first_id=950))
    outs = []
    for gpc in (1, 2, 4, 0):
        cs.cs_tune(h.ptr, cs.CS_TUNE_GROUPS_PER_CTA, gpc)
        assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_GROUPS_PER_CTA) == gpc
        outs.append(host(h.collide(f)))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    cs.cs_tune(h.ptr, cs.CS_TUNE_GROUPS_PER_CTA, 4)
    assert np.array_equal(host(h.collide(dev(host(f)[:96]))), outs[0][:96])  # three groups: two per CTA
    with pytest.raises(cs.CSError):
        cs.cs_tune(h.ptr, cs.CS_TUNE_GROUPS_PER_CTA, 3)
    cs.cs_status(h.ptr)
    h.close()


def test_fma_probe_rates_are_plausible(cs):
    """The pipe probes land between a quarter of and just above the rates the
    unit counts give at the maximum clock (152 SMs x 128 FP32 lanes x 2.07 GHz
    = 40.3 T lane-ops/s; FP64 at 1/64 of that)."""
    ffma, ffma2, dfma = (cs.cs_fma_probe(k) / 1e12 for k in (0, 1, 2))
    assert 10.0 < ffma < 42.0 and 10.0 < ffma2 < 42.0, (ffma, ffma2)
    assert 0.1 < dfma < 1.5, dfma
    with pytest.raises(cs.CSError):
        cs.cs_fma_probe(3)


@pytest.mark.parametrize("N", [32])
def test_few_cells_two_strips_per_warp_is_exact(cs, orc, N):
    """At most 16 cells: the convolution puts two strips in each warp (16
    lanes each) instead of leaving half the lanes on padding.  Every (cell,
    output) runs the same operations in the same order, so the result is the
    same bit for bit as with one strip per warp (forced by one group per
    CTA), and matches the oracle."""
    f = I.random_mixture_cells(N, L, 16, first_id=1500)
    h = cs.Handle(N, L, 1.0, "fp32")
    cs.cs_tune(h.ptr, cs.CS_TUNE_FEW_CELLS, -1)  # the strip kernels only
    fd = dev(f)
    few = host(h.collide(fd))  # automatic: two strips per warp
    cs.cs_tune(h.ptr, cs.CS_TUNE_GROUPS_PER_CTA, 1)
    one = host(h.collide(fd))
    assert np.array_equal(few, one)
    cs.cs_tune(h.ptr, cs.CS_TUNE_GROUPS_PER_CTA, 0)
    assert np.array_equal(host(h.collide(dev(f[:5]))), few[:5])
    ref = orc.collide(f[[0, 15]], N, L, 1.0)
    assert rel(few[0], ref[0]) < 1e-5 and rel(few[15], ref[1]) < 1e-5
    cs.cs_status(h.ptr)
    h.close()


@pytest.mark.parametrize("N,split", [(24, 0), (32, 0), (32, 2), (32, 4)])
def test_few_cell_kernel_is_exact(cs, orc, N, split):
    """At most 16 cells (N = 24, 32) a warp can hold one cell and its lanes
    the outputs of a pencil.  Each output adds the same terms in the same
    order as in the strip kernels, also with a pencil's tiles split into 2 or
    4 ranges (N = 32), so every cell count from 1 to 16 gives the same bits
    either way (and the same bits as the cell inside a larger launch); the
    oracle checks two of the cells, and a split changes only the rounding."""
    f = I.random_mixture_cells(N, L, 40, first_id=1900)
    h = cs.Handle(N, L, 1.0, "fp32")
    assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_FEW_CELLS) == 0  # its default limit (6 cells at N = 32, 9 at 24)
    if split:
        whole = host(h.collide(dev(f)))
        cs.cs_tune(h.ptr, cs.CS_TUNE_SPLIT, split)
    big = host(h.collide(dev(f)))  # 40 cells: the strip kernel
    if split:
        assert 0 < np.max(np.abs(big - whole)) <= 1e-6 * np.max(np.abs(whole))
    for nc in (1, 3, 16):
        fd = dev(f[:nc])
        cs.cs_tune(h.ptr, cs.CS_TUNE_FEW_CELLS, 16)
        lane = host(h.collide(fd))
        cs.cs_tune(h.ptr, cs.CS_TUNE_FEW_CELLS, -1)
        strip = host(h.collide(fd))
        assert np.array_equal(lane, strip), nc
        assert np.array_equal(lane, big[:nc]), nc
    cs.cs_tune(h.ptr, cs.CS_TUNE_FEW_CELLS, 2)  # at most 2 cells: 3 take the strip kernel
    assert np.array_equal(host(h.collide(dev(f[:3]))), big[:3])
    for bad in (-2, 17):
        with pytest.raises(cs.CSError):
            cs.cs_tune(h.ptr, cs.CS_TUNE_FEW_CELLS, bad)
    cs.cs_tune(h.ptr, cs.CS_TUNE_FEW_CELLS, 0)
    ref = orc.collide(f[[0, 2]], N, L, 1.0)
    assert rel(big[0], ref[0]) < 1e-5 and rel(big[2], ref[1]) < 1e-5
    cs.cs_status(h.ptr)
    h.close()


@pytest.mark.parametrize("N,nc,split", [(16, 64, 2), (16, 40, 4), (32, 40, 0)])
def test_tile_shapes_give_identical_results(cs, N, nc, split):
    """The xi-tile (blocks of 8 or 4 uniform rows) and the ring depth (2, 3 or
    4 stages) change neither the terms nor the order each output adds them
    in: every tile shape gives the same bits, and unsupported requests are
    refused."""
    h = cs.Handle(N, L, 1.0, "fp32")
    if split:
        cs.cs_tune(h.ptr, cs.CS_TUNE_SPLIT, split)
    f = dev(I.random_mixture_cells(N, L, nc, first_id=1700))
    outs = []
    for tile in (1, 2, 3, 4):
        cs.cs_tune(h.ptr, cs.CS_TUNE_TILE, tile)
        assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_TILE) == tile
        outs.append(host(h.collide(f)))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    cs.cs_tune(h.ptr, cs.CS_TUNE_TILE, 0)
    assert cs.cs_autotune(h.ptr, nc) > 0
    tuned = host(h.collide(f))
    if cs.cs_tune_get(h.ptr, cs.CS_TUNE_SPLIT) in (0, split):
        assert np.array_equal(tuned, outs[0])
    else:  # the autotuner also picks the split, which groups the terms differently
        assert rel(tuned, outs[0]) < 1e-6
    cs.cs_status(h.ptr)
    h.close()
    h8 = cs.Handle(8, L, 1.0, "fp32")
    with pytest.raises(cs.CSError) as e:
        cs.cs_tune(h8.ptr, cs.CS_TUNE_TILE, 2)
    assert e.value.code == cs.CS_ENOTSUP
    h8.close()
