"""Oracle parity at the sizes and launch shapes the bench times.

* The 128-cell N = 16 wall problem (cells dx_j = min(1/8 1.05^j, 1/2), so
  the capped cells from j = 29 on are included; wall at T_w = 1.5, far field
  the unit Maxwellian), one and three Strang steps through cs_step (the
  replayed step graph the bench times) against the oracle's Strang step on
  all 128 cells: FP64 1e-12, FP32 1e-5 of the largest state value.  The
  bench's own initial state (the unit Maxwellian everywhere) has a
  collision term that is zero up to spectral accuracy, so the same step is
  also taken from random 2-3 Maxwellian mixtures in every cell, where the
  collision term is large, and the step's increment f_{n+1} - f_n is compared
  as well (FP64 1e-10, FP32 1e-5 of the largest increment).
* cs_collide at N = 24 on 70 cells (three 32-cell groups, the last one
  partial), lambda = 0 and 1, both precisions, on sampled cells from every
  group against the oracle's operator (FP64 1e-12, FP32 1e-5), with the
  moment drift of every cell <= 1e-12.
* cs_relax in float at N = 16 and 24 (the Heun step whose first inverse
  launch also transforms forward for the second evaluation) against the
  oracle's Heun steps on sampled cells (1e-5), and with that fusion switched
  off (CS_TUNE_FORWARD_NEXT = 2) bit for bit equal to it switched on.
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
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / np.abs(np.asarray(ref)).max())


def drift(Q, N):
    """max over cells and rows of |C Q| / sum |C| |Q| (rounding-relative moment drift)."""
    v = I.velocity_grid(N, L)
    w = (2 * L / N) ** 3
    rows = np.stack([np.ones_like(v[0]), v[0], v[1], v[2], v[0] ** 2 + v[1] ** 2 + v[2] ** 2]).reshape(5, -1) * w
    q = Q.reshape(Q.shape[0], -1)
    return float((np.abs(q @ rows.T) / (np.abs(q) @ np.abs(rows).T)).max())


# ------------------------------------------------------------------ the bench's step, all 128 cells
N16, NC16 = 16, 128
_oracle_runs = {}


def _initial(kind):
    if kind == "unit":
        return I.wall_initial(N16, L, NC16)  # the bench's state
    return I.random_mixture_cells(N16, L, NC16, first_id=3000)


def _oracle_states(orc, kind, nsteps):
    """Oracle states after 0 .. nsteps Strang steps (cached across precisions)."""
    key = (kind, nsteps)
    if key not in _oracle_runs:
        dx = I.wall_grid(NC16)
        far = I.maxwellian(N16, L, 1.0, (0, 0, 0), 1.0)
        states = [_initial(kind)]
        for _ in range(nsteps):
            states.append(orc.strang_step(states[-1], N16, L, 1.0, dx, TW, (0, 0, 0), far, DT))
        _oracle_runs[key] = states
    return _oracle_runs[key]


@pytest.mark.parametrize("prec,tol,tol_inc", [("fp64", 1e-12, 1e-10), ("fp32", 1e-5, 1e-5)])
@pytest.mark.parametrize("kind,nsteps", [("unit", 1), ("unit", 3), ("mix", 1)])
def test_wall16_128_cells_strang_matches_oracle(cs, orc, prec, tol, tol_inc, kind, nsteps):
    ref = _oracle_states(orc, kind, nsteps)
    h = cs.Handle(N16, L, 1.0, prec)
    if prec == "fp32":
        cs.cs_autotune(h.ptr, NC16)  # the bench's launch choices
    f = dev(ref[0])
    dx = dev(I.wall_grid(NC16))
    far = dev(I.maxwellian(N16, L, 1.0, (0, 0, 0), 1.0))
    prev = None
    for s in range(nsteps):  # one cs_step call per step (the bench's replayed graph)
        prev = host(f)
        h.step(f, dx, far, TW, (0.0, 0.0, 0.0), DT, nsteps=1)
    got = host(f)
    cs.cs_status(h.ptr)
    assert rel(got, ref[-1]) < tol
    if kind == "mix":  # the increment of the step, where the collision term is large
        assert rel(got - prev, ref[-1] - ref[-2]) < tol_inc
    h.close()


# ------------------------------------------------------------------ N = 24, several groups
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_collide_n24_three_groups_matches_oracle(cs, orc, prec, tol, lam):
    N, nc = 24, 70
    f = I.random_mixture_cells(N, L, nc, first_id=4000)
    h = cs.Handle(N, L, lam, prec)
    got = host(h.collide(dev(f)))
    idx = [0, 31, 32, 50, 64, 69]  # every group, the last (partial) one included
    ref = orc.collide(f[idx], N, L, lam)
    for i, c in enumerate(idx):
        assert rel(got[c], ref[i]) < tol, c
    assert drift(got, N) < 1e-12
    raw = host(h.collide(dev(f), conserve=False))
    refr = orc.collide(f[idx[-2:]], N, L, lam, conserve=False)
    for i, c in enumerate(idx[-2:]):
        assert rel(raw[c], refr[i]) < tol, c
    cs.cs_status(h.ptr)
    h.close()


# ------------------------------------------------------------------ Heun steps with the fused forward transform
@pytest.mark.parametrize("N,nc", [(16, 40), (24, 36)])
def test_relax_float_matches_oracle_and_fusion_is_exact(cs, orc, N, nc):
    f0 = I.random_mixture_cells(N, L, nc, first_id=4500)
    h = cs.Handle(N, L, 1.0, "fp32")
    outs = {}
    for mode in (0, 2):  # 0: the first inverse launch transforms forward (default); 2: a separate launch
        cs.cs_tune(h.ptr, cs.CS_TUNE_FORWARD_NEXT, mode)
        assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_FORWARD_NEXT) == mode
        fd = dev(f0)
        cs.cs_launch_count(reset=True)
        h.relax(fd, DT, 3)
        outs[mode] = (host(fd), cs.cs_launch_count(reset=True))
    assert np.array_equal(outs[0][0], outs[2][0])
    assert outs[2][1] == outs[0][1] + 3  # one forward launch more per step
    idx = [0, nc // 2, nc - 1]
    ref = orc.rk2_homogeneous(f0[idx], N, L, 1.0, DT, 3)
    for i, c in enumerate(idx):
        assert rel(outs[0][0][c], ref[i]) < 1e-5, c
        # the change over the three steps (six float evaluations of Q) to the same bar
        assert rel(outs[0][0][c] - f0[c], ref[i] - f0[c]) < 1e-5, c
    cs.cs_status(h.ptr)
    h.close()
