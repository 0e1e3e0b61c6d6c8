"""Failure detection on the GPU in the forms that neither fault nor hang it.

* Bounded waits: the convolution's mbarrier waits have a limit (2 s by
  default, CS_TUNE_WAIT_US).  With the test stall on (CS_TUNE_TEST_STALL) the
  first CTA of a launch issues no copy for its first work item, so nothing
  ever completes the barrier its warps wait on: the waits run out after the
  limit, the CTA records the expiry and returns, the launch ends, and
  cs_status reports CS_ETIMEOUT.  With the stall off again the next call on
  the same handle is correct (bit for bit equal to a clean handle's) and
  cs_status is clear.  The same in a shared (mixed) convolution launch.
* Non-finite input: with the input scan on (CS_TUNE_CHECK_INPUT = 1) a NaN
  or an infinity put into f on the host makes cs_status report
  CS_ENONFINITE after cs_collide, cs_relax or cs_step; mode 2 also reports a
  negative value; with the scan off nothing is reported.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("N,nc", [(16, 64), (32, 32), (32, 3), (24, 5)])  # the last two: the few-cell kernel
def test_expired_wait_reports_timeout_and_the_handle_recovers(cs, N, nc):
    f = dev(I.random_mixture_cells(N, L, nc, first_id=8100))
    clean = cs.Handle(N, L, 1.0, "fp32")
    ref = host(clean.collide(f))
    cs.cs_status(clean.ptr)
    clean.close()
    h = cs.Handle(N, L, 1.0, "fp32")
    cs.cs_tune(h.ptr, cs.CS_TUNE_WAIT_US, 2000)  # 2 ms
    assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_WAIT_US) == 2000
    cs.cs_tune(h.ptr, cs.CS_TUNE_TEST_STALL, 1)
    h.collide(f)
    with pytest.raises(cs.CSError) as e:
        cs.cs_status(h.ptr)
    assert e.value.code == cs.CS_ETIMEOUT
    cs.cs_status(h.ptr)  # cs_status cleared the record
    cs.cs_tune(h.ptr, cs.CS_TUNE_TEST_STALL, 0)
    cs.cs_tune(h.ptr, cs.CS_TUNE_WAIT_US, 0)
    got = host(h.collide(f))
    cs.cs_status(h.ptr)
    assert np.array_equal(got, ref)
    h.close()


def test_expired_wait_in_a_shared_launch(cs):
    """Two float handles whose convolutions share one persistent launch: the
    stall set on one of them makes the launch's first CTA time out; the
    status is reported, and the next batched call is correct again."""
    specs = [(16, 64), (24, 40)]
    hs = [cs.Handle(N, L, 1.0, "fp32") for N, _ in specs]
    fs = [dev(I.random_mixture_cells(N, L, n, first_id=8200 + 100 * i)) for i, (N, n) in enumerate(specs)]
    refs = [host(h.collide(f)) for h, f in zip(hs, fs)]
    qs = [torch.empty_like(f) for f in fs]
    entries = [(h.ptr, f, q, n) for h, f, q, (_, n) in zip(hs, fs, qs, specs)]
    for h in hs:
        cs.cs_tune(h.ptr, cs.CS_TUNE_WAIT_US, 2000)
        cs.cs_tune(h.ptr, cs.CS_TUNE_TEST_STALL, 1)
    cs.cs_collide_batched(entries)
    torch.cuda.synchronize()
    codes = []
    for h in hs:
        try:
            cs.cs_status(h.ptr)
            codes.append(cs.CS_OK)
        except cs.CSError as e:
            codes.append(e.code)
    # the CTA that timed out records the expiry in the status of the handle whose item it held
    assert cs.CS_ETIMEOUT in codes and set(codes) <= {cs.CS_OK, cs.CS_ETIMEOUT}
    for h in hs:
        cs.cs_tune(h.ptr, cs.CS_TUNE_TEST_STALL, 0)
        cs.cs_tune(h.ptr, cs.CS_TUNE_WAIT_US, 0)
    cs.cs_collide_batched(entries)
    for h, q, r in zip(hs, qs, refs):
        cs.cs_status(h.ptr)
        assert np.array_equal(host(q), r)
    for h in hs:
        h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonfinite_input_is_reported(cs, prec):
    N, nc = 16, 40
    f0 = I.random_mixture_cells(N, L, nc, first_id=8300)
    bad = f0.copy()
    bad[17, 3, 4, 5] = np.nan
    inf = f0.copy()
    inf[39, 15, 0, 7] = np.inf
    neg = f0.copy()
    neg[5, 8, 8, 8] = -1e-3
    h = cs.Handle(N, L, 1.0, prec)
    # scan off (default): nothing is reported
    h.collide(dev(bad))
    cs.cs_status(h.ptr)
    cs.cs_tune(h.ptr, cs.CS_TUNE_CHECK_INPUT, 1)
    assert cs.cs_tune_get(h.ptr, cs.CS_TUNE_CHECK_INPUT) == 1
    for arr in (bad, inf):
        h.collide(dev(arr))
        with pytest.raises(cs.CSError) as e:
            cs.cs_status(h.ptr)
        assert e.value.code == cs.CS_ENONFINITE and "non-finite" in str(e.value)
    # a finite input passes, and a negative value only counts in mode 2
    h.collide(dev(f0))
    h.collide(dev(neg))
    cs.cs_status(h.ptr)
    cs.cs_tune(h.ptr, cs.CS_TUNE_CHECK_INPUT, 2)
    h.collide(dev(neg))
    with pytest.raises(cs.CSError) as e:
        cs.cs_status(h.ptr)
    assert e.value.code == cs.CS_ENONFINITE and "negative" in str(e.value)
    # every step of a relaxation and of a Strang step scans its state
    cs.cs_tune(h.ptr, cs.CS_TUNE_CHECK_INPUT, 1)
    fd = dev(bad)
    h.relax(fd, 0.01, 2)
    with pytest.raises(cs.CSError) as e:
        cs.cs_status(h.ptr)
    assert e.value.code == cs.CS_ENONFINITE
    dx = dev(I.wall_grid(nc))
    far = dev(I.maxwellian(N, L, 1.0, (0, 0, 0), 1.0))
    fd = dev(bad)
    h.step(fd, dx, far, 1.5, (0.0, 0.0, 0.0), 0.01, nsteps=1)
    with pytest.raises(cs.CSError) as e:
        cs.cs_status(h.ptr)
    assert e.value.code == cs.CS_ENONFINITE
    # the scan changes no result
    cs.cs_tune(h.ptr, cs.CS_TUNE_CHECK_INPUT, 0)
    a = host(h.collide(dev(f0)))
    cs.cs_tune(h.ptr, cs.CS_TUNE_CHECK_INPUT, 1)
    b = host(h.collide(dev(f0)))
    cs.cs_status(h.ptr)
    assert np.array_equal(a, b)
    h.close()
