"""cs_collide_noalloc, the entry point for callers that cannot allocate device memory.

Some callers may not call cudaMalloc at all (a plugin or host callback inside a
runtime that owns every allocation, a real-time loop that must not block on
the allocator).  For them the library keeps the collision operator's
intermediate arrays in one fixed array compiled into it.  These tests call
that entry point through the C ABI and check that it returns what
cs_collide returns, on two calls in a row (the second call reuses the array
the first one left behind), and that requests beyond the fixed size are
refused.  The file is named so pytest collects it last.
"""
import ctypes

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
    fn = api.lib().cs_collide_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                   ctypes.c_int, ctypes.c_void_p]
    return api


def _noalloc(api, h, f, Q, ncells):
    stream = torch.cuda.current_stream().cuda_stream
    return api.lib().cs_collide_noalloc(h.ptr, f.data_ptr(), ncells, 1.0, Q.data_ptr(), 1, stream)


@pytest.mark.parametrize("N,prec,split,n1,n2", [(8, "fp64", 0, 33, 5), (16, "fp32", 0, 40, 64),
                                                (16, "fp32", 4, 384, 7), (32, "fp32", 0, 64, 3),
                                                (32, "fp32", 4, 32, 5)])
def test_noalloc_matches_cs_collide_twice(cs, N, prec, split, n1, n2):
    """Both entry points run the same kernels in the same order on the same
    launch choices, so their results must agree bit for bit; any overlap of
    the intermediate buffers inside the fixed array would break that.  The
    four-way split (the launches that write all four partial sums and the
    counters of finished ranges) is run at its limits: 384 cells at N = 16,
    32 at N = 32."""
    h = cs.Handle(N, L, 1.0, prec)
    if split:
        cs.cs_tune(h.ptr, cs.CS_TUNE_SPLIT, split)
    for ncells, first in ((n1, 0), (n2, 500)):
        f = torch.from_numpy(I.random_mixture_cells(N, L, ncells, first_id=first)).cuda()
        ref = torch.empty_like(f)
        cs.cs_collide(h.ptr, f, ncells, 1.0, ref, 1)
        got = torch.full_like(f, float("nan"))
        assert _noalloc(cs, h, f, got, ncells) == cs.CS_OK, cs.lib().cs_last_error()
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(g).all()
        assert np.array_equal(g, r)
    cs.cs_status(h.ptr)
    h.close()


@pytest.mark.parametrize("N,prec,split,limit", [(32, "fp64", 0, 32), (16, "fp32", 4, 384), (16, "fp32", 0, 672),
                                                (32, "fp32", 0, 64), (32, "fp32", 4, 32)])
def test_noalloc_refuses_more_cells_than_the_fixed_array_holds(cs, N, prec, split, limit):
    """The limit follows from the buffers a call needs: three spectral
    arrays, two more for a four-way split."""
    h = cs.Handle(N, L, 1.0, prec)
    if split:
        cs.cs_tune(h.ptr, cs.CS_TUNE_SPLIT, split)
    f = torch.zeros((limit + 1, N, N, N), dtype=torch.float64, device="cuda")
    Q = torch.empty_like(f)
    rc = _noalloc(cs, h, f, Q, limit + 1)
    assert rc == cs.CS_EINVAL
    msg = cs.lib().cs_last_error().decode()
    assert f"at most {limit} cells" in msg
    h.close()
