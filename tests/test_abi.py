"""The C-ABI library builds, loads and exports every entry point include/cs.h declares.

No call here launches GPU work: only host-side queries and argument checks
that fail before anything is enqueued.
"""
import ctypes
import pathlib
import re

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def libcs():
    from paper_1301_4195_gb300 import build
    build.build()
    import torch  # noqa: F401  (brings the CUDA runtime into the process)
    from paper_1301_4195_gb300 import api
    return api


def declared_symbols():
    text = (ROOT / "include" / "cs.h").read_text()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(cs_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("cs_weights_build", "cs_collide", "cs_conserve", "cs_step", "cs_moments",
                     "cs_weights_bytes", "cs_handle_destroy", "cs_relax", "cs_transport"):
        assert required in names


def test_library_exports_every_declared_symbol(libcs):
    lib = ctypes.CDLL(str(libcs.library_path()))
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_queries(libcs):
    assert libcs.cs_version() >= 100
    b16 = libcs.cs_weights_bytes(16, libcs.CS_FP32)
    b32 = libcs.cs_weights_bytes(32, libcs.CS_FP32)
    # symmetrised half of the 27 N^6 / 64 valid pairs, 4 bytes each, rows padded to
    # multiples of 4 entries (+13% at N = 16, +6% at N = 32), plus small tables
    assert 0.49 * 27 * 16 ** 6 / 64 * 4 < b16 < 0.58 * 27 * 16 ** 6 / 64 * 4 + 1e5
    assert 0.49 * 27 * 32 ** 6 / 64 * 4 < b32 < 0.55 * 27 * 32 ** 6 / 64 * 4 + 1e5
    assert b32 > 50 * b16
    assert libcs.cs_weights_bytes(32, libcs.CS_FP64) > 1.9 * b32


def test_radius_table_bytes(libcs):
    """CS_WEIGHTS_RADIUS: A has (3 (N/2)^2 + 1) x (3 (N-1)^2 + 1) floats and
    B 3 (N/2)^2 + 1; the flag leaves the table of every pair out, and needs a
    float handle of the strip kernel."""
    R = libcs.CS_WEIGHTS_RADIUS
    for N in (16, 32, 64):
        full = libcs.cs_weights_bytes(N, libcs.CS_FP32)
        rad = libcs.cs_weights_bytes(N, libcs.CS_FP32 | R)
        KK, BB = 3 * (N // 2) ** 2 + 1, 3 * (N - 1) ** 2 + 1
        assert 4 * (KK * BB + KK) <= rad < 4 * (KK * BB + KK) + 1e6
        assert full > rad
    assert libcs.cs_weights_bytes(64, libcs.CS_FP32 | R) < 2e8 < 5e10 < libcs.cs_weights_bytes(64, libcs.CS_FP32)
    for N, prec in ((16, libcs.CS_FP64 | R), (12, libcs.CS_FP32 | R)):
        with pytest.raises(libcs.CSError) as e:
            libcs.cs_weights_bytes(N, prec)
        assert e.value.code == libcs.CS_EINVAL
        with pytest.raises(libcs.CSError) as e:
            libcs.cs_weights_build(N, 6.0, 1.0, prec, stream=0)
        assert e.value.code == libcs.CS_EINVAL


def test_launch_count_is_host_side(libcs):
    libcs.cs_launch_count(reset=True)
    assert libcs.cs_launch_count() == 0
    assert libcs.lib().cs_launch_count(None, 0) == libcs.CS_EINVAL


@pytest.mark.parametrize("N,L,lam,prec", [(5, 6.0, 1.0, 0), (66, 6.0, 1.0, 0), (2, 6.0, 1.0, 0),
                                          (8, -1.0, 1.0, 0), (8, 6.0, 1.5, 0), (8, 6.0, -3.0, 0),
                                          (8, 6.0, 1.0, 7), (8, float("nan"), 1.0, 0)])
def test_weights_build_rejects_bad_arguments(libcs, N, L, lam, prec):
    with pytest.raises(libcs.CSError) as e:
        libcs.cs_weights_build(N, L, lam, prec, stream=0)
    assert e.value.code == libcs.CS_EINVAL
    assert libcs.lib().cs_last_error().decode()


def test_null_handle_is_rejected(libcs):
    lib = libcs.lib()
    assert lib.cs_collide(None, None, 1, 1.0, None, 1, None) == libcs.CS_EINVAL
    assert lib.cs_handle_destroy(None) == libcs.CS_OK
    assert lib.cs_weights_bytes(16, 0, None) == libcs.CS_EINVAL


def test_batched_calls_and_probe_check_arguments_on_the_host(libcs):
    """Refused before any device work: too many or negative entries, a NULL
    list, bad eps/dt/nsteps, an unknown probe kind, tuning a NULL handle."""
    lib = libcs.lib()
    ent = (libcs.BatchEntry * 17)()
    rel = (libcs.RelaxEntry * 17)()
    assert lib.cs_collide_batched(ent, 17, 1.0, 1, None) == libcs.CS_EINVAL
    assert lib.cs_collide_batched(None, 2, 1.0, 1, None) == libcs.CS_EINVAL
    assert lib.cs_collide_batched(ent, -1, 1.0, 1, None) == libcs.CS_EINVAL
    assert lib.cs_collide_batched(ent, 0, 0.0, 1, None) == libcs.CS_EINVAL
    assert lib.cs_collide_batched(ent, 0, 1.0, 1, None) == libcs.CS_OK  # nothing to do
    assert lib.cs_relax_batched(rel, 17, 0.01, 1.0, 1, None) == libcs.CS_EINVAL
    assert lib.cs_relax_batched(rel, 0, float("nan"), 1.0, 1, None) == libcs.CS_EINVAL
    assert lib.cs_relax_batched(rel, 0, 0.01, 1.0, -1, None) == libcs.CS_EINVAL
    assert lib.cs_relax_batched(rel, 0, 0.01, 1.0, 5, None) == libcs.CS_OK
    out = libcs._d()
    assert lib.cs_fma_probe(3, None, libcs.ctypes.byref(out)) == libcs.CS_EINVAL
    assert lib.cs_fma_probe(0, None, None) == libcs.CS_EINVAL
    assert lib.cs_tune(None, libcs.CS_TUNE_SPLIT, 4) == libcs.CS_EINVAL
    assert lib.cs_last_error().decode()


@pytest.mark.parametrize("N", list(range(4, 33, 2)) + [40, 48, 64])
@pytest.mark.parametrize("prec", [0, 1])
def test_tile_layout_covers_every_valid_pair_once(libcs, N, prec):
    """Sec. 3.2: the pairs (m3, k3) with k3 - m3 + N/2 in [0, N-1]; every one of them
    must sit at exactly one entry of a tile, the rest being padding."""
    m = libcs.cs_tile_layout(N, prec)
    assert len(m) % 4 == 0
    got = sorted(e for e in m if e >= 0)
    want = sorted(m3 * 256 + k3 for m3 in range(N) for k3 in range(N) if 0 <= k3 - m3 + N // 2 <= N - 1)
    assert got == want
    assert len(want) == 3 * N * N // 4


def test_aniso_build_checks_its_moments_on_the_host(libcs):
    lib = libcs.lib()
    h = libcs._vp()
    good = (libcs._d * 3)(1.0, 0.0, 0.3)
    bad0 = (libcs._d * 2)(0.0, 0.1)
    nan = (libcs._d * 2)(1.0, float("nan"))
    assert lib.cs_weights_build_aniso(16, 6.0, 1.0, None, 1, 0, None, libcs.ctypes.byref(h)) == libcs.CS_EINVAL
    assert lib.cs_weights_build_aniso(16, 6.0, 1.0, good, 0, 0, None, libcs.ctypes.byref(h)) == libcs.CS_EINVAL
    assert lib.cs_weights_build_aniso(16, 6.0, 1.0, good, 17, 0, None, libcs.ctypes.byref(h)) == libcs.CS_EINVAL
    assert lib.cs_weights_build_aniso(16, 6.0, 1.0, bad0, 2, 0, None, libcs.ctypes.byref(h)) == libcs.CS_EINVAL
    assert lib.cs_weights_build_aniso(16, 6.0, 1.0, nan, 2, 0, None, libcs.ctypes.byref(h)) == libcs.CS_EINVAL
    assert lib.cs_weights_build_aniso(16, 6.0, 1.0, good, 3, libcs.CS_FP32 | libcs.CS_WEIGHTS_RADIUS, None,
                                      libcs.ctypes.byref(h)) == libcs.CS_EINVAL
    assert lib.cs_weights_build_aniso(5, 6.0, 1.0, good, 3, 0, None, libcs.ctypes.byref(h)) == libcs.CS_EINVAL


def test_transport3d_checks_its_domain_on_the_host(libcs):
    lib = libcs.lib()
    assert lib.cs_transport3d(None, None, 4, None, 0.01, None) == libcs.CS_EINVAL
    assert lib.cs_step3d(None, None, 4, None, 0.01, 1.0, 1, None) == libcs.CS_EINVAL
