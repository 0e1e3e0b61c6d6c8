"""Python binding of the C ABI in include/cs.h (argument marshalling only).

Every ``cs_*`` function here calls the function of the same name in
``libcs.so``; PyTorch provides device memory and streams.  There is no
fallback: if the library is missing or fails to load, the first call raises
``CSError``.  Arrays follow the layouts of include/cs.h (float64,
``[ncells, N, N, N]`` for distributions, ``[ncells, N, N, N, 2]`` for the
spectral arrays of the step-level calls, ``[ncells, 5]`` for moments).
"""
from __future__ import annotations

import ctypes
import pathlib
import threading

import torch

CS_OK = 0
CS_EINVAL = -1
CS_ENOMEM = -2
CS_ENOTSUP = -3
CS_ECUDA = -4
CS_ETIMEOUT = -5
CS_ENONFINITE = -6
CS_FP64 = 0
CS_FP32 = 1
CS_WEIGHTS_RADIUS = 16  # OR'd into the precision: radius tables only, no table of every pair

_LIB_PATH = pathlib.Path(__file__).resolve().parent / "_build" / "libcs.so"
_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


class CSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libcs error {code}: {msg}")
        self.code = code


class Domain(ctypes.Structure):
    """cs_domain: dx (device), f_far (device), wall_T, wall_V[3]."""
    _fields_ = [("dx", _vp), ("f_far", _vp), ("wall_T", _d), ("wall_V", _d * 3)]


class Domain2D(ctypes.Structure):
    """cs_domain2d: dx (device), f_far (device), wall_T, wall_V[3], ny, dy."""
    _fields_ = [("dx", _vp), ("f_far", _vp), ("wall_T", _d), ("wall_V", _d * 3), ("ny", _i), ("dy", _d)]


class Domain3D(ctypes.Structure):
    """cs_domain3d: dx (device), f_far (device), wall_T, wall_V[3], ny, dy, nz, dz."""
    _fields_ = [("dx", _vp), ("f_far", _vp), ("wall_T", _d), ("wall_V", _d * 3), ("ny", _i), ("dy", _d),
                ("nz", _i), ("dz", _d)]


class BatchEntry(ctypes.Structure):
    """cs_batch_entry: handle, f (device), Q (device), ncells."""
    _fields_ = [("handle", _vp), ("f", _vp), ("Q", _vp), ("ncells", _i)]


class RelaxEntry(ctypes.Structure):
    """cs_relax_entry: handle, f (device, advanced in place), ncells."""
    _fields_ = [("handle", _vp), ("f", _vp), ("ncells", _i)]


_SIGS = {
    "cs_version": (_i, []),
    "cs_last_error": (ctypes.c_char_p, []),
    "cs_weights_bytes": (_i, [_i, _i, ctypes.POINTER(ctypes.c_size_t)]),
    "cs_weights_build": (_i, [_i, _d, _d, _i, _vp, ctypes.POINTER(_vp)]),
    "cs_weights_build_aniso": (_i, [_i, _d, _d, ctypes.POINTER(_d), _i, _i, _vp, ctypes.POINTER(_vp)]),
    "cs_handle_destroy": (_i, [_vp]),
    "cs_handle_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(_d),
                            ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_size_t)]),
    "cs_reserve": (_i, [_vp, _i]),
    "cs_weights_sample": (_i, [_vp, ctypes.POINTER(_i), _i, ctypes.POINTER(_d)]),
    "cs_transform": (_i, [_vp, _vp, _i, _vp, _vp]),
    "cs_convolve": (_i, [_vp, _vp, _i, _vp, _vp]),
    "cs_inverse": (_i, [_vp, _vp, _i, _d, _vp, _vp]),
    "cs_collide": (_i, [_vp, _vp, _i, _d, _vp, _i, _vp]),
    "cs_conserve": (_i, [_vp, _vp, _i, _vp, _vp]),
    "cs_moments": (_i, [_vp, _vp, _i, _vp, _vp]),
    "cs_relax": (_i, [_vp, _vp, _i, _d, _d, _i, _vp]),
    "cs_transport": (_i, [_vp, _vp, _i, ctypes.POINTER(Domain), _d, _vp]),
    "cs_step": (_i, [_vp, _vp, _i, ctypes.POINTER(Domain), _d, _d, _i, _vp]),
    "cs_tile_layout": (_i, [_i, _i, ctypes.POINTER(_i), _i, ctypes.POINTER(_i)]),
    "cs_status": (_i, [_vp]),
    "cs_collide_batched": (_i, [ctypes.POINTER(BatchEntry), _i, _d, _i, _vp]),
    "cs_relax_batched": (_i, [ctypes.POINTER(RelaxEntry), _i, _d, _d, _i, _vp]),
    "cs_fma_probe": (_i, [_i, _vp, ctypes.POINTER(_d)]),
    "cs_tune": (_i, [_vp, _i, _i]),
    "cs_tune_get": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "cs_autotune": (_i, [_vp, _i, _vp, ctypes.POINTER(_d)]),
    "cs_profile": (_i, [_vp, _i]),
    "cs_profile_read": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_longlong), _i]),
    "cs_launch_count": (_i, [ctypes.POINTER(ctypes.c_longlong), _i]),
    "cs_transport2d": (_i, [_vp, _vp, _i, ctypes.POINTER(Domain2D), _d, _vp]),
    "cs_step2d": (_i, [_vp, _vp, _i, ctypes.POINTER(Domain2D), _d, _d, _i, _vp]),
    "cs_transport3d": (_i, [_vp, _vp, _i, ctypes.POINTER(Domain3D), _d, _vp]),
    "cs_step3d": (_i, [_vp, _vp, _i, ctypes.POINTER(Domain3D), _d, _d, _i, _vp]),
    "cs_transport_shard_prepare": (_i, [_vp, _i, _i, _i, ctypes.POINTER(Domain), _vp]),
    "cs_transport_shard_stage": (_i, [_vp, _vp, _i, _i, _i, ctypes.POINTER(Domain), _d, _vp, _d, _vp, _d, _vp,
                                      _vp]),
}

STAGES = ("forward", "convolve", "inverse", "conserve", "transport")


def library_path() -> pathlib.Path:
    return _LIB_PATH


def lib():
    """The loaded libcs.so (raises CSError if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not _LIB_PATH.exists():
                raise CSError(CS_ENOTSUP, f"{_LIB_PATH} is missing: run paper_1301_4195_gb300.build.build()")
            L = ctypes.CDLL(str(_LIB_PATH))
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != CS_OK:
        raise CSError(rc, lib().cs_last_error().decode(errors="replace"))


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dptr(t: torch.Tensor, name: str):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise CSError(CS_EINVAL, f"{name} must be a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _ncells(t: torch.Tensor, N: int) -> int:
    n = t.numel() // N ** 3
    if n * N ** 3 != t.numel():
        raise CSError(CS_EINVAL, f"tensor of {t.numel()} elements is not a whole number of N^3 cells")
    return n


# ------------------------------------------------------------------ C ABI, same names
def cs_version() -> int:
    return lib().cs_version()


def cs_weights_bytes(N: int, precision: int) -> int:
    out = ctypes.c_size_t()
    _check(lib().cs_weights_bytes(N, precision, ctypes.byref(out)))
    return out.value


def cs_tile_layout(N: int, precision: int) -> list:
    n = _i()
    _check(lib().cs_tile_layout(N, precision, None, 0, ctypes.byref(n)))
    arr = (_i * n.value)()
    _check(lib().cs_tile_layout(N, precision, arr, n.value, ctypes.byref(n)))
    return list(arr)


def cs_status(h: int):
    """Raise CSError(CS_ETIMEOUT) if a bounded device wait expired (synchronises)."""
    _check(lib().cs_status(h))


def cs_weights_build(N: int, L: float, lam: float, precision: int = CS_FP64, stream=None) -> int:
    h = _vp()
    _check(lib().cs_weights_build(N, L, lam, precision, _stream(stream), ctypes.byref(h)))
    return h.value


def cs_weights_build_aniso(N: int, L: float, lam: float, moments, precision: int = CS_FP64, stream=None) -> int:
    """Weights of B = |u|^lam b(cos theta), b by its Legendre moments
    moments[l] = int_{S^2} b P_l dsigma (see include/cs.h)."""
    m = [float(x) for x in moments]
    arr = (_d * max(1, len(m)))(*m)
    h = _vp()
    _check(lib().cs_weights_build_aniso(N, L, lam, arr, len(m), precision, _stream(stream), ctypes.byref(h)))
    return h.value


def cs_handle_destroy(h: int):
    _check(lib().cs_handle_destroy(h))


def cs_handle_info(h: int):
    N, L, lam, p, b = _i(), _d(), _d(), _i(), ctypes.c_size_t()
    _check(lib().cs_handle_info(h, ctypes.byref(N), ctypes.byref(L), ctypes.byref(lam), ctypes.byref(p),
                                ctypes.byref(b)))
    return N.value, L.value, lam.value, p.value, b.value


def cs_reserve(h: int, ncells: int):
    _check(lib().cs_reserve(h, ncells))


def cs_weights_sample(h: int, km) -> list:
    flat = [int(v) for row in km for v in row]
    n = len(flat) // 6
    arr = (_i * len(flat))(*flat)
    out = (_d * max(n, 1))()
    _check(lib().cs_weights_sample(h, arr, n, out))
    return list(out)[:n]


def cs_transform(h, f, ncells, fhat, stream=None):
    _check(lib().cs_transform(h, _dptr(f, "f"), ncells, _dptr(fhat, "fhat"), _stream(stream)))


def cs_convolve(h, fhat, ncells, qhat, stream=None):
    _check(lib().cs_convolve(h, _dptr(fhat, "fhat"), ncells, _dptr(qhat, "qhat"), _stream(stream)))


def cs_inverse(h, qhat, ncells, eps, Q, stream=None):
    _check(lib().cs_inverse(h, _dptr(qhat, "qhat"), ncells, eps, _dptr(Q, "Q"), _stream(stream)))


def cs_collide(h, f, ncells, eps, Q, conserve=1, stream=None):
    _check(lib().cs_collide(h, _dptr(f, "f"), ncells, eps, _dptr(Q, "Q"), int(conserve), _stream(stream)))


def cs_collide_batched(entries, eps=1.0, conserve=1, stream=None):
    """entries: list of (handle_ptr, f, Q, ncells) with device tensors f, Q."""
    arr = (BatchEntry * max(1, len(entries)))()
    for i, (h, f, Q, n) in enumerate(entries):
        arr[i] = BatchEntry(h, _dptr(f, "f"), _dptr(Q, "Q"), int(n))
    _check(lib().cs_collide_batched(arr, len(entries), eps, int(conserve), _stream(stream)))


def cs_relax_batched(entries, dt, nsteps=1, eps=1.0, stream=None):
    """entries: list of (handle_ptr, f, ncells) with device state tensors f, advanced in place."""
    arr = (RelaxEntry * max(1, len(entries)))()
    for i, (h, f, n) in enumerate(entries):
        arr[i] = RelaxEntry(h, _dptr(f, "f"), int(n))
    _check(lib().cs_relax_batched(arr, len(entries), dt, eps, int(nsteps), _stream(stream)))


def cs_conserve(h, Q, ncells, moments=None, stream=None):
    _check(lib().cs_conserve(h, _dptr(Q, "Q"), ncells, _dptr(moments, "moments"), _stream(stream)))


def cs_moments(h, f, ncells, out, stream=None):
    _check(lib().cs_moments(h, _dptr(f, "f"), ncells, _dptr(out, "out"), _stream(stream)))


def cs_relax(h, f, ncells, dt, eps, nsteps, stream=None):
    _check(lib().cs_relax(h, _dptr(f, "f"), ncells, dt, eps, nsteps, _stream(stream)))


def _domain(dx, f_far, wall_T, wall_V):
    return Domain(_dptr(dx, "dx"), _dptr(f_far, "f_far"), float(wall_T), (_d * 3)(*[float(v) for v in wall_V]))


def cs_transport(h, f, ncells, dom: Domain, dt, stream=None):
    _check(lib().cs_transport(h, _dptr(f, "f"), ncells, ctypes.byref(dom), dt, _stream(stream)))


def cs_step(h, f, ncells, dom: Domain, dt, eps, nsteps, stream=None):
    _check(lib().cs_step(h, _dptr(f, "f"), ncells, ctypes.byref(dom), dt, eps, nsteps, _stream(stream)))


def _domain2d(dx, f_far, wall_T, wall_V, ny, dy):
    return Domain2D(_dptr(dx, "dx"), _dptr(f_far, "f_far"), float(wall_T), (_d * 3)(*[float(v) for v in wall_V]),
                    int(ny), float(dy))


def cs_transport2d(h, f, nx, dom: Domain2D, dt, stream=None):
    _check(lib().cs_transport2d(h, _dptr(f, "f"), nx, ctypes.byref(dom), dt, _stream(stream)))


def cs_step2d(h, f, nx, dom: Domain2D, dt, eps, nsteps, stream=None):
    _check(lib().cs_step2d(h, _dptr(f, "f"), nx, ctypes.byref(dom), dt, eps, nsteps, _stream(stream)))


def _domain3d(dx, f_far, wall_T, wall_V, ny, dy, nz, dz):
    return Domain3D(_dptr(dx, "dx"), _dptr(f_far, "f_far"), float(wall_T), (_d * 3)(*[float(v) for v in wall_V]),
                    int(ny), float(dy), int(nz), float(dz))


def cs_transport3d(h, f, nx, dom: Domain3D, dt, stream=None):
    _check(lib().cs_transport3d(h, _dptr(f, "f"), nx, ctypes.byref(dom), dt, _stream(stream)))


def cs_step3d(h, f, nx, dom: Domain3D, dt, eps, nsteps, stream=None):
    _check(lib().cs_step3d(h, _dptr(f, "f"), nx, ctypes.byref(dom), dt, eps, nsteps, _stream(stream)))


def cs_transport_shard_prepare(h, ncells, first_cell, total_cells, dom: Domain, stream=None):
    _check(lib().cs_transport_shard_prepare(h, ncells, first_cell, total_cells, ctypes.byref(dom), _stream(stream)))


def cs_transport_shard_stage(h, f_win, ncells, first_cell, total_cells, dom: Domain, a, x, b, y, c, out,
                             stream=None):
    """out = a x + b y + c R(f) on a shard; f_win holds ncells + 4 cells (two ghosts per side)."""
    _check(lib().cs_transport_shard_stage(h, _dptr(f_win, "f_win"), ncells, first_cell, total_cells,
                                          ctypes.byref(dom), float(a), _dptr(x, "x"), float(b), _dptr(y, "y"),
                                          float(c), _dptr(out, "out"), _stream(stream)))


CS_TUNE_GROUPS_PER_CTA = 1
CS_TUNE_WEIGHTS = 3
CS_TUNE_SPLIT = 4
CS_TUNE_CTAS_PER_SM = 2
CS_TUNE_WAIT_US = 5        # limit of the convolution's bounded waits, microseconds (0: 2 s)
CS_TUNE_TEST_STALL = 6     # 1: the first CTA of each convolution launch issues no copy (its waits run out)
CS_TUNE_CHECK_INPUT = 7    # 1: scan inputs for non-finite values, 2: also for negative ones
CS_TUNE_FORWARD_NEXT = 8   # 2: a Heun step's second forward transform in a launch of its own
CS_TUNE_L2_HINT = 9        # 1: plain copies; 2 (default): L2 eviction priorities (weights first, rows last)
CS_TUNE_TILE = 10          # xi-tile and ring depth at N = 16, 32: 1 (default) U 8 / 3 stages (2: two groups at 32), 2 U 4, 3 4 stages, 4 2
CS_TUNE_FEW_CELLS = 11     # most cells the few-cell kernel (N = 24, 32) serves: 0 its default, -1 never, 1 .. 16


def cs_tune(h, param: int, value: int):
    _check(lib().cs_tune(h, param, value))


def cs_tune_get(h, param: int) -> int:
    v = _i()
    _check(lib().cs_tune_get(h, param, ctypes.byref(v)))
    return v.value


def cs_autotune(h, ncells: int, stream=None) -> float:
    """Time the convolution launch choices on ncells cells, keep the fastest; returns ms."""
    ms = _d()
    _check(lib().cs_autotune(h, ncells, _stream(stream), ctypes.byref(ms)))
    return ms.value


def cs_fma_probe(kind: int, stream=None) -> float:
    """Measured lane operations per second of FFMA (0), packed FFMA2 (1) or DFMA (2)."""
    out = _d()
    _check(lib().cs_fma_probe(int(kind), _stream(stream), ctypes.byref(out)))
    return out.value


def cs_profile(h, enable: bool):
    _check(lib().cs_profile(h, int(bool(enable))))


def cs_profile_read(h, reset: bool = True) -> dict:
    """{stage: (total_ms, launches)} of the stages bracketed since the last reset."""
    ms = (_d * len(STAGES))()
    n = (ctypes.c_longlong * len(STAGES))()
    _check(lib().cs_profile_read(h, ms, n, int(bool(reset))))
    return {k: (ms[i], n[i]) for i, k in enumerate(STAGES)}


def cs_launch_count(reset: bool = False) -> int:
    """Kernels the library has enqueued (graph replays count their kernel nodes)."""
    n = ctypes.c_longlong()
    _check(lib().cs_launch_count(ctypes.byref(n), int(bool(reset))))
    return n.value


def cs_collide_noalloc(h, f, ncells, eps, Q, conserve=1, stream=None):
    """cs_collide for callers that must not allocate device memory: the
    intermediates live in a fixed 64 MiB array inside the library (see cs.h
    for the cell limits and the rule that overlapping calls race)."""
    fn = lib().cs_collide_noalloc
    fn.restype = _i
    fn.argtypes = [_vp, _vp, _i, _d, _vp, _i, _vp]
    _check(fn(h, _dptr(f, "f"), ncells, eps, _dptr(Q, "Q"), int(conserve), _stream(stream)))


# ------------------------------------------------------------------ convenience object
class Handle:
    """Owns one cs_handle_t (weights for one (N, L, lambda, precision))."""

    def __init__(self, N: int, L: float, lam: float, precision: str | int = "fp64", stream=None, moments=None):
        """moments: Legendre moments of an anisotropic b(cos theta) (None: isotropic)."""
        p = precision if isinstance(precision, int) else {
            "fp64": CS_FP64, "fp32": CS_FP32, "fp32-radius": CS_FP32 | CS_WEIGHTS_RADIUS}[precision]
        self.N, self.L, self.lam, self.precision = int(N), float(L), float(lam), p
        self._h = None
        if moments is None:
            self._h = cs_weights_build(self.N, self.L, self.lam, p, stream)
        else:
            self._h = cs_weights_build_aniso(self.N, self.L, self.lam, moments, p, stream)

    @property
    def ptr(self) -> int:
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            cs_handle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def weight_bytes(self) -> int:
        return cs_handle_info(self._h)[4]

    def reserve(self, ncells: int):
        cs_reserve(self._h, ncells)

    def _cells(self, f):
        return _ncells(f, self.N)

    def collide(self, f: torch.Tensor, eps: float = 1.0, conserve: bool = True, out=None, stream=None):
        """P_N Qt(f)/eps.  A CPU tensor is copied to the device and the result copied back."""
        host = not f.is_cuda
        fd = f.to("cuda", non_blocking=True) if host else f
        fd = fd.contiguous()
        Q = torch.empty_like(fd) if (out is None or host) else out
        cs_collide(self._h, fd, self._cells(fd), eps, Q, int(conserve), stream)
        if host:
            res = out if out is not None else torch.empty(f.shape, dtype=f.dtype, pin_memory=f.is_pinned())
            res.copy_(Q, non_blocking=False)
            return res
        return Q

    def transform(self, f, stream=None):
        n = self._cells(f)
        out = torch.empty(f.shape + (2,), dtype=torch.float64, device=f.device)
        cs_transform(self._h, f, n, out, stream)
        return out

    def convolve(self, fhat, stream=None):
        n = fhat.numel() // (2 * self.N ** 3)
        out = torch.empty_like(fhat)
        cs_convolve(self._h, fhat, n, out, stream)
        return out

    def inverse(self, qhat, eps=1.0, stream=None):
        n = qhat.numel() // (2 * self.N ** 3)
        out = torch.empty(qhat.shape[:-1], dtype=torch.float64, device=qhat.device)
        cs_inverse(self._h, qhat, n, eps, out, stream)
        return out

    def conserve(self, Q, want_moments=False, stream=None):
        n = self._cells(Q)
        mom = torch.empty((n, 5), dtype=torch.float64, device=Q.device) if want_moments else None
        cs_conserve(self._h, Q, n, mom, stream)
        return mom

    def moments(self, f, stream=None):
        n = self._cells(f)
        out = torch.empty((n, 5), dtype=torch.float64, device=f.device)
        cs_moments(self._h, f, n, out, stream)
        return out

    def relax(self, f, dt, nsteps, eps=1.0, stream=None):
        cs_relax(self._h, f, self._cells(f), dt, eps, nsteps, stream)
        return f

    def transport(self, f, dx, f_far, wall_T, wall_V, dt, stream=None):
        dom = _domain(dx, f_far, wall_T, wall_V)
        cs_transport(self._h, f, self._cells(f), dom, dt, stream)
        return f

    def step(self, f, dx, f_far, wall_T, wall_V, dt, nsteps=1, eps=1.0, stream=None):
        dom = _domain(dx, f_far, wall_T, wall_V)
        cs_step(self._h, f, self._cells(f), dom, dt, eps, nsteps, stream)
        return f

    def transport2d(self, f, dx, f_far, wall_T, wall_V, ny, dy, dt, stream=None):
        """f: [nx][ny][N][N][N] float64 CUDA tensor (x wall-normal, y periodic)."""
        nx = _ncells(f, self.N) // int(ny)
        cs_transport2d(self._h, f, nx, _domain2d(dx, f_far, wall_T, wall_V, ny, dy), dt, stream)
        return f

    def step2d(self, f, dx, f_far, wall_T, wall_V, ny, dy, dt, nsteps=1, eps=1.0, stream=None):
        nx = _ncells(f, self.N) // int(ny)
        cs_step2d(self._h, f, nx, _domain2d(dx, f_far, wall_T, wall_V, ny, dy), dt, eps, nsteps, stream)
        return f

    def transport3d(self, f, dx, f_far, wall_T, wall_V, ny, dy, nz, dz, dt, stream=None):
        """f: [nx][ny][nz][N][N][N] float64 CUDA tensor (x wall-normal, y and z periodic)."""
        nx = _ncells(f, self.N) // (int(ny) * int(nz))
        cs_transport3d(self._h, f, nx, _domain3d(dx, f_far, wall_T, wall_V, ny, dy, nz, dz), dt, stream)
        return f

    def step3d(self, f, dx, f_far, wall_T, wall_V, ny, dy, nz, dz, dt, nsteps=1, eps=1.0, stream=None):
        nx = _ncells(f, self.N) // (int(ny) * int(nz))
        cs_step3d(self._h, f, nx, _domain3d(dx, f_far, wall_T, wall_V, ny, dy, nz, dz), dt, eps, nsteps, stream)
        return f

    def sample_weights(self, km):
        return cs_weights_sample(self._h, km)
