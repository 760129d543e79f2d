"""Python binding of liblbm.so (the C ABI declared in include/lbm.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  There is no CPU fallback -- if the library cannot be built or loaded, or no
CUDA device is present, the calls raise.

The functions carry the C names (lbm_create, lbm_init_phi, lbm_step, ...).  Device
memory comes from PyTorch's caching allocator by default, and the solver runs on a
caller-chosen CUDA stream (PyTorch's current stream by default).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, Structure, c_char_p, c_double, c_int, c_longlong,
                    c_size_t, c_uint, c_void_p)
from typing import Optional

import numpy as np

from . import _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EBUSY = range(7)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA",
                4: "LBM_EUNSTABLE", 5: "LBM_ETIMEOUT", 6: "LBM_EBUSY"}

LBM_FLAG_BUOYANCY, LBM_FLAG_SRT_FLOW, LBM_FLAG_D3Q7_STENCIL = 1, 2, 4
LBM_STORAGE_FP32, LBM_STORAGE_FP16, LBM_STORAGE_BF16 = 0, 1, 2
STORAGES = {"fp32": LBM_STORAGE_FP32, "fp16": LBM_STORAGE_FP16, "bf16": LBM_STORAGE_BF16}
LBM_PATTERN_AB, LBM_PATTERN_AA = 0, 1
PATTERNS = {"ab": LBM_PATTERN_AB, "aa": LBM_PATTERN_AA}

LBM_FIELD_PHI, LBM_FIELD_RHO, LBM_FIELD_P, LBM_FIELD_U, LBM_FIELD_MU = 1, 2, 4, 8, 16
LBM_FIELD_ALL = 31

LBM_VELOCITY_NONE, LBM_VELOCITY_UNIFORM, LBM_VELOCITY_ROTATION, LBM_VELOCITY_DEFORMATION = 0, 1, 2, 3
VELOCITY_KINDS = {"uniform": LBM_VELOCITY_UNIFORM, "rotation": LBM_VELOCITY_ROTATION,
                  "deformation": LBM_VELOCITY_DEFORMATION}

(LBM_TUNE_PREFETCH_COLLIDE, LBM_TUNE_PREFETCH_PHI, LBM_TUNE_MU_TMA, LBM_TUNE_GRAPHS,
 LBM_TUNE_TMA_WAIT_POLLS, LBM_TUNE_ROWS, LBM_TUNE_FUSED, LBM_TUNE_FUSED_SEGMENT,
 LBM_TUNE_FUSED_PREFETCH, LBM_TUNE_CELL_PAIRS, LBM_TUNE_STENCIL_STAGE,
 LBM_TUNE_PREFETCH_COLLIDE_SUMS) = range(12)

KERNEL_PHI, KERNEL_MU, KERNEL_COLLIDE = 0, 1, 2
KERNEL_NAMES = ("k_phi", "k_mu", "k_collide")


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class LbmGrid(Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("walls_z", c_int)]


class LbmParams(Structure):
    _fields_ = [("rho_l", c_double), ("rho_g", c_double), ("nu_l", c_double), ("nu_g", c_double),
                ("mobility", c_double), ("D", c_double), ("sigma", c_double),
                ("g", c_double * 3), ("A", c_double), ("sf", c_double * 7),
                ("sg", c_double * 15), ("flags", c_uint), ("storage", c_int),
                ("pattern", c_int)]


ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_void_p)


class LbmAllocator(Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p)]


_LIB = None

_SIGNATURES = {
    "lbm_create": (c_int, [POINTER(LbmGrid), POINTER(LbmParams), POINTER(LbmAllocator), c_void_p,
                           POINTER(c_void_p)]),
    "lbm_init_phi": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_step": (c_int, [c_void_p, c_int]),
    "lbm_read_fields": (c_int, [c_void_p, c_uint, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_reduce": (c_int, [c_void_p, POINTER(c_double), POINTER(c_double)]),
    "lbm_read_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_longlong)]),
    "lbm_read_state_at": (c_int, [c_void_p, c_void_p, c_longlong, c_void_p, c_void_p, c_void_p,
                                  POINTER(c_longlong)]),
    "lbm_write_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_longlong]),
    "lbm_get_step": (c_int, [c_void_p, POINTER(c_longlong)]),
    "lbm_set_velocity": (c_int, [c_void_p, c_int, c_double, c_double]),
    "lbm_set_tuning": (c_int, [c_void_p, c_int, c_int]),
    "lbm_get_tuning": (c_int, [c_void_p, c_int, POINTER(c_int)]),
    "lbm_profile": (c_int, [c_void_p, c_int]),
    "lbm_profile_read": (c_int, [c_void_p, c_int, POINTER(c_double), POINTER(c_longlong)]),
    "lbm_field_sum_noalloc": (c_int, [c_void_p, c_longlong, c_void_p, c_void_p]),
    "lbm_memory_bytes": (c_int, [POINTER(LbmGrid), POINTER(LbmParams), POINTER(c_size_t)]),
    "lbm_batch_create": (c_int, [POINTER(LbmAllocator), c_void_p, POINTER(c_void_p)]),
    "lbm_batch_step": (c_int, [c_void_p, POINTER(c_void_p), c_int, c_int]),
    "lbm_batch_set_grid": (c_int, [c_void_p, c_int, c_int]),
    "lbm_reduce_async": (c_int, [c_void_p, c_void_p]),
    "lbm_step_reduce": (c_int, [c_void_p, c_int, POINTER(c_double), POINTER(c_double)]),
    "lbm_step_reduce_async": (c_int, [c_void_p, c_int, c_void_p]),
    "lbm_batch_get_grid": (c_int, [c_void_p, c_int, POINTER(c_int)]),
    "lbm_batch_set_prefetch": (c_int, [c_void_p, c_int, c_int]),
    "lbm_batch_set_split": (c_int, [c_void_p, c_longlong]),
    "lbm_batch_get_split": (c_int, [c_void_p, POINTER(c_longlong)]),
    "lbm_batch_get_prefetch": (c_int, [c_void_p, c_int, POINTER(c_int)]),
    "lbm_batch_destroy": (c_int, [c_void_p]),
    "lbm_batch_last_error": (c_char_p, [c_void_p]),
    "lbm_destroy": (c_int, [c_void_p]),
    "lbm_last_error": (c_char_p, [c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load_library(build: bool = True):
    """Load liblbm.so, compiling it first when missing or stale (build=True)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not found at {path}; build it with "
                           "__graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(lib, status: int, ctx) -> None:
    if status != LBM_OK:
        msg = lib.lbm_last_error(ctx)
        raise LbmError(status, msg.decode() if msg else "")


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(c_void_p)


def make_params(rho_l, rho_g, nu_l, nu_g, mobility, D, sigma, g=(0.0, 0.0, 0.0), A=0.25,
                sf=(1.0, 1.25, 1.25, 1.25, 1.2, 1.0, 1.0), sg=(1.0,) * 15, buoyancy=False,
                storage=LBM_STORAGE_FP32, pattern=LBM_PATTERN_AB, srt_flow=False,
                stencil="d3q15") -> LbmParams:
    p = LbmParams()
    p.rho_l, p.rho_g, p.nu_l, p.nu_g = rho_l, rho_g, nu_l, nu_g
    p.mobility, p.D, p.sigma, p.A = mobility, D, sigma, A
    p.g[:] = [float(v) for v in g]
    p.sf[:] = [float(v) for v in sf]
    p.sg[:] = [float(v) for v in sg]
    p.flags = ((LBM_FLAG_BUOYANCY if buoyancy else 0) | (LBM_FLAG_SRT_FLOW if srt_flow else 0)
               | (LBM_FLAG_D3Q7_STENCIL if stencil == "d3q7" else 0))
    p.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
    p.pattern = PATTERNS[pattern] if isinstance(pattern, str) else int(pattern)
    return p


def params_from_workload(w, pattern=LBM_PATTERN_AB, storage=LBM_STORAGE_FP32) -> tuple:
    grid = LbmGrid(w.nx, w.ny, w.nz, 1 if w.walls_z else 0)
    params = make_params(w.rho_l, w.rho_g, w.nu_l, w.nu_g, w.mobility, w.D, w.sigma, w.g, w.A,
                         w.sf, w.sg, w.buoyancy, pattern=pattern, storage=storage,
                         srt_flow=getattr(w, "srt_flow", False),
                         stencil=getattr(w, "stencil", "d3q15"))
    return grid, params


class _TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self, stream_handle: int):
        import torch
        self._torch = torch
        self._stream = int(stream_handle)

        def _alloc(nbytes, user):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), stream=self._stream)
            except Exception:  # out of memory: the library reports LBM_ENOMEM
                return None

        def _free(ptr, user):
            self._torch.cuda.caching_allocator_delete(ptr)

        self._alloc = ALLOC_FN(_alloc)
        self._free = FREE_FN(_free)
        self.struct = LbmAllocator(self._alloc, self._free, None)


# --------------------------------------------------------------------------------
# The C entry points, one to one.
# --------------------------------------------------------------------------------

class Context:
    """Handle of an lbm_ctx plus the Python objects that must outlive it."""

    def __init__(self, handle: c_void_p, n: int, shape, allocator=None, stream: int = 0):
        self.handle = handle
        self.n = n
        self.shape = shape
        self.stream = stream  # the cudaStream_t (as int) the context's work runs on
        self._allocator = allocator

    @property
    def value(self):
        return self.handle.value


def lbm_create(grid: LbmGrid, params: LbmParams, stream: Optional[int] = None,
               allocator: str = "torch") -> Context:
    """lbm_create.  stream: a cudaStream_t as int (None: PyTorch's current stream).
    allocator: "torch" (caching allocator) or "cuda" (cudaMalloc inside the library)."""
    lib = load_library()
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: this solver runs only on the GPU")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    alloc = _TorchAllocator(stream) if allocator == "torch" else None
    out = c_void_p()
    st = lib.lbm_create(ctypes.byref(grid), ctypes.byref(params),
                        ctypes.byref(alloc.struct) if alloc else None, c_void_p(stream),
                        ctypes.byref(out))
    _check(lib, st, None)
    n = grid.nx * grid.ny * grid.nz
    return Context(out, n, (grid.nz, grid.ny, grid.nx), alloc, int(stream))


def lbm_init_phi(ctx: Context, phi, u=None, p=None) -> None:
    lib = load_library()
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
    u = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    p = None if p is None else np.ascontiguousarray(p, dtype=np.float64).reshape(-1)
    if phi.size != ctx.n or (u is not None and u.size != 3 * ctx.n) or (p is not None and p.size != ctx.n):
        raise ValueError("field sizes do not match the grid")
    _check(lib, lib.lbm_init_phi(ctx.handle, _ptr(phi), _ptr(u), _ptr(p)), ctx.handle)


def lbm_step(ctx: Context, n: int = 1) -> None:
    lib = load_library()
    _check(lib, lib.lbm_step(ctx.handle, int(n)), ctx.handle)


def lbm_read_fields(ctx: Context, mask: int = LBM_FIELD_ALL, out: Optional[dict] = None) -> dict:
    """Returns a dict of float64 arrays shaped [z, y, x] (u: [3, z, y, x]).  `out` may
    hold preallocated float64 arrays (e.g. page-locked) for the selected fields."""
    lib = load_library()
    given = out or {}
    out = {}
    bufs = {}
    for name, bit, comps in (("phi", LBM_FIELD_PHI, 1), ("rho", LBM_FIELD_RHO, 1),
                             ("p", LBM_FIELD_P, 1), ("u", LBM_FIELD_U, 3), ("mu", LBM_FIELD_MU, 1)):
        if not mask & bit:
            bufs[name] = None
        elif name in given:
            a = given[name]
            if a.dtype != np.float64 or a.size != comps * ctx.n or not a.flags.c_contiguous:
                raise ValueError(f"out[{name!r}] must be a contiguous float64 array of "
                                 f"{comps * ctx.n} values")
            bufs[name] = a.reshape(-1)
        else:
            bufs[name] = np.empty(comps * ctx.n)
    _check(lib, lib.lbm_read_fields(ctx.handle, mask, _ptr(bufs["phi"]), _ptr(bufs["rho"]),
                                    _ptr(bufs["p"]), _ptr(bufs["u"]), _ptr(bufs["mu"])), ctx.handle)
    for name, a in bufs.items():
        if a is not None:
            out[name] = a.reshape((3,) + ctx.shape) if name == "u" else a.reshape(ctx.shape)
    return out


def lbm_reduce(ctx: Context, check: bool = True):
    """Returns (sum_phi, momentum[3]).  With check=False an LBM_EUNSTABLE status is
    returned as a third element instead of raised."""
    lib = load_library()
    s = c_double()
    mom = (c_double * 3)()
    st = lib.lbm_reduce(ctx.handle, ctypes.byref(s), mom)
    if check:
        _check(lib, st, ctx.handle)
        return s.value, np.array(mom[:])
    if st not in (LBM_OK, LBM_EUNSTABLE):
        _check(lib, st, ctx.handle)
    return s.value, np.array(mom[:]), st


def lbm_step_reduce(ctx: Context, n: int = 1, check: bool = True):
    """Advances n steps; returns (sum_phi, momentum[3]) of the new state (the last
    step's stream-collide pass computes them).  check=False: like lbm_reduce."""
    lib = load_library()
    s = c_double()
    mom = (c_double * 3)()
    st = lib.lbm_step_reduce(ctx.handle, int(n), ctypes.byref(s), mom)
    if check:
        _check(lib, st, ctx.handle)
        return s.value, np.array(mom[:])
    if st not in (LBM_OK, LBM_EUNSTABLE):
        _check(lib, st, ctx.handle)
    return s.value, np.array(mom[:]), st


def lbm_step_reduce_async(ctx: Context, n: int, out_dev: int) -> None:
    """Advances n steps and enqueues the sums of the new state into 5 doubles at device
    address out_dev.  No synchronisation."""
    lib = load_library()
    _check(lib, lib.lbm_step_reduce_async(ctx.handle, int(n), c_void_p(out_dev)), ctx.handle)


def lbm_reduce_async(ctx: Context, out_dev: int) -> None:
    """Enqueues the FP64 sums into 5 doubles at device address out_dev: sum phi,
    momentum x, y, z, count of non-finite cells.  No synchronisation."""
    lib = load_library()
    _check(lib, lib.lbm_reduce_async(ctx.handle, c_void_p(out_dev)), ctx.handle)


def lbm_read_state(ctx: Context):
    """Returns (f[7, z, y, x], g[15, z, y, x], phiu_prev[3, z, y, x], step), float32."""
    lib = load_library()
    f = np.empty((7,) + ctx.shape, np.float32)
    g = np.empty((15,) + ctx.shape, np.float32)
    phiu = np.empty((3,) + ctx.shape, np.float32)
    step = c_longlong()
    _check(lib, lib.lbm_read_state(ctx.handle, _ptr(f), _ptr(g), _ptr(phiu), ctypes.byref(step)),
           ctx.handle)
    return f, g, phiu, step.value


def lbm_read_state_at(ctx: Context, cells):
    """The state of lbm_read_state at listed cells only: cells is a sequence of linear
    indices x + nx (y + ny z) or of (z, y, x) triples.  Returns (f[7, k], g[15, k],
    phiu_prev[3, k], step), float32."""
    lib = load_library()
    c = np.asarray(cells, dtype=np.int64)
    if c.ndim == 2:
        nz, ny, nx = ctx.shape
        c = (c[:, 0] * ny + c[:, 1]) * nx + c[:, 2]
    c = np.ascontiguousarray(c.reshape(-1), dtype=np.int64)
    k = c.size
    f = np.empty((7, k), np.float32)
    g = np.empty((15, k), np.float32)
    phiu = np.empty((3, k), np.float32)
    step = c_longlong()
    _check(lib, lib.lbm_read_state_at(ctx.handle, _ptr(c), k, _ptr(f), _ptr(g), _ptr(phiu),
                                      ctypes.byref(step)), ctx.handle)
    return f, g, phiu, step.value


def lbm_write_state(ctx: Context, f, g, phiu_prev=None, step: int = 0) -> None:
    lib = load_library()
    f = np.ascontiguousarray(f, dtype=np.float32)
    g = np.ascontiguousarray(g, dtype=np.float32)
    phiu = None if phiu_prev is None else np.ascontiguousarray(phiu_prev, dtype=np.float32)
    if f.size != 7 * ctx.n or g.size != 15 * ctx.n or (phiu is not None and phiu.size != 3 * ctx.n):
        raise ValueError("state sizes do not match the grid")
    _check(lib, lib.lbm_write_state(ctx.handle, _ptr(f), _ptr(g), _ptr(phiu), int(step)), ctx.handle)


def lbm_set_velocity(ctx: Context, kind, U: float = 0.0, period: float = 1.0) -> None:
    """Interface-tracking mode: kind "uniform", "rotation", "deformation" (or the C
    constants); call before lbm_init_phi."""
    lib = load_library()
    k = VELOCITY_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib, lib.lbm_set_velocity(ctx.handle, k, float(U), float(period)), ctx.handle)


def lbm_set_tuning(ctx: Context, param: int, value: int) -> None:
    lib = load_library()
    _check(lib, lib.lbm_set_tuning(ctx.handle, int(param), int(value)), ctx.handle)


def lbm_get_tuning(ctx: Context, param: int) -> int:
    lib = load_library()
    v = c_int()
    _check(lib, lib.lbm_get_tuning(ctx.handle, int(param), ctypes.byref(v)), ctx.handle)
    return v.value


def lbm_get_step(ctx: Context) -> int:
    lib = load_library()
    s = c_longlong()
    _check(lib, lib.lbm_get_step(ctx.handle, ctypes.byref(s)), ctx.handle)
    return s.value


def lbm_profile(ctx: Context, enable: bool) -> None:
    lib = load_library()
    _check(lib, lib.lbm_profile(ctx.handle, 1 if enable else 0), ctx.handle)


def lbm_profile_read(ctx: Context, kernel: int):
    """Returns (total_ms, launches) of kernel 0 (k_phi), 1 (k_mu) or 2 (k_collide)."""
    lib = load_library()
    ms = c_double()
    n = c_longlong()
    _check(lib, lib.lbm_profile_read(ctx.handle, kernel, ctypes.byref(ms), ctypes.byref(n)),
           ctx.handle)
    return ms.value, n.value


def lbm_field_sum_noalloc(field_ptr: int, n: int, out_ptr: int, stream: Optional[int] = None) -> None:
    """lbm_field_sum_noalloc on device pointers (e.g. torch tensors' data_ptr())."""
    lib = load_library()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib, lib.lbm_field_sum_noalloc(c_void_p(field_ptr), int(n), c_void_p(out_ptr),
                                          c_void_p(stream)), None)


def lbm_memory_bytes(grid: LbmGrid, params: LbmParams) -> int:
    """Device bytes lbm_create would allocate (no GPU needed)."""
    lib = load_library()
    out = c_size_t()
    _check(lib, lib.lbm_memory_bytes(ctypes.byref(grid), ctypes.byref(params), ctypes.byref(out)),
           None)
    return out.value


class Batch:
    """lbm_batch: advances many contexts together (one launch per pass for all)."""

    def __init__(self, stream: Optional[int] = None, allocator: str = "torch"):
        lib = load_library()
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._alloc = _TorchAllocator(stream) if allocator == "torch" else None
        out = c_void_p()
        st = lib.lbm_batch_create(ctypes.byref(self._alloc.struct) if self._alloc else None,
                                  c_void_p(stream), ctypes.byref(out))
        _check(lib, st, None)
        self.handle = out
        self.lib = lib

    def _check(self, st):
        if st != LBM_OK:
            msg = self.lib.lbm_batch_last_error(self.handle)
            raise LbmError(st, msg.decode() if msg else "")

    def step(self, contexts, steps: int) -> None:
        """lbm_batch_step over the given Contexts (or Solvers)."""
        handles = [(c.ctx if hasattr(c, "ctx") else c).handle.value for c in contexts]
        arr = (c_void_p * len(handles))(*handles)
        self._check(self.lib.lbm_batch_step(self.handle, arr, len(handles), int(steps)))

    def set_grid(self, pass_index: int, blocks: int) -> None:
        self._check(self.lib.lbm_batch_set_grid(self.handle, int(pass_index), int(blocks)))

    def get_grid(self, pass_index: int) -> int:
        v = c_int()
        self._check(self.lib.lbm_batch_get_grid(self.handle, int(pass_index), ctypes.byref(v)))
        return v.value

    def set_split(self, cells: int) -> None:
        """Runs of at least `cells` cells take their own launches (0: none do)."""
        self._check(self.lib.lbm_batch_set_split(self.handle, int(cells)))

    def get_split(self) -> int:
        v = c_longlong()
        self._check(self.lib.lbm_batch_get_split(self.handle, ctypes.byref(v)))
        return v.value

    def set_prefetch(self, pass_index: int, items: int) -> None:
        self._check(self.lib.lbm_batch_set_prefetch(self.handle, int(pass_index), int(items)))

    def get_prefetch(self, pass_index: int) -> int:
        v = c_int()
        self._check(self.lib.lbm_batch_get_prefetch(self.handle, int(pass_index), ctypes.byref(v)))
        return v.value

    def close(self) -> None:
        if self.handle is not None and self.handle.value is not None:
            self.lib.lbm_batch_destroy(self.handle)
            self.handle = c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_destroy(ctx: Context) -> None:
    if ctx.handle is None or ctx.handle.value is None:
        return
    lib = load_library()
    st = lib.lbm_destroy(ctx.handle)
    ctx.handle = c_void_p()
    _check(lib, st, None)


def lbm_last_error(ctx: Optional[Context] = None) -> str:
    lib = load_library()
    msg = lib.lbm_last_error(ctx.handle if ctx else None)
    return msg.decode() if msg else ""


# --------------------------------------------------------------------------------
# Convenience wrapper.
# --------------------------------------------------------------------------------

class Solver:
    """One simulation: create from a workload, initialise, step, read."""

    def __init__(self, workload, stream: Optional[int] = None, allocator: str = "torch",
                 init: bool = True, pattern=LBM_PATTERN_AB, storage=LBM_STORAGE_FP32):
        self.workload = workload
        grid, params = params_from_workload(workload, pattern, storage)
        self.ctx = lbm_create(grid, params, stream=stream, allocator=allocator)
        v = getattr(workload, "velocity", None)
        if v is not None:
            lbm_set_velocity(self.ctx, v[0], v[1], v[2] if len(v) > 2 else 1.0)
        if init:
            lbm_init_phi(self.ctx, workload.phi0, workload.u0, workload.p0)

    def step(self, n: int = 1):
        lbm_step(self.ctx, n)

    def fields(self, mask: int = LBM_FIELD_ALL) -> dict:
        return lbm_read_fields(self.ctx, mask)

    def reduce(self):
        return lbm_reduce(self.ctx)

    def state(self):
        return lbm_read_state(self.ctx)

    def state_at(self, cells):
        return lbm_read_state_at(self.ctx, cells)

    def set_state(self, f, g, phiu_prev=None, step=0):
        lbm_write_state(self.ctx, f, g, phiu_prev, step)

    @property
    def t(self) -> int:
        return lbm_get_step(self.ctx)

    def close(self):
        lbm_destroy(self.ctx)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
