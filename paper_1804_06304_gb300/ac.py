"""Thin ctypes binding of libac (include/ac.h), with the C ABI's names.

Argument marshalling only: every step of the method runs in the CUDA library.
``load()`` builds (if stale) and loads ``libac.so``; when the library cannot be
built or loaded it fails loudly -- there is no CPU path.  With the environment
variable ``AC_BUILD=checked`` the bounds-checked build is loaded instead.  Arrays
may be numpy (host) or torch tensors (host or CUDA).
"""
from __future__ import annotations

import ctypes as ct
import dataclasses
import math
import os
import re

import numpy as np

from . import build as _build

AC_OK, AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA, AC_ERR_STATE, AC_ERR_TIMEOUT, AC_ERR_BUDGET, AC_ERR_NUMERIC = range(8)
AC_U8, AC_U16, AC_F16, AC_F32 = range(4)
AC_PATH_BRICK, AC_PATH_PLAIN, AC_PATH_GRID = 0, 1, 2
STATUS_NAMES = {0: "AC_OK", 1: "AC_ERR_ARG", 2: "AC_ERR_OOM", 3: "AC_ERR_CUDA", 4: "AC_ERR_STATE",
                5: "AC_ERR_TIMEOUT", 6: "AC_ERR_BUDGET", 7: "AC_ERR_NUMERIC"}


class ACError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ac_seed_params(ct.Structure):
    _fields_ = [("stride", ct.c_double), ("R0", ct.c_double)]


class ac_evolve_params(ct.Structure):
    _fields_ = [("N", ct.c_int32), ("T", ct.c_int32), ("eps0", ct.c_float), ("dR", ct.c_float),
                ("Rmin", ct.c_float), ("Rmax", ct.c_float), ("max_step", ct.c_float), ("seed", ct.c_uint64),
                ("stream_id", ct.c_uint32), ("path", ct.c_int32), ("lanes_per_contour", ct.c_int32),
                ("compensated", ct.c_int32), ("brick", ct.c_int32 * 3), ("warps_per_block", ct.c_int32),
                ("first_iter", ct.c_int32), ("update_last", ct.c_int32), ("sampling", ct.c_int32),
                ("halo_factor", ct.c_float), ("freeze_tol", ct.c_float), ("freeze_iters", ct.c_int32),
                ("cull_iter", ct.c_int32), ("cull_E", ct.c_float)]


class ac_trace(ct.Structure):
    _fields_ = [("device_buf", ct.c_void_p), ("k_begin", ct.c_int64), ("k_end", ct.c_int64),
                ("t_begin", ct.c_int32), ("t_end", ct.c_int32)]


class ac_batch_item(ct.Structure):
    _fields_ = [("stream_id", ct.c_uint32), ("first_iter", ct.c_int32), ("n_iter", ct.c_int32),
                ("update_last", ct.c_int32)]


class ac_layout(ct.Structure):
    _fields_ = [("lanes_per_contour", ct.c_int32), ("warps_per_block", ct.c_int32), ("brick", ct.c_int32 * 3),
                ("halo", ct.c_int32 * 3), ("region", ct.c_int32 * 3), ("smem_bytes", ct.c_int32)]


class ac_localize_params(ct.Structure):
    _fields_ = [("E0", ct.c_float)]


class ac_cell(ct.Structure):
    _fields_ = [("c", ct.c_float * 3), ("r", ct.c_float), ("E", ct.c_float), ("id", ct.c_int32)]


CELL_DTYPE = np.dtype([("c", np.float32, 3), ("r", np.float32), ("E", np.float32), ("id", np.int32)])


class ac_server_params(ct.Structure):
    _fields_ = [("evolve", ac_evolve_params), ("dtype", ct.c_int32), ("ndim", ct.c_int32), ("stride", ct.c_float),
                ("R0", ct.c_float), ("E0", ct.c_float), ("iters_per_round", ct.c_int32),
                ("max_resident", ct.c_int32), ("hbm_budget_bytes", ct.c_int64),
                ("max_resident_contours", ct.c_int64), ("balance_rounds", ct.c_int32), ("reserved_", ct.c_int32)]


class ac_tile_result(ct.Structure):
    _fields_ = [("ticket", ct.c_int64), ("status", ct.c_int32), ("rounds", ct.c_int32), ("n_cells", ct.c_int64),
                ("contours", ct.c_int64), ("voxels", ct.c_int64), ("est_bytes", ct.c_int64),
                ("queue_ms", ct.c_double), ("run_ms", ct.c_double), ("total_ms", ct.c_double)]


class ac_server_stats(ct.Structure):
    _fields_ = [("pending", ct.c_int64), ("resident", ct.c_int64), ("finished", ct.c_int64),
                ("completed", ct.c_int64), ("failed", ct.c_int64), ("rounds", ct.c_int64),
                ("resident_bytes", ct.c_int64), ("peak_resident_bytes", ct.c_int64), ("budget_bytes", ct.c_int64)]

_SIGS = {
    "ac_create_volume": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_int64), ct.c_int64,
                                    ct.c_int64, ct.POINTER(ct.c_float), ct.c_float, ct.c_void_p,
                                    ct.POINTER(ct.c_void_p)]),
    "ac_destroy_volume": (None, [ct.c_void_p]),
    "ac_load_volume": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_int64, ct.c_int64, ct.c_void_p]),
    "ac_reseed": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "ac_seed": (ct.c_int, [ct.c_void_p, ct.POINTER(ac_seed_params), ct.c_void_p, ct.c_int64, ct.c_void_p,
                           ct.POINTER(ct.c_void_p)]),
    "ac_contour_count": (ct.c_int64, [ct.c_void_p]),
    "ac_destroy_contours": (None, [ct.c_void_p]),
    "ac_evolve": (ct.c_int, [ct.c_void_p, ct.POINTER(ac_evolve_params), ct.POINTER(ac_trace), ct.c_void_p]),
    "ac_evolve_batch": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.POINTER(ac_batch_item), ct.c_int32,
                                   ct.POINTER(ac_evolve_params), ct.c_void_p]),
    "ac_localize": (ct.c_int, [ct.c_void_p, ct.POINTER(ac_localize_params), ct.c_void_p, ct.c_int64,
                               ct.POINTER(ct.c_int64), ct.c_void_p]),
    "ac_localize_batch": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int32, ct.POINTER(ac_localize_params),
                                     ct.POINTER(ct.c_void_p), ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64),
                                     ct.c_void_p]),
    "ac_get_state": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "ac_set_state": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "ac_state_device_ptr": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "ac_philox4x32_10": (ct.c_int, [ct.c_void_p, ct.c_uint64, ct.c_void_p, ct.c_int64, ct.c_void_p]),
    "ac_evolve_kernel_ms": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_float)]),
    "ac_kernel_launches": (ct.c_int64, []),
    "ac_evolve_stats": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int64), ct.c_void_p]),
    "ac_evolve_stops": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int64), ct.c_void_p]),
    "ac_evolve_static": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.POINTER(ct.c_int64), ct.c_int64, ct.c_int64,
                                    ct.POINTER(ct.c_float), ct.c_float, ct.c_void_p, ct.c_int64, ct.c_float,
                                    ct.c_float, ct.POINTER(ac_evolve_params), ct.c_void_p]),
    "ac_plan_layout": (ct.c_int, [ct.c_int32, ct.c_int, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_float), ct.c_double,
                                  ct.c_double, ct.POINTER(ac_evolve_params), ct.POINTER(ac_layout)]),
    "ac_plan_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.POINTER(ac_batch_item), ct.c_int32,
                                  ct.POINTER(ac_evolve_params), ct.POINTER(ct.c_void_p)]),
    "ac_plan_rebind": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_void_p), ct.POINTER(ac_batch_item), ct.c_int32,
                                  ct.c_void_p]),
    "ac_plan_set_items": (ct.c_int, [ct.c_void_p, ct.POINTER(ac_batch_item), ct.c_void_p]),
    "ac_plan_launch": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p]),
    "ac_destroy_plan": (None, [ct.c_void_p]),
    "ac_autotune": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int32, ct.POINTER(ac_evolve_params), ct.c_void_p]),
    "ac_last_error": (ct.c_char_p, []),
    "ac_set_wait_limits": (ct.c_int, [ct.c_int64, ct.c_int64]),
    "ac_server_create": (ct.c_int, [ct.POINTER(ac_server_params), ct.POINTER(ct.c_void_p)]),
    "ac_server_submit": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_int64), ct.c_int64, ct.c_int64,
                                    ct.POINTER(ct.c_float), ct.c_float, ct.c_uint32, ct.POINTER(ct.c_int64)]),
    "ac_server_submit_traced": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_int64), ct.c_int64, ct.c_int64,
                                           ct.POINTER(ct.c_float), ct.c_float, ct.c_uint32, ct.POINTER(ac_trace),
                                           ct.POINTER(ct.c_int64)]),
    "ac_server_wait": (ct.c_int, [ct.c_void_p, ct.c_int64, ct.c_double, ct.c_void_p, ct.c_int64,
                                  ct.POINTER(ac_tile_result)]),
    "ac_server_get_stats": (ct.c_int, [ct.c_void_p, ct.POINTER(ac_server_stats)]),
    "ac_server_destroy": (None, [ct.c_void_p]),
}

_lib = None


def _checked() -> bool:
    v = os.environ.get("AC_BUILD", "")
    if v not in ("", "checked"):
        raise ACError(AC_ERR_ARG, f"AC_BUILD must be unset or 'checked', not {v!r}")
    return v == "checked"


def lib_path() -> str:
    return _build.lib_path(_checked())


def load():
    """Build (if stale) and load libac.so; raises if either fails."""
    global _lib
    if _lib is None:
        path = _build.build(checked=_checked())
        l = ct.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


def header_symbols() -> list:
    """Entry points declared in include/*.h."""
    inc = os.path.join(os.path.dirname(_build.HERE), "include")
    h = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    return sorted(set(re.findall(r"\b(ac_[a-z0-9_]+)\s*\(", h)))


def _check(status: int):
    if status != AC_OK:
        raise ACError(status, load().ac_last_error().decode())


def _stream(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def _ptr(arr):
    """(pointer, on_device, dtype code, shape, element strides) of numpy / torch data."""
    try:
        import torch
        if isinstance(arr, torch.Tensor):
            code = {torch.uint8: AC_U8, torch.int16: AC_U16, torch.float16: AC_F16, torch.float32: AC_F32}
            if hasattr(torch, "uint16"):
                code[torch.uint16] = AC_U16
            return arr.data_ptr(), int(arr.is_cuda), code.get(arr.dtype), tuple(arr.shape), tuple(arr.stride())
    except ImportError:
        pass
    a = np.asarray(arr)
    code = {np.dtype(np.uint8): AC_U8, np.dtype(np.uint16): AC_U16, np.dtype(np.float16): AC_F16,
            np.dtype(np.float32): AC_F32}.get(a.dtype)
    return a.ctypes.data, 0, code, a.shape, tuple(s // a.itemsize for s in a.strides)


# ------------------------------------------------------------------------ handles
class Volume:
    def __init__(self, handle, ndim, dims, spacing, keepalive=None):
        self.handle = handle
        self.ndim = ndim
        self.dims = dims
        self.spacing = spacing
        self._keep = keepalive

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ac_destroy_volume(self.handle)
            self.handle = None


class Contours:
    def __init__(self, handle, vol: Volume):
        self.handle = handle
        self.vol = vol

    @property
    def count(self) -> int:
        return int(load().ac_contour_count(self.handle))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ac_destroy_contours(self.handle)
            self.handle = None


# ------------------------------------------------------------------------ entry points
def ac_create_volume(data, spacing=(1.0, 1.0, 1.0), intensity_scale: float = 1.0, stream=None,
                     dtype: int | None = None) -> Volume:
    """``data`` indexed [z, y, x] (3D) or [y, x] (2D), x fastest."""
    l = load()
    ptr, on_dev, code, shape, strides = _ptr(data)
    if dtype is not None:
        code = dtype
    if code is None:
        raise ACError(AC_ERR_ARG, "unsupported element type")
    ndim = len(shape)
    if ndim not in (2, 3) or strides[-1] != 1:
        raise ACError(AC_ERR_ARG, "need a 2D or 3D array with unit x stride")
    dims = (ct.c_int64 * 3)(*(list(shape[::-1]) + [1] * (3 - ndim)))
    row = strides[-2]
    plane = strides[-3] if ndim == 3 else 0
    sp = (ct.c_float * 3)(*[float(s) for s in (list(spacing) + [1.0] * 3)[:3]])
    out = ct.c_void_p()
    _check(l.ac_create_volume(ct.c_void_p(ptr), on_dev, code, ndim, dims, row, plane, sp, intensity_scale,
                              ct.c_void_p(_stream(stream)), ct.byref(out)))
    return Volume(out, ndim, tuple(dims), tuple(sp), keepalive=data)


def ac_load_volume(vol: Volume, data, stream=None):
    """New voxels (same extents and type) into an existing volume."""
    ptr, on_dev, code, shape, strides = _ptr(data)
    if tuple(shape[::-1]) != tuple(vol.dims[:len(shape)]):
        raise ACError(AC_ERR_ARG, "extents differ from the volume's")
    row = strides[-2]
    plane = strides[-3] if len(shape) == 3 else 0
    _check(load().ac_load_volume(vol.handle, ct.c_void_p(ptr), on_dev, row, plane, ct.c_void_p(_stream(stream))))
    vol._keep = data


def ac_reseed(ctr: Contours, stream=None):
    _check(load().ac_reseed(ctr.handle, ct.c_void_p(_stream(stream))))


def ac_destroy_volume(vol: Volume):
    if vol.handle:
        load().ac_destroy_volume(vol.handle)
        vol.handle = None


def ac_seed(vol: Volume, stride: float | None = None, R0: float = 0.0, explicit=None, stream=None) -> Contours:
    l = load()
    p = ac_seed_params(float(stride or 0.0), float(R0))
    out = ct.c_void_p()
    if explicit is not None:
        e = np.ascontiguousarray(explicit, dtype=np.float32).reshape(-1, 4)
        buf = e if len(e) else np.zeros((1, 4), np.float32)   # a valid pointer for an empty set
        _check(l.ac_seed(vol.handle, ct.byref(p), ct.c_void_p(buf.ctypes.data), len(e), ct.c_void_p(_stream(stream)),
                         ct.byref(out)))
    else:
        _check(l.ac_seed(vol.handle, ct.byref(p), None, 0, ct.c_void_p(_stream(stream)), ct.byref(out)))
    return Contours(out, vol)


def ac_contour_count(ctr: Contours) -> int:
    return int(load().ac_contour_count(ctr.handle))


def ac_destroy_contours(ctr: Contours):
    if ctr.handle:
        load().ac_destroy_contours(ctr.handle)
        ctr.handle = None


@dataclasses.dataclass
class EvolveParams:
    N: int
    T: int
    eps0: float
    dR: float = 1.0
    Rmin: float = 0.5
    Rmax: float = 1e6
    max_step: float = 0.5
    seed: int = 0
    stream_id: int = 0
    path: int = AC_PATH_BRICK
    lanes_per_contour: int = 0
    compensated: int = 1
    brick: tuple = (0, 0, 0)
    warps_per_block: int = 0
    first_iter: int = 0
    update_last: int = 0
    sampling: int = 0
    halo_factor: float = 0.0
    freeze_tol: float = 0.0
    freeze_iters: int = 0
    cull_iter: int = 0
    cull_E: float = 0.0

    def to_c(self) -> ac_evolve_params:
        p = ac_evolve_params()
        for f in dataclasses.fields(self):
            if f.name == "brick":
                p.brick[:] = tuple(int(b) for b in self.brick)
            else:
                setattr(p, f.name, getattr(self, f.name))
        return p


def default_params(ndim: int, R0: float, contrast: float, N: int, T: int, seed: int = 0, **kw) -> EvolveParams:
    """Defaults for the values the paper leaves open: eps0 = 8 R0^2 / A (A = the
    expected foreground-background contrast in scaled intensity), dR = 1,
    Rmin = max(dR/2, R0/2), Rmax = 3 R0, max_step = 0.5."""
    dR = kw.pop("dR", 1.0)
    base = dict(eps0=8.0 * R0 * R0 / contrast, dR=dR, Rmin=max(0.5 * dR, 0.5 * R0), Rmax=3.0 * R0)
    base.update(kw)   # explicit values win
    return EvolveParams(N=N, T=T, seed=seed, **base)


def default_E0(ndim: int, contrast: float) -> float:
    """A quarter of the ideal-blob minimum energy (-A pi/12 in 3D, -A pi/8 in 2D):
    real nuclei (blurred, elongated, dimmer than the typical contrast A) reach
    only part of the ideal minimum."""
    return -math.pi * contrast / 48.0 if ndim == 3 else -math.pi * contrast / 32.0


def ac_evolve(ctr: Contours, params: EvolveParams, trace=None, stream=None):
    """``trace``: None or (device tensor, k_begin, k_end, t_begin, t_end)."""
    l = load()
    p = params.to_c()
    tr = None
    if trace is not None:
        buf, k0, k1, t0, t1 = trace
        need = (t1 - t0) * (k1 - k0) * 9
        if buf.numel() < need or not buf.is_cuda or buf.dtype.itemsize != 4:
            raise ACError(AC_ERR_ARG, "trace buffer too small or not a float32 CUDA tensor")
        tr = ac_trace(buf.data_ptr(), k0, k1, t0, t1)
    _check(l.ac_evolve(ctr.handle, ct.byref(p), ct.byref(tr) if tr is not None else None,
                       ct.c_void_p(_stream(stream))))


def _handles(sets):
    return (ct.c_void_p * len(sets))(*[s.handle.value if isinstance(s.handle, ct.c_void_p) else s.handle for s in sets])


def _items(items, n):
    if items is None:
        return None
    arr = (ac_batch_item * n)()
    for i, it in enumerate(items):
        arr[i].stream_id, arr[i].first_iter, arr[i].n_iter, arr[i].update_last = (int(v) for v in it)
    return arr


def ac_evolve_batch(sets, params: EvolveParams, items=None, stream=None):
    """One launch over several contour sets.  ``items``: None or per set
    (stream_id, first_iter, n_iter, update_last); the Philox key is params.seed."""
    p = params.to_c()
    _check(load().ac_evolve_batch(_handles(sets), _items(items, len(sets)), len(sets), ct.byref(p),
                                  ct.c_void_p(_stream(stream))))


class Plan:
    def __init__(self, handle, sets):
        self.handle = handle
        self.sets = list(sets)   # keep the contour sets alive

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ac_destroy_plan(self.handle)
            self.handle = None


def ac_plan_create(sets, params: EvolveParams, items=None) -> Plan:
    out = ct.c_void_p()
    p = params.to_c()
    _check(load().ac_plan_create(_handles(sets), _items(items, len(sets)), len(sets), ct.byref(p), ct.byref(out)))
    return Plan(out, sets)


def ac_plan_rebind(plan: Plan, sets, items=None, stream=None):
    """New contour sets (and items) for later launches of the plan."""
    _check(load().ac_plan_rebind(plan.handle, _handles(sets), _items(items, len(sets)), len(sets),
                                 ct.c_void_p(_stream(stream))))
    plan.sets = list(sets)


def ac_plan_set_items(plan: Plan, items, stream=None):
    _check(load().ac_plan_set_items(plan.handle, _items(items, len(plan.sets)), ct.c_void_p(_stream(stream))))


def ac_plan_launch(plan: Plan, use_graph: bool = True, stream=None):
    _check(load().ac_plan_launch(plan.handle, int(use_graph), ct.c_void_p(_stream(stream))))


def ac_destroy_plan(plan: Plan):
    if plan.handle:
        load().ac_destroy_plan(plan.handle)
        plan.handle = None


def ac_autotune(sets, params: EvolveParams, stream=None) -> EvolveParams:
    """Returns a copy of ``params`` with lanes_per_contour, brick and
    warps_per_block chosen by timed trials on copies of the sets' state."""
    p = params.to_c()
    _check(load().ac_autotune(_handles(sets), len(sets), ct.byref(p), ct.c_void_p(_stream(stream))))
    return dataclasses.replace(params, lanes_per_contour=int(p.lanes_per_contour),
                               warps_per_block=int(p.warps_per_block), brick=tuple(int(b) for b in p.brick))


def ac_localize(ctr: Contours, E0: float, cap: int | None = None, stream=None) -> np.ndarray:
    l = load()
    cap = ctr.count if cap is None else cap
    out = np.zeros(max(cap, 1), dtype=CELL_DTYPE)
    n = ct.c_int64()
    _check(l.ac_localize(ctr.handle, ct.byref(ac_localize_params(E0)), ct.c_void_p(out.ctypes.data), cap,
                         ct.byref(n), ct.c_void_p(_stream(stream))))
    return out[:min(n.value, cap)]


def ac_localize_batch(sets, E0, caps=None, stream=None) -> list:
    """ac_localize of several distinct contour sets in one call (one threshold for
    all, or one per set); returns one cell array per set."""
    l = load()
    n = len(sets)
    E0s = [float(E0)] * n if np.isscalar(E0) else [float(e) for e in E0]
    if len(E0s) != n:
        raise ValueError("ac_localize_batch: one E0 or one per set")
    caps = [c.count for c in sets] if caps is None else [int(c) for c in caps]
    outs = [np.zeros(max(c, 1), dtype=CELL_DTYPE) for c in caps]
    handles = _handles(sets) if n else (ct.c_void_p * 1)()
    params = (ac_localize_params * max(n, 1))(*[ac_localize_params(e) for e in E0s])
    ptrs = (ct.c_void_p * max(n, 1))(*[o.ctypes.data for o in outs])
    capv = (ct.c_int64 * max(n, 1))(*caps)
    nout = (ct.c_int64 * max(n, 1))()
    _check(l.ac_localize_batch(handles, n, params, ptrs, capv, nout, ct.c_void_p(_stream(stream))))
    return [o[:min(nout[i], caps[i])] for i, o in enumerate(outs)]


def ac_get_state(ctr: Contours, stream=None) -> np.ndarray:
    """(5, C) float32: cx, cy, cz, R, E."""
    l = load()
    out = np.empty((5, ctr.count), dtype=np.float32)
    _check(l.ac_get_state(ctr.handle, ct.c_void_p(out.ctypes.data), ct.c_void_p(_stream(stream))))
    return out


def ac_set_state(ctr: Contours, state: np.ndarray, stream=None):
    l = load()
    s = np.ascontiguousarray(state, dtype=np.float32).reshape(5, -1)
    _check(l.ac_set_state(ctr.handle, ct.c_void_p(s.ctypes.data), ct.c_void_p(_stream(stream))))


def ac_state_device_ptr(ctr: Contours) -> int:
    out = ct.c_void_p()
    _check(load().ac_state_device_ptr(ctr.handle, ct.byref(out)))
    return out.value


def ac_philox4x32_10(ctr_dev, key: int, stream=None):
    """``ctr_dev``: CUDA int32/uint32 tensor of shape (n, 4); returns words likewise."""
    import torch
    out = torch.empty_like(ctr_dev)
    _check(load().ac_philox4x32_10(ct.c_void_p(ctr_dev.data_ptr()), key, ct.c_void_p(out.data_ptr()),
                                   ctr_dev.shape[0], ct.c_void_p(_stream(stream))))
    return out


def ac_evolve_kernel_ms(ctr: Contours) -> float:
    ms = ct.c_float()
    _check(load().ac_evolve_kernel_ms(ctr.handle, ct.byref(ms)))
    return float(ms.value)


def ac_evolve_stats(ctr: Contours, stream=None) -> tuple:
    """(fast, clamped, global) contour-iterations of the last evolution."""
    c = (ct.c_int64 * 3)()
    _check(load().ac_evolve_stats(ctr.handle, c, ct.c_void_p(_stream(stream))))
    return tuple(int(v) for v in c)


def ac_evolve_stops(ctr: Contours, stream=None) -> tuple:
    """(contours stopped by the step rule, by the energy rule) so far."""
    out = (ct.c_int64 * 2)()
    _check(load().ac_evolve_stops(ctr.handle, out, ct.c_void_p(_stream(stream))))
    return int(out[0]), int(out[1])


def ac_kernel_launches() -> int:
    return int(load().ac_kernel_launches())


def ac_plan_layout(ndim: int, dtype: int, dims, spacing, stride: float, r0: float, params: EvolveParams) -> dict:
    """The launch layout ac_evolve takes for one contour set (host logic; no GPU
    needed): dims and spacing are (x, y[, z]); returns lanes_per_contour,
    warps_per_block, brick, halo, region (voxels, x y z) and smem_bytes."""
    d = (ct.c_int64 * 3)(*(list(dims) + [1] * 3)[:3])
    sp = (ct.c_float * 3)(*[float(v) for v in (list(spacing) + [1.0] * 3)[:3]])
    out = ac_layout()
    p = params.to_c()
    _check(load().ac_plan_layout(int(ndim), int(dtype), d, sp, float(stride), float(r0), ct.byref(p), ct.byref(out)))
    return {"lanes_per_contour": out.lanes_per_contour, "warps_per_block": out.warps_per_block,
            "brick": tuple(out.brick), "halo": tuple(out.halo), "region": tuple(out.region),
            "smem_bytes": out.smem_bytes}


AC_STATIC_MAX_CONTOURS = 1 << 20


def ac_evolve_static(volume_dev, state_dev, params: EvolveParams, r0: float, stride: float,
                     spacing=(1.0, 1.0, 1.0), intensity_scale: float = 1.0, dtype: int | None = None,
                     n_contours: int | None = None, stream=None):
    """Allocation-free evolve for callers that own all device memory: ``volume_dev``
    (CUDA tensor, [z, y, x] or [y, x]) and ``state_dev`` (CUDA float32 tensor of
    shape (5, C), updated in place) belong to the caller; the library's temporaries
    live in its fixed device array.  Synchronizes the stream."""
    import torch
    if not (isinstance(volume_dev, torch.Tensor) and volume_dev.is_cuda):
        raise ACError(AC_ERR_ARG, "ac_evolve_static: volume_dev must be a CUDA tensor")
    if not (isinstance(state_dev, torch.Tensor) and state_dev.is_cuda and state_dev.dtype == torch.float32 and
            state_dev.dim() == 2 and state_dev.shape[0] == 5 and state_dev.is_contiguous()):
        raise ACError(AC_ERR_ARG, "ac_evolve_static: state_dev must be a contiguous CUDA float32 tensor of shape (5, C)")
    if volume_dev.device != state_dev.device:
        raise ACError(AC_ERR_ARG, "ac_evolve_static: volume_dev and state_dev must be on the same device")
    ptr, on_dev, code, shape, strides = _ptr(volume_dev)
    if dtype is not None:
        code = dtype
    ndim = len(shape)
    if ndim not in (2, 3) or strides[-1] != 1 or code is None:
        raise ACError(AC_ERR_ARG, "ac_evolve_static: volume_dev must be 2D or 3D with unit x stride and a "
                                  "uint8 / uint16 (int16) / float16 / float32 dtype")
    dims = (ct.c_int64 * 3)(*(list(shape[::-1]) + [1] * (3 - ndim)))
    sp = (ct.c_float * 3)(*[float(v) for v in (list(spacing) + [1.0] * 3)[:3]])
    C = int(state_dev.shape[1]) if n_contours is None else int(n_contours)
    if C < 1 or (C > int(state_dev.shape[1]) and C <= AC_STATIC_MAX_CONTOURS):
        raise ACError(AC_ERR_ARG, "ac_evolve_static: need 1 <= n_contours <= state_dev.shape[1]")
    p = params.to_c()
    _check(load().ac_evolve_static(ct.c_void_p(ptr), code, ndim, dims, strides[-2], strides[-3] if ndim == 3 else 0,
                                   sp, intensity_scale, ct.c_void_p(state_dev.data_ptr()), C, float(r0), float(stride),
                                   ct.byref(p), ct.c_void_p(_stream(stream))))


def ac_last_error() -> str:
    return load().ac_last_error().decode()


def ac_set_wait_limits(tma_polls: int = -1, localize_rounds: int = -1):
    """Lower the bounds of the device waits (testing): polls of the brick kernel's
    first wait for its TMA load and rounds of the overlap competition; -1 restores
    the defaults."""
    _check(load().ac_set_wait_limits(int(tma_polls), int(localize_rounds)))


# ------------------------------------------------------------------------ serving form
class Server:
    """Request loop over image tiles (include/ac_serve.h).  ``submit`` keeps a
    reference to each tile's array until its ticket is collected by ``wait``."""

    def __init__(self, params: EvolveParams, dtype: int, ndim: int, stride: float, E0: float,
                 hbm_budget_bytes: int, iters_per_round: int = 10, max_resident: int = 0, R0: float = 0.0,
                 max_resident_contours: int = 0, balance_rounds: bool = True):
        sp = ac_server_params()
        sp.evolve = params.to_c()
        sp.dtype, sp.ndim, sp.stride, sp.R0, sp.E0 = int(dtype), int(ndim), float(stride), float(R0), float(E0)
        sp.iters_per_round, sp.max_resident, sp.hbm_budget_bytes = int(iters_per_round), int(max_resident), \
            int(hbm_budget_bytes)
        sp.max_resident_contours = int(max_resident_contours)
        sp.balance_rounds = int(bool(balance_rounds))
        self.handle = None
        out = ct.c_void_p()
        _check(load().ac_server_create(ct.byref(sp), ct.byref(out)))
        self.handle = out
        self._arrays = {}
        self._caps = {}
        self.ndim, self.stride = int(ndim), float(stride)

    def submit(self, volume: np.ndarray, spacing=(1.0, 1.0, 1.0), intensity_scale: float = 1.0,
               stream_id: int = 0, trace=None) -> int:
        """``volume`` indexed [z, y, x] (3D) or [y, x] (2D), host memory, x fastest.
        ``trace`` = (device tensor, k0, k1, t0, t1) records the tile's evaluations as
        ac_evolve's trace does (ac_server_submit_traced)."""
        a = np.asarray(volume)
        ptr, _, _, shape, strides = _ptr(a)
        if strides[-1] != 1 or len(shape) not in (2, 3):
            raise ACError(AC_ERR_ARG, "need a 2D or 3D host array with unit x stride")
        dims = (ct.c_int64 * 3)(*(list(shape[::-1]) + [1] * (3 - len(shape))))
        sp = (ct.c_float * 3)(*[float(s) for s in (list(spacing) + [1.0] * 3)[:3]])
        t = ct.c_int64()
        tr = None
        if trace is not None:
            buf, k0, k1, t0, t1 = trace
            tr = ac_trace(ct.c_void_p(buf.data_ptr()), int(k0), int(k1), int(t0), int(t1))
        _check(load().ac_server_submit_traced(self.handle, ct.c_void_p(ptr), dims, strides[-2],
                                              strides[-3] if len(shape) == 3 else 0, sp, float(intensity_scale),
                                              int(stream_id), ct.byref(tr) if tr is not None else None,
                                              ct.byref(t)))
        self._arrays[t.value] = (a, trace)
        lattice = 1
        for d in range(self.ndim):   # ac_seed's lattice size bounds the number of cells
            lattice *= max(1, int(math.floor(dims[d] * sp[d] / self.stride)))
        self._caps[t.value] = lattice
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0, cap: int | None = None):
        """(cells, result dict) of a finished tile; raises ACError on the tile's
        error or (AC_ERR_TIMEOUT) when it is not finished within ``timeout`` s."""
        r = ac_tile_result()
        cap = self._caps.get(ticket, 1) if cap is None else cap
        out = np.zeros(max(cap, 1), dtype=CELL_DTYPE)
        st = load().ac_server_wait(self.handle, int(ticket), float(timeout), ct.c_void_p(out.ctypes.data), cap,
                                   ct.byref(r))
        if st != AC_ERR_TIMEOUT:
            self._arrays.pop(ticket, None)
            self._caps.pop(ticket, None)
        _check(st)
        res = {f: getattr(r, f) for f, _ in ac_tile_result._fields_}
        return out[:min(cap, r.n_cells)].copy(), res

    def stats(self) -> dict:
        s = ac_server_stats()
        _check(load().ac_server_get_stats(self.handle, ct.byref(s)))
        return {f: int(getattr(s, f)) for f, _ in ac_server_stats._fields_}

    def close(self):
        if self.handle:
            load().ac_server_destroy(self.handle)
            self.handle = None
            self._arrays.clear()

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ac_server_destroy(self.handle)
            self.handle = None
