"""ctypes wrapper around ``ac_oracle.c``, the plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  The C source follows the
paper's equations step by step (Eqs. 5-15, the Monte-Carlo Integration section and
the overlap competition of the Results section); see its header for the readings
taken where the paper is silent.  This module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ac_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

E, DEDP, DEDQ, DEDR, DEDC, MAG_E, MAG_R, MAG_C, FLAGS, SUM_SI, VAR_E, VAR_R, VAR_C, MAG_G, MAG_I, RES_LEN = (
    0, 1, 4, 7, 8, 11, 12, 13, 16, 17, 18, 19, 20, 23, 24, 25)
TRACE_LEN = 9
DTYPES = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float16): 2, np.dtype(np.float32): 3}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Image(ct.Structure):
    _fields_ = [
        ("data", ct.c_void_p), ("dtype", ct.c_int32), ("ndim", ct.c_int32),
        ("n", ct.c_int64 * 3), ("pitch", ct.c_int64 * 3), ("spacing", ct.c_double * 3),
        ("scale", ct.c_double), ("analytic", ct.c_int32), ("pad_", ct.c_int32),
        ("blob_c", ct.c_double * 3), ("blob_r", ct.c_double), ("blob_amp", ct.c_double),
        ("offset", ct.c_double), ("grad", ct.c_double * 3),
    ]


class Params(ct.Structure):
    _fields_ = [
        ("ndim", ct.c_int32), ("N", ct.c_int32), ("T", ct.c_int32), ("pad_", ct.c_int32),
        ("eps0", ct.c_double), ("dR", ct.c_double), ("Rmin", ct.c_double), ("Rmax", ct.c_double),
        ("max_step", ct.c_double), ("edge_tol", ct.c_double),
        ("key", ct.c_uint32 * 2), ("stream_id", ct.c_uint32), ("integration", ct.c_int32),
        ("freeze_tol", ct.c_double), ("freeze_iters", ct.c_int32), ("cull_iter", ct.c_int32),
        ("cull_E", ct.c_double),
    ]


def _P(a, t):
    return a.ctypes.data_as(ct.POINTER(t))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ct.CDLL(build())
            D, I64, U32 = ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64), ct.POINTER(ct.c_uint32)
            IP, PP = ct.POINTER(Image), ct.POINTER(Params)
            sig = {
                "or_philox4x32_10": (None, [U32, U32, U32]),
                "or_philox_batch": (None, [ct.c_int64, U32, U32, U32]),
                "or_uniform24": (ct.c_double, [ct.c_uint32]),
                "or_uniforms21": (None, [ct.c_uint32, ct.c_uint32, D]),
                "or_half_to_double": (ct.c_double, [ct.c_uint16]),
                "or_image_value": (ct.c_double, [IP, D]),
                "or_image_values": (None, [IP, ct.c_int64, D, D]),
                "or_rho": (ct.c_double, [ct.c_int]),
                "or_weight": (None, [ct.c_int, ct.c_double, ct.c_double, ct.c_double, D]),
                "or_weight_batch": (None, [ct.c_int, ct.c_int64, D, ct.c_double, ct.c_double, D]),
                "or_eval_pq": (None, [IP, PP, D, D, ct.c_int64, ct.c_int64, D]),
                "or_eval_cr": (None, [IP, PP, D, ct.c_double, ct.c_int64, ct.c_int64, D]),
                "or_energy_grid": (ct.c_double, [IP, ct.c_int, D, ct.c_double, ct.c_double]),
                "or_update_pq": (None, [IP, PP, ct.c_int64, D, D, D]),
                "or_evolve": (None, [IP, PP, ct.c_int64, I64, D, D, D, ct.POINTER(ct.c_int32),
                                     ct.POINTER(ct.c_int32), ct.c_int]),
                "or_eval_grid_pq": (None, [IP, PP, D, D, D]),
                "or_max_threads": (ct.c_int, []),
                "or_seed_lattice": (ct.c_int64, [ct.c_int, I64, D, ct.c_double, D]),
                "or_localize": (ct.c_int64, [ct.c_int, ct.c_int64, D, D, ct.c_double, I64]),
                "or_unit_samples": (None, [PP, ct.c_int64, ct.c_int64, D]),
                "or_eval_many": (None, [IP, PP, ct.c_int64, D, I64, I64, D, ct.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


# --------------------------------------------------------------------------- images
class VolumeImage:
    """A voxel volume as the oracle sees it.  ``arr`` is indexed [z, y, x] (3D) or
    [y, x] (2D), x fastest in memory."""

    def __init__(self, arr: np.ndarray, spacing=(1.0, 1.0, 1.0), scale: float = 1.0):
        arr = np.ascontiguousarray(arr)
        self.arr = arr
        s = Image()
        s.data = arr.ctypes.data
        s.dtype = DTYPES[arr.dtype]
        s.ndim = arr.ndim
        shape = arr.shape[::-1] + (1,) * (3 - arr.ndim)
        s.n[:] = shape
        s.pitch[:] = (1, shape[0], shape[0] * shape[1])
        s.spacing[:] = tuple(float(v) for v in spacing)
        s.scale = float(scale)
        s.analytic = 0
        self.s = s
        self.ndim = arr.ndim


class BlobImage:
    """Analytic image offset + grad.x + amp [|x - centre| < radius] (used by pins)."""

    def __init__(self, ndim, centre, radius, amp, offset=0.0, grad=(0.0, 0.0, 0.0), n=(1 << 20,) * 3):
        s = Image()
        s.ndim = ndim
        s.analytic = 1
        s.n[:] = n
        s.spacing[:] = (1.0, 1.0, 1.0)
        s.scale = 1.0
        s.blob_c[:] = tuple(float(v) for v in centre) + (0.0,) * (3 - len(centre))
        s.blob_r = float(radius)
        s.blob_amp = float(amp)
        s.offset = float(offset)
        s.grad[:] = tuple(float(v) for v in grad) + (0.0,) * (3 - len(grad))
        self.s = s
        self.ndim = ndim


def make_params(ndim, N, T=1, eps0=0.0, dR=1.0, Rmin=0.5, Rmax=1e9, max_step=0.5, seed=0, stream_id=0,
                edge_tol=1e-5, integration=0, freeze_tol=0.0, freeze_iters=0, cull_iter=0, cull_E=0.0) -> Params:
    """integration 0: Monte-Carlo samples, 1: the voxel grid of Eq. 5.  Stopping
    rules (0 disables): freeze after ``freeze_iters`` consecutive proposed steps
    below ``freeze_tol``; stop at iteration ``cull_iter`` when E > ``cull_E``."""
    p = Params()
    p.integration, p.freeze_tol, p.freeze_iters, p.cull_iter, p.cull_E = (int(integration), float(freeze_tol),
                                                                           int(freeze_iters), int(cull_iter),
                                                                           float(cull_E))
    p.ndim, p.N, p.T = ndim, N, T
    p.eps0, p.dR, p.Rmin, p.Rmax, p.max_step, p.edge_tol = eps0, dR, Rmin, Rmax, max_step, edge_tol
    p.key[0] = seed & 0xFFFFFFFF
    p.key[1] = (seed >> 32) & 0xFFFFFFFF
    p.stream_id = stream_id
    return p


# --------------------------------------------------------------------------- functions
def philox(ctrs: np.ndarray, key) -> np.ndarray:
    ctrs = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty_like(ctrs)
    lib().or_philox_batch(len(ctrs), _P(ctrs, ct.c_uint32), _P(k, ct.c_uint32), _P(out, ct.c_uint32))
    return out


def uniform24(w: int) -> float:
    return lib().or_uniform24(int(w))


def uniforms21(w0: int, w1: int):
    """The three 21-bit uniforms a 3D sample draws from its two words."""
    out = np.empty(3)
    lib().or_uniforms21(int(w0), int(w1), _P(out, ct.c_double))
    return tuple(out)


def half_to_double(bits: int) -> float:
    return lib().or_half_to_double(int(bits))


def rho(ndim: int) -> float:
    return lib().or_rho(ndim)


def weight(ndim, r, R, dR):
    r = np.ascontiguousarray(np.atleast_1d(r), dtype=np.float64)
    out = np.empty((len(r), 3))
    lib().or_weight_batch(ndim, len(r), _P(r, ct.c_double), R, dR, _P(out, ct.c_double))
    return out


def image_values(img, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    out = np.empty(len(x))
    lib().or_image_values(ct.byref(img.s), len(x), _P(x, ct.c_double), _P(out, ct.c_double))
    return out


def unit_samples(params: Params, it: int, k: int) -> np.ndarray:
    out = np.empty((params.N, 3))
    lib().or_unit_samples(ct.byref(params), it, k, _P(out, ct.c_double))
    return out


def eval_pq(img, params, p, q, it, k) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    res = np.empty(RES_LEN)
    lib().or_eval_pq(ct.byref(img.s), ct.byref(params), _P(p, ct.c_double), _P(q, ct.c_double), it, k,
                     _P(res, ct.c_double))
    return res


def eval_grid_pq(img, params, p, q) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    res = np.empty(RES_LEN)
    lib().or_eval_grid_pq(ct.byref(img.s), ct.byref(params), _P(p, ct.c_double), _P(q, ct.c_double),
                          _P(res, ct.c_double))
    return res


def eval_cr(img, params, c, R, it, k) -> np.ndarray:
    c = np.ascontiguousarray(list(c) + [0.0] * (3 - len(c)), dtype=np.float64)
    res = np.empty(RES_LEN)
    lib().or_eval_cr(ct.byref(img.s), ct.byref(params), _P(c, ct.c_double), float(R), it, k, _P(res, ct.c_double))
    return res


def eval_many(img, params, cR, iters, ks, nthreads: int = 0) -> np.ndarray:
    """Teacher-forced evaluations: rows (cx, cy, cz, R) at iterations ``iters`` for
    contour indices ``ks``; returns (m, RES_LEN)."""
    cR = np.ascontiguousarray(cR, dtype=np.float64).reshape(-1, 4)
    m = len(cR)
    it = np.ascontiguousarray(np.broadcast_to(np.asarray(iters, dtype=np.int64), (m,)))
    kk = np.ascontiguousarray(np.broadcast_to(np.asarray(ks, dtype=np.int64), (m,)))
    res = np.empty((m, RES_LEN))
    lib().or_eval_many(ct.byref(img.s), ct.byref(params), m, _P(cR, ct.c_double), _P(it, ct.c_int64),
                       _P(kk, ct.c_int64), _P(res, ct.c_double), nthreads)
    return res


def energy_grid(img, ndim, c, R, dR) -> float:
    c = np.ascontiguousarray(list(c) + [0.0] * (3 - len(c)), dtype=np.float64)
    return lib().or_energy_grid(ct.byref(img.s), ndim, _P(c, ct.c_double), float(R), float(dR))


def update_pq(img, params, it, res, p, q):
    p = np.array(p, dtype=np.float64, order="C")
    q = np.array(q, dtype=np.float64, order="C")
    res = np.ascontiguousarray(res, dtype=np.float64)
    lib().or_update_pq(ct.byref(img.s), ct.byref(params), it, _P(res, ct.c_double), _P(p, ct.c_double),
                       _P(q, ct.c_double))
    return p, q


def evolve(img, params, cR: np.ndarray, ids=None, trace: bool = False, nthreads: int = 0, stops: bool = False):
    """Returns (final cR (C x 4), E (C,), trace (T x C x 9) or None), and with
    ``stops`` also (stop reason (C,): 0 none, 1 step rule, 2 energy rule;
    evaluations made (C,)).  Trace rows after a stop are NaN."""
    cR = np.array(cR, dtype=np.float64, order="C").reshape(-1, 4)   # a C-ordered copy (updated in place)
    C = len(cR)
    ids = np.arange(C, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
    E = np.empty(C)
    tr = np.full((params.T, C, TRACE_LEN), np.nan) if trace else None
    st = np.zeros(C, dtype=np.int32)
    ne = np.zeros(C, dtype=np.int32)
    lib().or_evolve(ct.byref(img.s), ct.byref(params), C, _P(ids, ct.c_int64), _P(cR, ct.c_double),
                    _P(E, ct.c_double), _P(tr, ct.c_double) if trace else None, _P(st, ct.c_int32),
                    _P(ne, ct.c_int32), nthreads)
    return (cR, E, tr, st, ne) if stops else (cR, E, tr)


def max_threads() -> int:
    return lib().or_max_threads()


def seed_lattice(ndim, n_xyz, spacing, stride) -> np.ndarray:
    n = np.ascontiguousarray(list(n_xyz) + [1] * (3 - len(n_xyz)), dtype=np.int64)
    sp = np.ascontiguousarray(list(spacing) + [1.0] * (3 - len(spacing)), dtype=np.float64)
    cnt = lib().or_seed_lattice(ndim, _P(n, ct.c_int64), _P(sp, ct.c_double), float(stride), None)
    out = np.empty((cnt, 4))
    lib().or_seed_lattice(ndim, _P(n, ct.c_int64), _P(sp, ct.c_double), float(stride), _P(out, ct.c_double))
    return out


def localize(ndim, cR, E, E0) -> np.ndarray:
    cR = np.ascontiguousarray(cR, dtype=np.float64).reshape(-1, 4)
    E = np.ascontiguousarray(E, dtype=np.float64)
    out = np.empty(max(len(cR), 1), dtype=np.int64)
    m = lib().or_localize(ndim, len(cR), _P(cR, ct.c_double), _P(E, ct.c_double), float(E0), _P(out, ct.c_int64))
    return out[:m].copy()
