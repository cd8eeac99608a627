"""ctypes front end of the FP64 CPU oracle (gwn_oracle.c).

TEST INFRASTRUCTURE ONLY.  Geometry is passed to the C code as one flat
float64 record stream:

* curve  : p, n, ctrl (2n), weights (n), knots (n + p + 1)
* patch  : du, dv, nu, nv, ctrl (3 nu nv, [i_u][i_v] order), weights (nu nv),
           knots_u, knots_v, n_trims, then n_trims curve records
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Sequence

import numpy as np

FLAG_NEAR = 1
FLAG_ON_BOUNDARY = 2
FLAG_DEGENERATE = 4
FLAG_NOT_CONVERGED = 8

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gwn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP).  Returns the shared-library path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle())
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        L = ctypes.c_long
        for name in ("or_gwn2d", "or_gwn3d"):
            f = getattr(_lib, name)
            f.argtypes = [D, L, ctypes.c_int, D, L, ctypes.c_double, ctypes.c_int, D, I]
            f.restype = ctypes.c_int
        for name in ("or_gwn2d_each", "or_gwn3d_each"):
            f = getattr(_lib, name)
            f.argtypes = [D, L, ctypes.c_int, D, L, D]
            f.restype = ctypes.c_int
        _lib.or_curve_eval.argtypes = [D, L, ctypes.c_int, ctypes.c_int, D, L, D]
        _lib.or_patch_eval.argtypes = [D, L, ctypes.c_int, ctypes.c_int, D, L, D]
        _lib.or_segment_moments.argtypes = [D, L, D, D]
        _lib.or_patch_moments.argtypes = [D, L, ctypes.c_int, ctypes.c_int, D, ctypes.c_int, D]
        _lib.or_taylor.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D, D, D, D]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _curve_record(c) -> List[np.ndarray]:
    return [np.array([c.degree, c.n_ctrl], dtype=np.float64), c.ctrl.reshape(-1), c.weights.reshape(-1),
            c.knots.reshape(-1)]


def pack_curves(curves: Sequence) -> np.ndarray:
    parts: List[np.ndarray] = []
    for c in curves:
        parts.extend(_curve_record(c))
    return np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros(1))


def pack_patches(patches: Sequence) -> np.ndarray:
    parts: List[np.ndarray] = []
    for p in patches:
        parts.append(np.array([p.deg_u, p.deg_v, p.n_u, p.n_v], dtype=np.float64))
        parts.extend([p.ctrl.reshape(-1), p.weights.reshape(-1), p.knots_u, p.knots_v,
                      np.array([len(p.trims)], dtype=np.float64)])
        for c in p.trims:
            parts.extend(_curve_record(c))
    return np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros(1))


def _threads(n_threads):
    return int(n_threads) if n_threads else (os.cpu_count() or 1)


def gwn2d(curves, q, near_thr: float = 0.0, n_threads: int = 0):
    """Exact GWN of the curve collection at each query (n, 2): (w, flags)."""
    lib = _load()
    rec = pack_curves(curves)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 2)
    w = np.zeros(q.shape[0])
    fl = np.zeros(q.shape[0], dtype=np.int32)
    rc = lib.or_gwn2d(_ptr(rec), rec.size, len(curves), _ptr(q), q.shape[0], near_thr, _threads(n_threads),
                      _ptr(w), _iptr(fl))
    if rc:
        raise ValueError("oracle: invalid curve input")
    return w, fl


def gwn3d(patches, q, near_thr: float = 0.0, n_threads: int = 0):
    """Exact GWN of the trimmed-patch collection at each query (n, 3): (w, flags)."""
    lib = _load()
    rec = pack_patches(patches)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 3)
    w = np.zeros(q.shape[0])
    fl = np.zeros(q.shape[0], dtype=np.int32)
    rc = lib.or_gwn3d(_ptr(rec), rec.size, len(patches), _ptr(q), q.shape[0], near_thr, _threads(n_threads),
                      _ptr(w), _iptr(fl))
    if rc:
        raise ValueError("oracle: invalid patch input")
    return w, fl


def gwn2d_each(curves, q):
    lib = _load()
    rec = pack_curves(curves)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 2)
    out = np.zeros((q.shape[0], len(curves)))
    if lib.or_gwn2d_each(_ptr(rec), rec.size, len(curves), _ptr(q), q.shape[0], _ptr(out)):
        raise ValueError("oracle: invalid curve input")
    return out


def gwn3d_each(patches, q):
    lib = _load()
    rec = pack_patches(patches)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((q.shape[0], len(patches)))
    if lib.or_gwn3d_each(_ptr(rec), rec.size, len(patches), _ptr(q), q.shape[0], _ptr(out)):
        raise ValueError("oracle: invalid patch input")
    return out


def curve_eval(curve, t):
    lib = _load()
    rec = pack_curves([curve])
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    out = np.zeros((t.size, 2))
    if lib.or_curve_eval(_ptr(rec), rec.size, 1, 0, _ptr(t), t.size, _ptr(out)):
        raise ValueError("oracle: invalid curve input")
    return out


def patch_eval(patch, uv):
    """S, S_u, S_v at parameter pairs uv (n, 2): (n, 3, 3)."""
    lib = _load()
    rec = pack_patches([patch])
    uv = np.ascontiguousarray(uv, dtype=np.float64).reshape(-1, 2)
    out = np.zeros((uv.shape[0], 9))
    if lib.or_patch_eval(_ptr(rec), rec.size, 1, 0, _ptr(uv), uv.shape[0], _ptr(out)):
        raise ValueError("oracle: invalid patch input")
    return out.reshape(-1, 3, 3)


def _split_moments(out, dim):
    m0 = out[:dim].copy()
    m1 = out[dim:dim + dim * dim].reshape(dim, dim).copy()
    o = dim + dim * dim
    m2 = out[o:o + dim ** 3].reshape(dim, dim, dim).copy()
    o += dim ** 3
    return {"m0": m0, "m1": m1, "m2": m2, "area": float(out[o]), "c": out[o + 1:o + 1 + dim].copy()}


def segment_moments(segments, x0):
    """Moments about x0 of straight segments (n, 4) = (ax, ay, bx, by), by quadrature."""
    lib = _load()
    seg = np.ascontiguousarray(segments, dtype=np.float64).reshape(-1, 4)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    out = np.zeros(17)
    lib.or_segment_moments(_ptr(seg), seg.shape[0], _ptr(x0), _ptr(out))
    return _split_moments(out, 2)


def patch_moments(patch, x0, nsub: int = 4):
    """Moments about x0 of a trimmed patch by fan cubature of its visible region."""
    lib = _load()
    rec = pack_patches([patch])
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    out = np.zeros(43)
    if lib.or_patch_moments(_ptr(rec), rec.size, 1, 0, _ptr(x0), int(nsub), _ptr(out)):
        raise ValueError("oracle: invalid patch input")
    return _split_moments(out, 3)


def taylor(dim, order, x0, m0, m1, m2, q):
    """Eq. 3 with full derivative tensors for moments centred at x0."""
    lib = _load()
    a = [np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in (x0, m0, m1, m2, q)]
    out = np.zeros(1)
    lib.or_taylor(dim, order, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(a[3]), _ptr(a[4]), _ptr(out))
    return float(out[0])
