"""Python binding of the C ABI in include/gwn.h (argument marshalling only).

Functions keep the C names (gwn_build_2d, gwn_query, ...).  Geometry comes in
as synth-style objects with ``degree/ctrl/weights/knots`` (curves) and
``deg_u/deg_v/ctrl/weights/knots_u/knots_v/trims`` (patches); points and
outputs are torch tensors (device or host) or numpy arrays (host).  Every
computation happens in libgwn.so; this module never evaluates a winding
number itself.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import native

GWN_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "INVALID_GEOMETRY", 3: "OOM", 4: "CUDA", 5: "TIMEOUT",
                6: "BUSY", 7: "INTERNAL", 8: "NOT_FOUND"}
PREC_FP32_REPAIR, PREC_FP32, PREC_FP64 = 0, 1, 2
MODE_BVH, MODE_DIRECT = 0, 1
F32, F64 = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
QS_REPAIRED, QS_NEAR, QS_STACK_OVERFLOW, QS_UNRESOLVED = 1, 2, 4, 8


class GwnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class gwn_curve2d(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32), ("n_ctrl", ctypes.c_int32), ("ctrl", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("knots", ctypes.c_void_p)]


class gwn_patch3d(ctypes.Structure):
    _fields_ = [("deg_u", ctypes.c_int32), ("deg_v", ctypes.c_int32), ("n_u", ctypes.c_int32),
                ("n_v", ctypes.c_int32), ("ctrl", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("knots_u", ctypes.c_void_p), ("knots_v", ctypes.c_void_p), ("n_trims", ctypes.c_int32),
                ("trims", ctypes.c_void_p)]


class gwn_build_opts(ctypes.Structure):
    _fields_ = [("tolerance", ctypes.c_double), ("max_aabb_frac", ctypes.c_double), ("order", ctypes.c_int32),
                ("beta", ctypes.c_double), ("beta_repair", ctypes.c_double), ("repair_band", ctypes.c_double),
                ("quad_nodes", ctypes.c_int32), ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("n_threads", ctypes.c_int32), ("leaf_far", ctypes.c_int32), ("beta_leaf", ctypes.c_double),
                ("adaptive_beta", ctypes.c_int32), ("device_build", ctypes.c_int32), ("tree_builder", ctypes.c_int32),
                ("local_ratio", ctypes.c_double)]


class gwn_query_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("beta", ctypes.c_double),
                ("count_work", ctypes.c_int32), ("profile", ctypes.c_int32), ("beta_leaf", ctypes.c_double),
                ("repair_band", ctypes.c_double), ("local_ratio", ctypes.c_double)]


class gwn_model_stats(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_primitives", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_nodes", ctypes.c_int64), ("max_depth", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("build_ms", ctypes.c_double), ("beta", ctypes.c_double), ("beta_repair", ctypes.c_double),
                ("repair_band", ctypes.c_double), ("order", ctypes.c_int32), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("beta_leaf", ctypes.c_double), ("device", ctypes.c_int32),
                ("bin_points_per_cell", ctypes.c_int32), ("stack_depth", ctypes.c_int32),
                ("beta_repair_leaf", ctypes.c_double), ("eval_order", ctypes.c_int32),
                ("local_ratio", ctypes.c_double)]


class gwn_serve_opts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("n_slots", ctypes.c_int32), ("device", ctypes.c_int32)]


class gwn_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("points_completed", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("queries_per_s", ctypes.c_double),
                ("budget_used_bytes", ctypes.c_int64), ("max_in_flight", ctypes.c_int64),
                ("max_gpu_overlap", ctypes.c_int64)]


class gwn_query_item(ctypes.Structure):
    _fields_ = [("model", ctypes.c_void_p), ("points", ctypes.c_void_p), ("points_dtype", ctypes.c_int32),
                ("n", ctypes.c_size_t), ("out_w", ctypes.c_void_p), ("out_label", ctypes.c_void_p),
                ("out_status", ctypes.c_void_p)]


_P = ctypes.c_void_p
_SIGS = {
    "gwn_default_build_opts": (None, [ctypes.POINTER(gwn_build_opts)]),
    "gwn_default_query_opts": (None, [ctypes.POINTER(gwn_query_opts)]),
    "gwn_build_2d": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.POINTER(gwn_build_opts), ctypes.POINTER(_P)]),
    "gwn_build_3d": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.POINTER(gwn_build_opts), ctypes.POINTER(_P)]),
    "gwn_query": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_size_t, _P, _P, _P,
                                 ctypes.POINTER(gwn_query_opts), _P]),
    "gwn_model_info": (ctypes.c_int, [_P, ctypes.POINTER(gwn_model_stats)]),
    "gwn_query_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_size_t, _P, _P, _P, _P]),
    "gwn_last_query_stats": (ctypes.c_int, [_P, _P]),
    "gwn_model_leaves": (ctypes.c_int, [_P, _P, _P]),
    "gwn_model_tree": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "gwn_release": (ctypes.c_int, [_P]),
    "gwn_model_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "gwn_model_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int32, ctypes.POINTER(_P)]),
    "gwn_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)]),
    "gwn_query_batch": (ctypes.c_int, [_P, ctypes.POINTER(gwn_query_item), ctypes.c_size_t, _P]),
    "gwn_query_batch_host": (ctypes.c_int, [_P, ctypes.POINTER(gwn_query_item), ctypes.c_size_t, _P]),
    "gwn_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64)]),
    "gwn_batch_release": (ctypes.c_int, [_P]),
    "gwn_default_serve_opts": (None, [ctypes.POINTER(gwn_serve_opts)]),
    "gwn_serve_create": (ctypes.c_int, [ctypes.POINTER(gwn_serve_opts), ctypes.POINTER(_P)]),
    "gwn_serve_add_model": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "gwn_serve_submit": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_size_t,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "gwn_serve_poll": (ctypes.c_int, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32]),
    "gwn_serve_stats": (ctypes.c_int, [_P, ctypes.POINTER(gwn_server_stats)]),
    "gwn_serve_destroy": (ctypes.c_int, [_P]),
    "gwn_last_error": (ctypes.c_char_p, []),
    "gwn_version": (ctypes.c_char_p, []),
}


def lib() -> ctypes.CDLL:
    L = native.load()
    if not getattr(L, "_gwn_sigs", False):
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        L._gwn_sigs = True
    return L


def _check(code: int):
    if code != GWN_OK:
        raise GwnError(code, lib().gwn_last_error().decode())


def default_build_opts(**kw) -> gwn_build_opts:
    o = gwn_build_opts()
    lib().gwn_default_build_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown build option {k}")
        setattr(o, k, v)
    return o


def default_query_opts(**kw) -> gwn_query_opts:
    o = gwn_query_opts()
    lib().gwn_default_query_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown query option {k}")
        setattr(o, k, v)
    return o


class _Pack:
    """Contiguous float64 buffers that keep the ABI structs' pointers alive."""

    def __init__(self):
        self.parts = []
        self.size = 0

    def add(self, a) -> int:
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        off = self.size
        self.parts.append(a)
        self.size += a.size
        return off

    def finish(self):
        self.buf = np.concatenate(self.parts) if self.parts else np.zeros(1)
        self.base = self.buf.ctypes.data
        return self.base


def _curve_array(curves: Sequence, pack: _Pack):
    arr = (gwn_curve2d * max(1, len(curves)))()
    offs = []
    for c in curves:
        offs.append((pack.add(c.ctrl), pack.add(c.weights), pack.add(c.knots)))
    return arr, offs


def _fill_curves(arr, curves, offs, base):
    for i, (c, (o1, o2, o3)) in enumerate(zip(curves, offs)):
        arr[i].degree = int(c.degree)
        arr[i].n_ctrl = int(c.ctrl.shape[0])
        arr[i].ctrl = base + 8 * o1
        arr[i].weights = base + 8 * o2
        arr[i].knots = base + 8 * o3


class Model:
    """Owning wrapper of a gwn_model handle."""

    def __init__(self, handle: int, dim: int):
        self.handle = ctypes.c_void_p(handle)
        self.dim = dim

    def release(self):
        if self.handle is not None and self.handle.value:
            _check(lib().gwn_release(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass

    def info(self) -> dict:
        s = gwn_model_stats()
        _check(lib().gwn_model_info(self.handle, ctypes.byref(s)))
        return {f: (list(getattr(s, f)) if f in ("lo", "hi") else getattr(s, f)) for f, _ in s._fields_}

    def last_query_stats(self) -> dict:
        out = np.zeros(20, dtype=np.int64)
        _check(lib().gwn_last_query_stats(self.handle, out.ctypes.data))
        names = ["pairs", "repaired", "near_band", "overflow", "nodes", "leaf_tests", "far", "leaves",
                 "gl_nodes", "gl_deg", "hits", "chords", "trav_us", "leaf_us", "full_pairs", "fast_nodes",
                 "fast_us", "full_us", "local_nodes"]
        return {k: int(out[i]) for i, k in enumerate(names)}

    def leaves(self):
        n = self.info()["n_leaves"]
        prim = np.zeros(n, dtype=np.int64)
        param = np.zeros((n, 4))
        _check(lib().gwn_model_leaves(self.handle, prim.ctypes.data, param.ctypes.data))
        return prim, param

    def tree(self):
        info = self.info()
        ni, d = info["n_nodes"], self.dim
        M = 14 if d == 2 else 120   # orders 0-2 in 2D, 0-3 in 3D
        child = np.zeros((max(ni, 1), 2), dtype=np.int32)
        x0 = np.zeros((max(ni, 1), d))
        r = np.zeros(max(ni, 1))
        mom = np.zeros((max(ni, 1), M))
        _check(lib().gwn_model_tree(self.handle, child.ctypes.data, x0.ctypes.data, r.ctypes.data, mom.ctypes.data))
        return {"child": child[:ni], "x0": x0[:ni], "r": r[:ni], "mom": mom[:ni]}

    def query(self, points, mode: int = MODE_BVH, precision: int = -1, beta: float = 0.0, stream=None,
              want_label: bool = True, want_status: bool = True, count_work: bool = False, profile: bool = False,
              out=None, beta_leaf: float = 0.0, repair_band: float = 0.0, local_ratio: float = 0.0):
        return gwn_query(self, points, mode=mode, precision=precision, beta=beta, stream=stream,
                         want_label=want_label, want_status=want_status, count_work=count_work, profile=profile,
                         out=out, beta_leaf=beta_leaf, repair_band=repair_band, local_ratio=local_ratio)


def marshal_curves(curves: Sequence):
    """gwn_curve2d array for `curves` (synth.geometry.Curve-like objects) and the
    buffers that keep its pointers valid: (array, keepalive)."""
    pack = _Pack()
    arr, offs = _curve_array(curves, pack)
    base = pack.finish()
    _fill_curves(arr, curves, offs, base)
    return arr, pack


def marshal_patches(patches: Sequence):
    """gwn_patch3d array for `patches` (synth.geometry.Patch-like objects) and the
    buffers that keep its pointers valid: (array, keepalive)."""
    pack = _Pack()
    parr = (gwn_patch3d * max(1, len(patches)))()
    poffs = []
    trim_arrays = []
    all_trims = []
    for p in patches:
        poffs.append((pack.add(p.ctrl), pack.add(p.weights), pack.add(p.knots_u), pack.add(p.knots_v)))
        tarr, toffs = _curve_array(p.trims, pack)
        trim_arrays.append(tarr)
        all_trims.append(toffs)
    base = pack.finish()
    for i, p in enumerate(patches):
        o1, o2, o3, o4 = poffs[i]
        s = parr[i]
        s.deg_u, s.deg_v = int(p.deg_u), int(p.deg_v)
        s.n_u, s.n_v = int(p.ctrl.shape[0]), int(p.ctrl.shape[1])
        s.ctrl, s.weights = base + 8 * o1, base + 8 * o2
        s.knots_u, s.knots_v = base + 8 * o3, base + 8 * o4
        s.n_trims = len(p.trims)
        _fill_curves(trim_arrays[i], p.trims, all_trims[i], base)
        s.trims = ctypes.cast(trim_arrays[i], _P).value if p.trims else None
    return parr, (pack, trim_arrays)


def gwn_build_2d(curves: Sequence, opts: Optional[gwn_build_opts] = None, **kw) -> Model:
    opts = opts or default_build_opts(**kw)
    arr, keep = marshal_curves(curves)
    h = ctypes.c_void_p()
    _check(lib().gwn_build_2d(ctypes.cast(arr, _P), len(curves), ctypes.byref(opts), ctypes.byref(h)))
    return Model(h.value, 2)


def gwn_build_3d(patches: Sequence, opts: Optional[gwn_build_opts] = None, **kw) -> Model:
    opts = opts or default_build_opts(**kw)
    parr, keep = marshal_patches(patches)
    h = ctypes.c_void_p()
    _check(lib().gwn_build_3d(ctypes.cast(parr, _P), len(patches), ctypes.byref(opts), ctypes.byref(h)))
    return Model(h.value, 3)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _check_shapes(model: Model, pts, out):
    """The C ABI reads n x dim points and writes n outputs: refuse shapes that
    would make it read or write past the caller's buffers."""
    if len(pts.shape) != 2 or pts.shape[1] != model.dim:
        raise ValueError(f"points must have shape (n, {model.dim})")
    if out is not None:
        n = pts.shape[0]
        for t in out:
            if t is not None and (len(t.shape) != 1 or t.shape[0] < n):
                raise ValueError("every output must be 1-D with at least n entries")
            if t is not None and not (t.is_contiguous() if hasattr(t, "is_contiguous") else t.flags["C_CONTIGUOUS"]):
                raise ValueError("outputs must be contiguous")
        w, lab, st = out
        if str(w.dtype) not in ("float64", "torch.float64"):
            raise TypeError("out w must be float64")
        for t in (lab, st):
            size = None if t is None else (t.element_size() if hasattr(t, "element_size") else t.itemsize)
            if size is not None and size != 4:
                raise TypeError("label and status outputs must be 32-bit")


def _check_device(model: Model, pts, out):
    """Device calls hand raw pointers to the kernels: every tensor must be a
    CUDA tensor on the model's GPU, else the kernels would read host memory or
    another GPU's memory as if it were their own."""
    dev = model.info()["device"]
    for name, t in (("points", pts),) + tuple(("output", t) for t in (out or ()) if t is not None):
        if not getattr(t, "is_cuda", False):
            raise TypeError(f"{name} must be a CUDA tensor for a device call")
        if t.device.index != dev:
            raise TypeError(f"{name} lives on cuda:{t.device.index}, the model on cuda:{dev}")


def gwn_query(model: Model, points, mode: int = MODE_BVH, precision: int = -1, beta: float = 0.0, stream=None,
              want_label: bool = True, want_status: bool = True, count_work: bool = False, profile: bool = False,
              out=None, beta_leaf: float = 0.0, repair_band: float = 0.0, local_ratio: float = 0.0):
    """GWN at points.  torch CUDA tensor -> asynchronous device call with device
    outputs; numpy array or CPU tensor -> host call (staged, synchronous).
    Returns (w float64, label int32 or None, status uint32/int32 or None).
    `out` may supply preallocated outputs (w, label or None, status or None)."""
    q = default_query_opts(mode=mode, precision=precision, beta=beta, count_work=int(count_work),
                           profile=int(profile), beta_leaf=beta_leaf, repair_band=repair_band,
                           local_ratio=local_ratio)
    try:
        import torch
    except Exception:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(points, torch.Tensor) and points.is_cuda:
        pts = points.contiguous()
        if pts.dtype not in (torch.float32, torch.float64):
            pts = pts.float()
        _check_shapes(model, pts, out)
        _check_device(model, pts, out)
        n = pts.shape[0]
        dt = F32 if pts.dtype == torch.float32 else F64
        if out is not None:
            w, lab, st = out
        else:
            w = torch.empty(n, dtype=torch.float64, device=pts.device)
            lab = torch.empty(n, dtype=torch.int32, device=pts.device) if want_label else None
            st = torch.empty(n, dtype=torch.int32, device=pts.device) if want_status else None
        _check(lib().gwn_query(model.handle, pts.data_ptr(), dt, MEM_DEVICE, n, w.data_ptr(),
                               lab.data_ptr() if lab is not None else None,
                               st.data_ptr() if st is not None else None, ctypes.byref(q),
                               _stream_handle(stream)))
        return w, lab, st
    if torch is not None and isinstance(points, torch.Tensor):
        points = points.numpy()
    pts = np.ascontiguousarray(points)

    def _addr(a):
        if a is None:
            return None
        if torch is not None and isinstance(a, torch.Tensor):
            return a.data_ptr()
        return a.ctypes.data
    if pts.dtype not in (np.float32, np.float64):
        pts = pts.astype(np.float64)
    _check_shapes(model, pts, out)
    n = pts.shape[0]
    dt = F32 if pts.dtype == np.float32 else F64
    if out is not None:
        w, lab, st = out
    else:
        w = np.zeros(n)
        lab = np.zeros(n, dtype=np.int32) if want_label else None
        st = np.zeros(n, dtype=np.uint32) if want_status else None
    _check(lib().gwn_query(model.handle, pts.ctypes.data, dt, MEM_HOST, n, _addr(w), _addr(lab), _addr(st),
                           ctypes.byref(q), _stream_handle(stream)))
    return w, lab, st


def gwn_model_info(model: Model) -> dict:
    return model.info()


def gwn_release(model: Model):
    model.release()


def gwn_model_save(model: Model, path: str):
    """Write a built model to `path` (gwn_model_load restores it without rebuilding)."""
    _check(lib().gwn_model_save(model.handle, os.fsencode(path)))


def gwn_model_load(path: str, device: int = -1) -> Model:
    """Restore a model written by gwn_model_save (device -2: host copy only)."""
    h = ctypes.c_void_p()
    _check(lib().gwn_model_load(os.fsencode(path), int(device), ctypes.byref(h)))
    m = Model(h.value, 0)
    m.dim = m.info()["dim"]
    return m


def gwn_version() -> str:
    return lib().gwn_version().decode()


def gwn_query_noalloc(model: Model, points, out, stream=None):
    """Query through gwn_query_noalloc: `points` a CUDA tensor (n x dim, float32
    or float64), `out` = (w float64, label int32 or None, status int32 or
    None) CUDA tensors supplied by the caller; the library allocates nothing."""
    if out is None:
        raise TypeError("gwn_query_noalloc writes into caller-supplied outputs: pass out=(w, label, status)")
    _check_shapes(model, points, out)
    _check_device(model, points, out)
    if str(points.dtype) not in ("torch.float32", "torch.float64") or not points.is_contiguous():
        raise TypeError("points must be a contiguous float32 or float64 CUDA tensor")
    w, lab, st = out
    dt = F32 if str(points.dtype).endswith("float32") else F64
    _check(lib().gwn_query_noalloc(model.handle, points.data_ptr(), dt, points.shape[0], w.data_ptr(),
                                   lab.data_ptr() if lab is not None else None,
                                   st.data_ptr() if st is not None else None, _stream_handle(stream)))
    return w, lab, st


class Server:
    """The gwn_serve_* request loop (continuous batching over resident models)."""

    def __init__(self, mem_budget_bytes: int = 40 << 30, n_slots: int = 4, device: int = -1):
        o = gwn_serve_opts()
        lib().gwn_default_serve_opts(ctypes.byref(o))
        o.mem_budget_bytes, o.n_slots, o.device = int(mem_budget_bytes), int(n_slots), int(device)
        h = ctypes.c_void_p()
        _check(lib().gwn_serve_create(ctypes.byref(o), ctypes.byref(h)))
        self.handle = h
        self.models = []
        self.dims = []

    def add_model(self, model: Model) -> int:
        mid = ctypes.c_int32()
        _check(lib().gwn_serve_add_model(self.handle, model.handle, ctypes.byref(mid)))
        self.models.append(model)
        self.dims.append(model.dim)
        return mid.value

    def submit(self, model_id: int, points) -> int:
        pts = np.ascontiguousarray(points)
        if pts.dtype not in (np.float32, np.float64):
            pts = pts.astype(np.float64)
        if 0 <= int(model_id) < len(self.dims) and (pts.ndim != 2 or pts.shape[1] != self.dims[int(model_id)]):
            raise ValueError(f"points must be (n, {self.dims[int(model_id)]}) for model {model_id}")
        rid = ctypes.c_uint64()
        _check(lib().gwn_serve_submit(self.handle, int(model_id), pts.ctypes.data,
                                      F32 if pts.dtype == np.float32 else F64, pts.shape[0], ctypes.byref(rid)))
        return rid.value

    def poll(self, request_id: int, n: int, timeout_ms: int = 60000):
        w = np.zeros(n)
        lab = np.zeros(n, dtype=np.int32)
        _check(lib().gwn_serve_poll(self.handle, ctypes.c_uint64(request_id), w.ctypes.data, lab.ctypes.data,
                                    int(timeout_ms)))
        return w, lab

    def stats(self) -> dict:
        s = gwn_server_stats()
        _check(lib().gwn_serve_stats(self.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().gwn_serve_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """gwn_query_batch: many models and point sets in one (graph) launch."""

    def __init__(self, n_streams: int = 4, device: int = -1):
        h = ctypes.c_void_p()
        _check(lib().gwn_batch_create(int(n_streams), int(device), ctypes.byref(h)))
        self.handle = h
        self._items = None
        self._keep = None

    def query(self, models, points, outs, stream=None):
        """models: list of Model; points: list of CUDA tensors (n x dim, float32
        or float64); outs: list of (w float64, label int32 or None, status int32
        or None) CUDA tensors.  Enqueues on `stream`; returns outs."""
        n = len(models)
        if not (len(points) == n and len(outs) == n):
            raise ValueError("models, points and outs must have the same length")
        arr = (gwn_query_item * n)()
        for k, (m, p, o) in enumerate(zip(models, points, outs)):
            w, lab, st = o
            if str(p.dtype) not in ("torch.float32", "torch.float64") or not p.is_contiguous():
                raise TypeError("points must be contiguous float32 or float64 tensors")
            if p.dim() != 2 or p.shape[1] != m.dim:
                raise ValueError("points must be (n, dim)")
            if str(w.dtype) != "torch.float64" or w.shape[0] < p.shape[0]:
                raise TypeError("out w must be float64 with n entries")
            for t in (lab, st):
                if t is not None and (t.element_size() != 4 or t.shape[0] < p.shape[0]):
                    raise TypeError("label and status outputs must be 32-bit with n entries")
            _check_device(m, p, o)
            arr[k].model = m.handle.value
            arr[k].points = p.data_ptr()
            arr[k].points_dtype = F32 if str(p.dtype).endswith("float32") else F64
            arr[k].n = p.shape[0]
            arr[k].out_w = w.data_ptr()
            arr[k].out_label = lab.data_ptr() if lab is not None else None
            arr[k].out_status = st.data_ptr() if st is not None else None
        self._keep = (list(models), list(points), list(outs))
        _check(lib().gwn_query_batch(self.handle, arr, n, _stream_handle(stream)))
        return outs

    def query_host(self, models, points, outs, stream=None):
        """gwn_query_batch_host: points and outputs in host memory (CPU torch
        tensors or numpy arrays; page-locked buffers let the library capture
        the copies in its graph).  Synchronous; returns outs."""
        n = len(models)
        if not (len(points) == n and len(outs) == n):
            raise ValueError("models, points and outs must have the same length")

        def _host(a, what):
            if hasattr(a, "is_cuda") and a.is_cuda:
                raise TypeError(f"{what} must be in host memory for query_host")
            if hasattr(a, "is_contiguous"):
                if not a.is_contiguous():
                    raise ValueError(f"{what} must be contiguous")
                return a.data_ptr(), str(a.dtype).replace("torch.", ""), a.element_size(), tuple(a.shape)
            if not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"{what} must be contiguous")
            return a.ctypes.data, str(a.dtype), a.itemsize, tuple(a.shape)

        arr = (gwn_query_item * n)()
        for k, (m, p, o) in enumerate(zip(models, points, outs)):
            pp, pdt, _, pshape = _host(p, "points")
            if pdt not in ("float32", "float64") or len(pshape) != 2 or pshape[1] != m.dim:
                raise TypeError("points must be (n, dim) float32 or float64")
            w, lab, st = o
            wp, wdt, _, wshape = _host(w, "out w")
            if wdt != "float64" or wshape[0] < pshape[0]:
                raise TypeError("out w must be float64 with n entries")
            ptrs = []
            for t in (lab, st):
                if t is None:
                    ptrs.append(None)
                    continue
                tp, _, es, tshape = _host(t, "label/status output")
                if es != 4 or tshape[0] < pshape[0]:
                    raise TypeError("label and status outputs must be 32-bit with n entries")
                ptrs.append(tp)
            arr[k].model = m.handle.value
            arr[k].points = pp
            arr[k].points_dtype = F32 if pdt == "float32" else F64
            arr[k].n = pshape[0]
            arr[k].out_w = wp
            arr[k].out_label, arr[k].out_status = ptrs
        self._keep = (list(models), list(points), list(outs))
        _check(lib().gwn_query_batch_host(self.handle, arr, n, _stream_handle(stream)))
        return outs

    def info(self) -> dict:
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().gwn_batch_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"graph_launches": a.value, "captures": b.value, "workspace_bytes": c.value}

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().gwn_batch_release(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
