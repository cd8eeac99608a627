"""Accuracy / throughput sweeps over the method's parameters.

Section 4.2 studies the Taylor order of the far field (orders 0, 1, 2) and the
far-field factor beta; Section 4.3 the subdivision threshold (the fraction of
the shape's bounding-box diagonal below which leaves stop being split).  This
module runs such sweeps on the GPU for any curve or patch set: for every
(order, subdivision fraction) it builds a model, and for every beta it times
the FP32 query (CUDA events) and measures its error against an exact
reference.  The reference defaults to the FP64 direct sum on the GPU over the
unsubdivided primitives (the plain definition of Eq. 1, evaluated by this
library), so the sweep needs nothing but the GPU.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np

from . import api


def _build(dim: int, prims, **kw) -> api.Model:
    return api.gwn_build_2d(prims, **kw) if dim == 2 else api.gwn_build_3d(prims, **kw)


def exact_reference(dim: int, prims, points) -> np.ndarray:
    """FP64 direct sum over every unsubdivided primitive (GPU)."""
    m = _build(dim, prims, max_aabb_frac=0.0)
    w, _, _ = m.query(points, mode=api.MODE_DIRECT, precision=api.PREC_FP64)
    return w.cpu().numpy()


def sweep(dim: int, prims, points, orders: Sequence[int] = (0, 1, 2), betas: Sequence[float] = (2.0, 3.0, 4.0, 6.0, 8.0),
          fracs: Sequence[float] = (0.1,), reference: Optional[np.ndarray] = None, reps: int = 3,
          precision: int = api.PREC_FP32) -> List[Dict]:
    """One row per (order, subdivision fraction, beta): max and mean |dGWN| against
    the reference, queries/s of the FP32 query (no repair unless `precision` asks
    for it), leaves and build time.  `points` is a CUDA tensor (n, dim)."""
    import torch

    if reference is None:
        reference = exact_reference(dim, prims, points.double())
    ok = np.isfinite(reference)
    rows = []
    n = points.shape[0]
    stream = torch.cuda.current_stream(points.device)
    for frac in fracs:
        for order in orders:
            m = _build(dim, prims, order=order, max_aabb_frac=frac, beta=max(betas))
            info = m.info()
            outs = (torch.empty(n, dtype=torch.float64, device=points.device), None, None)
            for beta in betas:
                # the leaves' far test keeps its default ratio to beta (2D leaves have none)
                m.query(points, precision=precision, beta=beta, beta_leaf=beta, out=outs, stream=stream)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(reps):
                    m.query(points, precision=precision, beta=beta, beta_leaf=beta, out=outs, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                w = outs[0].cpu().numpy()
                err = np.abs(w[ok] - reference[ok])
                rows.append({"order": order, "max_aabb_frac": frac, "beta": beta,
                             "max_abs_dgwn": float(err.max()), "mean_abs_dgwn": float(err.mean()),
                             "queries_per_s": n * reps / (a.elapsed_time(b) / 1e3),
                             "leaves": info["n_leaves"], "build_ms": info["build_ms"]})
            m.release()
    return rows
