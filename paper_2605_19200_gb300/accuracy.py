"""Accuracy of the agglomerated query against the exact direct sum, on the GPU.

Section 4.2 measures the error of the far-field approximation against direct
evaluation: the exact winding number summed over every primitive, with no
far field.  This module runs that reference in the library itself, so that
millions of queries can be checked (the FP64 CPU oracle evaluates a few queries
per second on a many-patch model, and the GPU's own FP64 direct sum is limited
by the FP64 pipe, ~1/64 of the FP32 rate on this part):

* a model built without subdivision (max_aabb_frac = 0), queried in
  GWN_MODE_DIRECT: every primitive evaluated exactly for every query, FP32
  leaves with the FP64 near band, the per-leaf values summed in FP64;
* every query whose reference value lies within REFERENCE_BAND of a
  half-integer is evaluated again by the exact FP64 direct sum (beta_repair =
  0), so the reference's rounded labels are FP64-exact wherever a label could
  flip.

The reference's own error against the oracle and the GPU FP64 direct sum is
measured by the GPU tests.  compare() reports max |dGWN| and label mismatches
the way the tests judge them: labels of queries whose reference value lies
within `half_band` of a half-integer are not compared (Section 4.3: there is no
single correct containment decision next to a half-integer), and their count
is reported.
"""
from __future__ import annotations

import numpy as np

from . import api

REFERENCE_BAND = 0.05


def build_reference(prims, dim: int, **kw) -> api.Model:
    """Model for the exact direct sum over every unsubdivided primitive."""
    opts = dict(max_aabb_frac=0.0, beta_repair=0.0, beta=2.0)
    opts.update(kw)
    return api.gwn_build_2d(prims, **opts) if dim == 2 else api.gwn_build_3d(prims, **opts)


def reference_values(ref: api.Model, points, stream=None, band: float = REFERENCE_BAND):
    """Exact direct sum at `points` (CUDA tensor): (w, label, status) tensors."""
    return ref.query(points, mode=api.MODE_DIRECT, precision=api.PREC_FP32_REPAIR, repair_band=band,
                     stream=stream)


def compare(w, lab, w_ref, half_band: float = 1e-6) -> dict:
    """Error statistics of values w / labels lab against reference values w_ref
    (numpy arrays of one query set)."""
    w = np.asarray(w, dtype=np.float64)
    w_ref = np.asarray(w_ref, dtype=np.float64)
    lab = np.asarray(lab)
    ok = np.isfinite(w_ref) & np.isfinite(w)
    d = np.abs(w[ok] - w_ref[ok])
    frac = w_ref - np.floor(w_ref)
    half = ok & (np.abs(frac - 0.5) <= half_band)
    keep = ok & ~half
    ref_lab = np.where(w_ref >= 0, np.floor(w_ref + 0.5), np.ceil(w_ref - 0.5))  # round half away from zero
    mism = int(np.sum(lab[keep].astype(np.int64) != ref_lab[keep].astype(np.int64)))
    return {"checked": int(ok.sum()), "max_abs_dgwn": float(d.max()) if d.size else 0.0,
            "mean_abs_dgwn": float(d.mean()) if d.size else 0.0, "label_mismatches": mism,
            "labels_compared": int(keep.sum()), "half_integer_excluded": int(half.sum())}


def merge(stats) -> dict:
    """Combine compare() results of several query sets."""
    stats = list(stats)
    n = sum(s["checked"] for s in stats)
    return {"checked": n, "max_abs_dgwn": max((s["max_abs_dgwn"] for s in stats), default=0.0),
            "mean_abs_dgwn": (sum(s["mean_abs_dgwn"] * s["checked"] for s in stats) / n) if n else 0.0,
            "label_mismatches": sum(s["label_mismatches"] for s in stats),
            "labels_compared": sum(s["labels_compared"] for s in stats),
            "half_integer_excluded": sum(s["half_integer_excluded"] for s in stats)}
