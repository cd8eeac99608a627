"""Plain containers for NURBS input and a few exact test shapes.

This module holds input geometry only: control points, weights and knot
vectors of curves and trimmed patches.  It contains none of the winding
number arithmetic, so both the oracle tests and the CUDA-path tests may use
it without sharing any of the method's code.

Conventions
-----------
* A 2D curve is a clamped NURBS curve: ``degree`` p, ``ctrl`` (n, 2),
  ``weights`` (n,), ``knots`` (n + p + 1,), first and last knot repeated
  p + 1 times.
* A 3D patch is a clamped tensor-product NURBS surface with ``ctrl``
  (n_u, n_v, 3) indexed [i_u, i_v], ``weights`` (n_u, n_v), and a list of
  trimming curves given as 2D NURBS curves in the patch's (u, v) parameter
  domain.  Trimming curves form closed loops; the visible region is counted
  with the loops' winding number (outer loops counter-clockwise, holes
  clockwise).  A patch with no trimming curves is untrimmed: its boundary is
  the parameter rectangle, traversed counter-clockwise.
* Surface normals are S_u x S_v, so a counter-clockwise trim loop in (u, v)
  is the positively oriented boundary of the visible surface.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class Curve:
    degree: int
    ctrl: np.ndarray
    weights: np.ndarray
    knots: np.ndarray

    def __post_init__(self):
        self.ctrl = np.ascontiguousarray(self.ctrl, dtype=np.float64).reshape(-1, 2)
        self.weights = np.ascontiguousarray(self.weights, dtype=np.float64).reshape(-1)
        self.knots = np.ascontiguousarray(self.knots, dtype=np.float64).reshape(-1)

    @property
    def n_ctrl(self) -> int:
        return self.ctrl.shape[0]

    def reversed(self) -> "Curve":
        """Same point set traversed backwards (knots mirrored)."""
        k = self.knots
        return Curve(self.degree, self.ctrl[::-1].copy(), self.weights[::-1].copy(),
                     (k[0] + k[-1] - k[::-1]).copy())


@dataclass
class Patch:
    deg_u: int
    deg_v: int
    ctrl: np.ndarray
    weights: np.ndarray
    knots_u: np.ndarray
    knots_v: np.ndarray
    trims: List[Curve] = field(default_factory=list)

    def __post_init__(self):
        self.ctrl = np.ascontiguousarray(self.ctrl, dtype=np.float64)
        nu, nv = self.ctrl.shape[:2]
        self.ctrl = self.ctrl.reshape(nu, nv, 3)
        self.weights = np.ascontiguousarray(self.weights, dtype=np.float64).reshape(nu, nv)
        self.knots_u = np.ascontiguousarray(self.knots_u, dtype=np.float64).reshape(-1)
        self.knots_v = np.ascontiguousarray(self.knots_v, dtype=np.float64).reshape(-1)

    @property
    def n_u(self) -> int:
        return self.ctrl.shape[0]

    @property
    def n_v(self) -> int:
        return self.ctrl.shape[1]

    def flipped(self) -> "Patch":
        """Same visible surface with u and v exchanged, so the normal S_u x S_v flips.

        Trim curves are mirrored into the swapped domain and reversed, so the
        visible region keeps winding number +1.
        """
        trims = [Curve(c.degree, c.ctrl[:, ::-1].copy(), c.weights, c.knots).reversed()
                 for c in self.trims]
        return Patch(self.deg_v, self.deg_u, self.ctrl.transpose(1, 0, 2).copy(),
                     self.weights.T.copy(), self.knots_v.copy(), self.knots_u.copy(), trims)


def clamped_uniform_knots(n_ctrl: int, degree: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    n_inner = n_ctrl - degree - 1
    inner = np.linspace(lo, hi, n_inner + 2)[1:-1] if n_inner > 0 else np.zeros(0)
    return np.concatenate([np.full(degree + 1, lo), inner, np.full(degree + 1, hi)])


def bezier_knots(degree: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return np.concatenate([np.full(degree + 1, lo), np.full(degree + 1, hi)])


# ---------------------------------------------------------------- 2D shapes

def circle(center=(0.0, 0.0), radius=1.0, ccw=True) -> Curve:
    """Exact circle: 9-point rational quadratic NURBS (four quarter arcs)."""
    c = np.asarray(center, dtype=np.float64)
    unit = np.array([[1, 0], [1, 1], [0, 1], [-1, 1], [-1, 0], [-1, -1], [0, -1], [1, -1], [1, 0]],
                    dtype=np.float64)
    s = np.sqrt(0.5)
    w = np.array([1, s, 1, s, 1, s, 1, s, 1], dtype=np.float64)
    knots = np.array([0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 4], dtype=np.float64) / 4.0
    cur = Curve(2, c + radius * unit, w, knots)
    return cur if ccw else cur.reversed()


def arc(center, radius, theta0, theta1) -> Curve:
    """Exact circular arc (|theta1 - theta0| < pi) as one rational quadratic."""
    c = np.asarray(center, dtype=np.float64)
    half = 0.5 * (theta1 - theta0)
    tm = 0.5 * (theta0 + theta1)
    p0 = c + radius * np.array([np.cos(theta0), np.sin(theta0)])
    p2 = c + radius * np.array([np.cos(theta1), np.sin(theta1)])
    p1 = c + radius / np.cos(half) * np.array([np.cos(tm), np.sin(tm)])
    return Curve(2, np.stack([p0, p1, p2]), np.array([1.0, np.cos(half), 1.0]), bezier_knots(2))


def polyline(vertices, closed=True) -> Curve:
    """Degree-1 NURBS through the vertices (closed: last vertex joins the first)."""
    v = np.asarray(vertices, dtype=np.float64).reshape(-1, 2)
    if closed:
        v = np.concatenate([v, v[:1]], axis=0)
    n = v.shape[0]
    knots = np.concatenate([[0.0], np.arange(n, dtype=np.float64), [n - 1.0]]) / (n - 1.0)
    return Curve(1, v, np.ones(n), knots)


def bezier_curve(ctrl, weights=None) -> Curve:
    ctrl = np.asarray(ctrl, dtype=np.float64).reshape(-1, 2)
    p = ctrl.shape[0] - 1
    w = np.ones(p + 1) if weights is None else np.asarray(weights, dtype=np.float64)
    return Curve(p, ctrl, w, bezier_knots(p))


# ---------------------------------------------------------------- 3D shapes

def bilinear_patch(p00, p10, p01, p11, trims=None) -> Patch:
    ctrl = np.array([[p00, p01], [p10, p11]], dtype=np.float64)
    return Patch(1, 1, ctrl, np.ones((2, 2)), bezier_knots(1), bezier_knots(1), list(trims or []))


def planar_patch(origin, a, b, trims=None) -> Patch:
    """Affine planar patch S(u, v) = origin + u a + v b on [0, 1]^2."""
    o, a, b = (np.asarray(x, dtype=np.float64) for x in (origin, a, b))
    return bilinear_patch(o, o + a, o + b, o + a + b, trims)


def cube_shell(center=(0, 0, 0), half=1.0) -> List[Patch]:
    """Six bilinear patches bounding an axis-aligned cube, outward normals."""
    c = np.asarray(center, dtype=np.float64)
    h = float(half)
    out = []
    for axis in range(3):
        for sgn in (-1.0, 1.0):
            e = np.zeros(3)
            e[axis] = sgn * h
            i1, i2 = (axis + 1) % 3, (axis + 2) % 3
            a = np.zeros(3)
            b = np.zeros(3)
            a[i1] = 2 * h
            b[i2] = 2 * h
            origin = c + e - 0.5 * a - 0.5 * b
            # a x b points along +axis; flip for the negative face
            if sgn > 0:
                out.append(planar_patch(origin, a, b))
            else:
                out.append(planar_patch(origin, b, a))
    return out


def nurbs_sphere(center=(0, 0, 0), radius=1.0) -> Patch:
    """Exact sphere: degree (2, 2) rational patch, u around the axis, v pole to pole.

    Oriented with outward normals (S_u x S_v points away from the centre).
    """
    c = np.asarray(center, dtype=np.float64)
    s = np.sqrt(0.5)
    ring = np.array([[1, 0], [1, 1], [0, 1], [-1, 1], [-1, 0], [-1, -1], [0, -1], [1, -1], [1, 0]],
                    dtype=np.float64)
    wr = np.array([1, s, 1, s, 1, s, 1, s, 1])
    # profile from the south pole to the north pole in the (rho, z) half plane
    prof = np.array([[0, -1], [1, -1], [1, 0], [1, 1], [0, 1]], dtype=np.float64)
    wp = np.array([1, s, 1, s, 1])
    ctrl = np.zeros((9, 5, 3))
    w = np.zeros((9, 5))
    for i in range(9):
        for j in range(5):
            ctrl[i, j, 0:2] = ring[i] * prof[j, 0]
            ctrl[i, j, 2] = prof[j, 1]
            w[i, j] = wr[i] * wp[j]
    ctrl = c + radius * ctrl
    ku = np.array([0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 4], dtype=np.float64) / 4.0
    kv = np.array([0, 0, 0, 1, 1, 2, 2, 2], dtype=np.float64) / 2.0
    return Patch(2, 2, ctrl, w, ku, kv, [])


def shape_bbox_2d(curves: List[Curve]):
    pts = np.concatenate([c.ctrl for c in curves], axis=0)
    return pts.min(axis=0), pts.max(axis=0)


def shape_bbox_3d(patches: List[Patch]):
    pts = np.concatenate([p.ctrl.reshape(-1, 3) for p in patches], axis=0)
    return pts.min(axis=0), pts.max(axis=0)
