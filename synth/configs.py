"""Seeded synthetic workloads shaped like the paper's 2D and 3D experiments.

The paper evaluates SVG clip-art (cubic and rational Bezier curves, queried on a
regular grid over the view box) and CAD parts from a STEP collection
(trimmed NURBS patches, queried on a grid over the bounding box), Section 4.
Neither collection is available here, so these generators stand in for them.
Every function is deterministic for a given seed.  Query coordinates are
rounded to float32-representable values so that a float32 and a float64
consumer see the same points.

Workloads
---------
* ``star_2d``      one closed loop of 64 cubic Bezier curves around the star
                   r = 1 + 0.3 sin(5 theta) + N(0, 0.02^2), 4 curves removed;
                   16,384 queries uniform in the bounding box scaled 1.2x.
* ``loops_2d``     200 randomly placed, randomly oriented perturbed circles of
                   100 curves each (cubic with unit weights, or rational
                   quadratic with middle weight U[0.5, 2], half each), 5% of the
                   curves removed; 1024 x 1024 grid over the box scaled 1.05x.
* ``sphere_3d``    a unit sphere deformed by low-order harmonics (l <= 3,
                   coefficients 0.1 N(0, 1)), tiled by 6 x 8 x 8 = 384 bicubic
                   Bezier patches on a cubed-sphere layout, each trimmed to one
                   random disc in parameter space; queries uniform in the box.
* ``cad_3d``       a union of 3-8 overlapping perturbed boxes and cylinders made
                   of N bicubic rational patches (weights U[0.8, 1.2]) with an
                   outer polygonal trim loop and 0-2 polygonal holes each.
* ``cad_batch_3d`` 16 ``cad_3d`` models, N log-uniform in [1000, 40000],
                   queries per model log-uniform in [65,536, 4,194,304].
* ``serve_models`` / ``serve_trace``  8 resident models (2 ``loops_2d``-type,
                   2 ``sphere_3d``-type, 4 ``cad_3d``-type) and an open-loop
                   request trace: Poisson arrivals, sizes log-normal with median
                   16,384 points and sigma 1.5 clamped to [1,000, 2,000,000],
                   model chosen uniformly; points uniform in the model's box.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

from .geometry import Curve, Patch, bezier_knots

BASE_SEED = 260519200


def _f32(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def uniform_queries(lo, hi, n, rng, scale=1.0) -> np.ndarray:
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo) * scale
    q = rng.uniform(c - h, c + h, size=(n, lo.shape[0]))
    return _f32(q)


def grid_queries_2d(lo, hi, res, scale=1.0) -> np.ndarray:
    """Cell centres of a res x res grid over the box scaled about its centre."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo) * scale
    xs = c[0] - h[0] + (np.arange(res) + 0.5) * (2 * h[0] / res)
    ys = c[1] - h[1] + (np.arange(res) + 0.5) * (2 * h[1] / res)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return _f32(np.stack([X.ravel(), Y.ravel()], axis=1))


def _bbox(pts):
    return pts.min(axis=0), pts.max(axis=0)


# ------------------------------------------------------------------ 2D


def _catmull_rom_cubics(p: np.ndarray) -> np.ndarray:
    """Closed C1 cubic Bezier spline through the points p (K, 2): (K, 4, 2)."""
    pm = np.roll(p, 1, axis=0)
    pp = np.roll(p, -1, axis=0)
    ppp = np.roll(p, -2, axis=0)
    b0 = p
    b1 = p + (pp - pm) / 6.0
    b2 = pp - (ppp - p) / 6.0
    b3 = pp
    return np.stack([b0, b1, b2, b3], axis=1)


def star_2d(seed: int = BASE_SEED + 1, n_queries: int = 16384) -> Tuple[List[Curve], np.ndarray]:
    rng = np.random.default_rng(seed)
    K = 64
    th = 2 * np.pi * np.arange(K) / K
    r = 1.0 + 0.3 * np.sin(5 * th) + rng.normal(0.0, 0.02, K)
    pts = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    bez = _catmull_rom_cubics(pts)
    drop = set(rng.choice(K, size=4, replace=False).tolist())
    curves = [Curve(3, bez[k], np.ones(4), bezier_knots(3)) for k in range(K) if k not in drop]
    lo, hi = _bbox(np.concatenate([c.ctrl for c in curves]))
    q = uniform_queries(lo, hi, n_queries, rng, scale=1.2)
    return curves, q


def _loop_curves(rng, center, radius, ccw, per_loop) -> List[Curve]:
    K = per_loop
    th = 2 * np.pi * (np.arange(K) + rng.uniform(-0.3, 0.3, K)) / K
    th = np.sort(th)
    amps = rng.uniform(0.0, 0.06, 4)
    phases = rng.uniform(0, 2 * np.pi, 4)

    def rad(t):
        return radius * (1.0 + sum(amps[i] * np.sin((i + 2) * t + phases[i]) for i in range(4)))

    def pt(t):
        return np.stack([center[0] + rad(t) * np.cos(t), center[1] + rad(t) * np.sin(t)], axis=-1)

    P = pt(th)
    bez = _catmull_rom_cubics(P)
    th_next = np.roll(th, -1)
    th_next[-1] += 2 * np.pi
    mid = pt(0.5 * (th + th_next))
    out = []
    for k in range(K):
        if rng.uniform() < 0.5:
            c = Curve(3, bez[k], np.ones(4), bezier_knots(3))
        else:
            w = rng.uniform(0.5, 2.0)
            p0, p2 = P[k], P[(k + 1) % K]
            # middle control point chosen so the curve passes through the mid sample
            p1 = ((2 + 2 * w) * mid[k] - p0 - p2) / (2 * w)
            c = Curve(2, np.stack([p0, p1, p2]), np.array([1.0, w, 1.0]), bezier_knots(2))
        out.append(c if ccw else c.reversed())
    return out


def loops_2d(seed: int = BASE_SEED + 2, n_loops: int = 200, per_loop: int = 100,
             drop_frac: float = 0.05, res: int = 1024) -> Tuple[List[Curve], np.ndarray]:
    rng = np.random.default_rng(seed)
    curves: List[Curve] = []
    for _ in range(n_loops):
        c = rng.uniform(0.15, 0.85, 2)
        R = math.exp(rng.uniform(math.log(0.02), math.log(0.35)))
        curves.extend(_loop_curves(rng, c, R, rng.uniform() < 0.5, per_loop))
    n = len(curves)
    keep = np.ones(n, dtype=bool)
    keep[rng.choice(n, size=int(round(drop_frac * n)), replace=False)] = False
    curves = [c for c, k in zip(curves, keep) if k]
    lo, hi = _bbox(np.concatenate([c.ctrl for c in curves]))
    q = grid_queries_2d(lo, hi, res, scale=1.05)
    return curves, q


# ------------------------------------------------------------------ 3D helpers

_B3 = np.array([[math.comb(3, k) * (s ** k) * ((1 - s) ** (3 - k)) for k in range(4)]
                for s in (0.0, 1.0 / 3.0, 2.0 / 3.0, 1.0)])
_B3_INV = np.linalg.inv(_B3)


def _interp_bicubic(samples: np.ndarray) -> np.ndarray:
    """Bezier control net (4, 4, 3) interpolating a 4x4 grid of samples at s = 0, 1/3, 2/3, 1."""
    return np.einsum("ia,abk,jb->ijk", _B3_INV, samples, _B3_INV)


def _real_harmonics(d: np.ndarray) -> np.ndarray:
    """Low-order (1 <= l <= 3) real harmonic polynomials on unit vectors d (..., 3)."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    return np.stack([
        x, y, z,
        x * y, y * z, x * z, 0.5 * (x * x - y * y), 0.5 * (3 * z * z - 1),
        0.25 * y * (3 * x * x - y * y), x * y * z, 0.5 * y * (5 * z * z - 1),
        0.5 * z * (5 * z * z - 3), 0.5 * x * (5 * z * z - 1), 0.5 * z * (x * x - y * y),
        0.25 * x * (x * x - 3 * y * y),
    ], axis=-1)


_CUBE_FACES = [  # (normal, e1, e2) with e1 x e2 = normal
    (np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0])),
    (np.array([-1.0, 0, 0]), np.array([0, 0, 1.0]), np.array([0, 1.0, 0])),
    (np.array([0, 1.0, 0]), np.array([0, 0, 1.0]), np.array([1.0, 0, 0])),
    (np.array([0, -1.0, 0]), np.array([1.0, 0, 0]), np.array([0, 0, 1.0])),
    (np.array([0, 0, 1.0]), np.array([1.0, 0, 0]), np.array([0, 1.0, 0])),
    (np.array([0, 0, -1.0]), np.array([0, 1.0, 0]), np.array([1.0, 0, 0])),
]


def _circle_trim(rng) -> Curve:
    c = rng.uniform(0.35, 0.65, 2)
    r = rng.uniform(0.2, 0.3)
    unit = np.array([[1, 0], [1, 1], [0, 1], [-1, 1], [-1, 0], [-1, -1], [0, -1], [1, -1], [1, 0]],
                    dtype=np.float64)
    s = math.sqrt(0.5)
    w = np.array([1, s, 1, s, 1, s, 1, s, 1])
    knots = np.array([0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 4], dtype=np.float64) / 4.0
    return Curve(2, c + r * unit, w, knots)


def sphere_3d(seed: int = BASE_SEED + 3, cells: int = 8, n_queries: int = 1 << 20
              ) -> Tuple[List[Patch], np.ndarray]:
    rng = np.random.default_rng(seed)
    coef = 0.1 * rng.normal(0.0, 1.0, 15)
    s4 = np.array([0.0, 1.0 / 3.0, 2.0 / 3.0, 1.0])
    patches: List[Patch] = []
    for normal, e1, e2 in _CUBE_FACES:
        for i in range(cells):
            for j in range(cells):
                a = -1 + 2 * (i + s4) / cells          # face coordinates of the 4 samples
                b = -1 + 2 * (j + s4) / cells
                ta = np.tan(0.25 * np.pi * a)          # equi-angular cube-sphere mapping
                tb = np.tan(0.25 * np.pi * b)
                P = normal[None, None, :] + ta[:, None, None] * e1 + tb[None, :, None] * e2
                d = P / np.linalg.norm(P, axis=-1, keepdims=True)
                r = 1.0 + _real_harmonics(d) @ coef
                net = _interp_bicubic(r[..., None] * d)
                patches.append(Patch(3, 3, net, np.ones((4, 4)), bezier_knots(3), bezier_knots(3),
                                     [_circle_trim(rng)]))
    lo, hi = _bbox(np.concatenate([p.ctrl.reshape(-1, 3) for p in patches]))
    q = uniform_queries(lo, hi, n_queries, rng)
    return patches, q


# ------------------------------------------------------------------ CAD-like models


def _star_polygon(rng, center, rmin_frac, rmax_frac, nv, max_radius_fn, ccw):
    th = 2 * np.pi * (np.arange(nv) + rng.uniform(0.1, 0.9, nv)) / nv
    rad = rng.uniform(rmin_frac, rmax_frac, nv) * max_radius_fn(th)
    pts = np.stack([center[0] + rad * np.cos(th), center[1] + rad * np.sin(th)], axis=1)
    if not ccw:
        pts = pts[::-1]
    pts = np.concatenate([pts, pts[:1]], axis=0)
    n = pts.shape[0]
    knots = np.concatenate([[0.0], np.arange(n, dtype=np.float64), [n - 1.0]]) / (n - 1.0)
    return Curve(1, pts, np.ones(n), knots)


def _cad_trims(rng) -> List[Curve]:
    """Outer CCW polygon near the domain boundary plus 0-2 small CW polygonal holes."""
    def to_square(th):
        return 0.5 / np.maximum(np.abs(np.cos(th)), np.abs(np.sin(th)))
    loops = [_star_polygon(rng, (0.5, 0.5), 0.80, 0.96, int(rng.integers(6, 13)), to_square, True)]
    n_holes = int(rng.integers(0, 3))
    phi = rng.uniform(0, 2 * np.pi)
    for h in range(n_holes):
        sgn = 1.0 if h == 0 else -1.0
        c = (0.5 + sgn * 0.09 * math.cos(phi), 0.5 + sgn * 0.09 * math.sin(phi))
        R = rng.uniform(0.03, 0.06)
        loops.append(_star_polygon(rng, c, 0.7, 1.0, int(rng.integers(5, 9)),
                                   lambda th, R=R: np.full_like(th, R), False))
    return loops


def _elevate_quadratic(h: np.ndarray) -> np.ndarray:
    """Exact degree elevation 2 -> 3 of homogeneous control points (3, k)."""
    return np.stack([h[0], (h[0] + 2 * h[1]) / 3, (2 * h[1] + h[2]) / 3, h[2]])


def _grid_patches(origin, a, b, na, nb):
    """Planar bicubic nets tiling origin + s a + t b, s,t in [0,1]: list of (4,4,3), (4,4)."""
    out = []
    s4 = np.arange(4) / 3.0
    for i in range(na):
        for j in range(nb):
            s = (i + s4) / na
            t = (j + s4) / nb
            net = origin + s[:, None, None] * a + t[None, :, None] * b
            out.append((net, np.ones((4, 4))))
    return out


def _box_nets(size, budget):
    sx, sy, sz = size
    faces = []
    h = 0.5 * np.asarray(size)
    for axis in range(3):
        i1, i2 = (axis + 1) % 3, (axis + 2) % 3
        for sgn in (-1.0, 1.0):
            a = np.zeros(3)
            b = np.zeros(3)
            a[i1] = 2 * h[i1]
            b[i2] = 2 * h[i2]
            o = np.zeros(3)
            o[axis] = sgn * h[axis]
            o = o - 0.5 * a - 0.5 * b
            if sgn < 0:
                a, b = b, a
            faces.append((o, a, b))
    areas = np.array([np.linalg.norm(np.cross(a, b)) for _, a, b in faces])
    out = []
    for (o, a, b), ar in zip(faces, areas):
        n_face = max(1, budget * ar / areas.sum())
        la, lb = np.linalg.norm(a), np.linalg.norm(b)
        na = max(1, int(round(math.sqrt(n_face * la / lb))))
        nb = max(1, int(round(n_face / na)))
        out.extend(_grid_patches(o, a, b, na, nb))
    return out


def _cylinder_nets(radius, height, budget):
    side_area = 2 * np.pi * radius * height
    cap_area = np.pi * radius ** 2
    total = side_area + 2 * cap_area
    n_side = max(4, budget * side_area / total)
    # arc segments of at most 90 degrees, roughly square side patches
    n_th = max(4, 4 * int(round(math.sqrt(n_side * 2 * np.pi * radius / height) / 4)))
    n_z = max(1, int(round(n_side / n_th)))
    out = []
    s4 = np.arange(4) / 3.0
    for k in range(n_th):
        t0 = 2 * np.pi * k / n_th
        t1 = 2 * np.pi * (k + 1) / n_th
        half = 0.5 * (t1 - t0)
        tm = 0.5 * (t0 + t1)
        arc = np.array([[math.cos(t0), math.sin(t0)],
                        [math.cos(tm) / math.cos(half), math.sin(tm) / math.cos(half)],
                        [math.cos(t1), math.sin(t1)]]) * radius
        wa = np.array([1.0, math.cos(half), 1.0])
        hom = np.concatenate([arc * wa[:, None], wa[:, None]], axis=1)
        hom3 = _elevate_quadratic(hom)
        xy = hom3[:, :2] / hom3[:, 2:3]
        w3 = hom3[:, 2]
        for m in range(n_z):
            z = -0.5 * height + height * (m + s4) / n_z
            net = np.zeros((4, 4, 3))
            net[:, :, 0:2] = xy[:, None, :]
            net[:, :, 2] = z[None, :]
            out.append((net, np.repeat(w3[:, None], 4, axis=1)))
    # caps: square cells whose centre lies inside the disc
    n_cap = max(1, budget * cap_area / total)
    nc = max(2, int(round(math.sqrt(n_cap * 4 / np.pi))))
    cell = 2 * radius / nc
    for sgn in (-1.0, 1.0):
        for i in range(nc):
            for j in range(nc):
                cx = -radius + (i + 0.5) * cell
                cy = -radius + (j + 0.5) * cell
                if cx * cx + cy * cy > radius * radius:
                    continue
                o = np.array([-radius + i * cell, -radius + j * cell, sgn * 0.5 * height])
                a = np.array([cell, 0.0, 0.0])
                b = np.array([0.0, cell, 0.0])
                if sgn < 0:
                    a, b = b, a
                out.extend(_grid_patches(o, a, b, 1, 1))
    return out


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def cad_3d(seed: int, n_patches: int, n_queries: int = 0) -> Tuple[List[Patch], np.ndarray]:
    rng = np.random.default_rng(seed)
    n_solids = int(rng.integers(3, 9))
    kinds = rng.uniform(size=n_solids) < 0.5       # True: box, False: cylinder
    dims = rng.uniform(0.3, 1.0, size=(n_solids, 3))
    areas = np.where(kinds, 2 * (dims[:, 0] * dims[:, 1] + dims[:, 1] * dims[:, 2] + dims[:, 0] * dims[:, 2]),
                     2 * np.pi * (0.5 * dims[:, 0]) * dims[:, 2] + 2 * np.pi * (0.5 * dims[:, 0]) ** 2)
    budgets = n_patches * areas / areas.sum()
    patches: List[Patch] = []
    for k in range(n_solids):
        nets = _box_nets(dims[k], budgets[k]) if kinds[k] else _cylinder_nets(0.5 * dims[k, 0], dims[k, 2], budgets[k])
        R = _random_rotation(rng)
        t = rng.uniform(-0.5, 0.5, 3)
        freq = rng.normal(0, 3.0, size=(3, 3))
        phase = rng.uniform(0, 2 * np.pi, 3)
        amp = 0.01 * float(dims[k].mean())
        for net, w in nets:
            x = net @ R.T + t
            disp = amp * np.sin(x @ freq.T + phase)     # smooth perturbation field
            x = x + disp
            ww = w * rng.uniform(0.8, 1.2, size=w.shape)
            patches.append(Patch(3, 3, x, ww, bezier_knots(3), bezier_knots(3), _cad_trims(rng)))
    q = np.zeros((0, 3))
    if n_queries > 0:
        lo, hi = _bbox(np.concatenate([p.ctrl.reshape(-1, 3) for p in patches]))
        q = uniform_queries(lo, hi, n_queries, rng)
    return patches, q


@dataclass
class CadModelSpec:
    seed: int
    n_patches: int
    n_queries: int


def cad_batch_specs(seed: int = BASE_SEED + 4, n_models: int = 16) -> List[CadModelSpec]:
    rng = np.random.default_rng(seed)
    n_p = np.exp(rng.uniform(math.log(1000), math.log(40000), n_models)).astype(int)
    n_q = np.exp(rng.uniform(math.log(65536), math.log(4194304), n_models)).astype(int)
    return [CadModelSpec(seed * 100 + m, int(n_p[m]), int(n_q[m])) for m in range(n_models)]


def cad_batch_3d(seed: int = BASE_SEED + 4, n_models: int = 16, query_scale: float = 1.0,
                 patch_scale: float = 1.0):
    """List of (patches, queries) for the batched workload (optionally scaled down)."""
    out = []
    for spec in cad_batch_specs(seed, n_models):
        npch = max(50, int(spec.n_patches * patch_scale))
        nq = max(64, int(spec.n_queries * query_scale))
        out.append(cad_3d(spec.seed, npch, nq))
    return out


# ------------------------------------------------------------------ serving workload


def serve_models(seed: int = BASE_SEED + 5, cad_patches: Tuple[int, ...] = (1500, 4000, 9000, 17000)):
    """The 8 resident models of the serving workload: list of (dim, primitives, box lo, box hi)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(2):
        curves, _ = loops_2d(seed=int(rng.integers(1 << 30)), res=2)
        lo, hi = _bbox(np.concatenate([c.ctrl for c in curves]))
        out.append((2, curves, lo, hi))
    for k in range(2):
        patches, _ = sphere_3d(seed=int(rng.integers(1 << 30)), n_queries=1)
        lo, hi = _bbox(np.concatenate([p.ctrl.reshape(-1, 3) for p in patches]))
        out.append((3, patches, lo, hi))
    for npch in cad_patches:
        patches, _ = cad_3d(int(rng.integers(1 << 30)), npch)
        lo, hi = _bbox(np.concatenate([p.ctrl.reshape(-1, 3) for p in patches]))
        out.append((3, patches, lo, hi))
    return out


def serve_trace(rate_per_s: float, duration_s: float, n_models: int = 8, seed: int = BASE_SEED + 6,
                median: int = 16384, sigma: float = 1.5, lo: int = 1000, hi: int = 2000000):
    """Open-loop request trace: arrays (arrival time s, model index, n points)."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate_per_s * duration_s))
    t = np.sort(rng.uniform(0.0, duration_s, n))
    model = rng.integers(0, n_models, n)
    size = np.clip(np.exp(rng.normal(math.log(median), sigma, n)), lo, hi).astype(np.int64)
    return t, model, size
