"""Pins of the oracle's near-boundary flag and of its curve evaluator.

Every label check of the GPU tests exempts the queries that the oracle flags
as near the geometry (FLAG_NEAR, set when a query lies within `near_thr` of a
primitive): the rounded containment decision is not unique next to the
boundary, where the winding number jumps by one (Section 4.3).  A mistake in
that flag -- a threshold off by a factor, or a proxy that flags every query
inside a primitive's box -- would silently widen the exemption, so the flag is
pinned here against exact distances to shapes whose distance function is known
in closed form:

* 2D: a rational-quadratic circle (distance | |q - c| - r |) and the end of
  a straight segment (distance to the endpoint);
* 3D: a trimmed planar disc seen on its axis (distance |h| to the plane), a
  planar patch seen in its own plane past an edge and past a corner, and the
  exact rational sphere (distance | |q| - R |, queries inside the patch's box).

The flag is conservative by construction (the oracle subdivides until a piece's
box is smaller than the threshold and flags a query within the threshold of
such a box, so a flagged query lies within (1 + sqrt(dim)) x the threshold of
the curve or of the untrimmed surface); the pins hold it to "set at distance <=
thr, clear at distance >= 4 thr".

The curve evaluator (or_curve_eval, a homogeneous de Boor recurrence) is pinned
against scipy's B-spline basis with rational weights.
"""
import numpy as np
import pytest

from synth import geometry as G
from tests import refgeom as R


def _near(flags):
    return (np.asarray(flags) & 1) != 0


# ----------------------------------------------------------------- 2D


@pytest.mark.parametrize("thr", [1e-3, 1e-5, 1e-7])
def test_near_flag_circle_radial_distance(oracle_lib, thr):
    c, r = np.array([0.2, -0.1]), 0.8
    rng = np.random.default_rng(11)
    theta = rng.uniform(0, 2 * np.pi, 24)
    u = np.stack([np.cos(theta), np.sin(theta)], axis=1)
    for frac, expect in ((0.0, True), (0.25, True), (0.999, True), (4.0, False), (10.0, False), (1e3, False)):
        for sgn in (1.0, -1.0):
            d = frac * thr
            q = c + (r + sgn * d) * u
            _, fl = oracle_lib.gwn2d([G.circle(c, r)], q, near_thr=thr)
            assert np.all(_near(fl) == expect), (thr, frac, sgn, fl)


def test_near_flag_segment_end(oracle_lib):
    """Past the end of a straight piece the distance is to its endpoint."""
    thr = 1e-4
    seg = G.polyline([[0.0, 0.0], [1.0, 0.0]], closed=False)
    rng = np.random.default_rng(2)
    ang = rng.uniform(-0.5 * np.pi, 0.5 * np.pi, 16)   # directions away from the segment
    dirs = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    for d, expect in ((0.5 * thr, True), (thr, True), (4 * thr, False), (50 * thr, False)):
        q = np.array([1.0, 0.0]) + d * dirs
        _, fl = oracle_lib.gwn2d([seg], q, near_thr=thr)
        assert np.all(_near(fl) == expect), (d, fl)


def test_near_flag_off_for_far_queries(oracle_lib):
    """Far from every piece nothing is flagged, whatever the box overlap."""
    curves = [G.circle((0, 0), 1.0), G.circle((0.3, 0.1), 0.4, ccw=False)]
    rng = np.random.default_rng(5)
    q = rng.uniform(-1.3, 1.3, size=(3000, 2))
    d1 = np.abs(np.linalg.norm(q, axis=1) - 1.0)
    d2 = np.abs(np.linalg.norm(q - [0.3, 0.1], axis=1) - 0.4)
    dist = np.minimum(d1, d2)
    thr = 1e-2
    _, fl = oracle_lib.gwn2d(curves, q, near_thr=thr)
    near = _near(fl)
    assert np.all(near[dist <= thr])
    assert not np.any(near[dist >= 4 * thr])
    assert near.sum() < 0.2 * q.shape[0]


# ----------------------------------------------------------------- 3D


@pytest.mark.parametrize("thr", [1e-3, 1e-6])
def test_near_flag_disc_on_axis(oracle_lib, thr):
    disc = G.planar_patch((-0.5, -0.5, 0.0), (1, 0, 0), (0, 1, 0), trims=[G.circle((0.5, 0.5), 0.3)])
    for frac, expect in ((0.0, True), (0.5, True), (1.0, True), (4.0, False), (30.0, False)):
        for sgn in (1.0, -1.0):
            h = sgn * frac * thr
            q = np.array([[0.0, 0.0, h], [0.1, -0.05, h], [0.2, 0.2, h]])
            _, fl = oracle_lib.gwn3d([disc], q, near_thr=thr)
            if frac == 0.0:
                # on the visible disc: undefined value, flagged on the boundary
                assert np.all(_near(fl) | ((fl & 2) != 0))
            else:
                assert np.all(_near(fl) == expect), (thr, frac, sgn, fl)


def test_near_flag_in_plane_past_edge_and_corner(oracle_lib):
    """In the patch's plane, outside its rectangle: the distance is to the edge
    (or to the corner), and the flag follows it."""
    thr = 1e-4
    sq = G.planar_patch((-0.5, -0.5, 0.0), (1, 0, 0), (0, 1, 0))
    for d, expect in ((0.5 * thr, True), (thr, True), (4 * thr, False), (40 * thr, False)):
        q = np.array([[0.5 + d, 0.0, 0.0], [0.0, -0.5 - d, 0.0], [-0.5 - d, 0.3, 0.0],
                      [0.5 + d / np.sqrt(2), 0.5 + d / np.sqrt(2), 0.0]])
        _, fl = oracle_lib.gwn3d([sq], q, near_thr=thr)
        assert np.all(_near(fl) == expect), (d, fl)


@pytest.mark.parametrize("thr", [1e-3, 1e-5])
def test_near_flag_sphere_inside_its_box(oracle_lib, thr):
    """Queries inside the sphere patch's box at a known distance | |q| - R |:
    the proxy flags the near ones only, so it does not flag a whole box."""
    sph = G.nurbs_sphere((0, 0, 0), 1.0)
    rng = np.random.default_rng(3)
    d = rng.normal(size=(40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    for frac, expect in ((0.5, True), (1.0, True), (4.0, False), (20.0, False)):
        for sgn in (1.0, -1.0):
            q = (1.0 + sgn * frac * thr) * d
            _, fl = oracle_lib.gwn3d([sph], q, near_thr=thr)
            assert np.all(_near(fl) == expect), (thr, frac, sgn, fl)
    # deep inside (distance >= 0.2) nothing is flagged, though every point is in the box
    q = 0.8 * rng.uniform(-1, 1, size=(200, 3)) / np.sqrt(3)
    _, fl = oracle_lib.gwn3d([sph], q, near_thr=thr)
    assert not np.any(_near(fl))


# ----------------------------------------------------------------- curve evaluator


def test_curve_eval_matches_scipy_bspline(oracle_lib):
    rng = np.random.default_rng(17)
    curves = [G.circle((0.3, -0.4), 1.7), G.polyline(rng.uniform(-1, 1, (7, 2)))]
    for p, n in ((1, 5), (2, 6), (3, 9), (3, 4), (2, 3)):
        knots = np.concatenate([np.zeros(p + 1), np.sort(rng.uniform(0.05, 0.95, n - p - 1)), np.ones(p + 1)])
        curves.append(G.Curve(p, rng.uniform(-2, 2, (n, 2)), rng.uniform(0.3, 3.0, n), knots))
    # a knot vector with a repeated interior knot and a range other than [0, 1]
    curves.append(G.Curve(3, rng.uniform(-1, 1, (8, 2)), rng.uniform(0.5, 2.0, 8),
                          np.array([2, 2, 2, 2, 2.4, 2.4, 3.1, 3.5, 5, 5, 5, 5.0])))
    for c in curves:
        a, b = c.knots[0], c.knots[-1]
        t = np.concatenate([[a, b], rng.uniform(a, b, 60), np.unique(c.knots)])
        got = oracle_lib.curve_eval(c, t)
        ref, _ = R.curve_point_deriv(c, t)
        np.testing.assert_allclose(got, ref, atol=1e-12, rtol=0)
