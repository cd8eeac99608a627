"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

The oracle computes the exact generalized winding number (Eq. 1, Eq. 2;
direct evaluation of Section 4.2).  Each test checks it against something
that is not the oracle itself: closed forms, the classical polygon winding
number, integer winding on closed curves and shells, additivity and
reversal, the unit jump across the boundary (Section 4.3), scipy-based
brute-force quadrature, the divergence theorem for the moments of
Section 3.1, and the decay rate of the Taylor remainder of Eq. 3.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from synth import geometry as G
from synth import configs
from tests import refgeom as R


# ----------------------------------------------------------------- 2D


def test_polygon_matches_crossing_rule(oracle_lib):
    rng = np.random.default_rng(7)
    for trial in range(6):
        nv = int(rng.integers(3, 12))
        poly = rng.uniform(-1, 1, size=(nv, 2))          # possibly self-intersecting
        q = rng.uniform(-1.2, 1.2, size=(200, 2))
        w, fl = oracle_lib.gwn2d([G.polyline(poly)], q)
        ref = np.array([R.crossing_winding(poly, x) for x in q])
        assert np.all(fl == 0)
        np.testing.assert_allclose(w, ref, atol=1e-12)


def test_circle_integer_and_orientation(oracle_lib):
    rng = np.random.default_rng(1)
    c, r = np.array([0.3, -0.2]), 0.7
    q = rng.uniform(-1.5, 1.5, size=(400, 2))
    d = np.linalg.norm(q - c, axis=1)
    q = q[np.abs(d - r) > 1e-3]
    d = np.linalg.norm(q - c, axis=1)
    w, _ = oracle_lib.gwn2d([G.circle(c, r)], q)
    np.testing.assert_allclose(w, (d < r).astype(float), atol=1e-12)
    w2, _ = oracle_lib.gwn2d([G.circle(c, r, ccw=False)], q)
    np.testing.assert_allclose(w2, -(d < r).astype(float), atol=1e-12)


def test_arc_from_centre_is_angle_over_2pi(oracle_lib):
    for t0, t1 in [(0.1, 1.3), (-2.0, 0.5), (2.0, 4.5)]:
        w, _ = oracle_lib.gwn2d([G.arc((0.4, 0.1), 0.8, t0, t1)], np.array([[0.4, 0.1]]))
        assert abs(w[0] - (t1 - t0) / (2 * math.pi)) < 1e-14


def _brute_curve(c, q):
    """(1/2pi) int (C - q) x C' / |C - q|^2 dt over each knot span (scipy quad)."""
    br = np.unique(c.knots)
    acc = 0.0
    for a, b in zip(br[:-1], br[1:]):
        def f(t):
            P, dP = R.curve_point_deriv(c, t)
            r = P[0] - q
            return (r[0] * dP[0, 1] - r[1] * dP[0, 0]) / (r @ r)
        val, err = integrate.quad(f, a, b, epsabs=1e-15, epsrel=1e-14, limit=400)
        acc += val
    return acc / (2 * math.pi)


def test_bruteforce_quadrature_2d(oracle_lib):
    rng = np.random.default_rng(3)
    curves = [
        G.Curve(3, rng.uniform(-1, 1, (6, 2)), rng.uniform(0.5, 2.0, 6), G.clamped_uniform_knots(6, 3)),
        G.Curve(2, rng.uniform(-1, 1, (5, 2)), rng.uniform(0.5, 2.0, 5), np.array([0, 0, 0, .3, .3, 1, 1, 1.])),
        G.bezier_curve(rng.uniform(-1, 1, (4, 2)), [1.0, 0.6, 1.7, 1.0]),
    ]
    q = rng.uniform(-2.0, 2.0, size=(12, 2))
    for c in curves:
        w, fl = oracle_lib.gwn2d([c], q)
        ref = np.array([_brute_curve(c, x) for x in q])
        assert np.all(fl == 0)
        np.testing.assert_allclose(w, ref, atol=1e-11)


def test_additivity_and_reversal_2d(oracle_lib):
    rng = np.random.default_rng(5)
    q = rng.uniform(-1.5, 1.5, size=(300, 2))
    for _ in range(4):
        c = G.bezier_curve(rng.uniform(-1, 1, (4, 2)), rng.uniform(0.5, 2.0, 4))
        L, Rr = R.bezier_split_curve(c, float(rng.uniform(0.2, 0.8)))
        each = oracle_lib.gwn2d_each([c, L, Rr, c.reversed()], q)
        np.testing.assert_allclose(each[:, 0], each[:, 1] + each[:, 2], atol=1e-12)
        np.testing.assert_allclose(each[:, 3], -each[:, 0], atol=1e-12)


def test_unit_jump_across_curve(oracle_lib):
    c, _ = configs.star_2d(n_queries=16)
    ts = np.linspace(0.1, 0.9, 7)
    for k in (0, 17, 40):
        P, dP = R.curve_point_deriv(c[k], ts)
        n = np.stack([dP[:, 1], -dP[:, 0]], axis=1)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        eps = 1e-7
        w_out, _ = oracle_lib.gwn2d(c, P + eps * n)
        w_in, _ = oracle_lib.gwn2d(c, P - eps * n)
        np.testing.assert_allclose(w_in - w_out, 1.0, atol=1e-5)


def test_nonclamped_knots_rejected(oracle_lib):
    bad = G.Curve(2, np.zeros((4, 2)), np.ones(4), np.array([0, 0.1, 0.2, 0.3, 0.7, 0.8, 1.0]))
    with pytest.raises(ValueError):
        oracle_lib.gwn2d([bad], np.zeros((1, 2)))


# ----------------------------------------------------------------- 3D


def _disk(R_, trims_ccw=True):
    return G.planar_patch((-0.5, -0.5, 0.0), (1, 0, 0), (0, 1, 0),
                          trims=[G.circle((0.5, 0.5), R_, ccw=trims_ccw)])


def test_disk_on_axis_closed_form(oracle_lib):
    Rd = 0.3
    hs = np.array([2.0, 0.7, 0.1, 1e-3, 1e-6, -1e-6, -0.05, -0.4, -3.0])
    q = np.stack([np.zeros_like(hs), np.zeros_like(hs), hs], axis=1)
    w, fl = oracle_lib.gwn3d([_disk(Rd)], q)
    # normal +z: points above see the back face (negative solid angle)
    exact = -np.sign(hs) * 0.5 * (1 - np.abs(hs) / np.sqrt(hs * hs + Rd * Rd))
    np.testing.assert_allclose(w, exact, atol=1e-12)
    w2, _ = oracle_lib.gwn3d([_disk(Rd).flipped()], q)
    np.testing.assert_allclose(w2, -exact, atol=1e-12)


def test_planar_polygon_solid_angle(oracle_lib):
    rng = np.random.default_rng(11)
    o, a, b = np.array([0.2, -0.1, 0.3]), np.array([1.1, 0.2, -0.1]), np.array([-0.2, 0.9, 0.4])
    th = np.sort(rng.uniform(0, 2 * np.pi, 7))
    uv = np.stack([0.5 + 0.4 * np.cos(th), 0.5 + 0.4 * np.sin(th)], axis=1)
    patch = G.planar_patch(o, a, b, trims=[G.polyline(uv)])
    verts = o + uv[:, :1] * a + uv[:, 1:] * b
    q = rng.uniform(-1.0, 2.0, size=(60, 3))
    w, fl = oracle_lib.gwn3d([patch], q)
    ref = np.array([sum(R.triangle_solid_angle(verts[0], verts[i], verts[i + 1], x)
                        for i in range(1, len(verts) - 1)) for x in q]) / (4 * math.pi)
    np.testing.assert_allclose(w, ref, atol=1e-11)


def test_closed_shells_integer(oracle_lib):
    rng = np.random.default_rng(2)
    q = rng.uniform(-1.6, 1.6, size=(120, 3))
    cube = G.cube_shell(half=1.0)
    w, fl = oracle_lib.gwn3d(cube, q)
    inside = np.all(np.abs(q) < 1.0, axis=1)
    ok = np.all(np.abs(np.abs(q) - 1.0) > 1e-3, axis=1)
    np.testing.assert_allclose(w[ok], inside[ok].astype(float), atol=1e-10)
    sph = G.nurbs_sphere(center=(0.1, 0.0, -0.1), radius=1.2)
    d = np.linalg.norm(q - np.array([0.1, 0.0, -0.1]), axis=1)
    keep = np.abs(d - 1.2) > 1e-3
    w, fl = oracle_lib.gwn3d([sph], q[keep])
    np.testing.assert_allclose(w, (d[keep] < 1.2).astype(float), atol=1e-10)


def test_trimmed_face_split_stays_watertight(oracle_lib):
    """Cube whose +z face is cut into a trimmed polygon and its complement."""
    cube = G.cube_shell(half=1.0)
    top = cube[5]
    hole = np.array([[0.3, 0.2], [0.7, 0.3], [0.6, 0.75], [0.25, 0.6]])
    inner = G.Patch(top.deg_u, top.deg_v, top.ctrl, top.weights, top.knots_u, top.knots_v,
                    [G.polyline(hole)])
    outer = G.Patch(top.deg_u, top.deg_v, top.ctrl, top.weights, top.knots_u, top.knots_v,
                    [G.polyline([[0, 0], [1, 0], [1, 1], [0, 1]]), G.polyline(hole[::-1])])
    shell = cube[:5] + [inner, outer]
    rng = np.random.default_rng(9)
    q = rng.uniform(-1.5, 1.5, size=(80, 3))
    q = q[np.all(np.abs(np.abs(q) - 1.0) > 1e-3, axis=1)]
    w, fl = oracle_lib.gwn3d(shell, q)
    np.testing.assert_allclose(w, np.all(np.abs(q) < 1, axis=1).astype(float), atol=1e-10)


def _brute_patch(p, q, n=24, nsub=4):
    """Solid-angle integrand over the visible region (scipy bases).

    Untrimmed patches: tensor Gauss-Legendre on every knot-span rectangle.
    Trimmed (single-span) patches: fan cubature from the domain centre."""
    x, w = R.gl01(n)
    if not p.trims:
        acc = 0.0
        bu, bv = np.unique(p.knots_u), np.unique(p.knots_v)
        for u0, u1 in zip(bu[:-1], bu[1:]):
            for v0, v1 in zip(bv[:-1], bv[1:]):
                U, V = np.meshgrid(u0 + (u1 - u0) * x, v0 + (v1 - v0) * x, indexing="ij")
                S, Su, Sv = R.surface_point_derivs(p, U.ravel(), V.ravel())
                r = S - q
                f = np.einsum("ij,ij->i", r, np.cross(Su, Sv)) / np.linalg.norm(r, axis=1) ** 3
                acc += (u1 - u0) * (v1 - v0) * np.sum(np.outer(w, w).ravel() * f)
        return acc / (4 * math.pi)
    loops = p.trims
    c = np.array([0.5 * (p.knots_u[0] + p.knots_u[-1]), 0.5 * (p.knots_v[0] + p.knots_v[-1])])
    acc = 0.0
    for cur in loops:
        br = np.unique(cur.knots)
        for a0, b0 in zip(br[:-1], br[1:]):
            for k in range(nsub):
                ta = a0 + (b0 - a0) * (k + x) / nsub
                wt = w * (b0 - a0) / nsub
                g, dg = R.curve_point_deriv(cur, ta)
                jac = (g[:, 0] - c[0]) * dg[:, 1] - (g[:, 1] - c[1]) * dg[:, 0]
                for m in range(nsub):
                    sg = (m + x) / nsub
                    ws = w / nsub
                    U = c[0] + sg[None, :] * (g[:, :1] - c[0])
                    V = c[1] + sg[None, :] * (g[:, 1:] - c[1])
                    S, Su, Sv = R.surface_point_derivs(p, U.ravel(), V.ravel())
                    nrm = np.cross(Su, Sv)
                    r = S - q
                    f = np.einsum("ij,ij->i", r, nrm) / np.linalg.norm(r, axis=1) ** 3
                    f = f.reshape(U.shape)
                    acc += np.sum(wt[:, None] * ws[None, :] * sg[None, :] * jac[:, None] * f)
    return acc / (4 * math.pi)


def test_bruteforce_cubature_3d(oracle_lib):
    patches, _ = configs.sphere_3d(n_queries=8)
    cads, _ = configs.cad_3d(99, 60)
    rng = np.random.default_rng(4)
    for p in [patches[3], patches[200], cads[5], cads[17], G.nurbs_sphere(radius=0.5)]:
        lo = p.ctrl.reshape(-1, 3).min(0)
        hi = p.ctrl.reshape(-1, 3).max(0)
        diag = np.linalg.norm(hi - lo)
        c = 0.5 * (lo + hi)
        dirs = rng.normal(size=(4, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        q = c + dirs * diag * rng.uniform(0.6, 1.5, size=(4, 1))
        w, fl = oracle_lib.gwn3d([p], q)
        ref = np.array([_brute_patch(p, x) for x in q])
        np.testing.assert_allclose(w, ref, atol=1e-11)


def test_patch_additivity_and_reversal(oracle_lib):
    patches, _ = configs.sphere_3d(n_queries=8)
    base = patches[11]
    untrimmed = G.Patch(3, 3, base.ctrl, base.weights, base.knots_u, base.knots_v, [])
    L, Rr = R.bezier_split_patch_u(untrimmed, 0.37)
    rng = np.random.default_rng(8)
    lo, hi = untrimmed.ctrl.reshape(-1, 3).min(0), untrimmed.ctrl.reshape(-1, 3).max(0)
    q = rng.uniform(lo - 0.2, hi + 0.2, size=(30, 3))
    each = oracle_lib.gwn3d_each([untrimmed, L, Rr, base, base.flipped()], q)
    np.testing.assert_allclose(each[:, 0], each[:, 1] + each[:, 2], atol=1e-11)
    np.testing.assert_allclose(each[:, 4], -each[:, 3], atol=1e-11)


def test_trim_loop_additivity(oracle_lib):
    o, a, b = np.array([0, 0, 0.0]), np.array([1, 0.1, 0.2]), np.array([0, 1, -0.3])
    outer = G.polyline([[0.1, 0.1], [0.9, 0.15], [0.85, 0.9], [0.1, 0.8]])
    hole_ccw = G.circle((0.45, 0.5), 0.15)
    hole_cw = G.circle((0.45, 0.5), 0.15, ccw=False)
    pD = G.planar_patch(o, a, b, [outer])
    pDH = G.planar_patch(o, a, b, [outer, hole_cw])
    pH = G.planar_patch(o, a, b, [hole_ccw])
    rng = np.random.default_rng(12)
    q = rng.uniform(-0.5, 1.5, size=(40, 3))
    each = oracle_lib.gwn3d_each([pD, pDH, pH], q)
    np.testing.assert_allclose(each[:, 0], each[:, 1] + each[:, 2], atol=1e-11)


def test_unit_jump_across_patch(oracle_lib):
    patches, _ = configs.sphere_3d(n_queries=8)
    p = patches[40]
    ctr = p.trims[0].ctrl[:-1].mean(axis=0)           # centre of the disc trim
    uv = ctr + 0.05 * np.array([[0, 0], [1, 0], [0, -1], [0.7, 0.7]])
    S, Su, Sv = R.surface_point_derivs(p, uv[:, 0], uv[:, 1])
    n = np.cross(Su, Sv)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    eps = 1e-7
    w_out, _ = oracle_lib.gwn3d(patches, S + eps * n)
    w_in, _ = oracle_lib.gwn3d(patches, S - eps * n)
    np.testing.assert_allclose(w_in - w_out, 1.0, atol=1e-5)


# ----------------------------------------------------------------- moments and Eq. 3


def test_moments_divergence_theorem_2d(oracle_lib):
    rng = np.random.default_rng(21)
    poly = np.array([[0, 0], [2, 0.3], [1.6, 1.4], [0.4, 1.1], [-0.3, 0.6]], dtype=float)
    seg = np.concatenate([poly, np.roll(poly, -1, axis=0)], axis=1)
    area = 0.5 * np.sum(poly[:, 0] * np.roll(poly[:, 1], -1) - np.roll(poly[:, 0], -1) * poly[:, 1])
    x0 = rng.uniform(-1, 1, 2)
    m = oracle_lib.segment_moments(seg, x0)
    np.testing.assert_allclose(m["m0"], 0, atol=1e-13)
    np.testing.assert_allclose(m["m1"], area * np.eye(2), atol=1e-12)
    # m2_ijk = delta_ik int (x - x0)_j + delta_jk int (x - x0)_i  (divergence theorem)
    cx = np.array([np.sum((poly[:, 0] + np.roll(poly[:, 0], -1)) * (poly[:, 0] * np.roll(poly[:, 1], -1) - np.roll(poly[:, 0], -1) * poly[:, 1])),
                   np.sum((poly[:, 1] + np.roll(poly[:, 1], -1)) * (poly[:, 0] * np.roll(poly[:, 1], -1) - np.roll(poly[:, 0], -1) * poly[:, 1]))]) / 6.0
    mx = cx - area * x0
    ref = np.einsum("ik,j->ijk", np.eye(2), mx) + np.einsum("jk,i->ijk", np.eye(2), mx)
    np.testing.assert_allclose(m["m2"], ref, atol=1e-12)


def test_moments_divergence_theorem_3d(oracle_lib):
    x0 = np.array([0.3, -0.2, 0.1])
    tot = {k: 0 for k in ("m0", "m1", "m2")}
    for p in G.cube_shell(center=(0.1, 0.2, -0.3), half=0.7):
        m = oracle_lib.patch_moments(p, x0, nsub=1)
        for k in tot:
            tot[k] = tot[k] + m[k]
    V = 1.4 ** 3
    mx = V * (np.array([0.1, 0.2, -0.3]) - x0)
    np.testing.assert_allclose(tot["m0"], 0, atol=1e-12)
    np.testing.assert_allclose(tot["m1"], V * np.eye(3), atol=1e-12)
    ref = np.einsum("ik,j->ijk", np.eye(3), mx) + np.einsum("jk,i->ijk", np.eye(3), mx)
    np.testing.assert_allclose(tot["m2"], ref, atol=1e-12)
    # exact sphere: volume 4/3 pi r^3, area 4 pi r^2
    sph = G.nurbs_sphere(center=(0, 0, 0), radius=0.8)
    m = oracle_lib.patch_moments(sph, np.zeros(3), nsub=6)
    np.testing.assert_allclose(m["m1"], 4 / 3 * math.pi * 0.8 ** 3 * np.eye(3), atol=1e-9)
    assert abs(m["area"] - 4 * math.pi * 0.8 ** 2) < 1e-9


def test_open_disk_moment_is_area_normal(oracle_lib):
    m = oracle_lib.patch_moments(_disk(0.3), np.zeros(3), nsub=4)
    np.testing.assert_allclose(m["m0"], [0, 0, math.pi * 0.09], atol=1e-12)
    assert abs(m["area"] - math.pi * 0.09) < 1e-12


def test_taylor_of_closed_shell_vanishes(oracle_lib):
    x0 = np.array([0.3, -0.2, 0.1])
    tot = {k: 0 for k in ("m0", "m1", "m2")}
    for p in G.cube_shell(center=(0.0, 0.0, 0.0), half=0.5):
        m = oracle_lib.patch_moments(p, x0, nsub=1)
        for k in tot:
            tot[k] = tot[k] + m[k]
    for q in ([3.0, 1.0, -2.0], [0.0, 5.0, 0.5]):
        assert abs(oracle_lib.taylor(3, 2, x0, tot["m0"], tot["m1"], tot["m2"], np.array(q))) < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_taylor_remainder_decay(oracle_lib, dim):
    """Order-k truncation error falls like rho^-(k+dim) (Eq. 3 with correct tensors)."""
    if dim == 2:
        arcs = [G.arc((0.1, -0.05), 0.3, 0.2, 1.9)]
        x0 = np.array([0.05, 0.1])
        # moments of the chord, the paper's 2D substitution
        P = R.curve_point_deriv(arcs[0], [0.0, 1.0])[0]
        m = oracle_lib.segment_moments(np.concatenate([P[0], P[1]])[None, :], x0)
        exact_fn = lambda q: oracle_lib.gwn2d(arcs, q[None, :])[0][0]
        direction = np.array([0.6, 0.8])
    else:
        patch = configs.sphere_3d(n_queries=4)[0][3]      # curved, trimmed bicubic patch
        x0 = patch.ctrl.reshape(-1, 3).mean(0) + np.array([0.02, -0.01, 0.015])
        m = oracle_lib.patch_moments(patch, x0, nsub=4)
        exact_fn = lambda q: oracle_lib.gwn3d([patch], q[None, :])[0][0]
        direction = np.array([0.48, 0.6, 0.64])
    for order in (0, 1, 2):
        errs = []
        for rho in (8.0, 16.0):
            q = x0 + rho * direction
            errs.append(abs(oracle_lib.taylor(dim, order, x0, m["m0"], m["m1"], m["m2"], q) - exact_fn(q)))
        rate = math.log2(errs[0] / errs[1])
        assert abs(rate - (order + dim)) < 0.35, (order, errs, rate)
