"""Test-side geometry helpers that pin the oracle against independent routines.

Nothing here is used by the oracle or by the CUDA path.  NURBS evaluation goes
through scipy's B-spline implementation (a library routine), solid angles of
triangles use the Van Oosterom-Strackee formula (IEEE Trans. Biomed. Eng.
1983), polygon winding uses the classical crossing rule, and brute-force
integrals use scipy quadrature or plain Gauss-Legendre products.
"""
from __future__ import annotations

import numpy as np
from scipy.interpolate import BSpline


def _basis(knots, degree, x, nu=0):
    n = len(knots) - degree - 1
    spl = BSpline(knots, np.eye(n), degree, extrapolate=False)
    if nu:
        spl = spl.derivative(nu)
    x = np.clip(np.asarray(x, dtype=np.float64), knots[degree], knots[n] - 1e-300)
    out = spl(x)
    return np.nan_to_num(out)


def curve_point_deriv(c, t):
    """C(t), C'(t) of a NURBS curve via scipy B-spline bases (homogeneous form)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    end = c.knots[-1]
    tt = np.where(t >= end, end - 1e-14 * (end - c.knots[0]), t)
    B = _basis(c.knots, c.degree, tt)
    dB = _basis(c.knots, c.degree, tt, 1)
    H = B @ (c.ctrl * c.weights[:, None])
    W = B @ c.weights
    dH = dB @ (c.ctrl * c.weights[:, None])
    dW = dB @ c.weights
    P = H / W[:, None]
    dP = (dH - P * dW[:, None]) / W[:, None]
    return P, dP


def surface_point_derivs(p, u, v):
    """S, S_u, S_v of a NURBS patch at arrays u, v via scipy B-spline bases."""
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))
    eu = p.knots_u[-1] - 1e-14 * (p.knots_u[-1] - p.knots_u[0])
    ev = p.knots_v[-1] - 1e-14 * (p.knots_v[-1] - p.knots_v[0])
    u = np.minimum(u, eu)
    v = np.minimum(v, ev)
    Bu, dBu = _basis(p.knots_u, p.deg_u, u), _basis(p.knots_u, p.deg_u, u, 1)
    Bv, dBv = _basis(p.knots_v, p.deg_v, v), _basis(p.knots_v, p.deg_v, v, 1)
    HW = np.concatenate([p.ctrl * p.weights[..., None], p.weights[..., None]], axis=-1)  # nu, nv, 4
    H = np.einsum("ni,nj,ijk->nk", Bu, Bv, HW)
    Hu = np.einsum("ni,nj,ijk->nk", dBu, Bv, HW)
    Hv = np.einsum("ni,nj,ijk->nk", Bu, dBv, HW)
    S = H[:, :3] / H[:, 3:]
    Su = (Hu[:, :3] - S * Hu[:, 3:]) / H[:, 3:]
    Sv = (Hv[:, :3] - S * Hv[:, 3:]) / H[:, 3:]
    return S, Su, Sv


def crossing_winding(poly, q):
    """Classical crossing-rule winding number of a closed polygon around q."""
    poly = np.asarray(poly, dtype=np.float64)
    wn = 0
    n = len(poly)
    for i in range(n):
        a, b = poly[i], poly[(i + 1) % n]
        isl = (b[0] - a[0]) * (q[1] - a[1]) - (q[0] - a[0]) * (b[1] - a[1])
        if a[1] <= q[1]:
            if b[1] > q[1] and isl > 0:
                wn += 1
        else:
            if b[1] <= q[1] and isl < 0:
                wn -= 1
    return wn


def triangle_solid_angle(a, b, c, q):
    """Signed solid angle of triangle abc seen from q (Van Oosterom-Strackee)."""
    R1, R2, R3 = (np.asarray(x, dtype=np.float64) - q for x in (a, b, c))
    r1, r2, r3 = (np.linalg.norm(x) for x in (R1, R2, R3))
    num = np.dot(R1, np.cross(R2, R3))
    den = r1 * r2 * r3 + np.dot(R1, R2) * r3 + np.dot(R1, R3) * r2 + np.dot(R2, R3) * r1
    return 2.0 * np.arctan2(num, den)


def gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def bezier_split_curve(c, s):
    """de Casteljau split of a single-span rational Bezier curve at s (test-side)."""
    from synth.geometry import Curve, bezier_knots
    H = np.concatenate([c.ctrl * c.weights[:, None], c.weights[:, None]], axis=1)
    p = c.degree
    L, R = [H[0].copy()], [H[p].copy()]
    T = H.copy()
    for j in range(1, p + 1):
        T = (1 - s) * T[:-1] + s * T[1:]
        L.append(T[0].copy())
        R.append(T[-1].copy())
    L = np.array(L)
    R = np.array(R[::-1])
    mk = lambda A: Curve(p, A[:, :2] / A[:, 2:], A[:, 2], bezier_knots(p))
    return mk(L), mk(R)


def bezier_split_patch_u(pt, s):
    """Split a single-span rational Bezier patch at u = s into two untrimmed patches."""
    from synth.geometry import Patch, bezier_knots
    HW = np.concatenate([pt.ctrl * pt.weights[..., None], pt.weights[..., None]], axis=-1)
    p = pt.deg_u
    L, R = [HW[0].copy()], [HW[p].copy()]
    T = HW.copy()
    for j in range(1, p + 1):
        T = (1 - s) * T[:-1] + s * T[1:]
        L.append(T[0].copy())
        R.append(T[-1].copy())
    L = np.array(L)
    R = np.array(R[::-1])
    mk = lambda A: Patch(p, pt.deg_v, A[..., :3] / A[..., 3:], A[..., 3], bezier_knots(p), pt.knots_v.copy(), [])
    return mk(L), mk(R)
