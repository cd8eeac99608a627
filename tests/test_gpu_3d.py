"""GPU parity of the 3D path (trimmed NURBS patches) against the FP64 oracle.

Acceptance: max |dGWN| <= 1e-4 on the FP32-bulk path, the all-FP64 direct sum at
<= 1e-9 (the repair, whose panels are coarser, at <= 1e-6),
and rounded containment identical away from the surface (1e-6 of the box
diagonal) and away from half-integers (Section 4.3).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_19200_gb300 as gwn
from paper_2605_19200_gb300 import api
from synth import configs
from synth import geometry as G

HALF_BAND = 1e-6


def _diag(patches):
    lo, hi = G.shape_bbox_3d(patches)
    return float(np.linalg.norm(hi - lo))


def _labels_ok(w, w_ref, near):
    keep = (~near) & (np.abs((w_ref - np.floor(w_ref)) - 0.5) > HALF_BAND)
    return np.array_equal(np.round(w[keep]).astype(int), np.round(w_ref[keep]).astype(int))


def _q(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_cube_shell_integer():
    cube = G.cube_shell(half=1.0)
    rng = np.random.default_rng(1)
    q = rng.uniform(-1.5, 1.5, size=(4000, 3))
    q = q[np.all(np.abs(np.abs(q) - 1.0) > 1e-3, axis=1)]
    inside = np.all(np.abs(q) < 1, axis=1).astype(float)
    m = gwn.gwn_build_3d(cube, beta=8.0)
    w64, _, _ = m.query(_q(q), precision=gwn.PREC_FP64, mode=gwn.MODE_DIRECT)
    assert np.max(np.abs(w64.cpu().numpy() - inside)) <= 1e-8
    w, lab, st = m.query(_q(q.astype(np.float32)))
    assert np.max(np.abs(w.cpu().numpy() - inside)) <= 1e-4
    assert np.array_equal(lab.cpu().numpy(), inside.astype(np.int32))


def test_disk_on_axis_closed_form():
    R = 0.3
    disk = G.planar_patch((-0.5, -0.5, 0.0), (1, 0, 0), (0, 1, 0), trims=[G.circle((0.5, 0.5), R)])
    hs = np.array([2.0, 0.7, 0.1, 1e-2, 1e-3, 1e-4, -1e-4, -1e-3, -0.05, -0.4, -3.0])
    q = np.stack([np.zeros_like(hs), np.zeros_like(hs), hs], axis=1)
    exact = -np.sign(hs) * 0.5 * (1 - np.abs(hs) / np.sqrt(hs * hs + R * R))
    m = gwn.gwn_build_3d([disk], max_aabb_frac=0.0)
    for prec, tol in ((gwn.PREC_FP64, 1e-9), (gwn.PREC_FP32, 1e-5)):
        w, _, _ = m.query(_q(q), precision=prec, mode=gwn.MODE_DIRECT)
        np.testing.assert_allclose(w.cpu().numpy(), exact, atol=tol)


@pytest.fixture(scope="module")
def sphere(oracle_lib):
    patches, q = configs.sphere_3d(n_queries=1 << 20)
    rng = np.random.default_rng(77)
    idx = np.sort(rng.choice(q.shape[0], size=1500, replace=False))
    # near-surface probes on both sides of random visible points
    p = patches[rng.integers(len(patches))]
    w_ref, fl = oracle_lib.gwn3d(patches, q[idx], near_thr=1e-6 * _diag(patches))
    return patches, q, idx, w_ref, fl


def test_sphere_fp64_direct(sphere):
    patches, q, idx, w_ref, fl = sphere
    m = gwn.gwn_build_3d(patches, max_aabb_frac=0.0)
    w, _, st = m.query(_q(q[idx]), precision=gwn.PREC_FP64, mode=gwn.MODE_DIRECT)
    ok = np.isfinite(w_ref)
    assert np.max(np.abs(w.cpu().numpy()[ok] - w_ref[ok])) <= 1e-9


def test_sphere_fp32_repair(sphere):
    patches, q, idx, w_ref, fl = sphere
    m = gwn.gwn_build_3d(patches, beta=6.0)
    w, lab, st = m.query(_q(q.astype(np.float32)))
    w = w.cpu().numpy()[idx]
    ok = np.isfinite(w_ref)
    err = np.abs(w[ok] - w_ref[ok])
    assert err.max() <= 1e-4, err.max()
    assert _labels_ok(w[ok], w_ref[ok], (fl[ok] & 1) != 0)


def test_sphere_near_surface(oracle_lib):
    """Queries 1e-3 .. 1e-6 of the diagonal off the surface, both sides."""
    patches, _ = configs.sphere_3d(n_queries=4)
    rng = np.random.default_rng(5)
    pts = []
    from tests import refgeom as R
    for k in rng.choice(len(patches), size=12, replace=False):
        p = patches[k]
        c = p.trims[0].ctrl[:-1].mean(axis=0)
        uv = c + 0.1 * rng.uniform(-1, 1, size=(2, 2))
        S, Su, Sv = R.surface_point_derivs(p, uv[:, 0], uv[:, 1])
        n = np.cross(Su, Sv)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        for h in (1e-3, 1e-4, 1e-5):
            pts.append(S + h * n)
            pts.append(S - h * n)
    q = np.concatenate(pts).astype(np.float32).astype(np.float64)
    w_ref, fl = oracle_lib.gwn3d(patches, q)
    m = gwn.gwn_build_3d(patches, beta=6.0)
    w, lab, st = m.query(_q(q))
    w = w.cpu().numpy()
    ok = np.isfinite(w_ref)
    assert np.max(np.abs(w[ok] - w_ref[ok])) <= 1e-4
    assert np.array_equal(np.round(w[ok]), np.round(w_ref[ok]))


@pytest.mark.parametrize("tree_builder", [1, 0])
def test_cad_model_fp32_and_direct(oracle_lib, tree_builder):
    """A CAD solid through the FP32 traversal over either hierarchy (top-down
    sweep, Karras LBVH) and through the plain FP32 direct sum, against the oracle."""
    patches, q = configs.cad_3d(1234, 400, 4000)
    w_ref, fl = oracle_lib.gwn3d(patches, q[:600], near_thr=1e-6 * _diag(patches))
    ok = np.isfinite(w_ref)
    m = gwn.gwn_build_3d(patches, beta=6.0, tree_builder=tree_builder)
    w, lab, st = m.query(_q(q))
    w = w.cpu().numpy()[:600]
    assert np.max(np.abs(w[ok] - w_ref[ok])) <= 1e-4
    assert _labels_ok(w[ok], w_ref[ok], (fl[ok] & 1) != 0)
    md = gwn.gwn_build_3d(patches, max_aabb_frac=0.0)
    wd, _, _ = md.query(_q(q[:600]), mode=gwn.MODE_DIRECT, precision=gwn.PREC_FP32)
    assert np.max(np.abs(wd.cpu().numpy()[ok] - w_ref[ok])) <= 1e-4


def test_autotuned_beta_meets_tolerance(oracle_lib):
    """beta = 0: the build picks (beta, beta_leaf) for max |dGWN| <= tolerance."""
    patches, q = configs.cad_3d(4321, 600, 6000)
    m = gwn.gwn_build_3d(patches, beta=0.0, tolerance=1e-4)
    info = m.info()
    assert info["beta"] >= 2.0 and 2.0 <= info["beta_leaf"] <= info["beta"]
    rng = np.random.default_rng(6)
    sel = rng.choice(q.shape[0], 400, replace=False)
    w_ref, fl = oracle_lib.gwn3d(patches, q[sel], near_thr=1e-6 * _diag(patches))
    w, _, _ = m.query(_q(q.astype(np.float32)))
    w = w.cpu().numpy()[sel]
    ok = np.isfinite(w_ref)
    assert np.max(np.abs(w[ok] - w_ref[ok])) <= 1e-4


@pytest.mark.parametrize("beta,beta_leaf", [(0.0, 0.0), (4.0, 3.5)])
def test_order3_far_field_against_the_oracle(oracle_lib, beta, beta_leaf):
    """A CAD solid built with order 3 (third-order moments, one term beyond
    Eq. 3): with beta autotuned the build evaluates order 2 or 3, whichever is
    faster at the tolerance; with beta = 4, beta_leaf = 3.5 it evaluates order 3
    at factors where order 2 is less accurate.  Both stay within 1e-4 of the
    oracle's exact GWN, with labels equal away from the surface; the FP64
    repair, which reads the same FP64 moment blocks at 3 beta (or the factors
    the autotuner lowered while it stays within 1e-7 of the FP64 direct sum),
    within 1e-5 (1e-6 when tuned)."""
    patches, q = configs.cad_3d(4321, 600, 6000)
    m = gwn.gwn_build_3d(patches, beta=beta, beta_leaf=beta_leaf, order=3, tolerance=1e-4)
    info = m.info()
    assert info["order"] == 3 and info["eval_order"] in ((2, 3) if beta == 0.0 else (3,))
    rng = np.random.default_rng(16)
    sel = rng.choice(q.shape[0], 400, replace=False)
    w_ref, fl = oracle_lib.gwn3d(patches, q[sel], near_thr=1e-6 * _diag(patches))
    w, lab, st = m.query(_q(q.astype(np.float32)))
    w = w.cpu().numpy()[sel]
    ok = np.isfinite(w_ref)
    assert np.max(np.abs(w[ok] - w_ref[ok])) <= 1e-4
    assert _labels_ok(w[ok], w_ref[ok], fl[ok] != 0)
    wr, _, str_ = m.query(_q(q[sel].astype(np.float32)), repair_band=0.4999)
    wr, str_ = wr.cpu().numpy(), str_.cpu().numpy()
    rep = ok & ((str_ & api.QS_REPAIRED) != 0)
    assert rep.sum() > 0 and np.max(np.abs(wr[rep] - w_ref[rep])) <= (1e-6 if beta == 0.0 else 1e-5)


def test_packet_local_expansion_against_the_oracle(oracle_lib):
    """The packet local expansion (query option local_ratio; a local-expansion
    far field, one step beyond the paper): 2^20 queries packed into a cube of
    4 % of the box side, so that a warp's 32 binned queries lie close together
    and the expansion takes many clusters.  With it on at ratio 32 the values
    stay within 2e-5 of the per-query terms (the remainders of the ~700
    clusters a packet takes add up: at ratio 16 the difference reached 7.6e-5)
    and within 1e-4 of the oracle's exact GWN on a seeded sample, with labels
    equal away from the surface."""
    patches, _ = configs.cad_3d(4321, 600, 0)
    m = gwn.gwn_build_3d(patches, beta=5.0, beta_leaf=3.5)
    lo, hi = np.array(m.info()["lo"]), np.array(m.info()["hi"])
    rng = np.random.default_rng(21)
    side = 0.04 * (hi - lo)
    corner = lo + rng.uniform(0.2, 0.7, size=3) * (hi - lo)
    q = (corner + rng.uniform(size=(1 << 20, 3)) * side).astype(np.float32)
    qd = _q(q)
    w_off, _, _ = m.query(qd, local_ratio=-1.0)
    w_on, lab, _ = m.query(qd, local_ratio=32.0, count_work=True)
    local = m.last_query_stats()["local_nodes"] / q.shape[0]
    assert local > 50, local
    w_off, w_on, lab = w_off.cpu().numpy(), w_on.cpu().numpy(), lab.cpu().numpy()
    assert np.max(np.abs(w_on - w_off)) <= 2e-5
    sel = rng.choice(q.shape[0], 300, replace=False)
    w_ref, fl = oracle_lib.gwn3d(patches, q[sel].astype(np.float64), near_thr=1e-6 * _diag(patches))
    ok = np.isfinite(w_ref)
    assert np.max(np.abs(w_on[sel][ok] - w_ref[ok])) <= 1e-4
    assert _labels_ok(w_on[sel][ok], w_ref[ok], fl[ok] != 0)


@pytest.mark.parametrize("shape,beta_repair,tol", [("sphere", 0.0, 1e-6), ("sphere", 12.0, 1e-4),
                                                    ("cad_open", 0.0, 1e-6)])
def test_repair_of_most_points(oracle_lib, shape, beta_repair, tol):
    """The trimmed sphere (disc trims: rational boundary curves of degree 12) and
    every other patch of a CAD solid (polygon trims: degree 6) are open surfaces,
    so their GWN takes every value in (0, 1); a repair band of 0.4999 then sends
    almost every query through the FP64 repair (warp traversal and the FP64 pair
    list, one warp per pair, 8- or 4-point panels by degree).  With
    beta_repair = 0 the repair is the exact sum over every leaf, held to 1e-6;
    with beta_repair = 12 its far field is Taylor, held to 1e-4."""
    if shape == "sphere":
        patches, q = configs.sphere_3d(n_queries=3000)
    else:
        patches, q = configs.cad_3d(2468, 400, 3000)
        patches = patches[::2]
    sel = q[:500]
    w_ref, fl = oracle_lib.gwn3d(patches, sel, near_thr=1e-6 * _diag(patches))
    ok = np.isfinite(w_ref)
    m = gwn.gwn_build_3d(patches, beta=6.0, beta_leaf=4.0, repair_band=0.4999, beta_repair=beta_repair)
    w, lab, st = m.query(_q(sel.astype(np.float32)))
    w, st = w.cpu().numpy(), st.cpu().numpy()
    rep = ok & ((st & gwn.QS_REPAIRED) != 0)
    assert rep.sum() > 0.5 * ok.sum()
    assert not np.any(st[ok] & gwn.QS_UNRESOLVED)
    assert np.max(np.abs(w[rep] - w_ref[rep])) <= tol
    assert np.max(np.abs(w[ok] - w_ref[ok])) <= 1e-4


def test_cad_fp64_direct_matches_oracle(oracle_lib):
    """The GPU FP64 direct sum (every unsubdivided patch exact, FP64) on a CAD
    solid, uniform queries plus queries 1e-2 .. 1e-5 off the surface on both
    sides: within 1e-9 of the oracle.  This is the reference the large label
    comparisons use, so it is held to the all-FP64 bound itself."""
    from tests import refgeom as R
    patches, q = configs.cad_3d(1234, 400, 400)
    rng = np.random.default_rng(8)
    pts = [q]
    for k in rng.choice(len(patches), size=10, replace=False):
        p = patches[k]
        c = p.trims[0].ctrl[:-1].mean(axis=0)
        uv = np.clip(c + 0.05 * rng.uniform(-1, 1, size=(2, 2)), 0.01, 0.99)
        S, Su, Sv = R.surface_point_derivs(p, uv[:, 0], uv[:, 1])
        n = np.cross(Su, Sv)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        for h in (1e-2, 1e-3, 1e-5):
            pts += [S + h * n, S - h * n]
    q = np.concatenate(pts)
    w_ref, fl = oracle_lib.gwn3d(patches, q, near_thr=1e-6 * _diag(patches))
    ok = np.isfinite(w_ref)
    md = gwn.gwn_build_3d(patches, max_aabb_frac=0.0)
    w, _, st = md.query(_q(q), precision=gwn.PREC_FP64, mode=gwn.MODE_DIRECT)
    w, st = w.cpu().numpy(), st.cpu().numpy()
    assert not np.any(st[ok] & gwn.QS_UNRESOLVED)
    assert np.max(np.abs(w[ok] - w_ref[ok])) <= 1e-9


def test_sphere_full_set_against_exact_reference(sphere):
    """All 1,048,576 queries of the trimmed-sphere workload: the autotuned FP32 +
    repair traversal against the exact GPU direct sum (held to the oracle on the
    module's seeded sample here): max |dGWN| <= 1e-4, identical labels away from
    half-integers."""
    from paper_2605_19200_gb300 import accuracy
    patches, q, idx, w_ref, fl = sphere
    pts = _q(q.astype(np.float32))
    m = gwn.gwn_build_3d(patches, beta=0.0, tolerance=1e-4)
    w, lab, st = m.query(pts)
    ref = accuracy.build_reference(patches, 3)
    wr, lr, sr = accuracy.reference_values(ref, pts)
    wr = wr.cpu().numpy()
    ok = np.isfinite(w_ref)
    assert np.max(np.abs(wr[idx][ok] - w_ref[ok])) <= 5e-6   # the reference itself
    s = accuracy.compare(w.cpu().numpy(), lab.cpu().numpy(), wr)
    assert s["checked"] == q.shape[0]
    assert s["max_abs_dgwn"] <= 1e-4, s
    assert s["label_mismatches"] == 0, s
