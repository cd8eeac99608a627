"""CPU-side checks of libgwn.so: exported ABI, host-side build (Algorithm 1
preprocessing) against the oracle's plain moment integrals, and input
validation.  No GPU is used: models are built with GWN_DEVICE_HOST_ONLY."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2605_19200_gb300 as gwn
from synth import configs
from synth import geometry as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOST_ONLY = -2


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "gwn.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(gwn_[a-z0-9_]+)\s*\(", hdr))
    assert len(names) >= 10
    lib = ctypes.CDLL(gwn.native.build())
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def _leaves_under(child, node):
    out, st = [], [node]
    while st:
        k = st.pop()
        for c in child[k]:
            if c < 0:
                out.append(~c)
            else:
                st.append(c)
    return out


@pytest.mark.parametrize("tree_builder", [0, 1])
def test_tree_is_a_valid_binary_tree(tree_builder):
    """Both builders: every leaf under the root exactly once, every internal node
    but the root the child of exactly one node; the top-down sweep numbers its
    nodes in preorder (an internal left child is its parent + 1)."""
    curves, _ = configs.loops_2d(n_loops=20, per_loop=30, res=8)
    m = gwn.gwn_build_2d(curves, device=HOST_ONLY, tree_builder=tree_builder)
    info = m.info()
    tr = m.tree()
    n = info["n_leaves"]
    assert info["n_nodes"] == n - 1
    leaves = _leaves_under(tr["child"], 0)
    assert sorted(leaves) == list(range(n))
    internal = [c for pair in tr["child"] for c in pair if c >= 0]
    assert sorted(internal) == list(range(1, n - 1))
    if tree_builder == 1:
        left = tr["child"][:, 0]
        k = np.nonzero(left >= 0)[0]
        np.testing.assert_array_equal(left[k], k + 1)
        # leaves in depth-first order: each subtree covers a contiguous range of them
        for node in range(0, n - 1, 97):
            L = sorted(_leaves_under(tr["child"], node))
            assert L == list(range(L[0], L[0] + len(L)))


def test_topdown_tree_stays_shallow_on_coincident_leaves():
    """Forty copies of the same cube shell: the sweep's split costs tie on runs
    of coincident boxes, and the tie goes to the balanced split, so the tree
    stays about log2(leaves) deep (peeling one leaf per level gave depth 51
    here, and enough copies would overflow the traversal's warp stack)."""
    import math
    m = gwn.gwn_build_3d(G.cube_shell(half=1.0) * 40, device=HOST_ONLY, beta=6.0, tree_builder=1)
    info = m.info()
    assert info["max_depth"] <= math.log2(info["n_leaves"]) + 8, info["max_depth"]


def _sum_r3_and_visits(m, q, beta):
    """Sum of cubed node radii and the internal-node visits per query of
    Algorithm 1's traversal (far test |q - x0| > beta r), counted on the host."""
    tr = m.tree()
    child, x0, r = tr["child"], tr["x0"], tr["r"]
    visits, front = 0, [(0, np.arange(len(q)))]
    while front:
        node, idx = front.pop()
        visits += len(idx)
        near = idx[np.sum((q[idx] - x0[node]) ** 2, 1) <= (beta * r[node]) ** 2]
        if len(near):
            front.extend((c, near) for c in child[node] if c >= 0)
    return float(np.sum(r ** 3)), visits / len(q)


def test_topdown_tree_has_smaller_radii_than_the_lbvh():
    """On a CAD solid the top-down sweep's nodes are tighter than the Karras
    LBVH's: smaller summed r^3 and fewer internal-node visits per uniform query
    at beta = 5 (the same leaves, the same radius definition)."""
    patches, q = configs.cad_3d(4321, 1400, 4000)
    res = {}
    for tb in (0, 1):
        m = gwn.gwn_build_3d(patches, device=HOST_ONLY, tree_builder=tb, beta=5.0, beta_leaf=3.5)
        res[tb] = _sum_r3_and_visits(m, q, 5.0)
    assert res[1][0] < 0.95 * res[0][0] and res[1][1] < 0.95 * res[0][1], res


def test_subdivision_respects_the_box_threshold(oracle_lib):
    curves = [G.circle((0, 0), 1.0), G.arc((0.3, 0.1), 0.2, 0.0, 1.0)]
    m = gwn.gwn_build_2d(curves, device=HOST_ONLY, max_aabb_frac=0.1)
    prim, param = m.leaves()
    lo, hi = G.shape_bbox_2d(curves)
    lim = 0.1 * np.linalg.norm(hi - lo)
    for c in range(len(curves)):
        sel = np.nonzero(prim == c)[0]
        iv = param[sel, :2]
        iv = iv[np.argsort(iv[:, 0])]
        assert iv[0, 0] == curves[c].knots[0] and iv[-1, 1] == curves[c].knots[-1]
        np.testing.assert_array_equal(iv[1:, 0], iv[:-1, 1])      # contiguous cover
    # each leaf's curve lies in a box below the threshold (sampled from the oracle's evaluator)
    for i in range(len(prim)):
        t = np.linspace(param[i, 0], param[i, 1], 50)
        P = oracle_lib.curve_eval(curves[prim[i]], t)
        assert np.linalg.norm(P.max(0) - P.min(0)) < lim


def test_node_moments_match_plain_integrals(oracle_lib):
    """Up-swept, centred moments (Section 3.1) equal the oracle's quadrature of
    the chords of the node's leaves about the node centroid."""
    curves, _ = configs.star_2d(n_queries=4)
    m = gwn.gwn_build_2d(curves, device=HOST_ONLY)
    prim, param = m.leaves()
    tr = m.tree()
    chords = np.zeros((len(prim), 4))
    for i in range(len(prim)):
        P = oracle_lib.curve_eval(curves[prim[i]], param[i, :2])
        chords[i] = [P[0, 0], P[0, 1], P[1, 0], P[1, 1]]
    for node in [0, 1, 5, 17, len(prim) - 2]:
        L = _leaves_under(tr["child"], node)
        ref = oracle_lib.segment_moments(chords[L], tr["x0"][node])
        got = tr["mom"][node]
        np.testing.assert_allclose(got[:2], ref["m0"], atol=1e-12)
        np.testing.assert_allclose(got[2:6], ref["m1"].ravel(), atol=1e-12)
        np.testing.assert_allclose(got[6:14], ref["m2"].ravel(), atol=1e-12)
        # centroid = chord-length-weighted centroid, radius = half box diagonal
        lens = np.linalg.norm(chords[L, 2:] - chords[L, :2], axis=1)
        mids = 0.5 * (chords[L, :2] + chords[L, 2:])
        np.testing.assert_allclose(tr["x0"][node], (lens[:, None] * mids).sum(0) / lens.sum(), atol=1e-12)


@pytest.mark.parametrize("bad,code", [
    (G.Curve(4, np.zeros((5, 2)), np.ones(5), G.bezier_knots(4)), "INVALID_ARG"),
    (G.Curve(2, np.zeros((4, 2)), np.ones(4), np.array([0, 0.1, 0.2, 0.3, 0.7, 0.8, 1.0])), "INVALID_GEOMETRY"),
    (G.Curve(1, np.zeros((2, 2)), np.array([1.0, -1.0]), G.bezier_knots(1)), "INVALID_GEOMETRY"),
    (G.Curve(1, np.array([[0, 0], [np.nan, 1]]), np.ones(2), G.bezier_knots(1)), "INVALID_GEOMETRY"),
])
def test_invalid_input_rejected(bad, code):
    with pytest.raises(gwn.GwnError, match=code):
        gwn.gwn_build_2d([bad], device=HOST_ONLY)


def test_invalid_options_rejected():
    curves = [G.circle()]
    for kw in ({"beta": 1.5}, {"order": 3}, {"repair_band": 0.7}, {"beta_repair": 1.0}):   # order 3 is 3D only
        with pytest.raises(gwn.GwnError, match="INVALID_ARG"):
            gwn.gwn_build_2d(curves, device=HOST_ONLY, **kw)


def test_3d_root_moments_match_plain_integrals(oracle_lib):
    """Leaves cut by the subdivision (trims clipped to the leaf rectangles),
    Green's-theorem quadrature per leaf and the up-sweep: the root's centred
    moments equal the oracle's fan cubature of every patch about the root
    centroid."""
    patches, _ = configs.sphere_3d(n_queries=4)
    m = gwn.gwn_build_3d(patches, device=HOST_ONLY)
    prim, param = m.leaves()
    assert len(prim) > len(patches)          # some patches were subdivided
    tr = m.tree()
    x0 = tr["x0"][0]
    tot = {k: 0 for k in ("m0", "m1", "m2")}
    area = 0.0
    for p in patches:
        r = oracle_lib.patch_moments(p, x0, nsub=2)
        for k in tot:
            tot[k] = tot[k] + r[k]
        area += r["area"]
    got = tr["mom"][0]
    scale = area
    np.testing.assert_allclose(got[:3], tot["m0"], atol=1e-10 * scale)
    np.testing.assert_allclose(got[3:12], tot["m1"].ravel(), atol=1e-10 * scale)
    np.testing.assert_allclose(got[12:39], tot["m2"].ravel(), atol=1e-10 * scale)


def test_3d_root_moments_of_two_cubes_closed_form():
    """Moments of orders 1-3 about the root centroid c for two disjoint cube
    shells, from the divergence theorem: int y_i n_k = d_ik V,
    int y_i y_j n_k = d_ik P_j + d_jk P_i and
    int y_i y_j y_l n_k = d_ik J_jl + d_jk J_il + d_lk J_ij, with P = int_V y dV
    and J = int_V y y dV over the solids (y = x - c).  The centroid differs from
    the scene's reference point, so the binomial shift of every order is used."""
    cubes = [((0.0, 0.0, 0.0), 1.0), ((3.0, 0.0, 0.0), 0.5)]
    patches = G.cube_shell(*cubes[0]) + G.cube_shell(*cubes[1])
    m = gwn.gwn_build_3d(patches, device=HOST_ONLY, order=3)
    tr = m.tree()
    c = tr["x0"][0]
    np.testing.assert_allclose(c, [0.6, 0.0, 0.0], atol=1e-12)   # area-weighted: (24 * 0 + 6 * 3) / 30
    V, P, J = 0.0, np.zeros(3), np.zeros((3, 3))
    for a, h in cubes:
        vol = (2 * h) ** 3
        d = np.asarray(a) - c
        V += vol
        P += vol * d
        J += vol * np.outer(d, d) + np.eye(3) * vol * h * h / 3
    I = np.eye(3)
    m1 = V * I
    m2 = np.einsum("ik,j->ijk", I, P) + np.einsum("jk,i->ijk", I, P)
    m3 = (np.einsum("ik,jl->ijlk", I, J) + np.einsum("jk,il->ijlk", I, J) + np.einsum("lk,ij->ijlk", I, J))
    got = tr["mom"][0]
    assert got.shape == (120,)
    np.testing.assert_allclose(got[:3], 0.0, atol=1e-12)          # closed surfaces: int n = 0
    np.testing.assert_allclose(got[3:12], m1.ravel(), atol=1e-11)
    np.testing.assert_allclose(got[12:39], m2.ravel(), atol=1e-11)
    np.testing.assert_allclose(got[39:120], m3.ravel(), atol=1e-11)


def test_3d_leaf_moments_additive_over_subdivision(oracle_lib):
    """A trimmed patch split into many leaves: the subtree of its leaves carries
    the patch's moments (checked on a single-patch model)."""
    patches, _ = configs.sphere_3d(n_queries=4)
    p = patches[7]
    m = gwn.gwn_build_3d([p], device=HOST_ONLY, max_aabb_frac=0.2)
    prim, param = m.leaves()
    assert len(prim) >= 4
    tr = m.tree()
    ref = oracle_lib.patch_moments(p, tr["x0"][0], nsub=2)
    np.testing.assert_allclose(tr["mom"][0][:3], ref["m0"], atol=1e-12)
    np.testing.assert_allclose(tr["mom"][0][3:12], ref["m1"].ravel(), atol=1e-12)
    np.testing.assert_allclose(tr["mom"][0][12:39], ref["m2"].ravel(), atol=1e-12)


def test_3d_invalid_input_rejected():
    good = G.planar_patch((0, 0, 0), (1, 0, 0), (0, 1, 0))
    bad_trim = G.planar_patch((0, 0, 0), (1, 0, 0), (0, 1, 0), trims=[G.circle((0.9, 0.5), 0.3)])
    with pytest.raises(gwn.GwnError, match="INVALID_GEOMETRY"):
        gwn.gwn_build_3d([good, bad_trim], device=HOST_ONLY)
    bad_w = G.Patch(1, 1, good.ctrl, -good.weights, good.knots_u, good.knots_v, [])
    with pytest.raises(gwn.GwnError, match="INVALID_GEOMETRY"):
        gwn.gwn_build_3d([bad_w], device=HOST_ONLY)


def test_binding_refuses_shapes_that_would_overrun_buffers():
    """The C ABI reads n x dim points and writes n outputs; the binding refuses
    arrays whose shapes would make it read or write past them (host path, no GPU)."""
    import numpy as np
    import paper_2605_19200_gb300 as gwn
    from synth import geometry as G
    m = gwn.gwn_build_2d([G.circle()], device=-2)     # host-only model: no query reaches the device
    with pytest.raises(ValueError):
        gwn.gwn_query(m, np.zeros((5, 3)))            # 3 coordinates for a 2D model
    with pytest.raises(ValueError):
        gwn.gwn_query(m, np.zeros(10))                # flat array
    with pytest.raises(ValueError):
        gwn.gwn_query(m, np.zeros((5, 2)), out=(np.zeros(4), None, None))   # output too short
    with pytest.raises(TypeError):
        gwn.gwn_query(m, np.zeros((5, 2)), out=(np.zeros(5, dtype=np.float32), None, None))
    with pytest.raises(ValueError):
        gwn.gwn_query(m, np.zeros((5, 2)), out=(np.zeros(10)[::2], None, None))  # strided


def test_shape_checks_accept_the_tensors_the_device_path_passes():
    """The same checks on torch tensors (as the CUDA path receives them)."""
    torch = pytest.importorskip("torch")
    from paper_2605_19200_gb300 import api
    m = gwn.gwn_build_3d(G.cube_shell(), device=-2)
    ok = (torch.zeros(5, dtype=torch.float64), torch.zeros(5, dtype=torch.int32), torch.zeros(5, dtype=torch.int32))
    api._check_shapes(m, torch.zeros((5, 3)), ok)
    api._check_shapes(m, torch.zeros((5, 3), dtype=torch.float64), (ok[0], None, None))
    api._check_shapes(m, torch.zeros((0, 3)), None)
    with pytest.raises(ValueError):
        api._check_shapes(m, torch.zeros((5, 2)), ok)
    with pytest.raises(TypeError):
        api._check_shapes(m, torch.zeros((5, 3)), (torch.zeros(5), None, None))
    with pytest.raises(TypeError):
        api._check_shapes(m, torch.zeros((5, 3)), (ok[0], torch.zeros(5, dtype=torch.int64), None))
    with pytest.raises(ValueError):
        api._check_shapes(m, torch.zeros((5, 3)), (torch.zeros(10, dtype=torch.float64)[::2], None, None))


@pytest.mark.parametrize("dim", [2, 3])
def test_model_checkpoint_roundtrip(tmp_path, dim):
    """gwn_model_save / gwn_model_load restore every host array and option of a
    model bit for bit (host copies; the device upload is the build's own)."""
    if dim == 2:
        curves, _ = configs.star_2d(n_queries=4)
        m = gwn.gwn_build_2d(curves, beta=6.0, device=-2)
    else:
        patches, _ = configs.cad_3d(31, 80, 0)
        m = gwn.gwn_build_3d(patches, beta=6.0, beta_leaf=4.0, adaptive_beta=1, device=-2)
    path = str(tmp_path / "model.gwn")
    gwn.gwn_model_save(m, path)
    r = gwn.gwn_model_load(path, device=-2)
    a, b = m.info(), r.info()
    for k in ("dim", "n_primitives", "n_leaves", "n_nodes", "max_depth", "beta", "beta_leaf", "order",
              "repair_band", "beta_repair"):
        assert a[k] == b[k], k
    ta, tb = m.tree(), r.tree()
    for k in ("child", "x0", "r", "mom"):
        assert ta[k].size > 0 and np.array_equal(ta[k], tb[k]), k
    pa, qa = m.leaves()
    pb, qb = r.leaves()
    assert np.array_equal(pa, pb) and np.array_equal(qa, qb)
    # every array (leaf geometry, boundary curves, FP64 copies) survives: the
    # restored model writes the same bytes
    again = str(tmp_path / "again.gwn")
    gwn.gwn_model_save(r, again)
    assert open(path, "rb").read() == open(again, "rb").read()


def test_model_load_rejects_bad_files(tmp_path):
    curves, _ = configs.star_2d(n_queries=4)
    m = gwn.gwn_build_2d(curves, beta=6.0, device=-2)
    good = tmp_path / "m.gwn"
    gwn.gwn_model_save(m, str(good))
    data = good.read_bytes()
    for name, blob in (("magic", b"XXXXXXXX" + data[8:]), ("truncated", data[: len(data) // 2]), ("empty", b"")):
        p = tmp_path / (name + ".gwn")
        p.write_bytes(blob)
        with pytest.raises(gwn.GwnError):
            gwn.gwn_model_load(str(p), device=-2)
    with pytest.raises(gwn.GwnError):
        gwn.gwn_model_load(str(tmp_path / "missing.gwn"), device=-2)


# element sizes of the model file's arrays, in file order (gwn_model_save)
_ARRAY_ELEM = [("child", 8), ("hdr", 16), ("mom", 16), ("hdr64", 8), ("mom64", 8), ("lhdr", 16), ("lmom", 16),
               ("lhdr64", 8), ("lmom64", 8), ("x0", 8), ("r", 8), ("mom_c", 8), ("leaf_prim", 8),
               ("leaf_param", 8), ("leaf2", 16), ("leaf2_64", 8), ("leaf3", 48), ("net3", 16), ("net3_64", 8),
               ("c3", 16), ("c3pts", 16), ("c3pts64", 8), ("c3n", 16), ("c3n64", 8), ("c2", 16), ("c2_64", 8), ("c2mult", 4)]


def _split_model_file(data):
    """(header bytes, [(name, count, payload bytes)]) of a model file."""
    import ctypes
    from paper_2605_19200_gb300 import api
    # magic, 4 int32, primitive count, options, 5 int32 (tree header, binning, order), 3 doubles (repair factors, local ratio), box
    off = 8 + 16 + 8 + ctypes.sizeof(api.gwn_build_opts) + 20 + 24 + 48
    head, arrays = data[:off], []
    for name, es in _ARRAY_ELEM:
        n = int(np.frombuffer(data[off:off + 8], dtype=np.uint64)[0])
        arrays.append((name, n, data[off + 8:off + 8 + n * es]))
        off += 8 + n * es
    assert off == len(data)
    return head, arrays


def _join_model_file(head, arrays):
    out = bytearray(head)
    for _, n, payload in arrays:
        out += np.uint64(n).tobytes() + payload
    return bytes(out)


@pytest.mark.parametrize("dim", [2, 3])
def test_model_load_rejects_inconsistent_arrays(tmp_path, dim):
    """A file whose arrays disagree with the model's leaf count, whose child
    indices leave the tree, or whose counts exceed the file, is refused before
    anything reaches a device (the kernels would read out of bounds)."""
    if dim == 2:
        curves, _ = configs.star_2d(n_queries=4)
        m = gwn.gwn_build_2d(curves, beta=6.0, device=-2)
    else:
        patches, _ = configs.cad_3d(31, 60, 0)
        m = gwn.gwn_build_3d(patches, beta=6.0, beta_leaf=4.0, device=-2)
    good = tmp_path / "m.gwn"
    gwn.gwn_model_save(m, str(good))
    data = good.read_bytes()
    head, arrays = _split_model_file(data)
    assert _join_model_file(head, arrays) == data
    idx = {name: k for k, (name, _, _) in enumerate(arrays)}
    es = dict(_ARRAY_ELEM)
    bad = {}
    # one moment block short
    a = list(arrays)
    name, n, pl = a[idx["mom"]]
    a[idx["mom"]] = (name, n - 1, pl[:-es["mom"]])
    bad["short_mom"] = _join_model_file(head, a)
    # a child index past the last leaf
    a = list(arrays)
    name, n, pl = a[idx["child"]]
    ch = np.frombuffer(pl, dtype=np.int32).copy()
    ch[1] = -(m.info()["n_leaves"] + 5)
    a[idx["child"]] = (name, n, ch.tobytes())
    bad["child_range"] = _join_model_file(head, a)
    # a child that points back at the root (the traversal would not end)
    ch = np.frombuffer(pl, dtype=np.int32).copy()
    ch[2 * (len(ch) // 2 - 1)] = 0
    a[idx["child"]] = (name, n, ch.tobytes())
    bad["child_root"] = _join_model_file(head, a)
    # a count far beyond the file's size
    a = list(arrays)
    name, n, pl = a[idx["r"]]
    blob = bytearray(_join_model_file(head, a))
    off = len(head) + sum(8 + len(p) for _, _, p in arrays[:idx["r"]])
    blob[off:off + 8] = np.uint64(1 << 40).tobytes()
    bad["huge_count"] = bytes(blob)
    # bytes after the last array
    bad["trailing"] = data + b"\0" * 16
    if dim == 3:
        # a boundary curve whose points run past the point table
        a = list(arrays)
        name, n, pl = a[idx["c3"]]
        c3 = np.frombuffer(pl, dtype=np.int32).copy().reshape(-1, 4)
        c3[-1, 0] = len(arrays[idx["c3pts"]][2]) // 16 - 2
        a[idx["c3"]] = (name, n, c3.tobytes())
        bad["c3_range"] = _join_model_file(head, a)
    for key, blob in bad.items():
        p = tmp_path / (key + ".gwn")
        p.write_bytes(blob)
        with pytest.raises(gwn.GwnError, match="INVALID_ARG"):
            gwn.gwn_model_load(str(p), device=-2)
    # the unmodified file still loads
    gwn.gwn_model_load(str(good), device=-2)


def test_device_calls_refuse_host_tensors():
    """A device call hands raw pointers to the kernels: host tensors, or tensors
    on another GPU, are refused in Python before any query reaches the library."""
    import torch
    from paper_2605_19200_gb300 import api
    curves, _ = configs.star_2d(n_queries=4)
    m = gwn.gwn_build_2d(curves, beta=6.0, device=-2)
    pts = torch.zeros((5, 2), dtype=torch.float32)
    outs = (torch.zeros(5, dtype=torch.float64), None, None)
    with pytest.raises(TypeError, match="CUDA"):
        api.gwn_query_noalloc(m, pts, outs)
    with pytest.raises(TypeError):
        api.gwn_query_noalloc(m, pts, None)

    class _OnGpu:  # stands in for a CUDA tensor on another device
        is_cuda = True

        def __init__(self, index):
            self.device = torch.device("cuda", index)

    with pytest.raises(TypeError, match="CUDA"):
        api._check_device(m, pts, (torch.zeros(5, dtype=torch.float64), None, None))
    # the host-only model lives on no GPU: any device index is another GPU's
    with pytest.raises(TypeError, match="lives on"):
        api._check_device(m, _OnGpu(3), None)
