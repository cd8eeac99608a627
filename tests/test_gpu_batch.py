"""GPU tests of gwn_query_batch: many models and point sets in one graph launch.

Each item's values must equal what gwn_query gives for the same model and
points (the same pipeline runs; only FP32 atomic summation order may differ),
a repeated call must replay the captured graph, and a changed item list must
be captured again.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_19200_gb300 as gwn
from synth import configs


def _outs(n):
    return (torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty(n, dtype=torch.int32, device="cuda"))


@pytest.fixture(scope="module")
def items():
    models, points = [], []
    for seed, npch, nq in ((31, 300, 70000), (32, 900, 5000), (33, 150, 1), (34, 500, 600000)):
        patches, q = configs.cad_3d(seed, npch, nq)
        models.append(gwn.gwn_build_3d(patches, beta=6.0, beta_leaf=4.0))
        points.append(torch.from_numpy(q.astype(np.float32)).cuda())
    curves, q2 = configs.star_2d(n_queries=30000)
    models.append(gwn.gwn_build_2d(curves, beta=8.0))
    points.append(torch.from_numpy(q2).cuda())          # float64 points
    return models, points


def test_batch_matches_single_queries_and_replays(items):
    models, points = items
    ref = []
    for m, p in zip(models, points):
        w, lab, _ = m.query(p)
        ref.append((w.cpu().numpy(), lab.cpu().numpy()))
    b = gwn.Batch(n_streams=3)
    outs = [_outs(p.shape[0]) for p in points]
    for rep in range(3):
        for o in outs:
            o[0].fill_(float("nan"))
        b.query(models, points, outs)
        torch.cuda.synchronize()
        for (w, lab, st), (wr, lr) in zip(outs, ref):
            np.testing.assert_allclose(w.cpu().numpy(), wr, rtol=0, atol=1e-5)
            assert np.array_equal(lab.cpu().numpy(), lr)
    info = b.info()
    assert info["graph_launches"] == 3 and info["captures"] == 1
    # a different item list is captured again
    sub = [p[: max(1, p.shape[0] // 3)] for p in points]
    outs2 = [_outs(p.shape[0]) for p in sub]
    b.query(models, sub, outs2)
    torch.cuda.synchronize()
    for (w, lab, st), (wr, lr), p in zip(outs2, ref, sub):
        np.testing.assert_allclose(w.cpu().numpy(), wr[: p.shape[0]], rtol=0, atol=1e-5)
    assert b.info()["captures"] == 2
    b.close()


def test_batch_rejects_bad_items(items):
    models, points = items
    b = gwn.Batch(n_streams=2)
    patches, _ = configs.cad_3d(35, 60, 0)
    host_only = gwn.gwn_build_3d(patches, beta=6.0, device=-2)
    with pytest.raises((gwn.GwnError, TypeError)):
        b.query([host_only], [points[0]], [_outs(points[0].shape[0])])
    with pytest.raises(TypeError):
        b.query([models[0]], [points[0].to(torch.int32)], [_outs(points[0].shape[0])])
    b.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_batch_host_buffers_match_device_batch(items, pinned):
    """gwn_query_batch_host (points and outputs in host memory, copies made by
    the library on the items' streams) gives the device batch's results; with
    page-locked buffers the copies are captured in the graph and replayed."""
    models, points = items
    b = gwn.Batch(n_streams=3)
    dev_outs = [_outs(p.shape[0]) for p in points]
    b.query(models, points, dev_outs)
    torch.cuda.synchronize()
    ref = [(o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy()) for o in dev_outs]
    if pinned:
        hp = [p.cpu().pin_memory() for p in points]
        mk = lambda n, dt: torch.empty(n, dtype=dt).pin_memory()
        hout = [(mk(p.shape[0], torch.float64), mk(p.shape[0], torch.int32), mk(p.shape[0], torch.int32))
                for p in points]
    else:
        hp = [p.cpu().numpy() for p in points]
        hout = [(np.empty(p.shape[0]), np.empty(p.shape[0], np.int32), np.empty(p.shape[0], np.int32))
                for p in points]
    caps0 = b.info()["captures"]
    for rep in range(2):
        for o in hout:
            o[0][:] = float("nan")
        b.query_host(models, hp, hout)
        for (w, lab, st), (wr, lr, sr) in zip(hout, ref):
            w, lab = np.asarray(w), np.asarray(lab)
            np.testing.assert_allclose(w, wr, rtol=0, atol=1e-5)
            assert np.array_equal(lab, lr)
    caps = b.info()["captures"] - caps0
    assert caps == (1 if pinned else 0)
    # the device batch still works after host calls (captured again)
    b.query(models, points, dev_outs)
    torch.cuda.synchronize()
    np.testing.assert_allclose(dev_outs[0][0].cpu().numpy(), ref[0][0], rtol=0, atol=1e-5)
    b.close()
