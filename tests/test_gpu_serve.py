"""GPU tests of the serving loop (gwn_serve_*): continuous batching over
resident 2D and 3D models with memory-budget admission.

The property checked is that a request returns the same values and labels
whether it runs alone or mixed with other requests (other models, sizes and
point precisions) queued behind a small memory budget, and that those values
are the ones the direct query entry point gives; in the mixed run, requests
must have been in flight together and their device work must have overlapped
(timing events around each request's work on its slot's stream).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_19200_gb300 as gwn
from synth import configs


@pytest.fixture(scope="module")
def models():
    curves, q2 = configs.star_2d(n_queries=20000)
    patches, q3 = configs.cad_3d(seed=7101, n_patches=600, n_queries=30000)
    m2 = gwn.gwn_build_2d(curves)
    m3 = gwn.gwn_build_3d(patches, beta=6.0, beta_leaf=4.0)
    return (m2, q2), (m3, q3)


def _requests(models, rng):
    (m2, q2), (m3, q3) = models
    reqs = []
    for k in range(14):
        which = k % 2
        q = q2 if which == 0 else q3
        n = int(rng.integers(1, 9000)) if k % 5 else 1
        lo = int(rng.integers(0, q.shape[0] - n))
        pts = q[lo:lo + n]
        if k % 3 == 0:
            pts = pts.astype(np.float32)
        reqs.append((which, np.ascontiguousarray(pts)))
    return reqs


def _direct(model, pts):
    w, lab, _ = model.query(torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    return w.cpu().numpy(), lab.cpu().numpy()


def test_serve_alone_equals_mixed_equals_direct(models):
    rng = np.random.default_rng(11)
    reqs = _requests(models, rng)
    mods = [models[0][0], models[1][0]]

    # alone: one slot, each request submitted after the previous one finished
    alone = []
    srv = gwn.Server(n_slots=1)
    ids = [srv.add_model(m) for m in mods]
    for which, pts in reqs:
        rid = srv.submit(ids[which], pts)
        alone.append(srv.poll(rid, pts.shape[0]))
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0 and st["in_flight"] == 0
    srv.close()

    # mixed: three slots, every request queued at once behind a budget that
    # holds about two of the larger requests
    budget = 2 * 9000 * (3 * 8 + 12) + 4096
    srv = gwn.Server(n_slots=3, mem_budget_bytes=budget)
    ids = [srv.add_model(m) for m in mods]
    rids = [srv.submit(ids[which], pts) for which, pts in reqs]
    mixed = [srv.poll(rid, pts.shape[0]) for rid, (_, pts) in zip(rids, reqs)]
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["points_completed"] == sum(p.shape[0] for _, p in reqs)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert st["budget_used_bytes"] == 0
    # continuous batching: requests were admitted while others were in flight,
    # and their device work (copy in, query, copy out) overlapped on the GPU
    assert st["max_in_flight"] >= 2
    assert st["max_gpu_overlap"] >= 2
    srv.close()

    for (which, pts), (wa, la), (wm, lm) in zip(reqs, alone, mixed):
        wd, ld = _direct(mods[which], pts)
        # pair contributions are summed in FP32 with atomics, in an order that varies from
        # run to run: values agree to a few float32 ulps of |w| (2.4e-7 at |w| = 2)
        np.testing.assert_allclose(wa, wd, rtol=0, atol=1e-5)
        np.testing.assert_allclose(wm, wa, rtol=0, atol=1e-5)
        assert np.array_equal(la, ld) and np.array_equal(lm, la)


def test_serve_errors(models):
    (m2, q2), _ = models
    srv = gwn.Server(n_slots=2, mem_budget_bytes=1 << 16)
    mid = srv.add_model(m2)
    with pytest.raises(gwn.GwnError):
        srv.submit(mid, q2[:20000])           # larger than the budget
    with pytest.raises(gwn.GwnError):
        srv.submit(mid + 5, q2[:10])          # unknown model
    with pytest.raises(gwn.GwnError):
        srv.poll(12345, 1, timeout_ms=10)     # unknown request
    rid = srv.submit(mid, q2[:100])
    w, lab = srv.poll(rid, 100)
    wd, ld = _direct(m2, np.ascontiguousarray(q2[:100]))
    np.testing.assert_allclose(w, wd, rtol=0, atol=1e-5)
    with pytest.raises(gwn.GwnError):
        srv.poll(rid, 100, timeout_ms=10)     # already collected
    srv.close()
