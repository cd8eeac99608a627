"""Parity at full size: the 16-model CAD workload (80,804 trimmed patches,
19,727,937 queries) built with the autotuner and queried in the launch
configuration the benchmark times (one gwn_query_batch graph launch over four
streams), checked against the FP64 oracle on sampled outputs that it computes
one by one (three queries per model, seeded).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_19200_gb300 as gwn
from synth import configs
from synth import geometry as G


def test_full_cad16_batch_against_oracle(oracle_lib):
    workload = configs.cad_batch_3d()
    models, points, outs = [], [], []
    for patches, q in workload:
        models.append(gwn.gwn_build_3d(patches, beta=0.0, tolerance=1e-4))
        p = torch.from_numpy(q.astype(np.float32)).cuda()
        points.append(p)
        n = p.shape[0]
        outs.append((torch.empty(n, dtype=torch.float64, device="cuda"),
                     torch.empty(n, dtype=torch.int32, device="cuda"),
                     torch.empty(n, dtype=torch.int32, device="cuda")))
    assert sum(p.shape[0] for p in points) == 19727937
    b = gwn.Batch(n_streams=4)
    for _ in range(2):  # capture, then replay
        b.query(models, points, outs)
    torch.cuda.synchronize()
    assert b.info()["captures"] == 1
    rng = np.random.default_rng(2026)
    for (patches, q), (w, lab, st) in zip(workload, outs):
        idx = rng.choice(q.shape[0], size=3, replace=False)
        lo, hi = G.shape_bbox_3d(patches)
        w_ref, fl = oracle_lib.gwn3d(patches, q[idx], near_thr=1e-6 * float(np.linalg.norm(hi - lo)))
        wg = w.cpu().numpy()[idx]
        lg = lab.cpu().numpy()[idx]
        ok = np.isfinite(w_ref)
        assert np.max(np.abs(wg[ok] - w_ref[ok])) <= 1e-4
        keep = ok & ((fl & 1) == 0) & (np.abs((w_ref - np.floor(w_ref)) - 0.5) > 1e-6)
        assert np.array_equal(lg[keep], np.round(w_ref[keep]).astype(np.int32))
    b.close()
