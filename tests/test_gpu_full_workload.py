"""Parity at full size: the 16-model CAD workload (80,804 trimmed patches,
19,727,937 queries) built with the autotuner and queried in the launch
configuration the benchmark times (one gwn_query_batch graph launch over four
streams).

Three checks, after Section 4.2 (direct evaluation is the error reference) and
Section 4.3 (containment by rounding; no unique decision next to the surface
or next to a half-integer):

1. the exact GPU direct-sum reference (paper_2605_19200_gb300.accuracy) is
   itself held to the GPU FP64 direct sum on seeded queries of the four
   smallest models;
2. the batch's values and labels against that reference on 65,536 seeded
   queries of every model: max |dGWN| <= 1e-4, identical labels;
3. the queries the GPU flagged (FP64 repair or near band), up to 6 per model,
   plus 2 seeded ones per model, against the FP64 CPU oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_19200_gb300 as gwn
from paper_2605_19200_gb300 import accuracy
from synth import configs
from synth import geometry as G

SAMPLE = 65536
REF_TOL = 3e-6   # the reference against the FP64 direct sum


def test_full_cad16_batch_against_reference_and_oracle(oracle_lib):
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
    b.close()

    sizes = [len(p) for p, _ in workload]
    smallest = set(np.argsort(sizes)[:4].tolist())
    stats = []
    flag = gwn.QS_REPAIRED | gwn.QS_NEAR
    for mi, ((patches, q), p, (w, lab, st)) in enumerate(zip(workload, points, outs)):
        ref = accuracy.build_reference(patches, 3)
        rng = np.random.default_rng(2026 + mi)
        sel = np.sort(rng.choice(q.shape[0], size=SAMPLE, replace=False))
        ps = p[torch.from_numpy(sel).cuda()].contiguous()
        wr, lr, sr = accuracy.reference_values(ref, ps)
        wr = wr.cpu().numpy()
        if mi in smallest:
            # 1. the reference against the GPU FP64 direct sum (exact to ~1e-9)
            w64, _, s64 = ref.query(ps[:1024], mode=gwn.MODE_DIRECT, precision=gwn.PREC_FP64)
            assert not np.any(s64.cpu().numpy() & gwn.QS_UNRESOLVED)
            err = np.max(np.abs(wr[:1024] - w64.cpu().numpy()))
            assert err <= REF_TOL, (mi, err)
        # 2. the batch against the reference
        s = accuracy.compare(w.cpu().numpy()[sel], lab.cpu().numpy()[sel], wr)
        assert s["max_abs_dgwn"] <= 1e-4, (mi, s)
        assert s["label_mismatches"] == 0, (mi, s)
        stats.append(s)
        # 3. flagged and seeded queries against the CPU oracle
        stv = st.cpu().numpy()
        idx = np.unique(np.concatenate([np.flatnonzero(stv & flag)[:6], rng.choice(q.shape[0], 2, replace=False)]))
        lo, hi = G.shape_bbox_3d(patches)
        w_o, fl = oracle_lib.gwn3d(patches, q[idx], near_thr=1e-6 * float(np.linalg.norm(hi - lo)))
        ok = np.isfinite(w_o)
        wg = w.cpu().numpy()[idx]
        lg = lab.cpu().numpy()[idx]
        assert np.max(np.abs(wg[ok] - w_o[ok])) <= 1e-4, mi
        keep = ok & ((fl & 1) == 0) & (np.abs((w_o - np.floor(w_o)) - 0.5) > 1e-6)
        assert np.array_equal(lg[keep], np.round(w_o[keep]).astype(np.int32)), mi
    tot = accuracy.merge(stats)
    assert tot["checked"] == SAMPLE * len(workload)
