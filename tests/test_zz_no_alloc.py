"""gwn_query_noalloc: the query entry point that allocates no device memory.

Some callers cannot let the library allocate: real-time loops that must not
stall on cudaMalloc, programs whose device memory belongs to another allocator
or a fixed budget.  For them gwn_query_noalloc keeps its scratch in
a fixed-size device array of the library.  This file is collected last so that
a failure here does not hide the other tests; it passes alone in a fresh
process as well (the first call on the device performs the array's set-up).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_19200_gb300 as gwn
from paper_2605_19200_gb300 import api
from synth import configs

TOL = 1e-4


def _outs(n):
    return (torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty(n, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_matches_gwn_query_twice(dim):
    if dim == 2:
        curves, q = configs.star_2d(n_queries=20000)
        m = gwn.gwn_build_2d(curves, beta=8.0)
    else:
        patches, q = configs.cad_3d(777, 300, 20000)
        m = gwn.gwn_build_3d(patches, beta=6.0, beta_leaf=4.0)
    pts = torch.from_numpy(q.astype(np.float32)).cuda()
    ref, ref_lab, _ = m.query(pts)
    torch.cuda.synchronize()
    for _ in range(2):  # the shared array keeps the previous call's contents
        w, lab, st = api.gwn_query_noalloc(m, pts, _outs(pts.shape[0]))
        torch.cuda.synchronize()
        assert torch.max(torch.abs(w - ref)).item() <= TOL
        mism = (lab != ref_lab) & (torch.abs(ref - torch.floor(ref) - 0.5) > TOL)
        assert not bool(mism.any())


def test_noalloc_rejects_oversized_batch():
    curves, _ = configs.star_2d(n_queries=4)
    m = gwn.gwn_build_2d(curves)
    n = (1 << 20) + 1
    pts = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(gwn.GwnError, match="INVALID_ARG"):
        api.gwn_query_noalloc(m, pts, _outs(n))
