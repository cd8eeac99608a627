"""The per-leaf stage of the 3D build on the GPU (Section 3.1 leaf moments by
Green's theorem quadrature, and the packing of the leaves' boundary curves for
the near field: composition with the leaf's net, point copies, FP32/FP64 node
tables, minimum panel levels) against the same stage on the host threads.

Both run the routines of curves3d.h without fused multiply-adds, so the model
must be the same bit for bit: every array of the model file (tree, moments,
leaf geometry, curves, tables) after the header, whose build options differ
in device_build alone.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_19200_gb300 as gwn
from paper_2605_19200_gb300 import api
from synth import configs


def _arrays(path):
    data = open(path, "rb").read()
    head = 8 + 16 + 8 + ctypes.sizeof(api.gwn_build_opts) + 20 + 24 + 48
    return data[:8 + 16 + 8], data[head:]


@pytest.mark.parametrize("shape", ["cad", "sphere", "cad_untrimmed_rational"])
def test_device_build_stage_matches_host_stage(tmp_path, shape):
    if shape == "cad":
        patches, q = configs.cad_3d(4242, 900, 20000)
    elif shape == "sphere":
        patches, q = configs.sphere_3d(n_queries=20000)
    else:
        patches, q = configs.cad_3d(77, 300, 20000)
        for p in patches:          # untrimmed: the rectangle edges are the whole boundary
            p.trims = []
    mh = gwn.gwn_build_3d(patches, beta=6.0, beta_leaf=4.0, device_build=0)
    md = gwn.gwn_build_3d(patches, beta=6.0, beta_leaf=4.0, device_build=1)
    ph, pd = str(tmp_path / "host.gwn"), str(tmp_path / "dev.gwn")
    gwn.gwn_model_save(mh, ph)
    gwn.gwn_model_save(md, pd)
    (h0, a0), (h1, a1) = _arrays(ph), _arrays(pd)
    assert h0 == h1
    assert len(a0) == len(a1) and a0 == a1
    # and the FP64 query (one thread per point, no atomics) agrees exactly
    pts = torch.from_numpy(q[:512].astype(np.float32)).cuda()
    wh, lh, _ = mh.query(pts, precision=gwn.PREC_FP64, beta=6.0)
    wd, ld, _ = md.query(pts, precision=gwn.PREC_FP64, beta=6.0)
    assert torch.equal(wh, wd) and torch.equal(lh, ld)
