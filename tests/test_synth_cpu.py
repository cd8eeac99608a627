"""The seeded input generators: deterministic for a seed, distinct across seeds,
and shaped as their documentation states (the benchmark's workload recipe)."""
import math

import numpy as np

from synth import configs


def test_generators_are_deterministic():
    a = configs.cad_3d(77, 60, 100)
    b = configs.cad_3d(77, 60, 100)
    assert len(a[0]) == len(b[0]) and np.array_equal(a[1], b[1])
    assert all(np.array_equal(p.ctrl, r.ctrl) and np.array_equal(p.weights, r.weights) for p, r in zip(a[0], b[0]))
    c = configs.cad_3d(78, 60, 100)
    assert not np.array_equal(a[1], c[1])
    s1, q1 = configs.star_2d()
    s2, q2 = configs.star_2d()
    assert np.array_equal(q1, q2) and len(s1) == len(s2) == 60


def test_workload_recipe():
    specs = configs.cad_batch_specs()
    assert len(specs) == 16
    assert all(1000 <= s.n_patches <= 40000 for s in specs)
    assert all(65536 <= s.n_queries <= 4194304 for s in specs)
    assert sum(s.n_queries for s in specs) == 19727937
    curves, q = configs.loops_2d(res=8)
    assert len(curves) == 19000 and q.shape == (64, 2)
    # queries are float32-representable
    assert np.array_equal(q, q.astype(np.float32).astype(np.float64))
    t, model, size = configs.serve_trace(2000.0, 1.0)
    assert abs(len(t) - 2000) < 200 and model.max() < 8
    assert size.min() >= 1000 and size.max() <= 2000000
    assert abs(math.log(np.median(size)) - math.log(16384)) < 0.3
