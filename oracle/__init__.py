"""TEST INFRASTRUCTURE ONLY: the FP64 CPU oracle for exact generalized winding
numbers.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
may import this package; the product library never does."""
from .oracle import (build_oracle, gwn2d, gwn2d_each, gwn3d, gwn3d_each, curve_eval, patch_eval,
                     segment_moments, patch_moments, taylor, FLAG_NEAR, FLAG_ON_BOUNDARY,
                     FLAG_DEGENERATE, FLAG_NOT_CONVERGED)
