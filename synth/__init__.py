"""Seeded synthetic inputs (geometry and query points) shared by the oracle
tests and the CUDA-path tests.  Holds no winding-number arithmetic."""
from .geometry import (Curve, Patch, arc, bezier_curve, bezier_knots, bilinear_patch, circle,
                       clamped_uniform_knots, cube_shell, nurbs_sphere, planar_patch, polyline,
                       shape_bbox_2d, shape_bbox_3d)
from . import configs
