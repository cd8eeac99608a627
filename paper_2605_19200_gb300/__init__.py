"""GB300-native generalized winding numbers for NURBS curves and trimmed
NURBS patches (agglomerated BVH + moment evaluation).

The compute path is libgwn.so (include/gwn.h), built from csrc/ with nvcc for
sm_103a; this package is its Python binding.
"""
from .api import (F32, F64, MEM_DEVICE, MEM_HOST, MODE_BVH, MODE_DIRECT, PREC_FP32, PREC_FP32_REPAIR,
                  PREC_FP64, QS_NEAR, QS_REPAIRED, QS_STACK_OVERFLOW, QS_UNRESOLVED, GwnError, Model,
                  default_build_opts, default_query_opts, gwn_build_2d, gwn_build_3d, gwn_model_info,
                  gwn_query, gwn_release, gwn_version, lib, Server, Batch,
                  gwn_model_save, gwn_model_load)
from .native import build as build_native
