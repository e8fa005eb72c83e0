"""B300 (sm_103a) hot path of GS-Scale 3DGS training: frustum cull, gather with
deferred restore, differentiable tile rasterizer, deferred Adam.

The compute lives in ``libgs_b300.so`` (hand-written CUDA behind the C ABI of
include/gs_b300.h); this package only marshals arguments.  Importing it loads
the library and fails if it has not been built.
"""
from . import _lib
from ._lib import (GS_BF16_SH_MOM, GS_BF16_SH_MOM_RN, GS_FP32, GS_OPT_ADAM, GS_OPT_ADAMW, GS_OPT_SGDM,  # noqa: F401
                   GS_TIER_DEVICE, GS_TIER_HOST_CPU_OPT, GS_TIER_HOST_SH)
from .api import (Context, GaussianScene, RegionCamera, adam_struct, adam_tables, camera_struct,  # noqa: F401
                  cpu_deferred_step, cpu_forward, n_params, render, split_regions)

_lib.load()
