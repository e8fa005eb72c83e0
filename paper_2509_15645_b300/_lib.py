"""ctypes declarations of the C ABI in include/gs_b300.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs_b300.so")

c_i32, c_i64, c_f32, c_vp = C.c_int32, C.c_int64, C.c_float, C.c_void_p

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_OOM, GS_ERR_CUDA, GS_ERR_BUDGET, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, GS_ERR_NUMERIC = range(8)
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_OOM", 3: "GS_ERR_CUDA", 4: "GS_ERR_BUDGET",
                5: "GS_ERR_CAPACITY", 6: "GS_ERR_TIMEOUT", 7: "GS_ERR_NUMERIC"}
GS_FP32, GS_BF16_SH_MOM, GS_BF16_SH_MOM_RN = 0, 1, 2
RASTER_VARIANTS = 10
SPANS = ("step", "cull", "fwd", "bwd", "adam", "adam_apply", "raster_bwd")
GS_ADAM_DEFERRED, GS_ADAM_EAGER = 0, 2
GS_OPT_ADAM, GS_OPT_ADAMW, GS_OPT_SGDM = 0, 1, 2
GS_TIER_DEVICE, GS_TIER_HOST_SH, GS_TIER_HOST_CPU_OPT = 0, 1, 2


class Camera(C.Structure):
    _fields_ = [("R", c_f32 * 9), ("t", c_f32 * 3), ("fx", c_f32), ("fy", c_f32), ("cx", c_f32), ("cy", c_f32),
                ("near_z", c_f32), ("far_z", c_f32), ("width", c_i32), ("height", c_i32), ("x0", c_i32),
                ("y0", c_i32), ("full_width", c_i32), ("full_height", c_i32)]


class Scene(C.Structure):
    _fields_ = [("n", c_i64), ("pitch", c_i64), ("sh_degree", c_i32), ("precision", c_i32), ("geo", c_vp),
                ("sh", c_vp), ("m", c_vp), ("v", c_vp), ("rdir", c_vp), ("counter", c_vp), ("step", c_i32),
                ("tier", c_i32), ("host_sh", c_vp), ("host_m", c_vp), ("host_v", c_vp), ("host_rdir", c_vp)]


class AdamCfg(C.Structure):
    _fields_ = [("lr", c_f32 * 6), ("beta1", c_f32), ("beta2", c_f32), ("eps", c_f32), ("max_defer", c_i32),
                ("mode", c_i32), ("seed", c_i32), ("optimizer", c_i32), ("weight_decay", c_f32)]


class Config(C.Structure):
    _fields_ = [("max_gaussians", c_i64), ("max_visible", c_i64), ("max_keys", c_i64), ("max_width", c_i32),
                ("max_height", c_i32), ("tile_w", c_i32), ("tile_h", c_i32), ("max_views", c_i32),
                ("max_sh_degree", c_i32), ("stage_chunks", c_i64), ("chunk_shift", c_i32), ("stage_elem_bytes", c_i32),
                ("render_views", c_i32), ("list_records", c_i32), ("cpu_opt", c_i32)]


EXPORTS = {
    "gs_workspace_size": (c_i32, [C.POINTER(Config), C.POINTER(C.c_size_t)]),
    "gs_create": (c_i32, [C.POINTER(c_vp), C.POINTER(Config), C.c_int, c_vp, C.c_size_t]),
    "gs_destroy": (c_i32, [c_vp]),
    "gs_last_error": (C.c_char_p, [c_vp]),
    "gs_sync_status": (c_i32, [c_vp, c_vp]),
    "gs_wait_copies": (c_i32, [c_vp, c_vp]),
    "gs_device_counters": (c_vp, [c_vp]),
    "gs_cull": (c_i32, [c_vp, C.POINTER(Scene), C.POINTER(Camera), C.POINTER(AdamCfg), c_vp, c_vp, c_vp]),
    "gs_render_fwd": (c_i32, [c_vp, C.POINTER(Scene), C.POINTER(Camera), C.POINTER(AdamCfg), c_vp, c_vp, c_vp, c_vp]),
    "gs_render_bwd": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp]),
    "gs_loss_l1": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "gs_adam_deferred": (c_i32, [c_vp, C.POINTER(Scene), c_vp, c_vp, c_vp, c_i64, C.POINTER(AdamCfg), c_vp]),
    "gs_refresh_rdir": (c_i32, [c_vp, C.POINTER(Scene), C.POINTER(AdamCfg), c_vp]),
    "gs_adam_materialize": (c_i32, [c_vp, C.POINTER(Scene), C.POINTER(AdamCfg), c_vp, c_vp, c_vp, c_vp]),
    "gs_grad_scatter": (c_i32, [c_vp, C.POINTER(Scene), c_vp, c_vp, c_vp, c_i64, c_vp, c_vp]),
    "gs_timing_enable": (c_i32, [c_vp, c_i32]),
    "gs_timing_read": (c_i32, [c_vp, C.POINTER(c_f32), c_i32, C.POINTER(c_i32)]),
    "gs_raster_pair_counts": (c_i32, [c_vp, C.POINTER(Scene), C.POINTER(Camera), C.POINTER(C.c_uint64), c_vp]),
    "gs_step_kernel_count": (c_i32, [c_vp, C.POINTER(c_i32)]),
    "gs_autotune": (c_i32, [c_vp, C.POINTER(Scene), C.POINTER(Camera), C.POINTER(c_i32), C.POINTER(c_f32), c_vp]),
    "gs_set_raster_variant": (c_i32, [c_vp, c_i32]),
    "gs_set_raster_variants": (c_i32, [c_vp, c_i32, c_i32]),
    "gs_cull_noalloc": (c_i32, [C.POINTER(Scene), C.POINTER(Camera), C.POINTER(AdamCfg), c_i32, c_i32, c_vp, c_vp,
                                c_vp, c_vp]),
    "gs_set_cull_wait_limit": (c_i32, [c_vp, C.c_uint32]),
    "gs_densify": (c_i32, [c_vp, C.POINTER(Scene), C.POINTER(Scene), C.POINTER(AdamCfg), c_vp, c_vp, c_vp, c_f32, c_f32,
                           c_f32, c_f32, c_vp]),
    "gs_render_lists": (c_i32, [c_vp, C.POINTER(c_vp), C.POINTER(c_vp), C.POINTER(c_vp), C.POINTER(c_vp)]),
    "gs_render_splats": (c_i32, [c_vp, C.POINTER(c_vp), C.POINTER(c_vp), C.POINTER(c_vp)]),
    "gs_step_gradients": (c_i32, [c_vp, C.POINTER(c_vp), C.POINTER(c_i64), C.POINTER(c_vp), C.POINTER(c_vp)]),
    "gs_host_tier_stats": (c_i32, [c_vp, C.POINTER(c_i64), C.POINTER(c_i64)]),
    "gs_split_point": (c_i32, [c_vp, C.POINTER(Scene), C.POINTER(Camera), C.POINTER(AdamCfg), c_i32, c_i32,
                               C.POINTER(c_i32), C.POINTER(c_i64), c_vp]),
    "gs_adam_tables": (c_i32, [C.POINTER(AdamCfg), c_i32, C.POINTER(c_f32), C.POINTER(c_f32), C.POINTER(c_f32),
                               C.POINTER(c_f32), C.POINTER(c_f32), C.POINTER(c_f32)]),
    "gs_step": (c_i32, [c_vp, C.POINTER(Scene), C.POINTER(Camera), C.POINTER(c_vp), c_i32, C.POINTER(AdamCfg),
                        c_vp, c_vp]),
    "gs_cpu_deferred_step": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_i32, c_i32, c_vp, c_vp, c_i64, c_vp, c_vp,
                                     c_i64, c_i64, C.POINTER(AdamCfg), c_i32, c_i32]),
    "gs_cpu_forward": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_i32, c_i32, c_vp, c_vp, c_i64, c_vp, c_vp, c_i64,
                               c_vp, c_vp, c_i64, c_i64, C.POINTER(AdamCfg), c_i32, c_vp, c_i64, c_i32]),
    "gs_set_cpu_threads": (c_i32, [c_vp, c_i32]),
    "gs_cpu_tier_stats": (c_i32, [c_vp, C.POINTER(C.c_double)]),
}

_lib = None


def load():
    """Load the CUDA library; raises if it has not been built (there is no
    fallback implementation)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library {LIB_PATH} is missing: run `python -m paper_2509_15645_b300.build`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class GsError(RuntimeError):
    def __init__(self, status, message=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
