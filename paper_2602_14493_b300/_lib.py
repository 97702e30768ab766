"""ctypes declarations of the C ABI in include/gmr.h (argument marshalling
only; every step of the renderer runs in libgmr.so's CUDA kernels).

The library is built in-tree by ``paper_2602_14493_b300.build``. Loading
fails loudly when it is missing: there is no fallback path.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgmr.so")

GMR_OK = 0
STATUS_NAMES = {0: "GMR_OK", 1: "GMR_ERR_INVALID_ARG", 2: "GMR_ERR_CUDA", 3: "GMR_ERR_OOM", 4: "GMR_ERR_CAPACITY",
                5: "GMR_ERR_TIMEOUT", 6: "GMR_ERR_STATE"}
GMR_DEV_BAD_FACE_INDEX = 1
GMR_DEV_PAIR_OVERFLOW = 2
GMR_COV_AREA, GMR_COV_EMBED_RAW = 0, 1
GMR_COLOR_PER_FACE, GMR_COLOR_PER_VERTEX, GMR_COLOR_SH = 0, 1, 2
GMR_FLAG_SYNC_CHECK = 1
GMR_FLAG_PROFILE = 2
GMR_FLAG_DEBUG_COUNTS = 4
GMR_FLAG_PERSISTENT = 8
GMR_FLAG_HALF_WARP_FWD = 16
GMR_FLAG_HALF_WARP_BWD = 32
GMR_FLAG_WARP_STAGE_FWD = 64
GMR_FLAG_WARP_STAGE_BWD = 128
GMR_FLAG_DETERMINISTIC = 256
GMR_L2_NOALLOC_MAX_ELEMS = 67108864
STAGES = ["project", "scan", "bin", "raster_fwd", "loss", "raster_bwd", "project_bwd"]

# Every function the header declares (checked by the CPU test suite).
EXPORTS = [
    "gmr_config_default", "gmr_create", "gmr_destroy", "gmr_set_config", "gmr_last_error", "gmr_status_string",
    "gmr_image_offsets", "gmr_reserve", "gmr_convert", "gmr_render_fwd", "gmr_render_fwd_l2", "gmr_render_bwd",
    "gmr_l2_loss",
    "gmr_get_device_status", "gmr_get_stats", "gmr_get_stage_times", "gmr_debug_forward_state",
    "gmr_l2_loss_noalloc", "gmr_adam_step", "gmr_chamfer", "gmr_render_bwd_ex", "gmr_silhouette_bce",
    "gmr_mesh_regularizers", "gmr_render_bwd_l2", "gmr_copy_h2d", "gmr_set_workspace_limit",
]


class GmrConfig(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("threads", ctypes.c_int32), ("threads_bwd", ctypes.c_int32),
                ("batch", ctypes.c_int32),
                ("cov_mode", ctypes.c_int32),
                ("color_mode", ctypes.c_int32), ("bg", ctypes.c_float * 3), ("flags", ctypes.c_int32),
                ("profile_stages", ctypes.c_uint32), ("sh_degree", ctypes.c_int32)]


class GmrCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("znear", ctypes.c_float)]


class GmrStats(ctypes.Structure):
    _fields_ = [("n_records", ctypes.c_int64), ("n_pairs", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("n_pixels", ctypes.c_int64), ("evals_fwd", ctypes.c_int64), ("evals_bwd", ctypes.c_int64), ("contribs", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("pair_capacity", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64)]


class GmrError(RuntimeError):
    pass


_LIB = None


def load(path: str = LIB_PATH):
    """Load libgmr.so and declare its signatures (no CUDA call is made)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise GmrError(f"{path} is missing: build it with `python -m paper_2602_14493_b300.build` "
                       "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    st = ctypes.c_int
    sig = {
        "gmr_config_default": (st, [ctypes.POINTER(GmrConfig)]),
        "gmr_create": (st, [ctypes.POINTER(GmrConfig), ctypes.POINTER(P)]),
        "gmr_destroy": (st, [P]),
        "gmr_set_config": (st, [P, ctypes.POINTER(GmrConfig)]),
        "gmr_last_error": (ctypes.c_char_p, [P]),
        "gmr_status_string": (ctypes.c_char_p, [st]),
        "gmr_image_offsets": (st, [P, i32, P]),
        "gmr_reserve": (st, [P, i64, i32, i64, i64]),
        "gmr_set_workspace_limit": (st, [P, i64]),
        "gmr_convert": (st, [P, P, i32, P, i32, P, P, P, P, P, P, P]),
        "gmr_render_fwd": (st, [P, P, i32, P, i32, P, P, P, i32, P, P, P]),
        "gmr_render_fwd_l2": (st, [P, P, i32, P, i32, P, P, P, i32, P, P, P, P, P, P]),
        "gmr_render_bwd": (st, [P, P, P, P, P, i32, P]),
        "gmr_l2_loss": (st, [P, P, P, i64, P, P, P]),
        "gmr_l2_loss_noalloc": (st, [P, P, i64, P, P, P]),
        "gmr_adam_step": (st, [P, P, P, P, P, i64, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, i32, P]),
        "gmr_chamfer": (st, [P, P, i64, P, i64, P, P]),
        "gmr_render_bwd_ex": (st, [P, P, P, P, P, P, i32, P]),
        "gmr_render_bwd_l2": (st, [P, P, P, P, P, P, P, P, i32, P]),
        "gmr_copy_h2d": (st, [P, P, i64, P]),
        "gmr_silhouette_bce": (st, [P, P, P, i64, ctypes.c_float, P, P, P]),
        "gmr_mesh_regularizers": (st, [P, P, i32, P, i32, ctypes.c_float, ctypes.c_float, P, P, P]),
        "gmr_get_device_status": (st, [P, P, ctypes.POINTER(ctypes.c_uint32)]),
        "gmr_get_stats": (st, [P, P, ctypes.POINTER(GmrStats)]),
        "gmr_get_stage_times": (st, [P, P, ctypes.POINTER(ctypes.c_float)]),
        "gmr_debug_forward_state": (st, [P, P, P, P, P, i64, P, P, P, P, P, ctypes.POINTER(ctypes.c_int64), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L
