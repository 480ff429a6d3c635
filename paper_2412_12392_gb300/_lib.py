"""ctypes loader for libmslam.so, the sm_103a CUDA library (include/mslam.h).

There is no fallback: if the library cannot be found or loaded, every entry
point raises.  Build it with ``paper_2412_12392_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

MSLAM_OK = 0
MSLAM_ERR_ARG = 1
MSLAM_ERR_CUDA = 2
MSLAM_ERR_NOT_PD = 3
MSLAM_ERR_TIMEOUT = 4
MSLAM_ERR_NONFINITE = 5
MSLAM_ERR_RANGE = 6
MSLAM_F32 = 0
MSLAM_F16 = 1
MSLAM_FLAG_PER_EDGE = 1
MSLAM_OP_LINEARIZE = 1
MSLAM_OP_SOLVE = 2
MSLAM_OP_BACKWARD = 3
MSLAM_OP_PACK_F32 = 4
MSLAM_OP_PACK_F16 = 5
MSLAM_OP_STATS = 6
MSLAM_OP_TRACK = 7
MSLAM_OP_MATCH = 8
MSLAM_RES_RAY, MSLAM_RES_POINT, MSLAM_RES_PIXEL = 0, 1, 2

STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_NOT_PD", 4: "ERR_TIMEOUT", 5: "ERR_NONFINITE",
                6: "ERR_RANGE"}


class Params(C.Structure):
    """Mirror of mslam_params."""
    _fields_ = [
        ("sigma_ray", C.c_float), ("sigma_dist", C.c_float), ("huber_delta", C.c_float), ("q_min", C.c_float),
        ("lm_lambda", C.c_float), ("lm_iters", C.c_int32), ("win_radius", C.c_int32), ("n_levels", C.c_int32),
        ("win_dilation", C.c_int32 * 4), ("max_rel_dist3d", C.c_float), ("conv_tol", C.c_double),
        ("residual", C.c_int32), ("sigma_point", C.c_float), ("sigma_pixel", C.c_float), ("sigma_depth", C.c_float),
        ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
    ]


class PlanOpts(C.Structure):
    """Mirror of mslam_plan_opts."""
    _fields_ = [("lin_tile", C.c_int32), ("lin_blocks_per_sm", C.c_int32), ("match_block_w", C.c_int32),
                ("lin_form", C.c_int32), ("solve_form", C.c_int32), ("match_form", C.c_int32),
                ("match_ppt", C.c_int32), ("wait_limit", C.c_int32)]


class MslamError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}: {last_error()}")
        self.status = status


_lib = None

vp = C.c_void_p
i32 = C.c_int32
i64 = C.c_int64
u32 = C.c_uint32
sz = C.c_size_t

# name -> (argtypes, restype)
SIGNATURES = {
    "mslam_default_params": ([C.POINTER(Params)], None),
    "mslam_last_error": ([], C.c_char_p),
    "mslam_version": ([], C.c_char_p),
    "mslam_plan_create": ([i32, vp, i32, vp, vp, C.POINTER(vp)], C.c_int),
    "mslam_plan_destroy": ([vp], None),
    "mslam_default_plan_opts": ([C.POINTER(PlanOpts)], None),
    "mslam_plan_create_ex": ([i32, vp, i32, vp, vp, C.POINTER(PlanOpts), C.POINTER(vp)], C.c_int),
    "mslam_plan_device_bytes": ([vp], sz),
    "mslam_plan_upload": ([vp, vp, sz, vp], C.c_int),
    "mslam_plan_kf_pixels": ([vp], i64),
    "mslam_plan_edge_pixels": ([vp], i64),
    "mslam_plan_num_graphs": ([vp], i32),
    "mslam_plan_offsets": ([vp, vp, vp], None),
    "mslam_plan_stats": ([vp, vp, vp], None),
    "mslam_workspace_bytes": ([vp, i32], sz),
    "mslam_match": ([vp, vp, C.c_int, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, sz, u32,
                     vp], C.c_int),
    "mslam_gn_linearize": ([vp, vp, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, u32, vp], C.c_int),
    "mslam_gn_linearize_noalloc": ([vp, vp, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp, u32, vp], C.c_int),
    "mslam_gn_pack": ([vp, vp, C.c_int, vp, vp, vp, vp, sz, vp], C.c_int),
    "mslam_gn_linearize_packed": ([vp, vp, C.c_int, vp, vp, sz, vp, vp, vp, vp, vp, vp, sz, u32, vp], C.c_int),
    "mslam_gn_track": ([vp, vp, C.c_int, vp, vp, sz, i32, vp, vp, sz, vp], C.c_int),
    "mslam_gn_solve": ([vp, vp, vp, vp, vp, vp, vp, vp, sz, vp], C.c_int),
    "mslam_match_stats": ([vp, vp, vp, vp, vp, sz, vp], C.c_int),
    "mslam_keyframe_criterion": ([i32, vp, vp, vp, C.c_double, vp], C.c_int),
    "mslam_desc_to_chunked": ([C.c_int, i32, i64, vp, vp, i64, vp], C.c_int),
    "mslam_ray_image": ([C.c_int, C.c_int64, vp, vp, vp], C.c_int),
    "mslam_calib_backproject": ([C.c_int, i32, i32, i32, C.c_float, C.c_float, C.c_float, C.c_float, vp, vp],
                                C.c_int),
    "mslam_gn_solve_launches": ([vp], i32),
    "mslam_fuse": ([C.c_int, vp, i32, i32, i64, vp, vp, vp, vp, vp], C.c_int),
    "mslam_gn_backward": ([vp, vp, C.c_int, vp, vp, vp, vp, vp, vp, vp, C.c_double, vp, vp, vp, vp, sz, vp],
                          C.c_int),
    "mslam_gn_step_backward": ([vp, vp, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp, C.c_double, vp, vp, vp, vp, vp,
                                sz, vp], C.c_int),
}


def lib():
    """Load libmslam.so once; raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libmslam.so not built ({LIB}); run paper_2412_12392_gb300.build.build()")
        L = C.CDLL(LIB)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def last_error() -> str:
    if _lib is None:
        return ""
    return (_lib.mslam_last_error() or b"").decode()


def check(status: int, what: str) -> None:
    if status != MSLAM_OK:
        raise MslamError(status, what)
