"""GB300-native (sm_103a) CUDA implementation of the data-parallel hot path of
MASt3R-SLAM (arXiv 2412.12392): iterative projective matching of two-view
pointmaps feeding a ray-error Sim(3) Gauss-Newton over a keyframe graph.

The kernels live in libmslam.so behind the C ABI of include/mslam.h; this
package holds its build script and a thin ctypes binding.
"""
from . import _lib  # noqa: F401
from .api import (GaussNewton, Plan, chunk_descriptors, default_params, gn_backward, gn_linearize,  # noqa: F401
                  gn_linearize_packed, gn_pack, gn_solve, match, match_stats, pack_bytes, params_dict, fuse,
                  calib_backproject, ray_image, gn_track, keyframe_needed)

__all__ = ["Plan", "GaussNewton", "chunk_descriptors", "default_params", "params_dict", "match", "gn_linearize", "gn_solve",
           "gn_backward", "gn_pack", "gn_linearize_packed", "pack_bytes", "fuse", "match_stats",
           "calib_backproject", "ray_image", "gn_track", "keyframe_needed"]
