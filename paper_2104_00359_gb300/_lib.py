"""ctypes binding of ``libshshadow.so`` (the C ABI declared in include/shs.h).

Argument marshalling only: every step of the shading path runs in the CUDA
library.  Importing this module loads the library and raises if it has not
been built; there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_float, c_int32, c_int64, c_size_t, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libshshadow.so")

SHS_OK = 0
SHS_FP32, SHS_TF32, SHS_BF16, SHS_FP16 = 0, 1, 2, 3
STATUS_NAMES = {0: "SHS_OK", 1: "SHS_ERR_INVALID_ARG", 2: "SHS_ERR_UNSUPPORTED", 3: "SHS_ERR_OOM",
                4: "SHS_ERR_CUDA", 5: "SHS_ERR_TIMEOUT", 6: "SHS_ERR_BUSY"}


class ShsConfig(ctypes.Structure):
    """Mirror of ``shs_config``."""
    _fields_ = [
        ("n_bands", c_int32),
        ("epsilon", c_float),
        ("exp_tau", c_float),
        ("exp_kmax", c_int32),
        ("fixed_k", c_int32),
        ("precision", c_int32),
        ("deterministic", c_int32),
        ("horizon_cull", c_int32),
        ("exp_mode", c_int32),
    ]


class ShsRequest(ctypes.Structure):
    """Mirror of ``shs_request`` (one job's request in a batch call)."""
    _fields_ = [("scene", c_void_p), ("n_points", c_int64)] + [
        (n, c_void_p) for n in ("points", "normals", "albedo", "radiance", "saved", "target", "loss",
                                "d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals",
                                "d_radiance")]


class ShsError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_F = POINTER(c_float)
_SIGS = {
    "shs_config_default": (c_int32, [POINTER(ShsConfig)]),
    "shs_scene_create": (c_int32, [POINTER(ShsConfig), c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                   POINTER(c_void_p)]),
    "shs_scene_update": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "shs_scene_set_ol_table": (c_int32, [c_void_p, _F, c_int32, c_float]),
    "shs_scene_destroy": (c_int32, [c_void_p]),
    "shs_scene_info": (c_int32, [c_void_p, POINTER(ShsConfig), POINTER(c_int32)]),
    "shs_saved_bytes": (c_size_t, [c_void_p, c_int64]),
    "shs_shade": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "shs_shade_tail": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "shs_shade_backward": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "shs_shade_backward_l2": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_void_p]),
    "shs_shade_backward_noalloc": (c_int32, [POINTER(ShsConfig), c_int32, c_void_p, c_void_p, c_void_p, c_int64,
                                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "shs_noalloc_device_status": (c_int32, [c_void_p, POINTER(c_int32)]),
    "shs_batch_create": (c_int32, [POINTER(c_void_p)]),
    "shs_batch_destroy": (c_int32, [c_void_p]),
    "shs_shade_batch": (c_int32, [c_void_p, POINTER(ShsRequest), c_int32, c_void_p]),
    "shs_envmap_workspace_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "shs_project_envmap": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "shs_raster_workspace_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "shs_rasterize": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_int32,
                                c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "shs_rasterize_backward": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_int32,
                                         c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                         c_void_p]),
    "shs_chain_forward": (c_int32, [c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_int32, c_void_p,
                                    c_void_p, c_void_p]),
    "shs_chain_workspace_bytes": (c_size_t, [c_int64, c_int32]),
    "shs_chain_views_workspace_bytes": (c_size_t, [c_int64, c_int32, c_int32]),
    "shs_chain_forward_views": (c_int32, [c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_int32, c_int32,
                                          c_void_p, c_void_p, c_void_p]),
    "shs_chain_backward_views": (c_int32, [c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_int32,
                                           c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "shs_chain_backward": (c_int32, [c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_int32, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "shs_fp32_fma_probe": (c_int32, [c_int32, c_int64, c_void_p, c_void_p]),
    "shs_tc_gemm_selftest": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                       c_void_p]),
    "shs_scene_device_status": (c_int32, [c_void_p, c_void_p, POINTER(c_int32)]),
    "shs_launch_count": (c_int64, []),
    "shs_status_string": (c_char_p, [c_int32]),
    "shs_last_error": (c_char_p, []),
}

_lib = None


def load():
    """Load the library (once) and declare every entry point's signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2104_00359_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status, where):
    if status != SHS_OK:
        msg = load().shs_last_error()
        raise ShsError(status, where, msg.decode() if msg else "")


def ptr(t):
    """Device (or host) address of a tensor, or None."""
    return None if t is None else ctypes.c_void_p(t.data_ptr())
