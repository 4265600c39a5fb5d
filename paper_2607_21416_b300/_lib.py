"""ctypes declarations of libgs (include/gs.h).  Argument marshalling only.

Loading fails loudly when the shared library is missing: there is no CPU or
PyTorch fallback for any step of the rendering path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs.so")

GS_OK = 0
GS_ERR_INVALID_ARG = -1
GS_ERR_CAPACITY = -2
GS_ERR_CUDA = -3
GS_ERR_TIMEOUT = -4
GS_ERR_UNSUPPORTED = -5
GS_TILE = 16
GS_MAX_VIEWS = 64
GS_PREC_FP32 = 0
GS_PREC_BF16 = 1

i32, i64, vp, sz = C.c_int32, C.c_int64, C.c_void_p, C.c_size_t


class gs_view(C.Structure):
    _fields_ = [("width", i32), ("height", i32)]


class gs_status(C.Structure):
    _fields_ = [("code", i32), ("where", i32), ("needed", i64)]


class gs_anchors(C.Structure):
    _fields_ = [("N", i32), ("F", i32), ("k", i32), ("hidden", i32), ("M", i32), ("xyz", vp),
                ("feat", vp), ("log_scaling", vp), ("offsets", vp), ("part", vp), ("mlp", vp)]


class gs_gauss3d(C.Structure):
    _fields_ = [("k", i32), ("cap_rows", i64), ("row_anchor", vp), ("view_start", vp), ("mu", vp),
                ("scale", vp), ("quat", vp), ("opacity", vp), ("colour", vp)]


class gs_gauss3d_grad(C.Structure):
    _fields_ = [("dmu", vp), ("dscale", vp), ("dquat", vp), ("dopacity", vp), ("dcolour", vp)]


class gs_splats(C.Structure):
    _fields_ = [("cap", i64), ("rec", vp), ("tiles", vp)]


class gs_splat_grad(C.Structure):
    _fields_ = [("g", vp), ("layout", i32)]


GS_SGRAD_CANDIDATE = 0
GS_SGRAD_ROW_TILES = 1


class gs_bins(C.Structure):
    _fields_ = [("cap_pairs", i64), ("vals", vp), ("keys", vp), ("ranges", vp), ("n_pairs", vp)]


class gs_anchor_grad(C.Structure):
    _fields_ = [("dxyz", vp), ("dfeat", vp), ("dlog_scaling", vp), ("doffsets", vp), ("dmlp", vp)]


class gs_adam_group(C.Structure):
    _fields_ = [("param", vp), ("grad", vp), ("m", vp), ("v", vp), ("n", i64), ("lr", C.c_float)]


class gs_tuning(C.Structure):
    _fields_ = [("fwd_ctas_per_sm", i32), ("bwd_ctas_per_sm", i32), ("sort_ctas_per_sm", i32),
                ("emit_ctas_per_sm", i32)]


GS_ADAM_MAX_GROUPS = 16
DEFAULT_CHUNK = 384   # splats per compositing work item when gs_render_fwd gets chunk = 0

P = C.POINTER

EXPORTS = {
    "gs_mlp_floats": (i64, [i32, i32, i32]),
    "gs_total_tiles": (i64, [P(gs_view), i32]),
    "gs_total_pixels": (i64, [P(gs_view), i32]),
    "gs_decode_workspace": (sz, [i32, i32, i32, i64]),
    "gs_bin_sort_workspace": (sz, [P(gs_view), i32, i64, i64]),
    "gs_decode_bwd_workspace": (sz, [i32, i32, i32, i64]),
    "gs_status_string": (C.c_char_p, [i32]),
    "gs_kernel_launches": (C.c_uint64, []),
    "gs_set_wait_limit": (i32, [i64]),
    "gs_set_tuning": (i32, [P(gs_tuning)]),
    "gs_get_tuning": (i32, [P(gs_tuning)]),
    "gs_probe_peak": (i32, [i32, i32, i32, vp, C.POINTER(C.c_int64), vp]),
    "gs_decode": (C.c_int, [P(gs_anchors), vp, P(gs_view), i32, i32, P(gs_gauss3d), vp, sz, vp, vp]),
    "gs_decode_noalloc": (C.c_int, [P(gs_anchors), vp, P(gs_view), i32, i32, P(gs_gauss3d), vp, vp]),
    "gs_project": (C.c_int, [P(gs_gauss3d), vp, P(gs_view), i32, P(gs_splats), vp, vp]),
    "gs_bin_sort": (C.c_int, [P(gs_splats), i32, vp, i64, P(gs_view), i32, P(gs_bins), vp, sz, vp, vp]),
    "gs_render_workspace": (sz, [P(gs_view), i32, i64, i32]),
    "gs_render_fwd": (C.c_int, [P(gs_splats), P(gs_bins), P(gs_view), i32, P(C.c_float), i32, vp, sz,
                                vp, vp, vp, vp, vp, vp]),
    "gs_l1_loss": (C.c_int, [vp, vp, P(gs_view), i32, vp, vp, vp]),
    "gs_photometric_workspace": (sz, [P(gs_view), i32]),
    "gs_adam_step": (C.c_int, [P(gs_adam_group), i32, i64, C.c_double, C.c_double, C.c_double, vp]),
    "gs_densify_stats": (C.c_int, [P(gs_gauss3d), i32, vp, vp, i32, vp, vp, vp, vp, vp, vp]),
    "gs_densify_masks": (C.c_int, [i64, i32, vp, vp, vp, vp, C.c_float, C.c_float, i32, vp, vp, vp]),
    "gs_voxelize_workspace": (sz, [i64]),
    "gs_voxelize": (C.c_int, [vp, i64, C.c_float, vp, i64, vp, vp, i64, vp, vp, sz, vp, vp]),
    "gs_loop_closure": (C.c_int, [vp, i32, vp, vp, vp, i32, C.c_float, vp, vp]),
    "gs_flow_workspace": (sz, [i32]),
    "gs_flow_triangulate": (C.c_int, [vp, vp, i32, i32, vp, vp, i32, C.c_double, vp, vp, vp, i64, vp, vp, sz,
                                      vp, vp]),
    "gs_photometric_loss": (C.c_int, [vp, vp, P(gs_view), i32, C.c_float, vp, sz, vp, vp, vp]),
    "gs_render_bwd": (C.c_int, [P(gs_gauss3d), vp, P(gs_splats), P(gs_bins), P(gs_view), i32,
                                i32, vp, sz, vp, vp, vp, P(gs_splat_grad), P(gs_gauss3d_grad), vp, vp]),
    "gs_decode_project": (C.c_int, [P(gs_anchors), vp, P(gs_view), i32, i32, P(gs_gauss3d), P(gs_splats), vp,
                                    sz, vp, vp]),
    "gs_project_bwd": (C.c_int, [P(gs_gauss3d), vp, P(gs_splats), P(gs_view), i32, P(gs_splat_grad),
                                 P(gs_gauss3d_grad), vp, vp]),
    "gs_decode_project_bwd_workspace": (sz, [i32, i64, i32]),
    "gs_decode_project_bwd": (C.c_int, [P(gs_anchors), vp, P(gs_view), i32, i32, P(gs_gauss3d), P(gs_splats),
                                        P(gs_splat_grad), P(gs_anchor_grad), vp, sz, vp, vp]),
    "gs_decode_bwd": (C.c_int, [P(gs_anchors), vp, P(gs_view), i32, i32, P(gs_gauss3d),
                                P(gs_gauss3d_grad), P(gs_anchor_grad), vp, sz, vp, vp]),
}

_lib = None


def load():
    """Loads libgs.so from the package directory (built by build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgs.so not built ({LIB_PATH}); run paper_2607_21416_b300/build.py")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class GsError(RuntimeError):
    def __init__(self, call, code):
        super().__init__(f"{call}: {load().gs_status_string(code).decode()} ({code})")
        self.code = code


def check(call, code):
    if code != GS_OK:
        raise GsError(call, code)
