"""ctypes declarations of the qrt C ABI (include/qrt.h), names unchanged.

Argument marshalling only: every computation happens in libqrt.so.  Loading
fails loudly when the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqrt.so")

QRT_OK = 0
QRT_ERR_INVALID_ARG = -1
QRT_ERR_ALIGN = -2
QRT_ERR_OOM = -3
QRT_ERR_CUDA = -4
QRT_ERR_STACK_OVERFLOW = -5
QRT_ERR_STEP_LIMIT = -6
QRT_ERR_NOT_READY = -7

QRT_FLAG_STAGE_TIMES = 1
STAGES = ("gen", "trace_closest", "shade", "trace_shadow", "accumulate")

ERROR_NAMES = {
    QRT_ERR_INVALID_ARG: "QRT_ERR_INVALID_ARG", QRT_ERR_ALIGN: "QRT_ERR_ALIGN",
    QRT_ERR_OOM: "QRT_ERR_OOM", QRT_ERR_CUDA: "QRT_ERR_CUDA",
    QRT_ERR_STACK_OVERFLOW: "QRT_ERR_STACK_OVERFLOW", QRT_ERR_STEP_LIMIT: "QRT_ERR_STEP_LIMIT",
    QRT_ERR_NOT_READY: "QRT_ERR_NOT_READY",
}


class qrt_mesh(C.Structure):
    _fields_ = [("verts", C.POINTER(C.c_float)), ("n_verts", C.c_uint32),
                ("quads", C.POINTER(C.c_uint32)), ("n_quads", C.c_uint32)]


class qrt_view(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("w", C.c_uint32), ("h", C.c_uint32),
                ("spp", C.c_uint32), ("sample_base", C.c_uint32), ("pixel_base", C.c_uint64),
                ("out_rgb", C.c_void_p), ("crop_x", C.c_uint32), ("crop_y", C.c_uint32),
                ("crop_w", C.c_uint32), ("crop_h", C.c_uint32)]


class qrt_tuning(C.Structure):
    _fields_ = [("block", C.c_uint32), ("blocks_per_sm", C.c_uint32), ("batch", C.c_uint32),
                ("stack", C.c_uint32), ("fetch", C.c_uint32), ("occupancy", C.c_uint32),
                ("mode", C.c_uint32), ("chunk_log2", C.c_uint32)]


class qrt_params(C.Structure):
    _fields_ = [("max_depth", C.c_uint32), ("flags", C.c_uint32), ("seed", C.c_uint64),
                ("env", C.c_float * 3), ("sun_dir", C.c_float * 3), ("sun_E", C.c_float * 3),
                ("max_steps", C.c_uint32), ("d_path_log", C.c_void_p), ("tuning", qrt_tuning),
                ("d_ray_log", C.c_void_p), ("d_tex", C.c_void_p), ("tex_res", C.c_uint32),
                ("n_lights", C.c_uint32), ("lights", C.POINTER(C.c_float))]


class qrt_build_opts(C.Structure):
    _fields_ = [("max_leaf", C.c_uint32), ("sah_bins", C.c_uint32), ("threads", C.c_uint32),
                ("degenerate", C.c_uint32), ("inst_boxes", C.c_uint32), ("tlas_builder", C.c_uint32),
                ("blas_builder", C.c_uint32)]


class qrt_scene_stats(C.Structure):
    _fields_ = [("n_meshes", C.c_uint64), ("n_instances", C.c_uint64), ("n_quads", C.c_uint64),
                ("blas_nodes", C.c_uint64), ("tlas_nodes", C.c_uint64),
                ("device_bytes", C.c_uint64), ("max_blas_depth", C.c_uint32),
                ("tlas_depth", C.c_uint32), ("build_seconds", C.c_double),
                ("phase_seconds", C.c_double * 6)]


_vp = C.c_void_p
_i = C.c_int
_u32 = C.c_uint32
_u64 = C.c_uint64

# name -> (restype, argtypes); one entry per function declared in qrt.h
SIGNATURES = {
    "qrt_last_error": (C.c_char_p, []),
    "qrt_version": (_i, []),
    "qrt_scene_create": (_i, [C.POINTER(qrt_mesh), _u32, C.POINTER(C.c_float),
                              C.POINTER(C.c_uint32), _u64, C.POINTER(qrt_build_opts),
                              C.POINTER(_vp)]),
    "qrt_scene_destroy": (_i, [_vp]),
    "qrt_scene_stats_get": (_i, [_vp, C.POINTER(qrt_scene_stats)]),
    "qrt_trace_closest": (_i, [_vp, _vp, _u64, _vp, C.POINTER(qrt_tuning), _vp]),
    "qrt_trace_any": (_i, [_vp, _vp, _u64, _vp, C.POINTER(qrt_tuning), _vp]),
    "qrt_render_spp": (_i, [_vp, C.POINTER(qrt_view), _u32, _vp, C.POINTER(qrt_params), _vp]),
    "qrt_render_spp_static": (_i, [_vp, C.POINTER(qrt_view), _u32, _vp, C.POINTER(qrt_params), _vp]),
    "qrt_render_adjoint": (_i, [_vp, C.POINTER(qrt_view), _u32, _vp, C.POINTER(_vp), _vp,
                                C.POINTER(qrt_params), _vp]),
    "qrt_accumulate": (_i, [_vp, _vp, _vp, _u64, _u32, _vp]),
    "qrt_l2_loss": (_i, [_vp, _vp, _u64, _vp, _vp, _vp]),
    "qrt_read_bandwidth": (_i, [_vp, _u64, _u32, _vp, _vp]),
    "qrt_render_graph_create": (_i, [_vp, C.POINTER(qrt_view), _u32, _vp, C.POINTER(qrt_params),
                                     C.POINTER(_vp)]),
    "qrt_graph_launch": (_i, [_vp, _vp]),
    "qrt_graph_destroy": (_i, [_vp]),
    "qrt_render_spp_stats": (_i, [_vp, C.POINTER(qrt_view), _u32, _vp, C.POINTER(qrt_params),
                                  _vp, _vp]),
    "qrt_render_cost": (_i, [_vp, C.POINTER(qrt_view), _u32, _vp, C.POINTER(qrt_params), _vp, _vp, _vp]),
    "qrt_trace_stats": (_i, [_vp, _i, _vp, _u64, _vp, C.POINTER(qrt_tuning), _vp, _vp]),
    "qrt_stage_times": (_i, [_vp, _vp, C.POINTER(C.c_double), C.POINTER(C.c_uint32), _i]),
    "qrt_check": (_i, [_vp, _vp]),
    "qrt_blas_build_check": (_i, [C.POINTER(qrt_mesh), C.POINTER(qrt_build_opts),
                                  C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]),
    "qrt_tlas_build_check": (_i, [_vp, _u64, C.POINTER(qrt_build_opts), C.POINTER(C.c_uint64),
                                  C.POINTER(C.c_uint32)]),
    "qrt_blases_build_check": (_i, [_vp, _u32, C.POINTER(qrt_build_opts), C.POINTER(C.c_uint64),
                                    C.POINTER(C.c_uint32)]),
    "qrt_test_sort_pairs": (_i, [_vp, _vp, _u64, _u32, _vp, _vp]),
}

_lock = threading.Lock()
_lib = None


class QrtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib():
    """The loaded libqrt.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libqrt.so not found at {LIB_PATH}: build it first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != QRT_OK:
        raise QrtError(rc, lib().qrt_last_error().decode(errors="replace"))
