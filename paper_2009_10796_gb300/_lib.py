"""ctypes declarations of ``include/ddgi.h``: argument marshalling only.

The shared library is built in-tree by ``build.py``.  Loading fails loudly if
it is missing: there is no CPU fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libddgi.so")

_lock = threading.Lock()
_lib = None

ERRORS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "TIMEOUT", 5: "NUMERIC", 6: "UNSUPPORTED"}

STATE_UNINIT, STATE_OFF, STATE_SLEEPING, STATE_NEWLY_VIGILANT, STATE_VIGILANT = 0, 1, 2, 3, 4
STATE_NEWLY_AWAKE, STATE_AWAKE = 5, 6
IRR_FP32, IRR_FP16, IRR_RGB9E5 = 0, 1, 2
DIST_FP32, DIST_FP16 = 0, 1
BLEND_FP32, BLEND_TF32, BLEND_BF16, BLEND_TF32X3 = 0, 1, 2, 3

F3 = C.c_float * 3


class Lights(C.Structure):
    _fields_ = [("sun_dir", F3), ("sun_irradiance", F3), ("sky_a", F3), ("sky_b", F3), ("sky_up", F3)]


class VolumeDesc(C.Structure):
    _fields_ = [("origin", F3), ("spacing", F3), ("counts", C.c_int32 * 3),
                ("rays_per_probe", C.c_int32), ("irr_n", C.c_int32), ("dist_n", C.c_int32),
                ("hysteresis_irr", C.c_float), ("hysteresis_vis", C.c_float), ("gamma", C.c_float),
                ("self_shadow_bias", C.c_float), ("dist_cos_power", C.c_float), ("t_max", C.c_float),
                ("thr_low", C.c_float), ("thr_high", C.c_float), ("thr_step", C.c_float),
                ("state_machine", C.c_int32), ("irr_format", C.c_int32), ("dist_format", C.c_int32),
                ("tracking", C.c_int32), ("seed", C.c_uint64), ("optimizer_iters", C.c_int32),
                ("offset_limit", C.c_float), ("converge_batches", C.c_int32)]


class VolumeInfo(C.Structure):
    _fields_ = [("n_probes", C.c_int64), ("irr_tile_texels", C.c_int64),
                ("dist_tile_texels", C.c_int64), ("irr_bytes", C.c_int64), ("dist_bytes", C.c_int64),
                ("irr_texel_bytes", C.c_int64), ("dist_texel_bytes", C.c_int64), ("t_max", C.c_float)]


class UpdateParams(C.Structure):
    _fields_ = [("frame", C.c_int64), ("irr_hyst_scale", C.c_float), ("vis_hyst_scale", C.c_float),
                ("blend_precision", C.c_int32), ("reserved", C.c_int32)]


class CascadeParams(C.Structure):
    _fields_ = [("frame", C.c_int64), ("camera_pos", F3), ("irr_hyst_scale", C.c_float),
                ("vis_hyst_scale", C.c_float), ("blend_precision", C.c_int32), ("use_graph", C.c_int32)]


_vp = C.c_void_p
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)

# name -> (restype, argtypes); every exported entry point of include/ddgi.h
SIGNATURES = {
    "ddgi_last_error": (C.c_char_p, []),
    "ddgi_version": (C.c_int32, []),
    "ddgi_texel_bytes": (C.c_int32, [C.c_int32, C.c_int32]),
    "ddgi_scene_create": (C.c_int, [_vp, C.c_int64, _vp, C.c_int64, _vp, C.c_int32, _vp, _vp, _vp,
                                    C.c_int32, _vp, C.POINTER(_vp)]),
    "ddgi_scene_destroy": (None, [_vp]),
    "ddgi_scene_info": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "ddgi_bvh_check": (C.c_int, [_vp, C.c_int64, _vp, C.c_int64, C.c_int64 * 9]),
    "ddgi_trace": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp, _vp]),
    "ddgi_raycast_gbuffer": (C.c_int, [_vp, F3, F3, F3, C.c_float, C.c_int32, C.c_int32, _vp, _vp, _vp]),
    "ddgi_volume_create": (C.c_int, [C.POINTER(VolumeDesc), C.POINTER(_vp)]),
    "ddgi_volume_destroy": (None, [_vp]),
    "ddgi_volume_get_info": (C.c_int, [_vp, C.POINTER(VolumeInfo)]),
    "ddgi_update": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.POINTER(UpdateParams), _vp]),
    "ddgi_query": (C.c_int, [_vp, _vp, _vp, C.c_int64, F3, _vp, _vp]),
    "ddgi_query_glossy": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, _vp, _vp]),
    "ddgi_frame_host": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.POINTER(UpdateParams), _vp, _vp, C.c_int64, F3,
                                  _vp, _vp]),
    "ddgi_set_dynamic_boxes": (C.c_int, [_vp, _vp, C.c_int32]),
    "ddgi_update_range": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.POINTER(UpdateParams), C.c_int64, C.c_int64,
                                    _vp]),
    "ddgi_get_buffer": (C.c_int, [_vp, C.c_int32, _vp, C.c_size_t, _vp]),
    "ddgi_set_buffer": (C.c_int, [_vp, C.c_int32, _vp, C.c_size_t, _vp]),
    "ddgi_get_ray_records": (C.c_int, [_vp, _vp, _vp, C.POINTER(C.c_int64), _vp]),
    "ddgi_enable_timing": (C.c_int, [_vp, C.c_int32]),
    "ddgi_read_timings": (C.c_int, [_vp, C.c_float * 8, C.c_int32 * 8]),
    "ddgi_poll_status": (C.c_int, [_vp, _vp]),
    "ddgi_trace_stats": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.c_uint64 * 7, _vp]),
    "ddgi_update_noalloc": (C.c_int, [_vp, C.POINTER(VolumeDesc), C.POINTER(Lights),
                                      C.POINTER(UpdateParams), _vp, _vp, _vp, _vp]),
    "ddgi_update_noalloc_poll_status": (C.c_int, [_vp]),
    "ddgi_measure_l2_read": (C.c_int, [_vp, C.c_size_t, C.c_int32, _vp, _vp]),
    "ddgi_volume_save": (C.c_int, [_vp, _vp, C.POINTER(C.c_size_t), _vp]),
    "ddgi_volume_load": (C.c_int, [_vp, _vp, C.c_size_t, _vp]),
    "ddgi_query_backward": (C.c_int, [_vp, _vp, _vp, C.c_int64, F3, _vp, C.c_int32, _vp, _vp]),
    "ddgi_diff_forward_f64": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.c_int64, C.c_int32, _vp, _vp, _vp, _vp,
                                        C.c_int64, F3, _vp, _vp]),
    "ddgi_diff_backward_f64": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.c_int64, C.c_int32, _vp, _vp, _vp,
                                         C.c_int64, F3, _vp, _vp, _vp, _vp]),
    "ddgi_cascade_create": (C.c_int, [C.POINTER(VolumeDesc), C.c_int32, C.POINTER(_vp)]),
    "ddgi_cascade_destroy": (None, [_vp]),
    "ddgi_cascade_update": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.POINTER(CascadeParams), _vp]),
    "ddgi_cascade_query": (C.c_int, [_vp, _vp, _vp, C.c_int64, F3, _vp, _vp]),
    "ddgi_cascade_get_buffer": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp, C.c_size_t, _vp]),
    "ddgi_cascade_get_window": (C.c_int, [_vp, C.c_int32, C.c_double * 3, C.c_int32 * 3]),
    "ddgi_cascade_get_ray_records": (C.c_int, [_vp, _vp, _vp, C.POINTER(C.c_int64), _vp]),
    "ddgi_cascade_set_tuning": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "ddgi_cascade_get_tuning": (C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "ddgi_cascade_autotune": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.POINTER(CascadeParams), C.c_char_p,
                                        C.POINTER(C.c_int32), _vp]),
    "ddgi_cascade_poll_status": (C.c_int, [_vp, _vp]),
    "ddgi_scene_set_materials": (C.c_int, [_vp, _vp, _vp, _vp]),
    "ddgi_diff_forward": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.c_int64, C.c_int32, _vp, _vp, C.c_int64, F3,
                                    _vp, _vp]),
    "ddgi_diff_backward": (C.c_int, [_vp, _vp, C.POINTER(Lights), C.c_int64, C.c_int32, _vp, _vp, C.c_int64, F3,
                                     _vp, _vp, _vp, _vp]),
}


class DDGIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ddgi error {ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libddgi.so (raise if it is missing) and declare every entry point."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"libddgi.so not found at {path}: build it with "
                "`python -m paper_2009_10796_gb300.build` (the CUDA path has no fallback)")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(code: int):
    if code != 0:
        raise DDGIError(code, load().ddgi_last_error().decode())
