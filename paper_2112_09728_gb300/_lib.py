"""ctypes mirror of include/pg.h and the loader of libpg.so.

The loader fails loudly when the CUDA library has not been built; there is no
CPU fallback anywhere in the package.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpg.so")
LIB_BOUNDS_PATH = os.path.join(HERE, "_lib", "libpg_bounds.so")

PG_OK, PG_ERR_ARG, PG_ERR_CUDA, PG_ERR_OOM, PG_ERR_STATE, PG_ERR_TIMEOUT, PG_ERR_NUMERIC, PG_ERR_BOUNDS = range(8)
PG_F32, PG_F16, PG_BF16 = 0, 1, 2
STATUS_NAMES = {0: "PG_OK", 1: "PG_ERR_ARG", 2: "PG_ERR_CUDA", 3: "PG_ERR_OOM", 4: "PG_ERR_STATE",
                5: "PG_ERR_TIMEOUT", 6: "PG_ERR_NUMERIC", 7: "PG_ERR_BOUNDS"}


class pg_config(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32),
                ("gamma_dtype", C.c_int32), ("seed", C.c_uint64), ("k_max", C.c_int32),
                ("pi_min", C.c_float), ("pi_max", C.c_float), ("pi_reinit", C.c_float),
                ("depth_tol", C.c_float), ("normal_tol", C.c_float), ("rough_min", C.c_float),
                ("sigma2_min", C.c_float), ("rho_max", C.c_float), ("init_mu", C.c_float * 2),
                ("init_sigma", C.c_float * 3), ("init_pi", C.c_float), ("reuse_radius", C.c_int32),
                ("stochastic_round", C.c_int32), ("ggx_f0", C.c_float),
                ("transparent", C.c_int32), ("adam_dtype", C.c_int32)]


class pg_camera(C.Structure):
    _fields_ = [("kind", C.c_int32), ("origin", C.c_float * 3), ("fwd", C.c_float * 3),
                ("right", C.c_float * 3), ("up", C.c_float * 3), ("pixel_size", C.c_float),
                ("tan_half_fov", C.c_float)]


class pg_gbuffer(C.Structure):
    _fields_ = [("g0", C.c_void_p), ("g1", C.c_void_p), ("camera", pg_camera)]


class pg_field(C.Structure):
    _fields_ = [("n_lobes", C.c_int32), ("dir", (C.c_float * 3) * 8), ("kappa", C.c_float * 8),
                ("amp", C.c_float * 8), ("constant", C.c_float), ("mask_kind", C.c_int32),
                ("mask", C.c_float * 4), ("rgb", C.c_int32), ("amp_rgb", (C.c_float * 3) * 8),
                ("constant_rgb", C.c_float * 3)]


class pg_samples(C.Structure):
    _fields_ = [("wx", C.c_void_p), ("wy", C.c_void_p), ("wz", C.c_void_p),
                ("radiance", C.c_void_p), ("pdf", C.c_void_p), ("mis", C.c_void_p),
                ("estimate", C.c_void_p), ("strategy", C.c_void_p)]


_P = C.c_void_p
_SIGNATURES = {
    "pg_config_default": (None, [C.POINTER(pg_config), C.c_int32, C.c_int32]),
    "pg_create": (C.c_int, [C.POINTER(pg_config), _P, C.POINTER(_P)]),
    "pg_set_stream": (C.c_int, [_P, _P]),
    "pg_reproject": (C.c_int, [_P, C.POINTER(pg_gbuffer), _P, _P]),
    "pg_sample": (C.c_int, [_P, C.POINTER(pg_gbuffer), C.POINTER(pg_field), C.c_uint32,
                            C.POINTER(pg_samples), _P]),
    "pg_update": (C.c_int, [_P, C.POINTER(pg_gbuffer), C.POINTER(pg_samples)]),
    "pg_frame": (C.c_int, [_P, C.POINTER(pg_gbuffer), _P, C.POINTER(pg_field), C.c_uint32, _P]),
    "pg_frames_host": (C.c_int, [_P, C.c_int32, _P, _P, C.POINTER(pg_camera), C.POINTER(pg_field), C.c_uint32,
                                 _P, _P]),
    "pg_eval": (C.c_int, [_P, C.POINTER(pg_gbuffer), C.POINTER(pg_field), C.c_int32, _P, _P]),
    "pg_gamma_bytes": (C.c_size_t, [_P]),
    "pg_get_gamma": (C.c_int, [_P, _P, C.c_int32]),
    "pg_set_gamma": (C.c_int, [_P, _P, C.c_int32]),
    "pg_gamma_to_f32": (C.c_int, [_P, _P]),
    "pg_gamma_from_f32": (C.c_int, [_P, _P]),
    "pg_get_reprojected": (C.c_int, [_P, _P]),
    "pg_check": (C.c_int, [_P]),
    "pg_philox": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int32, _P]),
    "pg_grad": (C.c_int, [_P, C.POINTER(pg_gbuffer), C.POINTER(pg_field), C.c_uint32, C.c_int32, _P, _P, _P]),
    "pg_adam_step": (C.c_int, [_P, _P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int32]),
    "pg_get_adam_state": (C.c_int, [_P, _P, _P]),
    "pg_set_adam_state": (C.c_int, [_P, _P, _P]),
    "pg_theta_from_gamma": (C.c_int, [_P, _P]),
    "pg_theta_to_gamma": (C.c_int, [_P, _P]),
    "pg_frame_noalloc": (C.c_int, [C.POINTER(pg_config), C.POINTER(pg_gbuffer), _P, C.POINTER(pg_field), C.c_uint32,
                                   _P, _P, C.POINTER(pg_samples), _P, _P]),
    "pg_last_error": (C.c_char_p, [_P]),
    "pg_destroy": (None, [_P]),
}

_libs = {}


def exported_names():
    return list(_SIGNATURES)


def load(bounds_check: bool = False):
    """Load libpg.so, or with bounds_check its bounds-checked build
    libpg_bounds.so (both built in-tree by __graft_entry__.build())."""
    path = LIB_BOUNDS_PATH if bounds_check else LIB_PATH
    if path not in _libs:
        if not os.path.exists(path):
            raise RuntimeError("%s is not built; run __graft_entry__.build() first" % path)
        lib = C.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _libs[path] = lib
    return _libs[path]


class PgError(RuntimeError):
    def __init__(self, status, where, msg=""):
        super().__init__("%s failed with %s%s" % (where, STATUS_NAMES.get(status, status),
                                                   (": " + msg) if msg else ""))
        self.status = status
