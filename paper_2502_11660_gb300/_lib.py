"""Loads libmsm377.so and declares the C signatures of include/msm377.h.

There is no fallback: if the library cannot be built or loaded, every call
raises. The library is built in-tree on first use when it is missing or older
than its sources.
"""
from __future__ import annotations

import ctypes
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_u32p = ctypes.c_void_p   # device pointers travel as plain addresses
c_size = ctypes.c_size_t
c_int = ctypes.c_int
c_void = ctypes.c_void_p


class MsmOpts(ctypes.Structure):
    _fields_ = [
        ("c", ctypes.c_int32),
        ("signed_digits", ctypes.c_int32),
        ("scalar_bits", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("stream", ctypes.c_void_p),
    ]


class MsmJob(ctypes.Structure):
    _fields_ = [
        ("points", ctypes.c_void_p),
        ("scalars", ctypes.c_void_p),
        ("n", ctypes.c_size_t),
        ("out", ctypes.c_void_p),
        ("c", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


SIGNATURES = {
    "msm377_last_error": (c_int, [ctypes.c_char_p, c_size]),
    "msm377_version": (c_int, []),
    "fq_mul_batch": (c_int, [c_u32p, c_u32p, c_u32p, c_size, c_int, c_void]),
    "fq_to_montgomery": (c_int, [c_u32p, c_u32p, c_size, c_void]),
    "fq_mul_batch_variant": (c_int, [c_u32p, c_u32p, c_u32p, c_size, c_int, c_void]),
    "fq_from_montgomery": (c_int, [c_u32p, c_u32p, c_size, c_void]),
    "padd_batch": (c_int, [c_u32p, c_u32p, c_u32p, c_size, c_int, c_void]),
    "xyzz_to_affine_batch": (c_int, [c_u32p, c_u32p, c_size, c_int, c_void]),
    "g1_generator_mul": (c_int, [c_u32p, c_size, c_u32p, c_void]),
    "msm_g1_workspace_bytes": (c_size, [c_size, ctypes.POINTER(MsmOpts)]),
    "msm_g1_default_c": (c_int, [c_size, c_int, ctypes.c_uint32]),
    "msm_g1_set_window_table": (c_int, [ctypes.POINTER(ctypes.c_int32), c_int, ctypes.c_uint32]),
    "msm_points_prepare": (c_int, [c_u32p, c_size, c_u32p, c_void]),
    "msm_points_prepare_ex": (c_int, [c_u32p, c_size, c_u32p, ctypes.c_uint32, c_void]),
    "msm_points_prepared_bytes": (c_size, [c_size, ctypes.c_uint32]),
    "msm_points_precomputed_bytes": (c_size, [c_size, ctypes.POINTER(MsmOpts)]),
    "msm_points_precompute": (c_int, [c_u32p, c_size, c_u32p, ctypes.POINTER(MsmOpts)]),
    "msm_g1": (c_int, [c_u32p, c_u32p, c_size, c_u32p, c_void, c_size, ctypes.POINTER(MsmOpts)]),
    "msm_g1_status": (c_int, [c_void, ctypes.POINTER(MsmOpts)]),
    "msm_g1_host_workspace_bytes": (c_size, [c_size, ctypes.POINTER(MsmOpts)]),
    "msm_g1_host": (c_int, [c_void, c_void, c_size, c_void, c_void, c_size, ctypes.POINTER(MsmOpts)]),
    "msm377_imad_probe": (c_int, [c_int, ctypes.POINTER(ctypes.c_double), c_void]),
    "msm377_profile_last": (c_int, [ctypes.POINTER(ctypes.c_float), c_int]),
    "msm377_launch_count": (ctypes.c_uint64, []),
    "msm_g1_noalloc": (c_int, [c_u32p, c_u32p, c_size, c_u32p, ctypes.POINTER(MsmOpts)]),
    "padd_chain": (c_int, [c_u32p, c_size, c_u32p, ctypes.c_uint32, c_int, c_void]),
    "msm_g1_batched_workspace_bytes": (c_size, [ctypes.POINTER(MsmJob), c_size, ctypes.POINTER(MsmOpts)]),
    "msm_g1_batched": (c_int, [ctypes.POINTER(MsmJob), c_size, c_void, c_size, ctypes.POINTER(MsmOpts)]),
    "msm_points_validate": (c_int, [c_u32p, c_size, ctypes.c_uint32, c_void]),
    "msm_g1_set_schedule": (c_int, [ctypes.c_uint32, c_int, c_int, c_int, c_int, c_int, c_int]),
    "msm_g1_schedule": (c_int, [c_size, ctypes.POINTER(MsmOpts), ctypes.POINTER(ctypes.c_int32)]),
    "msm_points_create": (c_int, [c_u32p, c_size, ctypes.POINTER(MsmOpts), ctypes.POINTER(ctypes.c_void_p)]),
    "msm_points_destroy": (c_int, [c_void]),
    "msm_points_count": (c_size, [c_void]),
    "msm_points_data": (c_void, [c_void, c_size]),
    "msm_g1_resident_workspace_bytes": (c_size, [c_void, c_size, ctypes.POINTER(MsmOpts)]),
    "msm_g1_resident": (c_int, [c_void, c_size, c_size, c_u32p, c_u32p, c_void, c_size, ctypes.POINTER(MsmOpts)]),
    "msm_g1_resident_host_workspace_bytes": (c_size, [c_void, c_size, ctypes.POINTER(MsmOpts)]),
    "msm_g1_resident_host": (c_int, [c_void, c_size, c_size, c_void, c_void, c_void, c_size,
                                     ctypes.POINTER(MsmOpts)]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class MsmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"msm377 error {code}: {msg}")
        self.code = code


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    lib().msm377_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def check(rc: int) -> int:
    if rc != 0:
        raise MsmError(rc, last_error())
    return rc
