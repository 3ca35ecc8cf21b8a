"""ctypes binding of libdressi.so (include/dressi.h): argument marshalling only.

Every step of the render and its adjoint runs in the library's CUDA kernels;
this module only packs torch tensors into the C structs and passes device
pointers and the current CUDA stream.  There is no CPU fallback: if the
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdressi.so")

DRESSI_OK, DRESSI_ERR_ARG, DRESSI_ERR_WORKSPACE, DRESSI_ERR_LAUNCH = 0, 1, 2, 3
DEV_TILE_OVERFLOW, DEV_FACE_RANGE, DEV_NONFINITE = 1, 2, 4
TEX_F32, TEX_F16 = 0, 1
MAX_K = 5


class DressiMesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_faces", C.c_int32), ("vert_off", C.c_int64),
                ("face_off", C.c_int64), ("tex_off", C.c_int64), ("tex_w", C.c_int32), ("tex_h", C.c_int32)]


class DressiScene(C.Structure):
    _fields_ = [("n_meshes", C.c_int32), ("meshes", C.POINTER(DressiMesh)), ("n_verts_total", C.c_int64),
                ("pos", C.c_void_p), ("col", C.c_void_p), ("uv", C.c_void_p), ("faces", C.c_void_p),
                ("tex", C.c_void_p), ("tex_dtype", C.c_int32), ("ntex", C.c_void_p)]


class DressiView(C.Structure):
    _fields_ = [("mvp", C.c_float * 16), ("light", C.c_float * 3), ("mesh", C.c_int32),
                ("width", C.c_int32), ("height", C.c_int32), ("pix_off", C.c_int64)]


class DressiParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("r", C.c_float), ("sigma", C.c_float), ("delta", C.c_float),
                ("gamma", C.c_float), ("edge_mode", C.c_int32), ("shade_mode", C.c_int32),
                ("texgrad_mode", C.c_int32), ("tile", C.c_int32), ("schedule", C.c_int32),
                ("list_cap", C.c_int64), ("uv_jitter", C.c_float * 2), ("reuse_setup", C.c_int32)]


# every symbol declared in include/dressi.h, with its ctypes signature
ABI_VERSION = 3   # DRESSI_ABI_VERSION of include/dressi.h

SIGNATURES = {
    "dressi_workspace_size": (C.c_size_t, [C.POINTER(DressiScene), C.POINTER(DressiView), C.c_int32,
                                           C.POINTER(DressiParams)]),
    "dressi_forward": (C.c_int, [C.POINTER(DressiScene), C.POINTER(DressiView), C.c_int32, C.POINTER(DressiParams),
                                 C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "dressi_forward_l2": (C.c_int, [C.POINTER(DressiScene), C.POINTER(DressiView), C.c_int32,
                                    C.POINTER(DressiParams), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "dressi_backward": (C.c_int, [C.POINTER(DressiScene), C.POINTER(DressiView), C.c_int32, C.POINTER(DressiParams),
                                  C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "dressi_backward_ex": (C.c_int, [C.POINTER(DressiScene), C.POINTER(DressiView), C.c_int32, C.POINTER(DressiParams),
                                     C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p,
                                     C.c_void_p]),
    "dressi_forward_from_layers": (C.c_int, [C.POINTER(DressiScene), C.POINTER(DressiView), C.c_int32,
                                             C.POINTER(DressiParams), C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                             C.c_size_t, C.c_void_p, C.c_void_p]),
    "dressi_forward_static_scratch": (C.c_int, [C.POINTER(DressiScene), C.POINTER(DressiView), C.c_int32,
                                                C.POINTER(DressiParams), C.c_void_p, C.c_void_p, C.c_int64,
                                                C.c_void_p, C.c_void_p]),
    "dressi_autotune": (C.c_int, [C.POINTER(DressiScene), C.POINTER(DressiView), C.c_int32, C.POINTER(DressiParams),
                                  C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_size_t, C.c_void_p, C.c_void_p, C.POINTER(C.c_float)]),
    "dressi_l2_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dressi_status_string": (C.c_char_p, [C.c_int]),
    "dressi_dev_status_string": (C.c_char_p, [C.c_int]),
    "dressi_abi_version": (C.c_int, []),
    "dressi_set_profile_events": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dressi_launch_count": (C.c_ulonglong, []),
    "dressi_set_stats_buffer": (C.c_int, [C.c_void_p]),
    "dressi_set_inverse_uv_buffer": (C.c_int, [C.c_void_p]),
    "dressi_set_tile_order_buffer": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dressi_measure_peak": (C.c_int, [C.c_int32, C.c_void_p, C.c_size_t, C.POINTER(C.c_double), C.c_void_p]),
}

_lock = threading.Lock()
_lib = None


class DressiError(RuntimeError):
    pass


def load(path: str = LIB_PATH):
    """Loads libdressi.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise DressiError(f"libdressi.so not built ({path}); run __graft_entry__.build()")
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            if lib.dressi_abi_version() != ABI_VERSION:
                raise DressiError("libdressi.so ABI version mismatch")
            _lib = lib
    return _lib


def check(code: int, what: str):
    if code != DRESSI_OK:
        msg = load().dressi_status_string(code).decode()
        raise DressiError(f"{what}: {msg} (code {code})")
