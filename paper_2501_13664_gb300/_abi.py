"""ctypes binding of libdrt3d (include/drt3d.h): names, signatures, status checks.

Argument marshalling only: every step of every transform runs in the CUDA
library.  If the library cannot be loaded the import raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

_lib = None

P = ctypes.c_void_p
I = ctypes.c_int
U32 = ctypes.c_uint32
SZ = ctypes.c_size_t
I64P = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); mirrors include/drt3d.h
SIGNATURES = {
    "drt3d_plan_create": (I, [ctypes.POINTER(P), I, I, ctypes.c_uint]),
    "drt3d_plan_destroy": (I, [P]),
    "drt3d_planes_out_shape": (I, [P, I64P]),
    "drt3d_lines_out_shape": (I, [P, I64P]),
    "drt3d_workspace_bytes": (I, [P, I, ctypes.POINTER(SZ)]),
    "drt3d_planes_forward": (I, [P, P, P, U32, P, SZ, P]),
    "drt3d_planes_forward_residual": (I, [P, P, P, P, U32, P, SZ, P]),
    "drt3d_planes_adjoint": (I, [P, P, P, U32, P, SZ, P]),
    "drt3d_planes_inverse": (I, [P, P, I, P, P, SZ, P]),
    "djt3d_lines_forward": (I, [P, P, P, U32, P, SZ, P]),
    "djt3d_lines_adjoint": (I, [P, P, P, U32, P, SZ, P]),
    "drt3d_planes_forward_global": (I, [P, P, P, P, SZ, P]),
    "drt2d_forward": (I, [P, P, I, P, U32, P, SZ, P]),
    "drt3d_planes_press_inverse": (I, [P, P, P, I, I, ctypes.POINTER(ctypes.c_float), P, SZ, P]),
    "drt3d_press_spectral_radius": (I, [P, I, P, I, ctypes.POINTER(ctypes.c_double), P, SZ, P]),
    "drt2d_workspace_bytes": (I, [P, I, U32, ctypes.POINTER(SZ)]),
    "drt3d_get_device_error": (I, [P, P]),
    "drt3d_status_string": (ctypes.c_char_p, [I]),
    "drt3d_set_profiling": (I, [P, I]),
    "drt3d_profiled_launches": (I, [P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double), I,
                                    ctypes.POINTER(I)]),
    "drt3d_profiled_launch_name": (ctypes.c_char_p, [P, I]),
    "drt3d_version": (I, []),
    "drt3d_planes_forward_noalloc": (I, [P, P, P, U32, P]),
    "drt3d_plan_set_schedule": (I, [P, I, ctypes.POINTER(I)]),
    "drt3d_plan_get_schedule": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
    "drt3d_batch_plan_create": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I), I, ctypes.c_uint]),
    "drt3d_batch_plan_destroy": (I, [P]),
    "drt3d_batch_set_schedule": (I, [P, I, I, ctypes.POINTER(I)]),
    "drt3d_batch_set_item_tiles": (I, [P, I, I, ctypes.POINTER(I)]),
    "drt3d_plan_set_adjoint_schedule": (I, [P, I, ctypes.POINTER(I)]),
    "drt3d_planes_forward_residual_loss": (I, [P, P, P, P, U32, P, P, SZ, P]),
    "drt3d_plan_get_adjoint_schedule": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
    "drt3d_batch_workspace_bytes": (I, [P, ctypes.POINTER(SZ)]),
    "drt3d_batch_bind": (I, [P, P, P, SZ]),
    "drt3d_planes_forward_batched": (I, [P, P]),
    "drt3d_batch_set_mode": (I, [P, I, I]),
    "drt3d_batch_get_device_error": (I, [P, P]),
    "drt3d_batch_set_wait_limit": (I, [P, ctypes.c_ulonglong, I, I]),
    "drt3d_noalloc_scratch_bytes": (SZ, []),
}

STATUS = {
    0: "DRT3D_OK", 1: "DRT3D_ERR_INVALID_ARG", 2: "DRT3D_ERR_SIZE", 3: "DRT3D_ERR_DTYPE",
    4: "DRT3D_ERR_ALIGN", 5: "DRT3D_ERR_WORKSPACE", 6: "DRT3D_ERR_NOT_IN_RANGE",
    7: "DRT3D_ERR_TIMEOUT", 8: "DRT3D_ERR_BOUNDS", 9: "DRT3D_ERR_CUDA", 10: "DRT3D_ERR_NO_MEMORY",
    11: "DRT3D_ERR_SCRATCH_LIMIT",
}
DTYPES = {"u8": 0, "i16": 1, "i32": 2, "f32": 3}
OPS = {"planes_forward": 0, "planes_adjoint": 1, "planes_inverse": 2, "lines_forward": 3, "lines_adjoint": 4,
       "planes_press": 5, "planes_residual_loss": 6}


class DRT3DError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


def header_functions(path: str | None = None) -> list:
    """Names of the functions declared in include/drt3d.h."""
    path = path or os.path.join(_build.INCLUDE, "drt3d.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*((?:drt3d|djt3d)_\w+)\s*\(", text, flags=re.M)


def lib(build: bool = True):
    """Load (building first if needed) libdrt3d.so and set its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libdrt3d.so not found at {path}; run the package build first")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(code: int, where: str) -> None:
    if code != 0:
        raise DRT3DError(code, where)
