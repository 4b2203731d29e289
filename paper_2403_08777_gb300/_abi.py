"""ctypes declarations of the nsrhs C ABI (include/nsrhs.h). Marshalling only."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

OK, EINVAL, ENOMEM, EMESH, ECUDA, EUNSUPPORTED = 0, 1, 2, 3, 4, 5
FP64, MIXED = 0, 1
SCATTER_AUTO, SCATTER_ATOMIC, SCATTER_BLOCK, SCATTER_COLOUR, SCATTER_BLOCK_COLOUR = 0, 1, 2, 3, 4
CONVECTIVE, SKEW = 0, 1
TAU_GAUSS, TAU_ELEMENT = 0, 1
GEOM_CACHED, GEOM_RECOMPUTE = 0, 1
EULER, SSPRK3 = 0, 1
ELEMENT_COLOUR, ELEMENT_BLOCK_COLOUR, ELEMENT_BLOCK = 0, 1, 2

# Every symbol include/nsrhs.h declares.
EXPORTED = ("nsrhs_params_default", "nsrhs_mesh_opts_default", "nsrhs_mesh_create",
            "nsrhs_mesh_get_info", "nsrhs_assemble", "nsrhs_assemble_vjp", "nsrhs_destroy",
            "nsrhs_status_string", "nsrhs_probe_fma", "nsrhs_mesh_check_noalloc",
            "nsrhs_probe_special", "nsrhs_lumped_mass", "nsrhs_explicit_step",
            "nsrhs_assemble_elmat", "nsrhs_mesh_element_colours", "nsrhs_assemble_rhs_vjp")


class Params(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("mu", ctypes.c_double), ("c_vreman", ctypes.c_double),
                ("c1", ctypes.c_double), ("c2", ctypes.c_double), ("precision", ctypes.c_int32),
                ("scatter", ctypes.c_int32), ("convection", ctypes.c_int32),
                ("tau_mode", ctypes.c_int32), ("geometry", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class MeshOpts(ctypes.Structure):
    _fields_ = [("ar_threshold", ctypes.c_double), ("colour", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class MeshCheckResult(ctypes.Structure):
    _fields_ = [("bad_index", ctypes.c_int64), ("bad_det", ctypes.c_int64),
                ("n_high_ar", ctypes.c_int64), ("min_detj", ctypes.c_double),
                ("max_ar", ctypes.c_double)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_elems", ctypes.c_int64),
                ("n_high_ar", ctypes.c_int64), ("n_blocks", ctypes.c_int64),
                ("block_elems", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("min_detj", ctypes.c_double), ("max_ar", ctypes.c_double),
                ("n_colours", ctypes.c_int64), ("n_block_colours", ctypes.c_int64)]


_lib = None


class NativeLibraryMissing(RuntimeError):
    pass


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libnsrhs.so. Raises NativeLibraryMissing if it has not been built:
    there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise NativeLibraryMissing(
            f"nsrhs CUDA library not found at {path}; build it with "
            "paper_2403_08777_gb300.build.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    lib.nsrhs_params_default.argtypes = [ctypes.POINTER(Params)]
    lib.nsrhs_params_default.restype = None
    lib.nsrhs_mesh_opts_default.argtypes = [ctypes.POINTER(MeshOpts)]
    lib.nsrhs_mesh_opts_default.restype = None
    lib.nsrhs_mesh_create.argtypes = [I64, I64, P, P, ctypes.POINTER(MeshOpts), P,
                                      ctypes.POINTER(P)]
    lib.nsrhs_mesh_create.restype = ctypes.c_int
    lib.nsrhs_mesh_get_info.argtypes = [P, ctypes.POINTER(MeshInfo)]
    lib.nsrhs_mesh_get_info.restype = ctypes.c_int
    lib.nsrhs_assemble.argtypes = [P, ctypes.POINTER(Params), P, P, P]
    lib.nsrhs_assemble.restype = ctypes.c_int
    lib.nsrhs_assemble_vjp.argtypes = [P, ctypes.POINTER(Params), P, P, P, P]
    lib.nsrhs_assemble_vjp.restype = ctypes.c_int
    lib.nsrhs_destroy.argtypes = [P]
    lib.nsrhs_destroy.restype = None
    lib.nsrhs_status_string.argtypes = [ctypes.c_int]
    lib.nsrhs_status_string.restype = ctypes.c_char_p
    lib.nsrhs_probe_fma.argtypes = [ctypes.c_int, I64, I64, P, P]
    lib.nsrhs_probe_fma.restype = ctypes.c_int
    lib.nsrhs_assemble_elmat.argtypes = [P, ctypes.POINTER(Params), P, P, P]
    lib.nsrhs_assemble_elmat.restype = ctypes.c_int
    lib.nsrhs_lumped_mass.argtypes = [P, P, P]
    lib.nsrhs_lumped_mass.restype = ctypes.c_int
    lib.nsrhs_explicit_step.argtypes = [P, ctypes.POINTER(Params), ctypes.c_double, ctypes.c_int32,
                                        P, P, P]
    lib.nsrhs_explicit_step.restype = ctypes.c_int
    lib.nsrhs_probe_special.argtypes = [ctypes.c_int, I64, P, P, P, P]
    lib.nsrhs_probe_special.restype = ctypes.c_int
    lib.nsrhs_mesh_check_noalloc.argtypes = [I64, I64, P, P, ctypes.c_double, P, P]
    lib.nsrhs_mesh_check_noalloc.restype = ctypes.c_int
    lib.nsrhs_mesh_element_colours.argtypes = [P, ctypes.c_int32, P, P]
    lib.nsrhs_mesh_element_colours.restype = ctypes.c_int
    lib.nsrhs_assemble_rhs_vjp.argtypes = [P, ctypes.POINTER(Params), P, P, P, P, P]
    lib.nsrhs_assemble_rhs_vjp.restype = ctypes.c_int
    _lib = lib
    return lib


class NSRHSError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = load().nsrhs_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})")
        self.status = status


def check(status: int, what: str) -> None:
    if status != OK:
        raise NSRHSError(status, what)
