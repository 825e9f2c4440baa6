"""ctypes binding of libmfcg.so (include/mfcg.h): argument marshalling only.

Every step of the solver runs in the CUDA library; this module converts torch
tensors to device pointers, checks shapes and dtypes, and turns status codes
into exceptions.  There is no fallback: if the library is missing the import
of the functions that need it raises.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libmfcg.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "mfcg.h")

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_DEGREE", 3: "OUT_OF_MEMORY", 4: "CUDA_ERROR",
          5: "NOT_CONVERGED", 6: "BREAKDOWN", 7: "DEVICE_TIMEOUT", 8: "SCRATCH_TOO_SMALL"}
OK, NOT_CONVERGED, BREAKDOWN = 0, 5, 6

GEOM = {"affine": 0, "deformed": 1, "deformed_tensor": 2, "user": 3, "deformed_quadratic": 4}
COEF = {"constant": 0, "sin_x": 1}
MODE = {"fused": 0, "unfused": 1, "semi_fused": 2, "loop_fused": 3}
PRECONDITIONER = {"jacobi": 0, "none": 1}
PRECISION = {"fp64": 0, "double_float": 1, "fp32_inner": 2, "double_float_inner": 3}
OPERATOR = {"laplace": 0, "mass": 1}
FP64_CONTRACTION = {"tensor_cores": 0, "fp64_pipe": 1}


class Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("amplitude", ctypes.c_double)]


class Geometry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("coefficient", ctypes.c_int32), ("user_data", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("graph_iterations", ctypes.c_int32), ("instrument", ctypes.c_int32),
                ("tile", ctypes.c_int32 * 3), ("precision", ctypes.c_int32), ("preconditioner", ctypes.c_int32),
                ("inner_rtol", ctypes.c_double), ("components", ctypes.c_int32), ("operator_kind", ctypes.c_int32),
                ("x_update_every_iteration", ctypes.c_int32), ("true_residual", ctypes.c_int32),
                ("fp64_contraction", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("status", ctypes.c_int32),
                ("main_kernel_launches", ctypes.c_int32), ("residual_sq_est", ctypes.c_double),
                ("rhs_norm_sq", ctypes.c_double), ("main_kernel_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("outer_cycles", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("true_residual_sq", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class MfcgError(RuntimeError):
    def __init__(self, call: str, status: int, text: str = ""):
        super().__init__(f"{call} failed: {STATUS.get(status, status)} ({text})")
        self.status = status


_lib = None


def declared_functions() -> list[str]:
    """Names of the functions declared in include/mfcg.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(mfcg_\w+)\s*\(", text, flags=re.M)))


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "mfcg_setup": [ctypes.POINTER(Mesh), i32, ctypes.POINTER(Geometry), ctypes.POINTER(Options), vp,
                       ctypes.POINTER(vp)],
        "mfcg_n_dofs": [vp, ctypes.POINTER(ctypes.c_int64)],
        "mfcg_apply_operator": [vp, vp, vp],
        "mfcg_diagonal": [vp, vp],
        "mfcg_rhs": [vp, vp],
        "mfcg_cg_solve": [vp, vp, vp, f64, i32, ctypes.POINTER(SolveInfo)],
        "mfcg_cg_solve_host": [vp, vp, vp, f64, i32, ctypes.POINTER(SolveInfo)],
        "mfcg_to_lexicographic": [vp, vp, vp],
        "mfcg_from_lexicographic": [vp, vp, vp],
        "mfcg_destroy": [vp],
        "mfcg_setup_batch": [i32, ctypes.POINTER(Mesh), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Geometry),
                             ctypes.POINTER(Options), vp, ctypes.POINTER(vp)],
        "mfcg_batch_member": [vp, i32, ctypes.POINTER(vp)],
        "mfcg_cg_solve_batch": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), f64, i32, ctypes.POINTER(SolveInfo)],
        "mfcg_destroy_batch": [vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.mfcg_status_string.argtypes = [ctypes.c_int]
    lib.mfcg_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(call: str, status: int, allowed=(OK,)) -> int:
    if status not in allowed:
        raise MfcgError(call, status, load().mfcg_status_string(status).decode())
    return status
