"""ctypes declarations of the C ABI in include/hpse.h (argument marshalling only).

Loading fails loudly when libhpse.so has not been built: there is no CPU
fallback for any entry point.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhpse.so")

HPSE_MAX_W = 10
HPSE_OK = 0
STATUS_NAMES = {
    0: "HPSE_OK", 1: "HPSE_ERR_INVALID_ARG", 2: "HPSE_ERR_NONMATCHING_FACE", 3: "HPSE_ERR_DEGREE",
    4: "HPSE_ERR_BREAKDOWN", 5: "HPSE_ERR_NO_CONVERGENCE", 6: "HPSE_ERR_TIMEOUT", 7: "HPSE_ERR_CUDA",
    8: "HPSE_ERR_OOM", 9: "HPSE_ERR_NO_DATA", 10: "HPSE_ERR_CAPACITY",
}
FP64, FP32 = 0, 1
COEF_LAPLACE, COEF_SCALAR, COEF_GENERAL = 0, 1, 2
PRECOND_SEPARABLE, PRECOND_BLOCK = 0, 1
COORD_CARTESIAN, COORD_EDGE, COORD_VERTEX, COORD_VERTEX_EDGE, COORD_CURVED = 0, 1, 2, 3, 4


class MeshDesc(C.Structure):
    _fields_ = [
        ("n_elem", C.c_int32), ("n_problem", C.c_int32), ("n_rhs", C.c_int32), ("coef_kind", C.c_int32),
        ("elem_W", C.c_void_p), ("elem_problem", C.c_void_p), ("elem_lo", C.c_void_p),
        ("elem_hi", C.c_void_p), ("elem_nbr", C.c_void_p),
        ("coord", C.c_int32), ("n_corner", C.c_int32), ("corner_W", C.c_void_p), ("corner_problem", C.c_void_p),
        ("face_bc", C.c_void_p), ("robin_gamma", C.c_void_p),
    ]


class Data(C.Structure):
    _fields_ = [("f", C.c_void_p), ("a", C.c_void_p), ("grad_a", C.c_void_p), ("g", C.c_void_p),
                ("op", C.c_void_p)]


class SolveOpts(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("max_iter", C.c_int32), ("prec", C.c_int32), ("inner_tol", C.c_double),
        ("max_sweeps", C.c_int32), ("check_every", C.c_int32), ("zero_init", C.c_int32),
        ("time_limit_s", C.c_double), ("refine_mode", C.c_int32),
    ]


class SolveReport(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iterations", C.c_int32), ("sweeps", C.c_int32), ("applies", C.c_int32),
        ("rel_residual", C.c_double),
    ]


# name -> (restype, argtypes); every symbol declared in include/hpse.h
SIGNATURES = {
    "hpse_setup_mesh": (C.c_int, [C.POINTER(MeshDesc), C.c_int, C.POINTER(C.c_void_p)]),
    "hpse_ndof": (C.c_int64, [C.c_void_p]),
    "hpse_nquad": (C.c_int64, [C.c_void_p]),
    "hpse_nface_points": (C.c_int64, [C.c_void_p]),
    "hpse_nrhs": (C.c_int32, [C.c_void_p]),
    "hpse_query_points": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_curved_n_face_points": (C.c_int64, [C.c_void_p]),
    "hpse_curved_points": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_set_geometry": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_n_boundary_faces": (C.c_int64, [C.c_void_p]),
    "hpse_set_data": (C.c_int, [C.c_void_p, C.POINTER(Data), C.c_void_p]),
    "hpse_apply_operator": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_apply_preconditioner": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_setup_block_preconditioner": (C.c_int, [C.c_void_p]),
    "hpse_select_preconditioner": (C.c_int, [C.c_void_p, C.c_int32]),
    "hpse_block_tile": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_set_block_tile": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "hpse_get_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_pcg_solve": (C.c_int, [C.c_void_p, C.POINTER(SolveOpts), C.c_void_p, C.POINTER(SolveReport),
                                 C.c_void_p]),
    "hpse_h1_error": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p]),
    "hpse_h1_error_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    "hpse_conforming_correction": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_apply_residual": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_apply_transpose": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_apply_transpose_ibp": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_apply_fields_transpose": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_data_gradient_bilinear": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_data_gradient_vjp": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_eval_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_apply_eval_transpose": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_quad_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_set_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_data_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_work_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hpse_set_block_threads": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "hpse_get_block_threads": (C.c_int32, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "hpse_kernel_launch_count": (C.c_int64, [C.c_int32]),
    "hpse_partition": (C.c_int, [C.POINTER(MeshDesc), C.c_int32, C.c_void_p]),
    "hpse_pack_blocks": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_int64,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_unpack_blocks": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_int64,
                                     C.c_void_p, C.c_void_p, C.c_void_p]),
    "hpse_status_string": (C.c_char_p, [C.c_int]),
    "hpse_destroy": (None, [C.c_void_p]),
}

_lib = None


def load():
    """Load libhpse.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libhpse.so is not built (expected at %s); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HpseError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        lib = load()
        msg = lib.hpse_status_string(self.status).decode()
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES.get(self.status, self.status), msg))


def check(status, where=""):
    if status != HPSE_OK:
        raise HpseError(status, where)
