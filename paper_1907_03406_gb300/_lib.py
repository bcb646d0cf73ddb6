"""ctypes declarations of the C ABI in include/sgf.h (marshalling only).

The shared library is built in-tree by `paper_1907_03406_gb300.build`.  There
is no CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsgf.so")


class sgf_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("dof", C.c_int), ("dirichlet", C.c_uint)]


class sgf_tuning(C.Structure):
    _fields_ = [("gemv_min_elems", C.c_int), ("gemv_max_elems", C.c_int), ("front_small", C.c_int),
                ("tensor_cores", C.c_int), ("gemv_cols", C.c_int), ("tc_min_dim", C.c_int)]


class sgf_opts(C.Structure):
    _fields_ = [("scheme", C.c_int), ("leaf", C.c_int), ("degree", C.c_int), ("basis", C.c_int),
                ("precision", C.c_int), ("tau", C.c_double), ("compress_from_level", C.c_int),
                ("nu", C.c_double)]


class sgf_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("seconds", C.c_double)]


_P = C.c_void_p
_I = C.c_int
_IP = C.POINTER(C.c_int)
_I64P = C.POINTER(C.c_int64)
_SZP = C.POINTER(C.c_size_t)

# name -> (restype, argtypes); every function declared in include/sgf.h
SIGNATURES = {
    "sgf_analyze": (_I, [C.POINTER(sgf_grid), _I, C.POINTER(sgf_opts), C.POINTER(_P)]),
    "sgf_plan_destroy": (None, [_P]),
    "sgf_plan_info": (_I, [_P, _IP, _I64P]),
    "sgf_plan_export_level": (_I, [_P, _I, _IP, _IP, _IP, _IP, _IP, _IP, _IP, _IP, _IP]),
    "sgf_plan_footprint": (_I, [_P, _SZP, _SZP]),
    "sgf_plan_get_tuning": (_I, [_P, C.POINTER(sgf_tuning)]),
    "sgf_factor_precision": (_I, [_P]),
    "sgf_plan_set_tuning": (_I, [_P, C.POINTER(sgf_tuning)]),
    "sgf_autotune": (_I, [_P, _P, _P, _I, C.POINTER(sgf_tuning), C.POINTER(C.c_double)]),
    "sgf_factor": (_I, [_P, _P, _P, C.POINTER(_P)]),
    "sgf_factor_destroy": (None, [_P]),
    "sgf_factor_level_stats": (_I, [_P, _I, _IP, _I64P, _I64P, _I64P]),
    "sgf_factor_ranks": (_I, [_P, _I, _IP, _IP]),
    "sgf_factor_status": (_I, [_P, _IP, _IP]),
    "sgf_apply": (_I, [_P, _P, _P, _I, _P]),
    "sgf_apply_forward": (_I, [_P, _P, _P, _I, _P]),
    "sgf_spmv": (_I, [_P, _P, _P, _I, _P]),
    "sgf_pcg_solve": (_I, [_P, _P, _P, _I, C.c_double, _I, _P, C.POINTER(sgf_solve_info)]),
    "sgf_solve_host": (_I, [_P, _P, _P, _P, _I, C.c_double, _I, _P, C.POINTER(sgf_solve_info)]),
    "sgf_pcg_solve_noalloc": (_I, [_P, _P, _P, C.c_double, _I, _P, C.POINTER(sgf_solve_info)]),
    "sgf_status_string": (C.c_char_p, [_I]),
    "sgf_last_error": (C.c_char_p, []),
    "sgf_dry_run_violations": (C.c_int64, [_I]),
    "sgf_dry_run_report": (C.c_char_p, []),
    "sgf_profile_reset": (None, [_I]),
    "sgf_profile_read": (_I, [_I, _I64P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sgf_profile_kind_name": (C.c_char_p, [_I]),
    "sgf_release_cached_memory": (_I, []),
    "sgf_sync": (_I, [_P]),
    "sgf_memory_stats": (_I, [_I64P, _I64P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the library once and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"SGF CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
