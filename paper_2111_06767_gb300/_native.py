"""ctypes binding of libdg_elliptic.so: the C ABI declared in include/dg_elliptic.h, one Python
name per C entry point, argument marshalling only. All compute runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# DG_DEBUG_BUILD=1 loads the bounds-checked build (paper_2111_06767_gb300/build.py --debug) instead
LIB_PATH = os.path.join(_HERE, "libdg_elliptic_debug.so" if os.environ.get("DG_DEBUG_BUILD") == "1"
                        else "libdg_elliptic.so")

DG_OK, DG_PENDING = 0, 1
DG_ERR_CANCELLED = -9
STATUS_NAMES = {0: "DG_OK", 1: "DG_PENDING", -1: "DG_ERR_INVALID_ARG", -2: "DG_ERR_OOM", -3: "DG_ERR_CUDA",
                -4: "DG_ERR_NOT_CONVERGED", -5: "DG_ERR_BREAKDOWN", -6: "DG_ERR_TIMEOUT", -7: "DG_ERR_BUSY",
                -8: "DG_ERR_NOT_FOUND", -9: "DG_ERR_CANCELLED"}
DG_MAX_N, DG_MAX_LEVELS, DG_MAX_PUNCTURES = 10, 8, 4
PRECISION_FP64, PRECISION_MIXED = 0, 1
PROBLEM_POISSON, PROBLEM_PUNCTURE = 0, 1


class dg_puncture(C.Structure):
    _fields_ = [("position", C.c_double * 3), ("mass", C.c_double), ("momentum", C.c_double * 3)]


class dg_domain_desc(C.Structure):
    _fields_ = [("lower", C.c_double * 3), ("upper", C.c_double * 3), ("n", C.c_int32 * 3), ("N", C.c_int32),
                ("penalty", C.c_double), ("precision", C.c_int32), ("mg_levels", C.c_int32),
                ("overlap", C.c_int32), ("presmooth", C.c_int32), ("postsmooth", C.c_int32),
                ("problem", C.c_int32), ("n_punctures", C.c_int32), ("punctures", dg_puncture * DG_MAX_PUNCTURES),
                ("subdomain_gemm", C.c_int32), ("neumann_faces", C.c_int32),
                ("node_xyz", C.POINTER(C.c_double)), ("coef", C.POINTER(C.c_double))]


class dg_layout(C.Structure):
    _fields_ = [("n_dof", C.c_int64), ("n_elements", C.c_int32), ("N", C.c_int32), ("n", C.c_int32 * 3),
                ("mg_levels", C.c_int32), ("level_n", (C.c_int32 * 3) * DG_MAX_LEVELS),
                ("n_classes", C.c_int32 * DG_MAX_LEVELS), ("subdomain_size", C.c_int32),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("device_bytes", C.c_size_t)]


class dg_solve_opts(C.Structure):
    _fields_ = [("max_iterations", C.c_int32), ("precondition", C.c_int32), ("linear_tol", C.c_double),
                ("max_newton_steps", C.c_int32), ("subdomain_iterations", C.c_int32), ("relative_to_b", C.c_int32),
                ("krylov", C.c_int32), ("subdomain_solver", C.c_int32)]


class dg_solve_report(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("newton_steps", C.c_int32),
                ("line_search_steps", C.c_int32), ("initial_residual", C.c_double),
                ("final_residual", C.c_double), ("relative_residual", C.c_double), ("seconds", C.c_double)]


PHASES = ("apply_fp64", "apply_fp32", "gather", "subdomain_gemm", "scatter", "transfer", "krylov", "coarse_smooth",
          "subdomain_build")


class dg_phase_stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("milliseconds", C.c_double), ("bytes", C.c_double), ("flops", C.c_double)]


class dg_serve_desc(C.Structure):
    _fields_ = [("memory_budget_bytes", C.c_size_t), ("max_active", C.c_int32), ("queue_capacity", C.c_int32),
                ("n_streams", C.c_int32)]


class dg_request(C.Structure):
    _fields_ = [("domain", dg_domain_desc), ("f_host", C.POINTER(C.c_double)), ("tol", C.c_double),
                ("opts", dg_solve_opts)]


class dg_result(C.Structure):
    _fields_ = [("report", dg_solve_report), ("u_host", C.POINTER(C.c_double)), ("n_dof", C.c_int64),
                ("submit_time", C.c_double), ("admit_time", C.c_double), ("finish_time", C.c_double)]


_vp = C.c_void_p
_i32 = C.c_int32
# name -> (restype, argtypes), exactly the functions of include/dg_elliptic.h
SIGNATURES = {
    "dg_domain_create": (C.c_int, [C.POINTER(dg_domain_desc), _vp, C.POINTER(_vp)]),
    "dg_domain_destroy": (None, [_vp]),
    "dg_domain_layout": (C.c_int, [_vp, C.POINTER(dg_layout)]),
    "dg_last_error": (C.c_char_p, [_vp]),
    "dg_apply": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dg_apply_f32": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "dg_apply_level": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "dg_rhs": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dg_mg_restrict": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "dg_mg_prolongate_add": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "dg_schwarz_smooth": (C.c_int, [_vp, _i32, _vp, _vp, _i32, _vp]),
    "dg_vcycle": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dg_dot": (C.c_int, [_vp, _i32, _vp, C.c_int64, _vp, _vp, _vp]),
    "dg_dot_noalloc": (C.c_int, [C.c_int64, _i32, _vp, C.c_int64, _vp, _vp, _vp]),
    "dg_debug_bounds_check": (_i32, []),
    "dg_nonlinear_residual": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "dg_set_linearization": (C.c_int, [_vp, _vp, _vp]),
    "dg_set_subdomain_solver": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp]),
    "dg_puncture_fields": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dg_copy_coordinates": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "dg_layout_coordinates_host": (C.c_int, [C.POINTER(dg_domain_desc), C.POINTER(C.c_double),
                                             C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "elliptic_solve": (C.c_int, [_vp, _vp, _vp, C.c_double, C.POINTER(dg_solve_opts), C.POINTER(dg_solve_report)]),
    "elliptic_solve_host": (C.c_int, [_vp, _vp, _vp, C.c_double, C.POINTER(dg_solve_opts),
                                      C.POINTER(dg_solve_report)]),
    "elliptic_batch_create": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), _i32, C.c_double,
                                        C.POINTER(dg_solve_opts), C.POINTER(_vp)]),
    "elliptic_batch_run": (C.c_int, [_vp, _vp, C.POINTER(dg_solve_report)]),
    "elliptic_batch_destroy": (None, [_vp]),
    "dg_kernel_launches": (C.c_int64, []),
    "dg_profile_enable": (C.c_int, [_vp, _i32]),
    "dg_profile_read": (C.c_int, [_vp, C.POINTER(dg_phase_stats)]),
    "elliptic_serve_create": (C.c_int, [C.POINTER(dg_serve_desc), C.POINTER(_vp)]),
    "elliptic_serve_submit": (C.c_int, [_vp, C.POINTER(dg_request), C.POINTER(C.c_uint64)]),
    "elliptic_serve_poll": (C.c_int, [_vp, C.c_uint64, C.POINTER(dg_result)]),
    "elliptic_serve_cancel": (C.c_int, [_vp, C.c_uint64]),
    "elliptic_serve_clock": (C.c_double, [_vp]),
    "elliptic_serve_destroy": (None, [_vp]),
}

_lib = None


class NativeError(RuntimeError):
    def __init__(self, status, message=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


def load(path: str = LIB_PATH):
    """Load the CUDA library; raise if it is missing (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python paper_2111_06767_gb300/build.py`"
                          + (" --debug" if path.endswith("_debug.so") else ""))
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status, handle=None):
    if status not in (DG_OK,):
        msg = load().dg_last_error(handle)
        raise NativeError(status, msg.decode() if msg else "")
    return status
