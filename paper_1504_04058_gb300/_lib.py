"""ctypes binding of libasp.so (include/asp.h), argument marshalling only.

Every compute step runs in the library's CUDA kernels; this module converts
torch tensors to device pointers and the current CUDA stream to a handle.  It
raises if the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libasp.so")

ASP_OK = 0
ASP_ERR_INVALID = -1
ASP_ERR_OOM = -2
ASP_ERR_CUDA = -3
ASP_ERR_SMALL_PIVOT = -4
ASP_ERR_NOT_CONVERGED = -5
ASP_ERR_TIMEOUT = -6
ASP_ERR_STATE = -7
ASP_ERR_UNSUPPORTED = -8

ASP_PREC_C128 = 0
ASP_PREC_C64 = 1
ASP_PREC_C64_SYM = 2
ASP_SLAB_BLOCK = 0
ASP_SLAB_ND = 1

KIND_M, KIND_R, KIND_L = 0, 1, 2

# every symbol include/asp.h declares
EXPORTS = [
    "asp_setup", "asp_footprint_bytes", "asp_num_layers", "asp_layer_range", "asp_factor",
    "asp_apply_preconditioner", "asp_matvec", "asp_subproblem_width", "asp_subproblem_solve",
    "asp_gmres_solve", "asp_take_launch_count", "asp_set_phase_timing", "asp_phase_times",
    "asp_destroy", "asp_error_string", "asp_last_error_detail", "asp_residual_norms_noalloc",
    "asp_selftest_bounded_wait", "asp_setup_layers", "asp_footprint_bytes_layers", "asp_layer_widths_from_velocity",
    "asp_autotune", "asp_set_solve_shape", "asp_nd_plan_check", "asp_testhook_fail_device_alloc",
]
NOALLOC_MAX_N = 4096
NOALLOC_MAX_RHS = 64
PHASES = ["factor", "tmap", "embed", "chain", "fill", "elementwise", "matvec", "krylov", "schur3d", "tdiag"]


class asp_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("pml", ctypes.c_int),
        ("pml_aux", ctypes.c_int),
        ("b", ctypes.c_int),
        ("C", ctypes.c_double),
        ("factor_prec", ctypes.c_int),
        ("max_rhs", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("slab_solver", ctypes.c_int),
    ]


class asp_solve_info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("rel_res_est", ctypes.c_double),
        ("rel_res_true", ctypes.c_double),
    ]


class AspError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (code {code})")
        self.code = code


_lib = None


def load() -> ctypes.CDLL:
    """Load libasp.so (built by ``paper_1504_04058_gb300.build``).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    sig = {
        "asp_setup": (I, [ctypes.POINTER(asp_params), P, I, ctypes.POINTER(P)]),
        "asp_footprint_bytes": (ctypes.c_size_t, [ctypes.POINTER(asp_params)]),
        "asp_setup_layers": (I, [ctypes.POINTER(asp_params), P, I, P, I, ctypes.POINTER(P)]),
        "asp_footprint_bytes_layers": (ctypes.c_size_t, [ctypes.POINTER(asp_params), P, I]),
        "asp_layer_widths_from_velocity": (I, [ctypes.POINTER(asp_params), P, I, I, P, I]),
        "asp_num_layers": (I, [P]),
        "asp_layer_range": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "asp_factor": (I, [P, P]),
        "asp_apply_preconditioner": (I, [P, P, P, I, P]),
        "asp_matvec": (I, [P, P, P, I, P]),
        "asp_subproblem_width": (I, [P, I, I]),
        "asp_subproblem_solve": (I, [P, I, I, P, P, I, P]),
        "asp_gmres_solve": (I, [P, P, P, I, D, I, I, ctypes.POINTER(asp_solve_info), P]),
        "asp_take_launch_count": (ctypes.c_longlong, [P]),
        "asp_autotune": (I, [P, I, P, P, P]),
        "asp_set_solve_shape": (I, [P, I, I, I, I]),
        "asp_nd_plan_check": (I, [I, I, P, I]),
        "asp_testhook_fail_device_alloc": (I, [I]),
        "asp_set_phase_timing": (I, [P, I]),
        "asp_phase_times": (I, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong), I]),
        "asp_destroy": (V, [P]),
        "asp_residual_norms_noalloc": (I, [ctypes.POINTER(asp_params), P, P, P, I, P, P]),
        "asp_selftest_bounded_wait": (I, [I, P]),
        "asp_error_string": (ctypes.c_char_p, [I]),
        "asp_last_error_detail": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int, where: str) -> int:
    if code != ASP_OK:
        lib = load()
        raise AspError(code, where, f"{lib.asp_error_string(code).decode()}: "
                                    f"{lib.asp_last_error_detail().decode()}")
    return code
