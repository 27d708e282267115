"""ctypes declarations of the libsdpgb C ABI (include/sdpgb.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from ._build import LIB

SDP_OK, SDP_ERR_ARG, SDP_ERR_OOM, SDP_ERR_NOT_PD, SDP_ERR_MAXIT = 0, 1, 2, 3, 4
SDP_ERR_UNSUPPORTED, SDP_ERR_NUMERIC, SDP_ERR_TIMEOUT, SDP_ERR_CUDA = 5, 6, 7, 8
SDP_FP64, SDP_FP32, SDP_BF16 = 0, 1, 2
SDP_STATIC_MAX_N = 512
SDP_K_MAX = 64
SDP_PRECOND_DIAG, SDP_PRECOND_WOODBURY, SDP_PRECOND_HAT = 0, 1, 2

PREC = {"fp64": SDP_FP64, "fp32": SDP_FP32, "bf16": SDP_BF16}


class sdp_params(C.Structure):
    _fields_ = [
        ("gap_tol", C.c_double),
        ("infeas_tol", C.c_double),
        ("pcg_rtol", C.c_double),
        ("ipm_maxit", C.c_int),
        ("pcg_maxit", C.c_int),
        ("refine_maxit", C.c_int),
        ("k", C.c_int),
        ("step_frac", C.c_double),
        ("prec", C.c_int),
        ("precond", C.c_int),
        ("inner_rtol", C.c_double),
        ("verbose", C.c_int),
        ("pcg_graph", C.c_int),
        ("inner_rtol_lp", C.c_double),
        ("wait_cycles", C.c_longlong),
        ("k_max", C.c_int),
        ("eta", C.c_double),
    ]


class sdp_ipm_info(C.Structure):
    _fields_ = [
        ("iter", C.c_int),
        ("mu", C.c_double),
        ("obj_p", C.c_double),
        ("obj_d", C.c_double),
        ("relgap", C.c_double),
        ("pinf", C.c_double),
        ("dinf", C.c_double),
        ("alpha_p", C.c_double),
        ("alpha_d", C.c_double),
        ("sigma", C.c_double),
        ("tau", C.c_double),
        ("pcg_iters_pred", C.c_int),
        ("pcg_iters_corr", C.c_int),
        ("pcg_relres_pred", C.c_double),
        ("pcg_relres_corr", C.c_double),
        ("converged", C.c_int),
        ("nt_fallback", C.c_int),
        ("k_split", C.c_int),
    ]


class sdp_result(C.Structure):
    _fields_ = [
        ("obj_p", C.c_double),
        ("obj_d", C.c_double),
        ("relgap", C.c_double),
        ("pinf", C.c_double),
        ("dinf", C.c_double),
        ("iters", C.c_int),
        ("pcg_iters_total", C.c_int),
        ("converged", C.c_int),
        ("seconds", C.c_double),
    ]


_P = C.c_void_p
_I32P = C.POINTER(C.c_int32)
_DP = C.POINTER(C.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "sdp_default_params": (None, [C.POINTER(sdp_params)]),
    "sdp_setup": (C.c_int, [C.c_int, C.c_int, C.c_int64, _I32P, _I32P, _DP, C.c_int64, _I32P, _I32P, _I32P,
                            _DP, _DP, C.c_int, C.POINTER(sdp_params), _P, C.POINTER(_P)]),
    "sdp_hessian_matvec": (C.c_int, [_P, _P, _P, C.c_int]),
    "sdp_precond_build": (C.c_int, [_P]),
    "sdp_precond_apply": (C.c_int, [_P, _P, _P, C.c_int]),
    "sdp_pcg_solve": (C.c_int, [_P, _P, _P, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int), _DP]),
    "sdp_ipm_step": (C.c_int, [_P, C.POINTER(sdp_ipm_info)]),
    "sdp_solve": (C.c_int, [_P, C.POINTER(sdp_result)]),
    "sdp_set_W": (C.c_int, [_P, _P]),
    "sdp_get_W": (C.c_int, [_P, _P]),
    "sdp_get_solution": (C.c_int, [_P, _P, _P, _P]),
    "sdp_set_state": (C.c_int, [_P, _P, _P, _P, C.c_int]),
    "sdp_get_state": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_int)]),
    "sdp_precond_info": (C.c_int, [_P, _DP, C.POINTER(C.c_int)]),
    "sdp_sizes": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "sdp_launch_count": (C.c_int64, [_P]),
    "sdp_device_bytes": (C.c_int64, [_P]),
    "sdp_reset": (C.c_int, [_P]),
    "sdp_timing_enable": (C.c_int, [_P, C.c_char_p]),
    "sdp_timing_read": (C.c_int, [_P, _DP, C.POINTER(C.c_int64), _DP, _DP]),
    "sdp_timing_report": (C.c_int64, [_P, C.c_char_p, C.c_int64]),
    "sdp_hessian_matvec_static": (C.c_int, [C.c_int, C.c_int, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sdp_batch_create": (C.c_int, [C.POINTER(_P), C.c_int, _P, C.POINTER(_P)]),
    "sdp_batch_solve": (C.c_int, [_P, C.POINTER(sdp_result)]),
    "sdp_batch_last_error": (C.c_char_p, [_P]),
    "sdp_batch_destroy": (None, [_P]),
    "sdp_batch_stage_seconds": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "sdp_batch_set_groups": (C.c_int, [_P, C.c_int]),
    "sdp_batch_tuning": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "sdp_batch_add": (C.c_int, [_P, _P]),
    "sdp_batch_step": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "sdp_batch_member": (C.c_int, [_P, _P, C.POINTER(sdp_result), C.POINTER(C.c_int)]),
    "sdp_batch_remove": (C.c_int, [_P, _P]),
    "sdp_mixed_gemm_work_bytes": (C.c_int64, [C.c_int, C.c_int, C.c_int]),
    "sdp_mixed_gemm": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _P, C.c_int, C.c_int, _P, C.c_int, C.c_int,
                                 _P, C.c_int, _P, C.c_int64, _P, _P]),
    "sdp_destroy": (None, [_P]),
    "sdp_status_str": (C.c_char_p, [C.c_int]),
    "sdp_last_error": (C.c_char_p, [_P]),
}

_lib = None


def load(path: str | None = None):
    """Load libsdpgb.so and declare every exported call; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"libsdpgb not built ({path} missing); run __graft_entry__.build() or "
            "python -m paper_1703_10973_gb300._build")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SDPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status
