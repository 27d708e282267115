"""Host-side checks of the C ABI (no GPU): the library loads, exports every
call that include/sdpgb.h declares, and rejects bad input before touching the
device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1703_10973_gb300 import _build, _lib
    if not os.path.exists(_build.LIB):
        _build.build()
    return _lib.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "sdpgb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sdp_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_paper_calls():
    names = _declared()
    for call in ["sdp_setup", "sdp_ipm_step", "sdp_hessian_matvec", "sdp_precond_build",
                 "sdp_precond_apply", "sdp_pcg_solve", "sdp_solve"]:
        assert call in names


def test_library_exports_every_declared_symbol():
    lib = _lib()
    from paper_1703_10973_gb300 import _lib as L
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in L.SIGNATURES, f"binding lacks {name}"


def test_default_params():
    from paper_1703_10973_gb300 import default_params
    p = default_params()
    assert p.gap_tol == 1e-6 and p.pcg_rtol == 1e-8 and p.step_frac == 0.9 and p.precond == 2   # Hhat of Section V


def _setup(n, m, C_trip, A_trip, b, k=1):
    lib = _lib()
    from paper_1703_10973_gb300 import _lib as L
    Ci, Cj, Cv = [np.ascontiguousarray(x) for x in C_trip]
    Ak, Ai, Aj, Av = [np.ascontiguousarray(x) for x in A_trip]
    b = np.ascontiguousarray(b, dtype=np.float64)
    h = C.c_void_p()
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    st = lib.sdp_setup(n, m, len(Ci), ip(Ci), ip(Cj), dp(Cv), len(Ak), ip(Ak), ip(Ai), ip(Aj), dp(Av), dp(b), k,
                       None, None, C.byref(h))
    if h.value:
        lib.sdp_destroy(h)
    return st, L


def _i(*a):
    return np.array(a, dtype=np.int32)


def _d(*a):
    return np.array(a, dtype=np.float64)


def test_setup_rejects_bad_sizes():
    st, L = _setup(0, 1, (_i(), _i(), _d()), (_i(0), _i(0), _i(0), _d(1.0)), _d(1.0))
    assert st == L.SDP_ERR_ARG


def test_setup_rejects_out_of_range_index():
    st, L = _setup(3, 1, (_i(0), _i(0), _d(1.0)), (_i(0), _i(0), _i(5), _d(1.0)), _d(1.0))
    assert st == L.SDP_ERR_ARG


def test_setup_rejects_empty_constraint():
    st, L = _setup(3, 2, (_i(0), _i(0), _d(1.0)), (_i(0), _i(0), _i(1), _d(1.0)), _d(1.0, 2.0))
    assert st == L.SDP_ERR_ARG


def test_setup_rejects_non_diagonal_AtA():
    """X_00 + X_11 = 1 and X_00 = 0.5 share a position: A_1 . A_2 = 1 != 0."""
    st, L = _setup(2, 2, (_i(0, 1), _i(0, 1), _d(1.0, 1.0)),
                   (_i(0, 0, 1), _i(0, 1, 0), _i(0, 1, 0), _d(1.0, 1.0, 1.0)), _d(1.0, 0.5))
    assert st == L.SDP_ERR_UNSUPPORTED


def test_status_strings():
    lib = _lib()
    for s in range(9):
        assert lib.sdp_status_str(s)
