"""Python binding of libsdpgb with the same names as the C ABI.

Device vectors are torch CUDA tensors (float64); torch supplies device memory
and the CUDA stream only.  Every operation is one call into the library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

try:  # torch is optional for host-only use (loading, symbol checks)
    import torch
except Exception:  # pragma: no cover
    torch = None


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def default_params(**kw) -> L.sdp_params:
    lib = L.load()
    p = L.sdp_params()
    lib.sdp_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = L.PREC[v]
        setattr(p, k, v)
    return p


def _prec(p):
    return L.PREC[p] if isinstance(p, str) else int(p)


def _check_dev(t, m, name):
    if torch is None or not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != m:
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor with {m} entries")


class SDPProblem:
    """One SDP (eq. SDP) resident on the GPU: sdp_setup ... sdp_destroy."""

    def __init__(self, n, m, C_trip, A_trip, b, k, params: L.sdp_params | None = None, stream=None):
        self.lib = L.load()
        Ci, Cj, Cv = (_i32(C_trip[0]), _i32(C_trip[1]), _f64(C_trip[2]))
        Ak, Ai, Aj, Av = (_i32(A_trip[0]), _i32(A_trip[1]), _i32(A_trip[2]), _f64(A_trip[3]))
        b = _f64(b)
        if b.shape[0] != m:
            raise ValueError("b must have m entries")
        self.params = params if params is not None else default_params()
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = C.c_void_p()
        st = self.lib.sdp_setup(int(n), int(m), int(Ci.shape[0]), _ip(Ci), _ip(Cj), _dp(Cv), int(Ak.shape[0]),
                                _ip(Ak), _ip(Ai), _ip(Aj), _dp(Av), _dp(b), int(k), C.byref(self.params),
                                C.c_void_p(stream) if stream else None, C.byref(h))
        if st != L.SDP_OK:
            raise L.SDPError(st, f"sdp_setup failed: {self.lib.sdp_status_str(st).decode()}")
        self.h = h
        self.n, self.m, self.k = int(n), int(m), int(k)

    @classmethod
    def from_data(cls, d, params=None, stream=None):
        """From any object with n, m, Ci, Cj, Cv, Ak, Ai, Aj, Av, b, k attributes."""
        return cls(d.n, d.m, (d.Ci, d.Cj, d.Cv), (d.Ak, d.Ai, d.Aj, d.Av), d.b, d.k, params, stream)

    # -- plumbing ---------------------------------------------------------
    def _raise(self, st, what, ok=(L.SDP_OK,)):
        if st in ok:
            return st
        msg = self.lib.sdp_last_error(self.h).decode() if self.h else ""
        raise L.SDPError(st, f"{what}: {self.lib.sdp_status_str(st).decode()}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.sdp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the C-ABI calls ----------------------------------------------------
    def hessian_matvec(self, v, out=None, prec="fp64"):
        _check_dev(v, self.m, "v")
        if out is None:
            out = torch.empty_like(v)
        _check_dev(out, self.m, "out")
        self._raise(self.lib.sdp_hessian_matvec(self.h, C.c_void_p(v.data_ptr()), C.c_void_p(out.data_ptr()),
                                                _prec(prec)), "sdp_hessian_matvec")
        return out

    def precond_build(self):
        self._raise(self.lib.sdp_precond_build(self.h), "sdp_precond_build")

    def precond_apply(self, r, out=None, prec="fp64"):
        _check_dev(r, self.m, "r")
        if out is None:
            out = torch.empty_like(r)
        self._raise(self.lib.sdp_precond_apply(self.h, C.c_void_p(r.data_ptr()), C.c_void_p(out.data_ptr()),
                                               _prec(prec)), "sdp_precond_apply")
        return out

    def pcg_solve(self, r, rtol=1e-8, maxit=1000, prec="fp64", out=None):
        _check_dev(r, self.m, "r")
        if out is None:
            out = torch.empty_like(r)
        its = C.c_int(0)
        rel = C.c_double(0.0)
        st = self.lib.sdp_pcg_solve(self.h, C.c_void_p(r.data_ptr()), C.c_void_p(out.data_ptr()), float(rtol),
                                    int(maxit), _prec(prec), C.byref(its), C.byref(rel))
        self._raise(st, "sdp_pcg_solve", ok=(L.SDP_OK, L.SDP_ERR_MAXIT))
        return out, its.value, rel.value, st

    def ipm_step(self):
        info = L.sdp_ipm_info()
        self._raise(self.lib.sdp_ipm_step(self.h, C.byref(info)), "sdp_ipm_step")
        return {f: getattr(info, f) for f, _ in L.sdp_ipm_info._fields_}

    def solve(self, allow_maxit=False):
        res = L.sdp_result()
        ok = (L.SDP_OK, L.SDP_ERR_MAXIT) if allow_maxit else (L.SDP_OK,)
        st = self._raise(self.lib.sdp_solve(self.h, C.byref(res)), "sdp_solve", ok=ok)
        out = {f: getattr(res, f) for f, _ in L.sdp_result._fields_}
        out["status"] = st
        return out

    def set_W(self, W):
        _check_dev(W, self.n * self.n, "W")
        self._raise(self.lib.sdp_set_W(self.h, C.c_void_p(W.data_ptr())), "sdp_set_W")

    def get_W(self):
        W = torch.empty(self.n, self.n, dtype=torch.float64, device="cuda")
        self._raise(self.lib.sdp_get_W(self.h, C.c_void_p(W.data_ptr())), "sdp_get_W")
        return W

    def get_solution(self):
        X = np.empty((self.n, self.n))
        y = np.empty(self.m)
        S = np.empty((self.n, self.n))
        self._raise(self.lib.sdp_get_solution(self.h, C.c_void_p(X.ctypes.data), C.c_void_p(y.ctypes.data),
                                              C.c_void_p(S.ctypes.data)), "sdp_get_solution")
        return X, y, S

    def get_state(self):
        """Checkpoint of the iterate: (X, y, S, iteration counter) on the host."""
        X = np.empty((self.n, self.n))
        y = np.empty(self.m)
        S = np.empty((self.n, self.n))
        it = C.c_int(0)
        self._raise(self.lib.sdp_get_state(self.h, C.c_void_p(X.ctypes.data), C.c_void_p(y.ctypes.data),
                                           C.c_void_p(S.ctypes.data), C.byref(it)), "sdp_get_state")
        return X, y, S, it.value

    def set_state(self, X, y, S, it=0):
        X, y, S = _f64(X), _f64(y), _f64(S)
        self._raise(self.lib.sdp_set_state(self.h, C.c_void_p(X.ctypes.data), C.c_void_p(y.ctypes.data),
                                           C.c_void_p(S.ctypes.data), int(it)), "sdp_set_state")

    def precond_info(self):
        tau = C.c_double(0.0)
        k = C.c_int(0)
        self._raise(self.lib.sdp_precond_info(self.h, C.byref(tau), C.byref(k)), "sdp_precond_info")
        return tau.value, k.value

    def sizes(self):
        n, m, k = C.c_int(), C.c_int(), C.c_int()
        nnz = C.c_int64()
        self._raise(self.lib.sdp_sizes(self.h, C.byref(n), C.byref(m), C.byref(k), C.byref(nnz)), "sdp_sizes")
        return n.value, m.value, k.value, nnz.value

    def device_bytes(self):
        return int(self.lib.sdp_device_bytes(self.h))

    def launch_count(self):
        return int(self.lib.sdp_launch_count(self.h))

    def reset(self):
        self._raise(self.lib.sdp_reset(self.h), "sdp_reset")

    def timing_enable(self, cls):
        self._raise(self.lib.sdp_timing_enable(self.h, cls.encode() if cls else None), "sdp_timing_enable")

    def timing_report(self):
        """Per-class device time since timing_enable: {class: (ms, launches, flops, bytes)}."""
        buf = C.create_string_buffer(1 << 16)
        self.lib.sdp_timing_report(self.h, buf, len(buf))
        out = {}
        for line in buf.value.decode().splitlines():
            name, ms, cnt, fl, by = line.split()
            out[name] = (float(ms), int(cnt), float(fl), float(by))
        return out

    def timing_read(self):
        ms = C.c_double()
        n = C.c_int64()
        f = C.c_double()
        b = C.c_double()
        self._raise(self.lib.sdp_timing_read(self.h, C.byref(ms), C.byref(n), C.byref(f), C.byref(b)),
                    "sdp_timing_read")
        return dict(ms=ms.value, launches=n.value, flops=f.value, bytes=b.value)


def hessian_matvec_static(n, m, Ak, Ai, Aj, Av, W, v, out=None, stream=None):
    """sdp_hessian_matvec_static: handle-free FP64 Hessian matvec with static scratch.

    Ak, Ai, Aj: int32 CUDA tensors (triplets), Av: float64 CUDA tensor, W: (n, n)
    float64 CUDA tensor, v: float64 CUDA tensor of length m.  n <= SDP_STATIC_MAX_N.
    """
    lib = L.load()
    nnz = int(Ak.numel())
    for t, name in ((Ak, "Ak"), (Ai, "Ai"), (Aj, "Aj")):
        if not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous() or t.numel() != nnz:
            raise ValueError(f"{name} must be a contiguous int32 CUDA tensor with {nnz} entries")
    _check_dev(Av, nnz, "Av")
    _check_dev(W, n * n, "W")
    _check_dev(v, m, "v")
    if out is None:
        out = torch.empty_like(v)
    _check_dev(out, m, "out")
    if out.data_ptr() == v.data_ptr():
        raise ValueError("out must not be v: the output is cleared before v is read")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.sdp_hessian_matvec_static(int(n), int(m), nnz, C.c_void_p(Ak.data_ptr()), C.c_void_p(Ai.data_ptr()),
                                       C.c_void_p(Aj.data_ptr()), C.c_void_p(Av.data_ptr()),
                                       C.c_void_p(W.data_ptr()), C.c_void_p(v.data_ptr()),
                                       C.c_void_p(out.data_ptr()), C.c_void_p(stream) if stream else None)
    if st != L.SDP_OK:
        raise L.SDPError(st, f"sdp_hessian_matvec_static: {lib.sdp_status_str(st).decode()}: "
                             f"{lib.sdp_last_error(None).decode()}")
    return out


class SDPBatch:
    """sdp_batch_*: solve several SDPProblem objects in lockstep with batched PCG launches."""

    def __init__(self, problems=(), stream=None, groups=0):
        self.lib = L.load()
        self.problems = list(problems)
        arr = (C.c_void_p * max(1, len(self.problems)))(*[p.h.value for p in self.problems])
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        b = C.c_void_p()
        st = self.lib.sdp_batch_create(arr, len(self.problems), C.c_void_p(stream) if stream else None, C.byref(b))
        if st != L.SDP_OK:
            raise L.SDPError(st, f"sdp_batch_create: {self.lib.sdp_status_str(st).decode()}")
        self.b = b
        st = self.lib.sdp_batch_set_groups(self.b, int(groups))
        if st != L.SDP_OK:
            raise L.SDPError(st, f"sdp_batch_set_groups: {self.lib.sdp_status_str(st).decode()}")

    def solve(self, allow_maxit=False):
        res = (L.sdp_result * len(self.problems))()
        st = self.lib.sdp_batch_solve(self.b, res)
        ok = (L.SDP_OK, L.SDP_ERR_MAXIT) if allow_maxit else (L.SDP_OK,)
        if st not in ok:
            raise L.SDPError(st, f"sdp_batch_solve: {self.lib.sdp_status_str(st).decode()}: "
                                 f"{self.lib.sdp_batch_last_error(self.b).decode()}")
        return [{f: getattr(r, f) for f, _ in L.sdp_result._fields_} for r in res]

    # -- continuous batching: members join and leave between IPM iterations --
    def add(self, prob):
        st = self.lib.sdp_batch_add(self.b, prob.h)
        if st != L.SDP_OK:
            raise L.SDPError(st, f"sdp_batch_add: {self.lib.sdp_status_str(st).decode()}: "
                                 f"{self.lib.sdp_batch_last_error(self.b).decode()}")
        self.problems.append(prob)

    def remove(self, prob):
        st = self.lib.sdp_batch_remove(self.b, prob.h)
        if st != L.SDP_OK:
            raise L.SDPError(st, "sdp_batch_remove")
        self.problems = [p for p in self.problems if p is not prob]

    def step(self):
        """One lockstep IPM iteration of every running member; returns how many still run."""
        run = C.c_int(0)
        st = self.lib.sdp_batch_step(self.b, C.byref(run))
        if st != L.SDP_OK:
            raise L.SDPError(st, f"sdp_batch_step: {self.lib.sdp_status_str(st).decode()}: "
                                 f"{self.lib.sdp_batch_last_error(self.b).decode()}")
        return run.value

    def tuning(self):
        """(chosen SpMM rows per CTA, {R: ms per launch}) of the batch's autotuner."""
        r = C.c_int(0)
        ms = (C.c_double * 4)()
        self.lib.sdp_batch_tuning(self.b, C.byref(r), ms)
        return r.value, {R: ms[i] for i, R in enumerate((1, 2, 4, 8)) if ms[i] > 0}

    MEMBER_STATES = ("running", "converged", "iteration_limit", "failed")

    def member(self, prob):
        """(result dict, state name, status) of a member."""
        r = L.sdp_result()
        state = C.c_int(0)
        st = self.lib.sdp_batch_member(self.b, prob.h, C.byref(r), C.byref(state))
        res = {f: getattr(r, f) for f, _ in L.sdp_result._fields_}
        return res, self.MEMBER_STATES[state.value], st

    STAGES = ("nt_precond", "pcg_pred", "step_pred", "pcg_corr", "step_update", "pcg_graph",
              "graph_launches", "batched_iters")

    def stage_seconds(self):
        """Wall seconds of the last solve per stage, then graph seconds, graph launches and
        batched PCG iterations (sdp_batch_stage_seconds)."""
        out = (C.c_double * 8)()
        self.lib.sdp_batch_stage_seconds(self.b, out)
        return dict(zip(self.STAGES, list(out)))

    def close(self):
        if getattr(self, "b", None):
            self.lib.sdp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
