"""sdp_hessian_matvec_static (static scratch, no allocation) against
sdp_hessian_matvec on the same W and v.

Collected last (file name) so that it also runs after every other GPU test has
used the library in the same process; it passes alone as well.  Two calls in a
row with different v check that the scratch is cleared between calls.
"""
import numpy as np
import pytest

import sdp_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10973_gb300 import _build, load
    _build.build()
    load()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * rng.uniform(0.1, 10.0, n)) @ Q.T


@pytest.mark.parametrize("make", [lambda: si.mc_instance(37, 61, 2, 900, 5),
                                  lambda: si.random_general(23, 40, 3, 2),
                                  lambda: si.unit_diag_instance(9)],
                         ids=["mc_ragged", "general", "unit_diag"])
def test_static_matches_handle_matvec_two_calls(make):
    from paper_1703_10973_gb300 import SDPProblem, hessian_matvec_static
    d = make()
    W = torch.from_numpy(_spd(d.n, 11)).cuda()
    trip = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).cuda() for x in (d.Ak, d.Ai, d.Aj)]
    Av = torch.from_numpy(np.ascontiguousarray(d.Av, dtype=np.float64)).cuda()
    vs = [torch.from_numpy(si.random_vec(d.m, s)).cuda() for s in (1, 2)]
    with SDPProblem.from_data(d) as prob:
        prob.set_W(W.reshape(-1).contiguous())
        ref = [prob.hessian_matvec(v).cpu().numpy() for v in vs]
    out = torch.full((d.m,), float("nan"), dtype=torch.float64, device="cuda")
    for v, r in zip(vs, ref):   # two calls in a row reuse the same scratch and output
        got = hessian_matvec_static(d.n, d.m, *trip, Av, W.reshape(-1).contiguous(), v, out=out)
        torch.cuda.synchronize()
        assert _rel(got.cpu().numpy(), r) <= 1e-12


def test_static_rejects_oversize_n():
    from paper_1703_10973_gb300 import _lib as L
    from paper_1703_10973_gb300 import hessian_matvec_static
    n = L.SDP_STATIC_MAX_N + 1
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    W = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.SDPError, match="SDP_STATIC_MAX_N"):
        hessian_matvec_static(n, 1, z, z, z, v, W, v)


def test_static_at_max_n_matches_handle_and_oracle():
    """n = SDP_STATIC_MAX_N fills the whole static scratch; the result agrees with
    the handle matvec and with the oracle's explicit H (closed form of eq. hesseqn2
    for one symmetric pair per constraint) times v."""
    from oracle import sdp_oracle as o
    from paper_1703_10973_gb300 import _lib as L
    from paper_1703_10973_gb300 import SDPProblem, hessian_matvec_static
    n = L.SDP_STATIC_MAX_N
    d = si.mc_instance(n // 2, n // 2, 2, 3000, 17)
    assert d.n == n
    Wn = _spd(d.n, 13)
    W = torch.from_numpy(Wn).cuda().reshape(-1).contiguous()
    trip = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).cuda() for x in (d.Ak, d.Ai, d.Aj)]
    Av = torch.from_numpy(np.ascontiguousarray(d.Av, dtype=np.float64)).cuda()
    vn = si.random_vec(d.m, 3)
    v = torch.from_numpy(vn).cuda()
    with SDPProblem.from_data(d) as prob:
        prob.set_W(W)
        ref = prob.hessian_matvec(v).cpu().numpy()
    got = hessian_matvec_static(d.n, d.m, *trip, Av, W, v).cpu().numpy()
    assert _rel(got, ref) <= 1e-12
    P = o.Problem.from_data(d)
    exact = o.hessian_auto(P, Wn) @ vn
    assert _rel(got, exact) <= 1e-12


def test_static_reports_out_of_range_triplets():
    """An index past n is skipped by the kernels (no access), counted and reported."""
    from paper_1703_10973_gb300 import _lib as L
    from paper_1703_10973_gb300 import hessian_matvec_static
    d = si.mc_instance(20, 30, 1, 200, 9)
    Ai = np.ascontiguousarray(d.Ai, dtype=np.int32).copy()
    Ai[7] = d.n + 5
    trip = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).cuda() for x in (d.Ak, Ai, d.Aj)]
    Av = torch.from_numpy(np.ascontiguousarray(d.Av, dtype=np.float64)).cuda()
    W = torch.from_numpy(_spd(d.n, 2)).cuda().reshape(-1).contiguous()
    v = torch.from_numpy(si.random_vec(d.m, 1)).cuda()
    with pytest.raises(L.SDPError, match="1 triplets had an index out of range"):
        hessian_matvec_static(d.n, d.m, *trip, Av, W, v)
    torch.cuda.synchronize()


def test_static_rejects_aliased_output():
    """Hv is cleared before v is read: an output that overlaps v is refused."""
    from paper_1703_10973_gb300 import _lib as L
    from paper_1703_10973_gb300 import hessian_matvec_static
    import ctypes as C
    d = si.mc_instance(10, 12, 1, 60, 3)
    trip = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).cuda() for x in (d.Ak, d.Ai, d.Aj)]
    Av = torch.from_numpy(np.ascontiguousarray(d.Av, dtype=np.float64)).cuda()
    W = torch.from_numpy(_spd(d.n, 2)).cuda().reshape(-1).contiguous()
    v = torch.from_numpy(si.random_vec(d.m, 1)).cuda()
    with pytest.raises(ValueError, match="must not be v"):
        hessian_matvec_static(d.n, d.m, *trip, Av, W, v, out=v)
    lib = L.load()
    st = lib.sdp_hessian_matvec_static(d.n, d.m, int(Av.numel()), C.c_void_p(trip[0].data_ptr()),
                                       C.c_void_p(trip[1].data_ptr()), C.c_void_p(trip[2].data_ptr()),
                                       C.c_void_p(Av.data_ptr()), C.c_void_p(W.data_ptr()),
                                       C.c_void_p(v.data_ptr()), C.c_void_p(v.data_ptr() + 8), None)
    assert st == L.SDP_ERR_ARG
    assert b"overlaps" in lib.sdp_last_error(None)
