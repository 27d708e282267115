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
