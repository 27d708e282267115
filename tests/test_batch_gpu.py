"""Batched solves (sdp_batch_*): problems advanced in lockstep with one launch per
PCG step for all of them give, problem by problem, the same iterates as alone."""
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


def _instances():
    specs = [dict(p=30, q=25, r=1, m=400, seed=81), dict(p=40, q=60, r=2, m=1500, seed=82),
             dict(p=90, q=70, r=2, m=3000, seed=83), dict(p=120, q=40, r=3, m=2600, seed=84),
             dict(p=65, q=172, r=1, m=3888, seed=4014)]
    return [si.mc_instance(s["p"], s["q"], s["r"], s["m"], s["seed"]) for s in specs]


def test_batch_equals_alone():
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem
    insts = _instances()
    alone = []
    for d in insts:
        with SDPProblem.from_data(d) as p:
            r = p.solve()
            alone.append((r, p.get_solution()))
    streams = [torch.cuda.Stream() for _ in insts]
    probs = [SDPProblem.from_data(d, stream=s.cuda_stream) for d, s in zip(insts, streams)]
    with SDPBatch(probs) as b:
        res = b.solve()
        sols = [p.get_solution() for p in probs]
    for p in probs:
        p.close()
    for (ra, sa), rb, sb in zip(alone, res, sols):
        assert ra["converged"] and rb["converged"]
        assert ra["iters"] == rb["iters"] and ra["pcg_iters_total"] == rb["pcg_iters_total"]
        assert ra["obj_p"] == rb["obj_p"]
        for xa, xb in zip(sa, sb):
            assert np.array_equal(xa, xb)


def test_batch_rejects_unsupported_precision():
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem, default_params
    from paper_1703_10973_gb300._lib import SDPError
    d = _instances()[0]
    with SDPProblem.from_data(d, params=default_params(prec="fp32")) as p:
        with pytest.raises(SDPError):
            SDPBatch([p])


def test_batch_matches_oracle():
    from oracle import sdp_oracle as o
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem
    insts = _instances()[:3]
    probs = [SDPProblem.from_data(d) for d in insts]
    with SDPBatch(probs) as b:
        res = b.solve()
    for d, p, r in zip(insts, probs, res):
        P = o.Problem.from_data(d)
        ref = o.ipm_solve(P)
        assert r["converged"] and abs(r["obj_p"] - ref.obj_p) <= 1e-6 * abs(ref.obj_p)
        X, y, S = p.get_solution()
        cert = o.kkt_certificate(P, X, y, S)
        assert cert["pinf"] <= 1e-6 and cert["dinf"] <= 1e-6
        p.close()
