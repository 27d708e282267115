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


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_batch_equals_alone(prec):
    """Batched kernels under the batch graph, and a solve on its own (which runs
    its Newton systems through a one-problem batch), both equal the
    single-problem kernels driven from the host (pcg_graph = 0) bit for bit."""
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem, default_params
    params = default_params(prec=prec)
    insts = _instances()
    alone = []
    for d in insts:
        with SDPProblem.from_data(d, params=default_params(prec=prec, pcg_graph=0)) as p:
            r = p.solve()
            alone.append((r, p.get_solution()))
        with SDPProblem.from_data(d, params=params) as p:
            r1 = p.solve()
            s1 = p.get_solution()
        assert r1["iters"] == r["iters"] and r1["pcg_iters_total"] == r["pcg_iters_total"]
        for xa, xb in zip(alone[-1][1], s1):
            assert np.array_equal(xa, xb)
    streams = [torch.cuda.Stream() for _ in insts]
    probs = [SDPProblem.from_data(d, params=params, stream=s.cuda_stream) for d, s in zip(insts, streams)]
    with SDPBatch(probs, groups=1) as b:
        res = b.solve()
        sols = [p.get_solution() for p in probs]
        stages = b.stage_seconds()
    assert set(stages) == set(SDPBatch.STAGES) and all(v >= 0.0 for v in stages.values())
    assert stages["pcg_pred"] > 0.0 and stages["nt_precond"] > 0.0
    for p in probs:
        p.close()
    for (ra, sa), rb, sb in zip(alone, res, sols):
        assert ra["converged"] and rb["converged"]
        assert ra["iters"] == rb["iters"] and ra["pcg_iters_total"] == rb["pcg_iters_total"]
        assert ra["obj_p"] == rb["obj_p"]
        for xa, xb in zip(sa, sb):
            assert np.array_equal(xa, xb)


def test_batch_rejects_unsupported_preconditioner():
    """Batched PCG applies the Hhat preconditioner only; Algorithm 1's dense core is refused."""
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem, default_params
    from paper_1703_10973_gb300._lib import SDPError
    d = _instances()[0]
    with SDPProblem.from_data(d, params=default_params(precond=1)) as p:
        with pytest.raises(SDPError):
            SDPBatch([p])


def test_batch_mixed_precisions_match_oracle():
    """FP32, FP64 and BF16 problems in one batch; each reaches the oracle's optimum."""
    from oracle import sdp_oracle as o
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem, default_params
    insts = _instances()[1:4]
    precs = ["fp32", "fp64", "bf16"]
    probs = [SDPProblem.from_data(d, params=default_params(prec=pr)) for d, pr in zip(insts, precs)]
    with SDPBatch(probs) as b:
        res = b.solve()
    for d, p, r in zip(insts, probs, res):
        P = o.Problem.from_data(d)
        ref = o.ipm_solve(P)
        assert r["converged"] and abs(r["obj_p"] - ref.obj_p) <= 1e-6 * abs(ref.obj_p)
        p.close()


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


def test_batch_host_loop_equals_graph():
    """pcg_graph = 0 drives the same batched kernels from the host: identical iterates."""
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem, default_params
    insts = _instances()[:3]
    out = []
    for g in (1, 0):
        params = default_params(pcg_graph=g)
        probs = [SDPProblem.from_data(d, params=params) for d in insts]
        with SDPBatch(probs) as b:
            res = b.solve()
            out.append((res, [p.get_solution() for p in probs]))
        for p in probs:
            p.close()
    (r1, s1), (r0, s0) = out
    for a, c in zip(r1, r0):
        assert a["iters"] == c["iters"] and a["pcg_iters_total"] == c["pcg_iters_total"] and a["obj_p"] == c["obj_p"]
    for a, c in zip(s1, s0):
        for xa, xc in zip(a, c):
            assert np.array_equal(xa, xc)


@pytest.mark.parametrize("groups", [0, 2, 5])
def test_batch_groups_equal_one_lockstep(groups):
    """Concurrent lockstep groups (0 = pairs) give every problem the same iterates."""
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem
    insts = _instances()
    out = []
    for g in (1, groups):
        streams = [torch.cuda.Stream() for _ in insts]
        probs = [SDPProblem.from_data(d, stream=s.cuda_stream) for d, s in zip(insts, streams)]
        with SDPBatch(probs, groups=g) as b:
            res = b.solve()
            out.append((res, [p.get_solution() for p in probs], b.stage_seconds()))
        for p in probs:
            p.close()
    (r1, s1, _), (rg, sg, stg) = out
    assert stg["graph_launches"] >= 1
    for a, c in zip(r1, rg):
        assert a["converged"] and c["converged"]
        assert a["iters"] == c["iters"] and a["pcg_iters_total"] == c["pcg_iters_total"] and a["obj_p"] == c["obj_p"]
    for a, c in zip(s1, sg):
        for xa, xc in zip(a, c):
            assert np.array_equal(xa, xc)


def test_dynamic_membership_equals_alone():
    """Members that join a running batch later (sdp_batch_add between steps) and
    leave when done (sdp_batch_remove) get the same iterates as alone."""
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem
    insts = _instances()[:4]
    alone = []
    for d in insts:
        with SDPProblem.from_data(d) as p:
            alone.append((p.solve(), p.get_solution()))
    streams = [torch.cuda.Stream() for _ in insts]
    probs = [SDPProblem.from_data(d, stream=s.cuda_stream) for d, s in zip(insts, streams)]
    got = {}
    with SDPBatch([]) as b:
        b.add(probs[0])
        b.add(probs[1])
        steps = 0
        joined = 2
        while len(got) < len(probs):
            if steps == 3 and joined < len(probs):
                b.add(probs[joined])
                joined += 1
            if steps == 5 and joined < len(probs):
                b.add(probs[joined])
                joined += 1
            b.step()
            steps += 1
            for i, p in enumerate(probs[:joined]):
                if i in got:
                    continue
                res, where, st = b.member(p)
                if where != "running":
                    got[i] = (res, where, p.get_solution())
                    b.remove(p)
            assert steps < 200
    for i, (ra, sa) in enumerate(alone):
        res, where, sb = got[i]
        assert where == "converged"
        assert res["iters"] == ra["iters"] and res["pcg_iters_total"] == ra["pcg_iters_total"]
        assert res["obj_p"] == ra["obj_p"]
        for xa, xb in zip(sa, sb):
            assert np.array_equal(xa, xb)
    for p in probs:
        p.close()


def test_spmm_autotuner_picks_a_measured_tile():
    """The batch times the SpMM tile candidates on its own data and keeps the fastest
    (the results above are bitwise the same whatever it picks)."""
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem
    insts = _instances()
    probs = [SDPProblem.from_data(d) for d in insts]
    with SDPBatch(probs, groups=1) as b:
        assert b.tuning()[0] == 0
        b.solve()
        r, ms = b.tuning()
    for p in probs:
        p.close()
    assert r in (1, 2, 4, 8) and r in ms
    assert ms[r] == min(ms.values()) and all(v > 0 for v in ms.values())
