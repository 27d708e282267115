"""Serving on the GPU: each result is the same alone and in a concurrent mix, and
the memory estimate bounds what a problem holds."""
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
    specs = [dict(p=30, q=25, r=1, m=400, seed=71), dict(p=40, q=60, r=2, m=1500, seed=72),
             dict(p=90, q=70, r=2, m=3000, seed=73), dict(p=120, q=40, r=3, m=2600, seed=74)]
    return [si.mc_instance(s["p"], s["q"], s["r"], s["m"], s["seed"]) for s in specs]


def test_alone_equals_mix():
    from paper_1703_10973_gb300.serve import Request, Server, cuda_solver
    insts = _instances()
    solver = cuda_solver(keep_solution=True)
    alone = Server(budget_bytes=1 << 40, slots=1, solver=solver).run(
        [Request(rid=i, data=d, arrival=0.0) for i, d in enumerate(insts)])
    srv = Server(budget_bytes=1 << 40, slots=4, solver=solver)
    mix = srv.run([Request(rid=i, data=d, arrival=0.0) for i, d in enumerate(insts)])
    assert srv.stats["max_concurrent"] >= 2
    for a, b in zip(alone, mix):
        assert a.ok and b.ok and a.converged and b.converged
        assert a.iters == b.iters
        assert abs(a.obj_p - b.obj_p) <= 1e-12 * abs(a.obj_p)
        for xa, xb in zip(a.solution, b.solution):
            assert np.max(np.abs(xa - xb)) <= 1e-12 * max(1.0, np.max(np.abs(xa)))


def test_estimate_bounds_device_bytes():
    from paper_1703_10973_gb300.serve import Request, Server, cuda_solver, estimate_request_bytes
    insts = _instances()
    res = Server(budget_bytes=1 << 40, slots=2, solver=cuda_solver()).run(
        [Request(rid=i, data=d, arrival=0.0) for i, d in enumerate(insts)])
    for d, r in zip(insts, res):
        assert r.ok and 0 < r.device_bytes <= estimate_request_bytes(d)


def test_budget_admission_on_gpu():
    from paper_1703_10973_gb300.serve import Request, Server, cuda_solver, estimate_request_bytes
    insts = _instances()
    budget = max(estimate_request_bytes(d) for d in insts)   # room for about one at a time
    srv = Server(budget_bytes=budget, slots=4, solver=cuda_solver())
    res = srv.run([Request(rid=i, data=d, arrival=0.01 * i) for i, d in enumerate(insts)])
    assert all(r.ok and r.converged for r in res)
    assert srv.stats["max_in_flight_bytes"] <= budget


def test_continuous_batching_alone_equals_mix_and_matches_oracle():
    """BatchServer: requests that arrive while others run join the running lockstep
    batch and share its launches; each result is the same as the request solved
    alone (bit for bit: the batched kernels run the single-problem code over the
    same partition), and it reaches the oracle's optimum."""
    from oracle import sdp_oracle as o
    from paper_1703_10973_gb300.serve import BatchServer, Request
    insts = _instances()
    alone = []
    for i, d in enumerate(insts):
        srv = BatchServer(budget_bytes=1 << 40, groups=1, keep_solution=True)
        alone += srv.run([Request(rid=i, data=d, arrival=0.0)])
    srv = BatchServer(budget_bytes=1 << 40, groups=2, keep_solution=True)
    mix = srv.run([Request(rid=i, data=d, arrival=0.05 * i) for i, d in enumerate(insts)])
    assert srv.stats["max_concurrent"] >= 2 and srv.stats["completed"] == len(insts)
    for d, a, b in zip(insts, alone, mix):
        assert a.ok and b.ok and a.converged and b.converged
        assert a.iters == b.iters and a.obj_p == b.obj_p
        for xa, xb in zip(a.solution, b.solution):
            assert np.array_equal(xa, xb)
        ref = o.ipm_solve(o.Problem.from_data(d))
        assert abs(b.obj_p - ref.obj_p) <= 1e-6 * abs(ref.obj_p)


def test_continuous_batching_budget_and_ranks():
    """Admission by the memory budget holds with continuous batching, and a rank
    serves only its own requests (rid % world == rank)."""
    from paper_1703_10973_gb300.serve import BatchServer, Request, estimate_request_bytes
    insts = _instances()
    budget = max(estimate_request_bytes(d) for d in insts) + min(estimate_request_bytes(d) for d in insts)
    srv = BatchServer(budget_bytes=budget, groups=2)
    res = srv.run([Request(rid=i, data=d, arrival=0.0) for i, d in enumerate(insts)])
    assert all(r.ok and r.converged for r in res)
    assert srv.stats["max_in_flight_bytes"] <= budget
    srv1 = BatchServer(budget_bytes=1 << 40, groups=1, rank=1, world=2)
    res1 = srv1.run([Request(rid=i, data=d, arrival=0.0) for i, d in enumerate(insts)])
    assert [r.rid for r in res1] == [1, 3] and all(r.ok for r in res1)
