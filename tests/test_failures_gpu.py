"""Failure paths of the C ABI, provoked without faulting or hanging the GPU.

Each error status is made to happen on purpose -- a bounded device wait that is
given almost no time, a non-finite right-hand side, an iteration cap, an
indefinite iterate or scaling matrix -- and the handle is checked to stay
usable afterwards.  The checkpoint pair sdp_get_state / sdp_set_state is checked
to resume a solve on the same iterates.
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


def _status_of(fn):
    from paper_1703_10973_gb300 import _lib as L
    try:
        fn()
    except L.SDPError as e:
        return e.status
    return L.SDP_OK


def test_grid_barrier_wait_runs_out_and_handle_survives():
    """n > 1024 runs the cooperative tridiagonalisation, whose grid barriers are
    bounded spin waits.  With a bound of one SM clock cycle the first wait runs
    out: the kernel sets its flag and returns, and the IPM step reports
    SDP_ERR_TIMEOUT.  The same instance then steps normally with the default bound."""
    from paper_1703_10973_gb300 import _lib as L
    from paper_1703_10973_gb300 import SDPProblem, default_params
    d = si.mc_instance(560, 540, 1, 4000, 31)
    assert d.n > 1024
    with SDPProblem.from_data(d, params=default_params(wait_cycles=1)) as p:
        assert _status_of(p.ipm_step) == L.SDP_ERR_TIMEOUT
        assert "timeout" in p.lib.sdp_last_error(p.h).decode()
    torch.cuda.synchronize()
    with SDPProblem.from_data(d) as p:
        info = p.ipm_step()
        assert info["pcg_relres_pred"] <= 1e-8 and np.isfinite(info["mu"])


def _ready_problem(seed=3):
    from paper_1703_10973_gb300 import SDPProblem
    d = si.mc_instance(30, 40, 2, 500, seed)
    p = SDPProblem.from_data(d)
    p.set_W(torch.from_numpy(si.random_spd(d.n, 5, cond=50.0)).cuda().reshape(-1).contiguous())
    p.precond_build()
    return d, p


def test_nonfinite_rhs_is_numeric_error():
    from paper_1703_10973_gb300 import _lib as L
    d, p = _ready_problem()
    with p:
        r = torch.from_numpy(si.random_vec(d.m, 1)).cuda()
        r[17] = float("nan")
        assert _status_of(lambda: p.pcg_solve(r)) == L.SDP_ERR_NUMERIC
        r[17] = 0.5                                  # the handle keeps working
        y, its, rel, st = p.pcg_solve(r)
        assert st == L.SDP_OK and rel <= 1e-8


def test_pcg_iteration_cap_returns_maxit_with_best_iterate():
    from paper_1703_10973_gb300 import _lib as L
    d, p = _ready_problem()
    with p:
        r = torch.from_numpy(si.random_vec(d.m, 2)).cuda()
        y, its, rel, st = p.pcg_solve(r, rtol=1e-14, maxit=2)
        assert st == L.SDP_ERR_MAXIT
        assert its <= 2 and 0.0 < rel < 1.0          # the iterate reduced the residual
        assert torch.isfinite(y).all()


def test_indefinite_scaling_matrix_rejected_by_preconditioner():
    from paper_1703_10973_gb300 import _lib as L
    from paper_1703_10973_gb300 import SDPProblem
    d = si.mc_instance(30, 40, 2, 500, 3)
    with SDPProblem.from_data(d) as p:
        W = si.random_spd(d.n, 5, cond=50.0) - 2.0 * np.eye(d.n) * 50.0
        p.set_W(torch.from_numpy(W).cuda().reshape(-1).contiguous())
        assert _status_of(p.precond_build) == L.SDP_ERR_NUMERIC
        assert "not positive" in p.lib.sdp_last_error(p.h).decode()
        p.set_W(torch.from_numpy(si.random_spd(d.n, 5, cond=50.0)).cuda().reshape(-1).contiguous())
        p.precond_build()


def test_indefinite_iterate_is_not_pd_and_recoverable():
    from paper_1703_10973_gb300 import _lib as L
    from paper_1703_10973_gb300 import SDPProblem
    d = si.mc_instance(20, 25, 1, 200, 4)
    with SDPProblem.from_data(d) as p:
        X0, y0, S0, it0 = p.get_state()
        bad = X0.copy()
        bad[3, 3] = -1.0
        p.set_state(bad, y0, S0, 0)
        assert _status_of(p.ipm_step) == L.SDP_ERR_NOT_PD
        assert "chol(X)" in p.lib.sdp_last_error(p.h).decode()
        p.set_state(X0, y0, S0, it0)                 # back to the start point: the solve runs
        res = p.solve()
        assert res["converged"] == 1


def test_checkpoint_resume_gives_the_same_iterates():
    from paper_1703_10973_gb300 import SDPProblem
    d = si.mc_instance(40, 50, 2, 900, 8)
    with SDPProblem.from_data(d) as a, SDPProblem.from_data(d) as b:
        for _ in range(4):
            a.ipm_step()
        X, y, S, it = a.get_state()
        assert it == 4
        b.set_state(X, y, S, it)
        for _ in range(3):
            ia = a.ipm_step()
            ib = b.ipm_step()
            assert ia["iter"] == ib["iter"]
        Xa, ya, Sa, ita = a.get_state()
        Xb, yb, Sb, itb = b.get_state()
        assert ita == itb == 7
        assert np.linalg.norm(Xa - Xb) <= 1e-12 * np.linalg.norm(Xa)
        assert np.linalg.norm(ya - yb) <= 1e-12 * max(np.linalg.norm(ya), 1.0)
