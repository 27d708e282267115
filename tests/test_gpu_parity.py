"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every input is seeded and synthetic; expected values come from ``oracle/`` run
on the same inputs.  Tolerances: FP64 matvec 1e-12 relative (2-norm);
preconditioner apply 1e-9; PCG to the requested true residual; the IPM end
point within 1e-6 relative objective error and 1e-5 relative Frobenius error
of the recovered matrix.
"""
import numpy as np
import pytest

import sdp_inputs as si
from oracle import sdp_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10973_gb300 import _build, load
    _build.build()
    load()


def _prob(d, **kw):
    from paper_1703_10973_gb300 import SDPProblem, default_params
    return SDPProblem.from_data(d, params=default_params(**kw))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _ipm_like_W(n, k, mu, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.concatenate([rng.uniform(1.0, 3.0, n - k), rng.uniform(1.0, 2.0, k) / mu])
    return (Q * ev) @ Q.T


# --------------------------------------------------------------------------
# hessian_matvec
# --------------------------------------------------------------------------

MATVEC_CASES = {
    "mc_tiny": lambda: si.mc_instance(5, 7, 1, 20, 3),
    "mc_C1": lambda: si.config_instance("C1"),
    "mc_ragged": lambda: si.mc_instance(37, 61, 2, 900, 5),   # n = 98: ragged tails everywhere
    "general": lambda: si.random_general(23, 40, 3, 2),
    "diag": lambda: si.diag_constraint_instance(17, 1),
    "unit_diag": lambda: si.unit_diag_instance(9),
}


@pytest.mark.parametrize("case", sorted(MATVEC_CASES))
def test_matvec_fp64_matches_oracle(case):
    d = MATVEC_CASES[case]()
    P = o.Problem.from_data(d)
    W = _ipm_like_W(d.n, min(2, d.n - 1), 1e-3, 11)
    with _prob(d) as prob:
        prob.set_W(_dev(W))
        for seed in (1, 2):
            v = si.random_vec(d.m, seed)
            hv = prob.hessian_matvec(_dev(v)).cpu().numpy()
            assert _rel(hv, o.hessian_matvec(P, W, v)) <= 1e-12


def test_matvec_fp64_C2_full_size():
    """Full C2 size (n = 1000, m = 8000) with W from a real oracle NT scaling."""
    d = si.config_instance("C2")
    P = o.Problem.from_data(d)
    X = si.random_spd(d.n, 5, cond=1e4)
    S = si.random_spd(d.n, 6, cond=1e4)
    W = o.nt_scaling(X, S)
    v = si.random_vec(d.m, 9)
    with _prob(d) as prob:
        prob.set_W(_dev(W))
        hv = prob.hessian_matvec(_dev(v)).cpu().numpy()
    assert _rel(hv, o.hessian_matvec(P, W, v)) <= 1e-12


def test_matvec_explicit_hessian_columns():
    """H e_j from the GPU equals column j of the explicit Hessian (closed form)."""
    d = si.mc_instance(6, 8, 2, 30, 4)
    P = o.Problem.from_data(d)
    W = si.random_spd(d.n, 2, cond=50.0)
    H = o.hessian_entries(P, W)
    with _prob(d) as prob:
        prob.set_W(_dev(W))
        E = np.eye(d.m)
        for j in (0, 7, d.m - 1):
            col = prob.hessian_matvec(_dev(E[:, j])).cpu().numpy()
            assert _rel(col, H[:, j]) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("bf16", 2e-2)])
def test_matvec_reduced_precision(prec, tol):
    d = si.mc_instance(40, 50, 2, 700, 8)
    P = o.Problem.from_data(d)
    W = si.random_spd(d.n, 3, cond=30.0)
    v = si.random_vec(d.m, 1)
    with _prob(d) as prob:
        prob.set_W(_dev(W))
        hv = prob.hessian_matvec(_dev(v), prec=prec).cpu().numpy()
    assert _rel(hv, o.hessian_matvec(P, W, v)) <= tol


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("bf16", 5e-2)])
def test_matvec_split_reduced_precision_near_optimum(prec, tol):
    """With the preconditioner built, the reduced-precision matvec splits W = W_l + W_s.
    On a W with k eigenvalues of order 1/mu (mu = 1e-4) the error, measured as
    ||H^{-1}(Hv_gpu - Hv)|| / ||v|| (the scale PCG works on), stays at the working
    precision, where rounding W whole loses the small part of W."""
    d = si.mc_instance(20, 25, 2, 300, 8)
    P = o.Problem.from_data(d)
    W = _ipm_like_W(d.n, 2, 1e-4, 3)
    H = o.hessian_entries(P, W)
    v = si.random_vec(d.m, 1)
    ref = H @ v
    with _prob(d) as prob:
        prob.set_W(_dev(W))
        plain = prob.hessian_matvec(_dev(v), prec=prec).cpu().numpy()
        prob.precond_build()
        split = prob.hessian_matvec(_dev(v), prec=prec).cpu().numpy()
    e_split = np.linalg.norm(np.linalg.solve(H, split - ref)) / np.linalg.norm(v)
    e_plain = np.linalg.norm(np.linalg.solve(H, plain - ref)) / np.linalg.norm(v)
    assert e_split <= tol
    assert e_split <= 0.1 * e_plain


# --------------------------------------------------------------------------
# preconditioner
# --------------------------------------------------------------------------

# Algorithm 1's Ht (eq. AtIUUtAt) and Section V's Hhat (eq. sparse_prec):
# sdp_params.precond code and the oracle's builder
PRECONDS = {"woodbury": (1, o.precond_build), "hat": (2, o.precond_hat_build)}


@pytest.mark.parametrize("kind", list(PRECONDS))
@pytest.mark.parametrize("mu", [1e-1, 1e-4, 1e-7])
def test_precond_apply_matches_dense_inverse(kind, mu):
    """eq. (SMW2) on the GPU equals the oracle's dense solve with eq. (AtIUUtAt) / (sparse_prec)."""
    code, build = PRECONDS[kind]
    d = si.mc_instance(9, 11, 2, 60, 6)
    P = o.Problem.from_data(d)
    W = _ipm_like_W(d.n, 2, mu, 3)
    pc = build(P, W, 2)
    Ht = o.precond_dense(P, pc)
    r = si.random_vec(d.m, 2)
    zref = np.linalg.solve(Ht, r)
    with _prob(d, precond=code) as prob:
        prob.set_W(_dev(W))
        prob.precond_build()
        tau, k = prob.precond_info()
        z = prob.precond_apply(_dev(r)).cpu().numpy()
    assert k == 2
    assert abs(tau - pc.tau) <= 1e-10 * abs(pc.tau) + 1e-14 * np.abs(W).max()
    # eq. (SMW2) is forward-accurate to about kappa(Ht) eps (the instability the
    # paper discusses in Section IV); the oracle's own SMW apply shows the same gap.
    kap = np.linalg.cond(Ht)
    tol = max(1e-12, 20.0 * kap * np.finfo(float).eps)
    assert _rel(z, zref) <= tol
    assert _rel(z, o.precond_apply(P, pc, r)) <= tol


@pytest.mark.parametrize("kind", list(PRECONDS))
def test_precond_general_constraints(kind):
    code, build = PRECONDS[kind]
    d = si.random_general(14, 20, 2, 7)
    P = o.Problem.from_data(d)
    W = _ipm_like_W(d.n, 2, 1e-3, 5)
    pc = build(P, W, 2)
    r = si.random_vec(d.m, 3)
    with _prob(d, precond=code) as prob:
        prob.set_W(_dev(W))
        prob.precond_build()
        z = prob.precond_apply(_dev(r)).cpu().numpy()
    assert _rel(z, o.precond_apply(P, pc, r)) <= 1e-9


@pytest.mark.parametrize("kind", list(PRECONDS))
def test_precond_exact_for_low_rank_W(kind):
    """W = tau I + U U^T makes Ht = H (PCG converges in one iteration) and H - Hhat
    of rank <= k(k+1)/2 (at most k(k+1)/2 + 1 iterations) on the GPU."""
    code, _ = PRECONDS[kind]
    d = si.mc_instance(10, 10, 2, 50, 9)
    rng = np.random.default_rng(5)
    U0 = rng.standard_normal((d.n, 2)) * 3.0
    W = 0.8 * np.eye(d.n) + U0 @ U0.T
    r = si.random_vec(d.m, 3)
    with _prob(d, precond=code) as prob:
        prob.set_W(_dev(W))
        prob.precond_build()
        y, its, rel, st = prob.pcg_solve(_dev(r), rtol=1e-10, maxit=50)
    assert its <= (1 if kind == "woodbury" else 4) and rel <= 1e-9


# --------------------------------------------------------------------------
# PCG
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", list(PRECONDS))
@pytest.mark.parametrize("mu", [1e-2, 1e-5])
def test_pcg_matches_direct_solve(mu, kind):
    code, _ = PRECONDS[kind]
    d = si.mc_instance(12, 14, 2, 100, 10)
    P = o.Problem.from_data(d)
    W = _ipm_like_W(d.n, 2, mu, 4)
    H = o.hessian_entries(P, W)
    # right-hand side with a solution of unit size, as for a Newton step
    ystar = si.random_vec(d.m, 5)
    ystar /= np.linalg.norm(ystar)
    r = H @ ystar
    with _prob(d, precond=code) as prob:
        prob.set_W(_dev(W))
        prob.precond_build()
        y, its, rel, st = prob.pcg_solve(_dev(r), rtol=1e-10, maxit=500)
    y = y.cpu().numpy()
    assert rel <= 1e-10
    assert np.linalg.norm(H @ y - r) <= 1e-9 * np.linalg.norm(r)
    assert _rel(y, ystar) <= 1e-10 * np.linalg.cond(H)
    # the preconditioned iteration count stays small and independent of mu
    # (Lemma Htilde; Lemma aug_prec with k^2 outliers), against m = 100 unknowns
    # and kappa(H) far above 1e6
    assert its <= 80


def test_pcg_host_loop_matches_graph_loop():
    """The host-driven PCG loop launches the same kernels as the graph's while node."""
    d = si.mc_instance(12, 14, 2, 100, 10)
    W = _ipm_like_W(d.n, 2, 1e-4, 4)
    r = si.random_vec(d.m, 5)
    out = []
    for g in (1, 0):
        with _prob(d, pcg_graph=g) as prob:
            prob.set_W(_dev(W))
            prob.precond_build()
            y, its, rel, st = prob.pcg_solve(_dev(r), rtol=1e-10, maxit=500)
            out.append((y.cpu().numpy(), its, rel))
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("mu", [1e-1, 1e-3])
def test_precond_apply_fp32_core_close_to_fp64(mu):
    """prec = SDP_FP32 in sdp_precond_apply: the Hhat core solve reads the FP32 copy
    of the Schur-factor inverse.  Rounding L_C^{-1} to FP32 perturbs the core solve
    by about kappa(core) 2^-24 relative, so the applied z stays within
    20 kappa(Hhat) 2^-24 of the exact z (the oracle's dense solve with eq. sparse_prec)."""
    d = si.mc_instance(30, 26, 2, 400, 12)
    P = o.Problem.from_data(d)
    W = _ipm_like_W(d.n, 2, mu, 3)
    pc = o.precond_hat_build(P, W, 2)
    Hh = o.precond_dense(P, pc)
    r = si.random_vec(d.m, 2)
    zref = np.linalg.solve(Hh, r)
    with _prob(d, precond=2) as prob:
        prob.set_W(_dev(W))
        prob.precond_build()
        z32 = prob.precond_apply(_dev(r), prec="fp32").cpu().numpy()
        z64 = prob.precond_apply(_dev(r), prec="fp64").cpu().numpy()
    tol = 20.0 * np.linalg.cond(Hh) * 2.0 ** -24
    assert 0.0 < _rel(z32, z64) <= tol            # a different (float) product ran
    assert _rel(z32, zref) <= tol
    assert _rel(z64, zref) <= max(1e-12, 20.0 * np.linalg.cond(Hh) * np.finfo(float).eps)


@pytest.mark.parametrize("prec,mu", [("fp32", 1e-3), ("bf16", 1e-1), ("bf16", 1e-5), ("fp32", 1e-5)])
def test_pcg_reduced_precision_refined_to_fp64(prec, mu):
    d = si.mc_instance(12, 14, 2, 100, 10)
    P = o.Problem.from_data(d)
    W = _ipm_like_W(d.n, 2, mu, 4)
    H = o.hessian_entries(P, W)
    r = si.random_vec(d.m, 5)
    with _prob(d) as prob:
        prob.set_W(_dev(W))
        prob.precond_build()
        y, its, rel, st = prob.pcg_solve(_dev(r), rtol=1e-8, maxit=2000, prec=prec)
    y = y.cpu().numpy()
    assert rel <= 1e-8
    # The oracle's residual H y - r is itself computed in FP64: each entry of H y
    # carries a rounding error up to m eps (|H| |y|)_i (the standard bound for a
    # dot product of length m), which near the optimum (|H| ~ 1/mu^2) is no
    # longer small against 1e-8 ||r||.
    slack = d.m * np.finfo(float).eps * np.linalg.norm(np.abs(H) @ np.abs(y))
    assert np.linalg.norm(H @ y - r) <= 1.01e-8 * np.linalg.norm(r) + slack


# --------------------------------------------------------------------------
# interior-point method
# --------------------------------------------------------------------------

def test_first_ipm_step_matches_oracle():
    """Same rules on both sides: after one step the iterates agree to PCG accuracy."""
    d = si.config_instance("C1")
    P = o.Problem.from_data(d)
    ref = o.ipm_solve(P, o.IPMParams(maxit=1))
    with _prob(d) as prob:
        info = prob.ipm_step()
        X, y, S = prob.get_solution()
    assert abs(info["alpha_p"] - ref.log[0]["alpha_p"]) <= 1e-6
    assert abs(info["alpha_d"] - ref.log[0]["alpha_d"]) <= 1e-6
    assert _rel(X, ref.X) <= 1e-6 and _rel(S, ref.S) <= 1e-6 and _rel(y, ref.y) <= 1e-6


def test_solve_C1_matches_oracle_and_recovers_M():
    d = si.config_instance("C1")
    P = o.Problem.from_data(d)
    ref = o.ipm_solve(P)
    with _prob(d) as prob:
        res = prob.solve()
        X, y, S = prob.get_solution()
    assert res["converged"] and res["relgap"] <= 1e-6
    assert abs(res["obj_p"] - ref.obj_p) <= 1e-6 * abs(ref.obj_p)
    Z = o.mc_recovered(P, X)
    assert _rel(Z, o.mc_recovered(P, ref.X)) <= 1e-5
    assert _rel(Z, d.meta["M"]) <= 1e-5
    cert = o.kkt_certificate(P, X, y, S)
    assert cert["pinf"] <= 1e-6 and cert["dinf"] <= 1e-6


def test_solve_unit_diagonal_closed_form():
    d = si.unit_diag_instance(12)
    with _prob(d) as prob:
        res = prob.solve()
        X, y, S = prob.get_solution()
    assert res["converged"]
    assert np.abs(X - np.eye(12)).max() <= 1e-5
    assert np.abs(y - 1.0).max() <= 1e-5


def test_solve_maxcut_bipartite_closed_form():
    d = si.maxcut_bipartite_instance(5, 6, 3, extra_edges=8)
    with _prob(d, gap_tol=1e-8, infeas_tol=1e-8) as prob:
        res = prob.solve()
        X, _, _ = prob.get_solution()
    z = d.meta["z"]
    assert abs(res["obj_p"] + 2 * d.meta["n_edges"]) <= 1e-5 * 2 * d.meta["n_edges"]
    assert np.abs(X - np.outer(z, z)).max() <= 1e-3


def _planted_general(n=30, m=100, nnz_per=3, rank=2, seed=21):
    """General sparse SDP (disjoint supports, A^T A diagonal) with a planted
    strictly complementary optimum: X* = V V^T of rank 2, S* on the orthogonal
    complement, y* random; b = A(X*) and C = A^T y* + S* are built with the
    oracle's operators, so (X*, y*, S*) is optimal with zero duality gap."""
    d = si.random_general(n, m, nnz_per, seed)
    P = o.Problem.from_data(d)
    rng = np.random.default_rng(seed + 100)
    V = rng.standard_normal((n, rank))
    Xs = V @ V.T
    Q, _ = np.linalg.qr(np.concatenate([V, rng.standard_normal((n, n - rank))], axis=1))
    Qp = Q[:, rank:]
    Ss = (Qp * rng.uniform(0.5, 2.0, n - rank)) @ Qp.T
    ys = rng.standard_normal(m)
    b = o.op_A(P, Xs)
    Cm = o.op_At(P, ys) + Ss
    iu, ju = np.triu_indices(n)
    d2 = si.SDPData(n=n, m=m, Ci=iu.astype(np.int32), Cj=ju.astype(np.int32), Cv=Cm[iu, ju],
                    Ak=d.Ak, Ai=d.Ai, Aj=d.Aj, Av=d.Av, b=b, k=rank, meta=dict(kind="planted"))
    return d2, Xs, ys, Ss


def test_solve_general_sparse_planted():
    d, Xs, ys, Ss = _planted_general()
    P = o.Problem.from_data(d)
    ref = o.ipm_solve(P)
    assert ref.converged
    with _prob(d) as prob:
        res = prob.solve()
        X, y, S = prob.get_solution()
    assert res["converged"]
    assert abs(res["obj_p"] - ref.obj_p) <= 1e-6 * (1 + abs(ref.obj_p))
    assert _rel(X, Xs) <= 1e-5 and _rel(X, ref.X) <= 1e-5
    cert = o.kkt_certificate(P, X, y, S)
    assert cert["pinf"] <= 1e-6 and cert["dinf"] <= 1e-6 and cert["relgap"] <= 1e-6


# The recovered matrix is held to 1e-5 relative Frobenius error.  A relative gap
# of 1e-6 bounds the objective, not the distance of the iterate to the optimum
# (near a rank-r optimum that distance shrinks only like the square root of mu),
# so the GPU solves run to the accuracy of the paper's experiments (Section VI
# reports 8 to 10 digits): gap and infeasibilities <= 1e-8.  The explicit-Hessian
# oracle cannot follow there: kappa(H) grows like 1/mu^2 and its Cholesky of H
# breaks down before mu reaches 1e-9, so it stops at the 1e-6 gap of the
# objective tolerance.  In the exact-recovery regime the optimum is the planted M, which
# pins the 1e-8 solve; the oracle pins the objective.
TIGHT = dict(gap_tol=1e-8, infeas_tol=1e-8)


def _gap_abs(r):
    """Absolute duality gap implied by a result's relative gap (the relgap definition)."""
    return r["relgap"] * (1.0 + abs(r["obj_p"]) + abs(r["obj_d"]))


@pytest.mark.parametrize("idx", [3, 14])
def test_solve_batched_instance_matches_oracle(idx):
    """Batched-workload instances (n >= 64: Lanczos step lengths, Hhat preconditioner,
    checked updates) reach the oracle's optimum and recover the planted matrix."""
    s = si.batched_specs(256)[idx]
    d = si.mc_instance(s["p"], s["q"], s["r"], s["m"], s["seed"])
    P = o.Problem.from_data(d)
    ref = o.ipm_solve(P)
    assert ref.converged
    M = d.meta["M"]
    with _prob(d, **TIGHT) as prob:
        res = prob.solve()
        X, y, S = prob.get_solution()
    assert res["converged"] and res["relgap"] <= 1e-8
    # both objectives lie within their own duality gaps of the optimal value,
    # which is ||M||_* here (exact recovery); the oracle's 1e-6 solve is only as
    # close to it as its gap, about 2e-6 relative under the relgap definition
    ref_gap = ref.relgap * (1.0 + abs(ref.obj_p) + abs(ref.obj_d))
    assert abs(res["obj_p"] - ref.obj_p) <= _gap_abs(res) + ref_gap
    nuc = float(np.linalg.svd(M, compute_uv=False).sum())
    assert abs(res["obj_p"] - nuc) <= 1e-6 * nuc
    Z = o.mc_recovered(P, X)
    assert _rel(Z, M) <= 1e-5
    # the oracle's 1e-6 point is as close to M as its gap allows, and so to Z
    assert _rel(Z, o.mc_recovered(P, ref.X)) <= 1e-5 + _rel(o.mc_recovered(P, ref.X), M)
    cert = o.kkt_certificate(P, X, y, S)
    assert cert["pinf"] <= 1e-6 and cert["dinf"] <= 1e-6 and cert["relgap"] <= 1e-6


def test_solve_batched_B0_recovers_planted_matrix():
    """B0 (n = 565, m = 37202), the largest instance of the bench batch, is beyond the
    explicit-Hessian oracle on test time (an m x m Cholesky of 1.7e13 flops per
    iteration).  It is pinned by what the mathematics fixes instead: in the exact
    recovery regime of Section V-A the optimum is the planted M, its objective is
    ||M||_* (sum of singular values, numpy SVD), and the FP64 KKT certificate holds."""
    s = si.batched_specs(256)[0]
    d = si.mc_instance(s["p"], s["q"], s["r"], s["m"], s["seed"])
    assert d.n == 565
    P = o.Problem.from_data(d)
    M = d.meta["M"]
    nuc = float(np.linalg.svd(M, compute_uv=False).sum())
    with _prob(d, **TIGHT) as prob:
        res = prob.solve()
        X, y, S = prob.get_solution()
    assert res["converged"] and res["relgap"] <= 1e-8
    assert abs(res["obj_p"] - nuc) <= 1e-6 * nuc
    assert _rel(o.mc_recovered(P, X), M) <= 1e-5
    cert = o.kkt_certificate(P, X, y, S)
    assert cert["pinf"] <= 1e-6 and cert["dinf"] <= 1e-6 and cert["relgap"] <= 1e-6
    assert cert["lmin_X"] >= -1e-8 * np.abs(X).max() and cert["lmin_S"] >= -1e-8 * np.abs(S).max()


# --------------------------------------------------------------------------
# orders above 1024: the cooperative-grid tridiagonalisation and the large
# dense factorisations
# --------------------------------------------------------------------------

def test_solve_maxcut_above_1024_matches_oracle_and_closed_form():
    """Bipartite max-cut with n = 1100 (> 1024, so every eigendecomposition runs the
    cooperative-grid tridiagonalisation): the optimum is X = z z^T with value -2|E|,
    and the oracle (explicit Hessian, m = n) reaches the same objective."""
    d = si.maxcut_bipartite_instance(550, 550, 7, extra_edges=1500)
    assert d.n > 1024
    P = o.Problem.from_data(d)
    ref = o.ipm_solve(P)
    assert ref.converged
    with _prob(d) as prob:
        res = prob.solve()
        X, y, S = prob.get_solution()
    assert res["converged"] and res["relgap"] <= 1e-6
    ne = d.meta["n_edges"]
    # each objective lies within its own duality gap of the optimal value -2|E|
    ref_gap = ref.relgap * (1.0 + abs(ref.obj_p) + abs(ref.obj_d))
    assert abs(res["obj_p"] - ref.obj_p) <= _gap_abs(res) + ref_gap
    assert abs(res["obj_p"] + 2 * ne) <= 1e-6 * 2 * ne
    z = d.meta["z"]
    assert np.abs(X - np.outer(z, z)).max() <= 1e-3
    cert = o.kkt_certificate(P, X, y, S)
    assert cert["pinf"] <= 1e-6 and cert["dinf"] <= 1e-6


def test_solve_mc_above_1024_recovers_planted_matrix():
    """Matrix completion with n = 1040 in the exact-recovery regime (m from the
    batched sampling rule, 21,675 observations): the solve recovers the planted M
    to 1e-5 and its objective is ||M||_*.  (The explicit-Hessian oracle would
    factor a 21,675-order matrix every iteration; the recovery, the nuclear norm
    and the KKT certificate pin the result instead.)  The solve runs at the default
    1e-6 tolerances: at this order the NT scaling falls back to the Denman-Beavers
    iterate from a 1e-5 gap on, and with it the primal step stalls near a 2e-8 gap, so
    the 1e-8 tolerances of the smaller instances are out of reach; the objective is
    then within its own duality gap of ||M||_*."""
    m = si.mc_m_rule(520, 520, 1)
    d = si.mc_instance(520, 520, 1, m, 1041)
    assert d.n > 1024
    P = o.Problem.from_data(d)
    M = d.meta["M"]
    nuc = float(np.linalg.svd(M, compute_uv=False).sum())
    with _prob(d) as prob:
        res = prob.solve()
        X, y, S = prob.get_solution()
    assert res["converged"] and res["relgap"] <= 1e-6
    assert abs(res["obj_p"] - nuc) <= _gap_abs(res) + 1e-6 * nuc
    assert _rel(o.mc_recovered(P, X), M) <= 1e-5
    cert = o.kkt_certificate(P, X, y, S)
    assert cert["pinf"] <= 1e-6 and cert["dinf"] <= 1e-6 and cert["relgap"] <= 1e-6


# --------------------------------------------------------------------------
# adaptive split rank (Section V implementation notes)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("eta,kmax", [(10.0, 12), (3.0, 12), (3.0, 4), (1.5, 20)])
def test_adaptive_rank_matches_oracle_rule(eta, kmax):
    """With eta > 0 the preconditioner build takes k~ = max{i <= k_max : lambda_i >=
    eta lambda_{i+1}} from the GPU eigenvalues of W; on a W with a prescribed
    spectrum it equals the oracle's rank_estimate (pinned on known spectra in the
    CPU tests), and the apply with that rank matches the oracle's Hhat solve."""
    d = si.mc_instance(40, 36, 3, 700, 19)
    P = o.Problem.from_data(d)
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((d.n, d.n)))
    top = np.array([400.0, 350.0, 90.0, 80.0, 70.0, 20.0, 18.0, 17.0, 5.0, 4.5, 4.0, 3.9, 3.8])
    ev = np.concatenate([top, rng.uniform(1.0, 1.2, d.n - top.size)])
    W = (Q * ev) @ Q.T
    want = o.rank_estimate(W, kmax, eta)
    with _prob(d, precond=2, k_max=kmax, eta=eta) as prob:
        prob.set_W(_dev(W))
        prob.precond_build()
        tau, k = prob.precond_info()
        r = si.random_vec(d.m, 4)
        z = prob.precond_apply(_dev(r)).cpu().numpy()
    assert k == want
    pc = o.precond_hat_build(P, W, want)
    Hh = o.precond_dense(P, pc)
    tol = max(1e-12, 20.0 * np.linalg.cond(Hh) * np.finfo(float).eps)
    assert _rel(z, np.linalg.solve(Hh, r)) <= tol


def test_hhat_core_above_eight_matches_oracle():
    """Split rank 20 (above the batched kernels' 8): the general-k formation,
    factorisation and solve of the Hhat core give the oracle's dense solve."""
    d = si.mc_instance(30, 34, 4, 900, 23)
    P = o.Problem.from_data(d)
    W = _ipm_like_W(d.n, 20, 1e-3, 8)
    pc = o.precond_hat_build(P, W, 20)
    Hh = o.precond_dense(P, pc)
    r = si.random_vec(d.m, 6)
    with _prob(d, precond=2, k=20) as prob:
        prob.set_W(_dev(W))
        prob.precond_build()
        tau, k = prob.precond_info()
        z = prob.precond_apply(_dev(r)).cpu().numpy()
        z32 = prob.precond_apply(_dev(r), prec="fp32").cpu().numpy()
    assert k == 20
    kap = np.linalg.cond(Hh)
    assert _rel(z, np.linalg.solve(Hh, r)) <= max(1e-12, 20.0 * kap * np.finfo(float).eps)
    assert _rel(z32, np.linalg.solve(Hh, r)) <= 20.0 * kap * 2.0 ** -24


@pytest.mark.parametrize("mu", [1e-2, 1e-5])
def test_hhat_apply_solves_the_augmented_system(mu):
    """The GPU Hhat apply (SMW with the block-sparse core) returns the solution of the
    sparse augmented system of eq. (aug_prec) as the oracle's LDL^T without
    pivoting computes it (the elimination the paper recommends for Hhat, whose
    first step leaves exactly the core the GPU factors)."""
    d = si.mc_instance(9, 11, 2, 60, 6)
    P = o.Problem.from_data(d)
    W = _ipm_like_W(d.n, 2, mu, 3)
    r = si.random_vec(d.m, 2)
    x = o.aug_prec_solve(P, W, 2, r)
    Hh = o.precond_hat_dense(P, W, 2)
    with _prob(d, precond=2) as prob:
        prob.set_W(_dev(W))
        prob.precond_build()
        z = prob.precond_apply(_dev(r)).cpu().numpy()
    tol = max(1e-12, 20.0 * np.linalg.cond(Hh) * np.finfo(float).eps)
    assert _rel(z, x) <= tol
