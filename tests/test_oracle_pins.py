"""Pins for the FP64 oracle: each check ties an oracle function to something
other than itself (an independent definition, a closed form, an invariant the
paper proves, brute force on a tiny case).  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import sdp_inputs as si
from oracle import sdp_oracle as o


def _mc(p, q, r, m, seed):
    return o.Problem.from_data(si.mc_instance(p, q, r, m, seed))


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# --------------------------------------------------------------------------
# Hessian (eq. hesseqn2 / hesseqn1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("maker", [
    lambda: _mc(4, 5, 1, 12, 11),
    lambda: o.Problem.from_data(si.random_general(7, 8, 2, 5)),
    lambda: o.Problem.from_data(si.diag_constraint_instance(6, 2)),
])
def test_hessian_forms_agree(maker):
    """Kronecker definition A^T (W kron W) A == tr(A_i W A_j W) == entry sum == matrix-free."""
    P = maker()
    W = si.random_spd(P.n, 7, cond=50.0)
    Hk = o.hessian_kron(P, W)
    Ht = o.hessian_trace(P, W)
    He = o.hessian_entries(P, W, chunk=5)
    assert _rel(Ht, Hk) < 1e-13
    assert _rel(He, Hk) < 1e-13
    v = si.random_vec(P.m, 3)
    assert _rel(o.hessian_matvec(P, W, v), Hk @ v) < 1e-13


def test_hessian_diag_constraints_is_hadamard():
    """A_i = e_i e_i^T gives H_ij = tr(e_i e_i^T W e_j e_j^T W) = W_ij^2, i.e. H = W o W."""
    P = o.Problem.from_data(si.diag_constraint_instance(9, 4))
    W = si.random_spd(9, 5, cond=30.0)
    assert _rel(o.hessian_entries(P, W), W * W) < 1e-14


def test_hessian_mc_closed_form():
    """For A_i = (e_p e_q^T + e_q e_p^T)/2: H_ij = (W_pp' W_qq' + W_pq' W_qp')/2."""
    P = _mc(5, 6, 2, 14, 3)
    W = si.random_spd(P.n, 9, cond=20.0)
    p, q = P.Ai, P.Aj
    Hc = 0.5 * (W[np.ix_(p, p)] * W[np.ix_(q, q)] + W[np.ix_(p, q)] * W[np.ix_(q, p)])
    assert _rel(o.hessian_entries(P, W), Hc) < 1e-14
    assert o.is_pair_structured(P)
    assert _rel(o.hessian_pairs(P, W), o.hessian_kron(P, W)) < 1e-14


def test_sym_kron_lemma():
    """Lemma sym_kron: A^T (X kron Y) A = A^T (Y kron X) A for any, even nonsymmetric, X, Y."""
    P = o.Problem.from_data(si.random_general(6, 5, 3, 8))
    rng = np.random.default_rng(1)
    X = rng.standard_normal((6, 6))
    Y = rng.standard_normal((6, 6))
    A = P.A_matrix()
    assert _rel(A.T @ np.kron(X, Y) @ A, A.T @ np.kron(Y, X) @ A) < 1e-13


def test_hessian_spd():
    """H is symmetric positive definite for W > 0 and linearly independent A_i."""
    P = _mc(6, 6, 2, 20, 4)
    H = o.hessian_entries(P, si.random_spd(P.n, 2, cond=100.0))
    assert np.allclose(H, H.T, atol=0, rtol=1e-14)
    assert np.linalg.eigvalsh(H)[0] > 0


# --------------------------------------------------------------------------
# NT scaling
# --------------------------------------------------------------------------

def test_nt_scaling_defining_property():
    """W S W = X with W positive definite (NT scaling, Section II-C)."""
    X = si.random_spd(12, 1, cond=1e4)
    S = si.random_spd(12, 2, cond=1e3)
    W = o.nt_scaling(X, S)
    assert _rel(W @ S @ W, X) < 1e-10
    assert np.linalg.eigvalsh(W)[0] > 0


def test_nt_scaling_commuting_closed_form():
    """For commuting (diagonal) X, S the NT matrix is diag(sqrt(x_i / s_i))."""
    x = np.linspace(0.5, 3.0, 7)
    s = np.linspace(2.0, 0.1, 7)
    W = o.nt_scaling(np.diag(x), np.diag(s))
    assert _rel(W, np.diag(np.sqrt(x / s))) < 1e-14


# --------------------------------------------------------------------------
# Split of W and the preconditioner (Section III)
# --------------------------------------------------------------------------

def _ipm_like_W(n, k, mu, seed):
    """W with k eigenvalues ~1/mu above n-k eigenvalues in [1, 3] (Prop. Weig)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.concatenate([rng.uniform(1.0, 3.0, n - k), rng.uniform(1.0, 2.0, k) / mu])
    return (Q * ev) @ Q.T


@pytest.mark.parametrize("z_kind", ["chol", "eig"])
def test_split_identities(z_kind):
    """eq. (Wsplit2): W = W0 + U U^T; eq. (hessExp2): H = H0 + UU UU^T for any valid Z."""
    P = _mc(4, 4, 2, 10, 6)
    W = _ipm_like_W(P.n, 2, 1e-3, 1)
    sp = o.split_W(W, 2, z_kind)
    assert _rel(sp.W0 + sp.U @ sp.U.T, W) < 1e-13
    assert _rel(sp.Z @ sp.Z.T, 2 * sp.W0 + sp.U @ sp.U.T) < 1e-12
    A = P.A_matrix()
    H0 = A.T @ np.kron(sp.W0, sp.W0) @ A
    UU = o.UU_kron(P, sp.U, sp.Z)
    assert _rel(H0 + UU @ UU.T, o.hessian_kron(P, W)) < 1e-11
    # tau lies in the admissible range of eq. (Wsplit2)
    lam_s = sp.lam[: P.n - 2]
    assert lam_s.min() <= sp.tau < lam_s.max()


def test_UU_matvec_matches_kron_and_is_adjoint():
    """eq. (Umv): columns from A_i.(Z X U^T) equal A^T (U kron Z); UU and UU^T are adjoint."""
    P = o.Problem.from_data(si.random_general(6, 6, 2, 9))
    rng = np.random.default_rng(2)
    U = rng.standard_normal((6, 2))
    Z = rng.standard_normal((6, 6))
    assert _rel(o.UU_explicit(P, U, Z), o.UU_kron(P, U, Z)) < 1e-14
    X = rng.standard_normal((6, 2))
    y = rng.standard_normal(P.m)
    lhs = o.UU_matvec(P, U, Z, X) @ y
    rhs = np.sum(X * o.UU_rmatvec(P, U, Z, y))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_wsmf_inverse():
    """eq. (wsmf): (tau I + U U^T)^{-1} = tau^{-1} I - tau^{-1} U S^{-1} U^T, S = tau I + U^T U."""
    rng = np.random.default_rng(3)
    U = rng.standard_normal((9, 3))
    tau = 0.7
    Ss = tau * np.eye(3) + U.T @ U
    inv = np.eye(9) / tau - U @ np.linalg.solve(Ss, U.T) / tau
    assert _rel(inv, np.linalg.inv(tau * np.eye(9) + U @ U.T)) < 1e-13


@pytest.mark.parametrize("z_kind", ["chol", "eig"])
def test_smw_apply_equals_dense_solve(z_kind):
    """eq. (SMW2) applied step by step equals a dense solve with eq. (AtIUUtAt)."""
    P = _mc(5, 5, 2, 15, 7)
    W = _ipm_like_W(P.n, 2, 1e-4, 3)
    pc = o.precond_build(P, W, 2, z_kind)
    Ht = pc.tau ** 2 * o.gram_AtA(P) + o.UU_kron(P, pc.U, pc.Z) @ o.UU_kron(P, pc.U, pc.Z).T
    r = si.random_vec(P.m, 1)
    assert _rel(o.precond_apply(P, pc, r), np.linalg.solve(Ht, r)) < 1e-9
    assert _rel(o.precond_dense(P, pc), Ht) < 1e-12


def test_core_needs_tau_squared():
    """Reading of Algorithm 1 step 2: with tau I instead of tau^2 I the SMW apply does not invert Ht."""
    P = _mc(5, 5, 2, 15, 7)
    W = _ipm_like_W(P.n, 2, 1e-2, 3)
    pc = o.precond_build(P, W, 2)
    r = si.random_vec(P.m, 1)
    Ht = o.precond_dense(P, pc)
    z = o.precond_apply(P, pc, r)
    assert _rel(Ht @ z, r) < 1e-10
    bad = o.Precond(tau=pc.tau, U=pc.U, Z=pc.Z, ginv=pc.ginv,
                    Sc=None, Lc=np.linalg.cholesky(pc.Sc - (pc.tau ** 2 - pc.tau) * np.eye(pc.Sc.shape[0])))
    assert _rel(Ht @ o.precond_apply(P, bad, r), r) > 1e-3


def test_preconditioner_independent_of_Z():
    """Ht^{-1} r does not depend on which factor Z of 2 W0 + U U^T is used."""
    P = _mc(4, 5, 1, 12, 8)
    W = _ipm_like_W(P.n, 1, 1e-5, 4)
    r = si.random_vec(P.m, 2)
    z1 = o.precond_apply(P, o.precond_build(P, W, 1, "chol"), r)
    z2 = o.precond_apply(P, o.precond_build(P, W, 1, "eig"), r)
    assert _rel(z1, z2) < 1e-8


def test_exact_low_rank_W_gives_exact_preconditioner():
    """W = tau I + U U^T exactly makes W0 = tau I, so Ht = H and PCG stops after one step."""
    P = _mc(5, 5, 2, 14, 9)
    rng = np.random.default_rng(5)
    U0 = rng.standard_normal((P.n, 2)) * 3.0
    W = 0.8 * np.eye(P.n) + U0 @ U0.T
    pc = o.precond_build(P, W, 2)
    H = o.hessian_entries(P, W)
    assert _rel(o.precond_dense(P, pc), H) < 1e-11
    r = si.random_vec(P.m, 3)
    res = o.pcg(lambda v: H @ v, lambda v: o.precond_apply(P, pc, v), r, rtol=1e-8)
    assert res.iters == 1


@pytest.mark.parametrize("mu", [1e-2, 1e-5])
def test_lemma_bounds(mu):
    """Lemma kappaW: kappa(W, Wt) <= kappa(W0); Lemma Htilde: kappa(H, Ht) <= kappa(W0)^2."""
    P = _mc(5, 5, 2, 16, 10)
    W = _ipm_like_W(P.n, 2, mu, 6)
    sp = o.split_W(W, 2)
    k0 = np.linalg.cond(sp.W0)
    Wt = sp.tau * np.eye(P.n) + sp.U @ sp.U.T
    ev = sla.eigh(W, Wt, eigvals_only=True)
    assert ev[-1] / ev[0] <= k0 * (1 + 1e-8)
    pc = o.precond_build(P, W, 2)
    evh = sla.eigh(o.hessian_entries(P, W), o.precond_dense(P, pc), eigvals_only=True)
    assert evh[-1] / evh[0] <= k0 ** 2 * (1 + 1e-8)
    # and the unpreconditioned Hessian is far worse conditioned
    assert np.linalg.cond(o.hessian_entries(P, W)) > 10 * k0 ** 2


def test_hat_smw_apply_equals_definition():
    """eq. (sparse_prec): the eq. (SMW2) apply with Z = sqrt(2 tau) I inverts
    A^T (tau^2 I + 2 tau U U^T kron I) A built with an explicit Kronecker product."""
    P = _mc(5, 5, 2, 15, 7)
    W = _ipm_like_W(P.n, 2, 1e-4, 3)
    pc = o.precond_hat_build(P, W, 2)
    Hh = o.precond_hat_dense(P, W, 2)
    assert _rel(o.precond_dense(P, pc), Hh) < 1e-12
    r = si.random_vec(P.m, 1)
    assert _rel(o.precond_apply(P, pc, r), np.linalg.solve(Hh, r)) < 1e-9


def test_hat_general_constraints():
    """Same identity for constraints with several entries each, and for diagonal ones."""
    for d in (si.random_general(10, 12, 3, 31), si.unit_diag_instance(8)):
        P = o.Problem.from_data(d)
        W = si.random_spd(P.n, 5, cond=1e3)
        pc = o.precond_hat_build(P, W, 2)
        Hh = o.precond_hat_dense(P, W, 2)
        r = si.random_vec(P.m, 2)
        assert _rel(o.precond_apply(P, pc, r), np.linalg.solve(Hh, r)) < 1e-9


def test_hat_exact_up_to_rank_k2_when_W0_is_tau_I():
    """W = tau I + U U^T: H - Hhat = A^T (U U^T kron U U^T) A (sym kron lemma), of rank
    <= k(k+1)/2 for symmetric A_i, so PCG with Hhat stops within k(k+1)/2 + 1 steps.
    With tau instead of 2 tau in eq. (sparse_prec) the difference has full rank."""
    P = _mc(6, 6, 2, 24, 9)
    rng = np.random.default_rng(5)
    U0 = rng.standard_normal((P.n, 2)) * 3.0
    W = 0.8 * np.eye(P.n) + U0 @ U0.T
    H = o.hessian_entries(P, W)
    Hh = o.precond_hat_dense(P, W, 2)
    s = np.linalg.svd(H - Hh, compute_uv=False)
    assert s[3] <= 1e-10 * s[0]
    r = si.random_vec(P.m, 3)
    pc = o.precond_hat_build(P, W, 2)
    res = o.pcg(lambda v: H @ v, lambda v: o.precond_apply(P, pc, v), r, rtol=1e-10)
    assert res.converged and res.iters <= 4
    A = P.A_matrix()
    bad = A.T @ (0.64 * np.eye(P.n ** 2) + 0.8 * np.kron(U0 @ U0.T, np.eye(P.n))) @ A
    sb = np.linalg.svd(H - bad, compute_uv=False)
    assert sb[3] > 1e-3 * sb[0]


@pytest.mark.parametrize("mu", [1e-2, 1e-5])
def test_lemma_aug_prec(mu):
    """Lemma aug_prec: apart from the k^2 largest, the eigenvalues of Hhat^{-1} H lie
    within a factor kappa(W0)^2 of the smallest."""
    P = _mc(5, 5, 2, 16, 10)
    W = _ipm_like_W(P.n, 2, mu, 6)
    sp = o.split_W(W, 2)
    k0 = np.linalg.cond(sp.W0)
    ev = sla.eigh(o.hessian_entries(P, W), o.precond_hat_dense(P, W, 2), eigvals_only=True)
    assert ev[:-4].max() / ev[0] <= k0 ** 2 * (1 + 1e-8)
    # while the Alg. 1 core is far worse conditioned than the Hhat core
    c1 = np.linalg.cond(o.precond_build(P, W, 2).Sc)
    c2 = np.linalg.cond(o.precond_hat_build(P, W, 2).Sc)
    assert c2 < c1


# --------------------------------------------------------------------------
# PCG
# --------------------------------------------------------------------------

def test_pcg_solves_and_respects_chebyshev_bound():
    """PCG reaches the residual tolerance; the A-norm error obeys eq. (cgcheb) with j = 1."""
    P = _mc(6, 6, 2, 24, 12)
    W = _ipm_like_W(P.n, 2, 1e-4, 7)
    H = o.hessian_entries(P, W)
    pc = o.precond_build(P, W, 2)
    r = si.random_vec(P.m, 4)
    xs = np.linalg.solve(H, r)
    res = o.pcg(lambda v: H @ v, lambda v: o.precond_apply(P, pc, v), r, rtol=1e-10)
    assert res.converged
    assert res.relres <= 1e-10
    # the true residual trails the recursively updated one by about kappa(H) eps
    assert np.linalg.norm(H @ res.x - r) <= 1e-8 * np.linalg.norm(r)
    assert _rel(res.x, xs) < 1e-6
    ev = sla.eigh(H, o.precond_dense(P, pc), eigvals_only=True)
    kap = ev[-1] / ev[0]
    rate = (math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)
    # error after i steps, measured in the H-norm, against 2 sqrt(kappa)... bound (Prop. CG/PCG)
    for i in (1, 2, 3):
        ri = o.pcg(lambda v: H @ v, lambda v: o.precond_apply(P, pc, v), r, rtol=0.0, maxit=i)
        e = ri.x - xs
        assert math.sqrt(e @ H @ e) <= 2 * rate ** i * math.sqrt(xs @ H @ xs) * (1 + 1e-8)


def test_pcg_identity_preconditioner_is_cg_and_exact_in_m_steps():
    """With no preconditioner PCG is CG, which is exact after m steps on a tiny system."""
    rng = np.random.default_rng(0)
    A = si.random_spd(8, 3, cond=10.0)
    b = rng.standard_normal(8)
    res = o.pcg(lambda v: A @ v, lambda v: v, b, rtol=1e-12, maxit=8)
    assert res.converged and res.iters <= 8
    assert _rel(res.x, np.linalg.solve(A, b)) < 1e-10


# --------------------------------------------------------------------------
# Interior-point method: closed forms, brute force, invariants
# --------------------------------------------------------------------------

def test_ipm_unit_diagonal_analytic_center():
    """min tr X s.t. X_ii = 1: optimal value n, analytic centre X = I, y = 1, S = 0."""
    P = o.Problem.from_data(si.unit_diag_instance(6))
    res = o.ipm_solve(P)
    assert res.converged
    assert abs(res.obj_p - 6) < 1e-5
    assert np.abs(res.X - np.eye(6)).max() < 1e-5
    assert np.abs(res.y - 1).max() < 1e-5
    assert np.abs(res.S).max() < 1e-5


def test_ipm_trace_one_gives_lambda_min():
    """min C.X s.t. tr X = 1 has value lambda_min(C) attained at X = v v^T."""
    d = si.trace_one_instance(7, 3)
    P = o.Problem.from_data(d)
    res = o.ipm_solve(P, o.IPMParams(gap_tol=1e-9, infeas_tol=1e-9))
    lam, V = np.linalg.eigh(d.meta["C"])
    assert abs(res.obj_p - lam[0]) < 1e-7 * (1 + abs(lam[0]))
    v = V[:, 0]
    assert np.abs(res.X - np.outer(v, v)).max() < 1e-4


def test_ipm_maxcut_bipartite():
    """min A_G.X s.t. X_ii = 1 on a connected bipartite graph: X = z z^T, value -2|E|."""
    d = si.maxcut_bipartite_instance(4, 5, 1, extra_edges=6)
    P = o.Problem.from_data(d)
    res = o.ipm_solve(P, o.IPMParams(gap_tol=1e-8, infeas_tol=1e-8))
    z = d.meta["z"]
    assert abs(res.obj_p + 2 * d.meta["n_edges"]) < 1e-5 * 2 * d.meta["n_edges"]
    assert np.abs(res.X - np.outer(z, z)).max() < 1e-3


def test_ipm_scalar_problem():
    """n = 1: min c x s.t. a x = b gives x = b / a and y = c / a."""
    P = o.Problem.from_data(si.scalar_instance(2.0, 3.0, 5.0))
    res = o.ipm_solve(P, o.IPMParams(gap_tol=1e-9, infeas_tol=1e-9))
    assert abs(res.X[0, 0] - 1.5) < 1e-7
    assert abs(res.y[0] - 2.5) < 1e-6


def _nuclear(M):
    return np.linalg.svd(M, compute_uv=False).sum()


def test_ipm_mc_brute_force_one_missing_entry():
    """p = q = 2 with one unobserved entry: the SDP value equals min_t ||[[m11, m12],[m21, t]]||_*."""
    Mfull = np.array([[1.3, -0.4], [0.7, 0.0]])
    rows = np.array([0, 0, 1])
    cols = np.array([0, 1, 0])
    d = si.SDPData(n=4, m=3, Ci=np.arange(4, dtype=np.int32), Cj=np.arange(4, dtype=np.int32),
                   Cv=np.full(4, 0.5), Ak=np.arange(3, dtype=np.int32), Ai=rows.astype(np.int32),
                   Aj=(2 + cols).astype(np.int32), Av=np.full(3, 0.5), b=Mfull[rows, cols], k=1,
                   meta=dict(kind="mc", p=2, q=2))
    P = o.Problem.from_data(d)
    res = o.ipm_solve(P, o.IPMParams(gap_tol=1e-9, infeas_tol=1e-9))
    f = lambda t: _nuclear(np.array([[1.3, -0.4], [0.7, t]]))
    grid = np.linspace(-5, 5, 20001)
    t0 = grid[np.argmin([f(t) for t in grid])]
    a, b = t0 - 1e-3, t0 + 1e-3
    g = (math.sqrt(5) - 1) / 2
    for _ in range(80):
        c1, c2 = b - g * (b - a), a + g * (b - a)
        if f(c1) < f(c2):
            b = c2
        else:
            a = c1
    tstar = (a + b) / 2
    assert abs(res.obj_p - f(tstar)) < 1e-7
    assert abs(o.mc_recovered(P, res.X)[1, 1] - tstar) < 1e-4


def test_ipm_mc_exact_recovery_C1():
    """Noiseless planted rank-1 M with m = 200 >> dof: Z = M and value ||M||_* (Section V-A)."""
    d = si.config_instance("C1")
    P = o.Problem.from_data(d)
    res = o.ipm_solve(P)
    assert res.converged and res.relgap <= 1e-6
    M = d.meta["M"]
    assert _rel(o.mc_recovered(P, res.X), M) <= 1e-5
    assert abs(res.obj_p - _nuclear(M)) <= 1e-5 * _nuclear(M)


def test_ipm_gap_identity_along_iterates():
    """C.X - b^T y = X.S + Rd.X - y^T Rp at every iterate (Section II duality-gap identity)."""
    P = _mc(6, 7, 2, 30, 13)
    X, y, S = o.start_point(P)
    for it in range(4):
        Rp, Rd, cx, by, *_ = o.residuals(P, X, y, S)
        assert abs((cx - by) - (np.sum(X * S) + np.sum(Rd * X) - y @ Rp)) < 1e-9 * (1 + abs(cx))
        res = o.ipm_solve(P, o.IPMParams(maxit=it + 1))
        X, y, S = res.X, res.y, res.S


def test_ipm_general_sparse_kkt():
    """Random sparse SDP with diagonal A^T A: the final point passes the KKT certificate."""
    P = o.Problem.from_data(si.random_general(10, 12, 2, 21))
    res = o.ipm_solve(P)
    assert res.converged
    cert = o.kkt_certificate(P, res.X, res.y, res.S)
    assert cert["pinf"] < 1e-6 and cert["dinf"] < 1e-6 and cert["relgap"] < 1e-6
    assert cert["lmin_X"] > -1e-8 and cert["lmin_S"] > -1e-8


def test_max_step_is_boundary():
    """max_step returns the alpha where X + alpha dX first becomes singular."""
    X = si.random_spd(6, 1)
    dX = si.random_sym(6, 2)
    a = o.max_step(X, dX)
    assert np.linalg.eigvalsh(X + 0.999 * a * dX)[0] > 0
    assert np.linalg.eigvalsh(X + 1.001 * a * dX)[0] < 0


# ---------------------------------------------------------------------------
# Adaptive rank k~ (Section V, implementation notes; Prop. Weig)
# ---------------------------------------------------------------------------
def _with_spectrum(lam_desc, seed=21):
    n = len(lam_desc)
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return (Q * np.asarray(lam_desc, dtype=float)) @ Q.T


def test_rank_estimate_rule_on_known_spectra():
    # the largest index with a ratio of at least eta wins, not the first or the biggest ratio
    W = _with_spectrum([100.0, 90.0, 1.0, 0.9, 0.8, 0.7])
    assert o.rank_estimate(W, kmax=4, eta=10.0) == 2
    W = _with_spectrum([1000.0, 100.0, 10.0, 1.0, 0.5])
    assert o.rank_estimate(W, kmax=4, eta=5.0) == 3
    assert o.rank_estimate(W, kmax=2, eta=5.0) == 2       # kmax caps the index
    assert o.rank_estimate(W, kmax=0, eta=5.0) == 0
    # a flat spectrum has no gap: k~ = 0 (lambda_0 = +inf is the only qualifying index)
    assert o.rank_estimate(3.0 * np.eye(6), kmax=5, eta=2.0) == 0
    # kmax beyond n - 1 is harmless
    W = _with_spectrum([8.0, 1.0, 1.0])
    assert o.rank_estimate(W, kmax=10, eta=4.0) == 1


def test_rank_estimate_equality_counts():
    # lambda_i = eta * lambda_{i+1} exactly qualifies (>=); eigenvalues exact in binary
    W = np.diag([16.0, 4.0, 1.0, 1.0])
    assert o.rank_estimate(W, kmax=3, eta=4.0) == 2
    assert o.rank_estimate(W, kmax=3, eta=4.5) == 0


@pytest.mark.parametrize("spec,r", [(dict(p=20, q=20, r=1, m=200, seed=1), 1),
                                    (dict(p=20, q=20, r=2, m=300, seed=13), 2)])
def test_rank_estimate_finds_rank_at_the_optimum(spec, r):
    """Prop. Weig: at the optimum of an exactly recovered completion, W has r eigenvalues
    of order one and the rest of order mu, so k~ = r = rank X* (and the planted rank)."""
    d = si.mc_instance(**spec)
    P = o.Problem.from_data(d)
    res = o.ipm_solve(P)
    assert res.converged
    assert _rel(o.mc_recovered(P, res.X), d.meta["M"]) <= 1e-5
    W = o.nt_scaling(res.X, res.S)
    assert o.rank_estimate(W, kmax=5, eta=10.0) == r
    # at the start point W is a multiple of I: no gap yet
    X0, _, S0 = o.start_point(P)
    assert o.rank_estimate(o.nt_scaling(X0, S0), kmax=5, eta=10.0) == 0


def test_rank_estimate_tracks_rank_of_X_when_recovery_fails():
    """Too few samples: the SDP optimum has rank above the planted r; k~ follows rank X*,
    the quantity Prop. Weig is about, not the planted rank."""
    d = si.mc_instance(16, 16, 3, 180, 12)
    P = o.Problem.from_data(d)
    res = o.ipm_solve(P)
    assert res.converged
    lx = np.sort(np.linalg.eigvalsh(res.X))[::-1]
    rank_x = int(np.sum(lx >= 1e-3 * lx[0]))
    assert rank_x > 3
    W = o.nt_scaling(res.X, res.S)
    assert o.rank_estimate(W, kmax=6, eta=10.0) == rank_x


def test_aug_prec_ldl_equals_hhat_and_its_core():
    """eq. (aug_prec): the augmented system of Section V, factored by LDL^T without
    pivoting, solves Hhat x = b (against the explicit Kronecker form of eq.
    sparse_prec), and eliminating its first block (tau^2 A^T A, diagonal under
    Assumption 2) leaves -1/2 of the core tau^2 I + 2 tau K that the SMW apply
    factors -- the paper's remark that elimination without pivoting on the
    augmented system takes the same steps as the SMW formula."""
    d = si.mc_instance(6, 7, 2, 30, 3)
    P = o.Problem.from_data(d)
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((d.n, d.n)))
    W = (Q * np.concatenate([rng.uniform(1, 3, d.n - 2), [50.0, 40.0]])) @ Q.T
    b = rng.standard_normal(d.m)
    x = o.aug_prec_solve(P, W, 2, b)
    Hh = o.precond_hat_dense(P, W, 2)
    assert np.linalg.norm(Hh @ x - b) <= 1e-12 * np.linalg.norm(b)
    K = o.aug_prec_matrix(P, W, 2)
    m = d.m
    schur = K[m:, m:] - K[m:, :m] @ np.linalg.solve(K[:m, :m], K[:m, m:])
    pc = o.precond_hat_build(P, W, 2)
    assert np.allclose(schur, -0.5 * pc.Sc, rtol=1e-12, atol=1e-12 * np.abs(pc.Sc).max())
    # a wrong scaling of the off-diagonal blocks breaks the identity
    K2 = K.copy()
    K2[m:, :m] *= 2.0
    K2[:m, m:] *= 2.0
    x2 = o.ldl_nopivot_solve(K2, np.concatenate([b, np.zeros(K.shape[0] - m)]))[:m]
    assert np.linalg.norm(Hh @ x2 - b) > 1e-3 * np.linalg.norm(b)
