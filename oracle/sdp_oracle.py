"""Plain FP64 CPU oracle for the modified interior-point method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library: it reads problems from the seeded generator ``sdp_inputs``
and otherwise uses NumPy/SciPy only.

Every function restates a definition or an algorithm step of Zhang & Lavaei,
"Modified Interior-Point Method for Large-and-Sparse Low-Rank Semidefinite
Programs" (arXiv 1703.10973), in the paper's notation:

* eq. (SDP)/(SDD): min C.X s.t. A_i.X = b_i, X psd / max b^T y s.t. sum y_i A_i + S = C.
* eq. (hesseqn2)/(hesseqn1): (H v)_i = A_i . (W (sum_j v_j A_j) W),  H = A^T (W kron W) A.
* eq. (Wsplit1)/(Wsplit2): W = W0 + U U^T from an eigendecomposition of W.
* eq. (hessExp2): H = H0 + UU UU^T with UU = A^T (U kron Z), Z Z^T = 2 W0 + U U^T.
* eq. (AtIUUtAt)/(SMW2): preconditioner Ht = tau^2 A^T A + UU UU^T and its inverse.
* eq. (Umv): UU x = [A_i . (Z X U^T)]_i,  UU^T y = Z^T (sum y_i A_i) U.
* Algorithm 1: formation, factorisation, PCG solution.
* eq. (sparse_prec), Lemma aug_prec, eq. (aug_prec): the Section V preconditioner Hhat
  and its augmented system, solved by LDL^T without pivoting.
* Section II / II-B: NT scaling (X = W S W) and the direct method (form H, Cholesky).

Readings where the paper is silent or inconsistent (each listed in the design notes):
* The core of eq. (SMW2) is S = tau^2 I + UU^T (A^T A)^{-1} UU (Algorithm 1 step 2
  prints tau I; the derivation of eq. (SMW2) needs tau^2).
* Vectorisation is row-major (the paper's identity vec(A X B^T) = (A kron B) vec X);
  the columns of UU are indexed (l, c) -> l*n + c for the k x n matrix X^T of eq. (Umv).
* The outer method is an infeasible NT predictor-corrector; the paper fixes only
  "NT-scaled path-following".  Start point X = S = xi I, y = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

# ---------------------------------------------------------------------------
# Problem data: dense symmetric matrices from triplets (eq. SDP).
# ---------------------------------------------------------------------------


def sym_from_triplets(n, i, j, v):
    """Dense symmetric matrix with M[i, j] = M[j, i] = v (duplicates add)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    v = np.asarray(v, dtype=np.float64)
    lo = np.minimum(i, j)
    hi = np.maximum(i, j)
    M = np.zeros((n, n))
    np.add.at(M, (lo, hi), v)
    off = lo != hi
    np.add.at(M, (hi[off], lo[off]), v[off])
    return M


@dataclass
class Problem:
    """The oracle's own copy of an SDP (eq. SDP): dense C, sparse A_i, b."""

    n: int
    m: int
    C: np.ndarray
    b: np.ndarray
    # sparse constraint data, one row per stored upper-triangular entry
    Ak: np.ndarray
    Ai: np.ndarray
    Aj: np.ndarray
    Av: np.ndarray
    k: int
    meta: dict = field(default_factory=dict)

    @classmethod
    def from_data(cls, d):
        lo = np.minimum(d.Ai, d.Aj).astype(np.int64)
        hi = np.maximum(d.Ai, d.Aj).astype(np.int64)
        return cls(n=d.n, m=d.m, C=sym_from_triplets(d.n, d.Ci, d.Cj, d.Cv),
                   b=np.asarray(d.b, dtype=np.float64).copy(),
                   Ak=np.asarray(d.Ak, dtype=np.int64), Ai=lo, Aj=hi,
                   Av=np.asarray(d.Av, dtype=np.float64), k=int(d.k), meta=dict(d.meta))

    def A_dense(self, i):
        sel = self.Ak == i
        return sym_from_triplets(self.n, self.Ai[sel], self.Aj[sel], self.Av[sel])

    def A_list(self):
        return [self.A_dense(i) for i in range(self.m)]

    def A_matrix(self):
        """The n^2 x m matrix A = [vec A_1, ..., vec A_m] (Assumption 2)."""
        return np.stack([a.reshape(-1) for a in self.A_list()], axis=1)


def op_A(P: Problem, X):
    """(A X)_i = A_i . X = tr(A_i^T X)  (eq. SDP constraints); X need not be symmetric."""
    both = X[P.Ai, P.Aj] + X[P.Aj, P.Ai]
    both = np.where(P.Ai == P.Aj, 0.5 * both, both)
    out = np.zeros(P.m)
    np.add.at(out, P.Ak, P.Av * both)
    return out


def op_At(P: Problem, y):
    """A^T y = sum_i y_i A_i  (eq. SDD)."""
    return sym_from_triplets(P.n, P.Ai, P.Aj, np.asarray(y)[P.Ak] * P.Av)


def gram_AtA(P: Problem):
    """G = A^T A with G_ij = A_i . A_j (dense m x m; small problems only)."""
    As = P.A_list()
    G = np.empty((P.m, P.m))
    for i in range(P.m):
        for j in range(P.m):
            G[i, j] = np.sum(As[i] * As[j])
    return G


def gram_AtA_diag(P: Problem):
    """Diagonal of A^T A, i.e. ||A_i||_F^2, from the stored entries."""
    mult = np.where(P.Ai == P.Aj, 1.0, 2.0)
    out = np.zeros(P.m)
    np.add.at(out, P.Ak, mult * P.Av ** 2)
    return out


# ---------------------------------------------------------------------------
# Hessian (eq. hesseqn2 / hesseqn1).
# ---------------------------------------------------------------------------


def hessian_kron(P: Problem, W):
    """H = A^T (W kron W) A with an explicit n^2 x n^2 Kronecker product (tiny n)."""
    A = P.A_matrix()
    return A.T @ np.kron(W, W) @ A


def hessian_trace(P: Problem, W):
    """H_ij = tr(A_i W A_j W), the entrywise form of eq. (hesseqn2)."""
    As = P.A_list()
    WA = [W @ a for a in As]
    H = np.empty((P.m, P.m))
    for i in range(P.m):
        for j in range(P.m):
            H[i, j] = np.sum(WA[i] * WA[j].T)
    return H


def _expanded_entries(P: Problem):
    """All nonzeros (constraint, row, col, value) of every A_i, both triangles."""
    off = P.Ai != P.Aj
    k = np.concatenate([P.Ak, P.Ak[off]])
    a = np.concatenate([P.Ai, P.Aj[off]])
    b = np.concatenate([P.Aj, P.Ai[off]])
    v = np.concatenate([P.Av, P.Av[off]])
    return k, a, b, v


def hessian_entries(P: Problem, W, chunk=2048):
    """H_ij = sum_{(a,b) in A_i} sum_{(c,d) in A_j} (A_i)_ab W_bc (A_j)_cd W_da.

    This is tr(A_i W A_j W) summed over the nonzeros of A_i and A_j, so it costs
    O(nnz^2) instead of O(m^2 n^3); used for every problem size the oracle runs.
    """
    import scipy.sparse as sp

    k, a, b, v = _expanded_entries(P)
    E = k.shape[0]
    inc = sp.csr_matrix((np.ones(E), (k, np.arange(E))), shape=(P.m, E))   # constraint <- entry
    H = np.zeros((P.m, P.m))
    for s in range(0, E, chunk):
        t = min(E, s + chunk)
        # contrib[e, f] = v_e v_f W[b_e, a_f] W[b_f, a_e]   (W symmetric)
        contrib = (v[s:t, None] * v[None, :]) * W[np.ix_(b[s:t], a)] * W[np.ix_(a[s:t], b)]
        R = inc @ contrib.T                      # m x (t-s): sum over the entries f of A_j
        H += inc[:, s:t] @ R.T                   # sum over the entries e of A_i
    return H


def hessian_pairs(P: Problem, W):
    """Closed form of eq. (hesseqn2) when every A_i is one symmetric off-diagonal pair.

    With A_i = a_i (e_p e_q^T + e_q e_p^T), tr(A_i W A_j W) expands into four
    terms, two by two equal because W is symmetric:
    H_ij = 2 a_i a_j (W_pp' W_qq' + W_pq' W_qp').
    """
    p, q, a = P.Ai, P.Aj, P.Av
    H = W[np.ix_(p, p)] * W[np.ix_(q, q)]
    H += W[np.ix_(p, q)] * W[np.ix_(q, p)]
    H *= 2.0 * np.outer(a, a)
    return H


def is_pair_structured(P: Problem):
    """True when constraint i is exactly one stored off-diagonal entry, in order."""
    return (P.Ak.shape[0] == P.m and np.array_equal(P.Ak, np.arange(P.m))
            and bool(np.all(P.Ai != P.Aj)))


def hessian_auto(P: Problem, W):
    """The explicit Hessian by the closed form when it applies, else by the entry sum."""
    return hessian_pairs(P, W) if is_pair_structured(P) else hessian_entries(P, W)


def hessian_matvec(P: Problem, W, v):
    """(H v)_i = A_i . [W (sum_j v_j A_j) W]  (eq. hesseqn2, matrix-free)."""
    return op_A(P, W @ op_At(P, v) @ W)


# ---------------------------------------------------------------------------
# NT scaling (Section II-C): W is the unique positive definite matrix with X = W S W.
# ---------------------------------------------------------------------------


def nt_scaling(X, S):
    """W = L Q Lambda^{-1/2} Q^T L^T with X = L L^T and L^T S L = Q Lambda Q^T.

    Then W S W = L Q Lambda^{-1/2} (Q^T L^T S L Q) Lambda^{-1/2} Q^T L^T = L L^T = X.
    """
    L = np.linalg.cholesky(X)
    lam, Q = np.linalg.eigh(L.T @ S @ L)
    G = L @ Q
    W = (G * lam ** -0.5) @ G.T
    return (W + W.T) / 2.0


# ---------------------------------------------------------------------------
# Splitting of W and the preconditioner (Section III, Algorithm 1).
# ---------------------------------------------------------------------------


@dataclass
class Split:
    tau: float
    lam: np.ndarray      # all eigenvalues of W, ascending
    V: np.ndarray        # eigenvectors (columns), same order
    U: np.ndarray        # n x k
    W0: np.ndarray
    Z: np.ndarray        # Z Z^T = 2 W0 + U U^T


def split_W(W, k, z_kind="chol"):
    """Algorithm 1 step 1: eig(W), tau = lambda_min(W), eq. (Wsplit2), and Z.

    eq. (Wsplit2): W0 = V diag(Lambda_s, tau I) V^T,  U U^T = V_l (Lambda_l - tau I) V_l^T,
    so U = V_l (Lambda_l - tau I)^{1/2}.  Z is any factor of 2 W0 + U U^T
    (eq. hessExp2); Algorithm 1 uses the Cholesky factor ("chol"); "eig" gives
    Z = V diag(sqrt(2 Lambda_s), sqrt(Lambda_l + tau)).
    """
    n = W.shape[0]
    lam, V = np.linalg.eigh(W)
    tau = lam[0]
    Vl = V[:, n - k:]
    Ll = lam[n - k:]
    U = Vl * np.sqrt(np.maximum(Ll - tau, 0.0))
    W0 = W - U @ U.T
    if z_kind == "chol":
        Z = np.linalg.cholesky(2.0 * W0 + U @ U.T)
    elif z_kind == "eig":
        d = np.concatenate([np.sqrt(2.0 * lam[: n - k]), np.sqrt(Ll + tau)])
        Z = V * d
    else:
        raise ValueError(z_kind)
    return Split(tau=float(tau), lam=lam, V=V, U=U, W0=W0, Z=Z)


def rank_estimate(W, kmax, eta):
    """Adaptive rank of the implementation notes of Section V:
    k~ = max{ i in {0, ..., kmax} : lambda_i(W) >= eta * lambda_{i+1}(W) },
    eigenvalues of W in decreasing order (lambda_1 the largest).

    Reading: lambda_0 = +inf, so i = 0 always qualifies and k~ >= 0; i is capped
    at n - 1 so that lambda_{i+1} exists.  Prop. Weig gives lambda_k / lambda_{k+1}
    in Theta(1/mu) for k = rank X*, so k~ tends to rank X* as mu -> 0.
    """
    lam = np.sort(np.linalg.eigvalsh(W))[::-1]
    best = 0
    for i in range(1, min(int(kmax), lam.size - 1) + 1):
        if lam[i - 1] >= eta * lam[i]:
            best = i
    return best


def UU_matvec(P: Problem, U, Z, X):
    """eq. (Umv a): (UU vec X)_i = A_i . (Z X U^T) for X in R^{n x k}."""
    return op_A(P, Z @ X @ U.T)


def UU_rmatvec(P: Problem, U, Z, y):
    """eq. (Umv b): UU^T y = Z^T (sum_i y_i A_i) U  in R^{n x k}."""
    return Z.T @ op_At(P, y) @ U


def UU_explicit(P: Problem, U, Z):
    """The m x nk matrix UU built column by column from eq. (Umv a).

    Column l*n + c is UU applied to X = e_c e_l^T (row-major vec of the k x n X^T).
    """
    n, k = U.shape
    out = np.empty((P.m, n * k))
    for l in range(k):
        for c in range(n):
            X = np.zeros((n, k))
            X[c, l] = 1.0
            out[:, l * n + c] = UU_matvec(P, U, Z, X)
    return out


def UU_kron(P: Problem, U, Z):
    """UU = A^T (U kron Z) with the explicit Kronecker product (tiny n)."""
    return P.A_matrix().T @ np.kron(U, Z)


@dataclass
class Precond:
    """Algorithm 1 steps 1-2: tau, U, Z, the core S and its Cholesky factor."""

    tau: float
    U: np.ndarray
    Z: np.ndarray
    ginv: np.ndarray     # diagonal of (A^T A)^{-1}
    Sc: np.ndarray       # core tau^2 I + UU^T G^{-1} UU  (nk x nk)
    Lc: np.ndarray       # its Cholesky factor


def precond_build(P: Problem, W, k, z_kind="chol"):
    """Algorithm 1 formation and factorisation (core with tau^2, eq. SMW2)."""
    sp = split_W(W, k, z_kind)
    g = gram_AtA_diag(P)
    ginv = 1.0 / g
    UU = UU_explicit(P, sp.U, sp.Z)
    n = W.shape[0]
    Sc = sp.tau ** 2 * np.eye(n * k) + UU.T @ (ginv[:, None] * UU)
    Lc = np.linalg.cholesky(Sc)
    return Precond(tau=sp.tau, U=sp.U, Z=sp.Z, ginv=ginv, Sc=Sc, Lc=Lc)


def precond_hat_build(P: Problem, W, k):
    """Section V, eq. (sparse_prec): Hhat = A^T (tau^2 I + 2 tau (U U^T kron I)) A.

    Hhat replaces Z Z^T = 2 W0 + U U^T of eq. (hessExp2) by 2 tau I, so it is the
    Algorithm 1 matrix tau^2 A^T A + UU UU^T with Z = sqrt(2 tau) I.  Its core
    tau^2 I + UU^T G^{-1} UU then has condition number of order lambda_max(W) / tau
    instead of (lambda_max(W) / tau)^2, which is what the section is after.  The
    same eq. (SMW2) apply (precond_apply) serves both; tau and U come from
    eq. (Wsplit2) as in Algorithm 1 step 1.
    """
    sp = split_W(W, k, "eig")
    n = W.shape[0]
    Z = math.sqrt(2.0 * sp.tau) * np.eye(n)
    ginv = 1.0 / gram_AtA_diag(P)
    UU = UU_explicit(P, sp.U, Z)
    Sc = sp.tau ** 2 * np.eye(n * k) + UU.T @ (ginv[:, None] * UU)
    Lc = np.linalg.cholesky(Sc)
    return Precond(tau=sp.tau, U=sp.U, Z=Z, ginv=ginv, Sc=Sc, Lc=Lc)


def precond_hat_dense(P: Problem, W, k):
    """eq. (sparse_prec) written out with an explicit n^2 x n^2 Kronecker product (tiny n)."""
    sp = split_W(W, k, "eig")
    n = W.shape[0]
    A = P.A_matrix()
    mid = sp.tau ** 2 * np.eye(n * n) + 2.0 * sp.tau * np.kron(sp.U @ sp.U.T, np.eye(n))
    return A.T @ mid @ A


def aug_prec_matrix(P: Problem, W, k):
    """The sparse augmented system of eq. (aug_prec) for Hhat (Section V):
        [[tau^2 A^T A,                 tau^{3/2} A^T (U kron I)],
         [tau^{3/2} (U kron I)^T A,   -tau^2 / 2 I_{nk}        ]],
    with A the n^2 x m matrix [vec A_1, ..., vec A_m] and (U kron I) the n^2 x nk
    matrix (row-major vec, columns (l, c) -> l n + c).  Eliminating its second block
    row leaves A^T (tau^2 I + 2 tau (U U^T kron I)) A = Hhat."""
    sp = split_W(W, k, "eig")
    n = W.shape[0]
    A = P.A_matrix()
    UI = np.kron(sp.U, np.eye(n))
    t = sp.tau
    top = np.hstack([t ** 2 * (A.T @ A), t ** 1.5 * (A.T @ UI)])
    bot = np.hstack([t ** 1.5 * (UI.T @ A), -0.5 * t ** 2 * np.eye(n * k)])
    return np.vstack([top, bot])


def ldl_nopivot_solve(K, b):
    """Solve K x = b by a plain LDL^T factorisation without pivoting (the recipe of
    Section V for eq. (aug_prec)): K = L D L^T with unit lower L and diagonal D,
    computed column by column; then forward, diagonal and backward substitution."""
    K = np.array(K, dtype=float)
    N = K.shape[0]
    L = np.eye(N)
    D = np.zeros(N)
    for j in range(N):
        D[j] = K[j, j] - np.dot(L[j, :j] ** 2, D[:j])
        for i in range(j + 1, N):
            L[i, j] = (K[i, j] - np.dot(L[i, :j] * L[j, :j], D[:j])) / D[j]
    y = np.zeros(N)
    for i in range(N):
        y[i] = b[i] - np.dot(L[i, :i], y[:i])
    z = y / D
    x = np.zeros(N)
    for i in range(N - 1, -1, -1):
        x[i] = z[i] - np.dot(L[i + 1:, i], x[i + 1:])
    return x


def aug_prec_solve(P: Problem, W, k, b):
    """Hhat^{-1} b through eq. (aug_prec): the first m entries of the solution of the
    augmented system with right-hand side [b; 0], by LDL^T without pivoting."""
    K = aug_prec_matrix(P, W, k)
    rhs = np.concatenate([np.asarray(b, dtype=float), np.zeros(K.shape[0] - P.m)])
    return ldl_nopivot_solve(K, rhs)[: P.m]


def precond_apply(P: Problem, pc: Precond, r):
    """eq. (SMW2): Ht^{-1} r = (tau^2 G)^{-1} (r - UU S^{-1} UU^T G^{-1} r).

    G^{-1} is diagonal (Assumption 2 with A^T A diagonal); S^{-1} = L^{-T} L^{-1}.
    """
    n, k = pc.U.shape
    t = pc.ginv * r
    u = UU_rmatvec(P, pc.U, pc.Z, t)                # n x k
    uvec = u.T.reshape(-1)                          # index l*n + c
    w = sla.solve_triangular(pc.Lc, uvec, lower=True)
    s = sla.solve_triangular(pc.Lc.T, w, lower=False)
    Smat = s.reshape(k, n).T                        # back to n x k
    return (pc.ginv / pc.tau ** 2) * (r - UU_matvec(P, pc.U, pc.Z, Smat))


def precond_dense(P: Problem, pc: Precond):
    """eq. (AtIUUtAt): Ht = tau^2 A^T A + UU UU^T as a dense m x m matrix."""
    UU = UU_explicit(P, pc.U, pc.Z)
    return pc.tau ** 2 * np.diag(1.0 / pc.ginv) + UU @ UU.T


# ---------------------------------------------------------------------------
# Preconditioned conjugate gradients (Prop. PCG; Algorithm 1 step 3).
# ---------------------------------------------------------------------------


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float
    converged: bool


def pcg(matvec, prec, r, rtol=1e-8, maxit=1000):
    """Textbook PCG from x0 = 0, stopping when ||r - H x|| <= rtol ||r||."""
    x = np.zeros_like(r)
    res = r.copy()
    nr0 = np.linalg.norm(r)
    if nr0 == 0.0:
        return PCGResult(x, 0, 0.0, True)
    z = prec(res)
    p = z.copy()
    rz = res @ z
    for it in range(1, maxit + 1):
        q = matvec(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        res = res - alpha * q
        rel = np.linalg.norm(res) / nr0
        if rel <= rtol:
            return PCGResult(x, it, rel, True)
        z = prec(res)
        rz_new = res @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return PCGResult(x, maxit, rel, False)


# ---------------------------------------------------------------------------
# Interior-point method: infeasible NT predictor-corrector whose Newton step
# solves H dy = r exactly by forming H and factoring it (Section II-B, direct method).
# ---------------------------------------------------------------------------


@dataclass
class IPMParams:
    gap_tol: float = 1e-6
    infeas_tol: float = 1e-6
    maxit: int = 100
    step_frac: float = 0.9


@dataclass
class IPMResult:
    X: np.ndarray
    y: np.ndarray
    S: np.ndarray
    obj_p: float
    obj_d: float
    relgap: float
    pinf: float
    dinf: float
    iters: int
    converged: bool
    log: list


def start_point(P: Problem):
    """X0 = S0 = xi I, y0 = 0 with xi = max(10, sqrt n, max_i sqrt n (1+|b_i|)/(1+||A_i||_F), (1+||C||_F)/sqrt n)."""
    n = P.n
    normA = np.sqrt(gram_AtA_diag(P))
    xi = max(10.0, math.sqrt(n),
             float(np.max(math.sqrt(n) * (1.0 + np.abs(P.b)) / (1.0 + normA))) if P.m else 0.0,
             (1.0 + np.linalg.norm(P.C)) / math.sqrt(n))
    return xi * np.eye(n), np.zeros(P.m), xi * np.eye(n)


def max_step(X, dX):
    """Largest alpha with X + alpha dX psd: 1 / max(0, -lambda_min(L^{-1} dX L^{-T})), X = L L^T."""
    L = np.linalg.cholesky(X)
    T = sla.solve_triangular(L, dX, lower=True)
    T = sla.solve_triangular(L, T.T, lower=True)
    lmin = np.linalg.eigvalsh((T + T.T) / 2.0)[0]
    return math.inf if lmin >= 0.0 else -1.0 / lmin


def residuals(P: Problem, X, y, S):
    Rp = P.b - op_A(P, X)
    Rd = P.C - S - op_At(P, y)
    cx = float(np.sum(P.C * X))
    by = float(P.b @ y)
    relgap = abs(cx - by) / (1.0 + abs(cx) + abs(by))
    pinf = np.linalg.norm(Rp) / (1.0 + np.linalg.norm(P.b))
    dinf = np.linalg.norm(Rd) / (1.0 + np.linalg.norm(P.C))
    return Rp, Rd, cx, by, relgap, pinf, dinf


def newton_direction(P: Problem, W, Hfactor, Rp, Rd, Rc):
    """Solve A(dX) = Rp, A^T dy + dS = Rd, dX + W dS W = Rc.

    Eliminating dX and dS gives eq. (hesseqn2) with right-hand side
    r = Rp - A(Rc) + A(W Rd W); then dS = Rd - A^T dy, dX = Rc - W dS W.
    """
    r = Rp - op_A(P, Rc) + op_A(P, W @ Rd @ W)
    dy = sla.cho_solve(Hfactor, r)
    dS = Rd - op_At(P, dy)
    dX = Rc - W @ dS @ W
    dX = (dX + dX.T) / 2.0
    return dX, dy, dS


def ipm_solve(P: Problem, prm: IPMParams | None = None, hessian=None):
    """Infeasible NT predictor-corrector; the Hessian is formed and Cholesky-factored."""
    prm = prm or IPMParams()
    hessian = hessian or hessian_auto
    X, y, S = start_point(P)
    n = P.n
    log = []
    converged = False
    for it in range(prm.maxit + 1):
        Rp, Rd, cx, by, relgap, pinf, dinf = residuals(P, X, y, S)
        mu = float(np.sum(X * S)) / n
        log.append(dict(it=it, mu=mu, obj_p=cx, obj_d=by, relgap=relgap, pinf=pinf, dinf=dinf))
        if relgap <= prm.gap_tol and pinf <= prm.infeas_tol and dinf <= prm.infeas_tol:
            converged = True
            break
        if it == prm.maxit:
            break
        W = nt_scaling(X, S)
        Hf = sla.cho_factor(hessian(P, W), lower=True)
        # predictor (sigma = 0): Rc = -X
        dX, dy, dS = newton_direction(P, W, Hf, Rp, Rd, -X)
        ap = min(1.0, prm.step_frac * max_step(X, dX))
        ad = min(1.0, prm.step_frac * max_step(S, dS))
        mu_aff = float(np.sum((X + ap * dX) * (S + ad * dS))) / n
        sigma = min(1.0, max(0.0, mu_aff / mu)) ** 3
        # corrector: Rc = sigma mu S^{-1} - X
        Sinv = np.linalg.inv(S)
        Rc = sigma * mu * (Sinv + Sinv.T) / 2.0 - X
        dX, dy, dS = newton_direction(P, W, Hf, Rp, Rd, Rc)
        ap = min(1.0, prm.step_frac * max_step(X, dX))
        ad = min(1.0, prm.step_frac * max_step(S, dS))
        X = X + ap * dX
        y = y + ad * dy
        S = S + ad * dS
        X = (X + X.T) / 2.0
        S = (S + S.T) / 2.0
        log[-1].update(alpha_p=ap, alpha_d=ad, sigma=sigma)
    return IPMResult(X=X, y=y, S=S, obj_p=cx, obj_d=by, relgap=relgap, pinf=pinf, dinf=dinf,
                     iters=it, converged=converged, log=log)


def kkt_certificate(P: Problem, X, y, S):
    """FP64 optimality certificate: infeasibilities, relative gap, extreme eigenvalues."""
    Rp, Rd, cx, by, relgap, pinf, dinf = residuals(P, X, y, S)
    return dict(pinf=pinf, dinf=dinf, relgap=relgap, obj_p=cx, obj_d=by,
                lmin_X=float(np.linalg.eigvalsh(X)[0]), lmin_S=float(np.linalg.eigvalsh(S)[0]))


def mc_recovered(P: Problem, X):
    """The p x q block Z of X = [[W1, Z], [Z^T, W2]] (eq. matcomp_sdp)."""
    p = P.meta["p"]
    return X[:p, p:]
