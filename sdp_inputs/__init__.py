"""Seeded synthetic inputs shared by the oracle and the GPU path.

This module only draws random numbers and lays out problem data (triplet lists,
dense test matrices). It holds none of the interior-point or preconditioner
arithmetic, so that the oracle (``oracle/``) and the CUDA library stay
independent of each other while being fed identical inputs.

Triplet convention for symmetric matrices: ``(k, i, j, v)`` with ``i <= j`` sets
``(A_k)[i, j] = (A_k)[j, i] = v``; a diagonal entry is set once.

Matrix-completion instances follow the random model of Section V-A of the
paper (Zhang & Lavaei, "Modified interior-point method for large-and-sparse
low-rank semidefinite programs"): the observed set Omega is drawn uniformly
without replacement among all p*q positions, and the planted matrix is
M = G1 G2^T with G1, G2 i.i.d. standard Gaussian.  The SDP (eq. matcomp_sdp)
has size n = p + q; constraint t observes entry (i, j) through
A_t = 1/2 (e_i e_{p+j}^T + e_{p+j} e_i^T), so A_t . X = X[i, p+j].  The cost
is C = I/2, which makes the optimal value equal to the nuclear norm ||M||_*.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "SDPData", "mc_instance", "mc_m_rule", "config_instance", "CONFIGS",
    "batched_specs", "serving_specs", "serving_arrivals",
    "diag_constraint_instance", "trace_one_instance", "maxcut_bipartite_instance",
    "scalar_instance", "unit_diag_instance", "random_sym", "random_spd", "random_vec",
    "random_general",
]


@dataclass
class SDPData:
    """An SDP in triplet form: min C.X s.t. A_k.X = b_k, X psd (eq. SDP)."""

    n: int
    m: int
    Ci: np.ndarray          # int32, i <= j
    Cj: np.ndarray          # int32
    Cv: np.ndarray          # float64
    Ak: np.ndarray          # int32 constraint index
    Ai: np.ndarray          # int32, i <= j
    Aj: np.ndarray          # int32
    Av: np.ndarray          # float64
    b: np.ndarray           # float64[m]
    k: int                  # rank parameter handed to the preconditioner
    meta: dict = field(default_factory=dict)

    @property
    def nnzA(self) -> int:
        return int(self.Ak.shape[0])

    @property
    def nnzC(self) -> int:
        return int(self.Ci.shape[0])


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def mc_m_rule(p: int, q: int, r: int) -> int:
    """Observation count of the batched and served workloads: min(pq/2, 3 r (p+q) ln(p+q))."""
    return int(min(p * q // 2, math.ceil(3.0 * r * (p + q) * math.log(p + q))))


def mc_instance(p: int, q: int, r: int, m: int, seed: int) -> SDPData:
    """Random matrix-completion SDP (Section V-A; eq. matcomp_sdp).

    Draw order (fixed, so both sides see the same numbers): G1 (p x r), G2 (q x r),
    then Omega = choice(p*q, m, replace=False), sorted; position t -> (t // q, t % q).
    """
    if m > p * q:
        raise ValueError("m exceeds p*q")
    rng = np.random.default_rng(seed)
    G1 = rng.standard_normal((p, r))
    G2 = rng.standard_normal((q, r))
    omega = np.sort(rng.choice(p * q, size=m, replace=False))
    rows = (omega // q).astype(np.int64)
    cols = (omega % q).astype(np.int64)
    M = G1 @ G2.T
    b = M[rows, cols]
    n = p + q
    diag = np.arange(n)
    return SDPData(
        n=n, m=m,
        Ci=_i32(diag), Cj=_i32(diag), Cv=_f64(np.full(n, 0.5)),
        Ak=_i32(np.arange(m)), Ai=_i32(rows), Aj=_i32(p + cols), Av=_f64(np.full(m, 0.5)),
        b=_f64(b), k=r,
        meta=dict(kind="mc", p=p, q=q, r=r, seed=seed, M=M, rows=rows, cols=cols),
    )


# The five workloads.  C1 is the small oracle case, C2 the single-instance FP64
# GPU case, C3 the mixed-precision case, C4 the batched case, C5 the served stream.
CONFIGS = {
    "C1": dict(p=20, q=20, r=1, m=200, seed=1),
    "C2": dict(p=500, q=500, r=2, m=8000, seed=2),
    "C3": dict(p=2000, q=2000, r=3, m=60000, seed=3),
}


def config_instance(name: str) -> SDPData:
    c = CONFIGS[name]
    return mc_instance(c["p"], c["q"], c["r"], c["m"], c["seed"])


def batched_specs(count: int = 256, seed0: int = 4000, lo: int = 50, hi: int = 400):
    """Shapes of the batched workload: p, q uniform integers in [lo, hi], r in {1..4}."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        p = int(rng.integers(lo, hi + 1))
        q = int(rng.integers(lo, hi + 1))
        r = int(rng.integers(1, 5))
        m = mc_m_rule(p, q, r)
        out.append(dict(p=p, q=q, r=r, m=m, seed=seed0 + i))
    return out


def serving_specs(count: int = 2000, seed0: int = 5000, lo: int = 50, hi: int = 3000):
    """Shapes of the served request stream: p, q log-uniform in [lo, hi], r in {1..5}."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        p = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        q = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        r = int(rng.integers(1, 6))
        m = mc_m_rule(p, q, r)
        out.append(dict(p=p, q=q, r=r, m=m, seed=seed0 + i))
    return out


def serving_arrivals(count: int, rate: float, seed: int = 5999) -> np.ndarray:
    """Poisson arrival times (seconds) for ``count`` requests at ``rate`` per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


# ---------------------------------------------------------------------------
# Small SDPs whose solutions are known in closed form (used as pins).
# ---------------------------------------------------------------------------

def unit_diag_instance(n: int, k: int = 1) -> SDPData:
    """min tr X s.t. X_ii = 1: every feasible X is optimal, analytic centre X = I."""
    d = np.arange(n)
    return SDPData(n=n, m=n, Ci=_i32(d), Cj=_i32(d), Cv=_f64(np.ones(n)),
                   Ak=_i32(d), Ai=_i32(d), Aj=_i32(d), Av=_f64(np.ones(n)),
                   b=_f64(np.ones(n)), k=k, meta=dict(kind="unit_diag"))


def trace_one_instance(n: int, seed: int) -> SDPData:
    """min C.X s.t. tr X = 1 with a random symmetric C: value lambda_min(C)."""
    C = random_sym(n, seed)
    iu, ju = np.triu_indices(n)
    d = np.arange(n)
    return SDPData(n=n, m=1, Ci=_i32(iu), Cj=_i32(ju), Cv=_f64(C[iu, ju]),
                   Ak=_i32(np.zeros(n)), Ai=_i32(d), Aj=_i32(d), Av=_f64(np.ones(n)),
                   b=_f64([1.0]), k=1, meta=dict(kind="trace_one", C=C))


def maxcut_bipartite_instance(n1: int, n2: int, seed: int, extra_edges: int = 0) -> SDPData:
    """min A_G.X s.t. X_ii = 1 for a connected bipartite graph G.

    A spanning path alternating sides keeps G connected; ``extra_edges`` random
    cross edges are added.  The optimum is X = z z^T with z the +-1 bipartition
    and value -2|E|.
    """
    rng = np.random.default_rng(seed)
    n = n1 + n2
    left = list(range(n1))
    right = list(range(n1, n))
    edges = set()
    # zig-zag path touching every vertex
    seq = []
    for t in range(max(n1, n2)):
        seq.append(left[min(t, n1 - 1)])
        seq.append(right[min(t, n2 - 1)])
    for a, b in zip(seq[:-1], seq[1:]):
        if a != b:
            edges.add((min(a, b), max(a, b)))
    for _ in range(extra_edges):
        a = int(rng.integers(0, n1))
        b = int(rng.integers(n1, n))
        edges.add((a, b))
    e = np.array(sorted(edges), dtype=np.int64)
    d = np.arange(n)
    z = np.concatenate([np.ones(n1), -np.ones(n2)])
    return SDPData(n=n, m=n, Ci=_i32(e[:, 0]), Cj=_i32(e[:, 1]), Cv=_f64(np.ones(len(e))),
                   Ak=_i32(d), Ai=_i32(d), Aj=_i32(d), Av=_f64(np.ones(n)),
                   b=_f64(np.ones(n)), k=1, meta=dict(kind="maxcut", z=z, n_edges=len(e)))


def scalar_instance(a: float, bval: float, c: float) -> SDPData:
    """n = 1: min c x s.t. a x = b, x >= 0."""
    return SDPData(n=1, m=1, Ci=_i32([0]), Cj=_i32([0]), Cv=_f64([c]),
                   Ak=_i32([0]), Ai=_i32([0]), Aj=_i32([0]), Av=_f64([a]),
                   b=_f64([bval]), k=1, meta=dict(kind="scalar"))


def diag_constraint_instance(n: int, seed: int) -> SDPData:
    """Constraints A_i = e_i e_i^T (m = n) with random positive right-hand sides."""
    rng = np.random.default_rng(seed)
    d = np.arange(n)
    return SDPData(n=n, m=n, Ci=_i32(d), Cj=_i32(d), Cv=_f64(np.ones(n)),
                   Ak=_i32(d), Ai=_i32(d), Aj=_i32(d), Av=_f64(np.ones(n)),
                   b=_f64(rng.uniform(0.5, 2.0, n)), k=1, meta=dict(kind="diag"))


def random_general(n: int, m: int, nnz_per: int, seed: int) -> SDPData:
    """Random sparse SDP whose constraints have pairwise disjoint off-diagonal supports.

    Disjoint supports make A^T A diagonal (the sparsity assumption of the paper,
    with (A^T A)^{-1} diagonal).  Every support lies strictly above the
    diagonal, so any right-hand side is strictly feasible (X = t I plus the
    prescribed off-diagonal entries is positive definite for large t); C is the
    identity plus a small symmetric perturbation that keeps it positive definite,
    so y = 0 is strictly dual feasible.
    """
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, k=1)
    total = iu.shape[0]
    need = m * nnz_per
    if need > total:
        raise ValueError("not enough positions for disjoint supports")
    pos = rng.choice(total, size=need, replace=False)
    Ak = np.repeat(np.arange(m), nnz_per)
    Av = rng.uniform(0.5, 1.5, need) * rng.choice([-1.0, 1.0], need)
    b = rng.standard_normal(m)
    P = rng.standard_normal((n, n))
    ci, cj = np.triu_indices(n)
    cv = 0.05 * (P + P.T)[ci, cj] / math.sqrt(n) + (ci == cj)
    return SDPData(n=n, m=m, Ci=_i32(ci), Cj=_i32(cj), Cv=_f64(cv),
                   Ak=_i32(Ak), Ai=_i32(iu[pos]), Aj=_i32(ju[pos]), Av=_f64(Av),
                   b=_f64(b), k=2, meta=dict(kind="general"))


# ---------------------------------------------------------------------------
# Dense random test inputs.
# ---------------------------------------------------------------------------

def random_sym(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    return (G + G.T) / 2.0


def random_spd(n: int, seed: int, cond: float = 10.0) -> np.ndarray:
    """Random symmetric positive definite matrix with eigenvalues log-spaced in [1, cond]."""
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.logspace(0.0, math.log10(cond), n)
    return (Qm * ev) @ Qm.T


def random_vec(m: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(m)
