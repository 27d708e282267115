// The preconditioner of Section III (Algorithm 1 steps 1-2, eq. SMW2).
//
// Build, for the current scaling matrix W:
//   tau = lambda_min(W);  U = V_l (Lambda_l - tau I)^{1/2}    (eq. Wsplit2)
//   Z   = chol(2 W0 + U U^T) = chol(2 W - U U^T)             (eq. hessExp2)
//   core S = tau^2 I + UU^T G^{-1} UU,  UU = A^T (U kron Z), G = A^T A diagonal
// Block (l, l') of S (n x n, columns of UU ordered l*n + c) is
//   tau^2 delta_ll' I + Z^T K_ll' Z,   K_ll' = sum_i g_i (A_i u_l)(A_i u_l')^T,
// so the formation is a sparse K_ll' Z product followed by a dense Z^T (K Z)
// GEMM per block -- k(k+1)/2 GEMMs of n^3 instead of an m x nk Gram matrix.
// The core is factored L L^T = S and L^{-1} is formed once, so every apply
// costs two triangular matrix-vector products instead of two dependent
// triangular solves.
//
// Apply (eq. SMW2):  t = G^{-1} r;  u = UU^T t = Z^T (sum t_i A_i) U;
//   s = L^{-T} L^{-1} u;  z = tau^{-2} G^{-1} (r - UU s),  (UU s)_i = A_i . (Z S U^T).
//
// Section V's Hhat = A^T (tau^2 I + 2 tau U U^T kron I) A (eq. sparse_prec) is
// the same construction with Z = sqrt(2 tau) I: the core blocks become
// tau^2 delta_ll' I + 2 tau K_ll' (K scattered, no dense GEMM), and both Z
// products of the apply become scalings.  Near the optimum the Algorithm 1
// core has condition number ~ (lambda_max(W) / tau)^2, beyond FP64 once
// mu ~ 1e-5, while the Hhat core stays near lambda_max(W) / tau.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <utility>

namespace sdpgb {

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// U[a][l] = Etop[l][a] * sqrt(max(wtop[l] - tau, 0))
__global__ void k_make_U(int n, int k, const double* __restrict__ Etop, const double* __restrict__ wtop,
                         const double* __restrict__ tau_dev, double* __restrict__ U) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int a = t / k, l = t % k;
  const double s = sqrt(fmax(wtop[l] - tau_dev[0], 0.0));
  U[t] = Etop[(size_t)l * n + a] * s;
}

// au[cr][l] = (A_i u_l)[row(cr)] = sum_{(b, coef) in row(cr) of A_i} coef U[b][l]
__global__ void k_au(int ncr, int k, const int* __restrict__ clptr, const int* __restrict__ clcol,
                     const double* __restrict__ clcoef, const double* __restrict__ U, double* __restrict__ au) {
  const int cr = blockIdx.x * blockDim.x + threadIdx.x;
  if (cr >= ncr) return;
  for (int l = 0; l < k; ++l) {
    double s = 0.0;
    for (int t = clptr[cr]; t < clptr[cr + 1]; ++t) s = fma(clcoef[t], U[(size_t)clcol[t] * k + l], s);
    au[(size_t)cr * k + l] = s;
  }
}

// Kval[s] = sum_{(i, cra, crb) in slot s} g_i au[cra][l] au[crb][l2]
__global__ void k_kvals(int nnzK, const int* __restrict__ kptr, const int* __restrict__ kcon,
                        const int* __restrict__ kcra, const int* __restrict__ kcrb, const double* __restrict__ ginv,
                        const double* __restrict__ au, int k, int l, int l2, double* __restrict__ Kval) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nnzK) return;
  double acc = 0.0;
  for (int t = kptr[s]; t < kptr[s + 1]; ++t)
    acc = fma(ginv[kcon[t]] * au[(size_t)kcra[t] * k + l], au[(size_t)kcrb[t] * k + l2], acc);
  Kval[s] = acc;
}

// out[a, c] = sum_{s in row a} val[s] B[col(s), c]   (generic CSR)
__global__ void k_csr_mm(int rows, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                         const double* __restrict__ val, const double* __restrict__ B, int ldb, int ncols,
                         double* __restrict__ out, int ldo) {
  const int a = blockIdx.y;
  if (a >= rows) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = rowptr[a]; s < rowptr[a + 1]; ++s) acc = fma(val[s], B[(size_t)colidx[s] * ldb + c], acc);
    out[(size_t)a * ldo + c] = acc;
  }
}

// z_i = (ginv_i / tau^2) (r_i - (UU s)_i),  (UU s)_i = A_i . (ZS U^T); with
// dout != nullptr also *dout = r . z (one deterministic grid reduction).
__device__ __forceinline__ void apply_tail_body(int lb, int nb, int m, int k, const int* __restrict__ eptr,
                                                const int* __restrict__ ep, const int* __restrict__ eq,
                                                const double* __restrict__ ecoef, const double* __restrict__ ZS,
                                                const double* __restrict__ U, const double* __restrict__ ginv,
                                                const double* __restrict__ r, double inv_tau2, double* __restrict__ z,
                                                double* dpart, unsigned int* ticket, double* dout) {
  const int i = lb * blockDim.x + threadIdx.x;
  double rz = 0.0;
  if (i < m) {
    double us = 0.0;
    for (int e = eptr[i]; e < eptr[i + 1]; ++e) {
      const int p = ep[e], q = eq[e];
      double s = 0.0;
      if (p == q) {
        for (int l = 0; l < k; ++l) s = fma(ZS[(size_t)p * k + l], U[(size_t)p * k + l], s);
        us = fma(ecoef[e], s, us);
      } else {
        for (int l = 0; l < k; ++l) {
          s = fma(ZS[(size_t)p * k + l], U[(size_t)q * k + l], s);
          s = fma(ZS[(size_t)q * k + l], U[(size_t)p * k + l], s);
        }
        us = fma(0.5 * ecoef[e], s, us);
      }
    }
    const double zi = ginv[i] * inv_tau2 * (r[i] - us);
    z[i] = zi;
    rz = r[i] * zi;
  }
  if (dout) {
    double tot;
    if (lb_reduce(rz, dpart, ticket, &tot, lb, nb)) *dout = tot;
  }
}
__global__ void k_apply_tail(int m, int k, const int* __restrict__ eptr, const int* __restrict__ ep,
                             const int* __restrict__ eq, const double* __restrict__ ecoef,
                             const double* __restrict__ ZS, const double* __restrict__ U,
                             const double* __restrict__ ginv, const double* __restrict__ r, double inv_tau2,
                             double* __restrict__ z, double* dpart, unsigned int* ticket, double* dout) {
  apply_tail_body(blockIdx.x, gridDim.x, m, k, eptr, ep, eq, ecoef, ZS, U, ginv, r, inv_tau2, z, dpart, ticket,
                  dout);
}

// Hhat apply, first product: u[l n + a] = scale * sum_{s in row a} V_s U[col(s)][l]
// with V = sum_i g_i^{-1} r_i A_i assembled on the fly; one warp per row a.
__device__ __forceinline__ void hat_u_body(int a, int lane, int n, int k, const int* __restrict__ rowptr,
                                           const int* __restrict__ colidx, const int* __restrict__ sptr,
                                           const int* __restrict__ scon, const double* __restrict__ scoef,
                                           const double* __restrict__ ginv, const double* __restrict__ r,
                                           const double* __restrict__ U, double scale, double* __restrict__ u) {
  if (a >= n) return;
  double acc[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) acc[l] = 0.0;
  for (int s = rowptr[a] + lane; s < rowptr[a + 1]; s += 32) {
    double v = 0.0;
    for (int c = sptr[s]; c < sptr[s + 1]; ++c) {
      const int i = scon[c];
      v = fma(scoef[c] * ginv[i], r[i], v);
    }
    const double* ur = U + (size_t)colidx[s] * k;
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (l < k) acc[l] = fma(v, ur[l], acc[l]);
  }
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    if (l >= k) break;
    double t = acc[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) u[(size_t)l * n + a] = scale * t;
  }
}
__global__ void k_hat_u(int n, int k, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                        const int* __restrict__ sptr, const int* __restrict__ scon, const double* __restrict__ scoef,
                        const double* __restrict__ ginv, const double* __restrict__ r, const double* __restrict__ U,
                        double scale, double* __restrict__ u) {
  hat_u_body((blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, n, k, rowptr, colidx, sptr, scon,
             scoef, ginv, r, U, scale, u);
}

// The same product for split ranks above 8 (up to 64): one warp per row a; the
// lanes first assemble V on 32 entries of the row at once, then every entry is
// broadcast and lane l accumulates columns l and l + 32 of u.
__global__ void k_hat_u_gen(int n, int k, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                            const int* __restrict__ sptr, const int* __restrict__ scon,
                            const double* __restrict__ scoef, const double* __restrict__ ginv,
                            const double* __restrict__ r, const double* __restrict__ U, double scale,
                            double* __restrict__ u) {
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (a >= n) return;
  double a0 = 0.0, a1 = 0.0;
  const int l0 = lane, l1 = lane + 32;
  for (int s0 = rowptr[a]; s0 < rowptr[a + 1]; s0 += 32) {
    const int cnt = min(32, rowptr[a + 1] - s0);
    double v = 0.0;
    int col = 0;
    if (lane < cnt) {
      const int s = s0 + lane;
      for (int c = sptr[s]; c < sptr[s + 1]; ++c) {
        const int i = scon[c];
        v = fma(scoef[c] * ginv[i], r[i], v);
      }
      col = colidx[s];
    }
    for (int t = 0; t < cnt; ++t) {
      const double vt = __shfl_sync(0xffffffffu, v, t);
      const int ct = __shfl_sync(0xffffffffu, col, t);
      const double* ur = U + (size_t)ct * k;
      if (l0 < k) a0 = fma(vt, ur[l0], a0);
      if (l1 < k) a1 = fma(vt, ur[l1], a1);
    }
  }
  if (l0 < k) u[(size_t)l0 * n + a] = scale * a0;
  if (l1 < k) u[(size_t)l1 * n + a] = scale * a1;
}

// Batched forms of the Hhat apply ends (the core solve is in schur.cu)
__global__ void kb_hat_u(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active) return;
  const int lb = blockIdx.x - off[i];
  hat_u_body((lb * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, D.n, D.k, D.rowptr, D.colidx, D.sptr, D.scon,
             D.scoef, D.ginv, D.pr, D.U, D.zscale, D.uvec);
}
__global__ void kb_apply_tail(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active) return;
  apply_tail_body(blockIdx.x - off[i], off[i + 1] - off[i], D.m, D.k, D.eptr, D.ep, D.eq, D.ecoef, D.Bn, D.U,
                  D.ginv, D.pr, D.inv_tau2, D.pz, D.part, D.ticket, D.scal + S_RZN);
}
int batch_blocks_hat_u(int n) { return (int)cdiv((size_t)n * 32, 256); }
int batch_blocks_tail(int m) { return (int)cdiv(m, 256); }
void batch_launch_hat_u(cudaStream_t st, const BDesc* desc, const int* off, int N, int nb) {
  count_launch();
  if (nb > 0) kb_hat_u<<<nb, 256, 0, st>>>(desc, off, N);
}
void batch_launch_tail(cudaStream_t st, const BDesc* desc, const int* off, int N, int nb) {
  count_launch();
  if (nb > 0) kb_apply_tail<<<nb, 256, 0, st>>>(desc, off, N);
}

__global__ void k_scale_ginv(int m, const double* __restrict__ ginv, const double* __restrict__ r, double s,
                             double* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) z[i] = ginv[i] * s * r[i];
}

// Tall-skinny products of the apply (k <= 32 columns; HBM/FP64-bound, not
// tensor-core work).  ut_part[chunk][l][c] = sum_{a in chunk} B[a][l] Z[a][c]:
// threads run over the columns c of Z (coalesced rows), the k sums stay in
// registers, and row chunks spread the work over the GPU; k_ts_ut_sum adds
// the chunks in a fixed order.
constexpr int TS_CHUNKS = 32;
template <int K>
__global__ void k_ts_ut(int n, const double* __restrict__ B, const double* __restrict__ Z,
                        double* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int rows = (n + TS_CHUNKS - 1) / TS_CHUNKS;
  const int a0 = blockIdx.y * rows, a1 = min(n, a0 + rows);
  if (c >= n) return;
  double acc[K];
#pragma unroll
  for (int l = 0; l < K; ++l) acc[l] = 0.0;
  for (int a = a0; a < a1; ++a) {
    const double z = Z[(size_t)a * n + c];
#pragma unroll
    for (int l = 0; l < K; ++l) acc[l] = fma(B[(size_t)a * K + l], z, acc[l]);
  }
#pragma unroll
  for (int l = 0; l < K; ++l) part[((size_t)blockIdx.y * K + l) * n + c] = acc[l];
}
__global__ void k_ts_ut_sum(int n, int k, const double* __restrict__ part, double* __restrict__ u) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int l = t / n, c = t % n;
  double s = 0.0;
  for (int ch = 0; ch < TS_CHUNKS; ++ch) s += part[((size_t)ch * k + l) * n + c];
  u[(size_t)l * n + c] = s;
}
// ZS[a][l] = sum_c Z[a][c] s[l n + c]: one warp per row a of Z.
template <int K>
__global__ void k_ts_zs(int n, const double* __restrict__ Z, const double* __restrict__ s,
                        double* __restrict__ ZS) {
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (a >= n) return;
  const double* za = Z + (size_t)a * n;
  double acc[K];
#pragma unroll
  for (int l = 0; l < K; ++l) acc[l] = 0.0;
  for (int c = lane; c < n; c += 32) {
    const double z = za[c];
#pragma unroll
    for (int l = 0; l < K; ++l) acc[l] = fma(z, s[(size_t)l * n + c], acc[l]);
  }
#pragma unroll
  for (int l = 0; l < K; ++l) {
    double v = acc[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ZS[(size_t)a * K + l] = v;
  }
}

template <int K>
static void ts_launch(cudaStream_t st, int n, const double* Bn, const double* Z, double* part, double* u,
                      const double* s, double* ZS, bool first) {
  if (first) {
    count_launch(2);
    k_ts_ut<K><<<dim3((n + 127) / 128, TS_CHUNKS), 128, 0, st>>>(n, Bn, Z, part);
    k_ts_ut_sum<<<cdiv((size_t)n * K, 256), 256, 0, st>>>(n, K, part, u);
  } else {
    count_launch();
    k_ts_zs<K><<<cdiv((size_t)n * 32, 256), 256, 0, st>>>(n, Z, s, ZS);
  }
}

// u (k x n) = Bn^T Z  or  ZS (n x k) = Z S_mat, dispatched on k.
static bool ts_product(cudaStream_t st, int n, int k, const double* Bn, const double* Z, double* part,
                       double* u, const double* s, double* ZS, bool first) {
  switch (k) {
    case 1: ts_launch<1>(st, n, Bn, Z, part, u, s, ZS, first); return true;
    case 2: ts_launch<2>(st, n, Bn, Z, part, u, s, ZS, first); return true;
    case 3: ts_launch<3>(st, n, Bn, Z, part, u, s, ZS, first); return true;
    case 4: ts_launch<4>(st, n, Bn, Z, part, u, s, ZS, first); return true;
    case 5: ts_launch<5>(st, n, Bn, Z, part, u, s, ZS, first); return true;
    case 6: ts_launch<6>(st, n, Bn, Z, part, u, s, ZS, first); return true;
    case 7: ts_launch<7>(st, n, Bn, Z, part, u, s, ZS, first); return true;
    case 8: ts_launch<8>(st, n, Bn, Z, part, u, s, ZS, first); return true;
    default: return false;
  }
}

// ---------------------------------------------------------------------------
// Subspace refinement of the top-k eigenpairs of W (k <= 31).  Inverse iteration
// on the tridiagonal form can return nearly parallel vectors for close top
// eigenvalues; two steps of subspace iteration with W itself (GEMMs) followed by
// Rayleigh-Ritz on the k x k projection restore an orthonormal basis of the
// dominant invariant subspace (the gap lambda_k / lambda_{k+1} grows like 1/mu,
// so the iteration converges in one or two steps where it matters).
// ---------------------------------------------------------------------------
// In place Gram-Schmidt (two passes) over k rows of length n, one CTA.
__global__ void k_rows_orth(int n, int k, double* E) {
  __shared__ double red[32];
  __shared__ double s_val;
  for (int a = 0; a < k; ++a) {
    double* xa = E + (size_t)a * n;
    for (int pass = 0; pass < 2; ++pass) {
      for (int b = 0; b < a; ++b) {
        const double* xb = E + (size_t)b * n;
        double s = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(xa[i], xb[i], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
          double t = 0.0;
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
          s_val = t;
        }
        __syncthreads();
        const double c = s_val;
        for (int i = threadIdx.x; i < n; i += blockDim.x) xa[i] -= c * xb[i];
        __syncthreads();
      }
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(xa[i], xa[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      s_val = (t > 0.0) ? 1.0 / sqrt(t) : 0.0;
    }
    __syncthreads();
    const double c = s_val;
    for (int i = threadIdx.x; i < n; i += blockDim.x) xa[i] *= c;
    __syncthreads();
  }
}

// Cyclic Jacobi on the k x k symmetric B (k <= 32) in one thread; Q (k x k, row
// j = eigenvector j) and ascending eigenvalues w.  Tiny, so one thread is enough.
__global__ void k_small_jacobi(int k, double* B, double* Q, double* w) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) Q[i * k + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        tot += B[i * k + j] * B[i * k + j];
        if (i != j) off += B[i * k + j] * B[i * k + j];
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = B[p * k + q];
        if (apq == 0.0) continue;
        const double theta = 0.5 * (B[q * k + q] - B[p * k + p]) / apq;
        const double t = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < k; ++r) {  // B <- J^T B J (columns, then rows)
          const double bp = B[r * k + p], bq = B[r * k + q];
          B[r * k + p] = c * bp - s * bq;
          B[r * k + q] = s * bp + c * bq;
        }
        for (int r = 0; r < k; ++r) {
          const double bp = B[p * k + r], bq = B[q * k + r];
          B[p * k + r] = c * bp - s * bq;
          B[q * k + r] = s * bp + c * bq;
        }
        for (int r = 0; r < k; ++r) {  // rows of Q are eigenvectors: Q <- J^T Q
          const double qp = Q[p * k + r], qq = Q[q * k + r];
          Q[p * k + r] = c * qp - s * qq;
          Q[q * k + r] = s * qp + c * qq;
        }
      }
  }
  // sort ascending (selection sort on k <= 32)
  for (int i = 0; i < k; ++i) w[i] = B[i * k + i];
  for (int i = 0; i < k; ++i) {
    int mi = i;
    for (int j = i + 1; j < k; ++j) if (w[j] < w[mi]) mi = j;
    if (mi != i) {
      const double tw = w[i]; w[i] = w[mi]; w[mi] = tw;
      for (int r = 0; r < k; ++r) { const double tq = Q[i * k + r]; Q[i * k + r] = Q[mi * k + r]; Q[mi * k + r] = tq; }
    }
  }
}

static sdp_status precond_alloc(sdp_problem* h) {
  if (h->U) return SDP_OK;
  // kcap + 1 eigenpairs are computed for the adaptive rule (it compares
  // lambda_k with lambda_{k+1}); the split itself uses at most kcap of them
  const int n = h->n, k = std::max(h->kcap + 1, 1), kc = std::max(h->kcap, 1);
  const size_t nk = (size_t)n * k, nkc = (size_t)n * kc;
  SDP_TRY(h->allocT(&h->U, nk));
  SDP_TRY(h->allocT(&h->Z, (size_t)n * n));
  if (h->prm.precond != SDP_PRECOND_HAT) {   // dense core (Hhat factors it sparsely, schur.cu)
    SDP_TRY(h->allocT(&h->Sc, nkc * nkc));
    SDP_TRY(h->allocT(&h->Linv, nkc * nkc));
  }
  SDP_TRY(h->allocT(&h->tau_dev, 8 + 2 * (size_t)(SDP_K_MAX + 1) * (SDP_K_MAX + 1)));
  SDP_TRY(h->allocT(&h->wtop, SDP_K_MAX + 1));
  SDP_TRY(h->allocT(&h->Etop, (size_t)(SDP_K_MAX + 1) * n));
  SDP_TRY(h->allocT(&h->au, (size_t)std::max(h->ncr, 1) * k));
  SDP_TRY(h->allocT(&h->Kval, std::max(h->nnzK, 1)));
  SDP_TRY(h->allocT(&h->KZ, (size_t)n * n));
  SDP_TRY(h->allocT(&h->Bn, nk));
  SDP_TRY(h->allocT(&h->uvec, nk));
  SDP_TRY(h->allocT(&h->uvec2, nk));
  SDP_TRY(h->allocT(&h->uvec3, nk));
  SDP_TRY(h->allocT(&h->pvec, std::max<size_t>(nk, (size_t)h->nnzV)));
  SDP_TRY(h->allocT(&h->trpart, std::max(trmv_part_doubles((int)nk), (size_t)TS_CHUNKS * nk)));
  SDP_TRY(h->allocT(&h->info, 8));
  const size_t wneed = std::max(std::max(potrf_work_doubles((int)nkc), trsm_work_doubles((int)nkc, (int)nkc)),
                                std::max(potrf_work_doubles(n), trsm_work_doubles(n, n)));
  if (wneed > h->work_doubles) {
    SDP_TRY(h->allocT(&h->work, wneed));
    h->work_doubles = wneed;
  }
  // n x n scratch, also the NT-scaling check's 16 n doubles when n < 16
  if (!h->M1) SDP_TRY(h->allocT(&h->M1, std::max((size_t)n * n, (size_t)16 * n)));
  if (!h->eig_base) {
    SDP_TRY(h->alloc(&h->eig_base, eig_work_bytes(n, true)));
    eig_work_carve(&h->eig, h->eig_base, n, true);
    eig_work_clear(h->stream, &h->eig);
    h->eig.spin_cycles = h->prm.wait_cycles;
  }
  return SDP_OK;
}

static sdp_status read_info(sdp_problem* h, const char* what) {
  int info = 0;
  SDP_CK(h, cudaMemcpyAsync(&info, h->info, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  SDP_CK(h, cudaStreamSynchronize(h->stream));
  if (info != 0) {
    h->last_error = std::string(what) + ": non-positive pivot at " + std::to_string(info - 1);
    return SDP_ERR_NOT_PD;
  }
  return SDP_OK;
}

// Sc = Z^T K_ll' Z block by block, plus shift on the diagonal.
// With a reduced-precision handle (params.prec = SDP_FP32 or SDP_BF16) the dense
// Z^T (K Z) products run on the tensor cores (tc_gemm) with TF32 operands and
// FP32 accumulation; the core is still factored in FP64.  BF16 operands (8-bit
// significands) are not used here: the core has kappa >= 1e2 already at mu ~ 0.1,
// and a BF16-formed core left PCG without convergence in the tests.
static sdp_status form_core(sdp_problem* h, int k, double shift) {
  cudaStream_t st = h->stream;
  const int n = h->n, nk = n * k;
  const bool mixed = (h->prm.prec == SDP_FP32 || h->prm.prec == SDP_BF16) && tc_available();
  int* tc_err = h->info + 4;
  if (mixed) {
    if (!h->tc_work) SDP_TRY(h->alloc(&h->tc_work, tc_work_bytes(n, n, n)));
    SDP_CK(h, cudaMemsetAsync(tc_err, 0, sizeof(int), st));
  }
  for (int l = 0; l < k; ++l) {
    for (int l2 = l; l2 < k; ++l2) {
      count_launch(2);
      k_kvals<<<cdiv(h->nnzK, 256), 256, 0, st>>>(h->nnzK, h->kptr, h->kcon, h->kcra, h->kcrb, h->ginv, h->au,
                                                 k, l, l2, h->Kval);
      const unsigned gx = std::max(1u, std::min(cdiv(n, 128), 64u));
      k_csr_mm<<<dim3(gx, n), 128, 0, st>>>(n, h->krowptr, h->kcol, h->Kval, h->Z, n, n, h->KZ, n);
      double* blk = h->Sc + (size_t)l * n * nk + (size_t)l2 * n;
      if (mixed) SDP_TRY(tc_gemm(st, SDP_FP32, n, n, n, h->Z, n, true, h->KZ, n, false, blk, nk, h->tc_work, tc_err));
      else gemm(st, true, false, n, n, n, 1.0, h->Z, n, h->KZ, n, 0.0, blk, nk);
      if (l2 != l) transpose(st, n, n, blk, nk, h->Sc + (size_t)l2 * n * nk + (size_t)l * n, nk);
    }
  }
  if (shift != 0.0) add_diag(st, nk, h->Sc, nk, shift);
  if (mixed) {
    int e = 0;
    SDP_CK(h, cudaMemcpyAsync(&e, tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SDP_CK(h, cudaStreamSynchronize(st));
    if (e) {
      h->last_error = "precond_build: a bounded wait of the tensor-core core formation ran out";
      return SDP_ERR_TIMEOUT;
    }
  }
  return SDP_OK;
}

sdp_status precond_build_impl(sdp_problem* h) {
  SDP_TRY(precond_alloc(h));
  cudaStream_t st = h->stream;
  const int n = h->n;
  const bool diag = (h->prm.precond == SDP_PRECOND_DIAG);
  const bool adaptive = !diag && h->prm.eta > 0.0;
  // eigenpairs to compute: the fixed k, or kcap + 1 for the adaptive rule
  const int kq = diag ? 0 : std::min(adaptive ? h->kcap + 1 : h->k, n - 1 > 0 ? n - 1 : 0);
  // ---- step 1a: eigenvalues of W (smallest and top kq with vectors)
  copy2d(st, n, n, h->W, n, h->M1, n);
  SDP_TRY(eig_extremes(st, n, h->M1, kq, h->tau_dev, h->wtop, h->Etop, &h->eig));
  int k = kq;
  if (adaptive) {
    // Section V implementation notes: k~ = max{i <= k_max : lambda_i >= eta lambda_{i+1}},
    // eigenvalues in decreasing order, lambda_0 = +inf (so i = 0 always qualifies);
    // wtop holds lambda_{kq}..lambda_1 in ascending order
    double lam[SDP_K_MAX + 1];
    SDP_CK(h, cudaMemcpyAsync(lam, h->wtop, kq * sizeof(double), cudaMemcpyDeviceToHost, st));
    SDP_CK(h, cudaStreamSynchronize(st));
    k = 0;
    for (int i = 1; i <= std::min(h->kcap, kq - 1); ++i)
      if (lam[kq - i] >= h->prm.eta * lam[kq - 1 - i]) k = i;
    h->kest = k;
    if (k > 0 && k < kq) {
      // keep the top k pairs at the front of Etop / wtop (rows kq - k .. kq - 1)
      SDP_CK(h, cudaMemcpyAsync(h->Bn, h->Etop + (size_t)(kq - k) * n, (size_t)k * n * sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
      SDP_CK(h, cudaMemcpyAsync(h->Etop, h->Bn, (size_t)k * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      SDP_CK(h, cudaMemcpyAsync(h->Bn, h->wtop + (kq - k), k * sizeof(double), cudaMemcpyDeviceToDevice, st));
      SDP_CK(h, cudaMemcpyAsync(h->wtop, h->Bn, k * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
  }
  const int nk = n * k;
  if (k > 0) {
    // refine Etop (k x n): two subspace steps with W, then Rayleigh-Ritz
    double* V = h->Bn;            // k x n scratch (Bn holds n k doubles)
    double* sm = h->tau_dev + 8;  // k x k projection, k x k rotation
    for (int step = 0; step < 2; ++step) {
      gemm(st, false, false, k, n, n, 1.0, h->Etop, n, h->W, n, 0.0, V, n);   // rows of E W
      count_launch();
      k_rows_orth<<<1, 256, 0, st>>>(n, k, V);
      copy2d(st, k, n, V, n, h->Etop, n);
    }
    gemm(st, false, false, k, n, n, 1.0, h->Etop, n, h->W, n, 0.0, V, n);     // E W
    gemm(st, false, true, k, k, n, 1.0, V, n, h->Etop, n, 0.0, sm, k);        // B = E W E^T
    symmetrize_avg(st, k, sm, k);
    count_launch();
    k_small_jacobi<<<1, 32, 0, st>>>(k, sm, sm + k * k, h->wtop);
    gemm(st, false, false, k, n, k, 1.0, sm + k * k, k, h->Etop, n, 0.0, V, n); // rotate
    copy2d(st, k, n, V, n, h->Etop, n);
  }
  double tau = 0.0;
  SDP_CK(h, cudaMemcpyAsync(&tau, h->tau_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaStreamSynchronize(st));
  if (eig_flag(st, &h->eig)) {
    h->last_error = "precond_build: grid barrier timeout in the tridiagonalisation";
    return SDP_ERR_TIMEOUT;
  }
  if (!(tau > 0.0) || !std::isfinite(tau)) {
    h->last_error = "precond_build: lambda_min(W) = " + std::to_string(tau) + " is not positive";
    return SDP_ERR_NUMERIC;
  }
  h->tau = tau;
  h->kpc = k;
  if (k == 0) {
    h->pc_valid = true;
    h->pc_generation++;
    return SDP_OK;
  }
  const bool hat = (h->prm.precond == SDP_PRECOND_HAT);
  h->pc_hat = hat;
  h->zscale = std::sqrt(2.0 * tau);
  // ---- step 1b: U, and Z = chol(2W - U U^T) (Algorithm 1) or sqrt(2 tau) I (Hhat)
  count_launch();
  k_make_U<<<cdiv((size_t)n * k, 256), 256, 0, st>>>(n, k, h->Etop, h->wtop, h->tau_dev, h->U);
  if (!hat) {
    axpby(st, (size_t)n * n, 2.0, h->W, 0.0, nullptr, h->Z);
    gemm(st, false, true, n, n, k, -1.0, h->U, k, h->U, k, 1.0, h->Z, n);
    potrf(st, n, h->Z, n, h->info, h->work);
    SDP_TRY(read_info(h, "precond_build: chol(2 W0 + U U^T)"));
  }
  // ---- step 2: core S = tau^2 I + Z^T K Z (block l, l'), Cholesky, inverse
  count_launch();
  k_au<<<cdiv(h->ncr, 256), 256, 0, st>>>(h->ncr, k, h->crlist_ptr, h->crlist_col, h->crlist_coef, h->U, h->au);
  // S = tau^2 I + UU^T G^{-1} UU >= tau^2 I exactly, so every Cholesky pivot of
  // S is at least tau^2.  Near the optimum S is ill conditioned (kappa ~
  // (lambda_max(W) / tau)^2) and FP64 rounding in its formation can push a pivot
  // below that bound or below zero; such pivots are raised to tau^2 (a
  // modified Cholesky with the bound the mathematics gives), which keeps the
  // factor of an SPD matrix close to S in every direction.
  h->core_shift = tau * tau;
  if (hat) {
    SDP_TRY(schur_build(h, k, tau));
  } else {
    SDP_TRY(form_core(h, k, tau * tau));
    potrf_floor(st, nk, h->Sc, nk, h->info, h->work, tau * tau);
    int inf2[2] = {0, 0};
    SDP_CK(h, cudaMemcpyAsync(inf2, h->info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    SDP_CK(h, cudaStreamSynchronize(st));
    h->core_floor_pivots = inf2[1];
    fill(st, h->Linv, (size_t)nk * nk, 0.0);
    add_diag(st, nk, h->Linv, nk, 1.0);
    trsm_left_lower_ex(st, false, nk, nk, h->Sc, nk, h->Linv, nk, h->work, true);
  }
  h->pc_valid = true;
  h->pc_generation++;
  return SDP_OK;
}

// prec != SDP_FP64 with the Hhat core: the two dense triangular products of the
// core solve read the FP32 copy of the Schur-factor inverse (schur_apply); every
// other step, and the whole Algorithm 1 apply, runs in FP64.
sdp_status precond_apply_impl(sdp_problem* h, const double* r, double* z, int prec, double* dot_out) {
  if (prec != SDP_FP64 && prec != SDP_FP32 && prec != SDP_BF16) {
    h->last_error = "precond_apply: unknown precision";
    return SDP_ERR_ARG;
  }
  cudaStream_t st = h->stream;
  const int n = h->n, m = h->m, k = h->kpc, nk = n * k;
  const double inv_tau2 = 1.0 / (h->tau * h->tau);
  if (k == 0) {
    count_launch();
    k_scale_ginv<<<cdiv(m, 256), 256, 0, st>>>(m, h->ginv, r, inv_tau2, z);
    if (dot_out) dot(st, m, r, z, dot_out, h->part);
    return SDP_OK;
  }
  if (h->pc_hat) {
    // u = sqrt(2 tau) (sum g_i r_i A_i) U (k x n); S^{-1} u through the block
    // factors, returned as ZS = sqrt(2 tau) S_mat (n x k)
    count_launch();
    if (k > 8)
      k_hat_u_gen<<<cdiv((size_t)n * 32, 256), 256, 0, st>>>(n, k, h->rowptr, h->colidx, h->sptr, h->scon,
                                                             h->scoef, h->ginv, r, h->U, h->zscale, h->uvec);
    else
      k_hat_u<<<cdiv((size_t)n * 32, 256), 256, 0, st>>>(n, k, h->rowptr, h->colidx, h->sptr, h->scon, h->scoef,
                                                         h->ginv, r, h->U, h->zscale, h->uvec);
    SDP_TRY(schur_apply(h, h->uvec, h->Bn, h->zscale, prec));
  } else {
    // u = Z^T (sum g_i r_i A_i) U, stored as k x n (row l = column l of u)
    assemble_V(h, r, h->ginv, h->pvec);
    spmm_rows(h, h->pvec, h->U, k, k, h->Bn, k);
    if (!ts_product(st, n, k, h->Bn, h->Z, h->trpart, h->uvec, nullptr, nullptr, true))
      gemm(st, true, false, k, n, n, 1.0, h->Bn, k, h->Z, n, 0.0, h->uvec, n);
    // s = L^{-T} L^{-1} u.  Multiplying by the stored inverse alone loses accuracy
    // once the core is ill conditioned (kappa(L) eps, late interior-point
    // iterations), so each triangular solve takes one step of iterative refinement
    // whose residual uses the factor itself:  y0 = L^{-1} u,  y = y0 + L^{-1}(u - L y0).
    // ||I - L^{-1} L|| stays far below one where the plain inverse has failed, and
    // the refined solve matches substitution.  Buffers: uvec = u, uvec2 = y0, uvec3 = scratch.
    for (int t = 0; t < 2; ++t) {
      const bool tr = (t == 1);
      trmv_lower_ex(st, tr, nk, h->Linv, nk, h->uvec, h->uvec2, h->trpart, 1.0, nullptr, 0.0);   // y0
      for (int it = 0; it < h->core_refine; ++it) {
        trmv_lower_ex(st, tr, nk, h->Sc, nk, h->uvec2, h->uvec3, h->trpart, -1.0, h->uvec, 1.0); // u - L y0
        trmv_lower_ex(st, tr, nk, h->Linv, nk, h->uvec3, h->uvec2, h->trpart, 1.0, h->uvec2, 1.0);  // y0 + L^{-1} res
      }
      std::swap(h->uvec, h->uvec2);   // result becomes the input of the next solve
    }
    // ZS = Z S_mat with S_mat[c][l] = s[l n + c]
    if (!ts_product(st, n, k, nullptr, h->Z, nullptr, nullptr, h->uvec, h->Bn, false))
      gemm(st, false, true, n, k, n, 1.0, h->Z, n, h->uvec, n, 0.0, h->Bn, k);
  }
  count_launch();
  k_apply_tail<<<cdiv(m, 256), 256, 0, st>>>(m, k, h->eptr, h->ep, h->eq, h->ecoef, h->Bn, h->U, h->ginv, r,
                                             inv_tau2, z, h->pcg_part, h->pcg_ticket, dot_out);
  return SDP_OK;
}

}  // namespace sdpgb
