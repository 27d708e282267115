// Sparse factorisation of the Section V core (eq. sparse_prec).
//
// For Hhat the core is S = tau^2 I + 2 tau K, with K_(l,x),(l',y) =
// sum_i g_i^{-1} (A_i u_l)_x (A_i u_l')_y nonzero only where rows x and y are
// touched by a common constraint (the K pattern) -- the paper notes that this
// matrix is sparse and that a sparse factorisation can cost far less than the
// dense (nk)^3 / 3.  Ordered by rows of W ("vertices"), S is block sparse with
// k x k blocks.  Rows of an independent set P of the K graph have no block
// between them, so S_PP is block diagonal, and
//   S = [[D, B], [B^T, E]],  D = diag(D_a),  L = [[L_P, 0], [F^T, L_C]],
//   L_P = diag(chol(D_a)),  F = L_P^{-1} B,  C = E - F^T F = L_C L_C^T,
// leaves a dense factorisation of the Schur complement C on the other rows R
// only.  For matrix completion the K graph is bipartite (rows of the observed
// matrix against its columns), P is the larger side and C has order
// min(p, q) k; the Schur complement needs about sum_a deg(a)^2 k^3 / 2 FMAs.
//
// Apply (S^{-1} u):  y_P = L_P^{-1} u_P;  y_R = L_C^{-1}(u_R - F^T y_P);
//                    x_R = L_C^{-T} y_R;  x_P = L_P^{-T}(y_P - F x_R).
// The two dense triangular solves use L_C^{-1} with one refinement step
// against L_C, as the dense core does.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <queue>

namespace sdpgb {

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Host: choose P and classify the K slots
// ---------------------------------------------------------------------------
// K graph: vertices = rows of W, edges = off-diagonal K slots.  If it is
// bipartite, each connected component contributes its larger colour class to
// P; otherwise P is a greedy maximal independent set taken in order of
// increasing degree.
void schur_plan(int n, const std::vector<int>& krowptr, const std::vector<int>& kcol, SchurPlanHost* out) {
  std::vector<int> color(n, -1);
  bool bip = true;
  std::vector<char> inP(n, 0);
  std::vector<int> comp;
  for (int s = 0; s < n && bip; ++s) {
    if (color[s] >= 0) continue;
    comp.clear();
    std::queue<int> q;
    q.push(s);
    color[s] = 0;
    while (!q.empty() && bip) {
      const int v = q.front();
      q.pop();
      comp.push_back(v);
      for (int t = krowptr[v]; t < krowptr[v + 1]; ++t) {
        const int u = kcol[t];
        if (u == v) continue;
        if (color[u] < 0) {
          color[u] = 1 - color[v];
          q.push(u);
        } else if (color[u] == color[v]) {
          bip = false;
          break;
        }
      }
    }
    if (!bip) break;
    int c0 = 0;
    for (int v : comp) c0 += (color[v] == 0);
    const int pick = (2 * c0 >= (int)comp.size()) ? 0 : 1;
    for (int v : comp) inP[v] = (color[v] == pick);
  }
  if (!bip) {
    std::fill(inP.begin(), inP.end(), 0);
    std::vector<int> order(n);
    for (int v = 0; v < n; ++v) order[v] = v;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return (krowptr[a + 1] - krowptr[a]) < (krowptr[b + 1] - krowptr[b]);
    });
    std::vector<char> blocked(n, 0);
    for (int v : order) {
      if (blocked[v]) continue;
      inP[v] = 1;
      for (int t = krowptr[v]; t < krowptr[v + 1]; ++t) blocked[kcol[t]] = 1;
    }
  }
  SchurPlanHost& P = *out;
  P = SchurPlanHost{};
  std::vector<int> pidx(n, -1), ridx(n, -1);
  for (int v = 0; v < n; ++v) {
    if (inP[v]) { pidx[v] = (int)P.pverts.size(); P.pverts.push_back(v); }
    else { ridx[v] = (int)P.rverts.size(); P.rverts.push_back(v); }
  }
  const int nnzK = krowptr[n];
  P.stype.assign(nnzK, 0);
  P.sa.assign(nnzK, 0);
  P.sb.assign(nnzK, 0);
  P.bptr.assign(P.pverts.size() + 1, 0);
  std::vector<int> bslot_of(nnzK, -1);
  for (int x = 0; x < n; ++x) {
    for (int s = krowptr[x]; s < krowptr[x + 1]; ++s) {
      const int y = kcol[s];
      if (pidx[x] >= 0 && y == x) {
        P.stype[s] = 1; P.sa[s] = pidx[x];
      } else if (pidx[x] >= 0) {          // y in R (P is independent)
        const int bi = (int)P.bcol.size();
        bslot_of[s] = bi;
        P.stype[s] = 2; P.sa[s] = bi;
        P.bcol.push_back(ridx[y]);
        P.bp.push_back(pidx[x]);
        P.bptr[pidx[x] + 1]++;
      } else if (pidx[y] >= 0) {
        P.stype[s] = 0;                  // mirror of a B block
      } else {
        P.stype[s] = 3; P.sa[s] = ridx[x]; P.sb[s] = ridx[y];
      }
    }
  }
  for (size_t a = 0; a < P.pverts.size(); ++a) P.bptr[a + 1] += P.bptr[a];
  // transpose lists: for each r in R, the B blocks (a, r)
  P.btptr.assign(P.rverts.size() + 1, 0);
  for (int bi = 0; bi < (int)P.bcol.size(); ++bi) P.btptr[P.bcol[bi] + 1]++;
  for (size_t r = 0; r < P.rverts.size(); ++r) P.btptr[r + 1] += P.btptr[r];
  P.btslot.assign(P.bcol.size(), 0);
  std::vector<int> fill(P.rverts.size(), 0);
  for (int bi = 0; bi < (int)P.bcol.size(); ++bi) {
    const int r = P.bcol[bi];
    P.btslot[P.btptr[r] + fill[r]++] = bi;
  }
  P.bipartite = bip;
}

// ---------------------------------------------------------------------------
// Device: formation and factorisation
// ---------------------------------------------------------------------------
constexpr int KMAX = 8;

// one thread per (slot, l): the k values 2 tau K_(l, l2)[x][y], written to the
// D, B or C target of the slot (mirror slots of B are skipped)
__global__ void k_hat_scatter(int nnzK, int k, const int* __restrict__ kptr, const int* __restrict__ kcon,
                              const int* __restrict__ kcra, const int* __restrict__ kcrb,
                              const double* __restrict__ ginv, const double* __restrict__ au, double two_tau,
                              const int* __restrict__ stype, const int* __restrict__ sa, const int* __restrict__ sb,
                              double* __restrict__ D, double* __restrict__ B, double* __restrict__ Cm, int Rk) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzK * k) return;
  const int s = t / k, l = t % k;
  const int ty = stype[s];
  if (ty == 0) return;
  double acc[KMAX];
#pragma unroll
  for (int l2 = 0; l2 < KMAX; ++l2) acc[l2] = 0.0;
  for (int c = kptr[s]; c < kptr[s + 1]; ++c) {
    const double ga = ginv[kcon[c]] * au[(size_t)kcra[c] * k + l];
    const double* ab = au + (size_t)kcrb[c] * k;
#pragma unroll
    for (int l2 = 0; l2 < KMAX; ++l2)
      if (l2 < k) acc[l2] = fma(ga, ab[l2], acc[l2]);
  }
  double* dst;
  if (ty == 1) dst = D + ((size_t)sa[s] * k + l) * k;
  else if (ty == 2) dst = B + ((size_t)sa[s] * k + l) * k;
  else dst = Cm + ((size_t)sa[s] * k + l) * Rk + (size_t)sb[s] * k;
#pragma unroll
  for (int l2 = 0; l2 < KMAX; ++l2)
    if (l2 < k) dst[l2] = two_tau * acc[l2];
}

// D_a += tau^2 I, then D_a = L_a L_a^T in place (lower), pivots below tau^2
// raised to it (S >= tau^2 I holds exactly); one thread per a.
__global__ void k_hat_factor_D(int np, int k, double tau2, double* __restrict__ D, int* info) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= np) return;
  double L[KMAX][KMAX];
  double* Da = D + (size_t)a * k * k;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) L[i][j] = Da[i * k + j] + ((i == j) ? tau2 : 0.0);
  for (int j = 0; j < k; ++j) {
    double p = L[j][j];
    for (int t = 0; t < j; ++t) p -= L[j][t] * L[j][t];
    if (!(p >= tau2)) {
      atomicAdd(info + 1, 1);
      p = tau2;
    }
    const double ljj = sqrt(p);
    L[j][j] = ljj;
    for (int i = j + 1; i < k; ++i) {
      double v = L[i][j];
      for (int t = 0; t < j; ++t) v -= L[i][t] * L[j][t];
      L[i][j] = v / ljj;
    }
  }
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) Da[i * k + j] = (j <= i) ? L[i][j] : 0.0;
}

// F = L_a^{-1} B_(a,y) in place; one thread per (block, column l2)
__global__ void k_hat_F(int nb, int k, const int* __restrict__ bp, const double* __restrict__ D,
                        double* __restrict__ B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * k) return;
  const int bi = t / k, c = t % k;
  const double* La = D + (size_t)bp[bi] * k * k;
  double* Bb = B + (size_t)bi * k * k;
  double x[KMAX];
  for (int i = 0; i < k; ++i) {
    double v = Bb[i * k + c];
    for (int j = 0; j < i; ++j) v -= La[i * k + j] * x[j];
    x[i] = v / La[i * k + i];
  }
  for (int i = 0; i < k; ++i) Bb[i * k + c] = x[i];
}

// C -= F^T F, lower triangle, one CTA per block row r of C (vertex rverts[r]):
// for every P-neighbour a of r in a fixed order, the blocks F_(a,r)^T F_(a,r')
// for the neighbours r' <= r of a.  Each CTA owns its rows, so the sums need no
// atomics and are the same on every run.
__global__ void __launch_bounds__(256) k_hat_schur_rows(int k, int Rk, const int* __restrict__ btptr,
                                                        const int* __restrict__ btslot, const int* __restrict__ bp,
                                                        const int* __restrict__ bptr, const int* __restrict__ bcol,
                                                        const double* __restrict__ F, double* __restrict__ Cm) {
  const int r = blockIdx.x;
  const int kk = k * k;
  for (int e = btptr[r]; e < btptr[r + 1]; ++e) {
    const int bi = btslot[e];
    const int a = bp[bi];
    const int b0 = bptr[a], deg = bptr[a + 1] - b0;
    const double* Fr = F + (size_t)bi * kk;
    for (int t = threadIdx.x; t < deg * kk; t += blockDim.x) {
      const int j = t / kk, l = (t % kk) / k, l2 = t % k;
      const int r2 = bcol[b0 + j];
      if (r2 > r || (r2 == r && l2 > l)) continue;
      const double* Fj = F + (size_t)(b0 + j) * kk;
      double v = 0.0;
      for (int q = 0; q < k; ++q) v = fma(Fr[q * k + l], Fj[q * k + l2], v);
      double* c = Cm + (size_t)(r * k + l) * Rk + (size_t)r2 * k + l2;
      *c -= v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Device: apply pieces (u and the result in the k x n layout u[l n + c])
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fwdP_body(int a, int np, int n, int k, const int* __restrict__ pverts,
                                          const double* __restrict__ D, const double* __restrict__ u,
                                          double* __restrict__ yP) {
  if (a >= np) return;
  const double* La = D + (size_t)a * k * k;
  const int v = pverts[a];
  double x[KMAX];
  for (int i = 0; i < k; ++i) {
    double s = u[(size_t)i * n + v];
    for (int j = 0; j < i; ++j) s -= La[i * k + j] * x[j];
    x[i] = s / La[i * k + i];
    yP[(size_t)a * k + i] = x[i];
  }
}
__global__ void k_hat_fwdP(int np, int n, int k, const int* __restrict__ pverts, const double* __restrict__ D,
                           const double* __restrict__ u, double* __restrict__ yP) {
  fwdP_body(blockIdx.x * blockDim.x + threadIdx.x, np, n, k, pverts, D, u, yP);
}

__device__ __forceinline__ double hs_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// tR[r k + l2] = u[l2 n + rverts[r]] - sum over blocks (a, r) of (F^T y_a)[l2];
// one warp per r, lanes over the blocks
__device__ __forceinline__ void fwdR_body(int r, int lane, int nr, int n, int k, const int* __restrict__ rverts,
                                          const int* __restrict__ btptr, const int* __restrict__ btslot,
                                          const int* __restrict__ bp, const double* __restrict__ F,
                                          const double* __restrict__ yP, const double* __restrict__ u,
                                          double* __restrict__ tR, float* __restrict__ tRf = nullptr) {
  if (r >= nr) return;
  double acc[KMAX];
#pragma unroll
  for (int c = 0; c < KMAX; ++c) acc[c] = 0.0;
  for (int e = btptr[r] + lane; e < btptr[r + 1]; e += 32) {
    const int bi = btslot[e];
    const double* Fb = F + (size_t)bi * k * k;
    const double* ya = yP + (size_t)bp[bi] * k;
    for (int i = 0; i < k; ++i) {
      const double yi = ya[i];
#pragma unroll
      for (int c = 0; c < KMAX; ++c)
        if (c < k) acc[c] = fma(Fb[i * k + c], yi, acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < KMAX; ++c) {
    if (c >= k) break;
    const double s = hs_warp_sum(acc[c]);
    if (lane == 0) {
      const double t = u[(size_t)c * n + rverts[r]] - s;
      tR[(size_t)r * k + c] = t;
      if (tRf) tRf[(size_t)r * k + c] = (float)t;
    }
  }
}
__global__ void k_hat_fwdR(int nr, int n, int k, const int* __restrict__ rverts, const int* __restrict__ btptr,
                           const int* __restrict__ btslot, const int* __restrict__ bp, const double* __restrict__ F,
                           const double* __restrict__ yP, const double* __restrict__ u, double* __restrict__ tR,
                           float* __restrict__ tRf) {
  fwdR_body((blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, nr, n, k, rverts, btptr, btslot, bp, F,
            yP, u, tR, tRf);
}

// y = A x for a triangular A (lower: columns 0..r of row r; upper: r..n-1), one
// warp per row (the two dense solves with the Schur factor: L_C^{-1} and its
// transpose, each stored row-major)
__device__ __forceinline__ void tri_gemv_body(int r, int lane, int n, bool lower, const double* __restrict__ A,
                                              const double* __restrict__ x, double* __restrict__ y) {
  if (r >= n) return;
  const int c0 = lower ? 0 : r, c1 = lower ? r + 1 : n;
  const double* ar = A + (size_t)r * n;
  double s = 0.0;
  for (int c = c0 + lane; c < c1; c += 32) s = fma(ar[c], x[c], s);
  s = hs_warp_sum(s);
  if (lane == 0) y[r] = s;
}
__global__ void k_tri_gemv(int n, int lower, const double* __restrict__ A, const double* __restrict__ x,
                           double* __restrict__ y) {
  tri_gemv_body((blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, n, lower != 0, A, x, y);
}
// The same product from the FP32 copy of the factor inverse with FP32 inputs and
// FP32 accumulation (reduced-precision applies; the FP64 pipe of this GPU would
// otherwise bound the product, and the float copy halves the bytes read).  The
// result goes to yf (float) or, when yf is null, to yd (double).
__device__ __forceinline__ float hs_warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ void tri_gemv32_body(int r, int lane, int n, bool lower, const float* __restrict__ A,
                                                const float* __restrict__ x, float* __restrict__ yf,
                                                double* __restrict__ yd) {
  if (r >= n) return;
  const int c0 = lower ? 0 : r, c1 = lower ? r + 1 : n;
  const float* ar = A + (size_t)r * n;
  float s = 0.f;
  for (int c = c0 + lane; c < c1; c += 32) s = fmaf(ar[c], x[c], s);
  s = hs_warp_sum_f(s);
  if (lane == 0) {
    if (yf) yf[r] = s;
    else yd[r] = (double)s;
  }
}
__global__ void k_tri_gemv32(int n, int lower, const float* __restrict__ A, const float* __restrict__ x,
                             float* __restrict__ yf, double* __restrict__ yd) {
  tri_gemv32_body((blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, n, lower != 0, A, x, yf, yd);
}

// x_a = L_a^{-T}(y_a - F_a x_R); out[pverts[a] k + l] = scale x_a[l]; one warp per a
__device__ __forceinline__ void bwdP_body(int a, int lane, int np, int k, const int* __restrict__ pverts,
                                          const int* __restrict__ bptr, const int* __restrict__ bcol,
                                          const double* __restrict__ F, const double* __restrict__ D,
                                          const double* __restrict__ yP, const double* __restrict__ xR,
                                          double scale, double* __restrict__ out) {
  if (a >= np) return;
  double acc[KMAX];
#pragma unroll
  for (int i = 0; i < KMAX; ++i) acc[i] = 0.0;
  for (int bi = bptr[a] + lane; bi < bptr[a + 1]; bi += 32) {
    const double* Fb = F + (size_t)bi * k * k;
    const double* xr = xR + (size_t)bcol[bi] * k;
    for (int c = 0; c < k; ++c) {
      const double xc = xr[c];
#pragma unroll
      for (int i = 0; i < KMAX; ++i)
        if (i < k) acc[i] = fma(Fb[i * k + c], xc, acc[i]);
    }
  }
  double z[KMAX];
#pragma unroll
  for (int i = 0; i < KMAX; ++i) z[i] = (i < k) ? yP[(size_t)a * k + i] - hs_warp_sum(acc[i]) : 0.0;
  if (lane != 0) return;
  const double* La = D + (size_t)a * k * k;
  const int v = pverts[a];
  for (int i = k - 1; i >= 0; --i) {
    double s = z[i];
    for (int j = i + 1; j < k; ++j) s -= La[j * k + i] * z[j];
    z[i] = s / La[i * k + i];
    out[(size_t)v * k + i] = scale * z[i];
  }
}
__global__ void k_hat_bwdP(int np, int n, int k, const int* __restrict__ pverts, const int* __restrict__ bptr,
                           const int* __restrict__ bcol, const double* __restrict__ F, const double* __restrict__ D,
                           const double* __restrict__ yP, const double* __restrict__ xR, double scale,
                           double* __restrict__ out) {
  (void)n;
  bwdP_body((blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, np, k, pverts, bptr, bcol, F, D, yP, xR,
            scale, out);
}

__device__ __forceinline__ void outR_body(int t, int nr, int k, const int* __restrict__ rverts,
                                          const double* __restrict__ xR, double scale, double* __restrict__ out) {
  if (t >= nr * k) return;
  const int r = t / k, l = t % k;
  out[(size_t)rverts[r] * k + l] = scale * xR[t];
}
__global__ void k_hat_outR(int nr, int k, const int* __restrict__ rverts, const double* __restrict__ xR,
                           double scale, double* __restrict__ out) {
  outR_body(blockIdx.x * blockDim.x + threadIdx.x, nr, k, rverts, xR, scale, out);
}

// ---------------------------------------------------------------------------
// Split ranks above KMAX (up to SDP_K_MAX, the adaptive rank of Section V's
// implementation notes): the same formation, factorisation and solve with the
// k x k blocks in shared memory or spread over a warp's lanes instead of one
// thread's registers.  Only single problems use them (batches keep k <= KMAX).
// ---------------------------------------------------------------------------
constexpr int KGEN = SDP_K_MAX;

// one thread per (slot, l, l2): 2 tau K_(l, l2)[x][y] into the D, B or C target
__global__ void k_hat_scatter_gen(int nnzK, int k, const int* __restrict__ kptr, const int* __restrict__ kcon,
                                  const int* __restrict__ kcra, const int* __restrict__ kcrb,
                                  const double* __restrict__ ginv, const double* __restrict__ au, double two_tau,
                                  const int* __restrict__ stype, const int* __restrict__ sa,
                                  const int* __restrict__ sb, double* __restrict__ D, double* __restrict__ B,
                                  double* __restrict__ Cm, int Rk) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t kk = (size_t)k * k;
  if (t >= (size_t)nnzK * kk) return;
  const int s = (int)(t / kk), l = (int)((t % kk) / k), l2 = (int)(t % k);
  const int ty = stype[s];
  if (ty == 0) return;
  double acc = 0.0;
  for (int c = kptr[s]; c < kptr[s + 1]; ++c)
    acc = fma(ginv[kcon[c]] * au[(size_t)kcra[c] * k + l], au[(size_t)kcrb[c] * k + l2], acc);
  double* dst;
  if (ty == 1) dst = D + ((size_t)sa[s] * k + l) * k;
  else if (ty == 2) dst = B + ((size_t)sa[s] * k + l) * k;
  else dst = Cm + ((size_t)sa[s] * k + l) * Rk + (size_t)sb[s] * k;
  dst[l2] = two_tau * acc;
}

// D_a += tau^2 I, then D_a = L_a L_a^T (lower, in place) with the tau^2 pivot
// floor; one CTA per a, the block in shared memory, right-looking by columns.
__global__ void __launch_bounds__(128) k_hat_factor_D_gen(int np, int k, double tau2, double* __restrict__ D,
                                                          int* info) {
  __shared__ double L[KGEN][KGEN + 1];
  const int a = blockIdx.x;
  if (a >= np) return;
  double* Da = D + (size_t)a * k * k;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t / k, j = t % k;
    L[i][j] = Da[t] + ((i == j) ? tau2 : 0.0);
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      double p = L[j][j];
      if (!(p >= tau2)) {
        atomicAdd(info + 1, 1);
        p = tau2;
      }
      L[j][j] = sqrt(p);
    }
    __syncthreads();
    const double r = 1.0 / L[j][j];
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) L[i][j] *= r;
    __syncthreads();
    const int rem = k - j - 1;
    for (int t = threadIdx.x; t < rem * rem; t += blockDim.x) {
      const int i = j + 1 + t / rem, c = j + 1 + t % rem;
      if (c <= i) L[i][c] = fma(-L[i][j], L[c][j], L[i][c]);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t / k, j = t % k;
    Da[t] = (j <= i) ? L[i][j] : 0.0;
  }
}

// F = L_a^{-1} B_(a,y) in place; one thread per (block, column)
__global__ void k_hat_F_gen(int nb, int k, const int* __restrict__ bp, const double* __restrict__ D,
                            double* __restrict__ B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * k) return;
  const int bi = t / k, c = t % k;
  const double* La = D + (size_t)bp[bi] * k * k;
  double* Bb = B + (size_t)bi * k * k;
  for (int i = 0; i < k; ++i) {
    double v = Bb[i * k + c];
    for (int j = 0; j < i; ++j) v = fma(-La[i * k + j], Bb[j * k + c], v);   // rows j < i already solved
    Bb[i * k + c] = v / La[i * k + i];
  }
}

// y_a = L_a^{-1} u_a; one warp per a (lane 0 substitutes; the row is short)
__global__ void k_hat_fwdP_gen(int np, int n, int k, const int* __restrict__ pverts, const double* __restrict__ D,
                               const double* __restrict__ u, double* __restrict__ yP) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= np) return;
  const double* La = D + (size_t)a * k * k;
  const int v = pverts[a];
  double* y = yP + (size_t)a * k;
  for (int i = 0; i < k; ++i) {
    double s = u[(size_t)i * n + v];
    for (int j = 0; j < i; ++j) s = fma(-La[i * k + j], y[j], s);
    y[i] = s / La[i * k + i];
  }
}

// tR[r k + c] = u[c n + rverts[r]] - sum over blocks (a, r) of (F^T y_a)[c];
// one warp per r, lane c (and c + 32) over the columns of F
__global__ void k_hat_fwdR_gen(int nr, int n, int k, const int* __restrict__ rverts, const int* __restrict__ btptr,
                               const int* __restrict__ btslot, const int* __restrict__ bp,
                               const double* __restrict__ F, const double* __restrict__ yP,
                               const double* __restrict__ u, double* __restrict__ tR, float* __restrict__ tRf) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= nr) return;
  double a0 = 0.0, a1 = 0.0;
  const int c0 = lane, c1 = lane + 32;
  for (int e = btptr[r]; e < btptr[r + 1]; ++e) {
    const int bi = btslot[e];
    const double* Fb = F + (size_t)bi * k * k;
    const double* ya = yP + (size_t)bp[bi] * k;
    for (int i = 0; i < k; ++i) {
      const double yi = ya[i];
      if (c0 < k) a0 = fma(Fb[i * k + c0], yi, a0);
      if (c1 < k) a1 = fma(Fb[i * k + c1], yi, a1);
    }
  }
  const int v = rverts[r];
  if (c0 < k) {
    const double t = u[(size_t)c0 * n + v] - a0;
    tR[(size_t)r * k + c0] = t;
    if (tRf) tRf[(size_t)r * k + c0] = (float)t;
  }
  if (c1 < k) {
    const double t = u[(size_t)c1 * n + v] - a1;
    tR[(size_t)r * k + c1] = t;
    if (tRf) tRf[(size_t)r * k + c1] = (float)t;
  }
}

// x_a = L_a^{-T}(y_a - F_a x_R); out[pverts[a] k + l] = scale x_a[l]; one warp per
// a: lanes i (and i + 32) over the rows of F, then lane 0 substitutes backwards
__global__ void k_hat_bwdP_gen(int np, int k, const int* __restrict__ pverts, const int* __restrict__ bptr,
                               const int* __restrict__ bcol, const double* __restrict__ F,
                               const double* __restrict__ D, const double* __restrict__ yP,
                               const double* __restrict__ xR, double scale, double* __restrict__ out,
                               double* __restrict__ zbuf) {
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (a >= np) return;
  double a0 = 0.0, a1 = 0.0;
  const int i0 = lane, i1 = lane + 32;
  if (xR) {
    for (int bi = bptr[a]; bi < bptr[a + 1]; ++bi) {
      const double* Fb = F + (size_t)bi * k * k;
      const double* xr = xR + (size_t)bcol[bi] * k;
      for (int c = 0; c < k; ++c) {
        const double xc = xr[c];
        if (i0 < k) a0 = fma(Fb[i0 * k + c], xc, a0);
        if (i1 < k) a1 = fma(Fb[i1 * k + c], xc, a1);
      }
    }
  }
  double* z = zbuf + (size_t)a * k;   // y_a - F_a x_R, then x_a
  const double* ya = yP + (size_t)a * k;
  if (i0 < k) z[i0] = ya[i0] - a0;
  if (i1 < k) z[i1] = ya[i1] - a1;
  __syncwarp();
  if (lane != 0) return;
  const double* La = D + (size_t)a * k * k;
  const int v = pverts[a];
  for (int i = k - 1; i >= 0; --i) {
    double s = z[i];
    for (int j = i + 1; j < k; ++j) s = fma(-La[j * k + i], z[j], s);
    z[i] = s / La[i * k + i];
    out[(size_t)v * k + i] = scale * z[i];
  }
}

// ---------------------------------------------------------------------------
// Batched forms of the core solve (one launch each for every problem of a batch)
// ---------------------------------------------------------------------------
#define HS_BATCH_PROLOGUE                                  \
  const int inst = batch_find(off, N, blockIdx.x);         \
  const BDesc& Dd = desc[inst];                            \
  if (!Dd.active) return;                                  \
  const int lb = blockIdx.x - off[inst];

__global__ void kb_fwdP(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  HS_BATCH_PROLOGUE
  fwdP_body(lb * blockDim.x + threadIdx.x, Dd.np, Dd.n, Dd.k, Dd.pverts, Dd.D, Dd.uvec, Dd.yP);
}
__global__ void kb_fwdR(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  HS_BATCH_PROLOGUE
  fwdR_body((lb * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, Dd.nr, Dd.n, Dd.k, Dd.rverts, Dd.btptr,
            Dd.btslot, Dd.bp, Dd.F, Dd.yP, Dd.uvec, Dd.v1, Dd.lpc ? Dd.v1f : nullptr);
}
__global__ void kb_gemv_lower(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  HS_BATCH_PROLOGUE
  if (Dd.lpc)
    tri_gemv32_body((lb * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, Dd.Rk, true, Dd.Cinv32, Dd.v1f, Dd.v2f,
                    nullptr);
  else
    tri_gemv_body((lb * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, Dd.Rk, true, Dd.Cinv, Dd.v1, Dd.v2);
}
__global__ void kb_gemv_upper(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  HS_BATCH_PROLOGUE
  if (Dd.lpc)
    tri_gemv32_body((lb * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, Dd.Rk, false, Dd.CinvT32, Dd.v2f,
                    nullptr, Dd.v1);
  else
    tri_gemv_body((lb * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, Dd.Rk, false, Dd.CinvT, Dd.v2, Dd.v1);
}
__global__ void kb_outR(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  HS_BATCH_PROLOGUE
  outR_body(lb * blockDim.x + threadIdx.x, Dd.nr, Dd.k, Dd.rverts, Dd.v1, Dd.zscale, Dd.Bn);
}
// The last step of the core solve in one launch: the first ceil(Rk / 256)
// blocks of a problem scatter x_R (outR), the rest substitute on the P rows
// (bwdP); both only read x_R.
__global__ void kb_out_bwd(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  HS_BATCH_PROLOGUE
  const int nout = (Dd.Rk + 255) / 256;
  if (lb < nout) outR_body(lb * blockDim.x + threadIdx.x, Dd.nr, Dd.k, Dd.rverts, Dd.v1, Dd.zscale, Dd.Bn);
  else
    bwdP_body(((lb - nout) * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, Dd.np, Dd.k, Dd.pverts, Dd.bptr,
              Dd.bcol, Dd.F, Dd.D, Dd.yP, Dd.v1, Dd.zscale, Dd.Bn);
}
int batch_blocks_out_bwd(int Rk, int np) { return (int)(cdiv(Rk, 256) + cdiv((size_t)np * 32, 256)); }
__global__ void kb_bwdP(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  HS_BATCH_PROLOGUE
  bwdP_body((lb * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, Dd.np, Dd.k, Dd.pverts, Dd.bptr, Dd.bcol, Dd.F,
            Dd.D, Dd.yP, Dd.v1, Dd.zscale, Dd.Bn);
}
int batch_blocks_fwdP(int np) { return (int)cdiv(np, 128); }
int batch_blocks_warp_rows(int rows) { return (int)cdiv((size_t)rows * 32, 256); }
int batch_blocks_outR(int Rk) { return (int)cdiv(Rk, 128); }
void batch_launch_core_solve(cudaStream_t st, const BDesc* desc, int N, const int* off_fwdP, int nb_fwdP,
                             const int* off_fwdR, int nb_fwdR, const int* off_gemv, int nb_gemv,
                             const int* off_outR, int nb_outR, const int* off_bwdP, int nb_bwdP) {
  // a batch with no rows of a kind (e.g. no vertex outside the independent
  // set) launches nothing for it: a grid of zero blocks is not a launch
  if (nb_fwdP > 0) {
    count_launch();
    kb_fwdP<<<nb_fwdP, 128, 0, st>>>(desc, off_fwdP, N);
  }
  if (nb_fwdR > 0) {
    count_launch();
    kb_fwdR<<<nb_fwdR, 256, 0, st>>>(desc, off_fwdR, N);
  }
  if (nb_gemv > 0) {
    count_launch(2);
    kb_gemv_lower<<<nb_gemv, 256, 0, st>>>(desc, off_gemv, N);
    kb_gemv_upper<<<nb_gemv, 256, 0, st>>>(desc, off_gemv, N);
  }
  // off_outR / nb_outR: the merged out_bwd partition (batch_blocks_out_bwd)
  (void)off_bwdP;
  (void)nb_bwdP;
  if (nb_outR > 0) {
    count_launch();
    kb_out_bwd<<<nb_outR, 256, 0, st>>>(desc, off_outR, N);
  }
}

// ---------------------------------------------------------------------------
// Host entry points
// ---------------------------------------------------------------------------
// Buffers of the factorisation for split rank k.  With the adaptive rank the
// rank changes between builds: the buffers are sized for the largest rank seen
// so far and reallocated (old ones released) only when a build needs more.
sdp_status schur_alloc(sdp_problem* h, int k) {
  const size_t np = h->hs_np, nb = h->hs_nb, Rk = (size_t)h->hs_nr * k;
  h->hs_k = k;   // trmv partials: h->trpart holds those of order n k >= R k
  if (h->hs_D && k <= h->hs_kcap) return SDP_OK;   // every buffer was sized for hs_kcap >= k
  for (double** b : {&h->hs_D, &h->hs_F, &h->hs_yP, &h->hs_C, &h->hs_Cinv, &h->hs_CinvT, &h->hs_v1, &h->hs_v2,
                     &h->hs_v3}) {
    h->release(*b);
    *b = nullptr;
  }
  SDP_TRY(h->allocT(&h->hs_D, std::max<size_t>(np * k * k, 1)));
  SDP_TRY(h->allocT(&h->hs_F, std::max<size_t>(nb * k * k, 1)));
  SDP_TRY(h->allocT(&h->hs_yP, std::max<size_t>(np * k, 1)));
  SDP_TRY(h->allocT(&h->hs_C, std::max<size_t>(Rk * Rk, 1)));
  SDP_TRY(h->allocT(&h->hs_Cinv, std::max<size_t>(Rk * Rk, 1)));
  SDP_TRY(h->allocT(&h->hs_CinvT, std::max<size_t>(Rk * Rk, 1)));
  SDP_TRY(h->allocT(&h->hs_v1, std::max<size_t>(Rk, 1)));
  SDP_TRY(h->allocT(&h->hs_v2, std::max<size_t>(Rk, 1)));
  SDP_TRY(h->allocT(&h->hs_v3, std::max<size_t>(std::max(Rk, np * k), 1)));
  const size_t wneed = std::max(potrf_work_doubles((int)Rk), trsm_work_doubles((int)Rk, (int)Rk));
  if (wneed > h->work_doubles) {
    h->release(h->work);
    h->work = nullptr;
    SDP_TRY(h->allocT(&h->work, wneed));
    h->work_doubles = wneed;
  }
  h->hs_cap = Rk;
  h->hs_kcap = k;
  return SDP_OK;
}

// Core of Hhat (needs h->au = A_i u_l on the support rows) -> L_P, F, L_C, L_C^{-1}.
sdp_status schur_build(sdp_problem* h, int k, double tau) {
  if (k > KGEN) {
    h->last_error = "precond_build: the sparse Hhat core supports k <= SDP_K_MAX";
    return SDP_ERR_UNSUPPORTED;
  }
  SDP_TRY(schur_alloc(h, k));
  const bool gen = k > KMAX;
  cudaStream_t st = h->stream;
  const int np = h->hs_np, nr = h->hs_nr, nb = h->hs_nb, Rk = nr * k;
  const double tau2 = tau * tau;
  fill(st, h->hs_D, (size_t)np * k * k, 0.0);
  if (Rk > 0) fill(st, h->hs_C, (size_t)Rk * Rk, 0.0);
  cudaMemsetAsync(h->info, 0, 2 * sizeof(int), st);
  count_launch();
  if (gen)
    k_hat_scatter_gen<<<cdiv((size_t)h->nnzK * k * k, 128), 128, 0, st>>>(
        h->nnzK, k, h->kptr, h->kcon, h->kcra, h->kcrb, h->ginv, h->au, 2.0 * tau, h->hs_stype, h->hs_sa, h->hs_sb,
        h->hs_D, h->hs_F, h->hs_C, Rk);
  else
    k_hat_scatter<<<cdiv((size_t)h->nnzK * k, 128), 128, 0, st>>>(h->nnzK, k, h->kptr, h->kcon, h->kcra, h->kcrb,
                                                                 h->ginv, h->au, 2.0 * tau, h->hs_stype, h->hs_sa,
                                                                 h->hs_sb, h->hs_D, h->hs_F, h->hs_C, Rk);
  if (np > 0) {
    count_launch();
    if (gen) k_hat_factor_D_gen<<<np, 128, 0, st>>>(np, k, tau2, h->hs_D, h->info);
    else k_hat_factor_D<<<cdiv(np, 128), 128, 0, st>>>(np, k, tau2, h->hs_D, h->info);
  }
  if (nb > 0) {
    count_launch(2);
    if (gen) k_hat_F_gen<<<cdiv((size_t)nb * k, 128), 128, 0, st>>>(nb, k, h->hs_bp, h->hs_D, h->hs_F);
    else k_hat_F<<<cdiv((size_t)nb * k, 128), 128, 0, st>>>(nb, k, h->hs_bp, h->hs_D, h->hs_F);
    k_hat_schur_rows<<<nr, 256, 0, st>>>(k, Rk, h->hs_btptr, h->hs_btslot, h->hs_bp, h->hs_bptr, h->hs_bcol,
                                         h->hs_F, h->hs_C);
  }
  int floored = 0;
  if (Rk > 0) {
    add_diag(st, Rk, h->hs_C, Rk, tau2);
    // a Schur complement of S >= tau^2 I is >= tau^2 I as well
    int inf0[2] = {0, 0};
    SDP_CK(h, cudaMemcpyAsync(inf0, h->info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    SDP_CK(h, cudaStreamSynchronize(st));
    floored = inf0[1];
    potrf_floor(st, Rk, h->hs_C, Rk, h->info, h->work, tau2);
    fill(st, h->hs_Cinv, (size_t)Rk * Rk, 0.0);
    add_diag(st, Rk, h->hs_Cinv, Rk, 1.0);
    trsm_left_lower_ex(st, false, Rk, Rk, h->hs_C, Rk, h->hs_Cinv, Rk, h->work, true);
    transpose(st, Rk, Rk, h->hs_Cinv, Rk, h->hs_CinvT, Rk);
  }
  int inf2[2] = {0, 0};
  SDP_CK(h, cudaMemcpyAsync(inf2, h->info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaStreamSynchronize(st));
  h->core_floor_pivots = floored + inf2[1];
  return SDP_OK;
}

// FP32 copies of L_C^{-1} and its transpose (and float work vectors), made once
// per preconditioner build when a reduced-precision apply first needs them.
sdp_status ensure_lowprec_core(sdp_problem* h) {
  if (!h->pc_valid || !h->pc_hat) return SDP_OK;
  const size_t Rk = (size_t)h->hs_nr * h->hs_k;
  if (Rk == 0 || h->hs_lp_gen == h->pc_generation) return SDP_OK;
  if (!h->hs_Cinv32 || h->hs_lp_cap < Rk) {
    for (float** b : {&h->hs_Cinv32, &h->hs_CinvT32, &h->hs_v1f, &h->hs_v2f}) {
      h->release(*b);
      *b = nullptr;
    }
    SDP_TRY(h->allocT(&h->hs_Cinv32, Rk * Rk));
    SDP_TRY(h->allocT(&h->hs_CinvT32, Rk * Rk));
    SDP_TRY(h->allocT(&h->hs_v1f, Rk));
    SDP_TRY(h->allocT(&h->hs_v2f, Rk));
    h->hs_lp_cap = Rk;
  }
  to_f32(h->stream, Rk * Rk, h->hs_Cinv, h->hs_Cinv32);
  to_f32(h->stream, Rk * Rk, h->hs_CinvT, h->hs_CinvT32);
  h->hs_lp_gen = h->pc_generation;
  return SDP_OK;
}

// out = scale S^{-1} u with u in the k x n layout u[l n + c] and out in the
// n x k layout out[c k + l]; u is not modified.  The dense solves take no
// refinement step: the Hhat core stays well enough conditioned (kappa ~ 1/mu)
// for the explicit inverse of the Schur factor.  With prec != SDP_FP64 the two
// dense products use the FP32 copy of that inverse (ensure_lowprec_core).
sdp_status schur_apply(sdp_problem* h, const double* u, double* out, double scale, int prec) {
  cudaStream_t st = h->stream;
  const int n = h->n, k = h->hs_k, np = h->hs_np, nr = h->hs_nr, Rk = nr * k;
  const bool lp = (prec != SDP_FP64) && Rk > 0;
  const bool gen = k > KMAX;
  if (lp) SDP_TRY(ensure_lowprec_core(h));
  if (np > 0) {
    count_launch();
    if (gen) k_hat_fwdP_gen<<<cdiv(np, 128), 128, 0, st>>>(np, n, k, h->hs_pverts, h->hs_D, u, h->hs_yP);
    else k_hat_fwdP<<<cdiv(np, 128), 128, 0, st>>>(np, n, k, h->hs_pverts, h->hs_D, u, h->hs_yP);
  }
  if (Rk > 0) {
    count_launch();
    if (gen)
      k_hat_fwdR_gen<<<cdiv((size_t)nr * 32, 256), 256, 0, st>>>(nr, n, k, h->hs_rverts, h->hs_btptr, h->hs_btslot,
                                                                  h->hs_bp, h->hs_F, h->hs_yP, u, h->hs_v1,
                                                                  lp ? h->hs_v1f : nullptr);
    else
      k_hat_fwdR<<<cdiv((size_t)nr * 32, 256), 256, 0, st>>>(nr, n, k, h->hs_rverts, h->hs_btptr, h->hs_btslot,
                                                              h->hs_bp, h->hs_F, h->hs_yP, u, h->hs_v1,
                                                              lp ? h->hs_v1f : nullptr);
    // y_R = L_C^{-1} t_R and x_R = L_C^{-T} y_R (both inverses stored row-major)
    count_launch(2);
    if (lp) {
      k_tri_gemv32<<<cdiv((size_t)Rk * 32, 256), 256, 0, st>>>(Rk, 1, h->hs_Cinv32, h->hs_v1f, h->hs_v2f, nullptr);
      k_tri_gemv32<<<cdiv((size_t)Rk * 32, 256), 256, 0, st>>>(Rk, 0, h->hs_CinvT32, h->hs_v2f, nullptr, h->hs_v1);
    } else {
      k_tri_gemv<<<cdiv((size_t)Rk * 32, 256), 256, 0, st>>>(Rk, 1, h->hs_Cinv, h->hs_v1, h->hs_v2);
      k_tri_gemv<<<cdiv((size_t)Rk * 32, 256), 256, 0, st>>>(Rk, 0, h->hs_CinvT, h->hs_v2, h->hs_v1);
    }
    count_launch();
    k_hat_outR<<<cdiv(Rk, 128), 128, 0, st>>>(nr, k, h->hs_rverts, h->hs_v1, scale, out);
  }
  if (np > 0) {
    const double* xR = (Rk > 0) ? h->hs_v1 : nullptr;
    count_launch();
    if (gen)
      k_hat_bwdP_gen<<<cdiv((size_t)np * 32, 256), 256, 0, st>>>(np, k, h->hs_pverts, h->hs_bptr, h->hs_bcol,
                                                                  h->hs_F, h->hs_D, h->hs_yP, xR, scale, out,
                                                                  h->hs_v3);
    else
      k_hat_bwdP<<<cdiv((size_t)np * 32, 256), 256, 0, st>>>(np, n, k, h->hs_pverts, h->hs_bptr, h->hs_bcol,
                                                              h->hs_F, h->hs_D, h->hs_yP, xR, scale, out);
  }
  return SDP_OK;
}

}  // namespace sdpgb
