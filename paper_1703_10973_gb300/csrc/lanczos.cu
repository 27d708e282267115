// Smallest eigenvalue of a dense symmetric matrix by Lanczos, in one
// thread-block cluster (the step-length test of the interior-point method
// needs lambda_min(L^{-1} dX L^{-T}) only, not a full spectrum).
//
// Lanczos with full reorthogonalisation (two classical Gram-Schmidt passes per
// step) builds the tridiagonal T_j = Q_j^T M Q_j.  The Ritz value theta =
// lambda_min(T_j) is never below lambda_min(M), and the residual of its Ritz
// vector is beta_j |s_j| (s the unit eigenvector of T_j for theta, s_j its last
// entry), so some eigenvalue of M lies in [theta - beta_j |s_j|, theta].  The
// iteration stops when that bound is small against |theta| and returns the
// conservative estimate theta - beta_j |s_j|, which can only shorten a step.
//
// The operator is M itself, or M = A1 A2 A3 applied as three products
// (the step length uses L^{-1} dX L^{-T} this way, from the explicit inverse of
// the Cholesky factor, without forming M).
//
// Layout: the LZ_CS CTAs of the cluster split the rows of each product
// w = M q (cyclically, for balance with triangular factors); each CTA writes its slice of w into every CTA's shared memory
// (distributed shared memory), and after one cluster barrier every CTA holds
// the whole w and performs the O(j n) vector work redundantly, so all CTAs
// compute bit-identical q, alpha, beta and take the same branches.  Each CTA
// keeps its own copy of the Lanczos basis in global memory (no cross-CTA
// visibility is needed for it).  One cluster barrier per step; w is double
// buffered so a CTA that runs ahead into step j+1 never overwrites the buffer
// a slower CTA still reads in step j.
#include "internal.cuh"

#include <cooperative_groups.h>

#include <cfloat>

#include <algorithm>
#include <cmath>

namespace cg = cooperative_groups;

namespace sdpgb {

constexpr int LZ_CS = 8;        // CTAs per cluster (portable cluster size)
constexpr int LZ_THREADS = 256;
constexpr int LZ_MAXIT = 120;   // Lanczos steps at most
constexpr int LZ_CHECK = 6;     // convergence test every LZ_CHECK steps

__device__ __forceinline__ double lz_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; every thread receives the result (red: 32 doubles of smem)
__device__ double lz_block_sum(double v, double* red) {
  v = lz_warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// deterministic start vector entry (splitmix64 of the index, mapped to [-1, 1])
__device__ __forceinline__ double lz_start(int i) {
  unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-52 - 1.0;
}

// Sturm count of T (diagonal a[0..j), off-diagonal b[0..j-1)) below x
__device__ int lz_sturm(int j, const double* a, const double* b, double x) {
  double pm = 1.0, p = a[0] - x;
  int sp = (p > 0.0) ? 1 : -1;
  int cnt = (sp < 0) ? 1 : 0;
  for (int i = 1; i < j; ++i) {
    const double pn = fma(a[i] - x, p, -b[i - 1] * b[i - 1] * pm);
    const int sn = (pn > 0.0) ? 1 : (pn < 0.0 ? -1 : -sp);
    cnt += (sn != sp);
    sp = sn;
    pm = p;
    p = pn;
    const double m = fmax(fabs(p), fabs(pm));
    if (m > 0x1p+400) { p *= 0x1p-400; pm *= 0x1p-400; }
    else if (m < 0x1p-400 && m > 0.0) { p *= 0x1p+400; pm *= 0x1p+400; }
  }
  return cnt;
}

// One warp: theta = lambda_min(T_j) by 32-way multisection, then the last
// entry of its unit eigenvector by two steps of inverse iteration (lane 0).
// res[0] = theta, res[1] = |s_last|.
__device__ void lz_ritz_min(int j, const double* a, const double* b, double* res, double* work) {
  const int lane = threadIdx.x & 31;
  double lo = a[0], hi = a[0];
  for (int i = 0; i < j; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < j ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  const double pad = 4.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) * j + DBL_MIN;
  lo -= pad;
  hi += pad;
  for (int it = 0; it < 14; ++it) {
    const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    const int c = lz_sturm(j, a, b, x);
    const unsigned ge = __ballot_sync(0xffffffffu, c >= 1);
    if (ge == 0u) {
      lo = lo + (hi - lo) * 32.0 / 33.0;
    } else {
      const int f = __ffs(ge) - 1;
      const double nh = lo + (hi - lo) * (double)(f + 1) / 33.0;
      const double nl = (f == 0) ? lo : lo + (hi - lo) * (double)f / 33.0;
      lo = nl;
      hi = nh;
    }
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi))) break;
  }
  if (lane == 0) {
    const double theta = 0.5 * (lo + hi);
    // inverse iteration: (T - theta I) s = s_prev, Gaussian elimination with
    // partial pivoting on the tridiagonal (work: 4 j doubles)
    double* s = work;
    double* dd = work + j;       // diagonal after elimination
    double* du = work + 2 * j;   // first superdiagonal
    double* du2 = work + 3 * j;  // second superdiagonal (from pivoting)
    const double tiny = fmax(fabs(theta), 1.0) * 1e-300 + DBL_MIN;
    for (int i = 0; i < j; ++i) s[i] = 1.0;
    for (int rep = 0; rep < 2; ++rep) {
      // factor rows in place into upper band (dd, du, du2), apply to s
      double cd = a[0] - theta, cu = (j > 1) ? b[0] : 0.0;
      for (int i = 0; i < j; ++i) {
        if (i + 1 < j) {
          const double sub = b[i];
          const double nd = a[i + 1] - theta;
          const double nu = (i + 2 < j) ? b[i + 1] : 0.0;
          if (fabs(cd) >= fabs(sub)) {
            const double piv = (cd != 0.0) ? cd : tiny;
            const double l = sub / piv;
            dd[i] = piv; du[i] = cu; du2[i] = 0.0;
            s[i + 1] -= l * s[i];
            cd = nd - l * cu;
            cu = nu;
          } else {
            const double l = cd / sub;
            dd[i] = sub; du[i] = nd; du2[i] = nu;
            const double t = s[i];
            s[i] = s[i + 1];
            s[i + 1] = t - l * s[i];
            cd = cu - l * nd;
            cu = -l * nu;
          }
        } else {
          dd[i] = (cd != 0.0) ? cd : tiny;
        }
      }
      for (int i = j - 1; i >= 0; --i) {
        double v = s[i];
        if (i + 1 < j) v -= du[i] * s[i + 1];
        if (i + 2 < j) v -= du2[i] * s[i + 2];
        s[i] = v / dd[i];
      }
      double nrm = 0.0;
      for (int i = 0; i < j; ++i) nrm = fmax(nrm, fabs(s[i]));
      const double sc = (nrm > 0.0 && isfinite(nrm)) ? 1.0 / nrm : 0.0;
      for (int i = 0; i < j; ++i) s[i] *= sc;
    }
    double n2 = 0.0;
    for (int i = 0; i < j; ++i) n2 += s[i] * s[i];
    res[0] = theta;
    res[1] = (n2 > 0.0) ? fabs(s[j - 1]) / sqrt(n2) : 1.0;
  }
  __syncwarp();
}

// out = A x for this CTA's rows (row r handled by warp r mod (LZ_CS * warps),
// cyclic over the cluster), each result written into every CTA's `out`
__device__ __forceinline__ void lz_gemv_bcast(cg::cluster_group& cluster, int n, const double* __restrict__ A,
                                              int lda, const double* x, double* out, int rank, int warp,
                                              int lane, int nw) {
  const int stride = LZ_CS * nw;
  for (int r = rank * nw + warp; r < n; r += stride) {
    const double* ar = A + (size_t)r * lda;
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) acc = fma(ar[c], x[c], acc);
    acc = lz_warp_sum(acc);
    if (lane < LZ_CS) {
      double* dst = cluster.map_shared_rank(out, lane);
      dst[r] = acc;
    }
  }
}

// out[0] = conservative lambda_min estimate, out[1] = theta, out[2] = bound,
// out[3] = steps, out[4] = 1 if converged.  Q: LZ_CS * (LZ_MAXIT + 1) * n doubles.
// Converged: bound <= rtol |theta|, or (after 2 LZ_CHECK steps) theta - bound >=
// accept_above (the caller only needs to know that lambda_min is above it).
__global__ void __cluster_dims__(LZ_CS, 1, 1) __launch_bounds__(LZ_THREADS)
    k_lanczos_min(int n, const double* __restrict__ M, const double* __restrict__ A2,
                  const double* __restrict__ A3, int ldm, double rtol, double accept_above,
                  double* __restrict__ Qall, double* __restrict__ out) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double sm[];
  double* q = sm;                 // n
  double* w0 = sm + n;            // n   (double-buffered product)
  double* w1 = sm + 2 * (size_t)n;
  double* qp = sm + 3 * (size_t)n;  // n   previous q
  double* t1 = sm + 4 * (size_t)n;  // n   A3 q   (three-factor operator)
  double* t2 = sm + 5 * (size_t)n;  // n   A2 A3 q
  __shared__ double alpha[LZ_MAXIT], beta[LZ_MAXIT], cdot[LZ_MAXIT + 1];
  __shared__ double red[32], ritz[2], twork[4 * LZ_MAXIT];
  __shared__ int stop;
  const int rank = (int)cluster.block_rank();
  double* Q = Qall + (size_t)rank * (LZ_MAXIT + 1) * n;
  const int maxit = min(LZ_MAXIT, n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;

  // q0: the deterministic start vector, normalised (identical in every CTA)
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = lz_start(i);
    q[i] = v;
    qp[i] = 0.0;
    s = fma(v, v, s);
  }
  s = lz_block_sum(s, red);
  const double inv0 = 1.0 / sqrt(s);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    q[i] *= inv0;
    Q[i] = q[i];
  }
  if (threadIdx.x == 0) stop = 0;
  double bprev = 0.0, theta = 0.0, bound = INFINITY;
  int steps = 0, conv = 0;
  cluster.sync();

  for (int j = 0; j < maxit; ++j) {
    double* wb = (j & 1) ? w1 : w0;
    if (A2) {
      lz_gemv_bcast(cluster, n, A3, ldm, q, t1, rank, warp, lane, nw);
      cluster.sync();
      lz_gemv_bcast(cluster, n, A2, ldm, t1, t2, rank, warp, lane, nw);
      cluster.sync();
      lz_gemv_bcast(cluster, n, M, ldm, t2, wb, rank, warp, lane, nw);
    } else {
      lz_gemv_bcast(cluster, n, M, ldm, q, wb, rank, warp, lane, nw);
    }
    cluster.sync();
    // alpha_j = q . w ;  w -= alpha q + beta_{j-1} q_{j-1}
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(q[i], wb[i], a);
    a = lz_block_sum(a, red);
    for (int i = threadIdx.x; i < n; i += blockDim.x) wb[i] = wb[i] - a * q[i] - bprev * qp[i];
    __syncthreads();
    // full reorthogonalisation against Q rows 0..j, two passes
    for (int pass = 0; pass < 2; ++pass) {
      for (int t = warp; t <= j; t += nw) {
        const double* qt = Q + (size_t)t * n;
        double c = 0.0;
        for (int i = lane; i < n; i += 32) c = fma(qt[i], wb[i], c);
        c = lz_warp_sum(c);
        if (lane == 0) cdot[t] = c;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = wb[i];
        for (int t = 0; t <= j; ++t) v = fma(-cdot[t], Q[(size_t)t * n + i], v);
        wb[i] = v;
      }
      __syncthreads();
    }
    double b2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) b2 = fma(wb[i], wb[i], b2);
    b2 = lz_block_sum(b2, red);
    const double b = sqrt(b2);
    if (threadIdx.x == 0) {
      alpha[j] = a;
      beta[j] = b;
    }
    steps = j + 1;
    __syncthreads();
    const bool invariant = !(b > 1e-14 * fmax(fabs(a), fabs(bprev)) + DBL_MIN);
    if (invariant || steps == maxit || (steps % LZ_CHECK) == 0) {
      if (warp == 0) lz_ritz_min(steps, alpha, beta, ritz, twork);
      __syncthreads();
      theta = ritz[0];
      bound = invariant ? 0.0 : b * ritz[1];
      const bool ok = invariant || bound <= rtol * fabs(theta) ||
                      (steps >= 2 * LZ_CHECK && theta - bound >= accept_above);
      if (threadIdx.x == 0 && (ok || steps == maxit)) stop = 1;
      conv = ok ? 1 : 0;
      __syncthreads();
    }
    if (stop) break;
    // q_{j+1} = w / beta_j
    const double ib = 1.0 / b;
    double* qn = Q + (size_t)(j + 1) * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      qp[i] = q[i];
      const double v = wb[i] * ib;
      q[i] = v;
      qn[i] = v;
    }
    bprev = b;
    __syncthreads();
  }
  if (rank == 0 && threadIdx.x == 0) {
    out[0] = theta - bound;
    out[1] = theta;
    out[2] = bound;
    out[3] = (double)steps;
    out[4] = conv ? 1.0 : 0.0;
  }
  cluster.sync();   // no CTA leaves while another may still write into its shared memory
}

size_t lanczos_work_doubles(int n) { return (size_t)LZ_CS * (LZ_MAXIT + 1) * n + 8; }

// Launch on st; results land in out_dev[0..4] (device).
// Operator M (A2 = A3 = nullptr) or M A2 A3.  Needs 6 n doubles of shared memory per CTA.
bool lanczos_fits(int n) { return n >= 2 && 6 * (size_t)n * sizeof(double) <= 200 * 1024; }

sdp_status lanczos_min(cudaStream_t st, int n, const double* M, const double* A2, const double* A3, int ldm,
                       double rtol, double accept_above, double* work, double* out_dev) {
  const size_t smem = 6 * (size_t)n * sizeof(double);
  if (!lanczos_fits(n) || (A2 == nullptr) != (A3 == nullptr)) return SDP_ERR_UNSUPPORTED;
  allow_max_smem((const void*)k_lanczos_min);
  count_launch();
  ktimer_begin(st, "lanczos");
  k_lanczos_min<<<LZ_CS, LZ_THREADS, smem, st>>>(n, M, A2, A3, ldm, rtol, accept_above, work, out_dev);
  ktimer_end(st, "lanczos", 0.0, 0.0);
  return cudaPeekAtLastError() == cudaSuccess ? SDP_OK : SDP_ERR_CUDA;
}

}  // namespace sdpgb
