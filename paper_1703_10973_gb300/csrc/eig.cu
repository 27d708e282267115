// FP64 symmetric eigensolver for Algorithm 1 step 1 (eig(W)), the NT scaling
// (eig(L^T S L)) and the step-length test (lambda_min).
//
//  1. Householder tridiagonalisation A = Q T Q^T in one cooperative persistent
//     kernel: per column, every CTA rebuilds the reflector from row j (cheap,
//     no barrier), warps own rows for the symmetric matrix-vector product and the
//     rank-2 update; two bounded grid barriers per column.
//  2. Eigenvalues of T by bisection on Sturm counts (one thread per eigenvalue).
//  3. Eigenvectors of T by inverse iteration with a pivoted tridiagonal LU (one
//     thread per eigenvalue, interleaved workspace so that the per-thread
//     sequential sweeps load coalesced).
//  4. Re-orthogonalisation of the eigenvector block by one Cholesky-QR pass
//     (Gram matrix GEMM, Cholesky, triangular solve), which repairs the loss of
//     orthogonality of inverse iteration inside eigenvalue clusters.
//  5. Back-transformation by the stored reflectors (one warp per eigenvector,
//     no inter-CTA communication).
#include "internal.cuh"

#include <cfloat>
#include <algorithm>

namespace sdpgb {

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double bsum(double v, double* sh) {
  v = wsum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < (int)(blockDim.x / 32)) ? sh[l] : 0.0;
    s = wsum(s);
  }
  __syncthreads();
  return s;  // valid in thread 0 (lane 0 of warp 0)
}

// Grid-wide barrier for a cooperative launch.  Every wait is bounded: after
// about two seconds of clock the waiting CTA sets *flag and returns false; all
// CTAs then leave the kernel at their next barrier.
constexpr long long SPIN_CYCLES = 4000000000LL;

__device__ bool grid_barrier(unsigned int* bar, int* flag) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_ok = 1;
    volatile unsigned int* vgen = bar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*(volatile int*)flag) { s_ok = 0; break; }
        if (clock64() - t0 > SPIN_CYCLES) { atomicExch(flag, 1); s_ok = 0; break; }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// 1. Tridiagonalisation (lower; A full symmetric storage, row-major)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sytrd(int n, double* A, int lda, double* d, double* e,
                                               double* tauh, double* p, double* part,
                                               unsigned int* bar, int* flag) {
  extern __shared__ double sm[];
  double* v = sm;       // n
  double* w = sm + n;   // n
  __shared__ double red[32];
  __shared__ double s_tau, s_beta, s_scale, s_K;
  const int wpb = blockDim.x / 32, wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int gwarp = blockIdx.x * wpb + wid, nwarps = gridDim.x * wpb;

  for (int j = 0; j < n - 2; ++j) {
    const int len = n - j - 1;
    const double* row = A + (size_t)j * lda + j + 1;
    // --- reflector H = I - tau v v^T with v[0] = 1 mapping row j onto beta e_1
    double s = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const double x = __ldcg(row + i);
      v[i] = x;
      if (i > 0) s = fma(x, x, s);
    }
    s = bsum(s, red);
    if (threadIdx.x == 0) {
      const double x0 = v[0];
      double tau = 0.0, beta = x0, scale = 0.0;
      if (s > 0.0) {
        beta = -copysign(sqrt(fma(x0, x0, s)), x0);
        tau = (beta - x0) / beta;
        scale = 1.0 / (x0 - beta);
      }
      s_tau = tau; s_beta = beta; s_scale = scale;
    }
    __syncthreads();
    const double tau = s_tau, scale = s_scale;
    for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) v[i] *= scale;
    if (threadIdx.x == 0) v[0] = 1.0;
    __syncthreads();
    // --- p = tau A22 v for the rows this CTA owns; partial sums of p^T v
    double kp = 0.0;
    for (int i = j + 1 + gwarp; i < n; i += nwarps) {
      const double* ai = A + (size_t)i * lda + j + 1;
      double acc = 0.0;
      for (int l = lane; l < len; l += 32) acc = fma(__ldcg(ai + l), v[l], acc);
      acc = wsum(acc) * tau;
      if (lane == 0) {
        p[i] = acc;
        kp = fma(acc, v[i - j - 1], kp);
      }
    }
    kp = bsum(kp, red);
    if (threadIdx.x == 0) part[blockIdx.x] = kp;
    if (!grid_barrier(bar, flag)) return;
    // --- w = p - (tau/2)(p^T v) v ; A22 -= v w^T + w v^T
    if (threadIdx.x == 0) {
      double K = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) K += __ldcg(part + b);
      s_K = 0.5 * tau * K;
    }
    __syncthreads();
    const double K = s_K;
    for (int l = threadIdx.x; l < len; l += blockDim.x) w[l] = __ldcg(p + j + 1 + l) - K * v[l];
    __syncthreads();
    for (int i = j + 1 + gwarp; i < n; i += nwarps) {
      double* ai = A + (size_t)i * lda + j + 1;
      const double vi = v[i - j - 1], wi = w[i - j - 1];
      for (int l = lane; l < len; l += 32) {
        const double x = __ldcg(ai + l);
        ai[l] = x - fma(vi, w[l], wi * v[l]);
      }
    }
    if (blockIdx.x == 0) {
      double* rj = A + (size_t)j * lda + j + 1;
      for (int l = threadIdx.x; l < len; l += blockDim.x) rj[l] = v[l];
      if (threadIdx.x == 0) {
        d[j] = __ldcg(A + (size_t)j * lda + j);
        e[j] = s_beta;
        tauh[j] = tau;
      }
    }
    if (!grid_barrier(bar, flag)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n >= 2) {
      d[n - 2] = __ldcg(A + (size_t)(n - 2) * lda + n - 2);
      e[n - 2] = __ldcg(A + (size_t)(n - 2) * lda + n - 1);
      tauh[n - 2] = 0.0;
    }
    d[n - 1] = __ldcg(A + (size_t)(n - 1) * lda + n - 1);
    e[n - 1] = 0.0;
    if (n >= 2) tauh[n - 1] = 0.0;
  }
}

static int sytrd_blocks(int n, size_t smem) {
  static int cached_sms = 0;
  if (!cached_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sytrd, 256, smem);
  occ = std::max(1, std::min(occ, 2));
  int blocks = cached_sms * occ;
  const int want = (n + 7) / 8;  // 8 warps per CTA, one row per warp is enough
  blocks = std::max(1, std::min(blocks, std::max(want, cached_sms)));
  return std::min(blocks, 4096);
}

static sdp_status sytrd(cudaStream_t st, int n, double* A, EigWork* w) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  if (smem > 200 * 1024) return SDP_ERR_UNSUPPORTED;
  static size_t attr = 0;
  if (smem > 48 * 1024 && smem > attr) {
    cudaFuncSetAttribute(k_sytrd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = smem;
  }
  cudaMemsetAsync(w->bar, 0, 2 * sizeof(unsigned int), st);
  cudaMemsetAsync(w->flag, 0, sizeof(int), st);
  const int blocks = sytrd_blocks(n, smem);
  int lda = n;
  void* args[] = {&n, &A, &lda, &w->d, &w->e, &w->tauh, &w->p, &w->part, &w->bar, &w->flag};
  count_launch();
  ktimer_begin(st, "sytrd");
  cudaError_t err = cudaLaunchCooperativeKernel((void*)k_sytrd, dim3(blocks), dim3(256), args, smem, st);
  // per column: symv 2 len^2 + rank-2 update 4 len^2 flops; the trailing block is read twice, written once
  ktimer_end(st, "sytrd", 2.0 * n * (double)n * n, 8.0 * n * (double)n * n);
  return err == cudaSuccess ? SDP_OK : SDP_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// 2. Bisection
// ---------------------------------------------------------------------------
__device__ __forceinline__ int sturm_count(int n, const double* d, const double* e, double x, double pivmin) {
  // number of eigenvalues of T strictly below x
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < n; ++i) {
    const double ei = e[i - 1];
    q = d[i] - x - (ei * ei) / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

__device__ void gersh(int n, const double* d, const double* e, double* lo, double* hi, double* pivmin) {
  double gl = d[0], gu = d[0], em = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    gl = fmin(gl, d[i] - r);
    gu = fmax(gu, d[i] + r);
    if (i + 1 < n) em = fmax(em, e[i] * e[i]);
  }
  const double tn = fmax(fabs(gl), fabs(gu));
  const double pad = 2.0 * DBL_EPSILON * tn * n + 4.0 * DBL_MIN;
  *lo = gl - pad;
  *hi = gu + pad;
  *pivmin = DBL_MIN * fmax(1.0, em);
}

// w[t] = eigenvalue number idx[t] (ascending, 0-based) of T.
__global__ void k_stebz(int n, const double* d, const double* e, int cnt, const int* idx, int i0, double* wout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int target = idx ? idx[t] : i0 + t;
  double lo, hi, pivmin;
  gersh(n, d, e, &lo, &hi, &pivmin);
  for (int it = 0; it < 256; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 2.0 * pivmin || mid == lo || mid == hi) break;
    if (sturm_count(n, d, e, mid, pivmin) > target) hi = mid; else lo = mid;
  }
  wout[t] = 0.5 * (lo + hi);
}

// Smallest eigenvalue by multisection with one warp (32 Sturm counts per round).
__global__ void k_eigmin_warp(int n, const double* d, const double* e, double* out) {
  __shared__ double s_lo, s_hi;
  __shared__ int cnts[32];
  const int lane = threadIdx.x;
  if (lane == 0) {
    double lo, hi, pm;
    gersh(n, d, e, &lo, &hi, &pm);
    s_lo = lo; s_hi = hi;
  }
  __syncwarp();
  double lo = s_lo, hi = s_hi, pivmin;
  {
    double a, b;
    gersh(n, d, e, &a, &b, &pivmin);
  }
  for (int round = 0; round < 64; ++round) {
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 2.0 * pivmin) break;
    const double h = (hi - lo) / 33.0;
    const double x = lo + h * (lane + 1);
    cnts[lane] = sturm_count(n, d, e, x, pivmin);
    __syncwarp();
    // first point with at least one eigenvalue below it
    int first = 32;
    for (int l = 0; l < 32; ++l) if (cnts[l] >= 1) { first = l; break; }
    const double nlo = (first == 0) ? lo : lo + h * first;
    const double nhi = (first == 32) ? hi : lo + h * (first + 1);
    __syncwarp();
    if (nlo == lo && nhi == hi) break;
    lo = nlo; hi = nhi;
  }
  if (lane == 0) out[0] = 0.5 * (lo + hi);
}

// ---------------------------------------------------------------------------
// 3. Inverse iteration (tridiagonal LU with partial pivoting)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double hash_unif(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;  // [-1, 1)
}

__global__ void k_stein(int n, const double* __restrict__ d, const double* __restrict__ e,
                        const double* __restrict__ wsel, int cnt, double* __restrict__ ws, int bstride,
                        double* __restrict__ Eout, int ldE, int tbase) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
#define WS(f, i) ws[((size_t)(f) * n + (i)) * bstride + t]
  const double lam = wsel[t];
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    tnorm = fmax(tnorm, r);
  }
  const double tol = fmax(DBL_EPSILON * tnorm, DBL_MIN);
  // fields: 0 a (diag of U), 1 b (super), 2 c (multipliers), 3 d2 (second super), 4 y, 5 pivot flag
  for (int i = 0; i < n; ++i) {
    WS(0, i) = d[i] - lam;
    WS(1, i) = (i + 1 < n) ? e[i] : 0.0;
    WS(2, i) = (i + 1 < n) ? e[i] : 0.0;
    WS(3, i) = 0.0;
    WS(5, i) = 0.0;
  }
  for (int k = 0; k + 1 < n; ++k) {
    const double ak = WS(0, k), bk = WS(1, k), ck = WS(2, k);
    const double ak1 = WS(0, k + 1);
    const double bk1 = (k + 2 < n) ? WS(1, k + 1) : 0.0;
    const double scale1 = fabs(ak) + fabs(bk);
    const double scale2 = fabs(ck) + fabs(ak1) + fabs(bk1);
    const double piv1 = (scale1 == 0.0) ? 0.0 : fabs(ak) / scale1;
    if (ck == 0.0) {
      WS(5, k) = 0.0;
      WS(3, k) = 0.0;
    } else {
      const double piv2 = fabs(ck) / scale2;
      if (piv2 <= piv1) {
        const double mult = ck / ak;
        WS(5, k) = 0.0;
        WS(2, k) = mult;
        WS(0, k + 1) = ak1 - mult * bk;
        WS(3, k) = 0.0;
      } else {
        const double mult = ak / ck;
        WS(5, k) = 1.0;
        WS(0, k) = ck;
        WS(0, k + 1) = bk - mult * ak1;
        if (k + 2 < n) {
          WS(3, k) = bk1;
          WS(1, k + 1) = -mult * bk1;
        } else {
          WS(3, k) = 0.0;
        }
        WS(1, k) = ak1;
        WS(2, k) = mult;
      }
    }
  }
  for (int i = 0; i < n; ++i) WS(4, i) = hash_unif(((unsigned long long)(tbase + t) << 32) ^ (unsigned long long)i);
  for (int iter = 0; iter < 3; ++iter) {
    // forward: P L^{-1}
    for (int k = 1; k < n; ++k) {
      if (WS(5, k - 1) == 0.0) {
        WS(4, k) = WS(4, k) - WS(2, k - 1) * WS(4, k - 1);
      } else {
        const double tmp = WS(4, k - 1);
        const double yk = WS(4, k);
        WS(4, k - 1) = yk;
        WS(4, k) = tmp - WS(2, k - 1) * yk;
      }
    }
    // backward: U^{-1} with tiny pivots replaced by +-tol
    double ymax = 0.0;
    for (int k = n - 1; k >= 0; --k) {
      double tmp = WS(4, k);
      if (k + 1 < n) tmp -= WS(1, k) * WS(4, k + 1);
      if (k + 2 < n) tmp -= WS(3, k) * WS(4, k + 2);
      double ak = WS(0, k);
      if (fabs(ak) < tol) ak = (ak >= 0.0) ? tol : -tol;
      const double yk = tmp / ak;
      WS(4, k) = yk;
      ymax = fmax(ymax, fabs(yk));
    }
    // normalise (scale by the max first to avoid overflow)
    const double inv = (ymax > 0.0) ? 1.0 / ymax : 1.0;
    double nrm = 0.0;
    for (int k = 0; k < n; ++k) {
      const double yk = WS(4, k) * inv;
      WS(4, k) = yk;
      nrm = fma(yk, yk, nrm);
    }
    const double sc = 1.0 / sqrt(nrm);
    for (int k = 0; k < n; ++k) WS(4, k) *= sc;
  }
  double* out = Eout + (size_t)t * ldE;
  for (int k = 0; k < n; ++k) out[k] = WS(4, k);
#undef WS
}

// ---------------------------------------------------------------------------
// 5. Back-transformation: row t of E <- Q row t (Q = H_0 ... H_{n-3})
// ---------------------------------------------------------------------------
__global__ void k_ormtr_rows(int n, const double* __restrict__ A, int lda, const double* __restrict__ tauh,
                             double* __restrict__ E, int ldE, int rows) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (t >= rows) return;
  double* x = E + (size_t)t * ldE;
  for (int j = n - 3; j >= 0; --j) {
    const double tau = tauh[j];
    if (tau == 0.0) continue;
    const double* vj = A + (size_t)j * lda + j + 1;
    const int len = n - j - 1;
    double s = 0.0;
    for (int l = lane; l < len; l += 32) s = fma(vj[l], x[j + 1 + l], s);
    s = wsum(s) * tau;
    for (int l = lane; l < len; l += 32) x[j + 1 + l] -= s * vj[l];
    __syncwarp();
  }
}

// Modified Gram-Schmidt over `rows` (<= 32) vectors of length n, one CTA.
__global__ void k_mgs(int n, double* E, int ldE, int rows) {
  __shared__ double red[32];
  __shared__ double s_val;
  for (int a = 0; a < rows; ++a) {
    double* xa = E + (size_t)a * ldE;
    for (int b = 0; b < a; ++b) {
      const double* xb = E + (size_t)b * ldE;
      double s = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(xa[i], xb[i], s);
      s = bsum(s, red);
      if (threadIdx.x == 0) s_val = s;
      __syncthreads();
      const double c = s_val;
      for (int i = threadIdx.x; i < n; i += blockDim.x) xa[i] -= c * xb[i];
      __syncthreads();
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(xa[i], xa[i], s);
    s = bsum(s, red);
    if (threadIdx.x == 0) s_val = s;
    __syncthreads();
    const double c = 1.0 / sqrt(s_val);
    for (int i = threadIdx.x; i < n; i += blockDim.x) xa[i] *= c;
    __syncthreads();
  }
}

__global__ void k_idx_extremes(int n, int k, int* idx) {
  const int t = threadIdx.x;
  if (t == 0) idx[0] = 0;
  if (t < k) idx[1 + t] = n - k + t;
}

// ---------------------------------------------------------------------------
// Host drivers
// ---------------------------------------------------------------------------
static int stein_batch(int n) {
  // keep the interleaved workspace near 256 MB
  size_t b = (size_t)(256u << 20) / (6 * sizeof(double) * (size_t)std::max(n, 1));
  b = std::max<size_t>(32, std::min<size_t>(b, (size_t)n));
  return (int)b;
}

size_t eig_work_bytes(int n, bool full) {
  size_t dbl = 5 * (size_t)n + 4096 + 64;
  if (full) {
    dbl += (size_t)6 * n * stein_batch(n);
    dbl += (size_t)n * n;  // Gram matrix
    dbl += std::max(potrf_work_doubles(n), trsm_work_doubles(n, n));
  } else {
    dbl += (size_t)6 * n * 64;
  }
  return dbl * sizeof(double) + 64 * sizeof(int) + 256;
}

void eig_work_carve(EigWork* w, void* base, int n, bool full) {
  double* p = (double*)base;
  w->d = p; p += n;
  w->e = p; p += n;
  w->tauh = p; p += n;
  w->p = p; p += n;
  w->wsel = p; p += n;
  w->part = p; p += 4096;
  p += 64;
  w->batch = full ? stein_batch(n) : 64;
  w->ws = p; p += (size_t)6 * n * w->batch;
  if (full) {
    w->G = p; p += (size_t)n * n;
    w->aux = p; p += std::max(potrf_work_doubles(n), trsm_work_doubles(n, n));
  } else {
    w->G = nullptr;
    w->aux = nullptr;
  }
  int* ip = (int*)p;
  w->bar = (unsigned int*)ip; ip += 4;
  w->flag = ip; ip += 4;
  w->info = ip; ip += 4;
}

int eig_flag(cudaStream_t st, EigWork* w) {
  int f = 0;
  cudaMemcpyAsync(&f, w->flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return f;
}

sdp_status eig_full(cudaStream_t st, int n, double* A, double* wout, double* E, EigWork* w) {
  SDP_TRY(sytrd(st, n, A, w));
  count_launch();
  k_stebz<<<cdiv(n, 128), 128, 0, st>>>(n, w->d, w->e, n, nullptr, 0, wout);
  for (int t0 = 0; t0 < n; t0 += w->batch) {
    const int cnt = std::min(w->batch, n - t0);
    count_launch();
    k_stein<<<cdiv(cnt, 64), 64, 0, st>>>(n, w->d, w->e, wout + t0, cnt, w->ws, w->batch,
                                          E + (size_t)t0 * n, n, t0);
  }
  // one Cholesky-QR pass on the rows of E
  gemm(st, false, true, n, n, n, 1.0, E, n, E, n, 0.0, w->G, n, 1);
  potrf(st, n, w->G, n, w->info, w->aux);
  trsm_left_lower(st, false, n, n, w->G, n, E, n, w->aux);
  count_launch();
  k_ormtr_rows<<<cdiv((size_t)n * 32, 256), 256, 0, st>>>(n, A, n, w->tauh, E, n, n);
  return SDP_OK;
}

sdp_status eig_min(cudaStream_t st, int n, double* A, double* lmin_dev, EigWork* w) {
  SDP_TRY(sytrd(st, n, A, w));
  count_launch();
  k_eigmin_warp<<<1, 32, 0, st>>>(n, w->d, w->e, lmin_dev);
  return SDP_OK;
}

sdp_status eig_extremes(cudaStream_t st, int n, double* A, int k, double* lmin_dev, double* wtop,
                        double* Etop, EigWork* w) {
  if (k < 0 || k > 31 || k > n) return SDP_ERR_ARG;
  SDP_TRY(sytrd(st, n, A, w));
  count_launch();
  k_eigmin_warp<<<1, 32, 0, st>>>(n, w->d, w->e, lmin_dev);
  if (k == 0) return SDP_OK;
  int* idx = (int*)w->part;  // small scratch (reinterpreted; part is idle here)
  count_launch(4);
  k_idx_extremes<<<1, 32, 0, st>>>(n, k, idx);
  k_stebz<<<1, 32, 0, st>>>(n, w->d, w->e, k, idx + 1, 0, wtop);
  k_stein<<<1, 32, 0, st>>>(n, w->d, w->e, wtop, k, w->ws, w->batch, Etop, n, n - k);
  k_ormtr_rows<<<cdiv((size_t)k * 32, 128), 128, 0, st>>>(n, A, n, w->tauh, Etop, n, k);
  k_mgs<<<1, 256, 0, st>>>(n, Etop, n, k);
  return SDP_OK;
}

}  // namespace sdpgb
