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
//  4. Re-orthogonalisation of the eigenvector block by up to two Cholesky-QR
//     passes (Gram matrix GEMM, Cholesky, triangular solve), which repair the
//     loss of orthogonality of inverse iteration inside eigenvalue clusters; a
//     pass whose Gram matrix is already the identity to 1e-12 stops there.
//  5. Back-transformation by the stored reflectors (one warp per eigenvector,
//     no inter-CTA communication).
#include <cstring>
#include "internal.cuh"

#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <algorithm>

namespace cg = cooperative_groups;

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
// `spin` cycles of the SM clock (default about two seconds) the waiting CTA sets
// *flag and returns false; all CTAs then leave the kernel at their next barrier.
constexpr long long SPIN_CYCLES = 4000000000LL;

__device__ bool grid_barrier(unsigned int* bar, int* flag, long long spin) {
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
      unsigned int spins = 0;
      while (*vgen == gen) {
        if (*(volatile int*)flag) { s_ok = 0; break; }
        if (clock64() - t0 > spin) { atomicExch(flag, 1); s_ok = 0; break; }
        if (++spins > 4096u) __nanosleep(64);
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
                                               unsigned int* bar, int* flag, long long spin) {
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
    if (!grid_barrier(bar, flag, spin)) return;
    // --- w = p - (tau/2)(p^T v) v ; A22 -= v w^T + w v^T
    if (threadIdx.x < 32) {
      double K = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) K += __ldcg(part + b);
      K = wsum(K);
      if (lane == 0) s_K = 0.5 * tau * K;
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
        ai[l] = fma(-vi, w[l], fma(-wi, v[l], x));
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
    if (!grid_barrier(bar, flag, spin)) return;
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

// Cluster form for small n: one thread-block cluster of SY_CS CTAs, so that
// the two barriers per column are hardware cluster barriers instead of grid
// barriers through global atomics, and the rest of the GPU stays free for
// other problems.  A stays in global memory (L2); warp g of the cluster owns
// rows i = g mod (number of warps) for the whole reduction.  Per column j:
//   every CTA rebuilds the reflector from row j (loaded through L2);
//   p_i = tau A22[i, :] v for the owned rows, each p_i broadcast into every
//   CTA's shared memory, and the CTA's share of p^T v likewise;
//   cluster barrier;  w = p - (tau / 2)(p^T v) v;  owned rows updated;
//   cluster barrier (row j + 1 is complete before anyone reads it).
// The shared arrays written remotely in column j + 1 are only read in steps of
// column j that precede its second barrier, so no buffer is overwritten early.
constexpr int SY_THREADS = 512;
__global__ void __launch_bounds__(SY_THREADS) k_sytrd_cluster(int n, double* A, int lda, double* d, double* e,
                                                               double* tauh) {
  cg::cluster_group cluster = cg::this_cluster();
  const int cs = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  extern __shared__ double sm[];
  double* v = sm;            // n
  double* w = sm + n;        // n
  double* p = sm + 2 * n;    // n   (written by every CTA)
  __shared__ double kpart[32];  // one partial of p^T v per CTA of the cluster
  __shared__ double red[32];
  __shared__ double s_tau, s_beta, s_scale;
  const int wpb = blockDim.x / 32, wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int gwarp = rank * wpb + wid, nwarps = cs * wpb;

  for (int j = 0; j < n - 2; ++j) {
    const int len = n - j - 1;
    const double* row = A + (size_t)j * lda + j + 1;
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
    // owned rows: first owned row index >= j + 1
    double kp = 0.0;
    int i = gwarp + ((j + 1 - gwarp + nwarps - 1) / nwarps) * nwarps;
    if (gwarp >= j + 1) i = gwarp;
    for (; i < n; i += nwarps) {
      const double* ai = A + (size_t)i * lda + j + 1;
      // four independent accumulators keep four L2 loads in flight per lane
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int l = lane;
      for (; l + 96 < len; l += 128) {
        const double x0 = __ldcg(ai + l), x1 = __ldcg(ai + l + 32), x2 = __ldcg(ai + l + 64),
                     x3 = __ldcg(ai + l + 96);
        a0 = fma(x0, v[l], a0);
        a1 = fma(x1, v[l + 32], a1);
        a2 = fma(x2, v[l + 64], a2);
        a3 = fma(x3, v[l + 96], a3);
      }
      for (; l < len; l += 32) a0 = fma(__ldcg(ai + l), v[l], a0);
      double acc = wsum((a0 + a1) + (a2 + a3)) * tau;
      if (lane < cs) {
        double* dst = cluster.map_shared_rank(p, lane);
        dst[i - j - 1] = acc;
      }
      if (lane == 0) kp = fma(acc, v[i - j - 1], kp);
    }
    kp = bsum(kp, red);                                  // valid in thread 0
    const double kp0 = __shfl_sync(0xffffffffu, kp, 0);  // warp 0: every lane gets it
    if (threadIdx.x < cs) {
      double* dst = cluster.map_shared_rank(kpart, (int)threadIdx.x);
      dst[rank] = kp0;
    }
    cluster.sync();
    double K = 0.0;
    for (int c = 0; c < cs; ++c) K += kpart[c];
    K *= 0.5 * tau;
    for (int l = threadIdx.x; l < len; l += blockDim.x) w[l] = p[l] - K * v[l];
    __syncthreads();
    i = gwarp + ((j + 1 - gwarp + nwarps - 1) / nwarps) * nwarps;
    if (gwarp >= j + 1) i = gwarp;
    for (; i < n; i += nwarps) {
      double* ai = A + (size_t)i * lda + j + 1;
      const double vi = v[i - j - 1], wi = w[i - j - 1];
      int l = lane;
      for (; l + 96 < len; l += 128) {
        const double x0 = __ldcg(ai + l), x1 = __ldcg(ai + l + 32), x2 = __ldcg(ai + l + 64),
                     x3 = __ldcg(ai + l + 96);
        ai[l] = fma(-vi, w[l], fma(-wi, v[l], x0));
        ai[l + 32] = fma(-vi, w[l + 32], fma(-wi, v[l + 32], x1));
        ai[l + 64] = fma(-vi, w[l + 64], fma(-wi, v[l + 64], x2));
        ai[l + 96] = fma(-vi, w[l + 96], fma(-wi, v[l + 96], x3));
      }
      for (; l < len; l += 32) {
        const double x = __ldcg(ai + l);
        ai[l] = fma(-vi, w[l], fma(-wi, v[l], x));
      }
    }
    if (rank == 0) {
      double* rj = A + (size_t)j * lda + j + 1;
      for (int l = threadIdx.x; l < len; l += blockDim.x) rj[l] = v[l];
      if (threadIdx.x == 0) {
        d[j] = __ldcg(A + (size_t)j * lda + j);
        e[j] = s_beta;
        tauh[j] = tau;
      }
    }
    cluster.sync();
  }
  if (rank == 0 && threadIdx.x == 0) {
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

// Shared-memory-resident cluster form for orders whose matrix fits in the
// distributed shared memory of one cluster: row i lives in CTA i mod cs (slot
// i / cs) for the whole reduction, so the matrix-vector product and the rank-2
// update of every column read and write shared memory instead of streaming the
// trailing matrix through L2.  Per column j: every CTA copies row j from the CTA
// that owns it (a distributed-shared-memory read) and rebuilds the reflector;
// p_i = tau A22[i, :] v for the owned rows, broadcast into every CTA's p;
// cluster barrier; w = p - (tau / 2)(p^T v) v; owned rows updated; the owner of
// row j stores the reflector in it; cluster barrier.  Row j is read by the other
// CTAs before the first barrier and overwritten by its owner after it, and row
// j + 1 is complete at the second barrier, before anyone reads it.  The rows
// return to global memory at the end (the back-transformation reads them).
__global__ void __launch_bounds__(SY_THREADS) k_sytrd_cluster_smem(int n, double* A, int lda, double* d, double* e,
                                                                    double* tauh) {
  cg::cluster_group cluster = cg::this_cluster();
  const int cs = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  extern __shared__ double sm[];
  const int slots = (n + cs - 1) / cs;
  double* rows = sm;                         // slots x n, row-major
  double* v = rows + (size_t)slots * n;      // n
  double* w = v + n;                         // n
  double* p = w + n;                         // n   (written by every CTA)
  __shared__ double kpart[32];
  __shared__ double red[32];
  __shared__ double s_tau, s_beta, s_scale;
  const int wpb = blockDim.x / 32, wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int sl = 0; sl < slots; ++sl) {
    const int i = sl * cs + rank;
    if (i >= n) break;
    for (int c = threadIdx.x; c < n; c += blockDim.x) rows[(size_t)sl * n + c] = __ldcg(A + (size_t)i * lda + c);
  }
  cluster.sync();
  for (int j = 0; j < n - 2; ++j) {
    const int len = n - j - 1;
    const double* rowj = cluster.map_shared_rank(rows, j % cs) + (size_t)(j / cs) * n + j + 1;
    double s = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const double x = rowj[i];
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
    // owned rows i = sl cs + rank > j
    const int sl0 = (j + 1 > rank) ? (j + 1 - rank + cs - 1) / cs : 0;
    double kp = 0.0;
    for (int sl = sl0 + wid; sl < slots; sl += wpb) {
      const int i = sl * cs + rank;
      if (i >= n) break;
      const double* ai = rows + (size_t)sl * n + j + 1;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int l = lane;
      for (; l + 96 < len; l += 128) {
        a0 = fma(ai[l], v[l], a0);
        a1 = fma(ai[l + 32], v[l + 32], a1);
        a2 = fma(ai[l + 64], v[l + 64], a2);
        a3 = fma(ai[l + 96], v[l + 96], a3);
      }
      for (; l < len; l += 32) a0 = fma(ai[l], v[l], a0);
      const double acc = wsum((a0 + a1) + (a2 + a3)) * tau;
      if (lane < cs) {
        double* dst = cluster.map_shared_rank(p, lane);
        dst[i - j - 1] = acc;
      }
      if (lane == 0) kp = fma(acc, v[i - j - 1], kp);
    }
    kp = bsum(kp, red);
    const double kp0 = __shfl_sync(0xffffffffu, kp, 0);
    if (threadIdx.x < cs) {
      double* dst = cluster.map_shared_rank(kpart, (int)threadIdx.x);
      dst[rank] = kp0;
    }
    cluster.sync();
    double K = 0.0;
    for (int c = 0; c < cs; ++c) K += kpart[c];
    K *= 0.5 * tau;
    for (int l = threadIdx.x; l < len; l += blockDim.x) w[l] = p[l] - K * v[l];
    __syncthreads();
    for (int sl = sl0 + wid; sl < slots; sl += wpb) {
      const int i = sl * cs + rank;
      if (i >= n) break;
      double* ai = rows + (size_t)sl * n + j + 1;
      const double vi = v[i - j - 1], wi = w[i - j - 1];
      for (int l = lane; l < len; l += 32) ai[l] = fma(-vi, w[l], fma(-wi, v[l], ai[l]));
    }
    if (rank == j % cs) {
      double* rj = rows + (size_t)(j / cs) * n;
      for (int l = threadIdx.x; l < len; l += blockDim.x) rj[j + 1 + l] = v[l];
      if (threadIdx.x == 0) {
        d[j] = rj[j];
        e[j] = s_beta;
        tauh[j] = tau;
      }
    }
    cluster.sync();
  }
  if (threadIdx.x == 0) {
    if (n >= 2 && rank == (n - 2) % cs) {
      const double* r2 = rows + (size_t)((n - 2) / cs) * n;
      d[n - 2] = r2[n - 2];
      e[n - 2] = r2[n - 1];
      tauh[n - 2] = 0.0;
    }
    if (rank == (n - 1) % cs) {
      d[n - 1] = rows[(size_t)((n - 1) / cs) * n + n - 1];
      e[n - 1] = 0.0;
      if (n >= 2) tauh[n - 1] = 0.0;
    }
  }
  for (int sl = 0; sl < slots; ++sl) {
    const int i = sl * cs + rank;
    if (i >= n) break;
    for (int c = threadIdx.x; c < n; c += blockDim.x) A[(size_t)i * lda + c] = rows[(size_t)sl * n + c];
  }
}

// One-triangle shared-memory cluster form.  Row i keeps only its lower part
// A[i][0..i] (packed) in CTA i mod cs, so the matrix of order up to ~880 fits
// one 16-CTA cluster, and the symmetric rank-2 update touches one triangle:
// 2 len^2 FMAs per column instead of the 3 len^2 of the full-storage form.
// With lower storage, p = A22 v splits into a row part (the owner's dot of its
// lower row with v) and a column part (for column c, the sum over rows i > c
// of A[i][c] v_i, which every CTA forms over its own rows).  Per column j:
//   0: every CTA builds the reflector from the column j that the owners of
//      rows i > j broadcast into vn at the end of column j - 1;
//   1: row parts (warp per owned row) and the CTA's column parts (thread per
//      column); cluster barrier;
//   2: the owner of row i adds its row part to the 16 CTAs' column parts for i
//      (fixed order), scales by tau and broadcasts p_i and its share of p^T v;
//      cluster barrier;
//   3: w = p - (tau / 2)(p^T v) v; owned rows updated on c in [j + 1, i];
//      the reflector is stored in column j of the owned rows, and column
//      j + 1 is broadcast into vn; cluster barrier.
// Remote buffers and the barriers that order them: vn is written in step 3
// and read in step 0 of the next column (barrier 3 between; the next writes
// come after barriers 1 and 2); part is read remotely between barriers 1 and
// 2 and reused as w after barrier 2; p and kpart are written remotely
// between barriers 1 and 2 and read after barrier 2.  Every sum runs in a
// fixed order, so the result does not depend on timing.  At the end the
// rows are written back with the lower part mirrored into the upper one:
// row j then holds the reflector in A[j][j+1..], as the back-transformation
// expects.
__device__ __forceinline__ size_t sy_off(int sl, int cs, int rank) {
  return (size_t)cs * sl * (sl - 1) / 2 + (size_t)sl * (rank + 1);
}
__global__ void __launch_bounds__(SY_THREADS) k_sytrd_cluster_lower(int n, double* A, int lda, double* d, double* e,
                                                                     double* tauh) {
  cg::cluster_group cluster = cg::this_cluster();
  const int cs = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  extern __shared__ double sm[];
  const int slots = (n - rank + cs - 1) / cs;      // owned rows i = sl cs + rank < n
  // the vectors come first, at the same offset in every CTA (a remote access
  // maps the local offset); the packed rows, whose length depends on the
  // rank, follow them
  double* v = sm;               // n: the reflector of the current column
  double* vn = v + n;           // n: the next column (written remotely)
  double* part = vn + n;        // n: column parts (read remotely), then w
  double* p = part + n;         // n: tau A22 v (written remotely)
  double* rowp = p + n;         // ceil(n / cs): row parts of the owned rows
  double* rows = rowp + (n + cs - 1) / cs;
  __shared__ double kpart[32];
  __shared__ double red[32];
  __shared__ double s_tau, s_beta, s_scale;
  const int wpb = blockDim.x / 32, wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int sl = 0; sl < slots; ++sl) {
    const int i = sl * cs + rank;
    double* ri = rows + sy_off(sl, cs, rank);
    for (int c = threadIdx.x; c <= i; c += blockDim.x) ri[c] = __ldcg(A + (size_t)i * lda + c);
  }
  cluster.sync();
  // column 0 into every CTA's vn
  for (int sl = wid; sl < slots; sl += wpb) {
    const int i = sl * cs + rank;
    if (i >= 1 && lane < cs) cluster.map_shared_rank(vn, lane)[i - 1] = rows[sy_off(sl, cs, rank)];
  }
  cluster.sync();
  for (int j = 0; j < n - 2; ++j) {
    const int len = n - j - 1;
    // ---- 0: reflector from the broadcast column
    double s = 0.0;
    for (int l = threadIdx.x; l < len; l += blockDim.x) {
      const double x = vn[l];
      v[l] = x;
      if (l > 0) s = fma(x, x, s);
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
    for (int l = 1 + threadIdx.x; l < len; l += blockDim.x) v[l] *= scale;
    if (threadIdx.x == 0) v[0] = 1.0;
    __syncthreads();
    // ---- 1: row parts and column parts
    const int sl0 = (j + 1 > rank) ? (j + 1 - rank + cs - 1) / cs : 0;   // first owned row > j
    for (int sl = sl0 + wid; sl < slots; sl += wpb) {
      const int i = sl * cs + rank;
      const double* ri = rows + sy_off(sl, cs, rank) + j + 1;
      const int cnt = i - j;                         // c = j + 1 .. i
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int l = lane;
      for (; l + 96 < cnt; l += 128) {
        a0 = fma(ri[l], v[l], a0);
        a1 = fma(ri[l + 32], v[l + 32], a1);
        a2 = fma(ri[l + 64], v[l + 64], a2);
        a3 = fma(ri[l + 96], v[l + 96], a3);
      }
      for (; l < cnt; l += 32) a0 = fma(ri[l], v[l], a0);
      const double rp = wsum((a0 + a1) + (a2 + a3));
      if (lane == 0) rowp[sl] = rp;
    }
    for (int l = threadIdx.x; l < len; l += blockDim.x) {
      const int c = j + 1 + l;
      int sl = (c >= rank) ? (c - rank) / cs + 1 : 0;   // first owned row > c
      double acc = 0.0;
      size_t o = sy_off(sl, cs, rank);
      for (int i = sl * cs + rank; i < n; i += cs) {
        acc = fma(rows[o + c], v[i - j - 1], acc);
        o += (size_t)i + 1;                          // row i holds i + 1 entries
      }
      part[l] = acc;
    }
    cluster.sync();
    // ---- 2: p_i for the owned rows, broadcast
    double kp = 0.0;
    for (int sl = sl0 + wid; sl < slots; sl += wpb) {
      const int i = sl * cs + rank;
      const int li = i - j - 1;
      double x = (lane < cs) ? cluster.map_shared_rank(part, lane)[li] : 0.0;
      x = wsum(x);
      const double pi = (rowp[sl] + x) * tau;
      if (lane < cs) cluster.map_shared_rank(p, lane)[li] = pi;
      if (lane == 0) kp = fma(pi, v[li], kp);
    }
    kp = bsum(kp, red);
    const double kp0 = __shfl_sync(0xffffffffu, kp, 0);
    if (threadIdx.x < cs) cluster.map_shared_rank(kpart, (int)threadIdx.x)[rank] = kp0;
    cluster.sync();
    // ---- 3: update, reflector, next column
    double K = 0.0;
    for (int c = 0; c < cs; ++c) K += kpart[c];
    K *= 0.5 * tau;
    double* w = part;
    for (int l = threadIdx.x; l < len; l += blockDim.x) w[l] = p[l] - K * v[l];
    __syncthreads();
    for (int sl = sl0 + wid; sl < slots; sl += wpb) {
      const int i = sl * cs + rank;
      const int li = i - j - 1;
      double* ri = rows + sy_off(sl, cs, rank);
      const double vi = v[li], wi = w[li];
      const int cnt = i - j;
      double* rr = ri + j + 1;
      for (int l = lane; l < cnt; l += 32) rr[l] = fma(-vi, w[l], fma(-wi, v[l], rr[l]));
      __syncwarp();
      if (lane == 0) ri[j] = vi;                       // reflector entry (row i, column j)
      if (i > j + 1 && lane < cs) cluster.map_shared_rank(vn, lane)[i - j - 2] = ri[j + 1];
    }
    if (threadIdx.x == 0) {
      if (rank == j % cs) d[j] = rows[sy_off(j / cs, cs, rank) + j];
      if (rank == 0) {
        e[j] = s_beta;
        tauh[j] = tau;
      }
    }
    cluster.sync();
  }
  if (threadIdx.x == 0) {
    if (rank == (n - 2) % cs) {
      d[n - 2] = rows[sy_off((n - 2) / cs, cs, rank) + n - 2];
      tauh[n - 2] = 0.0;
    }
    if (rank == (n - 1) % cs) {
      const double* r1 = rows + sy_off((n - 1) / cs, cs, rank);
      d[n - 1] = r1[n - 1];
      e[n - 2] = r1[n - 2];
      e[n - 1] = 0.0;
      tauh[n - 1] = 0.0;
    }
  }
  for (int sl = 0; sl < slots; ++sl) {
    const int i = sl * cs + rank;
    const double* ri = rows + sy_off(sl, cs, rank);
    for (int c = threadIdx.x; c <= i; c += blockDim.x) {
      const double x = ri[c];
      A[(size_t)i * lda + c] = x;
      A[(size_t)c * lda + i] = x;
    }
  }
}

static size_t sytrd_lower_smem_bytes(int n, int cs) {
  size_t most = 0;   // packed rows of the rank that holds the most
  for (int rank = 0; rank < cs; ++rank) {
    const int slots = (n - rank + cs - 1) / cs;
    most = std::max(most, (size_t)cs * slots * (slots - 1) / 2 + (size_t)slots * (rank + 1));
  }
  return (4 * (size_t)n + (size_t)(n + cs - 1) / cs + most) * sizeof(double);
}

// Cluster size of the shared-memory form for order n: 16 when the matrix and the
// work vectors fit in 16 CTAs' shared memory and the device runs such a
// cluster; 0 otherwise.
static size_t sytrd_smem_bytes(int n, int cs) {
  return ((size_t)((n + cs - 1) / cs) * n + 3 * (size_t)n) * sizeof(double);
}
static int sytrd_smem_cluster(int n) {
  static int max_optin = -1;
  static int ok16 = -1;
  if (max_optin < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  const int cs = 16;
  const size_t need = sytrd_smem_bytes(n, cs);
  if (need + 2048 > (size_t)max_optin) return 0;
  if (ok16 < 0) {
    allow_max_smem((const void*)k_sytrd_cluster_smem);
    cudaFuncSetAttribute((const void*)k_sytrd_cluster_smem, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(SY_THREADS);
    cfg.dynamicSmemBytes = (size_t)max_optin - 2048;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    ok16 = (cudaOccupancyMaxActiveClusters(&ncl, (const void*)k_sytrd_cluster_smem, &cfg) == cudaSuccess && ncl > 0)
               ? 1 : 0;
    cudaGetLastError();
  }
  return ok16 ? cs : 0;
}

// Cluster size of the one-triangle form for order n (16, or 0 when the packed
// rows and work vectors do not fit 16 CTAs' shared memory or the device does
// not run such a cluster).
static int sytrd_lower_cluster(int n) {
  static int max_optin = -1;
  static int ok16 = -1;
  if (max_optin < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  const int cs = 16;
  if (sytrd_lower_smem_bytes(n, cs) + 2048 > (size_t)max_optin) return 0;
  if (ok16 < 0) {
    allow_max_smem((const void*)k_sytrd_cluster_lower);
    cudaFuncSetAttribute((const void*)k_sytrd_cluster_lower, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(SY_THREADS);
    cfg.dynamicSmemBytes = (size_t)max_optin - 2048;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    ok16 = (cudaOccupancyMaxActiveClusters(&ncl, (const void*)k_sytrd_cluster_lower, &cfg) == cudaSuccess &&
            ncl > 0) ? 1 : 0;
    cudaGetLastError();
  }
  return ok16 ? cs : 0;
}

// Cluster size for k_sytrd_cluster: 16 where the device allows it, else 8
// (0 = cluster launch unavailable).
static int sytrd_cluster_size(size_t smem) {
  static int cached = -1;
  if (cached >= 0) return cached;
  allow_max_smem((const void*)k_sytrd_cluster);
  cudaFuncSetAttribute((const void*)k_sytrd_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaGetLastError();
  cached = 0;
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(SY_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, (const void*)k_sytrd_cluster, &cfg) == cudaSuccess && ncl > 0) {
      cached = cs;
      break;
    }
    cudaGetLastError();
  }
  return cached;
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

// Up to this order the cluster form is faster (the cooperative grid form wins
// once the O(n^3) work needs the whole GPU).
constexpr int SY_CLUSTER_MAX_N = 1024;

// Order of preference: the one-triangle form in cluster shared memory
// (n <= 880); the full-row form (n <= 656, where the device cannot run the
// first); the L2-streaming cluster form; the cooperative grid form.  Alone, the
// full-row form is as fast at n ~ 565 and faster for small n (two barriers per
// column instead of three), but in a batch of concurrent problems the
// one-triangle form's half-size shared-memory footprint leaves room on its 16
// SMs for the other problems' kernels, which measured faster end to end.
static sdp_status sytrd(cudaStream_t st, int n, double* A, EigWork* w) {
  if (n >= 3 && n <= SY_CLUSTER_MAX_N) {
    const int cs = sytrd_lower_cluster(n);
    if (cs > 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(SY_THREADS);
      cfg.dynamicSmemBytes = sytrd_lower_smem_bytes(n, cs);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int lda = n;
      count_launch();
      ktimer_begin(st, "sytrd");
      cudaError_t err = cudaLaunchKernelEx(&cfg, k_sytrd_cluster_lower, n, A, lda, w->d, w->e, w->tauh);
      ktimer_end(st, "sytrd", 4.0 / 3.0 * n * (double)n * n, 16.0 * n * (double)n);
      if (err == cudaSuccess) return SDP_OK;
      cudaGetLastError();
    }
  }
  if (n >= 3 && n <= SY_CLUSTER_MAX_N) {
    const int cs = sytrd_smem_cluster(n);
    if (cs > 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(SY_THREADS);
      cfg.dynamicSmemBytes = sytrd_smem_bytes(n, cs);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int lda = n;
      count_launch();
      ktimer_begin(st, "sytrd");
      cudaError_t err = cudaLaunchKernelEx(&cfg, k_sytrd_cluster_smem, n, A, lda, w->d, w->e, w->tauh);
      ktimer_end(st, "sytrd", 4.0 / 3.0 * n * (double)n * n, 16.0 * n * (double)n);
      if (err == cudaSuccess) return SDP_OK;
      cudaGetLastError();
    }
  }
  if (n <= SY_CLUSTER_MAX_N) {
    const size_t csm = 3 * (size_t)n * sizeof(double);
    const int cs = sytrd_cluster_size(200 * 1024);
    if (cs > 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(SY_THREADS);
      cfg.dynamicSmemBytes = csm;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int lda = n;
      count_launch();
      ktimer_begin(st, "sytrd");
      cudaError_t err = cudaLaunchKernelEx(&cfg, k_sytrd_cluster, n, A, lda, w->d, w->e, w->tauh);
      ktimer_end(st, "sytrd", 4.0 / 3.0 * n * (double)n * n, 24.0 * n * (double)n * n / 3.0);
      if (err == cudaSuccess) return SDP_OK;
      cudaGetLastError();
    }
  }
  const size_t smem = 2 * (size_t)n * sizeof(double);
  if (smem > 200 * 1024) return SDP_ERR_UNSUPPORTED;
  allow_max_smem((const void*)k_sytrd);
  cudaMemsetAsync(w->bar, 0, 2 * sizeof(unsigned int), st);
  cudaMemsetAsync(w->flag, 0, sizeof(int), st);
  const int blocks = sytrd_blocks(n, smem);
  int lda = n;
  long long spin = (w->spin_cycles > 0) ? w->spin_cycles : SPIN_CYCLES;
  void* args[] = {&n, &A, &lda, &w->d, &w->e, &w->tauh, &w->p, &w->part, &w->bar, &w->flag, &spin};
  count_launch();
  ktimer_begin(st, "sytrd");
  cudaError_t err = cudaLaunchCooperativeKernel((void*)k_sytrd, dim3(blocks), dim3(256), args, smem, st);
  // algorithmic work of the reduction: (4/3) n^3 flops (symmetric matrix-vector
  // product and rank-2 update per column); the trailing block is read twice and
  // written once per column: 3 * 8 * n^3 / 3 bytes
  ktimer_end(st, "sytrd", 4.0 / 3.0 * n * (double)n * n, 24.0 * n * (double)n * n / 3.0);
  return err == cudaSuccess ? SDP_OK : SDP_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// 2. Bisection
// ---------------------------------------------------------------------------
// Number of eigenvalues of T strictly below x, from the signs of the leading
// principal minors p_i(x) = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (Sturm sequence).
// The three-term form needs two FP64 multiply-adds per step and no division,
// which matters on GB300 where every FP64 op of a warp costs many cycles; the
// sequence is rescaled by a power of two every 16 steps to stay in range.
// A zero minor takes the sign opposite to its predecessor.
__device__ __forceinline__ int sturm_count(int n, const double* d, const double* e2, double x) {
  double pm = 1.0, p = d[0] - x;
  int sp = (p > 0.0) ? 1 : -1;       // sign of p_0 = 1 is +1; zero counts as a change
  int cnt = (sp < 0) ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    const double pn = fma(d[i] - x, p, -e2[i - 1] * pm);
    const int sn = (pn > 0.0) ? 1 : (pn < 0.0 ? -1 : -sp);
    cnt += (sn != sp);
    sp = sn;
    pm = p;
    p = pn;
    if ((i & 15) == 0) {
      const double a = fmax(fabs(p), fabs(pm));
      if (a > 0x1p+400) { p *= 0x1p-400; pm *= 0x1p-400; }
      else if (a < 0x1p-400 && a > 0.0) { p *= 0x1p+400; pm *= 0x1p+400; }
    }
  }
  return cnt;
}

__device__ void gersh(int n, const double* d, const double* e, double* lo, double* hi) {
  double gl = d[0], gu = d[0];
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    gl = fmin(gl, d[i] - r);
    gu = fmax(gu, d[i] + r);
  }
  const double tn = fmax(fabs(gl), fabs(gu));
  const double pad = 2.0 * DBL_EPSILON * tn * n + 4.0 * DBL_MIN;
  *lo = gl - pad;
  *hi = gu + pad;
}

// Stage d and e^2 in shared memory (2n doubles) and compute Gershgorin bounds.
__device__ void stage_tri(int n, const double* d, const double* e, double* sd, double* se2, double* s_lo,
                          double* s_hi) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sd[i] = d[i];
    se2[i] = (i + 1 < n) ? e[i] * e[i] : 0.0;
  }
  if (threadIdx.x == 0) gersh(n, d, e, s_lo, s_hi);
  __syncthreads();
}

__device__ __forceinline__ bool bis_done(double lo, double hi) {
  return hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 4.0 * DBL_MIN;
}

// w[t] = eigenvalue number idx[t] (ascending, 0-based) of T; one warp per
// eigenvalue, 32-point multisection per round (five bits per round).
__global__ void k_stebz(int n, const double* d, const double* e, int cnt, const int* idx, int i0, double* wout) {
  extern __shared__ double tri[];
  __shared__ double s_lo, s_hi;
  stage_tri(n, d, e, tri, tri + n, &s_lo, &s_hi);
  const int lane = threadIdx.x % 32;
  const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (t >= cnt) return;
  const int target = idx ? idx[t] : i0 + t;
  double lo = s_lo, hi = s_hi;
  for (int round = 0; round < 64 && !bis_done(lo, hi); ++round) {
    const double h = (hi - lo) / 33.0;
    const int c = sturm_count(n, tri, tri + n, lo + h * (lane + 1));
    const unsigned above = __ballot_sync(0xffffffffu, c > target);
    const int first = above ? __ffs(above) - 1 : 32;
    const double nlo = (first == 0) ? lo : lo + h * first;
    const double nhi = (first == 32) ? hi : lo + h * (first + 1);
    if (nlo == lo && nhi == hi) break;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) wout[t] = 0.5 * (lo + hi);
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

// One eigenvector per thread.  With blocks == nullptr the whole tridiagonal is
// used; otherwise thread t works on the unreduced diagonal block that owns the
// eigenvalue (src[t] is its row, blocks = {blockid, bstart, bend}) and the
// vector is zero outside that block.
__global__ void k_stein(int nfull, const double* __restrict__ dfull, const double* __restrict__ efull,
                        const double* __restrict__ wsel, int cnt, double* __restrict__ ws, int bstride,
                        double* __restrict__ Eout, int ldE, int tbase, const int* __restrict__ src,
                        const int* __restrict__ blocks) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  int s0 = 0, s1 = nfull;
  if (blocks) {
    const int b = blocks[src[t]];
    s0 = blocks[nfull + b];
    s1 = blocks[2 * nfull + b];
  }
  const int n = s1 - s0;
  const double* d = dfull + s0;
  const double* e = efull + s0;
#define WS(f, i) ws[((size_t)(f) * nfull + (i)) * bstride + t]
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
  // reciprocal pivots (tiny pivots replaced by +-tol) so the solves only multiply
  for (int k = 0; k < n; ++k) {
    double ak = WS(0, k);
    if (fabs(ak) < tol) ak = (ak >= 0.0) ? tol : -tol;
    WS(0, k) = 1.0 / ak;
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
    // backward: U^{-1} with tiny pivots replaced by +-tol.  Each tiny pivot
    // multiplies by up to 1/tol, so a cluster of them can overflow: whenever an
    // entry passes 2^400 the whole vector (solved part and remaining
    // right-hand side alike) is scaled by 2^-400, which keeps the system
    // consistent; the vector is normalised afterwards anyway.
    double ymax = 0.0;
    for (int k = n - 1; k >= 0; --k) {
      double tmp = WS(4, k);
      if (k + 1 < n) tmp -= WS(1, k) * WS(4, k + 1);
      if (k + 2 < n) tmp -= WS(3, k) * WS(4, k + 2);
      double yk = tmp * WS(0, k);
      if (!(fabs(yk) < 0x1p+400)) {
        for (int j = 0; j < n; ++j) WS(4, j) *= 0x1p-400;
        ymax *= 0x1p-400;
        yk = (tmp * 0x1p-400) * WS(0, k);
      }
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
  for (int k = 0; k < s0; ++k) out[k] = 0.0;
  for (int k = 0; k < n; ++k) out[s0 + k] = WS(4, k);
  for (int k = s1; k < nfull; ++k) out[k] = 0.0;
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
// Splitting into unreduced blocks.  Where e_i^2 <= eps^2 |d_i d_{i+1}| (+ tiny)
// the off-diagonal is set to zero and T falls apart into independent blocks.
// Equal eigenvalues of different blocks would otherwise share one shift, and
// inverse iteration would return the same null direction for all of them;
// per block, eigenvalues of an unreduced tridiagonal are distinct, the vectors
// of different blocks have disjoint supports and are exactly orthogonal.
// blocks[0..n) = block of each row, blocks[n + b] = first row, blocks[2n + b] =
// one past the last row, blocks[3n] = number of blocks.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_tri_split(int n, const double* __restrict__ d, const double* __restrict__ e,
                                                    double* __restrict__ es, int* __restrict__ blocks) {
  __shared__ int csum[1024];
  const int T = blockDim.x, tid = threadIdx.x;
  const int chunk = (n + T - 1) / T, i0 = tid * chunk, i1 = min(n, i0 + chunk);
  int cnt = 0;
  for (int i = i0; i < i1; ++i) {
    bool split = false;
    if (i + 1 < n) {
      const double e2 = e[i] * e[i];
      split = !(e2 > DBL_EPSILON * DBL_EPSILON * fabs(d[i] * d[i + 1]) + 4.0 * DBL_MIN);
      es[i] = split ? 0.0 : e[i];
    } else {
      es[i] = 0.0;
    }
    const int starts = (i == 0) ? 1 : 0;   // row i starts a block if i == 0 or e_{i-1} split
    cnt += starts;
    (void)split;
  }
  // rows that start a block because the previous off-diagonal split
  for (int i = i0; i < i1; ++i) {
    if (i > 0) {
      const double e2 = e[i - 1] * e[i - 1];
      if (!(e2 > DBL_EPSILON * DBL_EPSILON * fabs(d[i - 1] * d[i]) + 4.0 * DBL_MIN)) ++cnt;
    }
  }
  csum[tid] = cnt;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int q = 0; q < T; ++q) { const int c = csum[q]; csum[q] = run; run += c; }
    blocks[3 * n] = run;
  }
  __syncthreads();
  int b = csum[tid] - 1;
  for (int i = i0; i < i1; ++i) {
    bool start = (i == 0);
    if (i > 0) {
      const double e2 = e[i - 1] * e[i - 1];
      start = !(e2 > DBL_EPSILON * DBL_EPSILON * fabs(d[i - 1] * d[i]) + 4.0 * DBL_MIN);
    }
    if (start) {
      ++b;
      blocks[n + b] = i;
      if (b > 0) blocks[2 * n + b - 1] = i;
    }
    blocks[i] = b;
  }
  __syncthreads();
  if (tid == 0) blocks[2 * n + blocks[3 * n] - 1] = n;
}

// val[t] = eigenvalue number (t - first row) of the block that owns row t.
__global__ void k_stebz_blk(int n, const double* d, const double* es, const int* __restrict__ blocks, double* val) {
  extern __shared__ double tri[];
  double* sd = tri;
  double* se2 = tri + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sd[i] = d[i];
    se2[i] = es[i] * es[i];
  }
  __syncthreads();
  const int lane = threadIdx.x % 32;
  const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (t >= n) return;
  const int b = blocks[t], s0 = blocks[n + b], s1 = blocks[2 * n + b], ns = s1 - s0;
  const int target = t - s0;
  if (ns == 1) {
    if (lane == 0) val[t] = sd[s0];
    return;
  }
  double lo, hi;
  gersh(ns, d + s0, es + s0, &lo, &hi);
  for (int round = 0; round < 64 && !bis_done(lo, hi); ++round) {
    const double h = (hi - lo) / 33.0;
    const int c = sturm_count(ns, sd + s0, se2 + s0, lo + h * (lane + 1));
    const unsigned above = __ballot_sync(0xffffffffu, c > target);
    const int first = above ? __ffs(above) - 1 : 32;
    const double nlo = (first == 0) ? lo : lo + h * first;
    const double nhi = (first == 32) ? hi : lo + h * (first + 1);
    if (nlo == lo && nhi == hi) break;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) val[t] = 0.5 * (lo + hi);
}

// Global ascending order of the per-block eigenvalues (ties by row).
__global__ void k_rank(int n, const double* __restrict__ val, double* __restrict__ w, int* __restrict__ src) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double v = val[t];
  int r = 0;
  for (int u = 0; u < n; ++u) {
    const double x = val[u];
    r += (x < v) || (x == v && u < t);
  }
  w[r] = v;
  src[r] = t;
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
  size_t dbl = 7 * (size_t)n + 4096 + 64 + (4 * (size_t)n + 16) / 2 + 8;
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
  w->es = p; p += n;
  w->val = p; p += n;
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
  w->blocks = ip; ip += 3 * n + 4;
  w->src = ip; ip += n;
}

// The barrier counters, the timeout flag and the info word start at zero: the
// flag is read after every eigensolver call, also when no grid-barrier kernel
// ran (freshly allocated device memory holds whatever was there before).
void eig_work_clear(cudaStream_t st, EigWork* w) {
  cudaMemsetAsync(w->bar, 0, 12 * sizeof(int), st);   // bar[4], flag[4], info[4]
}

int eig_flag(cudaStream_t st, EigWork* w) {
  int f = 0;
  cudaMemcpyAsync(&f, w->flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return f;
}

static void launch_stebz(cudaStream_t st, int n, const double* d, const double* e, int cnt, const int* idx,
                         int i0, double* out) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  allow_max_smem((const void*)k_stebz);
  const int warps = 4;
  count_launch();
  k_stebz<<<cdiv(cnt, warps), 32 * warps, smem, st>>>(n, d, e, cnt, idx, i0, out);
}

// Splits T into unreduced blocks; returns the number of blocks (host sync).
static int split_blocks(cudaStream_t st, int n, EigWork* w) {
  count_launch();
  k_tri_split<<<1, 1024, 0, st>>>(n, w->d, w->e, w->es, w->blocks);
  int nb = 1;
  cudaMemcpyAsync(&nb, w->blocks + 3 * n, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return nb;
}

// All eigenvalues ascending (w) and, when blocked, the row of the block that owns each.
static void eigenvalues_all(cudaStream_t st, int n, EigWork* w, int nblocks, double* wout) {
  if (nblocks <= 1) {
    launch_stebz(st, n, w->d, w->e, n, nullptr, 0, wout);
    return;
  }
  allow_max_smem((const void*)k_stebz_blk);
  count_launch(2);
  k_stebz_blk<<<cdiv(n, 4), 128, 2 * (size_t)n * sizeof(double), st>>>(n, w->d, w->es, w->blocks, w->val);
  k_rank<<<cdiv(n, 128), 128, 0, st>>>(n, w->val, wout, w->src);
}

static void eigenvectors(cudaStream_t st, int n, EigWork* w, int nblocks, const double* wv, int first, int cnt,
                         double* E) {
  const double* e = (nblocks <= 1) ? w->e : w->es;
  for (int t0 = 0; t0 < cnt; t0 += w->batch) {
    const int c = std::min(w->batch, cnt - t0);
    count_launch();
    k_stein<<<cdiv(c, 64), 64, 0, st>>>(n, w->d, e, wv + first + t0, c, w->ws, w->batch, E + (size_t)t0 * n, n,
                                        first + t0, nblocks <= 1 ? nullptr : w->src + first + t0,
                                        nblocks <= 1 ? nullptr : w->blocks);
  }
}

// max over the lower triangle of |G_ij - delta_ij| (non-negative doubles order
// like their bit patterns, so an integer atomicMax takes the maximum)
constexpr double ORTH_TOL = 1e-12;
__global__ void k_gram_err(int n, const double* __restrict__ G, int ldg, unsigned long long* err) {
  double m = 0.0;
  const size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (j > i) continue;
    double v = fabs(G[(size_t)i * ldg + j] - (i == j ? 1.0 : 0.0));
    if (!(v == v)) v = INFINITY;   // NaN counts as not orthogonal
    m = fmax(m, v);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(err, (unsigned long long)__double_as_longlong(m));
}

sdp_status eig_full(cudaStream_t st, int n, double* A, double* wout, double* E, EigWork* w) {
  SDP_TRY(sytrd(st, n, A, w));
  const int nb = split_blocks(st, n, w);
  eigenvalues_all(st, n, w, nb, wout);
  eigenvectors(st, n, w, nb, wout, 0, n, E);
  // Up to two Cholesky-QR passes on the rows of E.  Inverse iteration leaves
  // vectors of well separated eigenvalues orthogonal to working accuracy; only
  // tight clusters inside one block lose orthogonality.  Each pass first forms
  // the Gram matrix and stops when max |E E^T - I| is already at rounding level,
  // so the factorisation and the triangular solve run only when needed.
  for (int pass = 0; pass < 2; ++pass) {
    gemm(st, false, true, n, n, n, 1.0, E, n, E, n, 0.0, w->G, n, GEMM_LOWER_C);
    unsigned long long* err = reinterpret_cast<unsigned long long*>(w->part);
    SDP_CK_ST(cudaMemsetAsync(err, 0, sizeof(unsigned long long), st));
    count_launch();
    k_gram_err<<<std::min<unsigned>(cdiv((size_t)n * n, 256), 1024), 256, 0, st>>>(n, w->G, n, err);
    unsigned long long bits = 0;
    SDP_CK_ST(cudaMemcpyAsync(&bits, err, sizeof(bits), cudaMemcpyDeviceToHost, st));
    SDP_CK_ST(cudaStreamSynchronize(st));
    double e;
    std::memcpy(&e, &bits, sizeof(e));
    if (e <= ORTH_TOL) break;
    potrf(st, n, w->G, n, w->info, w->aux);
    trsm_left_lower(st, false, n, n, w->G, n, E, n, w->aux);
  }
  count_launch();
  k_ormtr_rows<<<cdiv((size_t)n * 32, 256), 256, 0, st>>>(n, A, n, w->tauh, E, n, n);
  return SDP_OK;
}

sdp_status eig_min(cudaStream_t st, int n, double* A, double* lmin_dev, EigWork* w) {
  SDP_TRY(sytrd(st, n, A, w));
  launch_stebz(st, n, w->d, w->e, 1, nullptr, 0, lmin_dev);
  return SDP_OK;
}

sdp_status eig_extremes(cudaStream_t st, int n, double* A, int k, double* lmin_dev, double* wtop,
                        double* Etop, EigWork* w) {
  if (k < 0 || k > SDP_K_MAX + 1 || k > n) return SDP_ERR_ARG;
  SDP_TRY(sytrd(st, n, A, w));
  const int nb = (k > 0) ? split_blocks(st, n, w) : 1;
  if (nb <= 1) {
    launch_stebz(st, n, w->d, w->e, 1, nullptr, 0, lmin_dev);
    if (k == 0) return SDP_OK;
    int* idx = (int*)w->part;  // small scratch (part is idle here)
    count_launch(1);
    k_idx_extremes<<<1, 128, 0, st>>>(n, k, idx);
    launch_stebz(st, n, w->d, w->e, k, idx + 1, 0, wtop);
    eigenvectors(st, n, w, 1, wtop, 0, k, Etop);
  } else {
    eigenvalues_all(st, n, w, nb, w->wsel);
    SDP_CK_ST(cudaMemcpyAsync(lmin_dev, w->wsel, sizeof(double), cudaMemcpyDeviceToDevice, st));
    SDP_CK_ST(cudaMemcpyAsync(wtop, w->wsel + n - k, k * sizeof(double), cudaMemcpyDeviceToDevice, st));
    eigenvectors(st, n, w, nb, w->wsel, n - k, k, Etop);
  }
  count_launch(2);
  k_ormtr_rows<<<cdiv((size_t)k * 32, 128), 128, 0, st>>>(n, A, n, w->tauh, Etop, n, k);
  k_mgs<<<1, 256, 0, st>>>(n, Etop, n, k);
  return SDP_OK;
}

}  // namespace sdpgb
