// Dense FP64 building blocks: tiled GEMM, blocked Cholesky, blocked triangular
// solves, reductions and elementwise kernels.  All matrices are row-major.
//
// On GB300 the FP64 pipe runs at about 1/60 of the FP32 rate, so every FP64
// kernel here is arithmetic-bound long before it is memory-bound: the GEMM keeps
// a 64 x 64 tile per CTA (4 x 4 per thread) and does 16 FMAs per shared-memory
// operand pair, far above the ratio the FP64 pipe needs.
#include "internal.cuh"

#include <algorithm>

namespace sdpgb {

std::atomic<int64_t> g_launches{0};
thread_local int64_t t_launches = 0;

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// GEMM:  C = alpha op(A) op(B) + beta C
// ---------------------------------------------------------------------------
template <typename T, int BM, int BN, bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, T alpha, const T* __restrict__ A,
                                              int lda, const T* __restrict__ B, int ldb, T beta,
                                              T* __restrict__ C, int ldc, int flags,
                                              long long sA, long long sB, long long sC) {
  constexpr int BK = 16;
  constexpr int TM = BM / 16, TN = BN / 16;
  const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
  if ((flags & GEMM_LOWER_C) && bn > bm + BM - 1) return;
  // k range that can hold nonzero products when op(A) or op(B) is triangular
  // (the skipped entries are stored zeros, so the boundary chunk needs no mask)
  int kbeg = 0, kend = K;
  if (flags & GEMM_A_UPPER) kbeg = max(kbeg, bm);
  if (flags & GEMM_B_LOWER) kbeg = max(kbeg, bn);
  if (flags & GEMM_A_LOWER) kend = min(kend, bm + BM);
  if (flags & GEMM_B_UPPER) kend = min(kend, bn + BN);
  A += (long long)blockIdx.z * sA;
  B += (long long)blockIdx.z * sB;
  C += (long long)blockIdx.z * sC;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += 256) {
      int r, c;
      if (!TA) { r = t / BK; c = t % BK; } else { c = t / BM; r = t % BM; }
      const int gr = bm + r, gc = k0 + c;
      T v = T(0);
      if (gr < M && gc < K) v = TA ? A[(size_t)gc * lda + gr] : A[(size_t)gr * lda + gc];
      As[c][r] = v;
    }
    for (int t = threadIdx.x; t < BK * BN; t += 256) {
      int r, c;
      if (!TB) { r = t / BN; c = t % BN; } else { c = t / BK; r = t % BK; }
      const int gr = k0 + r, gc = bn + c;
      T v = T(0);
      if (gr < K && gc < N) v = TB ? B[(size_t)gc * ldb + gr] : B[(size_t)gr * ldb + gc];
      Bs[r][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = bm + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = bn + tx + 16 * j;
      if (c >= N) continue;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v = fma(beta, C[(size_t)r * ldc + c], v);
      C[(size_t)r * ldc + c] = v;
    }
  }
}

template <typename T, int BM, int BN>
static void gemm_launch(cudaStream_t st, bool tA, bool tB, int M, int N, int K, T alpha, const T* A,
                        int lda, const T* B, int ldb, T beta, T* C, int ldc, int flags,
                        int batch, long long sA, long long sB, long long sC) {
  dim3 grid(cdiv(N, BN), cdiv(M, BM), batch);
  count_launch();
  if (!tA && !tB)
    k_gemm<T, BM, BN, false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, sA, sB, sC);
  else if (!tA && tB)
    k_gemm<T, BM, BN, false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, sA, sB, sC);
  else if (tA && !tB)
    k_gemm<T, BM, BN, true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, sA, sB, sC);
  else
    k_gemm<T, BM, BN, true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, sA, sB, sC);
}

// Multiply-adds a gemm call performs on entries that are not structural zeros:
// the k range of every tile it runs, times the tile's rows and columns inside C.
double gemm_useful_fma(int M, int N, int K, int flags, int tile) {
  double f = 0.0;
  for (int bm = 0; bm < M; bm += tile)
    for (int bn = 0; bn < N; bn += tile) {
      if ((flags & GEMM_LOWER_C) && bn > bm + tile - 1) continue;
      int kbeg = 0, kend = K;
      if (flags & GEMM_A_UPPER) kbeg = std::max(kbeg, bm);
      if (flags & GEMM_B_LOWER) kbeg = std::max(kbeg, bn);
      if (flags & GEMM_A_LOWER) kend = std::min(kend, bm + tile);
      if (flags & GEMM_B_UPPER) kend = std::min(kend, bn + tile);
      if (kend > kbeg)
        f += (double)std::min(tile, M - bm) * std::min(tile, N - bn) * (kend - kbeg);
    }
  return f;
}

// Thin products C = alpha A op(B) + beta C with at most THIN_N columns (A not
// transposed): one warp per row of C, lanes over K, one accumulator per column,
// so a probe-vector check or a product with k eigenvectors costs about M K N
// FMAs instead of a 32 x 32 tile per 32 rows whose columns are mostly padding.
constexpr int THIN_N = 8;
template <bool TB>
__global__ void __launch_bounds__(256) k_gemm_thin(int M, int N, int K, double alpha, const double* __restrict__ A,
                                                   int lda, const double* __restrict__ B, int ldb, double beta,
                                                   double* __restrict__ C, int ldc) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (r >= M) return;
  const double* a = A + (size_t)r * lda;
  double acc[THIN_N];
#pragma unroll
  for (int j = 0; j < THIN_N; ++j) acc[j] = 0.0;
  for (int k = lane; k < K; k += 32) {
    const double x = a[k];
#pragma unroll
    for (int j = 0; j < THIN_N; ++j)
      if (j < N) acc[j] = fma(x, TB ? B[(size_t)j * ldb + k] : B[(size_t)k * ldb + j], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < THIN_N; ++j) {
    double v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == j && j < N) {
      double c = alpha * v;
      if (beta != 0.0) c = fma(beta, C[(size_t)r * ldc + j], c);
      C[(size_t)r * ldc + j] = c;
    }
  }
}

void gemm(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
          int lda, const double* B, int ldb, double beta, double* C, int ldc, int flags,
          int batch, long long sA, long long sB, long long sC) {
  if (M <= 0 || N <= 0) return;
  if (!tA && N <= THIN_N && K > 0 && flags == 0 && batch == 1) {
    const bool timed = ktimer_on("gemm_f64");
    if (timed) ktimer_begin(st, "gemm_f64");
    count_launch();
    const unsigned grid = cdiv((size_t)M * 32, 256);
    if (tB) k_gemm_thin<true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else k_gemm_thin<false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    if (timed) ktimer_end(st, "gemm_f64", 2.0 * M * N * (double)K, 8.0 * ((double)M * K + (double)K * N + 2.0 * M * N));
    return;
  }
  if (K <= 0) {  // C = beta C
    if (beta == 0.0) {
      for (int b = 0; b < batch; ++b) copy2d(st, M, N, nullptr, 0, C + b * sC, ldc);
    } else {
      gemm_launch<double, 32, 32>(st, false, false, M, N, 1, 0.0, C, ldc, C, ldc, beta, C, ldc,
                                  flags & GEMM_LOWER_C, batch, sC, sC, sC);
    }
    return;
  }
  const long long tiles64 = (long long)cdiv(M, 64) * cdiv(N, 64) * batch;
  const bool timed = ktimer_on("gemm_f64");
  if (timed) ktimer_begin(st, "gemm_f64");
  const int tile = (tiles64 >= 2 * 152) ? 64 : 32;
  if (tile == 64)
    gemm_launch<double, 64, 64>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, batch, sA, sB, sC);
  else
    gemm_launch<double, 32, 32>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, batch, sA, sB, sC);
  if (timed) {
    const double f = 2.0 * gemm_useful_fma(M, N, K, flags, tile) * batch;
    const double by = 8.0 * ((double)M * K + (double)K * N + 2.0 * M * N) * batch;
    ktimer_end(st, "gemm_f64", f, by);
  }
}

void gemm_f32(cudaStream_t st, bool tA, bool tB, int M, int N, int K, float alpha, const float* A,
              int lda, const float* B, int ldb, float beta, float* C, int ldc) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  gemm_launch<float, 64, 64>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0, 1, 0, 0, 0);
}

// ---------------------------------------------------------------------------
// Elementwise helpers
// ---------------------------------------------------------------------------
__global__ void k_fill(double* x, size_t count, double v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) x[i] = v;
}
void fill(cudaStream_t st, double* x, size_t count, double v) {
  if (!count) return;
  count_launch();
  k_fill<<<std::min<unsigned>(cdiv(count, 256), 4096), 256, 0, st>>>(x, count, v);
}

__global__ void k_copy2d(int rows, int cols, const double* __restrict__ s, int lds, double* __restrict__ d, int ldd) {
  const size_t total = (size_t)rows * cols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / cols), c = (int)(t % cols);
    d[(size_t)r * ldd + c] = s ? s[(size_t)r * lds + c] : 0.0;
  }
}
void copy2d(cudaStream_t st, int rows, int cols, const double* src, int lds, double* dst, int ldd) {
  if (rows <= 0 || cols <= 0) return;
  count_launch();
  k_copy2d<<<std::min<unsigned>(cdiv((size_t)rows * cols, 256), 8192), 256, 0, st>>>(rows, cols, src, lds, dst, ldd);
}

__global__ void k_transpose(int rows, int cols, const double* __restrict__ s, int lds, double* __restrict__ d, int ldd) {
  __shared__ double tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = s[(size_t)r * lds + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) d[(size_t)c * ldd + r] = tile[threadIdx.x][i];
  }
}
void transpose(cudaStream_t st, int rows, int cols, const double* src, int lds, double* dst, int ldd) {
  if (rows <= 0 || cols <= 0) return;
  count_launch();
  k_transpose<<<dim3(cdiv(cols, 32), cdiv(rows, 32)), dim3(32, 8), 0, st>>>(rows, cols, src, lds, dst, ldd);
}

// A_ij = A_ji for i < j (copy the lower triangle into the upper one) or average.
template <int MODE>
__global__ void k_sym(int n, double* A, int lda) {
  __shared__ double tl[32][33], tu[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  const int r0 = bi * 32, c0 = bj * 32;  // lower tile (r0, c0), mirror tile (c0, r0)
  for (int i = threadIdx.y; i < 32; i += 8) {
    int r = r0 + i, c = c0 + threadIdx.x;
    tl[i][threadIdx.x] = (r < n && c < n) ? A[(size_t)r * lda + c] : 0.0;
    r = c0 + i; c = r0 + threadIdx.x;
    tu[i][threadIdx.x] = (r < n && c < n) ? A[(size_t)r * lda + c] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    // element (c0+i, r0+tx) of the upper tile mirrors (r0+tx, c0+i) of the lower tile
    const int ru = c0 + i, cu = r0 + threadIdx.x;
    const int rl = r0 + i, cl = c0 + threadIdx.x;
    const double lo_m = tl[threadIdx.x][i];  // A[r0+tx][c0+i]
    const double up_m = tu[threadIdx.x][i];  // A[c0+tx][r0+i]
    if (MODE == 0) {
      if (ru < n && cu < n && cu > ru) A[(size_t)ru * lda + cu] = lo_m;
    } else {
      const double lo = tl[i][threadIdx.x];  // A[rl][cl]
      const double avg = 0.5 * (lo + up_m);
      if (rl < n && cl < n) A[(size_t)rl * lda + cl] = avg;
      if (ru < n && cu < n && ru != cu) A[(size_t)ru * lda + cu] = 0.5 * (tu[i][threadIdx.x] + lo_m);
    }
  }
}
void symmetrize_lower(cudaStream_t st, int n, double* A, int lda) {
  count_launch();
  k_sym<0><<<dim3(cdiv(n, 32), cdiv(n, 32)), dim3(32, 8), 0, st>>>(n, A, lda);
}
void symmetrize_avg(cudaStream_t st, int n, double* A, int lda) {
  count_launch();
  k_sym<1><<<dim3(cdiv(n, 32), cdiv(n, 32)), dim3(32, 8), 0, st>>>(n, A, lda);
}

__global__ void k_add_diag(int n, double* A, int lda, double v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) A[(size_t)i * lda + i] += v;
}
void add_diag(cudaStream_t st, int n, double* A, int lda, double v) {
  count_launch();
  k_add_diag<<<cdiv(n, 256), 256, 0, st>>>(n, A, lda, v);
}

__global__ void k_scale_cols(int rows, int cols, const double* __restrict__ A, int lda,
                             const double* __restrict__ s, double pw, double* __restrict__ B, int ldb) {
  const size_t total = (size_t)rows * cols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / cols), c = (int)(t % cols);
    const double f = (pw == 1.0) ? s[c] : (pw == -1.0) ? 1.0 / s[c] : pow(s[c], pw);
    B[(size_t)r * ldb + c] = A[(size_t)r * lda + c] * f;
  }
}
void scale_cols(cudaStream_t st, int rows, int cols, const double* A, int lda, const double* s,
                double pw, double* B, int ldb) {
  count_launch();
  k_scale_cols<<<std::min<unsigned>(cdiv((size_t)rows * cols, 256), 8192), 256, 0, st>>>(rows, cols, A, lda, s, pw, B, ldb);
}

__global__ void k_zero_upper(int n, double* A, int lda) {
  const size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / n), c = (int)(t % n);
    if (c > r) A[(size_t)r * lda + c] = 0.0;
  }
}
void zero_upper(cudaStream_t st, int n, double* A, int lda) {
  count_launch();
  k_zero_upper<<<std::min<unsigned>(cdiv((size_t)n * n, 256), 8192), 256, 0, st>>>(n, A, lda);
}

__global__ void k_axpby(size_t count, double a, const double* x, double b, const double* y, double* z) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    z[i] = a * x[i] + (y ? b * y[i] : 0.0);
}
void axpby(cudaStream_t st, size_t count, double a, const double* x, double b, const double* y, double* z) {
  if (!count) return;
  count_launch();
  k_axpby<<<std::min<unsigned>(cdiv(count, 256), 8192), 256, 0, st>>>(count, a, x, b, y, z);
}

__global__ void k_to_f32(size_t count, const double* x, float* y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) y[i] = (float)x[i];
}
void to_f32(cudaStream_t st, size_t count, const double* x, float* y) {
  count_launch();
  k_to_f32<<<std::min<unsigned>(cdiv(count, 256), 8192), 256, 0, st>>>(count, x, y);
}
__global__ void k_to_bf16(size_t count, const double* x, __nv_bfloat16* y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn((float)x[i]);
}
void to_bf16(cudaStream_t st, size_t count, const double* x, __nv_bfloat16* y) {
  count_launch();
  k_to_bf16<<<std::min<unsigned>(cdiv(count, 256), 8192), 256, 0, st>>>(count, x, y);
}

// ---------------------------------------------------------------------------
// Reductions (deterministic: fixed partition, fixed summation order)
// ---------------------------------------------------------------------------
constexpr int DOT_BLOCKS = 512;
size_t dot_part_doubles() { return DOT_BLOCKS; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < (int)(blockDim.x / 32)) ? sh[l] : 0.0;
    s = warp_sum(s);
  }
  return s;  // valid in thread 0
}

__global__ void k_dot_part(size_t count, const double* __restrict__ x, const double* __restrict__ y, double* part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void k_sum_part(int np, const double* part, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}
void dot_partials(cudaStream_t st, size_t count, const double* x, const double* y, double* part) {
  count_launch();
  k_dot_part<<<DOT_BLOCKS, 256, 0, st>>>(count, x, y, part);
}
void dot(cudaStream_t st, size_t count, const double* x, const double* y, double* out, double* part) {
  count_launch(2);
  k_dot_part<<<DOT_BLOCKS, 256, 0, st>>>(count, x, y, part);
  k_sum_part<<<1, 512, 0, st>>>(DOT_BLOCKS, part, out);
}

// ---------------------------------------------------------------------------
// Triangular matrix-vector products with a lower-triangular L
// ---------------------------------------------------------------------------
constexpr int TRMV_CHUNKS = 64;
size_t trmv_part_doubles(int n) { return (size_t)n * TRMV_CHUNKS; }

__global__ void k_trmv_n(int n, const double* __restrict__ L, int ldl, const double* __restrict__ x,
                         double* __restrict__ y, double alpha, const double* __restrict__ z, double beta) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (warp >= n) return;
  const double* row = L + (size_t)warp * ldl;
  double s = 0.0;
  for (int j = lane; j <= warp; j += 32) s = fma(row[j], x[j], s);
  s = warp_sum(s);
  if (lane == 0) y[warp] = alpha * s + (z ? beta * z[warp] : 0.0);
}
// part[c][j] = sum_{i in chunk c, i >= j} L[i][j] x[i]
__global__ void k_trmv_t_part(int n, const double* __restrict__ L, int ldl, const double* __restrict__ x, double* __restrict__ part) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  const int rows = (n + TRMV_CHUNKS - 1) / TRMV_CHUNKS;
  const int i0 = c * rows, i1 = min(n, i0 + rows);
  if (j >= n) return;
  double s = 0.0;
  for (int i = max(i0, j); i < i1; ++i) s = fma(L[(size_t)i * ldl + j], x[i], s);
  part[(size_t)c * n + j] = s;
}
__global__ void k_trmv_t_sum(int n, const double* __restrict__ part, double* __restrict__ y, double alpha,
                             const double* __restrict__ z, double beta) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int c = 0; c < TRMV_CHUNKS; ++c) s += part[(size_t)c * n + j];
  y[j] = alpha * s + (z ? beta * z[j] : 0.0);
}
void trmv_lower_ex(cudaStream_t st, bool trans, int n, const double* L, int ldl, const double* x, double* y,
                   double* part, double alpha, const double* z, double beta) {
  if (!trans) {
    count_launch();
    k_trmv_n<<<cdiv((size_t)n * 32, 256), 256, 0, st>>>(n, L, ldl, x, y, alpha, z, beta);
  } else {
    count_launch(2);
    k_trmv_t_part<<<dim3(cdiv(n, 128), TRMV_CHUNKS), 128, 0, st>>>(n, L, ldl, x, part);
    k_trmv_t_sum<<<cdiv(n, 256), 256, 0, st>>>(n, part, y, alpha, z, beta);
  }
}
void trmv_lower(cudaStream_t st, bool trans, int n, const double* L, int ldl, const double* x, double* y, double* part) {
  trmv_lower_ex(st, trans, n, L, ldl, x, y, part, 1.0, nullptr, 0.0);
}

// ---------------------------------------------------------------------------
// Blocked Cholesky and triangular solves
// ---------------------------------------------------------------------------
constexpr int NB = 64;

// Factor the nbs x nbs (nbs <= BS) diagonal block in place (lower).  256
// threads; thread t keeps the BS^2 / 256 entries (i, l) with l = t % BS and
// i = t / BS + (256 / BS) s in registers.  Per column j: the owner of (j, j)
// forms the pivot, the owners of column j scale it and publish it to shared
// memory, and every thread applies the rank-1 update to its entries -- two
// barriers per column and one reciprocal instead of a division per entry.  The
// published column alternates between two buffers, so the writers of column
// j + 1 never overwrite a value that a thread still finishing step j reads.
// FP64 issue slots are the scarce resource on this GPU (a warp instruction
// costs the same with most lanes masked), so the factorisation uses 32 x 32
// diagonal blocks: the per-column work of every thread stays at 4 entries.
template <int BS>
__global__ void __launch_bounds__(256) k_potrf_diag(int nbs, double* A, int lda, int* info, int base,
                                                    double floor_) {
  constexpr int RS = 256 / BS;        // row stride of a thread's entries
  constexpr int PER = BS / RS;        // entries per thread
  __shared__ double colbuf[2][BS];
  __shared__ double s_rinv;
  const int t = threadIdx.x;
  const int l = t % BS, i0 = t / BS;
  double a[PER];
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    const int i = i0 + RS * s;
    a[s] = (i < nbs && l < nbs && l <= i) ? A[(size_t)i * lda + l] : 0.0;
  }
  for (int j = 0; j < nbs; ++j) {
    double* colj = colbuf[j & 1];
    if (l == j) {
#pragma unroll
      for (int s = 0; s < PER; ++s) {
        if (i0 + RS * s != j) continue;
        double p = a[s];
        if (floor_ > 0.0) {
          // the matrix is known to satisfy A >= floor I, so every Cholesky pivot
          // (a Schur-complement diagonal) is >= floor; smaller ones are rounding
          if (!(p >= floor_)) {
            if (info) atomicAdd(info + 1, 1);
            p = floor_;
          }
        } else if (!(p > 0.0)) {
          if (info && *info == 0) *info = base + j + 1;
          p = 1.0;
        }
        const double dj = sqrt(p);
        a[s] = dj;
        colj[j] = dj;
        s_rinv = 1.0 / dj;
      }
    }
    __syncthreads();
    if (l == j) {
      const double r = s_rinv;
#pragma unroll
      for (int s = 0; s < PER; ++s) {
        const int i = i0 + RS * s;
        if (i > j && i < nbs) {
          a[s] *= r;
          colj[i] = a[s];
        }
      }
    }
    __syncthreads();
    if (l > j && l < nbs) {
      const double cl = colj[l];
#pragma unroll
      for (int s = 0; s < PER; ++s) {
        const int i = i0 + RS * s;
        if (i >= l && i < nbs) a[s] = fma(-colj[i], cl, a[s]);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    const int i = i0 + RS * s;
    if (i < nbs && l < nbs) A[(size_t)i * lda + l] = (l <= i) ? a[s] : 0.0;
  }
}

// Triangular solves with one kbs x kbs (kbs <= 64) diagonal block of L, one warp
// per right-hand-side vector: vector v has its entries at x0 + v * vstride +
// i * estride.  Lane q holds entries q and q + 32 in registers; column by column
// the finished entry is broadcast by a shuffle and the remaining entries are
// updated (no division: the reciprocals of the diagonal are precomputed).
//   trans = false:  L x = b  (forward);   trans = true:  L^T x = b  (backward)
// The right solve X L^T = P of the Cholesky panel is the forward solve on each
// row of P.
constexpr int TRSV_WARPS = 4;
__global__ void __launch_bounds__(32 * TRSV_WARPS) k_trsv_warp(int kbs, bool trans, const double* __restrict__ L,
                                                               int ldl, double* __restrict__ X, int nvec,
                                                               int vstride, int estride) {
  __shared__ double sl[NB][NB + 1];
  __shared__ double rd[NB];
  for (int t = threadIdx.x; t < kbs * kbs; t += blockDim.x) {
    const int i = t / kbs, j = t % kbs;
    sl[i][j] = (j <= i) ? L[(size_t)i * ldl + j] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kbs; i += blockDim.x) rd[i] = 1.0 / sl[i][i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int v = blockIdx.x * TRSV_WARPS + (threadIdx.x >> 5);
  if (v >= nvec) return;
  double* x = X + (size_t)v * vstride;
  const int e0 = lane, e1 = lane + 32;
  double x0 = (e0 < kbs) ? x[(size_t)e0 * estride] : 0.0;
  double x1 = (e1 < kbs) ? x[(size_t)e1 * estride] : 0.0;
  if (!trans) {
    for (int j = 0; j < kbs; ++j) {
      const double xj = __shfl_sync(0xffffffffu, (j < 32) ? x0 : x1, j & 31) * rd[j];
      if (e0 == j) x0 = xj;
      if (e1 == j) x1 = xj;
      if (e0 > j && e0 < kbs) x0 = fma(-sl[e0][j], xj, x0);
      if (e1 > j && e1 < kbs) x1 = fma(-sl[e1][j], xj, x1);
    }
  } else {
    for (int j = kbs - 1; j >= 0; --j) {
      const double xj = __shfl_sync(0xffffffffu, (j < 32) ? x0 : x1, j & 31) * rd[j];
      if (e0 == j) x0 = xj;
      if (e1 == j) x1 = xj;
      if (e0 < j) x0 = fma(-sl[j][e0], xj, x0);
      if (e1 < j) x1 = fma(-sl[j][e1], xj, x1);
    }
  }
  if (e0 < kbs) x[(size_t)e0 * estride] = x0;
  if (e1 < kbs) x[(size_t)e1 * estride] = x1;
}

size_t potrf_work_doubles(int n) { return (size_t)NB * NB + (size_t)n * NB; }

void potrf(cudaStream_t st, int n, double* A, int lda, int* info_dev, double* work) {
  potrf_floor(st, n, A, lda, info_dev, work, 0.0);
}

// Cholesky of a matrix known to satisfy A >= floor I (floor > 0): pivots below
// floor are raised to floor and counted in info_dev[1] instead of failing.
void potrf_floor(cudaStream_t st, int n, double* A, int lda, int* info_dev, double* work, double floor_) {

  (void)work;
  ktimer_begin(st, "potrf");
  cudaMemsetAsync(info_dev, 0, 2 * sizeof(int), st);
  constexpr int PB = 32;   // diagonal block of the factorisation (see k_potrf_diag)
  for (int k0 = 0; k0 < n; k0 += PB) {
    const int kbs = std::min(PB, n - k0);
    double* Akk = A + (size_t)k0 * lda + k0;
    count_launch();
    k_potrf_diag<PB><<<1, 256, 0, st>>>(kbs, Akk, lda, info_dev, k0, floor_);
    const int r0 = k0 + kbs;
    const int rows = n - r0;
    if (rows <= 0) break;
    double* P = A + (size_t)r0 * lda + k0;
    // panel: P <- P L_kk^{-T}, a forward solve on each row (one warp per row)
    count_launch();
    k_trsv_warp<<<cdiv(rows, TRSV_WARPS), 32 * TRSV_WARPS, 0, st>>>(kbs, false, Akk, lda, P, rows, lda, 1);
    // trailing: A22 -= P P^T (lower tiles only)
    gemm(st, false, true, rows, rows, kbs, -1.0, P, lda, P, lda, 1.0, A + (size_t)r0 * lda + r0, lda, 1);
  }
  zero_upper(st, n, A, lda);
  ktimer_end(st, "potrf", (double)n * n * n / 3.0, 8.0 * n * n);
}

size_t trsm_work_doubles(int n, int nrhs) {
  const int nblk = (n + NB - 1) / NB;
  return (size_t)nblk * NB * NB + (size_t)NB * nrhs;
}

void trsm_left_lower(cudaStream_t st, bool trans, int n, int nrhs, const double* L, int ldl, double* B,
                     int ldb, double* work) {
  trsm_left_lower_ex(st, trans, n, nrhs, L, ldl, B, ldb, work, false);
}

// lower_rhs: B is lower triangular (e.g. the identity when inverting L) and so
// is L^{-1} B, so block row k only has nonzero columns [0, k0 + kbs): the GEMMs
// are restricted to those columns, which brings the cost from n^3 to n^3 / 3.
void trsm_left_lower_ex(cudaStream_t st, bool trans, int n, int nrhs, const double* L, int ldl, double* B,
                        int ldb, double* work, bool lower_rhs) {
  (void)work;
  const int nblk = (n + NB - 1) / NB;
  ktimer_begin(st, "trsm");
  if (!trans) {
    for (int b = 0; b < nblk; ++b) {
      const int k0 = b * NB, kbs = std::min(NB, n - k0);
      const int nc = lower_rhs ? std::min(nrhs, k0 + kbs) : nrhs;
      double* Bk = B + (size_t)k0 * ldb;
      count_launch();
      k_trsv_warp<<<cdiv(nc, TRSV_WARPS), 32 * TRSV_WARPS, 0, st>>>(kbs, false, L + (size_t)k0 * ldl + k0, ldl, Bk, nc,
                                                                    1, ldb);
      const int r0 = k0 + kbs;
      if (r0 < n)
        gemm(st, false, false, n - r0, nc, kbs, -1.0, L + (size_t)r0 * ldl + k0, ldl, Bk, ldb, 1.0,
             B + (size_t)r0 * ldb, ldb);
    }
  } else {
    for (int b = nblk - 1; b >= 0; --b) {
      const int k0 = b * NB, kbs = std::min(NB, n - k0);
      double* Bk = B + (size_t)k0 * ldb;
      count_launch();
      k_trsv_warp<<<cdiv(nrhs, TRSV_WARPS), 32 * TRSV_WARPS, 0, st>>>(kbs, true, L + (size_t)k0 * ldl + k0, ldl, Bk,
                                                                      nrhs, 1, ldb);
      if (k0 > 0)
        gemm(st, true, false, k0, nrhs, kbs, -1.0, L + (size_t)k0 * ldl, ldl, Bk, ldb, 1.0, B, ldb);
    }
  }
  ktimer_end(st, "trsm", (double)n * n * nrhs, 8.0 * ((double)n * n / 2 + 2.0 * n * nrhs));
}

}  // namespace sdpgb
