// The Hessian operator of eq. (hesseqn2), applied matrix-free:
//   V  = sum_j v_j A_j          (gather over the CSR slots of the V pattern)
//   T  = W V                    (sparse-times-dense: T[r, l] = sum_{s in row l} V_ls W[r, s])
//   Hv_i = sum_{(p,q) in A_i} a_pq mult_pq W[p, :] . T[q, :]
// because (W V W)_pq = sum_l W_pl (V W)_lq = W[p, :] . (W V)[q, :] (V, W symmetric).
// T is produced row by row in its final layout, so no transpose is needed, and
// the per-entry dot products read two contiguous rows.
//
// The same CSR machinery serves the IPM: A(X) (op_A_dense), A^T y scattered into
// a dense matrix (scatter_V_dense) and sparse-times-dense products with U or Z.
//
// Reduced precision with the split W = W_l + W_s (W_l = E^T Lambda E, the top-k
// eigenpairs of the preconditioner build): near the optimum W_l holds the k
// eigenvalues of order 1/mu and W_s the rest, so rounding W itself to FP32 or
// BF16 erases W_s.  Instead only W_s V W_s runs in the reduced precision (SpMM
// and SDDMM as above); the other three terms are low rank,
//   (W_l V W_s + W_s V W_l)_pq = sum_l E[l][p] R[l][q] + E[l][q] R[l][p],
//   R = Lambda (E V) W_s  (k x n),
//   (W_l V W_l)_pq = E[:, p]^T Q E[:, q],  Q = Lambda (E V E^T) Lambda  (k x k),
// and are added per stored entry in FP64, so every term keeps a relative error
// of the working precision on its own scale.
#include "internal.cuh"

#include <algorithm>

namespace sdpgb {

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

template <typename T> __device__ __forceinline__ float tof(T x);
template <> __device__ __forceinline__ float tof<float>(float x) { return x; }
template <> __device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ double wsum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// K0: V values from v (gather form, no atomics)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void assemble_body(int s, int nnzV, const int* __restrict__ sptr,
                                              const int* __restrict__ scon, const double* __restrict__ scoef,
                                              const double* __restrict__ v, const double* __restrict__ scale,
                                              double* __restrict__ Vval) {
  if (s >= nnzV) return;
  double acc = 0.0;
  for (int c = sptr[s]; c < sptr[s + 1]; ++c) {
    const int k = scon[c];
    const double f = scale ? scale[k] : 1.0;
    acc = fma(scoef[c] * f, v[k], acc);
  }
  Vval[s] = acc;
}
__global__ void k_assemble(int nnzV, const int* __restrict__ sptr, const int* __restrict__ scon,
                           const double* __restrict__ scoef, const double* __restrict__ v,
                           const double* __restrict__ scale, double* __restrict__ Vval) {
  assemble_body(blockIdx.x * blockDim.x + threadIdx.x, nnzV, sptr, scon, scoef, v, scale, Vval);
}

void assemble_V(sdp_problem* h, const double* v, const double* scale, double* Vval) {
  count_launch();
  k_assemble<<<cdiv(h->nnzV, 256), 256, 0, h->stream>>>(h->nnzV, h->sptr, h->scon, h->scoef, v, scale, Vval);
}

// ---------------------------------------------------------------------------
// K1: T = W V, R rows of W per CTA staged in shared memory
// ---------------------------------------------------------------------------
constexpr int SPMM_UNROLL = 8;
// FP64: a CTA (SPMM_COLS threads) takes R rows of W and one chunk of SPMM_COLS
// rows of V: block blk = (row block) * chunks + chunk, so a problem has
// ceil(n / R) * ceil(n / SPMM_COLS) CTAs -- enough to fill the GPU when only a
// few problems of a batch are still iterating.  Thread t of chunk c handles
// row perm[c * SPMM_COLS + t] of V (rows by decreasing length, so that the
// lanes of a warp walk rows of about the same length).  Every entry of T is
// one thread's sum in the row's CSR order, whatever R and the chunking.
constexpr int SPMM_COLS = 256;
__host__ __device__ __forceinline__ int spmm_chunks(int n) { return (n + SPMM_COLS - 1) / SPMM_COLS; }
template <int R>
__device__ __forceinline__ void spmm_f64_body(int blk, int n, const int* __restrict__ rowptr,
                                              const int* __restrict__ perm, const int* __restrict__ colidx,
                                              const double* __restrict__ Vval, const double* __restrict__ W,
                                              double* __restrict__ T, double* wsh) {
  const int nc = spmm_chunks(n);
  const int r0 = (blk / nc) * R, t = (blk % nc) * SPMM_COLS + (int)threadIdx.x;
  for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
    const int rr = e / n, c = e % n;
    wsh[e] = (r0 + rr < n) ? W[(size_t)(r0 + rr) * n + c] : 0.0;
  }
  __syncthreads();
  if (t < n) {
    const int l = perm[t];
    double acc[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) acc[rr] = 0.0;
    const int s1 = rowptr[l + 1];
    int s = rowptr[l];
    // eight entries of column l per step: their loads are independent, so each
    // thread keeps eight L2 requests in flight instead of one
    for (; s + SPMM_UNROLL <= s1; s += SPMM_UNROLL) {
      int col[SPMM_UNROLL];
      double val[SPMM_UNROLL];
#pragma unroll
      for (int u = 0; u < SPMM_UNROLL; ++u) {
        col[u] = colidx[s + u];
        val[u] = Vval[s + u];
      }
#pragma unroll
      for (int u = 0; u < SPMM_UNROLL; ++u)
#pragma unroll
        for (int rr = 0; rr < R; ++rr) acc[rr] = fma(val[u], wsh[rr * n + col[u]], acc[rr]);
    }
    for (; s < s1; ++s) {
      const double val = Vval[s];
      const int col = colidx[s];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr] = fma(val, wsh[rr * n + col], acc[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (r0 + rr < n) T[(size_t)(r0 + rr) * n + l] = acc[rr];
  }
}
template <int R>
__global__ void __launch_bounds__(256) k_spmm_wv_f64(int n, const int* __restrict__ rowptr,
                                                     const int* __restrict__ perm,
                                                     const int* __restrict__ colidx,
                                                     const double* __restrict__ Vval,
                                                     const double* __restrict__ W, double* __restrict__ T) {
  extern __shared__ double wsh[];  // R x n
  spmm_f64_body<R>(blockIdx.x, n, rowptr, perm, colidx, Vval, W, T, wsh);
}

// Floats per staged column of the reduced-precision SpMM (see spmm_lp_body).
__host__ __device__ constexpr int spmm_lp_stride(int R) { return (R % 4 == 0) ? R + 4 : R; }
template <typename TW, int R>
__device__ __forceinline__ void spmm_lp_body(int blk, int n, const int* __restrict__ rowptr,
                                             const int* __restrict__ perm, const int* __restrict__ colidx,
                                             const double* __restrict__ Vval, const TW* __restrict__ W,
                                             float* __restrict__ T, float* fsh) {
  // no column chunks here: in FP32 the FMAs are cheap next to staging R rows
  // of W, so every CTA walks all rows of V for its R rows of W.  The R rows are
  // staged transposed with a row stride of RS = spmm_lp_stride(R) floats
  // (fsh[c * RS + rr]): the R values one stored entry of V needs are
  // contiguous (R / 4 vector loads), and the pad of 4 makes the stride an odd
  // number of 16-byte groups so that the random columns of a warp's lanes do
  // not all fall on the same banks (without it the kernel ran 1.4x slower;
  // with it, as fast as R scattered scalar loads: the CSR loads bound it).
  // Each acc[rr] sums in the same order as with any other layout.
  constexpr int RS = spmm_lp_stride(R);
  const int r0 = blk * R;
  for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
    const int rr = e / n, c = e % n;
    fsh[c * RS + rr] = (r0 + rr < n) ? tof<TW>(W[(size_t)(r0 + rr) * n + c]) : 0.f;
  }
  __syncthreads();
  auto fma_row = [&](float val, int col, float* acc) {
    const float* w = fsh + col * RS;
    if constexpr (R % 4 == 0) {
#pragma unroll
      for (int q = 0; q < R / 4; ++q) {
        const float4 w4 = reinterpret_cast<const float4*>(w)[q];
        acc[4 * q + 0] = fmaf(val, w4.x, acc[4 * q + 0]);
        acc[4 * q + 1] = fmaf(val, w4.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(val, w4.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(val, w4.w, acc[4 * q + 3]);
      }
    } else {
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr] = fmaf(val, w[rr], acc[rr]);
    }
  };
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int l = perm[t];
    float acc[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) acc[rr] = 0.f;
    const int s1 = rowptr[l + 1];
    int s = rowptr[l];
    for (; s + SPMM_UNROLL <= s1; s += SPMM_UNROLL) {
      int col[SPMM_UNROLL];
      float val[SPMM_UNROLL];
#pragma unroll
      for (int u = 0; u < SPMM_UNROLL; ++u) {
        col[u] = colidx[s + u];
        val[u] = (float)Vval[s + u];
      }
#pragma unroll
      for (int u = 0; u < SPMM_UNROLL; ++u) fma_row(val[u], col[u], acc);
    }
    for (; s < s1; ++s) fma_row((float)Vval[s], colidx[s], acc);
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (r0 + rr < n) T[(size_t)(r0 + rr) * n + l] = acc[rr];
  }
}
template <typename TW, int R>
__global__ void __launch_bounds__(256) k_spmm_wv_lp(int n, const int* __restrict__ rowptr,
                                                    const int* __restrict__ perm,
                                                    const int* __restrict__ colidx,
                                                    const double* __restrict__ Vval,
                                                    const TW* __restrict__ W, float* __restrict__ T) {
  extern __shared__ float fsh[];  // R x n
  spmm_lp_body<TW, R>(blockIdx.x, n, rowptr, perm, colidx, Vval, W, T, fsh);
}

// ---------------------------------------------------------------------------
// K2: per-constraint gather of W[p,:] . T[q,:]
// ---------------------------------------------------------------------------
// A warp serves SDDMM_G constraints, SDDMM_L = 32 / SDDMM_G lanes each: the
// cross-lane sums then cost log2(SDDMM_L) shuffle-adds per SDDMM_G constraints
// instead of five per constraint, which matters on a GPU whose FP64 pipe is
// the bound; the group's lanes read a row segment of SDDMM_L consecutive
// doubles, and the SDDMM_G groups of a warp read SDDMM_G rows at once.
// With dv != nullptr the kernel also forms dv . Hv (one deterministic grid
// reduction into *dout; PCG's p . Hp), first moving *pro_src to *pro_dst.
constexpr int SDDMM_G = 4;
constexpr int SDDMM_L = 32 / SDDMM_G;
constexpr int SDDMM_PER_BLOCK = (256 / 32) * SDDMM_G;   // constraints per 256-thread block
__device__ __forceinline__ double gsum_d(double v) {
#pragma unroll
  for (int o = SDDMM_L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float gsum_f(float v) {
#pragma unroll
  for (int o = SDDMM_L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ void sddmm_f64_body(int lb, int nb, int n, int m, const int* __restrict__ eptr,
                                               const int* __restrict__ ep, const int* __restrict__ eq,
                                               const double* __restrict__ ecoef, const double* __restrict__ W,
                                               const double* __restrict__ T, double* __restrict__ Hv,
                                               const double* __restrict__ dv, double* dpart, unsigned int* ticket,
                                               double* dout, double* pro_dst, const double* pro_src) {
  const int warp = (lb * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  const int gl = lane % SDDMM_L;
  const int i = warp * SDDMM_G + lane / SDDMM_L;
  const int e0 = (i < m) ? eptr[i] : 0, cnt = (i < m) ? eptr[i + 1] - e0 : 0;
  const int maxcnt = __reduce_max_sync(0xffffffffu, cnt);
  double acc = 0.0;
  for (int t = 0; t < maxcnt; ++t) {
    double s = 0.0;
    if (t < cnt) {
      const double* wp = W + (size_t)ep[e0 + t] * n;
      const double* tq = T + (size_t)eq[e0 + t] * n;
      int l = gl;
      for (; l + 3 * SDDMM_L < n; l += 4 * SDDMM_L) {   // four loads of each row in flight per lane
        const double w0 = wp[l], w1 = wp[l + SDDMM_L], w2 = wp[l + 2 * SDDMM_L], w3 = wp[l + 3 * SDDMM_L];
        const double t0 = tq[l], t1 = tq[l + SDDMM_L], t2 = tq[l + 2 * SDDMM_L], t3 = tq[l + 3 * SDDMM_L];
        s = fma(w0, t0, s);
        s = fma(w1, t1, s);
        s = fma(w2, t2, s);
        s = fma(w3, t3, s);
      }
      for (; l < n; l += SDDMM_L) s = fma(wp[l], tq[l], s);
    }
    s = gsum_d(s);   // every lane of the group holds the dot
    if (t < cnt) acc = fma(ecoef[e0 + t], s, acc);
  }
  if (i < m && gl == 0) Hv[i] = acc;
  if (dv) {
    const double c = (i < m && gl == 0) ? dv[i] * acc : 0.0;
    double tot;
    if (lb_reduce(c, dpart, ticket, &tot, lb, nb)) {
      if (pro_dst) *pro_dst = *pro_src;
      *dout = tot;
    }
  }
}
__global__ void __launch_bounds__(256) k_sddmm_f64(int n, int m, const int* __restrict__ eptr,
                                                   const int* __restrict__ ep, const int* __restrict__ eq,
                                                   const double* __restrict__ ecoef,
                                                   const double* __restrict__ W, const double* __restrict__ T,
                                                   double* __restrict__ Hv, const double* __restrict__ dv,
                                                   double* dpart, unsigned int* ticket, double* dout,
                                                   double* pro_dst, const double* pro_src) {
  sddmm_f64_body(blockIdx.x, gridDim.x, n, m, eptr, ep, eq, ecoef, W, T, Hv, dv, dpart, ticket, dout, pro_dst,
                 pro_src);
}

// ---------------------------------------------------------------------------
// Batched forms (one launch for every problem of a batch; see batch.cu)
// ---------------------------------------------------------------------------
__global__ void kb_assemble(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active) return;
  const int lb = blockIdx.x - off[i];
  assemble_body(lb * blockDim.x + threadIdx.x, D.nnzV, D.sptr, D.scon, D.scoef, D.pp, nullptr, D.Vval);
}
// R rows of W per CTA: chosen per batch by the autotuner (batch.cu); every R
// gives each entry of T by the same sequence of FMAs, so results do not depend on it
template <int R>
__global__ void __launch_bounds__(256) kb_spmm(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  extern __shared__ double wsh[];
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active || D.lp) return;
  spmm_f64_body<R>(blockIdx.x - off[i], D.n, D.rowptr, D.rowperm, D.colidx, D.Vval, D.W, D.T, wsh);
}
static void launch_kb_spmm(cudaStream_t st, int R, const BDesc* desc, const int* off, int N, int nb, int nmax) {
  const size_t smem = (size_t)R * nmax * sizeof(double);
  switch (R) {
    case 1: allow_max_smem((const void*)kb_spmm<1>); kb_spmm<1><<<nb, 256, smem, st>>>(desc, off, N); break;
    case 2: allow_max_smem((const void*)kb_spmm<2>); kb_spmm<2><<<nb, 256, smem, st>>>(desc, off, N); break;
    case 8: allow_max_smem((const void*)kb_spmm<8>); kb_spmm<8><<<nb, 256, smem, st>>>(desc, off, N); break;
    default: allow_max_smem((const void*)kb_spmm<4>); kb_spmm<4><<<nb, 256, smem, st>>>(desc, off, N); break;
  }
}
void batch_launch_spmm(cudaStream_t st, int R, const BDesc* desc, const int* off, int N, int nb, int nmax) {
  count_launch();
  if (nb > 0) launch_kb_spmm(st, R, desc, off, N, nb, nmax);
}
bool batch_spmm_fits(int R, int nmax) { return (size_t)R * nmax * sizeof(double) <= 200 * 1024; }
__global__ void __launch_bounds__(256) kb_sddmm(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active || D.lp) return;
  sddmm_f64_body(blockIdx.x - off[i], off[i + 1] - off[i], D.n, D.m, D.eptr, D.ep, D.eq, D.ecoef, D.W, D.T, D.pq,
                 D.pp, D.part, D.ticket, D.scal + S_PQ, D.scal + S_RZ, D.scal + S_RZN);
}
int batch_blocks_assemble(int nnzV) { return (int)cdiv(nnzV, 256); }
int batch_blocks_spmm(int n, int R) { return (int)cdiv(n, R) * spmm_chunks(n); }
int batch_blocks_sddmm(int m) { return (int)cdiv(m, SDDMM_PER_BLOCK); }
// nb_sddmm = 0 leaves the gather out (a mixed batch launches it with the
// reduced-precision one, batch_launch_sddmm_mixed)
void batch_launch_matvec(cudaStream_t st, const BDesc* desc, const int* off_asm, const int* off_spmm,
                         const int* off_sddmm, int N, int nb_asm, int nb_spmm, int nb_sddmm, int nmax, int spmm_r) {
  count_launch(nb_sddmm > 0 ? 3 : 2);
  if (nb_asm > 0) kb_assemble<<<nb_asm, 256, 0, st>>>(desc, off_asm, N);
  if (nb_spmm > 0) launch_kb_spmm(st, spmm_r, desc, off_spmm, N, nb_spmm, nmax);
  if (nb_sddmm > 0) kb_sddmm<<<nb_sddmm, 256, 0, st>>>(desc, off_sddmm, N);
}

template <typename TW>
__device__ __forceinline__ void sddmm_lp_body(int lb, int nb, int n, int m, const int* __restrict__ eptr,
                                              const int* __restrict__ ep, const int* __restrict__ eq,
                                              const double* __restrict__ ecoef, const TW* __restrict__ W,
                                              const float* __restrict__ T, double* __restrict__ Hv,
                                              const double* __restrict__ dv, double* dpart, unsigned int* ticket,
                                              double* dout, double* pro_dst, const double* pro_src, int k,
                                              const double* __restrict__ E, const float* __restrict__ R,
                                              const double* __restrict__ Q) {
  const int warp = (lb * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  const int gl = lane % SDDMM_L;
  const int i = warp * SDDMM_G + lane / SDDMM_L;
  const int e0 = (i < m) ? eptr[i] : 0, cnt = (i < m) ? eptr[i + 1] - e0 : 0;
  const int maxcnt = __reduce_max_sync(0xffffffffu, cnt);
  double hv = 0.0;
  for (int t = 0; t < maxcnt; ++t) {
    const bool on = t < cnt;
    const int p = on ? ep[e0 + t] : 0, q = on ? eq[e0 + t] : 0;
    float s = 0.f;
    if (on) {
      const TW* wp = W + (size_t)p * n;
      const float* tq = T + (size_t)q * n;
      int l = gl;
      for (; l + 3 * SDDMM_L < n; l += 4 * SDDMM_L) {
        const float w0 = tof<TW>(wp[l]), w1 = tof<TW>(wp[l + SDDMM_L]), w2 = tof<TW>(wp[l + 2 * SDDMM_L]),
                    w3 = tof<TW>(wp[l + 3 * SDDMM_L]);
        const float t0 = tq[l], t1 = tq[l + SDDMM_L], t2 = tq[l + 2 * SDDMM_L], t3 = tq[l + 3 * SDDMM_L];
        s = fmaf(w0, t0, s);
        s = fmaf(w1, t1, s);
        s = fmaf(w2, t2, s);
        s = fmaf(w3, t3, s);
      }
      for (; l < n; l += SDDMM_L) s = fmaf(tof<TW>(wp[l]), tq[l], s);
    }
    double v = (double)gsum_f(s);
    if (k > 0) {
      // low-rank terms of the split, in FP64, lane l of the group taking term l
      // (k <= SDDMM_L):  E[l][p] R[l][q] + E[l][q] R[l][p] + E[l][p] (Q E)[l][q]
      double tl = 0.0;
      if (on && gl < k) {
        const int l = gl;
        const double epl = E[(size_t)l * n + p], eql = E[(size_t)l * n + q];
        double qe = 0.0;
        for (int l2 = 0; l2 < k; ++l2) qe = fma(Q[l * k + l2], E[(size_t)l2 * n + q], qe);
        tl = epl * (double)R[(size_t)l * n + q];
        tl = fma(eql, (double)R[(size_t)l * n + p], tl);
        tl = fma(epl, qe, tl);
      }
      v += gsum_d(tl);
    }
    if (on) hv = fma(ecoef[e0 + t], v, hv);
  }
  if (i < m && gl == 0) Hv[i] = hv;
  if (dv) {
    const double c = (i < m && gl == 0) ? dv[i] * hv : 0.0;
    double tot;
    if (lb_reduce(c, dpart, ticket, &tot, lb, nb)) {
      if (pro_dst) *pro_dst = *pro_src;
      *dout = tot;
    }
  }
}
template <typename TW>
__global__ void __launch_bounds__(256) k_sddmm_lp(int n, int m, const int* __restrict__ eptr,
                                                  const int* __restrict__ ep, const int* __restrict__ eq,
                                                  const double* __restrict__ ecoef, const TW* __restrict__ W,
                                                  const float* __restrict__ T, double* __restrict__ Hv,
                                                  const double* __restrict__ dv, double* dpart, unsigned int* ticket,
                                                  double* dout, double* pro_dst, const double* pro_src, int k,
                                                  const double* __restrict__ E, const float* __restrict__ R,
                                                  const double* __restrict__ Q) {
  sddmm_lp_body<TW>(blockIdx.x, gridDim.x, n, m, eptr, ep, eq, ecoef, W, T, Hv, dv, dpart, ticket, dout, pro_dst,
                    pro_src, k, E, R, Q);
}

// Split: G^T[c][l] = (E V)[l][c] = sum_{s in row c} V[c][s] E[l][s] (V symmetric);
// one warp per row c.
__device__ __forceinline__ void split_G_body(int lb, int n, int k, const int* __restrict__ rowptr,
                                             const int* __restrict__ colidx, const double* __restrict__ Vval,
                                             const double* __restrict__ E, double* __restrict__ Gt) {
  const int c = (lb * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= n) return;
  double acc[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) acc[l] = 0.0;
  for (int s = rowptr[c] + lane; s < rowptr[c + 1]; s += 32) {
    const double v = Vval[s];
    const int col = colidx[s];
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (l < k) acc[l] = fma(v, E[(size_t)l * n + col], acc[l]);
  }
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    if (l >= k) break;
    const double t = wsum_d(acc[l]);
    if (lane == 0) Gt[(size_t)c * k + l] = t;
  }
}
__global__ void k_split_G(int n, int k, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                          const double* __restrict__ Vval, const double* __restrict__ E, double* __restrict__ Gt) {
  split_G_body(blockIdx.x, n, k, rowptr, colidx, Vval, E, Gt);
}

// Split: partial sums of (G W_s)[l][q] over a chunk of rows c (FP32; grid.y = chunk)
constexpr int SPLIT_CHUNKS = 16;
template <typename TW>
__device__ __forceinline__ void split_R_part_body(int bx, int by, int n, int k, const double* __restrict__ Gt,
                                                  const TW* __restrict__ Ws, float* __restrict__ part) {
  const int q = bx * blockDim.x + threadIdx.x;
  const int rows = (n + SPLIT_CHUNKS - 1) / SPLIT_CHUNKS;
  const int c0 = by * rows, c1 = min(n, c0 + rows);
  if (q >= n) return;
  float acc[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) acc[l] = 0.f;
#pragma unroll 4
  for (int c = c0; c < c1; ++c) {
    const float w = tof<TW>(Ws[(size_t)c * n + q]);
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (l < k) acc[l] = fmaf((float)Gt[(size_t)c * k + l], w, acc[l]);
  }
#pragma unroll
  for (int l = 0; l < 8; ++l)
    if (l < k) part[((size_t)by * k + l) * n + q] = acc[l];
}
template <typename TW>
__global__ void k_split_R_part(int n, int k, const double* __restrict__ Gt, const TW* __restrict__ Ws,
                               float* __restrict__ part) {
  split_R_part_body<TW>(blockIdx.x, blockIdx.y, n, k, Gt, Ws, part);
}
// R[l][q] = lambda_l sum_chunks part;  Q[l][l2] = lambda_l lambda_l2 sum_c G[l][c] E[l2][c]
// (the Q block is formed by the first k * k warps of the grid)
__device__ __forceinline__ void split_R_Q_body(int lb, int n, int k, const float* __restrict__ part,
                                               const double* __restrict__ lam, const double* __restrict__ Gt,
                                               const double* __restrict__ E, float* __restrict__ R,
                                               double* __restrict__ Q) {
  const int t = lb * blockDim.x + threadIdx.x;
  if (t < n * k) {
    const int l = t / n, q = t % n;
    float s = 0.f;
    for (int ch = 0; ch < SPLIT_CHUNKS; ++ch) s += part[((size_t)ch * k + l) * n + q];
    R[t] = (float)(lam[l] * (double)s);
  }
  const int w = t >> 5, lane = t & 31;
  if (w < k * k) {
    const int l = w / k, l2 = w % k;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s = fma(Gt[(size_t)c * k + l], E[(size_t)l2 * n + c], s);
    s = wsum_d(s);
    if (lane == 0) Q[l * k + l2] = lam[l] * lam[l2] * s;
  }
}
__global__ void k_split_R_Q(int n, int k, const float* __restrict__ part, const double* __restrict__ lam,
                            const double* __restrict__ Gt, const double* __restrict__ E, float* __restrict__ R,
                            double* __restrict__ Q) {
  split_R_Q_body(blockIdx.x, n, k, part, lam, Gt, E, R, Q);
}

// W_s = W - E^T diag(lam) E into Ws (n x n FP64)
__global__ void k_split_Ws(int n, int k, const double* __restrict__ W, const double* __restrict__ E,
                           const double* __restrict__ lam, double* __restrict__ Ws) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * n) return;
  const int a = (int)(t / n), b = (int)(t % n);
  double v = W[t];
  for (int l = 0; l < k; ++l) v = fma(-lam[l] * E[(size_t)l * n + a], E[(size_t)l * n + b], v);
  Ws[t] = v;
}

// Batched FP32 forms: the same bodies as the single-problem launches (problems
// in an FP64 sweep return at once).  Each entry of T is one thread's sum in the
// row's CSR order whatever the rows per CTA, so the batched SpMM may take more
// rows of W per CTA than a problem alone and still match it bit for bit: 16 (a
// quarter of the CSR re-reads of 4) while the staged rows of the batch's
// largest problem fit in 200 KB of shared memory, fewer for larger orders.
int batch_spmm_lp_rows(int nmax) {
  for (int r = 16; r > 1; r /= 2)
    if ((size_t)spmm_lp_stride(r) * nmax * sizeof(float) <= 200 * 1024) return r;
  return 1;
}
__global__ void __launch_bounds__(256) kb_split_G(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active || !D.lp || D.ks == 0) return;
  split_G_body(blockIdx.x - off[i], D.n, D.ks, D.rowptr, D.colidx, D.Vval, D.Etop, D.mvG);
}
__global__ void __launch_bounds__(128) kb_split_R_part(const BDesc* __restrict__ desc, const int* __restrict__ off,
                                                       int N) {
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active || !D.lp || D.ks == 0) return;
  const int lb = blockIdx.x - off[i], gx = (D.n + 127) / 128;
  if (D.bf) split_R_part_body<__nv_bfloat16>(lb % gx, lb / gx, D.n, D.ks, D.mvG, D.W16, D.mvPart);
  else split_R_part_body<float>(lb % gx, lb / gx, D.n, D.ks, D.mvG, D.W32, D.mvPart);
}
__global__ void __launch_bounds__(256) kb_split_R_Q(const BDesc* __restrict__ desc, const int* __restrict__ off,
                                                    int N) {
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active || !D.lp || D.ks == 0) return;
  split_R_Q_body(blockIdx.x - off[i], D.n, D.ks, D.mvPart, D.wtop, D.mvG, D.Etop, D.mvR, D.mvQ);
}
template <int R>
__global__ void __launch_bounds__(256) kb_spmm_lp(const BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  extern __shared__ float fsh[];
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active || !D.lp) return;
  if (D.bf)
    spmm_lp_body<__nv_bfloat16, R>(blockIdx.x - off[i], D.n, D.rowptr, D.rowperm, D.colidx, D.Vval,
                                                 D.W16, D.T32, fsh);
  else
    spmm_lp_body<float, R>(blockIdx.x - off[i], D.n, D.rowptr, D.rowperm, D.colidx, D.Vval, D.W32,
                                         D.T32, fsh);
}
__global__ void __launch_bounds__(256) kb_sddmm_lp(const BDesc* __restrict__ desc, const int* __restrict__ off,
                                                   int N) {
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active || !D.lp) return;
  if (D.bf)
    sddmm_lp_body<__nv_bfloat16>(blockIdx.x - off[i], off[i + 1] - off[i], D.n, D.m, D.eptr, D.ep, D.eq, D.ecoef,
                                 D.W16, D.T32, D.pq, D.pp, D.part, D.ticket, D.scal + S_PQ, D.scal + S_RZ,
                                 D.scal + S_RZN, D.ks, D.Etop, D.mvR, D.mvQ);
  else
    sddmm_lp_body<float>(blockIdx.x - off[i], off[i + 1] - off[i], D.n, D.m, D.eptr, D.ep, D.eq, D.ecoef, D.W32,
                         D.T32, D.pq, D.pp, D.part, D.ticket, D.scal + S_PQ, D.scal + S_RZ, D.scal + S_RZN, D.ks,
                         D.Etop, D.mvR, D.mvQ);
}
int batch_blocks_split_G(int n) { return (int)cdiv((size_t)n * 32, 256); }
int batch_blocks_split_R(int n) { return (int)cdiv(n, 128) * SPLIT_CHUNKS; }
int batch_blocks_split_Q(int n, int k) { return (int)cdiv(std::max((size_t)n * k, (size_t)k * k * 32), 256); }
int batch_blocks_spmm_lp(int n, int nmax) { return (int)cdiv(n, batch_spmm_lp_rows(nmax)); }
// Both gathers of a mixed batch in one launch: the two forms share the block
// partition (and the reduction groups), so each problem runs the same code as
// in its own launch.
__global__ void __launch_bounds__(256) kb_sddmm_mixed(const BDesc* __restrict__ desc, const int* __restrict__ off,
                                                      int N) {
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active) return;
  const int lb = blockIdx.x - off[i], nb = off[i + 1] - off[i];
  if (!D.lp)
    sddmm_f64_body(lb, nb, D.n, D.m, D.eptr, D.ep, D.eq, D.ecoef, D.W, D.T, D.pq, D.pp, D.part, D.ticket,
                   D.scal + S_PQ, D.scal + S_RZ, D.scal + S_RZN);
  else if (D.bf)
    sddmm_lp_body<__nv_bfloat16>(lb, nb, D.n, D.m, D.eptr, D.ep, D.eq, D.ecoef, D.W16, D.T32, D.pq, D.pp, D.part,
                                 D.ticket, D.scal + S_PQ, D.scal + S_RZ, D.scal + S_RZN, D.ks, D.Etop, D.mvR, D.mvQ);
  else
    sddmm_lp_body<float>(lb, nb, D.n, D.m, D.eptr, D.ep, D.eq, D.ecoef, D.W32, D.T32, D.pq, D.pp, D.part, D.ticket,
                         D.scal + S_PQ, D.scal + S_RZ, D.scal + S_RZN, D.ks, D.Etop, D.mvR, D.mvQ);
}
void batch_launch_sddmm_mixed(cudaStream_t st, const BDesc* desc, const int* off, int N, int nb) {
  count_launch();
  if (nb > 0) kb_sddmm_mixed<<<nb, 256, 0, st>>>(desc, off, N);
}

void batch_launch_matvec_lp(cudaStream_t st, const BDesc* desc, const int* off_g, const int* off_r,
                            const int* off_q, const int* off_spmm, const int* off_sddmm, int N, int nb_g, int nb_r,
                            int nb_q, int nb_spmm, int nb_sddmm, int nmax, bool with_sddmm) {
  const int R = batch_spmm_lp_rows(nmax);
  const size_t smem = (size_t)spmm_lp_stride(R) * nmax * sizeof(float);
  count_launch(with_sddmm ? 5 : 4);
  if (nb_g > 0) kb_split_G<<<nb_g, 256, 0, st>>>(desc, off_g, N);
  if (nb_r > 0) kb_split_R_part<<<nb_r, 128, 0, st>>>(desc, off_r, N);
  if (nb_q > 0) kb_split_R_Q<<<nb_q, 256, 0, st>>>(desc, off_q, N);
  if (nb_spmm > 0) {
    switch (R) {
      case 16: allow_max_smem((const void*)kb_spmm_lp<16>); kb_spmm_lp<16><<<nb_spmm, 256, smem, st>>>(desc, off_spmm, N); break;
      case 8: allow_max_smem((const void*)kb_spmm_lp<8>); kb_spmm_lp<8><<<nb_spmm, 256, smem, st>>>(desc, off_spmm, N); break;
      case 4: allow_max_smem((const void*)kb_spmm_lp<4>); kb_spmm_lp<4><<<nb_spmm, 256, smem, st>>>(desc, off_spmm, N); break;
      case 2: allow_max_smem((const void*)kb_spmm_lp<2>); kb_spmm_lp<2><<<nb_spmm, 256, smem, st>>>(desc, off_spmm, N); break;
      default: allow_max_smem((const void*)kb_spmm_lp<1>); kb_spmm_lp<1><<<nb_spmm, 256, smem, st>>>(desc, off_spmm, N); break;
    }
  }
  if (with_sddmm && nb_sddmm > 0) kb_sddmm_lp<<<nb_sddmm, 256, 0, st>>>(desc, off_sddmm, N);
}

// Reduced-precision copy of W, or of W_s when a preconditioner with top
// eigenpairs is built (the split form); keyed so that a new W or a rebuilt
// preconditioner refreshes it.
sdp_status ensure_lowprec_W(sdp_problem* h, int prec) {
  const int n = h->n;
  const size_t nn = (size_t)n * n;
  if (prec != SDP_FP32 && prec != SDP_BF16) return SDP_OK;
  if (!h->T32) SDP_TRY(h->allocT(&h->T32, nn));
  const bool split = h->pc_valid && h->kpc > 0 && h->Etop && h->KZ && h->kpc <= 8;
  const int64_t key = split ? h->pc_generation : -1;
  bool& valid = (prec == SDP_FP32) ? h->W32_valid : h->W16_valid;
  int64_t& have_key = (prec == SDP_FP32) ? h->W32_key : h->W16_key;
  if (valid && have_key == key) return SDP_OK;
  const double* src = h->W;
  cudaStream_t st = h->stream;
  if (split) {
    count_launch();
    k_split_Ws<<<cdiv(nn, 256), 256, 0, st>>>(n, h->kpc, h->W, h->Etop, h->wtop, h->KZ);
    src = h->KZ;
    if (!h->mv_G) {
      SDP_TRY(h->allocT(&h->mv_G, (size_t)n * 8));
      SDP_TRY(h->allocT(&h->mv_R, (size_t)n * 8));
      SDP_TRY(h->allocT(&h->mv_Q, 64));
      SDP_TRY(h->allocT(&h->mv_part, (size_t)SPLIT_CHUNKS * 8 * n));
    }
  }
  if (prec == SDP_FP32) {
    if (!h->W32) SDP_TRY(h->allocT(&h->W32, nn));
    to_f32(st, nn, src, h->W32);
  } else {
    if (!h->W16) SDP_TRY(h->allocT(&h->W16, nn));
    to_bf16(st, nn, src, h->W16);
  }
  valid = true;
  have_key = key;
  return SDP_OK;
}

// Rows of W per CTA of the SpMM: as many as shared memory allows (each CTA
// streams its chunk of the CSR of V once), but few enough that the grid still
// covers the SMs -- the FP64 form is bound by the SMs' DFMA rate, not by
// bandwidth.
static int rows_per_cta(int n, size_t elem) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const size_t budget = 96 * 1024;
  const int cap = (int)std::min<size_t>(8, budget / (elem * (size_t)n));
  for (int r = 8; r > 1; r /= 2)
    if (r <= cap && (n + r - 1) / r >= (sms * 9) / 10) return r;
  return 1;
}

template <int R>
static void launch_spmm_f64(sdp_problem* h, const double* Vval) {
  const size_t smem = (size_t)R * h->n * sizeof(double);
  allow_max_smem((const void*)k_spmm_wv_f64<R>);
  count_launch();
  k_spmm_wv_f64<R><<<cdiv(h->n, R) * spmm_chunks(h->n), SPMM_COLS, smem, h->stream>>>(h->n, h->rowptr, h->rowperm, h->colidx, Vval, h->W,
                                                              h->T);
}
template <typename TW, int R>
static void launch_spmm_lp(sdp_problem* h, const double* Vval, const TW* W) {
  const size_t smem = (size_t)spmm_lp_stride(R) * h->n * sizeof(float);
  allow_max_smem((const void*)k_spmm_wv_lp<TW, R>);
  count_launch();
  k_spmm_wv_lp<TW, R><<<cdiv(h->n, R), SPMM_COLS, smem, h->stream>>>(h->n, h->rowptr, h->rowperm, h->colidx, Vval, W,
                                                                 h->T32);
}

sdp_status matvec_impl(sdp_problem* h, const double* v, double* Hv, int prec, double* dot_out, double* pro_dst,
                       const double* pro_src) {
  const double* dv = dot_out ? v : nullptr;
  if (!h->have_W) {
    h->last_error = "hessian_matvec: no scaling matrix W (call sdp_set_W or sdp_ipm_step)";
    return SDP_ERR_ARG;
  }
  const int n = h->n;
  const bool timed = ktimer_on("matvec");
  if (timed) ktimer_begin(h->stream, "matvec");
  assemble_V(h, v, nullptr, h->Vval);
  if (prec == SDP_FP64) {
    switch (rows_per_cta(n, sizeof(double))) {
      case 8: launch_spmm_f64<8>(h, h->Vval); break;
      case 4: launch_spmm_f64<4>(h, h->Vval); break;
      case 2: launch_spmm_f64<2>(h, h->Vval); break;
      default: launch_spmm_f64<1>(h, h->Vval); break;
    }
    count_launch();
    k_sddmm_f64<<<cdiv(h->m, SDDMM_PER_BLOCK), 256, 0, h->stream>>>(n, h->m, h->eptr, h->ep, h->eq, h->ecoef,
                                                                     h->W, h->T, Hv, dv, h->pcg_part,
                                                                     h->pcg_ticket, dot_out, pro_dst, pro_src);
  } else if (prec == SDP_FP32 || prec == SDP_BF16) {
    SDP_TRY(ensure_lowprec_W(h, prec));
    const bool split = (prec == SDP_FP32 ? h->W32_key : h->W16_key) >= 0;
    const int ks = split ? h->kpc : 0;
    if (split) {
      count_launch(3);
      k_split_G<<<cdiv((size_t)n * 32, 256), 256, 0, h->stream>>>(n, ks, h->rowptr, h->colidx, h->Vval, h->Etop,
                                                                    h->mv_G);
      if (prec == SDP_FP32)
        k_split_R_part<float><<<dim3(cdiv(n, 128), SPLIT_CHUNKS), 128, 0, h->stream>>>(n, ks, h->mv_G, h->W32,
                                                                                       h->mv_part);
      else
        k_split_R_part<__nv_bfloat16><<<dim3(cdiv(n, 128), SPLIT_CHUNKS), 128, 0, h->stream>>>(
            n, ks, h->mv_G, h->W16, h->mv_part);
      const size_t th = std::max((size_t)n * ks, (size_t)ks * ks * 32);
      k_split_R_Q<<<cdiv(th, 256), 256, 0, h->stream>>>(n, ks, h->mv_part, h->wtop, h->mv_G, h->Etop, h->mv_R,
                                                        h->mv_Q);
    }
  }
  if (prec == SDP_FP32) {
    switch (rows_per_cta(n, sizeof(float))) {
      case 8: launch_spmm_lp<float, 8>(h, h->Vval, h->W32); break;
      case 4: launch_spmm_lp<float, 4>(h, h->Vval, h->W32); break;
      case 2: launch_spmm_lp<float, 2>(h, h->Vval, h->W32); break;
      default: launch_spmm_lp<float, 1>(h, h->Vval, h->W32); break;
    }
    count_launch();
    k_sddmm_lp<float><<<cdiv(h->m, SDDMM_PER_BLOCK), 256, 0, h->stream>>>(
        n, h->m, h->eptr, h->ep, h->eq, h->ecoef, h->W32, h->T32, Hv, dv, h->pcg_part, h->pcg_ticket, dot_out,
        pro_dst, pro_src, h->W32_key >= 0 ? h->kpc : 0, h->Etop, h->mv_R, h->mv_Q);
  } else if (prec == SDP_BF16) {
    switch (rows_per_cta(n, sizeof(float))) {
      case 8: launch_spmm_lp<__nv_bfloat16, 8>(h, h->Vval, h->W16); break;
      case 4: launch_spmm_lp<__nv_bfloat16, 4>(h, h->Vval, h->W16); break;
      case 2: launch_spmm_lp<__nv_bfloat16, 2>(h, h->Vval, h->W16); break;
      default: launch_spmm_lp<__nv_bfloat16, 1>(h, h->Vval, h->W16); break;
    }
    count_launch();
    k_sddmm_lp<__nv_bfloat16><<<cdiv(h->m, SDDMM_PER_BLOCK), 256, 0, h->stream>>>(
        n, h->m, h->eptr, h->ep, h->eq, h->ecoef, h->W16, h->T32, Hv, dv, h->pcg_part, h->pcg_ticket, dot_out,
        pro_dst, pro_src, h->W16_key >= 0 ? h->kpc : 0, h->Etop, h->mv_R, h->mv_Q);
  } else if (prec != SDP_FP64) {
    h->last_error = "hessian_matvec: unknown precision";
    return SDP_ERR_ARG;
  }
  if (timed) {
    // algorithmic work: T = W V (2 nnzV n flops), one length-n dot per stored entry;
    // bytes: W read for T, T written, W and T rows read by the gather (4 n^2 s) + sparse data
    const double s = (prec == SDP_FP64) ? 8.0 : (prec == SDP_FP32 ? 4.0 : 3.0);
    const double f = 2.0 * h->nnzV * (double)n + 2.0 * h->nent * (double)n;
    const double by = 4.0 * s * n * (double)n + 12.0 * h->nnzV + 16.0 * h->m;
    ktimer_end(h->stream, "matvec", f, by);
  }
  return SDP_OK;
}

// ---------------------------------------------------------------------------
// Sparse helpers for the IPM and the preconditioner
// ---------------------------------------------------------------------------
// out[i] = alpha * A_i . X + beta * add[i]   (X symmetric)
__global__ void k_opA(int m, const int* __restrict__ eptr, const int* __restrict__ ep,
                      const int* __restrict__ eq, const double* __restrict__ ecoef, int n,
                      const double* __restrict__ X, double* __restrict__ out, double alpha,
                      const double* __restrict__ add, double beta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int e = eptr[i]; e < eptr[i + 1]; ++e) s = fma(ecoef[e], X[(size_t)ep[e] * n + eq[e]], s);
  out[i] = alpha * s + (add ? beta * add[i] : 0.0);
}
void op_A_dense(sdp_problem* h, const double* X, double* out, double alpha, const double* add, double beta) {
  count_launch();
  k_opA<<<cdiv(h->m, 256), 256, 0, h->stream>>>(h->m, h->eptr, h->ep, h->eq, h->ecoef, h->n, X, out, alpha,
                                                add, beta);
}

// D[row][col] += alpha * Vval[s]  over every slot of the V pattern
__global__ void k_scatter(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                          const double* __restrict__ Vval, double alpha, double* __restrict__ D) {
  const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (r >= n) return;
  for (int s = rowptr[r] + lane; s < rowptr[r + 1]; s += 32) D[(size_t)r * n + colidx[s]] += alpha * Vval[s];
}
void scatter_V_dense(sdp_problem* h, const double* Vval, double alpha, double* D) {
  count_launch();
  k_scatter<<<cdiv((size_t)h->n * 32, 256), 256, 0, h->stream>>>(h->n, h->rowptr, h->colidx, Vval, alpha, D);
}

// out[a, c] = sum_{s in row a} val[s] B[col(s), c]   (c < ncols)
__global__ void k_spmm_rows(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                            const double* __restrict__ val, const double* __restrict__ B, int ldb, int ncols,
                            double* __restrict__ out, int ldo) {
  const int a = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = rowptr[a]; s < rowptr[a + 1]; ++s) acc = fma(val[s], B[(size_t)colidx[s] * ldb + c], acc);
    out[(size_t)a * ldo + c] = acc;
  }
}
void spmm_rows(sdp_problem* h, const double* Vval, const double* B, int ldb, int ncols, double* out, int ldo) {
  count_launch();
  const unsigned gx = std::max(1u, std::min(cdiv(ncols, 128), 64u));
  k_spmm_rows<<<dim3(gx, h->n), 128, 0, h->stream>>>(h->n, h->rowptr, h->colidx, Vval, B, ldb, ncols, out, ldo);
}

}  // namespace sdpgb
