// Tensor-core GEMM for the reduced-precision Woodbury core formation.
//
// Algorithm 1 step 2 forms the core blocks Z^T (K_ll' Z) -- n x n x n dense
// products, k(k+1)/2 of them per build.  With a reduced-precision PCG
// (params.prec = SDP_FP32 or SDP_BF16) these run on the 5th-generation tensor
// cores: the operands are rounded to TF32 (FP32) or BF16, the products
// accumulate in FP32 in tensor memory, and the block is written back in FP64,
// where the factorisation of the core stays (FP64 Cholesky with the tau^2 pivot
// floor).
//
// One CTA computes a 128 x 128 tile of C = A B^T with A (M x K) and B (N x K)
// both K-major in global memory (rows of K contiguous, padded to the tile
// sizes).  Four warps:
//   warp 0, one lane : TMA producer -- cp.async.bulk.tensor loads of 128 x 128-byte
//                      tiles of A and B (128-byte swizzle) into a STAGES-deep ring,
//                      completion counted on an mbarrier per stage;
//   warp 1, one lane : MMA issuer -- tcgen05.mma (M = N = 128, K = 32 bytes per
//                      instruction) from shared-memory descriptors into one
//                      128-column FP32 accumulator in tensor memory; tcgen05.commit
//                      frees a stage once its MMAs have read it;
//   all four warps   : epilogue -- tcgen05.ld of the warp's 32 accumulator lanes
//                      (rows), converted to FP64 and stored.
// Every mbarrier wait is bounded: a wait that runs out sets an error flag (read
// by the host as SDP_ERR_TIMEOUT) and the CTA skips ahead to free its tensor
// memory and return.
#include "internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

namespace sdpgb {

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

constexpr int TC_TM = 128;          // tile rows (accumulator lanes)
constexpr int TC_TN = 128;          // tile columns (accumulator columns)
constexpr int TC_ROWB = 128;        // bytes of K per tile row and stage (one 128-byte swizzle atom)
constexpr int TC_STAGES = 4;
constexpr int TC_TILE_BYTES = TC_TM * TC_ROWB;      // 16 KiB per operand tile
constexpr int TC_STAGE_BYTES = 2 * TC_TILE_BYTES;   // A and B
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
constexpr long long TC_WAIT_SPINS = 1ll << 26;       // bound of one mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the phase with the given parity; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < TC_WAIT_SPINS; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte
// swizzle layout that the TMA load writes: rows of 128 bytes, 8-row atoms of
// 1024 bytes (stride byte offset), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused by this layout)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, A and B K-major, M = 128, N = 128;
// fmt = 1 (BF16, kind::f16) or 2 (TF32, kind::tf32).
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_TN >> 3) << 17) | ((uint32_t)(TC_TM >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// C[M x N] (FP64, row stride ldc) = A B^T over nkb K blocks of 128 bytes.
template <bool BF16>
__global__ void __launch_bounds__(128) k_tc_gemm(const __grid_constant__ CUtensorMap mapA,
                                                 const __grid_constant__ CUtensorMap mapB, int M, int N, int nkb,
                                                 double* __restrict__ C, int ldc, int* err) {
  extern __shared__ uint8_t tc_smem_raw[];
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;          // swizzle atoms need 1024-byte alignment
  uint8_t* gbase = tc_smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + TC_STAGES * TC_STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_STAGES + 2);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (TC_STAGES + s); };
  const uint32_t done_bar = bar0 + 8u * (2 * TC_STAGES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_TM, n0 = blockIdx.x * TC_TN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % TC_STAGES;
      if (kb >= TC_STAGES && !mbar_wait(empty_bar(s), ((kb / TC_STAGES) - 1) & 1)) {
        atomicExch(err, 1);
        break;
      }
      const uint32_t sa = base + s * TC_STAGE_BYTES, sb = sa + TC_TILE_BYTES;
      mbar_expect_tx(full_bar(s), TC_STAGE_BYTES);
      const int x = kb * (TC_ROWB / (BF16 ? 2 : 4));   // element coordinate along K
      tma_load_2d(sa, &mapA, x, m0, full_bar(s));
      tma_load_2d(sb, &mapB, x, n0, full_bar(s));
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 instructions of 32 bytes of K per stage
    constexpr uint32_t idesc = tc_idesc(BF16 ? 1u : 2u);
    bool ok = true;
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int s = kb % TC_STAGES;
      if (!mbar_wait(full_bar(s), (kb / TC_STAGES) & 1)) {
        atomicExch(err, 1);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = base + s * TC_STAGE_BYTES, sb = sa + TC_TILE_BYTES;
#pragma unroll
      for (int kk = 0; kk < TC_ROWB / 32; ++kk)
        tc_mma<BF16>(tmem, sw128_desc(sa + 32 * kk), sw128_desc(sb + 32 * kk), idesc, (kb | kk) ? 1u : 0u);
      tc_commit(empty_bar(s));
    }
    tc_commit(done_bar);
  }
  __syncwarp();
  // epilogue: warp w reads accumulator lanes (rows) 32 w .. 32 w + 31
  const bool have = __all_sync(0xffffffffu, mbar_wait(done_bar, 0) ? 1 : 0) != 0;   // warp-uniform
  if (!have && lane == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have) {
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < TC_TN; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < M) {
        double* cr = C + (size_t)row * ldc + n0 + c0;
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (n0 + c0 + i < N) cr[i] = (double)v[i];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TN));
}

// dst[r][c] (R x Kp, K-major, zero padded) = src[c][r] (trans) or src[r][c], rounded
template <typename T>
__device__ __forceinline__ T tc_round(double x);
template <> __device__ __forceinline__ __nv_bfloat16 tc_round<__nv_bfloat16>(double x) {
  return __float2bfloat16_rn((float)x);
}
// TF32 operands: rounded to nearest here (the tensor core itself would drop the
// low 13 mantissa bits of an FP32 input, i.e. truncate)
template <> __device__ __forceinline__ float tc_round<float>(double x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)x));
  return __uint_as_float(r);
}

template <typename T>
__global__ void k_tc_pack(int rows, int cols, const double* __restrict__ src, int lds, bool trans, int R, int Kp,
                          T* __restrict__ dst) {
  __shared__ double tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  // dst rows r (operand rows) and columns c (K); the source tile is read along
  // its contiguous dimension and transposed through shared memory when needed
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    double v = 0.0;
    if (trans) {
      const int c = c0 + i, r = r0 + threadIdx.x;   // src[c][r]: threadIdx.x runs along r (contiguous)
      if (r < rows && c < cols) v = src[(size_t)c * lds + r];
      tile[threadIdx.x][i] = v;
    } else {
      const int r = r0 + i, c = c0 + threadIdx.x;
      if (r < rows && c < cols) v = src[(size_t)r * lds + c];
      tile[i][threadIdx.x] = v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < Kp) dst[(size_t)r * Kp + c] = tc_round<T>(tile[i][threadIdx.x]);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

static bool make_map(CUtensorMap* map, void* base, bool bf16, int rows, int kp) {
  auto fn = encode_fn();
  if (!fn) return false;
  const size_t es = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * es};
  cuuint32_t box[2] = {(cuuint32_t)(TC_ROWB / es), (cuuint32_t)TC_TM};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_available() { return encode_fn() != nullptr; }

size_t tc_work_bytes(int M, int N, int K) {
  const size_t Mp = cdiv(M, TC_TM) * (size_t)TC_TM, Np = cdiv(N, TC_TN) * (size_t)TC_TN;
  const size_t Kp = cdiv(K, 64) * (size_t)64;
  return (Mp + Np) * Kp * 4 + 256;   // room for FP32 (TF32) operands; BF16 uses half
}

// C = op(A) op(B) in reduced precision on the tensor cores; op(A) is M x K, op(B) is
// K x N.  The operands are packed K-major into work (tc_work_bytes), A from a
// row-major A (transA: A holds op(A)^T) and B likewise.  err_dev: one int, set on
// a bounded-wait timeout.
sdp_status tc_gemm(cudaStream_t st, int prec, int M, int N, int K, const double* A, int lda, bool transA,
                   const double* B, int ldb, bool transB, double* C, int ldc, void* work, int* err_dev) {
  if (M <= 0 || N <= 0 || K <= 0) return SDP_OK;
  const bool bf16 = (prec == SDP_BF16);
  const int Mp = (int)(cdiv(M, TC_TM) * TC_TM), Np = (int)(cdiv(N, TC_TN) * TC_TN);
  const int kpe = TC_ROWB / (bf16 ? 2 : 4);   // elements of K per block
  const int Kp = (int)(cdiv(K, kpe) * kpe);
  const size_t es = bf16 ? 2 : 4;
  uint8_t* wa = static_cast<uint8_t*>(work);
  uint8_t* wb = wa + (((size_t)Mp * Kp * es + 255) / 256) * 256;
  const dim3 tb(32, 8);
  // op(A)[r][k]: A row-major is op(A) itself (no trans) or its transpose (trans)
  count_launch(2);
  if (bf16) {
    k_tc_pack<__nv_bfloat16><<<dim3(cdiv(Kp, 32), cdiv(Mp, 32)), tb, 0, st>>>(
        M, K, A, lda, transA, Mp, Kp, reinterpret_cast<__nv_bfloat16*>(wa));
    // the B operand is op(B)^T (N x K): row n, column k = op(B)[k][n]
    k_tc_pack<__nv_bfloat16><<<dim3(cdiv(Kp, 32), cdiv(Np, 32)), tb, 0, st>>>(
        N, K, B, ldb, !transB, Np, Kp, reinterpret_cast<__nv_bfloat16*>(wb));
  } else {
    k_tc_pack<float><<<dim3(cdiv(Kp, 32), cdiv(Mp, 32)), tb, 0, st>>>(M, K, A, lda, transA, Mp, Kp,
                                                                       reinterpret_cast<float*>(wa));
    k_tc_pack<float><<<dim3(cdiv(Kp, 32), cdiv(Np, 32)), tb, 0, st>>>(N, K, B, ldb, !transB, Np, Kp,
                                                                       reinterpret_cast<float*>(wb));
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, wa, bf16, Mp, Kp) || !make_map(&mb, wb, bf16, Np, Kp)) return SDP_ERR_CUDA;
  const dim3 grid(Np / TC_TN, Mp / TC_TM);
  const int nkb = Kp / kpe;
  if (grid.y > 65535u) return SDP_ERR_ARG;
  count_launch();
  if (bf16) {
    allow_max_smem((const void*)k_tc_gemm<true>);
    k_tc_gemm<true><<<grid, 128, TC_SMEM, st>>>(ma, mb, M, N, nkb, C, ldc, err_dev);
  } else {
    allow_max_smem((const void*)k_tc_gemm<false>);
    k_tc_gemm<false><<<grid, 128, TC_SMEM, st>>>(ma, mb, M, N, nkb, C, ldc, err_dev);
  }
  return cudaGetLastError() == cudaSuccess ? SDP_OK : SDP_ERR_CUDA;
}

}  // namespace sdpgb

using namespace sdpgb;

extern "C" int64_t sdp_mixed_gemm_work_bytes(int M, int N, int K) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  return (int64_t)tc_work_bytes(M, N, K);
}

extern "C" sdp_status sdp_mixed_gemm(int prec, int M, int N, int K, const double* A_dev, int lda, int transA,
                                     const double* B_dev, int ldb, int transB, double* C_dev, int ldc,
                                     void* work_dev, int64_t work_bytes, int* err_dev, void* cuda_stream) {
  if ((prec != SDP_FP32 && prec != SDP_BF16) || M < 0 || N < 0 || K < 0 || !A_dev || !B_dev || !C_dev ||
      !work_dev || !err_dev || ldc < N)
    return SDP_ERR_ARG;
  if (lda < (transA ? M : K) || ldb < (transB ? K : N)) return SDP_ERR_ARG;
  if (work_bytes < sdp_mixed_gemm_work_bytes(M, N, K)) return SDP_ERR_ARG;
  if (!tc_available()) return SDP_ERR_UNSUPPORTED;
  return tc_gemm(static_cast<cudaStream_t>(cuda_stream), prec, M, N, K, A_dev, lda, transA != 0, B_dev, ldb,
                 transB != 0, C_dev, ldc, work_dev, err_dev);
}
