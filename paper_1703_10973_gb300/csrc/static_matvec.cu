// Handle-free Hessian matvec with statically allocated scratch.
//
// sdp_hessian_matvec_static computes the product of eq. (hesseqn2),
//   Hv_k = A_k . (W V W),  V = sum_j v_j A_j,
// like sdp_hessian_matvec, but straight from the constraint triplets and a
// caller-supplied W, for callers that cannot allocate device memory: there is
// no handle, and no cudaMalloc / cudaFree / allocating call on this path.  The
// scratch is two n x n FP64 matrices in one file-scope __device__ array, which
// caps n at SDP_STATIC_MAX_N = 512 (4 MiB of static device memory, present in
// every context that loads the library).
//
//   1. clear VW, Hv and the skipped-entry counter (all accumulate atomically)
//   2. for each entry (k, a, b, c) with w = c v_k:
//        VW[a, :] += w W[b, :];  VW[b, :] += w W[a, :] (a != b)   ->  VW = V W
//   3. T = VW^T = W V (tiled transpose)
//   4. Hv_k += c mult W[a, :] . T[b, :],  mult = 2 off the diagonal, because
//      (W V W)_ab = sum_l W_al (V W)_lb = W[a, :] . T[b, :]
//
// Entries with an index out of range are skipped and counted; the call then
// returns SDP_ERR_ARG.  Both scratch matrices are shared by every call in the
// process on a device, so calls that overlap in time (two streams, two host
// threads) race and must be serialised by the caller.
#include "internal.cuh"

#include <algorithm>
#include <mutex>

namespace sdpgb {

// ceil(a / b) clamped to [1, cap]
static inline unsigned cdiv_cap(int64_t a, int64_t b, int64_t cap) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((a + b - 1) / b, cap));
}

constexpr int SMAX = SDP_STATIC_MAX_N;
static __device__ __align__(256) double g_static_scratch[2 * SMAX * SMAX];
static __device__ __align__(256) unsigned long long g_static_skipped;

__global__ void k_st_clear(int nn, double* __restrict__ VW, int m, double* __restrict__ Hv,
                           unsigned long long* skipped) {
  const int stride = gridDim.x * blockDim.x;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += stride) VW[t] = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += stride) Hv[t] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *skipped = 0ull;
}

__device__ __forceinline__ bool st_entry_ok(int n, int m, int k, int a, int b) {
  return k >= 0 && k < m && a >= 0 && a < n && b >= 0 && b < n;
}

// one warp per entry (grid-stride over entries), lanes over the row
__global__ void k_st_scatter(int n, int m, int64_t nnz, const int32_t* __restrict__ Ak,
                             const int32_t* __restrict__ Ai, const int32_t* __restrict__ Aj,
                             const double* __restrict__ Av, const double* __restrict__ v,
                             const double* __restrict__ W, double* __restrict__ VW, unsigned long long* skipped) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nnz; e += nwarps) {
    const int k = Ak[e], a = Ai[e], b = Aj[e];
    if (!st_entry_ok(n, m, k, a, b)) {
      if (lane == 0) atomicAdd(skipped, 1ull);
      continue;
    }
    const double w = Av[e] * v[k];
    for (int r = lane; r < n; r += 32) {
      atomicAdd(&VW[(size_t)a * n + r], w * W[(size_t)b * n + r]);
      if (a != b) atomicAdd(&VW[(size_t)b * n + r], w * W[(size_t)a * n + r]);
    }
  }
}

// T[r][a] = VW[a][r], 32 x 32 tiles through shared memory
__global__ void k_st_transpose(int n, const double* __restrict__ VW, double* __restrict__ T) {
  __shared__ double tile[32][33];
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int y = y0 + dy, x = x0 + threadIdx.x;
    if (y < n && x < n) tile[dy][threadIdx.x] = VW[(size_t)y * n + x];
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int y = x0 + dy, x = y0 + threadIdx.x;   // output row y = input column
    if (y < n && x < n) T[(size_t)y * n + x] = tile[threadIdx.x][dy];
  }
}

__global__ void k_st_gather(int n, int m, int64_t nnz, const int32_t* __restrict__ Ak,
                            const int32_t* __restrict__ Ai, const int32_t* __restrict__ Aj,
                            const double* __restrict__ Av, const double* __restrict__ W,
                            const double* __restrict__ T, double* __restrict__ Hv) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nnz; e += nwarps) {
    const int k = Ak[e], a = Ai[e], b = Aj[e];
    if (!st_entry_ok(n, m, k, a, b)) continue;
    const double* wa = W + (size_t)a * n;
    const double* tb = T + (size_t)b * n;
    double s = 0.0;
    for (int l = lane; l < n; l += 32) s = fma(wa[l], tb[l], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicAdd(&Hv[k], (a != b ? 2.0 : 1.0) * Av[e] * s);
  }
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_sym_mu;
double* g_sym_scratch[kMaxDevices] = {};
unsigned long long* g_sym_skipped[kMaxDevices] = {};
}  // namespace

// Device addresses of the static scratch, looked up once per device.  The first
// lookup on a device may load the module into the current context.
static cudaError_t static_scratch(double** scratch, unsigned long long** skipped) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_sym_mu);
  if (!g_sym_scratch[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&q, g_static_skipped);
    if (e != cudaSuccess) return e;
    g_sym_scratch[dev] = static_cast<double*>(p);
    g_sym_skipped[dev] = static_cast<unsigned long long*>(q);
  }
  *scratch = g_sym_scratch[dev];
  *skipped = g_sym_skipped[dev];
  return cudaSuccess;
}

static thread_local std::string t_free_error;
const char* free_call_error() { return t_free_error.c_str(); }

static sdp_status fail(sdp_status s, const std::string& msg) {
  t_free_error = msg;
  return s;
}

}  // namespace sdpgb

extern "C" sdp_status sdp_hessian_matvec_static(int n, int m, int64_t nnzA, const int32_t* Ak_dev,
                                                const int32_t* Ai_dev, const int32_t* Aj_dev, const double* Av_dev,
                                                const double* W_dev, const double* v_dev, double* Hv_dev,
                                                void* cuda_stream) {
  using namespace sdpgb;
  t_free_error.clear();
  if (n < 1 || n > SDP_STATIC_MAX_N)
    return fail(SDP_ERR_ARG, "hessian_matvec_static: n = " + std::to_string(n) +
                                 " is outside [1, SDP_STATIC_MAX_N = " + std::to_string(SDP_STATIC_MAX_N) +
                                 "] (the static scratch holds two n x n matrices); use sdp_hessian_matvec");
  if (m < 1) return fail(SDP_ERR_ARG, "hessian_matvec_static: m must be positive");
  if (nnzA < 0) return fail(SDP_ERR_ARG, "hessian_matvec_static: nnzA must be non-negative");
  if (nnzA > 0 && (!Ak_dev || !Ai_dev || !Aj_dev || !Av_dev))
    return fail(SDP_ERR_ARG, "hessian_matvec_static: null triplet pointer");
  if (!W_dev || !v_dev || !Hv_dev) return fail(SDP_ERR_ARG, "hessian_matvec_static: null W, v or Hv pointer");
  // Hv is cleared before v and W are read, so it may share no byte with them
  auto overlap = [](const void* a, size_t na, const void* b, size_t nb) {
    const char *pa = static_cast<const char*>(a), *pb = static_cast<const char*>(b);
    return pa < pb + nb && pb < pa + na;
  };
  const size_t hv_bytes = (size_t)m * sizeof(double);
  if (overlap(Hv_dev, hv_bytes, v_dev, (size_t)m * sizeof(double)) ||
      overlap(Hv_dev, hv_bytes, W_dev, (size_t)n * n * sizeof(double)))
    return fail(SDP_ERR_ARG, "hessian_matvec_static: Hv overlaps v or W (the output is cleared before the "
                             "inputs are read)");
  double* scratch = nullptr;
  unsigned long long* skipped_dev = nullptr;
  cudaError_t e = static_scratch(&scratch, &skipped_dev);
  if (e != cudaSuccess) return fail(SDP_ERR_CUDA, std::string("hessian_matvec_static: ") + cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nn = n * n;
  double* VW = scratch;
  double* T = scratch + (size_t)SMAX * SMAX;
  count_launch(nnzA > 0 ? 4 : 2);
  k_st_clear<<<cdiv_cap(std::max(nn, m), 256, 1024), 256, 0, st>>>(nn, VW, m, Hv_dev, skipped_dev);
  const unsigned gw = cdiv_cap(nnzA, 8, 4096);   // 8 warps (entries) per CTA of 256
  if (nnzA > 0)
    k_st_scatter<<<gw, 256, 0, st>>>(n, m, nnzA, Ak_dev, Ai_dev, Aj_dev, Av_dev, v_dev, W_dev, VW, skipped_dev);
  k_st_transpose<<<dim3(cdiv_cap(n, 32, SMAX), cdiv_cap(n, 32, SMAX)), dim3(32, 8), 0, st>>>(n, VW, T);
  if (nnzA > 0) k_st_gather<<<gw, 256, 0, st>>>(n, m, nnzA, Ak_dev, Ai_dev, Aj_dev, Av_dev, W_dev, T, Hv_dev);
  unsigned long long skipped = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&skipped, skipped_dev, sizeof(skipped), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SDP_ERR_CUDA, std::string("hessian_matvec_static: ") + cudaGetErrorString(e));
  if (skipped)
    return fail(SDP_ERR_ARG, "hessian_matvec_static: " + std::to_string(skipped) +
                                 " triplets had an index out of range and were skipped");
  return SDP_OK;
}
