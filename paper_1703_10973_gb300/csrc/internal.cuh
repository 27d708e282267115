// Internal declarations shared by the translation units of libsdpgb.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/sdpgb.h"

namespace sdpgb {
// Deterministic grid-wide sum in one kernel: every block stores its partial in
// part[blockIdx.x]; the last block to arrive (atomic ticket) adds the partials
// in index order and, in its thread 0, returns true with the total in *total
// (then re-arms the ticket).  Every thread of every block must call it.
__device__ inline double lb_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double lb_block_sum(double v, double* sh) {
  v = lb_warp_sum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < (int)(blockDim.x / 32)) ? sh[l] : 0.0;
    s = lb_warp_sum(s);
  }
  return s;  // valid in thread 0
}
// Block b of a group of nb blocks (a whole grid, or one problem's share of a
// batched grid) stores its partial in part[b]; the last block of the group to
// arrive (atomic ticket) adds the partials in index order and, in its thread 0,
// returns true with the total in *total (then re-arms the ticket).
__device__ inline bool lb_reduce(double v, double* part, unsigned int* ticket, double* total, int b, int nb) {
  __shared__ double sh[32];
  __shared__ int s_last;
  const double s0 = lb_block_sum(v, sh);
  if (threadIdx.x == 0) {
    part[b] = s0;
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == (unsigned)nb - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += __ldcg(part + i);
  s = lb_block_sum(s, sh);
  if (threadIdx.x == 0) {
    *total = s;
    *ticket = 0u;
  }
  return threadIdx.x == 0;
}

// Scalar slots of a PCG run (device array scal[])
enum { S_PQ = 0, S_RR = 1, S_RZ = 2, S_RZN = 3, S_TMP = 4, S_NR0 = 5, S_TOL2 = 6, S_IT = 7, S_MAXIT = 8,
       S_BRK = 9, S_GO = 10, S_RRB = 11, S_NEWB = 12 };

// One problem of a batched PCG launch (FP64 or FP32 split matvec, Hhat preconditioner): the
// device pointers and sizes the batched kernels read, refreshed by the host
// before every batched solve.
struct BDesc {
  int n, m, k, np, nr, Rk, nnzV;
  int active;                       // the problem's PCG loop is still running
  double zscale, inv_tau2;
  const int *rowptr, *rowperm, *colidx, *sptr, *scon, *eptr, *ep, *eq;
  const double *scoef, *ecoef, *ginv;
  const double *W, *U;
  double *T, *Vval;
  const int *pverts, *rverts, *btptr, *btslot, *bp, *bptr, *bcol;
  const double *D, *F, *Cinv, *CinvT;
  double *yP, *v1, *v2, *uvec, *Bn;
  int lpc;                          // the core solve uses the FP32 copy of the Schur-factor inverse
  const float *Cinv32, *CinvT32;
  float *v1f, *v2f;
  double *px, *pr, *pp, *pq, *pz, *pxb;
  double *scal, *part;
  unsigned int* ticket;
  // FP32 split matvec (a problem in a reduced-precision sweep)
  int lp, ks;                       // lp: this sweep runs the FP32 matvec; ks: split rank (0: none)
  int bf;                           // the reduced-precision W_s copy is bfloat16 (W16), else float (W32)
  const __nv_bfloat16* W16;
  const float* W32;
  float *T32, *mvR, *mvPart;
  const double *Etop, *wtop;
  double *mvG, *mvQ;
};

// Finds the problem that owns block b of a batched grid: off[0..N] are the
// first blocks of each problem (off[N] = total).
__device__ inline int batch_find(const int* off, int N, int b) {
  int lo = 0, hi = N;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}
}  // namespace sdpgb

namespace sdpgb {
const char* free_call_error();   // error text of the last handle-free call on this thread

// ---------------------------------------------------------------------------
// Error plumbing: every CUDA call inside the library goes through CK(), which
// records the failing call on the handle and returns SDP_ERR_CUDA.
// ---------------------------------------------------------------------------
struct Err {
  sdp_status st = SDP_OK;
  std::string msg;
};

#define SDP_CK(h, call)                                                          \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      (h)->set_error(SDP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
      return SDP_ERR_CUDA;                                                       \
    }                                                                            \
  } while (0)

#define SDP_CK_ST(call)                                                          \
  do {                                                                           \
    if ((call) != cudaSuccess) return SDP_ERR_CUDA;                              \
  } while (0)

#define SDP_TRY(expr)                                                            \
  do {                                                                           \
    sdp_status s_ = (expr);                                                      \
    if (s_ != SDP_OK) return s_;                                                 \
  } while (0)

// Launch accounting: every kernel launch in the library increments this counter
// (per process); sdp_launch_count() reports it per handle via a snapshot.
extern std::atomic<int64_t> g_launches;
extern thread_local int64_t t_launches;   // this host thread's launches (graph capture accounting)
inline void count_launch(int k = 1) {
  g_launches.fetch_add(k, std::memory_order_relaxed);
  t_launches += k;
}

// Optional event timing of one kernel class (sdp_timing_enable / sdp_timing_read).
// ktimer_begin/ktimer_end bracket a launch; they do nothing unless `cls` is the
// class currently enabled.
bool ktimer_on(const char* cls);
void ktimer_begin(cudaStream_t st, const char* cls);
void ktimer_end(cudaStream_t st, const char* cls, double flops, double bytes);
void ktimer_set(const char* cls);
void ktimer_read(double* ms, int64_t* launches, double* flops, double* bytes);
void ktimer_pause(bool paused);   // no recording while a graph is being captured
size_t ktimer_report(char* buf, size_t len);

// Raise a kernel's dynamic shared-memory limit to the per-CTA maximum, once per
// kernel and process (thread-safe).  Setting the limit per launch to the size
// that launch needs races between host threads driving different problems: a
// smaller value written by one thread can land after a larger one, and the
// larger launch then fails.
void allow_max_smem(const void* func);

// Device buffer owned by a handle.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// ---------------------------------------------------------------------------
// Dense FP64 linear algebra (dense.cu).  Row-major storage; ld = row stride.
// ---------------------------------------------------------------------------
// C[M x N] = alpha * op(A) * op(B) + beta * C.  op(A) is M x K.
// flags: GEMM_LOWER_C skips tiles strictly above the diagonal of C (a symmetric
// product; symmetrize_lower completes it).  GEMM_A_LOWER / GEMM_A_UPPER /
// GEMM_B_LOWER / GEMM_B_UPPER declare op(A) or op(B) triangular with its other
// triangle STORED as zeros, and restrict each tile's k range to the band that
// can be nonzero.  Batched over `batch` with element strides sA, sB, sC.
enum GemmFlags : int {
  GEMM_LOWER_C = 1, GEMM_A_LOWER = 2, GEMM_A_UPPER = 4, GEMM_B_LOWER = 8, GEMM_B_UPPER = 16
};
void gemm(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha,
          const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
          int flags = 0, int batch = 1, long long sA = 0, long long sB = 0, long long sC = 0);
double gemm_useful_fma(int M, int N, int K, int flags, int tile);
void gemm_f32(cudaStream_t st, bool tA, bool tB, int M, int N, int K, float alpha,
              const float* A, int lda, const float* B, int ldb, float beta, float* C, int ldc);

// In-place lower Cholesky A = L L^T of an n x n matrix (strict upper part set to 0).
// info_dev receives 0 on success or (index + 1) of the first non-positive pivot.
// work: at least potrf_work_doubles(n) doubles.
size_t potrf_work_doubles(int n);
void potrf(cudaStream_t st, int n, double* A, int lda, int* info_dev, double* work);
// info_dev needs 2 ints; info_dev[1] counts pivots raised to floor.
void potrf_floor(cudaStream_t st, int n, double* A, int lda, int* info_dev, double* work, double floor_);

// Triangular solves with a lower-triangular L (n x n), in place on B (n x nrhs):
// trans == false: B <- L^{-1} B;  trans == true: B <- L^{-T} B.
size_t trsm_work_doubles(int n, int nrhs);
void trsm_left_lower(cudaStream_t st, bool trans, int n, int nrhs, const double* L, int ldl,
                     double* B, int ldb, double* work);
void trsm_left_lower_ex(cudaStream_t st, bool trans, int n, int nrhs, const double* L, int ldl,
                        double* B, int ldb, double* work, bool lower_rhs);

// Elementwise helpers.
void fill(cudaStream_t st, double* x, size_t count, double v);
void copy2d(cudaStream_t st, int rows, int cols, const double* src, int lds, double* dst, int ldd);
void transpose(cudaStream_t st, int rows, int cols, const double* src, int lds, double* dst, int ldd);
void symmetrize_lower(cudaStream_t st, int n, double* A, int lda);     // A_ij (i<j) = A_ji
void symmetrize_avg(cudaStream_t st, int n, double* A, int lda);       // A = (A + A^T)/2
void add_diag(cudaStream_t st, int n, double* A, int lda, double v);
void scale_cols(cudaStream_t st, int rows, int cols, const double* A, int lda, const double* s,
                double pw, double* B, int ldb);                        // B = A diag(s^pw)
void zero_upper(cudaStream_t st, int n, double* A, int lda);
void axpby(cudaStream_t st, size_t count, double a, const double* x, double b, const double* y,
           double* z);                                                 // z = a x + b y
void to_f32(cudaStream_t st, size_t count, const double* x, float* y);
void to_bf16(cudaStream_t st, size_t count, const double* x, __nv_bfloat16* y);

// Deterministic reductions into device memory (two stages, fixed order).
// out[0] = sum_i x_i y_i.
void dot(cudaStream_t st, size_t count, const double* x, const double* y, double* out, double* part);
void dot_partials(cudaStream_t st, size_t count, const double* x, const double* y, double* part);
size_t dot_part_doubles();

// Lower-triangular GEMV y = L x and y = L^T x (L n x n row-major).  part: n * TRMV_CHUNKS doubles.
void trmv_lower(cudaStream_t st, bool trans, int n, const double* L, int ldl, const double* x,
                double* y, double* part);
size_t trmv_part_doubles(int n);
// y = alpha op(L) x + beta z   (z may be NULL)
void trmv_lower_ex(cudaStream_t st, bool trans, int n, const double* L, int ldl, const double* x, double* y,
                   double* part, double alpha, const double* z, double beta);

// ---------------------------------------------------------------------------
// Symmetric eigensolver (eig.cu).  A is n x n row-major symmetric and is
// overwritten (it receives the Householder vectors of the tridiagonalisation).
// ---------------------------------------------------------------------------
struct EigWork {
  double* d = nullptr;      // n   diagonal of T
  double* e = nullptr;      // n   off-diagonal of T
  double* tauh = nullptr;   // n   Householder scalars
  double* p = nullptr;      // n   symv result
  double* part = nullptr;   // 4096 block partials
  unsigned int* bar = nullptr;  // 2 barrier words
  int* flag = nullptr;      // 1 error flag (barrier timeout)
  double* ws = nullptr;     // inverse-iteration workspace: 6 * n * batch doubles
  int batch = 0;
  double* G = nullptr;      // n x n Gram matrix for the re-orthogonalisation
  double* aux = nullptr;    // trsm / potrf work
  int* info = nullptr;      // potrf info
  double* wsel = nullptr;   // selected eigenvalues
  double* es = nullptr;     // n   off-diagonal with split positions zeroed
  double* val = nullptr;    // n   per-block eigenvalues before sorting
  int* blocks = nullptr;    // 3n+4  block of each row, block starts, block ends, count
  int* src = nullptr;       // n   row that owns each sorted eigenvalue
  long long spin_cycles = 0;   // bound of a grid-barrier wait (0: the default)
};
size_t eig_work_bytes(int n, bool full);
void eig_work_carve(EigWork* w, void* base, int n, bool full);

// Full eigendecomposition: w ascending, E row t = unit eigenvector of w[t].
sdp_status eig_full(cudaStream_t st, int n, double* A, double* w, double* E, EigWork* ws);
// Smallest eigenvalue only (result in *lmin_dev, device).
sdp_status eig_min(cudaStream_t st, int n, double* A, double* lmin_dev, EigWork* ws);
// lanczos.cu: lambda_min of a dense symmetric matrix (one thread-block cluster);
// out_dev[0..4] = estimate, Ritz value, residual bound, steps, converged flag
size_t lanczos_work_doubles(int n);
// schur.cu: sparse factorisation of the Hhat core
struct SchurPlanHost {
  std::vector<int> pverts, rverts, stype, sa, sb, bptr, bcol, bp, btptr, btslot;
  bool bipartite = false;
};
void schur_plan(int n, const std::vector<int>& krowptr, const std::vector<int>& kcol, SchurPlanHost* out);
sdp_status schur_build(sdp_problem* h, int k, double tau);
sdp_status schur_apply(sdp_problem* h, const double* u, double* out, double scale, int prec = SDP_FP64);
// FP32 copy of the Hhat core's dense factor inverse for applies in reduced precision
sdp_status ensure_lowprec_core(sdp_problem* h);
// tc_gemm.cu: C (FP64) = op(A) op(B) on the tensor cores with the operands
// rounded to BF16 (prec SDP_BF16) or TF32 (SDP_FP32), FP32 accumulation
bool tc_available();
size_t tc_work_bytes(int M, int N, int K);
sdp_status tc_gemm(cudaStream_t st, int prec, int M, int N, int K, const double* A, int lda, bool transA,
                   const double* B, int ldb, bool transB, double* C, int ldc, void* work, int* err_dev);
bool lanczos_fits(int n);
sdp_status lanczos_min(cudaStream_t st, int n, const double* M, const double* A2, const double* A3, int ldm,
                       double rtol, double accept_above, double* work, double* out_dev);
// Smallest eigenvalue and the top-k eigenpairs (k <= SDP_K_MAX + 1): wtop[0..k) ascending
// (= lambda_{n-k..n-1}), Etop rows = eigenvectors; *lmin_dev = lambda_0.
sdp_status eig_extremes(cudaStream_t st, int n, double* A, int k, double* lmin_dev, double* wtop,
                        double* Etop, EigWork* ws);
// Reads the barrier-timeout flag; nonzero -> SDP_ERR_TIMEOUT.
void eig_work_clear(cudaStream_t st, EigWork* w);
int eig_flag(cudaStream_t st, EigWork* ws);

}  // namespace sdpgb

// ---------------------------------------------------------------------------
// The handle.
// ---------------------------------------------------------------------------
struct sdp_problem {
  int n = 0, m = 0, k = 0;
  int kcap = 0;            // largest split rank a build can use (k, or k_max with the adaptive rule)
  int kest = -1;           // split rank chosen by the last build's adaptive rule (-1: fixed k)
  sdp_params prm{};
  cudaStream_t stream = nullptr;
  std::string last_error;
  int64_t launches_at_setup = 0;

  // ---- sparse constraint operator (device) ----
  int nnzV = 0;            // CSR pattern of V = sum v_i A_i (both triangles)
  int* rowptr = nullptr;   // n+1
  int* rowperm = nullptr;  // n   rows by decreasing length (SpMM thread -> row)
  int* colidx = nullptr;   // nnzV
  int* sptr = nullptr;     // nnzV+1  slot -> contributors
  int* scon = nullptr;     // contributors: constraint
  double* scoef = nullptr; // contributors: coefficient
  int ncontrib = 0;
  int nent = 0;            // stored upper entries over all constraints
  int* eptr = nullptr;     // m+1   constraint -> entries
  int* ep = nullptr;       // entry row (p <= q)
  int* eq = nullptr;       // entry col
  double* ecoef = nullptr; // entry value
  double* ginv = nullptr;  // m   1/||A_i||_F^2
  // K-pattern for the core formation (pairs of support rows of each constraint)
  int ncr = 0;             // constraint-row slots
  int* crptr = nullptr;    // m+1   constraint -> support rows
  int* crrow = nullptr;    // ncr   support row index
  int* crlist_ptr = nullptr;  // ncr+1  (constraint,row) -> entries (col, coef) of A_i in that row
  int* crlist_col = nullptr;
  double* crlist_coef = nullptr;
  int nnzK = 0;
  int* krowptr = nullptr;  // n+1
  int* kcol = nullptr;     // nnzK
  int* kptr = nullptr;     // nnzK+1  K slot -> contributor triples
  int* kcon = nullptr;     // constraint
  int* kcra = nullptr;     // cr slot of row a
  int* kcrb = nullptr;     // cr slot of row b
  int nkc = 0;

  // ---- data (device) ----
  double* C = nullptr;     // n*n dense
  double* b = nullptr;     // m
  double normb = 0, normC = 0;

  // ---- IPM state (device) ----
  double *X = nullptr, *y = nullptr, *S = nullptr, *W = nullptr;
  int iter = 0;
  int nt_fallbacks = 0;     // NT scalings computed by the Denman-Beavers fallback
  int pcg_prec_fallbacks = 0;  // restarted PCG sweeps that fell back from reduced precision to FP64
  bool have_W = false;
  double xi = 0;

  // ---- matvec work ----
  double* Vval = nullptr;  // nnzV
  double* T = nullptr;     // n*n
  float* W32 = nullptr;    // n*n (reduced-precision copies, lazily allocated)
  float* T32 = nullptr;
  __nv_bfloat16* W16 = nullptr;
  bool W32_valid = false, W16_valid = false;
  int64_t W32_key = -1, W16_key = -1;   // preconditioner generation of a split copy (-1: plain W)
  double* mv_G = nullptr;  // split matvec: (E V)^T, n x k
  float* mv_R = nullptr;   // Lambda (E V) W_s, k x n
  double* mv_Q = nullptr;  // Lambda (E V E^T) Lambda, k x k
  float* mv_part = nullptr;

  // ---- preconditioner ----
  bool pc_valid = false;
  double tau = 0;
  double core_shift = 0;   // diagonal added to the core (tau^2)
  int core_floor_pivots = 0;  // pivots raised to tau^2 in the last core Cholesky
  int kpc = 0;             // split rank used
  bool pc_hat = false;     // built as Hhat (Z = sqrt(2 tau) I, eq. sparse_prec)
  double zscale = 0;       // sqrt(2 tau)
  double* U = nullptr;     // n*k
  double* Z = nullptr;     // n*n
  double* Sc = nullptr;    // nk*nk core, then its Cholesky factor
  double* Linv = nullptr;  // nk*nk inverse of the factor
  double* tau_dev = nullptr;  // device scalars: [0] tau, [1] lmin scratch
  double* wtop = nullptr;  // k
  double* Etop = nullptr;  // k*n
  double* au = nullptr;    // ncr*k   (A_i u_l) restricted to support rows
  double* Kval = nullptr;  // nnzK
  double* KZ = nullptr;    // n*n
  void* tc_work = nullptr; // packed tensor-core operands of the mixed core formation
  double* pvec = nullptr;  // scratch vectors for the apply
  double* Bn = nullptr;    // n*k
  double* uvec = nullptr;  // nk
  double* uvec2 = nullptr; // nk
  double* uvec3 = nullptr; // nk
  int core_refine = 1;     // refinement steps of each core triangular solve
  // sparse Hhat core (schur.cu): independent set P of the K graph, rest R
  int hs_np = 0, hs_nr = 0, hs_nb = 0, hs_k = 0;
  int *hs_pverts = nullptr, *hs_rverts = nullptr;        // np, nr
  int *hs_stype = nullptr, *hs_sa = nullptr, *hs_sb = nullptr;   // per K slot
  int *hs_bptr = nullptr, *hs_bcol = nullptr, *hs_bp = nullptr;  // B blocks by row of P
  int *hs_btptr = nullptr, *hs_btslot = nullptr;         // B blocks by row of R
  double *hs_D = nullptr, *hs_F = nullptr, *hs_yP = nullptr;     // L_P, F = L_P^{-1} B, y_P
  double *hs_C = nullptr, *hs_Cinv = nullptr, *hs_CinvT = nullptr;   // Schur factor, inverse, its transpose
  double *hs_v1 = nullptr, *hs_v2 = nullptr, *hs_v3 = nullptr;
  // FP32 copy of the Schur-factor inverse and its transpose for reduced-precision
  // applies, refreshed once per preconditioner build (key hs_lp_gen)
  float *hs_Cinv32 = nullptr, *hs_CinvT32 = nullptr, *hs_v1f = nullptr, *hs_v2f = nullptr;
  int64_t hs_lp_gen = -1;
  size_t hs_lp_cap = 0;    // Rk the float copies were allocated for
  size_t hs_cap = 0;       // Rk the Schur buffers were allocated for (they grow, never shrink)
  int hs_kcap = 0;         // split rank they were allocated for
  double* trpart = nullptr;

  // ---- dense IPM work ----
  double *L = nullptr, *Rs = nullptr, *M1 = nullptr, *M2 = nullptr, *M3 = nullptr;
  bool chol_valid = false;   // L = chol(X) and Rs = chol(S) belong to the current X, S
  double* lz_work = nullptr; // Lanczos basis scratch (step length)
  // explicit inverses of the Cholesky factors (and their transposes) of X and S
  double *LinvX = nullptr, *LinvXT = nullptr, *LinvS = nullptr, *LinvST = nullptr;
  bool linv_valid = false;
  double *Gt = nullptr, *Sinv = nullptr, *Rd = nullptr, *Rc = nullptr, *dX = nullptr,
         *dS = nullptr, *E = nullptr, *lam = nullptr;
  double *Rp = nullptr, *rhs = nullptr, *dy = nullptr;
  double* work = nullptr;  // trsm / potrf work
  size_t work_doubles = 0;
  int* info = nullptr;
  double* scal = nullptr;  // device scalar scratch (64)
  double* part = nullptr;  // reduction partials
  sdpgb::EigWork eig;
  void* eig_base = nullptr;

  // ---- PCG as a device-side graph loop ----
  int64_t pc_generation = 0;            // bumped by every preconditioner build
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t pcg_graph = nullptr;
  cudaGraphExec_t pcg_exec = nullptr;
  int64_t pcg_key = -1;
  int64_t pcg_body_launches = 0;
  sdp_batch* self_batch = nullptr;   // one-problem batch driving this handle's Newton solves

  // ---- PCG vectors ----
  double *pr = nullptr, *pz = nullptr, *pp = nullptr, *pq = nullptr, *px = nullptr,
         *pbest = nullptr, *pcorr = nullptr, *pxb = nullptr;
  double* pcg_part = nullptr;          // per-block partials of the fused PCG reductions
  unsigned int* pcg_ticket = nullptr;  // their arrival tickets (one per reduction)

  std::vector<void*> owned;   // every cudaMalloc made for this handle
  std::vector<size_t> owned_bytes;
  int64_t device_bytes = 0;   // their total size

  void set_error(sdp_status s, const std::string& msg) {
    (void)s;
    last_error = msg;
  }
  sdp_status alloc(void** p, size_t bytes);
  void release(void* p);      // frees one allocation made by alloc (no-op for nullptr)
  template <typename T>
  sdp_status allocT(T** p, size_t count) {
    return alloc(reinterpret_cast<void**>(p), count * sizeof(T));
  }
};

namespace sdpgb {
// setup.cu: device memory of problems and batches, from one stream-ordered
// pool per device that keeps what is freed.  pool_malloc returns memory that
// every stream may use (it waits for the allocation on st); pool_free orders
// the free on st, so the caller must have finished every use on other streams.
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st);
void pool_free(void* p, cudaStream_t st);
// matvec.cu
// Optional epilogue (PCG): *dot_out = v . Hv, after *pro_dst = *pro_src.
sdp_status matvec_impl(sdp_problem* h, const double* v, double* Hv, int prec, double* dot_out = nullptr,
                       double* pro_dst = nullptr, const double* pro_src = nullptr);
sdp_status ensure_lowprec_W(sdp_problem* h, int prec);
// sparse helpers used by the IPM and the preconditioner (matvec.cu)
void assemble_V(sdp_problem* h, const double* v, const double* scale, double* Vval);
void op_A_dense(sdp_problem* h, const double* X, double* out, double alpha, const double* add,
                double beta);   // out = alpha * A(X) + beta * add
void scatter_V_dense(sdp_problem* h, const double* Vval, double alpha, double* D);  // D += alpha*V
void spmm_rows(sdp_problem* h, const double* Vval, const double* B, int ldb, int ncols, double* out,
               int ldo);   // out[a, :ncols] = sum_{s in row a} Vval[s] B[col(s), :ncols]
// precond.cu
sdp_status precond_build_impl(sdp_problem* h);
// Optional epilogue (PCG): *dot_out = r . z.
sdp_status precond_apply_impl(sdp_problem* h, const double* r, double* z, int prec, double* dot_out = nullptr);
// pcg.cu
sdp_status pcg_impl(sdp_problem* h, const double* r, double* y, double rtol, int maxit, int prec,
                    int* iters, double* relres);
// ipm.cu
sdp_status ipm_alloc(sdp_problem* h);
// Batched PCG pieces (one launch for all problems of a batch; block offsets per problem)
int batch_blocks_assemble(int nnzV);
int batch_blocks_spmm(int n, int R);
void batch_launch_spmm(cudaStream_t st, int R, const BDesc* desc, const int* off, int N, int nb, int nmax);
bool batch_spmm_fits(int R, int nmax);
int batch_blocks_sddmm(int m);
int batch_blocks_vec(int m);
int batch_blocks_hat_u(int n);
int batch_blocks_tail(int m);
int batch_blocks_fwdP(int np);
int batch_blocks_warp_rows(int rows);
int batch_blocks_outR(int Rk);
int batch_blocks_out_bwd(int Rk, int np);
int batch_blocks_split_G(int n);
int batch_blocks_split_R(int n);
int batch_blocks_split_Q(int n, int k);
int batch_blocks_spmm_lp(int n, int nmax);   // rows per CTA chosen from the batch's largest order
void batch_launch_matvec_lp(cudaStream_t st, const BDesc* desc, const int* off_g, const int* off_r,
                            const int* off_q, const int* off_spmm, const int* off_sddmm, int N, int nb_g, int nb_r,
                            int nb_q, int nb_spmm, int nb_sddmm, int nmax, bool with_sddmm = true);
void batch_launch_matvec(cudaStream_t st, const BDesc* desc, const int* off_asm, const int* off_spmm,
                         const int* off_sddmm, int N, int nb_asm, int nb_spmm, int nb_sddmm, int nmax, int spmm_r);
// the reduced-precision matvec pieces; with_sddmm = false leaves the gather to batch_launch_sddmm_mixed
void batch_launch_xr(cudaStream_t st, BDesc* desc, const int* off, int N, int nb);
// direction update; also sets the loop condition (graph) or the host-loop flags
void batch_launch_p(cudaStream_t st, const BDesc* desc, const int* off, int N, int nb,
                    cudaGraphConditionalHandle cond, int* flag);
// the FP64 and reduced-precision gathers of a mixed batch in one launch
void batch_launch_sddmm_mixed(cudaStream_t st, const BDesc* desc, const int* off, int N, int nb);
void batch_launch_hat_u(cudaStream_t st, const BDesc* desc, const int* off, int N, int nb);
void batch_launch_tail(cudaStream_t st, const BDesc* desc, const int* off, int N, int nb);
void batch_launch_core_solve(cudaStream_t st, const BDesc* desc, int N, const int* off_fwdP, int nb_fwdP,
                             const int* off_fwdR, int nb_fwdR, const int* off_gemv, int nb_gemv,
                             const int* off_outR, int nb_outR, const int* off_bwdP, int nb_bwdP);
// Restarted PCG as a state machine (pcg.cu), shared by single solves and batches
struct PcgSweeps {
  const double* r = nullptr;
  double* y = nullptr;
  double rtol = 0, inner_fp64 = 0, inner_lp = 0, tr = 1, nr0sq = 0;
  int maxit = 0, prec = 0, sweeps = 1, sweep = 0, total = 0, budget = 0;
  bool finished = false, graph = false;
  sdp_status result = SDP_ERR_MAXIT;
};
sdp_status pcg_sweeps_init(sdp_problem* h, PcgSweeps* S, const double* r, double* y, double rtol, int maxit,
                           int prec);
sdp_status pcg_sweep_begin(sdp_problem* h, PcgSweeps* S, bool graph, bool* run);
sdp_status pcg_sweep_end(sdp_problem* h, PcgSweeps* S);
// One IPM iteration split around its two Newton solves (H dy = h->rhs into h->dy)
struct IpmStepState {
  sdp_ipm_info inf{};
  double mu = 0, xs = 0;
};
sdp_status ipm_phase_a(sdp_problem* h, IpmStepState* s, bool* done);
sdp_status ipm_phase_b(sdp_problem* h, IpmStepState* s, int pcg_its, double pcg_rr);
sdp_status ipm_phase_c(sdp_problem* h, IpmStepState* s, int pcg_its, double pcg_rr);
sdp_status ipm_step_impl(sdp_problem* h, sdp_ipm_info* info);
// The Newton system H dy = h->rhs of one problem through its one-problem batch
// (batch.cu): the batched PCG graph is captured once per handle, where the
// single-problem graph is captured again for every new preconditioner.
// *used = false (nothing done) when the configuration is not batchable or the
// PCG loop is host-driven (pcg_graph = 0).
sdp_status self_batch_newton(sdp_problem* h, int* its, double* rr, bool* used);
}  // namespace sdpgb
