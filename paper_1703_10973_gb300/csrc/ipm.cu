// One iteration of the infeasible NT predictor-corrector around the PCG
// Hessian solve, and sdp_solve.
//
// Per iteration (all FP64 on the device; the host reads a few scalars):
//   residuals   Rp = b - A(X),  Rd = C - S - A^T y,  mu = X.S / n
//   NT scaling  X = L L^T,  L^T S L = Q Lambda Q^T,  Gt = L Q,
//               W = Gt Lambda^{-1/2} Gt^T (so W S W = X),  S^{-1} = Gt Lambda^{-1} Gt^T
//   precond     sdp_precond_build (Algorithm 1 steps 1-2)
//   Newton      H dy = Rp - A(Rc) + A(W Rd W)  (eq. hesseqn2), by PCG;
//               dS = Rd - A^T dy,  dX = Rc - W dS W
//   predictor   Rc = -X;  corrector Rc = sigma mu S^{-1} - X, sigma = (mu_aff / mu)^3
//   step        alpha = min(1, step_frac / max(0, -lambda_min(L^{-1} dX L^{-T}))) per side.
#include "internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <utility>

namespace sdpgb {

enum { R_RP = 8, R_RD, R_CX, R_BY, R_XS, R_XDS, R_DXS, R_DXDS, R_LMIN, R_LZ /* 5 slots */ };

// Step lengths use Lanczos from this order on (below it the full eigensolver is cheap).
constexpr int LZ_MIN_N = 64;

// Probe vectors of the NT-scaling check (declared here: ipm_alloc sizes the
// scratch that holds them).
constexpr int NT_PROBES = 4;

sdp_status ipm_alloc(sdp_problem* h) {
  if (h->L) return SDP_OK;
  const int n = h->n, m = h->m;
  const size_t nn = (size_t)n * n;
  // M1 also holds the check's four n x NT_PROBES products and Gt its probe
  // vectors, which exceed n^2 for n < 16
  const size_t nm1 = std::max(nn, (size_t)4 * NT_PROBES * n), ngt = std::max(nn, (size_t)NT_PROBES * n);
  SDP_TRY(h->allocT(&h->L, nn));
  SDP_TRY(h->allocT(&h->Rs, nn));
  if (!h->M1) SDP_TRY(h->allocT(&h->M1, nm1));
  SDP_TRY(h->allocT(&h->M2, nn));
  SDP_TRY(h->allocT(&h->M3, nn));
  SDP_TRY(h->allocT(&h->Gt, ngt));
  SDP_TRY(h->allocT(&h->Sinv, nn));
  SDP_TRY(h->allocT(&h->Rd, nn));
  SDP_TRY(h->allocT(&h->Rc, nn));
  SDP_TRY(h->allocT(&h->dX, nn));
  SDP_TRY(h->allocT(&h->dS, nn));
  SDP_TRY(h->allocT(&h->E, nn));
  SDP_TRY(h->allocT(&h->lam, n));
  SDP_TRY(h->allocT(&h->Rp, m));
  SDP_TRY(h->allocT(&h->rhs, m));
  SDP_TRY(h->allocT(&h->dy, m));
  if (!h->scal) SDP_TRY(h->allocT(&h->scal, 64));
  if (!h->part) SDP_TRY(h->allocT(&h->part, dot_part_doubles()));
  if (!h->info) SDP_TRY(h->allocT(&h->info, 8));
  const size_t wneed = std::max(potrf_work_doubles(n), trsm_work_doubles(n, n));
  if (wneed > h->work_doubles) {
    SDP_TRY(h->allocT(&h->work, wneed));
    h->work_doubles = wneed;
  }
  if (!h->eig_base) {
    SDP_TRY(h->alloc(&h->eig_base, eig_work_bytes(n, true)));
    eig_work_carve(&h->eig, h->eig_base, n, true);
    eig_work_clear(h->stream, &h->eig);
    h->eig.spin_cycles = h->prm.wait_cycles;
  }
  if (n >= LZ_MIN_N && lanczos_fits(n)) SDP_TRY(h->allocT(&h->lz_work, lanczos_work_doubles(n)));
  return SDP_OK;
}

static sdp_status chol_checked(sdp_problem* h, const double* src, double* L, const char* what) {
  const int n = h->n;
  copy2d(h->stream, n, n, src, n, L, n);
  potrf(h->stream, n, L, n, h->info, h->work);
  int info = 0;
  SDP_CK(h, cudaMemcpyAsync(&info, h->info, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  SDP_CK(h, cudaStreamSynchronize(h->stream));
  if (info) {
    h->last_error = std::string(what) + ": not positive definite (pivot " + std::to_string(info - 1) + ")";
    return SDP_ERR_NOT_PD;
  }
  return SDP_OK;
}

// Explicit inverses of L = chol(X) and Rs = chol(S) with their transposes, for
// the step-length operator L^{-1} D L^{-T}; computed once per pair of factors.
static sdp_status ensure_linv(sdp_problem* h) {
  if (h->linv_valid) return SDP_OK;
  cudaStream_t st = h->stream;
  const int n = h->n;
  const size_t nn = (size_t)n * n;
  if (!h->LinvX) {
    SDP_TRY(h->allocT(&h->LinvX, nn));
    SDP_TRY(h->allocT(&h->LinvXT, nn));
    SDP_TRY(h->allocT(&h->LinvS, nn));
    SDP_TRY(h->allocT(&h->LinvST, nn));
  }
  const double* F[2] = {h->L, h->Rs};
  double* I[2] = {h->LinvX, h->LinvS};
  double* IT[2] = {h->LinvXT, h->LinvST};
  for (int t = 0; t < 2; ++t) {
    fill(st, I[t], nn, 0.0);
    add_diag(st, n, I[t], n, 1.0);
    trsm_left_lower_ex(st, false, n, n, F[t], n, I[t], n, h->work, true);
    transpose(st, n, n, I[t], n, IT[t], n);
  }
  h->linv_valid = true;
  return SDP_OK;
}

// Largest alpha with (Lf Lf^T) + alpha D psd, from lambda_min(Lf^{-1} D Lf^{-T}).
// Lanczos applies that operator as three products with the explicit inverse
// (Linv, D, Linv^T); without the inverse it forms the matrix by two solves.
static sdp_status max_step(sdp_problem* h, const double* Lf, const double* Linv, const double* LinvT,
                           const double* D, double* alpha) {
  cudaStream_t st = h->stream;
  const int n = h->n;
  ktimer_begin(st, "max_step");
  double lmin = 0.0;
  bool have = false;
  const bool implicit = (Linv != nullptr) && h->lz_work;
  if (!implicit) {
    copy2d(st, n, n, D, n, h->M1, n);
    trsm_left_lower(st, false, n, n, Lf, n, h->M1, n, h->work);   // Lf^{-1} D
    transpose(st, n, n, h->M1, n, h->M2, n);                      // D Lf^{-T}
    trsm_left_lower(st, false, n, n, Lf, n, h->M2, n, h->work);   // Lf^{-1} D Lf^{-T}
    symmetrize_avg(st, n, h->M2, n);
  }
  if (h->lz_work) {
    // lambda_min by Lanczos; only whether it lies above -step_frac matters for a full step
    const sdp_status ls = implicit
        ? lanczos_min(st, n, Linv, D, LinvT, n, 1e-3, -h->prm.step_frac, h->lz_work, h->scal + R_LZ)
        : lanczos_min(st, n, h->M2, nullptr, nullptr, n, 1e-3, -h->prm.step_frac, h->lz_work, h->scal + R_LZ);
    if (ls == SDP_OK) {
      double o[5];
      SDP_CK(h, cudaMemcpyAsync(o, h->scal + R_LZ, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
      SDP_CK(h, cudaStreamSynchronize(st));
      if (o[4] != 0.0 && std::isfinite(o[0])) {
        lmin = o[0];
        have = true;
      }
    }
  }
  if (!have && implicit) {
    copy2d(st, n, n, D, n, h->M1, n);
    trsm_left_lower(st, false, n, n, Lf, n, h->M1, n, h->work);
    transpose(st, n, n, h->M1, n, h->M2, n);
    trsm_left_lower(st, false, n, n, Lf, n, h->M2, n, h->work);
    symmetrize_avg(st, n, h->M2, n);
  }
  if (!have) {
    SDP_TRY(eig_min(st, n, h->M2, h->scal + R_LMIN, &h->eig));
    SDP_CK(h, cudaMemcpyAsync(&lmin, h->scal + R_LMIN, sizeof(double), cudaMemcpyDeviceToHost, st));
    SDP_CK(h, cudaStreamSynchronize(st));
    if (eig_flag(st, &h->eig)) {
      h->last_error = "step length: grid barrier timeout";
      return SDP_ERR_TIMEOUT;
    }
  }
  ktimer_end(st, "max_step", 0.0, 0.0);
  if (!std::isfinite(lmin)) {
    h->last_error = "step length: non-finite eigenvalue";
    return SDP_ERR_NUMERIC;
  }
  *alpha = (lmin >= 0.0) ? INFINITY : -1.0 / lmin;
  return SDP_OK;
}

// Newton system (eq. hesseqn2): rhs = rhs0 - A(Rc), then dy from H dy = rhs,
// then dS = Rd - A^T dy and dX = Rc - W dS W.
static void newton_rhs(sdp_problem* h, const double* rhs0) {
  op_A_dense(h, h->Rc, h->rhs, -1.0, rhs0, 1.0);
}
static sdp_status newton_post(sdp_problem* h) {
  cudaStream_t st = h->stream;
  const int n = h->n;
  const size_t nn = (size_t)n * n;
  // dS = Rd - A^T dy
  SDP_CK(h, cudaMemcpyAsync(h->dS, h->Rd, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  assemble_V(h, h->dy, nullptr, h->Vval);
  scatter_V_dense(h, h->Vval, -1.0, h->dS);
  // dX = Rc - W dS W
  gemm(st, false, false, n, n, n, 1.0, h->W, n, h->dS, n, 0.0, h->M1, n);
  gemm(st, false, false, n, n, n, 1.0, h->M1, n, h->W, n, 0.0, h->M2, n, GEMM_LOWER_C);
  axpby(st, nn, 1.0, h->Rc, -1.0, h->M2, h->dX);   // upper triangle replaced next
  symmetrize_lower(st, n, h->dX, n);
  return SDP_OK;
}

// sum_i log A_ii into *out (one CTA, fixed summation order)
__global__ void k_logdiag(int n, const double* __restrict__ A, int lda, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += log(A[(size_t)i * lda + i]);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

// A <- A^{-1} for symmetric positive definite A; *logdet = log det A.  Lb is scratch (n x n).
static sdp_status spd_inverse(sdp_problem* h, double* A, double* Lb, double* logdet) {
  cudaStream_t st = h->stream;
  const int n = h->n;
  copy2d(st, n, n, A, n, Lb, n);
  potrf(st, n, Lb, n, h->info, h->work);
  count_launch();
  k_logdiag<<<1, 256, 0, st>>>(n, Lb, n, h->scal + R_LMIN);
  int info = 0;
  double ld = 0.0;
  SDP_CK(h, cudaMemcpyAsync(&info, h->info, sizeof(int), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaMemcpyAsync(&ld, h->scal + R_LMIN, sizeof(double), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaStreamSynchronize(st));
  if (info) {
    h->last_error = "nt scaling: Denman-Beavers iterate lost positive definiteness";
    return SDP_ERR_NOT_PD;
  }
  *logdet = 2.0 * ld;
  fill(st, A, (size_t)n * n, 0.0);
  add_diag(st, n, A, n, 1.0);
  trsm_left_lower_ex(st, false, n, n, Lb, n, A, n, h->work, true);   // A = L^{-1}
  gemm(st, true, false, n, n, n, 1.0, A, n, A, n, 0.0, Lb, n);        // L^{-T} L^{-1}
  copy2d(st, n, n, Lb, n, A, n);
  symmetrize_avg(st, n, A, n);
  return SDP_OK;
}

// M^{-1/2} by the scaled Denman-Beavers iteration
//   Y0 = M, Z0 = I;  Y+ = (mu Y + Z^{-1}/mu)/2,  Z+ = (mu Z + Y^{-1}/mu)/2,
//   mu = |det(Y) det(Z)|^{-1/(2n)} while the iterates are far from convergence;
// Y -> M^{1/2}, Z -> M^{-1/2}.  Every iterate is a rational function of M, so
// it stays symmetric positive definite and each inverse is a Cholesky inverse.
// Result in Zout; M is overwritten.  Uses the handle's n x n scratch buffers.
static sdp_status db_inv_sqrt(sdp_problem* h, double* M, double* Zout) {
  cudaStream_t st = h->stream;
  const int n = h->n;
  const size_t nn = (size_t)n * n;
  double* Y = M;
  double* Z = Zout;
  double* Yi = h->Gt;
  double* Zi = h->dX;
  double* Lb = h->dS;
  double* Yn = h->M1;
  fill(st, Z, nn, 0.0);
  add_diag(st, n, Z, n, 1.0);
  bool scale = true;
  for (int it = 0; it < 40; ++it) {
    double ly = 0.0, lz = 0.0;
    copy2d(st, n, n, Y, n, Yi, n);
    SDP_TRY(spd_inverse(h, Yi, Lb, &ly));
    copy2d(st, n, n, Z, n, Zi, n);
    SDP_TRY(spd_inverse(h, Zi, Lb, &lz));
    const double mu = scale ? std::exp(-(ly + lz) / (2.0 * n)) : 1.0;
    axpby(st, nn, 0.5 * mu, Y, 0.5 / mu, Zi, Yn);      // Y+
    axpby(st, nn, 0.5 * mu, Z, 0.5 / mu, Yi, Z);        // Z+ (in place)
    symmetrize_avg(st, n, Yn, n);
    symmetrize_avg(st, n, Z, n);
    axpby(st, nn, 1.0, Yn, -1.0, Y, Y);                 // Y <- Y+ - Y (difference)
    dot(st, nn, Y, Y, h->scal + R_XDS, h->part);
    dot(st, nn, Yn, Yn, h->scal + R_DXS, h->part);
    double v[2];
    SDP_CK(h, cudaMemcpyAsync(v, h->scal + R_XDS, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SDP_CK(h, cudaStreamSynchronize(st));
    std::swap(Y, Yn);
    const double rel = std::sqrt(v[0] / v[1]);
    if (!std::isfinite(rel)) {
      h->last_error = "nt scaling: non-finite Denman-Beavers iterate";
      return SDP_ERR_NUMERIC;
    }
    if (rel < 1e-2) scale = false;
    if (rel < 1e-13) break;
  }
  return SDP_OK;
}

// Probe vectors for the NT check: entries from a splitmix64 hash of the index, in [-1, 1].
__global__ void k_probe_fill(int count, double* Z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1) + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  Z[i] = (double)(z >> 11) * 0x1p-52 - 1.0;
}

// W = L Q Lambda^{-1/2} Q^T L^T and S^{-1} = L Q Lambda^{-1} Q^T L^T from
// L^T S L = Q Lambda Q^T.  The eigendecomposition path is checked through the
// defining property W S W = X (on a few probe vectors, four thin products
// instead of two n^3 GEMMs); when inverse iteration could not separate a
// tight eigenvalue cluster the check fails and the inverse square root of
// L^T S L comes from the Denman-Beavers iteration instead.
static sdp_status nt_scaling(sdp_problem* h) {
  cudaStream_t st = h->stream;
  const int n = h->n;
  const size_t nn = (size_t)n * n;
  // L is lower triangular with stored zeros: S L needs k >= j, L^T (S L) needs
  // k >= i, and only the lower triangle of the symmetric results is formed.
  gemm(st, false, false, n, n, n, 1.0, h->S, n, h->L, n, 0.0, h->M1, n, GEMM_B_LOWER);   // S L
  gemm(st, true, false, n, n, n, 1.0, h->L, n, h->M1, n, 0.0, h->M2, n,
       GEMM_A_UPPER | GEMM_LOWER_C);                                                       // M = L^T S L
  symmetrize_lower(st, n, h->M2, n);
  copy2d(st, n, n, h->M2, n, h->M3, n);                                      // keep M
  SDP_TRY(eig_full(st, n, h->M2, h->lam, h->E, &h->eig));
  gemm(st, false, true, n, n, n, 1.0, h->L, n, h->E, n, 0.0, h->Gt, n, GEMM_A_LOWER);   // Gt = L Q, Q = E^T
  scale_cols(st, n, n, h->Gt, n, h->lam, -0.5, h->M1, n);
  gemm(st, false, true, n, n, n, 1.0, h->M1, n, h->Gt, n, 0.0, h->W, n, GEMM_LOWER_C);
  symmetrize_lower(st, n, h->W, n);
  scale_cols(st, n, n, h->Gt, n, h->lam, -1.0, h->M1, n);
  gemm(st, false, true, n, n, n, 1.0, h->M1, n, h->Gt, n, 0.0, h->Sinv, n, GEMM_LOWER_C);
  symmetrize_lower(st, n, h->Sinv, n);
  // check W S W = X on NT_PROBES fixed pseudo-random vectors Z: W (S (W Z)) - X Z
  {
    const int pr = NT_PROBES;
    double* Zp = h->Gt;                       // n x pr
    double* T1 = h->M1;                       // n x pr each
    double* T2 = h->M1 + (size_t)n * pr;
    double* T3 = h->M1 + 2 * (size_t)n * pr;
    double* T4 = h->M1 + 3 * (size_t)n * pr;
    count_launch();
    k_probe_fill<<<(unsigned)((n * pr + 255) / 256), 256, 0, st>>>(n * pr, Zp);
    gemm(st, false, false, n, pr, n, 1.0, h->W, n, Zp, pr, 0.0, T1, pr);
    gemm(st, false, false, n, pr, n, 1.0, h->S, n, T1, pr, 0.0, T2, pr);
    gemm(st, false, false, n, pr, n, 1.0, h->W, n, T2, pr, 0.0, T3, pr);
    gemm(st, false, false, n, pr, n, 1.0, h->X, n, Zp, pr, 0.0, T4, pr);
    axpby(st, (size_t)n * pr, 1.0, T3, -1.0, T4, T3);
    dot(st, (size_t)n * pr, T3, T3, h->scal + R_XDS, h->part);
    dot(st, (size_t)n * pr, T4, T4, h->scal + R_DXS, h->part);
  }
  double v[2], lam0 = 0.0;
  SDP_CK(h, cudaMemcpyAsync(v, h->scal + R_XDS, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaMemcpyAsync(&lam0, h->lam, sizeof(double), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaStreamSynchronize(st));
  if (eig_flag(st, &h->eig)) {
    h->last_error = "ipm_step: grid barrier timeout in the eigensolver";
    return SDP_ERR_TIMEOUT;
  }
  const double rel = std::sqrt(v[0] / v[1]);
  // the check is there to catch eigenvectors that inverse iteration could not
  // separate (errors of order one); near the optimum rounding alone can take
  // the relative error past 1e-9 (kappa eps), and the fallback costs a
  // Denman-Beavers iteration of some twenty Cholesky inverses, so only an
  // error above 1e-6 counts as a failure
  if (std::isfinite(rel) && rel <= 1e-6 && lam0 > 0.0) return SDP_OK;
  // fallback: Z = M^{-1/2};  W = (L Z) L^T;  S^{-1} = (L Z)(L Z)^T
  h->nt_fallbacks++;
  SDP_TRY(db_inv_sqrt(h, h->M3, h->E));
  gemm(st, false, false, n, n, n, 1.0, h->L, n, h->E, n, 0.0, h->M1, n);   // L Z
  gemm(st, false, true, n, n, n, 1.0, h->M1, n, h->L, n, 0.0, h->W, n);
  symmetrize_avg(st, n, h->W, n);
  gemm(st, false, true, n, n, n, 1.0, h->M1, n, h->M1, n, 0.0, h->Sinv, n);
  symmetrize_avg(st, n, h->Sinv, n);
  return SDP_OK;
}

// X <- X + alpha dX (symmetrised) once chol(X + alpha dX) succeeds into Lout;
// alpha shrinks by 0.8 per failure (at most 8 times).
static sdp_status update_checked(sdp_problem* h, double* X, const double* dX, double* alpha, double* Lout,
                                 const char* what) {
  cudaStream_t st = h->stream;
  const int n = h->n;
  const size_t nn = (size_t)n * n;
  for (int t = 0; t < 8; ++t) {
    axpby(st, nn, 1.0, X, *alpha, dX, h->M1);
    symmetrize_avg(st, n, h->M1, n);
    copy2d(st, n, n, h->M1, n, Lout, n);
    potrf(st, n, Lout, n, h->info, h->work);
    int info = 0;
    SDP_CK(h, cudaMemcpyAsync(&info, h->info, sizeof(int), cudaMemcpyDeviceToHost, st));
    SDP_CK(h, cudaStreamSynchronize(st));
    if (info == 0) {
      copy2d(st, n, n, h->M1, n, X, n);
      return SDP_OK;
    }
    *alpha *= 0.8;
  }
  h->last_error = std::string(what) + ": no positive definite iterate along the step";
  return SDP_ERR_NOT_PD;
}

// One IPM iteration in three phases around the two Newton solves, so that a
// batch can solve the Newton systems of many problems together (batch.cu):
//   A: residuals, stopping test, NT scaling, preconditioner, predictor rhs
//   (solve)  B: predictor direction, step lengths, centering, corrector rhs
//   (solve)  C: corrector direction, step lengths, checked update
// Phase A sets *done when the iterate already meets the tolerances.
sdp_status ipm_phase_a(sdp_problem* h, IpmStepState* s, bool* done) {
  SDP_TRY(ipm_alloc(h));
  cudaStream_t st = h->stream;
  const int n = h->n, m = h->m;
  const size_t nn = (size_t)n * n;
  double* sc = h->scal;
  *done = false;
  s->inf = sdp_ipm_info{};
  sdp_ipm_info& inf = s->inf;
  inf.iter = h->iter;

  // ---- residuals and scalars
  op_A_dense(h, h->X, h->Rp, -1.0, h->b, 1.0);
  axpby(st, nn, 1.0, h->C, -1.0, h->S, h->Rd);
  assemble_V(h, h->y, nullptr, h->Vval);
  scatter_V_dense(h, h->Vval, -1.0, h->Rd);
  dot(st, m, h->Rp, h->Rp, sc + R_RP, h->part);
  dot(st, nn, h->Rd, h->Rd, sc + R_RD, h->part);
  dot(st, nn, h->C, h->X, sc + R_CX, h->part);
  dot(st, m, h->b, h->y, sc + R_BY, h->part);
  dot(st, nn, h->X, h->S, sc + R_XS, h->part);
  double v[5];
  SDP_CK(h, cudaMemcpyAsync(v, sc + R_RP, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaStreamSynchronize(st));
  const double cx = v[2], by = v[3], xs = v[4];
  const double mu = xs / n;
  s->mu = mu;
  s->xs = xs;
  inf.mu = mu;
  inf.obj_p = cx;
  inf.obj_d = by;
  inf.relgap = std::fabs(cx - by) / (1.0 + std::fabs(cx) + std::fabs(by));
  inf.pinf = std::sqrt(v[0]) / (1.0 + h->normb);
  inf.dinf = std::sqrt(v[1]) / (1.0 + h->normC);
  if (!std::isfinite(cx) || !std::isfinite(by) || !std::isfinite(xs)) {
    h->last_error = "ipm_step: non-finite iterate";
    return SDP_ERR_NUMERIC;
  }
  if (inf.relgap <= h->prm.gap_tol && inf.pinf <= h->prm.infeas_tol && inf.dinf <= h->prm.infeas_tol) {
    inf.converged = 1;
    *done = true;
    return SDP_OK;
  }

  // ---- NT scaling (L = chol(X) and Rs = chol(S) come from the previous step's check)
  if (!h->chol_valid) {
    h->linv_valid = false;
    SDP_TRY(chol_checked(h, h->X, h->L, "ipm_step: chol(X)"));
    SDP_TRY(chol_checked(h, h->S, h->Rs, "ipm_step: chol(S)"));
    h->chol_valid = true;
  }
  const int fb0 = h->nt_fallbacks;
  ktimer_begin(st, "nt_scaling");
  SDP_TRY(nt_scaling(h));
  ktimer_end(st, "nt_scaling", 0.0, 0.0);
  inf.nt_fallback = h->nt_fallbacks - fb0;
  h->have_W = true;
  h->W32_valid = h->W16_valid = false;
  h->pc_valid = false;

  // ---- preconditioner (Algorithm 1 steps 1-2)
  ktimer_begin(st, "precond_build");
  SDP_TRY(precond_build_impl(h));
  ktimer_end(st, "precond_build", 0.0, 0.0);
  inf.tau = h->tau;
  inf.k_split = h->kpc;

  // ---- common part of the right-hand side: Rp <- Rp + A(W Rd W) (nothing to add
  // once a full dual step has made the iterate dual feasible: Rd = 0 exactly)
  if (v[1] != 0.0) {
    gemm(st, false, false, n, n, n, 1.0, h->W, n, h->Rd, n, 0.0, h->M1, n);
    gemm(st, false, false, n, n, n, 1.0, h->M1, n, h->W, n, 0.0, h->M3, n, GEMM_LOWER_C);
    symmetrize_lower(st, n, h->M3, n);
    op_A_dense(h, h->M3, h->Rp, 1.0, h->Rp, 1.0);   // Rp <- Rp + A(W Rd W)
  }

  // ---- predictor right-hand side
  axpby(st, nn, -1.0, h->X, 0.0, nullptr, h->Rc);
  newton_rhs(h, h->Rp);
  return SDP_OK;
}

sdp_status ipm_phase_b(sdp_problem* h, IpmStepState* s, int its, double rr) {
  cudaStream_t st = h->stream;
  const int n = h->n;
  const size_t nn = (size_t)n * n;
  double* sc = h->scal;
  sdp_ipm_info& inf = s->inf;
  inf.pcg_iters_pred = its;
  inf.pcg_relres_pred = rr;
  SDP_TRY(newton_post(h));
  double ap = 0.0, ad = 0.0;
  if (h->lz_work) SDP_TRY(ensure_linv(h));
  SDP_TRY(max_step(h, h->L, h->LinvX, h->LinvXT, h->dX, &ap));
  SDP_TRY(max_step(h, h->Rs, h->LinvS, h->LinvST, h->dS, &ad));
  ap = std::min(1.0, h->prm.step_frac * ap);
  ad = std::min(1.0, h->prm.step_frac * ad);
  dot(st, nn, h->X, h->dS, sc + R_XDS, h->part);
  dot(st, nn, h->dX, h->S, sc + R_DXS, h->part);
  dot(st, nn, h->dX, h->dS, sc + R_DXDS, h->part);
  double w3[3];
  SDP_CK(h, cudaMemcpyAsync(w3, sc + R_XDS, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaStreamSynchronize(st));
  const double mu_aff = (s->xs + ad * w3[0] + ap * w3[1] + ap * ad * w3[2]) / n;
  const double ratio = std::min(1.0, std::max(0.0, mu_aff / s->mu));
  const double sigma = ratio * ratio * ratio;
  inf.sigma = sigma;
  // ---- corrector right-hand side
  axpby(st, nn, sigma * s->mu, h->Sinv, -1.0, h->X, h->Rc);
  newton_rhs(h, h->Rp);
  return SDP_OK;
}

sdp_status ipm_phase_c(sdp_problem* h, IpmStepState* s, int its, double rr) {
  cudaStream_t st = h->stream;
  const int m = h->m;
  sdp_ipm_info& inf = s->inf;
  inf.pcg_iters_corr = its;
  inf.pcg_relres_corr = rr;
  SDP_TRY(newton_post(h));
  double ap = 0.0, ad = 0.0;
  SDP_TRY(max_step(h, h->L, h->LinvX, h->LinvXT, h->dX, &ap));
  SDP_TRY(max_step(h, h->Rs, h->LinvS, h->LinvST, h->dS, &ad));
  ap = std::min(1.0, h->prm.step_frac * ap);
  ad = std::min(1.0, h->prm.step_frac * ad);

  // ---- update.  The Cholesky factors of the new X and S are the next step's
  // L and Rs; a factorisation that fails (a step length from a Lanczos estimate
  // that came out too long) shortens that side's step.
  h->chol_valid = false;
  h->linv_valid = false;
  SDP_TRY(update_checked(h, h->X, h->dX, &ap, h->L, "ipm_step: primal update"));
  SDP_TRY(update_checked(h, h->S, h->dS, &ad, h->Rs, "ipm_step: dual update"));
  h->chol_valid = true;
  inf.alpha_p = ap;
  inf.alpha_d = ad;
  axpby(st, m, 1.0, h->y, ad, h->dy, h->y);
  SDP_CK(h, cudaGetLastError());
  h->iter++;
  if (h->prm.verbose)
    fprintf(stderr, "ipm %3d mu %.3e gap %.3e pinf %.3e dinf %.3e ap %.3f ad %.3f sig %.3e k %d pcg %d/%d rel %.1e/%.1e\n",
            inf.iter, inf.mu, inf.relgap, inf.pinf, inf.dinf, ap, ad, inf.sigma, inf.k_split, inf.pcg_iters_pred,
            inf.pcg_iters_corr, inf.pcg_relres_pred, inf.pcg_relres_corr);
  return SDP_OK;
}

static sdp_status newton_solve(sdp_problem* h, int* its, double* rr) {
  bool used = false;
  sdp_status s = self_batch_newton(h, its, rr, &used);
  if (used) return s;
  s = pcg_impl(h, h->rhs, h->dy, h->prm.pcg_rtol, h->prm.pcg_maxit, h->prm.prec, its, rr);
  return (s == SDP_OK || s == SDP_ERR_MAXIT) ? SDP_OK : s;
}

sdp_status ipm_step_impl(sdp_problem* h, sdp_ipm_info* info) {
  IpmStepState s;
  bool done = false;
  sdp_status st = ipm_phase_a(h, &s, &done);
  if (st == SDP_OK && !done) {
    int its = 0;
    double rr = 0.0;
    st = newton_solve(h, &its, &rr);
    if (st == SDP_OK) st = ipm_phase_b(h, &s, its, rr);
    if (st == SDP_OK) st = newton_solve(h, &its, &rr);
    if (st == SDP_OK) st = ipm_phase_c(h, &s, its, rr);
  }
  if (info) *info = s.inf;
  return st;
}

}  // namespace sdpgb

extern "C" sdp_status sdp_solve(sdp_problem* h, sdp_result* res) {
  if (!h) return SDP_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  sdp_result r{};
  sdp_status s = SDP_OK;
  int pcg_total = 0;
  for (int it = 0; it <= h->prm.ipm_maxit; ++it) {
    sdp_ipm_info inf{};
    s = sdpgb::ipm_step_impl(h, &inf);
    r.obj_p = inf.obj_p;
    r.obj_d = inf.obj_d;
    r.relgap = inf.relgap;
    r.pinf = inf.pinf;
    r.dinf = inf.dinf;
    if (s != SDP_OK) break;
    if (inf.converged) {
      r.converged = 1;
      break;
    }
    pcg_total += inf.pcg_iters_pred + inf.pcg_iters_corr;
  }
  r.iters = h->iter;
  r.pcg_iters_total = pcg_total;
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (res) *res = r;
  if (s == SDP_OK && !r.converged) return SDP_ERR_MAXIT;
  return s;
}
