// Preconditioned conjugate gradients for H y = r (Prop. PCG; Algorithm 1 step 3).
//
// Scalars (r.z, p.q, ||r||^2) live in device memory; the update kernels read
// them directly, so one iteration is: matvec, dot(p, q), fused x/r update with
// the partial sums of ||r||^2, preconditioner apply, dot(r, z), direction update.
// The host reads ||r||^2 once per iteration for the stopping test.
//
// For reduced precision (prec != FP64) the solve is an FP64 iterative
// refinement: the true residual r - H y is recomputed with the FP64 matvec, an
// inner PCG in the reduced precision solves for a correction to a loose
// tolerance, and the correction is added in FP64.
#include "internal.cuh"

#include <algorithm>
#include <cmath>

namespace sdpgb {

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

enum { S_PQ = 0, S_RR = 1, S_RZ0 = 2, S_RZ1 = 3, S_TMP = 4, S_NR0 = 5 };

// x += a p ; r -= a q  with a = rz / pq
__global__ void k_pcg_xr(int m, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                         const double* __restrict__ q, const double* __restrict__ scal, int rz_slot) {
  const double a = scal[rz_slot] / scal[S_PQ];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    r[i] = fma(-a, q[i], r[i]);
  }
}
// p = z + beta p  with beta = rz_new / rz_old
__global__ void k_pcg_p(int m, double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ scal,
                        int rz_new, int rz_old) {
  const double beta = scal[rz_new] / scal[rz_old];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) p[i] = fma(beta, p[i], z[i]);
}

static sdp_status pcg_alloc(sdp_problem* h) {
  if (h->pr) return SDP_OK;
  const int m = h->m;
  SDP_TRY(h->allocT(&h->pr, m));
  SDP_TRY(h->allocT(&h->pz, m));
  SDP_TRY(h->allocT(&h->pp, m));
  SDP_TRY(h->allocT(&h->pq, m));
  SDP_TRY(h->allocT(&h->px, m));
  SDP_TRY(h->allocT(&h->pbest, m));
  SDP_TRY(h->allocT(&h->pcorr, m));
  if (!h->scal) SDP_TRY(h->allocT(&h->scal, 64));
  if (!h->part) SDP_TRY(h->allocT(&h->part, dot_part_doubles()));
  return SDP_OK;
}

static double read_scalar(sdp_problem* h, const double* dev) {
  double v = 0.0;
  cudaMemcpyAsync(&v, dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  return v;
}

// Plain PCG from x = 0 on (r, x) in precision prec.  Returns iterations; *rel = recursive relres.
static sdp_status pcg_core(sdp_problem* h, const double* rhs, double* x, double rtol, int maxit, int prec,
                           int* iters, double* rel) {
  cudaStream_t st = h->stream;
  const int m = h->m;
  const unsigned g = std::min(cdiv(m, 256), 2048u);
  double* scal = h->scal;
  SDP_CK(h, cudaMemcpyAsync(h->pr, rhs, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDP_CK(h, cudaMemsetAsync(x, 0, m * sizeof(double), st));
  dot(st, m, h->pr, h->pr, scal + S_NR0, h->part);
  const double nr0sq = read_scalar(h, scal + S_NR0);
  if (!std::isfinite(nr0sq)) {
    h->last_error = "pcg: non-finite right-hand side";
    return SDP_ERR_NUMERIC;
  }
  if (nr0sq == 0.0) {
    *iters = 0;
    *rel = 0.0;
    return SDP_OK;
  }
  SDP_TRY(precond_apply_impl(h, h->pr, h->pz, prec));
  SDP_CK(h, cudaMemcpyAsync(h->pp, h->pz, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  dot(st, m, h->pr, h->pz, scal + S_RZ0, h->part);
  int cur = S_RZ0;
  double relres = 1.0;
  for (int it = 1; it <= maxit; ++it) {
    SDP_TRY(matvec_impl(h, h->pp, h->pq, prec));
    dot(st, m, h->pp, h->pq, scal + S_PQ, h->part);
    count_launch();
    k_pcg_xr<<<g, 256, 0, st>>>(m, x, h->pr, h->pp, h->pq, scal, cur);
    dot(st, m, h->pr, h->pr, scal + S_RR, h->part);
    const double rr = read_scalar(h, scal + S_RR);
    if (!std::isfinite(rr)) {
      h->last_error = "pcg: non-finite residual";
      *iters = it;
      *rel = relres;
      return SDP_ERR_NUMERIC;
    }
    relres = std::sqrt(rr / nr0sq);
    if (relres <= rtol) {
      *iters = it;
      *rel = relres;
      return SDP_OK;
    }
    SDP_TRY(precond_apply_impl(h, h->pr, h->pz, prec));
    const int nxt = (cur == S_RZ0) ? S_RZ1 : S_RZ0;
    dot(st, m, h->pr, h->pz, scal + nxt, h->part);
    count_launch();
    k_pcg_p<<<g, 256, 0, st>>>(m, h->pp, h->pz, scal, nxt, cur);
    cur = nxt;
  }
  *iters = maxit;
  *rel = relres;
  return SDP_ERR_MAXIT;
}

// relres = ||r - H y|| / ||r|| with the FP64 matvec; leaves r - H y in out
static sdp_status true_residual(sdp_problem* h, const double* r, const double* y, double* out, double* relres) {
  cudaStream_t st = h->stream;
  const int m = h->m;
  SDP_TRY(matvec_impl(h, y, out, SDP_FP64));
  axpby(st, m, 1.0, r, -1.0, out, out);
  dot(st, m, out, out, h->scal + S_TMP, h->part);
  dot(st, m, r, r, h->scal + S_NR0, h->part);
  double v[6];
  SDP_CK(h, cudaMemcpyAsync(v, h->scal, 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaStreamSynchronize(st));
  *relres = (v[S_NR0] > 0.0) ? std::sqrt(v[S_TMP] / v[S_NR0]) : 0.0;
  return SDP_OK;
}

sdp_status pcg_impl(sdp_problem* h, const double* r, double* y, double rtol, int maxit, int prec, int* iters,
                    double* relres) {
  SDP_TRY(pcg_alloc(h));
  if (!h->pc_valid) SDP_TRY(precond_build_impl(h));
  cudaStream_t st = h->stream;
  const int m = h->m;
  // Restarted PCG = iterative refinement on the true FP64 residual.  Each sweep
  // runs PCG from zero on the current residual to a loose tolerance; restarting
  // discards the Krylov recurrences that rounding in the Woodbury apply (about
  // kappa(Ht) eps, Section IV) and in a reduced-precision matvec corrupts, so
  // the true residual keeps falling where one long PCG run stagnates.
  SDP_CK(h, cudaMemsetAsync(y, 0, m * sizeof(double), st));
  double* resid = h->pbest;
  double* corr = h->pcorr;
  SDP_CK(h, cudaMemcpyAsync(resid, r, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double tr = 1.0;
  int total = 0;
  sdp_status result = SDP_ERR_MAXIT;
  const int sweeps = std::max(1, h->prm.refine_maxit);
  const double inner = std::max(h->prm.inner_rtol, rtol);
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    int it = 0;
    double rr = 0.0;
    const int budget = std::max(1, std::min(maxit - total, 300));
    sdp_status s = pcg_core(h, resid, corr, inner, budget, prec, &it, &rr);
    total += it;
    if (s != SDP_OK && s != SDP_ERR_MAXIT) return s;
    if (it > 0) axpby(st, m, 1.0, y, 1.0, corr, y);
    SDP_TRY(true_residual(h, r, y, resid, &tr));
    if (!std::isfinite(tr)) {
      h->last_error = "pcg: non-finite true residual";
      return SDP_ERR_NUMERIC;
    }
    if (tr <= rtol) {
      result = SDP_OK;
      break;
    }
    if (total >= maxit) break;
  }
  if (iters) *iters = total;
  if (relres) *relres = tr;
  return result;
}

}  // namespace sdpgb
