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

enum { S_PQ = 0, S_RR = 1, S_RZ = 2, S_RZN = 3, S_TMP = 4, S_NR0 = 5, S_TOL2 = 6, S_IT = 7, S_MAXIT = 8, S_BRK = 9, S_GO = 10 };

// A breakdown (p.q or r.z not positive and finite: rounding has made the
// preconditioned operator indefinite in some direction) leaves x and r at the
// last good iterate, sets scal[S_BRK] and ends the loop; the restarted outer
// solve then continues from the true residual.

// p = z + beta p  with beta = rz_new / rz
__global__ void k_pcg_p(int m, double* __restrict__ p, const double* __restrict__ z, double* scal) {
  const double rzn = scal[S_RZN], rz = scal[S_RZ];
  if (!(rzn > 0.0 && isfinite(rzn) && rz > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[S_BRK] = 1.0;
    return;
  }
  const double beta = rzn / rz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) p[i] = fma(beta, p[i], z[i]);
}

// x += a p;  r -= a q  (a = rz / pq), ||r||^2, iteration count and the loop
// condition, in one kernel (the last block to finish reduces and decides).
__global__ void k_pcg_xr_check(int m, double* __restrict__ x, double* __restrict__ r,
                               const double* __restrict__ p, const double* __restrict__ q, double* scal,
                               double* part, unsigned int* ticket, cudaGraphConditionalHandle cond, int use_cond) {
  const double pq = scal[S_PQ], rz = scal[S_RZ];
  const bool ok = pq > 0.0 && rz > 0.0 && isfinite(pq) && isfinite(rz);
  const double a = ok ? rz / pq : 0.0;
  double rr = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double ri = r[i];
    if (ok) {
      x[i] = fma(a, p[i], x[i]);
      ri = fma(-a, q[i], ri);
      r[i] = ri;
    }
    rr = fma(ri, ri, rr);
  }
  double tot;
  if (lb_reduce(rr, part, ticket, &tot)) {
    scal[S_RR] = tot;
    const double it = scal[S_IT] + 1.0;
    scal[S_IT] = it;
    if (!ok) scal[S_BRK] = 1.0;
    const bool go = ok && (tot > scal[S_TOL2]) && (it < scal[S_MAXIT]) && isfinite(tot) && scal[S_BRK] == 0.0;
    scal[S_GO] = go ? 1.0 : 0.0;
    if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
}

__global__ void k_pcg_init(double* scal, double rtol, int maxit) {
  scal[S_RZN] = scal[S_RZ];
  scal[S_TOL2] = rtol * rtol * scal[S_NR0];
  scal[S_IT] = 0.0;
  scal[S_MAXIT] = (double)maxit;
  scal[S_BRK] = 0.0;
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
  SDP_TRY(h->allocT(&h->pcg_part, (size_t)m / 8 + 4096));
  SDP_TRY(h->allocT(&h->pcg_ticket, 4));
  SDP_CK(h, cudaMemsetAsync(h->pcg_ticket, 0, 4 * sizeof(unsigned int), h->stream));
  if (!h->scal) SDP_TRY(h->allocT(&h->scal, 64));
  if (!h->part) SDP_TRY(h->allocT(&h->part, dot_part_doubles()));
  return SDP_OK;
}


// One PCG iteration on h->stream (the body of the device-side loop): four
// launches plus those of the two operators, whose last kernels also form the
// two inner products (p . Hp with the move rz <- rz_new, and r . z).
static sdp_status pcg_body(sdp_problem* h, int prec, cudaGraphConditionalHandle cond, bool use_cond) {
  cudaStream_t st = h->stream;
  const int m = h->m;
  const unsigned g = std::min(cdiv(m, 256), 2048u);
  double* scal = h->scal;
  SDP_TRY(matvec_impl(h, h->pp, h->pq, prec, scal + S_PQ, scal + S_RZ, scal + S_RZN));
  count_launch();
  k_pcg_xr_check<<<g, 256, 0, st>>>(m, h->px, h->pr, h->pp, h->pq, scal, h->pcg_part, h->pcg_ticket, cond,
                                    use_cond ? 1 : 0);
  SDP_TRY(precond_apply_impl(h, h->pr, h->pz, prec, scal + S_RZN));
  count_launch();
  k_pcg_p<<<g, 256, 0, st>>>(m, h->pp, h->pz, scal);
  return SDP_OK;
}

// Build (or reuse) the executable graph: one while-node whose body is one PCG
// iteration; the loop runs on the device until the recursive residual meets the
// tolerance or the iteration budget is spent, with no host round trip.
static sdp_status pcg_graph(sdp_problem* h, int prec) {
  const int64_t key = h->pc_generation * 8 + prec;
  if (h->pcg_exec && h->pcg_key == key) return SDP_OK;
  if (h->pcg_exec) {
    cudaGraphExecDestroy(h->pcg_exec);
    h->pcg_exec = nullptr;
  }
  if (h->pcg_graph) {
    cudaGraphDestroy(h->pcg_graph);
    h->pcg_graph = nullptr;
  }
  SDP_TRY(ensure_lowprec_W(h, prec));
  cudaGraph_t g = nullptr;
  SDP_CK(h, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond;
  SDP_CK(h, cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  SDP_CK(h, cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t user = h->stream;
  h->stream = h->capture_stream;
  const int64_t l0 = t_launches;
  ktimer_pause(true);
  cudaError_t e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  sdp_status s = (e == cudaSuccess) ? pcg_body(h, prec, cond, true) : SDP_ERR_CUDA;
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(h->stream, &out);
  ktimer_pause(false);
  h->pcg_body_launches = t_launches - l0;   // captured, not launched: counted per iteration instead
  g_launches.fetch_sub(h->pcg_body_launches);
  t_launches = l0;
  h->stream = user;
  if (e != cudaSuccess || e2 != cudaSuccess || s != SDP_OK) {
    cudaGraphDestroy(g);
    h->last_error = std::string("pcg graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
    return s != SDP_OK ? s : SDP_ERR_CUDA;
  }
  SDP_CK(h, cudaGraphInstantiate(&h->pcg_exec, g, 0));
  h->pcg_graph = g;
  h->pcg_key = key;
  return SDP_OK;
}

static double read_scalar(sdp_problem* h, const double* dev) {
  double v = 0.0;
  cudaMemcpyAsync(&v, dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  return v;
}

// Plain PCG from x = 0 in precision prec; x receives the iterate.  *rel is the
// recursive relative residual at exit.
static sdp_status pcg_core(sdp_problem* h, const double* rhs, double* x, double rtol, int maxit, int prec,
                           int* iters, double* rel, bool* brk) {
  cudaStream_t st = h->stream;
  const int m = h->m;
  double* scal = h->scal;
  const bool use_graph = h->prm.pcg_graph != 0;
  if (use_graph) SDP_TRY(pcg_graph(h, prec));
  else SDP_TRY(ensure_lowprec_W(h, prec));
  SDP_CK(h, cudaMemcpyAsync(h->pr, rhs, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDP_CK(h, cudaMemsetAsync(h->px, 0, m * sizeof(double), st));
  dot(st, m, h->pr, h->pr, scal + S_NR0, h->part);
  const double nr0sq = read_scalar(h, scal + S_NR0);
  if (!std::isfinite(nr0sq)) {
    h->last_error = "pcg: non-finite right-hand side";
    return SDP_ERR_NUMERIC;
  }
  if (nr0sq == 0.0) {
    SDP_CK(h, cudaMemsetAsync(x, 0, m * sizeof(double), st));
    *iters = 0;
    *rel = 0.0;
    if (brk) *brk = false;
    return SDP_OK;
  }
  SDP_TRY(precond_apply_impl(h, h->pr, h->pz, prec, scal + S_RZ));
  SDP_CK(h, cudaMemcpyAsync(h->pp, h->pz, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  count_launch();
  k_pcg_init<<<1, 1, 0, st>>>(scal, rtol, maxit);
  double v[11];
  if (use_graph) {
    SDP_CK(h, cudaGraphLaunch(h->pcg_exec, st));
    SDP_CK(h, cudaMemcpyAsync(v, scal, 11 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SDP_CK(h, cudaStreamSynchronize(st));
  } else {
    // the same body, launched from the host one iteration at a time
    do {
      SDP_TRY(pcg_body(h, prec, cudaGraphConditionalHandle{}, false));
      SDP_CK(h, cudaMemcpyAsync(v, scal, 11 * sizeof(double), cudaMemcpyDeviceToHost, st));
      SDP_CK(h, cudaStreamSynchronize(st));
    } while (v[S_GO] != 0.0);
  }
  SDP_CK(h, cudaMemcpyAsync(x, h->px, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const int its = (int)v[S_IT];
  if (use_graph) g_launches.fetch_add((int64_t)its * h->pcg_body_launches);
  const double rr = v[S_RR];
  *iters = its;
  *rel = std::sqrt(rr / nr0sq);
  if (brk) *brk = (v[S_BRK] != 0.0);
  if (!std::isfinite(rr)) {
    h->last_error = "pcg: non-finite residual";
    return SDP_ERR_NUMERIC;
  }
  return (rr <= v[S_TOL2]) ? SDP_OK : SDP_ERR_MAXIT;
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

static sdp_status pcg_impl_(sdp_problem* h, const double* r, double* y, double rtol, int maxit, int prec,
                            int* iters, double* relres);
sdp_status pcg_impl(sdp_problem* h, const double* r, double* y, double rtol, int maxit, int prec, int* iters,
                    double* relres) {
  ktimer_begin(h->stream, "pcg");
  sdp_status s = pcg_impl_(h, r, y, rtol, maxit, prec, iters, relres);
  ktimer_end(h->stream, "pcg", 0.0, 0.0);
  return s;
}
static sdp_status pcg_impl_(sdp_problem* h, const double* r, double* y, double rtol, int maxit, int prec,
                            int* iters, double* relres) {
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
  const double inner_fp64 = std::max(h->prm.inner_rtol, rtol);
  const double inner_lp = std::max(h->prm.inner_rtol_lp, rtol);
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    int it = 0;
    double rr = 0.0;
    const int budget = std::max(1, std::min(maxit - total, 500));
    bool brk = false;
    sdp_status s = pcg_core(h, resid, corr, prec == SDP_FP64 ? inner_fp64 : inner_lp, budget, prec, &it, &rr,
                            &brk);
    total += it;
    if (s != SDP_OK && s != SDP_ERR_MAXIT) return s;
    if (brk && it <= 1 && prec == SDP_FP64) break;   // breakdown before any progress
    const double tr_prev = tr;
    if (it > 0) axpby(st, m, 1.0, y, 1.0, corr, y);
    SDP_TRY(true_residual(h, r, y, resid, &tr));
    if (!(tr < tr_prev)) {
      // the sweep did not reduce the FP64 residual: drop its correction; a
      // reduced-precision inner solve hands over to FP64, an FP64 one stops
      if (it > 0) axpby(st, m, 1.0, y, -1.0, corr, y);
      SDP_TRY(true_residual(h, r, y, resid, &tr));
      if (prec == SDP_FP64) break;
      prec = SDP_FP64;
      h->pcg_prec_fallbacks++;
      continue;
    }
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
