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
#include <cstdio>

namespace sdpgb {

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }


// A breakdown (p.q or r.z not positive and finite: rounding has made the
// preconditioned operator indefinite in some direction) leaves x and r at the
// last good iterate, sets scal[S_BRK] and ends the loop; the restarted outer
// solve then continues from the true residual.
//
// CG minimises the H-norm of the error, not the residual norm, which on an
// ill-conditioned system can rise far above its starting value before it
// falls.  A run therefore keeps the iterate of smallest recursive residual
// (xb, with ||r||^2 in scal[S_RRB]): the iteration that finds a new minimum sets
// scal[S_NEWB] and the direction update that follows copies x into xb, so a
// run that ends above its best returns the best.

// p = z + beta p  with beta = rz_new / rz
__device__ __forceinline__ void pcg_p_body(int lb, int nb, int m, double* __restrict__ p,
                                           const double* __restrict__ z, const double* __restrict__ x,
                                           double* __restrict__ xb, double* scal) {
  if (scal[S_NEWB] != 0.0)
    for (int i = lb * blockDim.x + threadIdx.x; i < m; i += nb * blockDim.x) xb[i] = x[i];
  if (scal[S_GO] == 0.0) return;   // the loop has stopped: r may be exactly zero
  const double rzn = scal[S_RZN], rz = scal[S_RZ];
  if (!(rzn > 0.0 && isfinite(rzn) && rz > 0.0)) {
    if (lb == 0 && threadIdx.x == 0) scal[S_BRK] = 1.0;
    return;
  }
  const double beta = rzn / rz;
  for (int i = lb * blockDim.x + threadIdx.x; i < m; i += nb * blockDim.x) p[i] = fma(beta, p[i], z[i]);
}
__global__ void k_pcg_p(int m, double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ x,
                        double* __restrict__ xb, double* scal) {
  pcg_p_body(blockIdx.x, gridDim.x, m, p, z, x, xb, scal);
}

// x += a p;  r -= a q  (a = rz / pq), ||r||^2, iteration count and the loop
// condition, in one kernel (the last block to finish reduces and decides).
// Returns true in the deciding thread when the loop must go on.
__device__ __forceinline__ bool pcg_xr_body(int lb, int nb, int m, double* __restrict__ x, double* __restrict__ r,
                                            const double* __restrict__ p, const double* __restrict__ q,
                                            double* scal, double* part, unsigned int* ticket, bool* decided) {
  const double pq = scal[S_PQ], rz = scal[S_RZ];
  const bool ok = pq > 0.0 && rz > 0.0 && isfinite(pq) && isfinite(rz);
  const double a = ok ? rz / pq : 0.0;
  double rr = 0.0;
  for (int i = lb * blockDim.x + threadIdx.x; i < m; i += nb * blockDim.x) {
    double ri = r[i];
    if (ok) {
      x[i] = fma(a, p[i], x[i]);
      ri = fma(-a, q[i], ri);
      r[i] = ri;
    }
    rr = fma(ri, ri, rr);
  }
  double tot;
  *decided = false;
  if (lb_reduce(rr, part, ticket, &tot, lb, nb)) {
    scal[S_RR] = tot;
    const double it = scal[S_IT] + 1.0;
    scal[S_IT] = it;
    if (!ok) scal[S_BRK] = 1.0;
    const bool best = tot < scal[S_RRB];
    if (best) scal[S_RRB] = tot;
    scal[S_NEWB] = best ? 1.0 : 0.0;
    const bool go = ok && (tot > scal[S_TOL2]) && (it < scal[S_MAXIT]) && isfinite(tot) && scal[S_BRK] == 0.0;
    scal[S_GO] = go ? 1.0 : 0.0;
    *decided = true;
    return go;
  }
  return false;
}
__global__ void k_pcg_xr_check(int m, double* __restrict__ x, double* __restrict__ r,
                               const double* __restrict__ p, const double* __restrict__ q, double* scal,
                               double* part, unsigned int* ticket, cudaGraphConditionalHandle cond, int use_cond) {
  bool decided = false;
  const bool go = pcg_xr_body(blockIdx.x, gridDim.x, m, x, r, p, q, scal, part, ticket, &decided);
  if (decided && use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
}

// Batched forms: the problems whose loop stops leave the batch's active set;
// the batch loop goes on while any problem is active.
__global__ void kb_pcg_xr(BDesc* __restrict__ desc, const int* __restrict__ off, int N) {
  const int i = batch_find(off, N, blockIdx.x);
  BDesc& D = desc[i];
  if (!D.active) return;
  bool decided = false;
  const bool go = pcg_xr_body(blockIdx.x - off[i], off[i + 1] - off[i], D.m, D.px, D.pr, D.pp, D.pq, D.scal,
                              D.part, D.ticket, &decided);
  if (decided && !go) D.active = 0;
}
// The direction update also decides the batch loop: block 0 reads every
// problem's active flag (final since kb_pcg_xr ran earlier in the stream) and
// sets the graph condition, or with flag != nullptr (host-driven loop) writes
// flag[0] = some problem active, flag[1 + i] = problem i active.
__global__ void kb_pcg_p(const BDesc* __restrict__ desc, const int* __restrict__ off, int N,
                         cudaGraphConditionalHandle cond, int* flag) {
  if (blockIdx.x == 0) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const int a = desc[i].active ? 1 : 0;
      if (flag) flag[1 + i] = a;
      if (a) any = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (flag) flag[0] = any;
      else cudaGraphSetConditional(cond, any ? 1u : 0u);
    }
  }
  const int i = batch_find(off, N, blockIdx.x);
  const BDesc& D = desc[i];
  if (!D.active) return;
  pcg_p_body(blockIdx.x - off[i], off[i + 1] - off[i], D.m, D.pp, D.pz, D.px, D.pxb, D.scal);
}
int batch_blocks_vec(int m) { return (int)std::min(cdiv(m, 256), 2048u); }
void batch_launch_xr(cudaStream_t st, BDesc* desc, const int* off, int N, int nb) {
  count_launch();
  if (nb > 0) kb_pcg_xr<<<nb, 256, 0, st>>>(desc, off, N);
}
void batch_launch_p(cudaStream_t st, const BDesc* desc, const int* off, int N, int nb,
                    cudaGraphConditionalHandle cond, int* flag) {
  count_launch();
  kb_pcg_p<<<nb > 0 ? nb : 1, 256, 0, st>>>(desc, off, N, cond, flag);
}

__global__ void k_pcg_init(double* scal, double rtol, int maxit) {
  scal[S_RZN] = scal[S_RZ];
  scal[S_TOL2] = rtol * rtol * scal[S_NR0];
  scal[S_IT] = 0.0;
  scal[S_MAXIT] = (double)maxit;
  scal[S_BRK] = 0.0;
  scal[S_GO] = 1.0;
  scal[S_RRB] = scal[S_NR0];   // the start x = 0 is the best so far
  scal[S_NEWB] = 0.0;
}

static sdp_status pcg_alloc(sdp_problem* h) {
  if (h->pr) return SDP_OK;
  const int m = h->m;
  SDP_TRY(h->allocT(&h->pr, m));
  SDP_TRY(h->allocT(&h->pz, m));
  SDP_TRY(h->allocT(&h->pp, m));
  SDP_TRY(h->allocT(&h->pq, m));
  SDP_TRY(h->allocT(&h->px, m));
  SDP_TRY(h->allocT(&h->pxb, m));
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
  // the core solve stays in FP64 inside PCG: near the optimum the Hhat core has
  // kappa ~ 1 / mu, and its FP32 inverse (what sdp_precond_apply uses for
  // prec != FP64) cost about twice the PCG iterations in measurements
  SDP_TRY(precond_apply_impl(h, h->pr, h->pz, SDP_FP64, scal + S_RZN));
  count_launch();
  k_pcg_p<<<g, 256, 0, st>>>(m, h->pp, h->pz, h->px, h->pxb, scal);
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

// Start of one PCG run from x = 0 on rhs (precision prec): r = rhs, z = M r,
// p = z, scalars initialised on the device.  *nr0sq = ||rhs||^2 (zero: nothing
// to run).  The loop itself is run by the caller (pcg_run, or a batch).
static sdp_status pcg_start(sdp_problem* h, const double* rhs, double rtol, int maxit, int prec, bool graph,
                            double* nr0sq) {
  cudaStream_t st = h->stream;
  const int m = h->m;
  double* scal = h->scal;
  if (graph) SDP_TRY(pcg_graph(h, prec));
  else SDP_TRY(ensure_lowprec_W(h, prec));
  SDP_CK(h, cudaMemcpyAsync(h->pr, rhs, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDP_CK(h, cudaMemsetAsync(h->px, 0, m * sizeof(double), st));
  SDP_CK(h, cudaMemsetAsync(h->pxb, 0, m * sizeof(double), st));
  dot(st, m, h->pr, h->pr, scal + S_NR0, h->part);
  *nr0sq = read_scalar(h, scal + S_NR0);
  if (!std::isfinite(*nr0sq)) {
    h->last_error = "pcg: non-finite right-hand side";
    return SDP_ERR_NUMERIC;
  }
  if (*nr0sq == 0.0) return SDP_OK;
  SDP_TRY(precond_apply_impl(h, h->pr, h->pz, SDP_FP64, scal + S_RZ));
  SDP_CK(h, cudaMemcpyAsync(h->pp, h->pz, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  count_launch();
  k_pcg_init<<<1, 1, 0, st>>>(scal, rtol, maxit);
  return SDP_OK;
}

// The loop on the handle's own stream: the device-side graph, or the host loop.
static sdp_status pcg_run(sdp_problem* h, int prec, bool graph) {
  cudaStream_t st = h->stream;
  if (graph) {
    SDP_CK(h, cudaGraphLaunch(h->pcg_exec, st));
    return SDP_OK;
  }
  double go = 1.0;
  while (go != 0.0) {
    SDP_TRY(pcg_body(h, prec, cudaGraphConditionalHandle{}, false));
    SDP_CK(h, cudaMemcpyAsync(&go, h->scal + S_GO, sizeof(double), cudaMemcpyDeviceToHost, st));
    SDP_CK(h, cudaStreamSynchronize(st));
  }
  return SDP_OK;
}

// End of a run: x = the iterate of smallest recursive residual (the last one
// when its iteration set a new minimum, else the copy in pxb), iteration
// count, that iterate's recursive relative residual.
static sdp_status pcg_finish(sdp_problem* h, double* x, double nr0sq, bool graph, int* iters, double* rel,
                             bool* brk) {
  cudaStream_t st = h->stream;
  const int m = h->m;
  double v[13];
  SDP_CK(h, cudaMemcpyAsync(v, h->scal, 13 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SDP_CK(h, cudaStreamSynchronize(st));
  SDP_CK(h, cudaMemcpyAsync(x, v[S_NEWB] != 0.0 ? h->px : h->pxb, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const int its = (int)v[S_IT];
  if (graph) g_launches.fetch_add((int64_t)its * h->pcg_body_launches);
  const double rr = v[S_RRB];
  *iters = its;
  *rel = std::sqrt(rr / nr0sq);
  if (brk) *brk = (v[S_BRK] != 0.0);
  if (!std::isfinite(rr) || !std::isfinite(v[S_RR])) {
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

// Restarted PCG = iterative refinement on the true FP64 residual.  Each sweep
// runs PCG from zero on the current residual to the inner tolerance; restarting
// discards the Krylov recurrences that rounding in the Woodbury apply (about
// kappa(Ht) eps, Section IV) and in a reduced-precision matvec corrupts, so
// the true residual keeps falling where one long PCG run stagnates.  The sweep
// logic lives in PcgSweeps so that a batch runs exactly the same rules.
sdp_status pcg_sweeps_init(sdp_problem* h, PcgSweeps* S, const double* r, double* y, double rtol, int maxit,
                           int prec) {
  SDP_TRY(pcg_alloc(h));
  if (!h->pc_valid) SDP_TRY(precond_build_impl(h));
  cudaStream_t st = h->stream;
  const int m = h->m;
  *S = PcgSweeps{};
  S->r = r;
  S->y = y;
  S->rtol = rtol;
  S->maxit = maxit;
  S->prec = prec;
  S->sweeps = std::max(1, h->prm.refine_maxit);
  S->inner_fp64 = std::max(h->prm.inner_rtol, rtol);
  S->inner_lp = std::max(h->prm.inner_rtol_lp, rtol);
  S->tr = 1.0;
  S->result = SDP_ERR_MAXIT;
  SDP_CK(h, cudaMemsetAsync(y, 0, m * sizeof(double), st));
  SDP_CK(h, cudaMemcpyAsync(h->pbest, r, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return SDP_OK;
}

// Starts the next sweep; *run = false when the solve is over, or when this
// sweep has nothing to iterate (it is then finished here).
sdp_status pcg_sweep_begin(sdp_problem* h, PcgSweeps* S, bool graph, bool* run) {
  *run = false;
  if (S->finished || S->sweep >= S->sweeps) {
    S->finished = true;
    return SDP_OK;
  }
  // iterations of one sweep: a restart discards the Krylov space, so a sweep must
  // be long enough to resolve the k(k+1)/2 outlying eigenvalues that H - Hhat
  // (rank <= k(k+1)/2, Section V) leaves, on top of the bulk; each later sweep gets twice the budget of the
  // one before (up to 8x), since the residual a sweep leaves is concentrated
  // on the slowest part of the spectrum
  const int kk = h->pc_hat ? h->kpc : 0;
  const int base = std::max(500, kk * (kk + 1) / 2 + 500);
  S->budget = std::max(1, std::min(S->maxit - S->total, base << std::min(S->sweep, 3)));
  S->graph = graph;
  SDP_TRY(pcg_start(h, h->pbest, S->prec == SDP_FP64 ? S->inner_fp64 : S->inner_lp, S->budget, S->prec, graph,
                    &S->nr0sq));
  if (S->nr0sq == 0.0) {
    S->finished = true;       // zero residual: y is exact already
    S->result = SDP_OK;
    S->tr = 0.0;
    return SDP_OK;
  }
  *run = true;
  return SDP_OK;
}

// Ends the running sweep: adds the correction and decides what comes next.
sdp_status pcg_sweep_end(sdp_problem* h, PcgSweeps* S) {
  cudaStream_t st = h->stream;
  const int m = h->m;
  int it = 0;
  double rr = 0.0;
  bool brk = false;
  sdp_status s = pcg_finish(h, h->pcorr, S->nr0sq, S->graph, &it, &rr, &brk);
  S->sweep++;
  S->total += it;
  if (s != SDP_OK && s != SDP_ERR_MAXIT) return s;
  if (brk && it <= 1 && s != SDP_OK && S->prec == SDP_FP64) {   // breakdown before any progress
    S->finished = true;
    return SDP_OK;
  }
  const double tr_prev = S->tr;
  if (it > 0) axpby(st, m, 1.0, S->y, 1.0, h->pcorr, S->y);
  SDP_TRY(true_residual(h, S->r, S->y, h->pbest, &S->tr));
  if (h->prm.verbose >= 2)
    std::fprintf(stderr, "  pcg sweep %d %s: %d its (budget %d), recursive %.2e, breakdown %d, true %.2e -> %.2e\n",
                 S->sweep - 1, S->prec == SDP_FP64 ? "fp64" : (S->prec == SDP_FP32 ? "fp32" : "bf16"), it,
                 S->budget, rr, brk ? 1 : 0, tr_prev, S->tr);
  if (!(S->tr < tr_prev)) {
    // the sweep did not reduce the FP64 residual: drop its correction; a
    // reduced-precision inner solve hands over to FP64, an FP64 one stops
    if (it > 0) axpby(st, m, 1.0, S->y, -1.0, h->pcorr, S->y);
    SDP_TRY(true_residual(h, S->r, S->y, h->pbest, &S->tr));
    if (S->prec == SDP_FP64) {
      S->finished = true;
    } else {
      S->prec = SDP_FP64;
      h->pcg_prec_fallbacks++;
    }
    return SDP_OK;
  }
  if (!std::isfinite(S->tr)) {
    h->last_error = "pcg: non-finite true residual";
    return SDP_ERR_NUMERIC;
  }
  if (S->tr <= S->rtol) {
    S->result = SDP_OK;
    S->finished = true;
  } else if (S->total >= S->maxit) {
    S->finished = true;
  } else if (S->prec != SDP_FP64 && S->tr > 0.1 * tr_prev) {
    // a reduced-precision sweep that gained less than one digit on the FP64
    // residual has reached what its rounding allows: the next sweeps run in FP64
    S->prec = SDP_FP64;
    h->pcg_prec_fallbacks++;
  }
  return SDP_OK;
}

static sdp_status pcg_impl_(sdp_problem* h, const double* r, double* y, double rtol, int maxit, int prec,
                            int* iters, double* relres) {
  PcgSweeps S;
  SDP_TRY(pcg_sweeps_init(h, &S, r, y, rtol, maxit, prec));
  const bool graph = h->prm.pcg_graph != 0;
  for (;;) {
    bool run = false;
    SDP_TRY(pcg_sweep_begin(h, &S, graph, &run));
    if (!run) break;
    SDP_TRY(pcg_run(h, S.prec, graph));
    SDP_TRY(pcg_sweep_end(h, &S));
  }
  if (iters) *iters = S.total;
  if (relres) *relres = S.tr;
  return S.result;
}

sdp_status pcg_impl(sdp_problem* h, const double* r, double* y, double rtol, int maxit, int prec, int* iters,
                    double* relres) {
  ktimer_begin(h->stream, "pcg");
  sdp_status s = pcg_impl_(h, r, y, rtol, maxit, prec, iters, relres);
  ktimer_end(h->stream, "pcg", 0.0, 0.0);
  return s;
}

}  // namespace sdpgb
