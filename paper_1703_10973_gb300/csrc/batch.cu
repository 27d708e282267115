// Batched solves: many SDPs advanced in lockstep, with every PCG iteration of
// all their Newton systems run as one sequence of launches over all problems.
//
// sdp_batch_solve runs the interior-point iterations of every problem of the
// batch together.  The dense per-problem phases (NT scaling, preconditioner,
// step lengths, update: ipm_phase_a/b/c) run on each problem's own stream from
// one host thread per problem.  The two Newton systems of an iteration are
// solved for all problems at once: each PCG iteration is one fixed sequence of
// batched kernels (assemble, SpMM, SDDMM with p.Hp, x/r update with the loop
// test, the Hhat apply, direction update), each launch covering every problem
// -- the grid is the concatenation of the problems' own grids, and a block
// finds its problem from a table of block offsets.  The sequence is captured
// once as a CUDA graph whose conditional while node runs until no problem is
// active; a problem leaves the active set when its own loop test fails, and its
// blocks then return at once.  Every batched kernel runs the same device code
// over the same block partition as the single-problem kernel, so a problem's
// iterates are bitwise the same in a batch and alone.
//
// The restarted outer loop (refinement on the FP64 true residual) is the
// single-problem PcgSweeps state machine, stepped for all problems together.
// Supported: the Hhat preconditioner (the default) with the FP64 matvec or the
// FP32 / BF16 split matvec; a problem whose reduced-precision sweep stalls hands
// over to FP64 on its own, so one batched iteration can mix the forms.
#include "internal.cuh"

#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

namespace sdpgb {

static inline int cdivi(int a, int b) { return (a + b - 1) / b; }

enum { BK_ASM, BK_SPMM, BK_SDDMM, BK_VEC, BK_HATU, BK_TAIL, BK_FWDP, BK_FWDR, BK_GEMV, BK_OUTR, BK_BWDP,
       BK_SPLG, BK_SPLR, BK_SPLQ, BK_SPMM_LP, BK_COUNT };

}  // namespace sdpgb

struct sdp_batch {
  std::vector<sdp_problem*> hs;
  cudaStream_t stream = nullptr;      // the batched launches
  cudaStream_t capture = nullptr;     // capture stream for the graph
  sdpgb::BDesc* ddesc = nullptr;
  int* doff = nullptr;                // BK_COUNT x (N + 1) block offsets
  std::vector<int> off;               // host copy
  int total[sdpgb::BK_COUNT] = {};
  int nmax = 0;
  bool any_lp = false;                // some problem runs FP32 sweeps: the graph holds the FP32 matvec
  bool host_loop = false;             // pcg_graph == 0: the host launches every iteration (profilers)
  int* dflag = nullptr;               // host loop: "some problem active" after each iteration
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t body_launches = 0;
  double stage_s[8] = {};             // wall seconds per stage of the last solve, then
                                      // graph seconds, graph launches, batched iterations
  int groups = 0;                     // lockstep groups solved concurrently (0: pairs)
  std::vector<sdp_batch*> child;      // one batch per group when groups > 1
  std::vector<std::vector<int>> members;   // problems of each group
  std::vector<cudaStream_t> child_streams;
  std::string last_error;
  // per-member interior-point state of the lockstep iterations (indices follow hs)
  std::vector<sdpgb::IpmStepState> ms;
  std::vector<sdp_status> mst;
  std::vector<char> mdone;            // 0 running, 1 converged, 2 iteration limit, 3 error
  std::vector<int> mpcg, mit, mits;   // PCG iterations so far, IPM iterations in this batch, last solve's
  std::vector<double> mrr, mstart, mfin;   // last true residual; seconds (from the epoch) joined / finished
  std::chrono::steady_clock::time_point epoch = std::chrono::steady_clock::now();
  bool dirty = true;                  // membership changed: offsets and the graph are rebuilt before use
  int spmm_r = 4;                     // rows of W per CTA of the batched SpMM (autotuned)
  bool tuned = false;                 // spmm_r chosen for the current members
  float tune_ms[4] = {};              // measured time per candidate R = 1, 2, 4, 8 (0: not run)
  int ndesc = 0, noff = 0;            // capacities of ddesc and doff
};

namespace sdpgb {

static bool batch_supported(sdp_problem* h, std::string* why) {
  if (h->prm.prec != SDP_FP64 && h->prm.prec != SDP_FP32 && h->prm.prec != SDP_BF16) {
    *why = "batched solves run the FP64, FP32 or BF16 split matvec";
    return false;
  }
  if (h->prm.precond != SDP_PRECOND_HAT) { *why = "batched solves use the Hhat preconditioner"; return false; }
  const int k = std::min(h->kcap, std::max(h->n - 1, 0));
  if (k < 1 || k > 8) { *why = "batched solves need a split rank (k, or k_max) in 1..8"; return false; }
  return true;
}

// Block offsets of every batched kernel (sizes only, fixed for the batch).
static void batch_offsets(sdp_batch* b) {
  const int N = (int)b->hs.size();
  b->off.assign((size_t)BK_COUNT * (N + 1), 0);
  b->nmax = 0;
  b->any_lp = false;
  for (int i = 0; i < N; ++i) b->nmax = std::max(b->nmax, b->hs[i]->n);
  for (int i = 0; i < N; ++i) {
    sdp_problem* h = b->hs[i];
    const int k = std::min(h->kcap, h->n - 1), Rk = h->hs_nr * k;   // grids for the largest rank
    const int cnt[BK_COUNT] = {batch_blocks_assemble(h->nnzV), batch_blocks_spmm(h->n, b->spmm_r), batch_blocks_sddmm(h->m),
                               batch_blocks_vec(h->m),         batch_blocks_hat_u(h->n), batch_blocks_tail(h->m),
                               batch_blocks_fwdP(h->hs_np),    batch_blocks_warp_rows(h->hs_nr),
                               batch_blocks_warp_rows(Rk),     batch_blocks_out_bwd(Rk, h->hs_np),
                               0,
                               batch_blocks_split_G(h->n),     batch_blocks_split_R(h->n),
                               batch_blocks_split_Q(h->n, k),  batch_blocks_spmm_lp(h->n, b->nmax)};
    for (int kd = 0; kd < BK_COUNT; ++kd)
      b->off[(size_t)kd * (N + 1) + i + 1] = b->off[(size_t)kd * (N + 1) + i] + cnt[kd];
    if (h->prm.prec == SDP_FP32 || h->prm.prec == SDP_BF16) b->any_lp = true;
  }
  for (int kd = 0; kd < BK_COUNT; ++kd) b->total[kd] = b->off[(size_t)kd * (N + 1) + N];
}

static BDesc make_desc(sdp_problem* h, int active, int prec) {
  BDesc D{};
  D.n = h->n; D.m = h->m; D.k = h->kpc; D.np = h->hs_np; D.nr = h->hs_nr; D.Rk = h->hs_nr * h->kpc;
  D.nnzV = h->nnzV;
  D.active = active;
  D.zscale = h->zscale;
  D.inv_tau2 = 1.0 / (h->tau * h->tau);
  D.rowptr = h->rowptr; D.rowperm = h->rowperm; D.colidx = h->colidx; D.sptr = h->sptr; D.scon = h->scon;
  D.eptr = h->eptr; D.ep = h->ep; D.eq = h->eq;
  D.scoef = h->scoef; D.ecoef = h->ecoef; D.ginv = h->ginv;
  D.W = h->W; D.U = h->U; D.T = h->T; D.Vval = h->Vval;
  D.pverts = h->hs_pverts; D.rverts = h->hs_rverts; D.btptr = h->hs_btptr; D.btslot = h->hs_btslot;
  D.bp = h->hs_bp; D.bptr = h->hs_bptr; D.bcol = h->hs_bcol;
  D.D = h->hs_D; D.F = h->hs_F; D.Cinv = h->hs_Cinv; D.CinvT = h->hs_CinvT;
  D.yP = h->hs_yP; D.v1 = h->hs_v1; D.v2 = h->hs_v2; D.uvec = h->uvec; D.Bn = h->Bn;
  D.px = h->px; D.pr = h->pr; D.pp = h->pp; D.pq = h->pq; D.pz = h->pz; D.pxb = h->pxb;
  D.scal = h->scal; D.part = h->pcg_part; D.ticket = h->pcg_ticket;
  D.lp = (prec == SDP_FP32 || prec == SDP_BF16) ? 1 : 0;
  D.bf = (prec == SDP_BF16) ? 1 : 0;
  D.ks = (D.lp && (D.bf ? h->W16_key : h->W32_key) >= 0) ? h->kpc : 0;
  D.W16 = h->W16;
  D.W32 = h->W32; D.T32 = h->T32; D.mvR = h->mv_R; D.mvPart = h->mv_part;
  D.Etop = h->Etop; D.wtop = h->wtop; D.mvG = h->mv_G; D.mvQ = h->mv_Q;
  // the core solve runs in FP64 in every sweep (see pcg_body); the FP32 copy of
  // the Schur-factor inverse serves sdp_precond_apply with prec != SDP_FP64
  D.lpc = 0;
  D.Cinv32 = h->hs_Cinv32; D.CinvT32 = h->hs_CinvT32; D.v1f = h->hs_v1f; D.v2f = h->hs_v2f;
  return D;
}

// One PCG iteration of every active problem (the body of the batched loop).
// mode (host loop only): per problem, 1 when it runs an FP64-matvec sweep this
// iteration, 2 for a reduced-precision sweep, 0 when inactive; the batched
// matvecs are then timed as classes "matvec_b" (FP64) and "matvec_lp_b" (split
// FP32 / BF16) with the algorithmic work of their problems.  FP64: T = W V
// (2 nnzV n flops) and one length-n dot per stored entry (2 nent n); bytes: W
// and T once each, the sparse data.  Split form: the same flops in FP32; bytes:
// W_s read by the SpMM and by the gather (2 n^2 s_W), T written and read
// (2 n^2 4), the sparse data.
static void batch_body(sdp_batch* b, cudaStream_t st, cudaGraphConditionalHandle cond, int* flag,
                       const std::vector<char>* mode = nullptr) {
  const int N = (int)b->hs.size();
  const int* o = b->doff;
  auto off = [&](int kd) { return o + (size_t)kd * (N + 1); };
  double fl = 0.0, by = 0.0, fl_lp = 0.0, by_lp = 0.0;
  if (mode) {
    for (int i = 0; i < N; ++i) {
      const sdp_problem* h = b->hs[i];
      const double f = 2.0 * h->nnzV * (double)h->n + 2.0 * h->nent * (double)h->n;
      if ((*mode)[i] == 1) {
        fl += f;
        by += 16.0 * h->n * (double)h->n + 12.0 * h->nnzV + 16.0 * h->m;
      } else if ((*mode)[i] == 2) {
        const double sw = (h->prm.prec == SDP_BF16) ? 2.0 : 4.0;
        fl_lp += f;
        by_lp += (2.0 * sw + 8.0) * h->n * (double)h->n + 12.0 * h->nnzV + 16.0 * h->m;
      }
    }
    ktimer_begin(st, "matvec_b");
  }
  // A mixed batch in the graph gathers both forms in one launch after the
  // reduced-precision pieces; the instrumented host loop keeps them apart so that
  // each class is timed on its own.  Same partitions either way, same results.
  const bool merge = b->any_lp && !mode;
  batch_launch_matvec(st, b->ddesc, off(BK_ASM), off(BK_SPMM), off(BK_SDDMM), N, b->total[BK_ASM],
                      b->total[BK_SPMM], merge ? 0 : b->total[BK_SDDMM], b->nmax, b->spmm_r);
  if (mode) ktimer_end(st, "matvec_b", fl, by);
  if (b->any_lp) {  // same SDDMM partition (and reduction groups) as the FP64 form
    if (mode) ktimer_begin(st, "matvec_lp_b");
    batch_launch_matvec_lp(st, b->ddesc, off(BK_SPLG), off(BK_SPLR), off(BK_SPLQ), off(BK_SPMM_LP), off(BK_SDDMM),
                           N, b->total[BK_SPLG], b->total[BK_SPLR], b->total[BK_SPLQ], b->total[BK_SPMM_LP],
                           b->total[BK_SDDMM], b->nmax, !merge);
    if (merge) batch_launch_sddmm_mixed(st, b->ddesc, off(BK_SDDMM), N, b->total[BK_SDDMM]);
    if (mode) ktimer_end(st, "matvec_lp_b", fl_lp, by_lp);
  }
  batch_launch_xr(st, b->ddesc, off(BK_VEC), N, b->total[BK_VEC]);
  batch_launch_hat_u(st, b->ddesc, off(BK_HATU), N, b->total[BK_HATU]);
  batch_launch_core_solve(st, b->ddesc, N, off(BK_FWDP), b->total[BK_FWDP], off(BK_FWDR), b->total[BK_FWDR],
                          off(BK_GEMV), b->total[BK_GEMV], off(BK_OUTR), b->total[BK_OUTR], off(BK_BWDP),
                          b->total[BK_BWDP]);
  batch_launch_tail(st, b->ddesc, off(BK_TAIL), N, b->total[BK_TAIL]);
  batch_launch_p(st, b->ddesc, off(BK_VEC), N, b->total[BK_VEC], cond, flag);
}

// Block offsets, device tables and the captured loop for the current members;
// rebuilt after a membership change (continuous batching: sdp_batch_add/remove).
static sdp_status batch_prepare(sdp_batch* b) {
  if (!b->dirty && (b->exec || b->host_loop)) return SDP_OK;
  const int N = (int)b->hs.size();
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->host_loop = false;
  batch_offsets(b);
  if (N > b->ndesc || (int)b->off.size() > b->noff) {
    pool_free(b->ddesc, b->stream);
    pool_free(b->doff, b->stream);
    pool_free(b->dflag, b->stream);
    b->ddesc = nullptr;
    b->doff = nullptr;
    b->dflag = nullptr;
    b->ndesc = b->noff = 0;
    const int cap = std::max(N, 2 * b->ndesc);
    const size_t offcap = (size_t)BK_COUNT * (cap + 1);
    if (pool_malloc((void**)&b->ddesc, sizeof(BDesc) * cap, b->stream) != cudaSuccess ||
        pool_malloc((void**)&b->doff, sizeof(int) * offcap, b->stream) != cudaSuccess ||
        pool_malloc((void**)&b->dflag, sizeof(int) * (cap + 1), b->stream) != cudaSuccess) {
      cudaGetLastError();
      b->last_error = "sdp_batch: device allocation failed";
      return SDP_ERR_OOM;
    }
    b->ndesc = cap;
    b->noff = (int)offcap;
  }
  cudaMemcpy(b->doff, b->off.data(), sizeof(int) * b->off.size(), cudaMemcpyHostToDevice);
  b->dirty = false;
  b->tuned = b->tuned && b->nmax > 0;
  if (b->hs[0]->prm.pcg_graph == 0) {
    b->host_loop = true;
    return SDP_OK;
  }
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle cond;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  if (cudaGraphCreate(&g, 0) != cudaSuccess || cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    b->last_error = "sdp_batch: graph creation failed";
    return SDP_ERR_CUDA;
  }
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) {
    cudaGraphDestroy(g);
    b->last_error = "sdp_batch: conditional node failed";
    return SDP_ERR_CUDA;
  }
  const int64_t l0 = t_launches;
  ktimer_pause(true);
  cudaError_t e = cudaStreamBeginCaptureToGraph(b->capture, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) batch_body(b, b->capture, cond, nullptr);
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->capture, &out);
  ktimer_pause(false);
  b->body_launches = t_launches - l0;
  g_launches.fetch_sub(b->body_launches);
  t_launches = l0;
  if (e != cudaSuccess || e2 != cudaSuccess || cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    b->last_error = std::string("sdp_batch: graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
    return SDP_ERR_CUDA;
  }
  b->graph = g;
  return SDP_OK;
}

// Autotuner of the batched SpMM tile: each candidate R (rows of W per CTA: 1, 2,
// 4, 8, within shared memory) runs on the batch's own data with the descriptors
// just uploaded, timed with CUDA events (five interleaved rounds of one warm-up
// and one timed launch, minimum kept); the fastest is kept and the launch
// structures are rebuilt for it.  T is
// scratch of the matvec, recomputed by every real launch, so the trial launches
// change nothing; every R computes each entry of T by the same FMA sequence.
static sdp_status batch_autotune(sdp_batch* b, const std::vector<BDesc>& hd) {
  const int N = (int)b->hs.size();
  // time the FP64 SpMM with every active problem in an FP64 sweep (problems in a
  // reduced-precision sweep would return at once), then restore the descriptors
  std::vector<BDesc> td(hd);
  for (BDesc& D : td) D.lp = 0;
  if (cudaMemcpyAsync(b->ddesc, td.data(), sizeof(BDesc) * N, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return SDP_ERR_CUDA;
  const int cand[4] = {1, 2, 4, 8};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SDP_ERR_CUDA;
  std::vector<int> off(N + 1, 0);
  int* doff = nullptr;
  if (pool_malloc((void**)&doff, sizeof(int) * (N + 1), b->stream) != cudaSuccess) {
    cudaGetLastError();
    return SDP_ERR_OOM;
  }
  // candidates interleaved over five rounds, the minimum per candidate kept: other
  // lockstep groups run their dense phases on the GPU meanwhile, and the minimum
  // is the least disturbed of the samples
  float best = 0.f;
  int best_r = b->spmm_r;
  for (int c = 0; c < 4; ++c) b->tune_ms[c] = 0.f;
  for (int round = 0; round < 5; ++round) {
    for (int c = 0; c < 4; ++c) {
      const int R = cand[c];
      if (!batch_spmm_fits(R, b->nmax)) continue;
      for (int i = 0; i < N; ++i) off[i + 1] = off[i] + batch_blocks_spmm(b->hs[i]->n, R);
      cudaMemcpyAsync(doff, off.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, b->stream);
      batch_launch_spmm(b->stream, R, b->ddesc, doff, N, off[N], b->nmax);   // warm-up
      cudaEventRecord(e0, b->stream);
      batch_launch_spmm(b->stream, R, b->ddesc, doff, N, off[N], b->nmax);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (b->tune_ms[c] == 0.f || ms < b->tune_ms[c]) b->tune_ms[c] = ms;
    }
  }
  for (int c = 0; c < 4; ++c) {
    if (b->tune_ms[c] == 0.f) continue;
    if (best == 0.f || b->tune_ms[c] < best) {
      best = b->tune_ms[c];
      best_r = cand[c];
    }
  }
  cudaMemcpyAsync(b->ddesc, hd.data(), sizeof(BDesc) * N, cudaMemcpyHostToDevice, b->stream);
  cudaStreamSynchronize(b->stream);
  pool_free(doff, b->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) {
    b->last_error = "sdp_batch: SpMM autotuning failed";
    return SDP_ERR_CUDA;
  }
  b->tuned = true;
  if (best_r != b->spmm_r) {
    b->spmm_r = best_r;
    b->dirty = true;
    SDP_TRY(batch_prepare(b));
  }
  return SDP_OK;
}

// The Newton systems H dy = rhs of the listed problems, solved together.
// While their Newton systems are solved, the listed problems issue all their
// work (sweep set-up, true residuals, the batched graph) on the batch's stream:
// their own streams are idle then, and a batch stream of high priority keeps
// this latency-bound work ahead of other lockstep groups' dense phases.  The
// guard hands each problem its own stream back, after the batch stream is idle.
struct StreamSwap {
  sdp_batch* b;
  std::vector<std::pair<sdp_problem*, cudaStream_t>> saved;
  StreamSwap(sdp_batch* bb, const std::vector<int>& idx) : b(bb) {
    if (!b->stream) return;
    for (int i : idx) {
      sdp_problem* h = b->hs[i];
      if (h->stream == b->stream) continue;
      cudaStreamSynchronize(h->stream);
      saved.push_back({h, h->stream});
      h->stream = b->stream;
    }
  }
  ~StreamSwap() {
    if (saved.empty()) return;
    cudaStreamSynchronize(b->stream);
    for (auto& sv : saved) sv.first->stream = sv.second;
  }
};

static sdp_status batch_newton(sdp_batch* b, const std::vector<int>& idx, std::vector<int>& its,
                               std::vector<double>& rr, std::vector<sdp_status>& st) {
  const int N = (int)b->hs.size();
  StreamSwap swap(b, idx);
  std::vector<PcgSweeps> S(N);
  std::vector<char> live(N, 0);
  for (int i : idx) {
    sdp_problem* h = b->hs[i];
    st[i] = pcg_sweeps_init(h, &S[i], h->rhs, h->dy, h->prm.pcg_rtol, h->prm.pcg_maxit, h->prm.prec);
    live[i] = (st[i] == SDP_OK);
  }
  SDP_TRY(batch_prepare(b));
  std::vector<BDesc> hd(N);
  for (;;) {
    std::vector<int> running;
    for (int i : idx) {
      if (!live[i]) continue;
      bool run = false;
      st[i] = pcg_sweep_begin(b->hs[i], &S[i], false, &run);
      if (st[i] != SDP_OK) { live[i] = 0; continue; }
      if (run) running.push_back(i);
      else live[i] = 0;
    }
    if (running.empty()) break;
    for (int i = 0; i < N; ++i) hd[i] = make_desc(b->hs[i], 0, S[i].prec);
    for (int i : running) {
      cudaStreamSynchronize(b->hs[i]->stream);
      hd[i].active = 1;
    }
    const auto g0 = std::chrono::steady_clock::now();
    if (cudaMemcpyAsync(b->ddesc, hd.data(), sizeof(BDesc) * N, cudaMemcpyHostToDevice, b->stream) != cudaSuccess) {
      b->last_error = std::string("sdp_batch: descriptor upload failed: ") + cudaGetErrorString(cudaGetLastError());
      return SDP_ERR_CUDA;
    }
    if (!b->tuned) SDP_TRY(batch_autotune(b, hd));
    if (b->host_loop) {
      // flags[0]: some problem active; flags[1 + i]: problem i active (read back
      // after every iteration, so each timed matvec knows its problems)
      std::vector<int> flags(N + 1, 0);
      std::vector<char> mode(N, 0);
      for (int i : running) mode[i] = (S[i].prec == SDP_FP64) ? 1 : 2;
      for (;;) {
        batch_body(b, b->stream, cudaGraphConditionalHandle{}, b->dflag, &mode);
        if (cudaMemcpyAsync(flags.data(), b->dflag, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost, b->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess) {
          b->last_error = std::string("sdp_batch: batched PCG failed: ") + cudaGetErrorString(cudaGetLastError());
          return SDP_ERR_CUDA;
        }
        if (!flags[0]) break;
        for (int i = 0; i < N; ++i) mode[i] = flags[1 + i] ? mode[i] : 0;
      }
    } else if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess) {
      b->last_error = std::string("sdp_batch: batched PCG failed: ") + cudaGetErrorString(cudaGetLastError());
      return SDP_ERR_CUDA;
    }
    b->stage_s[5] += std::chrono::duration<double>(std::chrono::steady_clock::now() - g0).count();
    b->stage_s[6] += 1.0;
    int max_it = 0;
    for (int i : running) {
      const int before = S[i].total;
      st[i] = pcg_sweep_end(b->hs[i], &S[i]);
      max_it = std::max(max_it, S[i].total - before);
      if (st[i] != SDP_OK) live[i] = 0;
    }
    if (!b->host_loop) g_launches.fetch_add((int64_t)max_it * b->body_launches);
    b->stage_s[7] += max_it;
  }
  for (int i : idx) {
    its[i] = S[i].total;
    rr[i] = S[i].tr;
    if (st[i] == SDP_OK && S[i].result != SDP_OK) st[i] = SDP_OK;   // MAXIT: keep the best iterate
  }
  return SDP_OK;
}

sdp_status self_batch_newton(sdp_problem* h, int* its, double* rr, bool* used) {
  *used = false;
  std::string why;
  if (h->prm.pcg_graph == 0 || !batch_supported(h, &why)) return SDP_OK;
  if (!h->self_batch) {
    sdp_problem* one[1] = {h};
    if (sdp_batch_create(one, 1, h->stream, &h->self_batch) != SDP_OK) return SDP_OK;   // old path
  }
  *used = true;
  std::vector<int> idx{0}, it(1, 0);
  std::vector<double> r(1, 0.0);
  std::vector<sdp_status> st(1, SDP_OK);
  ktimer_begin(h->stream, "pcg");
  const sdp_status s = batch_newton(h->self_batch, idx, it, r, st);
  ktimer_end(h->stream, "pcg", 0.0, 0.0);
  if (s != SDP_OK) {
    h->last_error = h->self_batch->last_error;
    return s;
  }
  *its = it[0];
  *rr = r[0];
  return st[0];
}

// Runs fn(i) for every listed problem on its own host thread.
template <typename F>
static void parallel_for(const std::vector<int>& idx, F fn) {
  std::vector<std::thread> th;
  th.reserve(idx.size());
  for (int i : idx) th.emplace_back([&fn, i] { fn(i); });
  for (auto& t : th) t.join();
}

}  // namespace sdpgb

using namespace sdpgb;

extern "C" sdp_status sdp_batch_create(sdp_problem* const* hs, int count, void* cuda_stream, sdp_batch** out) {
  if (!out || count < 0 || (count > 0 && !hs)) return SDP_ERR_ARG;
  *out = nullptr;
  std::string why;
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return SDP_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return SDP_ERR_ARG;
    if (!batch_supported(hs[i], &why)) return SDP_ERR_UNSUPPORTED;
  }
  sdp_batch* b = new sdp_batch();
  if (count > 0) b->hs.assign(hs, hs + count);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return SDP_ERR_CUDA;
  }
  *out = b;
  return SDP_OK;
}

static sdp_status batch_solve_lockstep(sdp_batch* b, sdp_result* results);

// Groups: problems sorted by order, largest first, dealt in a snake (0..G-1,
// G-1..0, ...), so that the group holding the largest problem gets the
// smallest of the next round and the groups carry similar work; each group is a lockstep batch of its own on
// its own stream and host thread.  One group's dense phases then overlap
// another group's batched PCG instead of all problems alternating together
// between latency-bound phases and the throughput-bound PCG.
static sdp_status batch_make_groups(sdp_batch* b, int G) {
  const int N = (int)b->hs.size();
  std::vector<int> order(N);
  for (int i = 0; i < N; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->hs[x]->n > b->hs[y]->n; });
  b->members.assign(G, {});
  for (int t = 0; t < N; ++t) {
    const int r = t % G;
    b->members[((t / G) % 2 == 0) ? r : G - 1 - r].push_back(order[t]);
  }
  for (int g = 0; g < G; ++g) {
    cudaStream_t s = nullptr;
    int lo = 0, hi = 0;   // the PCG of a group runs on its stream: highest priority
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, hi) != cudaSuccess) {
      cudaGetLastError();
      b->last_error = "sdp_batch: stream creation failed";
      return SDP_ERR_CUDA;
    }
    b->child_streams.push_back(s);
    std::vector<sdp_problem*> hs;
    for (int i : b->members[g]) hs.push_back(b->hs[i]);
    sdp_batch* c = nullptr;
    const sdp_status st = sdp_batch_create(hs.data(), (int)hs.size(), s, &c);
    if (st != SDP_OK) {
      b->last_error = "sdp_batch: group creation failed";
      return st;
    }
    c->groups = 1;
    b->child.push_back(c);
  }
  return SDP_OK;
}

extern "C" sdp_status sdp_batch_solve(sdp_batch* b, sdp_result* results) {
  if (!b || b->hs.empty()) return SDP_ERR_ARG;
  const int N = (int)b->hs.size();
  const int G = std::min(N, b->groups > 0 ? b->groups : (N + 1) / 2);
  if (G <= 1) return batch_solve_lockstep(b, results);
  if ((int)b->child.size() != G) {
    for (sdp_batch* c : b->child) sdp_batch_destroy(c);
    for (cudaStream_t s : b->child_streams) cudaStreamDestroy(s);
    b->child.clear();
    b->child_streams.clear();
    SDP_TRY(batch_make_groups(b, G));
  }
  std::vector<std::vector<sdp_result>> res(G);
  std::vector<sdp_status> st(G, SDP_OK);
  std::vector<std::thread> th;
  for (int g = 0; g < G; ++g) {
    res[g].resize(b->members[g].size());
    th.emplace_back([&, g] { st[g] = sdp_batch_solve(b->child[g], res[g].data()); });
  }
  for (auto& t : th) t.join();
  for (double& x : b->stage_s) x = 0.0;
  sdp_status worst = SDP_OK;
  for (int g = 0; g < G; ++g) {
    for (size_t t = 0; t < b->members[g].size(); ++t)
      if (results) results[b->members[g][t]] = res[g][t];
    for (int k = 0; k < 8; ++k)   // seconds: the slowest group; counts: all groups
      b->stage_s[k] = (k < 6) ? std::max(b->stage_s[k], b->child[g]->stage_s[k]) : b->stage_s[k] + b->child[g]->stage_s[k];
    if (st[g] == SDP_ERR_MAXIT && worst == SDP_OK) {
      worst = SDP_ERR_MAXIT;
    } else if (st[g] != SDP_OK && st[g] != SDP_ERR_MAXIT && (worst == SDP_OK || worst == SDP_ERR_MAXIT)) {
      worst = st[g];   // the first hard error wins over an iteration limit
      b->last_error = b->child[g]->last_error;
    }
  }
  return worst;
}

// Member state for a (re)start of problem i.
static void member_reset(sdp_batch* b, int i) {
  b->ms[i] = IpmStepState{};
  b->mst[i] = SDP_OK;
  b->mdone[i] = 0;
  b->mpcg[i] = b->mit[i] = b->mits[i] = 0;
  b->mrr[i] = 0.0;
  b->mstart[i] = std::chrono::duration<double>(std::chrono::steady_clock::now() - b->epoch).count();
  b->mfin[i] = -1.0;
}
static void members_resize(sdp_batch* b) {
  const size_t N = b->hs.size();
  b->ms.resize(N);
  b->mst.resize(N, SDP_OK);
  b->mdone.resize(N, 0);
  b->mpcg.resize(N, 0);
  b->mit.resize(N, 0);
  b->mits.resize(N, 0);
  b->mrr.resize(N, 0.0);
  b->mstart.resize(N, 0.0);
  b->mfin.resize(N, -1.0);
}

// One interior-point iteration of every running member, in lockstep: the dense
// phases of each on its own stream and host thread, the two Newton systems of
// all of them through the batched PCG.  A member leaves the running set when
// its iterate meets the tolerances (state 1), its iteration limit is reached
// (2) or a call fails (3); its finishing time is recorded then.
static sdp_status lockstep_iter(sdp_batch* b) {
  const int N = (int)b->hs.size();
  auto now_s = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - b->epoch).count(); };
  auto tick = std::chrono::steady_clock::now();
  auto lap = [&](int stage) {
    const auto t = std::chrono::steady_clock::now();
    b->stage_s[stage] += std::chrono::duration<double>(t - tick).count();
    tick = t;
  };
  auto fail_check = [&](const std::vector<int>& idx) {
    std::vector<int> ok;
    for (int i : idx) {
      if (b->mst[i] == SDP_OK) {
        ok.push_back(i);
      } else if (!b->mdone[i]) {
        b->mdone[i] = 3;
        b->mfin[i] = now_s();
      }
    }
    return ok;
  };
  std::vector<int> act;
  for (int i = 0; i < N; ++i)
    if (!b->mdone[i]) act.push_back(i);
  if (act.empty()) return SDP_OK;
  std::vector<char> conv(N, 0);
  parallel_for(act, [&](int i) {
    bool d = false;
    b->mst[i] = ipm_phase_a(b->hs[i], &b->ms[i], &d);
    conv[i] = d;
  });
  lap(0);
  std::vector<int> solve;
  for (int i : fail_check(act)) {
    if (conv[i]) b->mdone[i] = 1;
    else if (b->mit[i] < b->hs[i]->prm.ipm_maxit) solve.push_back(i);
    else b->mdone[i] = 2;   // iteration limit
    if (b->mdone[i]) b->mfin[i] = now_s();
  }
  if (solve.empty()) return SDP_OK;
  SDP_TRY(batch_newton(b, solve, b->mits, b->mrr, b->mst));
  lap(1);
  std::vector<int> nxt = fail_check(solve);
  parallel_for(nxt, [&](int i) {
    b->mpcg[i] += b->mits[i];
    b->mst[i] = ipm_phase_b(b->hs[i], &b->ms[i], b->mits[i], b->mrr[i]);
  });
  lap(2);
  std::vector<int> nxt2 = fail_check(nxt);
  SDP_TRY(batch_newton(b, nxt2, b->mits, b->mrr, b->mst));
  lap(3);
  std::vector<int> nxt3 = fail_check(nxt2);
  parallel_for(nxt3, [&](int i) {
    b->mpcg[i] += b->mits[i];
    b->mst[i] = ipm_phase_c(b->hs[i], &b->ms[i], b->mits[i], b->mrr[i]);
    if (b->mst[i] == SDP_OK) b->mit[i]++;
  });
  lap(4);
  fail_check(nxt3);
  return SDP_OK;
}

static sdp_result member_result(const sdp_batch* b, int i) {
  sdp_result r{};
  const IpmStepState& s = b->ms[i];
  r.obj_p = s.inf.obj_p;
  r.obj_d = s.inf.obj_d;
  r.relgap = s.inf.relgap;
  r.pinf = s.inf.pinf;
  r.dinf = s.inf.dinf;
  r.iters = b->hs[i]->iter;
  r.pcg_iters_total = b->mpcg[i];
  r.converged = (b->mdone[i] == 1) ? 1 : 0;
  const double end = (b->mfin[i] >= 0.0) ? b->mfin[i]
                                         : std::chrono::duration<double>(std::chrono::steady_clock::now() - b->epoch).count();
  r.seconds = end - b->mstart[i];   // this member's own time in the batch
  return r;
}

static sdp_status batch_solve_lockstep(sdp_batch* b, sdp_result* results) {
  const int N = (int)b->hs.size();
  members_resize(b);
  for (int i = 0; i < N; ++i) member_reset(b, i);
  for (double& x : b->stage_s) x = 0.0;
  int ipm_maxit = 0;
  for (auto* h : b->hs) ipm_maxit = std::max(ipm_maxit, h->prm.ipm_maxit);
  for (int it = 0; it <= ipm_maxit + 1; ++it) {
    bool any = false;
    for (int i = 0; i < N; ++i) any = any || !b->mdone[i];
    if (!any) break;
    SDP_TRY(lockstep_iter(b));
  }
  sdp_status worst = SDP_OK;
  for (int i = 0; i < N; ++i) {
    const sdp_result r = member_result(b, i);
    if (results) results[i] = r;
    if (b->mst[i] != SDP_OK && worst == SDP_OK) {
      worst = b->mst[i];
      b->last_error = "problem " + std::to_string(i) + ": " + b->hs[i]->last_error;
    }
    if (b->mst[i] == SDP_OK && !r.converged && worst == SDP_OK) worst = SDP_ERR_MAXIT;
  }
  return worst;
}

static int member_index(const sdp_batch* b, const sdp_problem* h) {
  for (size_t i = 0; i < b->hs.size(); ++i)
    if (b->hs[i] == h) return (int)i;
  return -1;
}

extern "C" sdp_status sdp_batch_tuning(const sdp_batch* b, int* spmm_rows, double* ms) {
  if (!b) return SDP_ERR_ARG;
  const sdp_batch* t = b->child.empty() ? b : b->child[0];
  if (spmm_rows) *spmm_rows = t->tuned ? t->spmm_r : 0;
  if (ms)
    for (int c = 0; c < 4; ++c) ms[c] = t->tune_ms[c];
  return SDP_OK;
}

extern "C" sdp_status sdp_batch_add(sdp_batch* b, sdp_problem* h) {
  if (!b || !h || member_index(b, h) >= 0 || !b->child.empty()) return SDP_ERR_ARG;
  std::string why;
  if (!batch_supported(h, &why)) {
    b->last_error = why;
    return SDP_ERR_UNSUPPORTED;
  }
  b->hs.push_back(h);
  members_resize(b);
  member_reset(b, (int)b->hs.size() - 1);
  b->dirty = true;
  return SDP_OK;
}

extern "C" sdp_status sdp_batch_remove(sdp_batch* b, sdp_problem* h) {
  if (!b) return SDP_ERR_ARG;
  const int i = member_index(b, h);
  if (i < 0) return SDP_ERR_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  auto erase = [i](auto& v) { v.erase(v.begin() + i); };
  erase(b->hs);
  erase(b->ms);
  erase(b->mst);
  erase(b->mdone);
  erase(b->mpcg);
  erase(b->mit);
  erase(b->mits);
  erase(b->mrr);
  erase(b->mstart);
  erase(b->mfin);
  b->dirty = true;
  return SDP_OK;
}

extern "C" sdp_status sdp_batch_step(sdp_batch* b, int* running) {
  if (!b || !b->child.empty()) return SDP_ERR_ARG;
  members_resize(b);
  sdp_status s = b->hs.empty() ? SDP_OK : lockstep_iter(b);
  int run = 0;
  for (char d : b->mdone) run += (d == 0);
  if (running) *running = run;
  return s;
}

extern "C" sdp_status sdp_batch_member(const sdp_batch* b, const sdp_problem* h, sdp_result* r, int* state) {
  if (!b) return SDP_ERR_ARG;
  const int i = member_index(b, h);
  if (i < 0 || i >= (int)b->mdone.size()) return SDP_ERR_ARG;
  if (r) *r = member_result(b, i);
  if (state) *state = b->mdone[i];
  return (b->mdone[i] == 3) ? b->mst[i] : SDP_OK;
}

extern "C" const char* sdp_batch_last_error(const sdp_batch* b) { return b ? b->last_error.c_str() : ""; }

extern "C" sdp_status sdp_batch_set_groups(sdp_batch* b, int groups) {
  if (!b || groups < 0) return SDP_ERR_ARG;
  b->groups = groups;
  return SDP_OK;
}

extern "C" sdp_status sdp_batch_stage_seconds(const sdp_batch* b, double* out) {
  if (!b || !out) return SDP_ERR_ARG;
  for (int i = 0; i < 8; ++i) out[i] = b->stage_s[i];
  return SDP_OK;
}

extern "C" void sdp_batch_destroy(sdp_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  pool_free(b->ddesc, b->stream);
  pool_free(b->doff, b->stream);
  pool_free(b->dflag, b->stream);
  for (sdp_batch* c : b->child) sdp_batch_destroy(c);
  for (cudaStream_t s : b->child_streams) cudaStreamDestroy(s);
  delete b;
}
