// sdp_setup and the small handle-level calls of the C ABI.
//
// sdp_setup turns the triplet lists of eq. (SDP) into the device-side sparse
// constraint operator:
//   * CSR pattern of V = sum_i v_i A_i (union of the supports, both triangles)
//     with a gather list slot -> (constraint, coefficient), so assembling V
//     needs no atomics;
//   * the per-constraint list of stored upper entries (p <= q) with the
//     coefficient pre-multiplied by 2 off the diagonal, so A_i . X is a plain sum;
//   * (A^T A)^{-1} = diag(1 / ||A_i||_F^2) after checking that A^T A is diagonal
//     (Assumption 2 in the form the Woodbury apply of eq. SMW2 needs);
//   * the pattern of K_ll' = sum_i g_i (A_i u_l)(A_i u_l')^T used to form the
//     preconditioner core, with its gather list.
#include "internal.cuh"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <unordered_map>

using namespace sdpgb;

namespace sdpgb {

// One pool per device that keeps up to 32 GiB of freed memory: what a finished
// problem frees stays with the pool and the next request reuses it without a
// new mapping, and a free is ordered on the freeing stream -- cudaFree waits
// for all work on the device, so one serving request's clean-up would stall
// every other request's kernels.
static cudaMemPool_t device_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = 32ull << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
  }
  return pools[dev];
}

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  cudaMemPool_t pool = device_pool();
  if (!pool) return cudaMalloc(p, bytes);
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

void pool_free(void* p, cudaStream_t st) {
  if (!p) return;
  if (device_pool()) cudaFreeAsync(p, st);
  else cudaFree(p);
}

}  // namespace sdpgb

sdp_status sdp_problem::alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = pool_malloc(p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    last_error = std::string("device allocation (") + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e);
    *p = nullptr;
    return SDP_ERR_OOM;
  }
  owned.push_back(*p);
  owned_bytes.push_back(bytes);
  device_bytes += (int64_t)bytes;
  return SDP_OK;
}

void sdp_problem::release(void* p) {
  if (!p) return;
  for (size_t i = 0; i < owned.size(); ++i) {
    if (owned[i] != p) continue;
    pool_free(p, stream);
    device_bytes -= (int64_t)owned_bytes[i];
    owned[i] = owned.back();
    owned.pop_back();
    owned_bytes[i] = owned_bytes.back();
    owned_bytes.pop_back();
    return;
  }
}

extern "C" void sdp_default_params(sdp_params* p) {
  if (!p) return;
  p->gap_tol = 1e-6;
  p->infeas_tol = 1e-6;
  p->pcg_rtol = 1e-8;
  p->ipm_maxit = 100;
  p->pcg_maxit = 1000;
  p->refine_maxit = 64;
  p->k = 0;
  p->step_frac = 0.9;
  p->prec = SDP_FP64;
  p->precond = SDP_PRECOND_HAT;
  p->inner_rtol = 1e-9;
  p->verbose = 0;
  p->pcg_graph = 1;
  p->inner_rtol_lp = 1e-4;
  p->wait_cycles = 0;
  p->k_max = 0;
  p->eta = 0.0;
}

extern "C" const char* sdp_status_str(sdp_status s) {
  switch (s) {
    case SDP_OK: return "ok";
    case SDP_ERR_ARG: return "invalid argument";
    case SDP_ERR_OOM: return "out of memory";
    case SDP_ERR_NOT_PD: return "matrix not positive definite";
    case SDP_ERR_MAXIT: return "iteration limit reached";
    case SDP_ERR_UNSUPPORTED: return "unsupported problem structure (A^T A not diagonal)";
    case SDP_ERR_NUMERIC: return "NaN or Inf encountered";
    case SDP_ERR_TIMEOUT: return "bounded device wait expired";
    case SDP_ERR_CUDA: return "CUDA runtime error";
  }
  return "unknown status";
}

extern "C" int64_t sdp_device_bytes(const sdp_problem* h) { return h ? h->device_bytes : -1; }

extern "C" const char* sdp_last_error(const sdp_problem* h) {
  return h ? h->last_error.c_str() : sdpgb::free_call_error();
}

extern "C" void sdp_destroy(sdp_problem* h) {
  if (!h) return;
  if (!h->owned.empty()) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
  }
  if (h->self_batch) sdp_batch_destroy(h->self_batch);
  if (h->pcg_exec) cudaGraphExecDestroy(h->pcg_exec);
  if (h->pcg_graph) cudaGraphDestroy(h->pcg_graph);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  for (void* p : h->owned) pool_free(p, h->stream);
  delete h;
}

template <typename T>
static sdp_status upload(sdp_problem* h, T** dst, const std::vector<T>& src) {
  SDP_TRY(h->allocT(dst, std::max<size_t>(src.size(), 1)));
  if (!src.empty()) SDP_CK(h, cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  return SDP_OK;
}

static inline uint64_t poskey(int i, int j) { return ((uint64_t)(uint32_t)i << 32) | (uint32_t)j; }

static sdp_status build(sdp_problem* h, int64_t nnzC, const int32_t* Ci, const int32_t* Cj, const double* Cv,
                        int64_t nnzA, const int32_t* Ak, const int32_t* Ai, const int32_t* Aj, const double* Av,
                        const double* b) {
  const int n = h->n, m = h->m;
  // ---- merge duplicate A entries, normalise to i <= j, sort by (k, i, j)
  struct Ent { int k, i, j; double v; };
  std::vector<Ent> ent;
  ent.reserve((size_t)nnzA);
  for (int64_t t = 0; t < nnzA; ++t) {
    const int k = Ak[t], i = Ai[t], j = Aj[t];
    if (k < 0 || k >= m || i < 0 || i >= n || j < 0 || j >= n) {
      h->last_error = "sdp_setup: A triplet index out of range at position " + std::to_string(t);
      return SDP_ERR_ARG;
    }
    if (!std::isfinite(Av[t])) {
      h->last_error = "sdp_setup: non-finite A value";
      return SDP_ERR_ARG;
    }
    ent.push_back({k, std::min(i, j), std::max(i, j), Av[t]});
  }
  std::sort(ent.begin(), ent.end(), [](const Ent& a, const Ent& c) {
    if (a.k != c.k) return a.k < c.k;
    if (a.i != c.i) return a.i < c.i;
    return a.j < c.j;
  });
  std::vector<Ent> me;
  for (const Ent& e : ent) {
    if (!me.empty() && me.back().k == e.k && me.back().i == e.i && me.back().j == e.j) me.back().v += e.v;
    else me.push_back(e);
  }
  me.erase(std::remove_if(me.begin(), me.end(), [](const Ent& e) { return e.v == 0.0; }), me.end());

  // ---- per-constraint entries and ||A_i||_F^2
  std::vector<int> eptr(m + 1, 0), ep, eq;
  std::vector<double> ecoef, g(m, 0.0);
  for (const Ent& e : me) {
    eptr[e.k + 1]++;
    ep.push_back(e.i);
    eq.push_back(e.j);
    const double mult = (e.i == e.j) ? 1.0 : 2.0;
    ecoef.push_back(e.v * mult);
    g[e.k] += mult * e.v * e.v;
  }
  for (int k = 0; k < m; ++k) eptr[k + 1] += eptr[k];
  for (int k = 0; k < m; ++k) {
    if (!(g[k] > 0.0)) {
      h->last_error = "sdp_setup: constraint " + std::to_string(k) + " has no nonzero entry";
      return SDP_ERR_ARG;
    }
  }
  // ---- positions -> contributors; A^T A diagonal check
  std::unordered_map<uint64_t, std::vector<std::pair<int, double>>> pos;
  pos.reserve(me.size() * 2);
  for (const Ent& e : me) pos[poskey(e.i, e.j)].push_back({e.k, e.v});
  {
    std::unordered_map<uint64_t, double> offd;
    for (auto& kv : pos) {
      auto& lst = kv.second;
      if (lst.size() < 2) continue;
      const int i = (int)(kv.first >> 32), j = (int)(kv.first & 0xffffffffu);
      const double mult = (i == j) ? 1.0 : 2.0;
      for (size_t a = 0; a < lst.size(); ++a)
        for (size_t c = a + 1; c < lst.size(); ++c) {
          const int k1 = std::min(lst[a].first, lst[c].first), k2 = std::max(lst[a].first, lst[c].first);
          offd[poskey(k1, k2)] += mult * lst[a].second * lst[c].second;
        }
    }
    for (auto& kv : offd) {
      const int k1 = (int)(kv.first >> 32), k2 = (int)(kv.first & 0xffffffffu);
      if (std::fabs(kv.second) > 1e-12 * std::sqrt(g[k1] * g[k2])) {
        h->last_error = "sdp_setup: A^T A is not diagonal (constraints " + std::to_string(k1) + " and " +
                        std::to_string(k2) + ")";
        return SDP_ERR_UNSUPPORTED;
      }
    }
  }
  // ---- CSR pattern of V (both triangles) with gather lists
  std::vector<std::vector<std::pair<int, uint64_t>>> rows(n);   // (col, key of the position)
  for (auto& kv : pos) {
    const int i = (int)(kv.first >> 32), j = (int)(kv.first & 0xffffffffu);
    rows[i].push_back({j, kv.first});
    if (i != j) rows[j].push_back({i, kv.first});
  }
  std::vector<int> rowptr(n + 1, 0), colidx, sptr(1, 0), scon;
  std::vector<double> scoef;
  for (int r = 0; r < n; ++r) {
    std::sort(rows[r].begin(), rows[r].end());
    for (auto& cv : rows[r]) {
      colidx.push_back(cv.first);
      for (auto& kc : pos[cv.second]) {
        scon.push_back(kc.first);
        scoef.push_back(kc.second);
      }
      sptr.push_back((int)scon.size());
    }
    rowptr[r + 1] = (int)colidx.size();
  }
  h->nnzV = (int)colidx.size();
  h->ncontrib = (int)scon.size();
  h->nent = (int)ep.size();

  // ---- support rows of each constraint, per-row entry lists, K pattern
  std::vector<int> crptr(m + 1, 0), crrow, clptr(1, 0), clcol;
  std::vector<double> clcoef;
  std::map<std::pair<int, int>, std::vector<std::array<int, 3>>> kslots;
  for (int k = 0; k < m; ++k) {
    std::vector<int> sup;
    for (int e = eptr[k]; e < eptr[k + 1]; ++e) {
      sup.push_back(ep[e]);
      sup.push_back(eq[e]);
    }
    std::sort(sup.begin(), sup.end());
    sup.erase(std::unique(sup.begin(), sup.end()), sup.end());
    const int base = (int)crrow.size();
    for (int a : sup) {
      crrow.push_back(a);
      // entries of row a of A_k: (b, value)
      for (int e = eptr[k]; e < eptr[k + 1]; ++e) {
        const double v = (ep[e] == eq[e]) ? ecoef[e] : 0.5 * ecoef[e];
        if (ep[e] == a) { clcol.push_back(eq[e]); clcoef.push_back(v); }
        else if (eq[e] == a) { clcol.push_back(ep[e]); clcoef.push_back(v); }
      }
      clptr.push_back((int)clcol.size());
    }
    crptr[k + 1] = (int)crrow.size();
    for (size_t x = 0; x < sup.size(); ++x)
      for (size_t y = 0; y < sup.size(); ++y)
        kslots[{sup[x], sup[y]}].push_back({k, base + (int)x, base + (int)y});
  }
  std::vector<int> krowptr(n + 1, 0), kcol, kptr(1, 0), kcon, kcra, kcrb;
  for (auto& kv : kslots) {
    krowptr[kv.first.first + 1]++;
    kcol.push_back(kv.first.second);
    for (auto& tr : kv.second) {
      kcon.push_back(tr[0]);
      kcra.push_back(tr[1]);
      kcrb.push_back(tr[2]);
    }
    kptr.push_back((int)kcon.size());
  }
  for (int r = 0; r < n; ++r) krowptr[r + 1] += krowptr[r];
  h->ncr = (int)crrow.size();
  h->nnzK = (int)kcol.size();
  h->nkc = (int)kcon.size();
  SchurPlanHost sp;
  schur_plan(n, krowptr, kcol, &sp);
  h->hs_np = (int)sp.pverts.size();
  h->hs_nr = (int)sp.rverts.size();
  h->hs_nb = (int)sp.bcol.size();

  // ---- dense C, b, norms, start point
  std::vector<double> Cd((size_t)n * n, 0.0);
  for (int64_t t = 0; t < nnzC; ++t) {
    const int i = Ci[t], j = Cj[t];
    if (i < 0 || i >= n || j < 0 || j >= n || !std::isfinite(Cv[t])) {
      h->last_error = "sdp_setup: invalid C triplet at position " + std::to_string(t);
      return SDP_ERR_ARG;
    }
    Cd[(size_t)i * n + j] += Cv[t];
    if (i != j) Cd[(size_t)j * n + i] += Cv[t];
  }
  double nC = 0.0, nb = 0.0, bmaxterm = 0.0;
  for (double x : Cd) nC += x * x;
  nC = std::sqrt(nC);
  const double sn = std::sqrt((double)n);
  for (int k = 0; k < m; ++k) {
    if (!std::isfinite(b[k])) {
      h->last_error = "sdp_setup: non-finite b";
      return SDP_ERR_ARG;
    }
    nb += b[k] * b[k];
    bmaxterm = std::max(bmaxterm, sn * (1.0 + std::fabs(b[k])) / (1.0 + std::sqrt(g[k])));
  }
  h->normb = std::sqrt(nb);
  h->normC = nC;
  h->xi = std::max(std::max(10.0, sn), std::max(bmaxterm, (1.0 + nC) / sn));

  std::vector<double> ginv(m);
  for (int k = 0; k < m; ++k) ginv[k] = 1.0 / g[k];

  // rows of V by decreasing length: the SpMM gives consecutive threads of a warp
  // rows of about the same length, so no lane idles while the longest finishes
  std::vector<int> rowperm(n);
  for (int r = 0; r < n; ++r) rowperm[r] = r;
  std::stable_sort(rowperm.begin(), rowperm.end(), [&](int a, int b2) {
    return rowptr[a + 1] - rowptr[a] > rowptr[b2 + 1] - rowptr[b2];
  });
  SDP_TRY(upload(h, &h->rowptr, rowptr));
  SDP_TRY(upload(h, &h->rowperm, rowperm));
  SDP_TRY(upload(h, &h->colidx, colidx));
  SDP_TRY(upload(h, &h->sptr, sptr));
  SDP_TRY(upload(h, &h->scon, scon));
  SDP_TRY(upload(h, &h->scoef, scoef));
  SDP_TRY(upload(h, &h->eptr, eptr));
  SDP_TRY(upload(h, &h->ep, ep));
  SDP_TRY(upload(h, &h->eq, eq));
  SDP_TRY(upload(h, &h->ecoef, ecoef));
  SDP_TRY(upload(h, &h->ginv, ginv));
  SDP_TRY(upload(h, &h->crptr, crptr));
  SDP_TRY(upload(h, &h->crrow, crrow));
  SDP_TRY(upload(h, &h->crlist_ptr, clptr));
  SDP_TRY(upload(h, &h->crlist_col, clcol));
  SDP_TRY(upload(h, &h->crlist_coef, clcoef));
  SDP_TRY(upload(h, &h->krowptr, krowptr));
  SDP_TRY(upload(h, &h->kcol, kcol));
  SDP_TRY(upload(h, &h->kptr, kptr));
  SDP_TRY(upload(h, &h->kcon, kcon));
  SDP_TRY(upload(h, &h->kcra, kcra));
  SDP_TRY(upload(h, &h->kcrb, kcrb));
  SDP_TRY(upload(h, &h->hs_pverts, sp.pverts));
  SDP_TRY(upload(h, &h->hs_rverts, sp.rverts));
  SDP_TRY(upload(h, &h->hs_stype, sp.stype));
  SDP_TRY(upload(h, &h->hs_sa, sp.sa));
  SDP_TRY(upload(h, &h->hs_sb, sp.sb));
  SDP_TRY(upload(h, &h->hs_bptr, sp.bptr));
  SDP_TRY(upload(h, &h->hs_bcol, sp.bcol));
  SDP_TRY(upload(h, &h->hs_bp, sp.bp));
  SDP_TRY(upload(h, &h->hs_btptr, sp.btptr));
  SDP_TRY(upload(h, &h->hs_btslot, sp.btslot));
  SDP_TRY(upload(h, &h->C, Cd));
  std::vector<double> bv(b, b + m);
  SDP_TRY(upload(h, &h->b, bv));

  const size_t nn = (size_t)n * n;
  SDP_TRY(h->allocT(&h->X, nn));
  SDP_TRY(h->allocT(&h->S, nn));
  SDP_TRY(h->allocT(&h->W, nn));
  SDP_TRY(h->allocT(&h->y, m));
  SDP_TRY(h->allocT(&h->T, nn));
  SDP_TRY(h->allocT(&h->Vval, std::max(h->nnzV, 1)));
  SDP_CK(h, cudaMemsetAsync(h->y, 0, m * sizeof(double), h->stream));
  fill(h->stream, h->X, nn, 0.0);
  add_diag(h->stream, n, h->X, n, h->xi);
  fill(h->stream, h->S, nn, 0.0);
  add_diag(h->stream, n, h->S, n, h->xi);
  SDP_CK(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
  SDP_CK(h, cudaStreamSynchronize(h->stream));
  return SDP_OK;
}

extern "C" sdp_status sdp_setup(int n, int m, int64_t nnzC, const int32_t* Ci, const int32_t* Cj,
                                const double* Cv, int64_t nnzA, const int32_t* Ak, const int32_t* Ai,
                                const int32_t* Aj, const double* Av, const double* b, int k,
                                const sdp_params* prm, void* cuda_stream, sdp_problem** out) {
  if (!out) return SDP_ERR_ARG;
  *out = nullptr;
  if (n < 1 || m < 1 || k < 0 || k > n || nnzC < 0 || nnzA < 1 || !b) return SDP_ERR_ARG;
  if (nnzC > 0 && (!Ci || !Cj || !Cv)) return SDP_ERR_ARG;
  if (!Ak || !Ai || !Aj || !Av) return SDP_ERR_ARG;
  if (n > 46000) return SDP_ERR_ARG;
  sdp_problem* h = new (std::nothrow) sdp_problem();
  if (!h) return SDP_ERR_OOM;
  h->n = n;
  h->m = m;
  if (prm) h->prm = *prm;
  else sdp_default_params(&h->prm);
  h->k = (h->prm.k > 0) ? std::min(h->prm.k, n) : k;
  if (h->k > SDP_K_MAX || h->prm.k_max < 0 || h->prm.k_max > SDP_K_MAX || !(h->prm.eta >= 0.0)) {
    delete h;
    return SDP_ERR_ARG;
  }
  // the adaptive rule (eta > 0) picks the split rank per build, up to k_max (or k)
  h->kcap = (h->prm.eta > 0.0 && h->prm.k_max > 0) ? h->prm.k_max : h->k;
  h->kcap = std::max(0, std::min(h->kcap, n - 1));
  h->stream = (cudaStream_t)cuda_stream;
  h->launches_at_setup = g_launches.load();
  sdp_status s = build(h, nnzC, Ci, Cj, Cv, nnzA, Ak, Ai, Aj, Av, b);
  if (s != SDP_OK) {
    fprintf(stderr, "sdp_setup: %s\n", h->last_error.c_str());
    sdp_destroy(h);
    return s;
  }
  *out = h;
  return SDP_OK;
}

extern "C" sdp_status sdp_set_W(sdp_problem* h, const double* W_dev) {
  if (!h || !W_dev) return SDP_ERR_ARG;
  SDP_CK(h, cudaMemcpyAsync(h->W, W_dev, (size_t)h->n * h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  h->have_W = true;
  h->W32_valid = h->W16_valid = false;
  h->pc_valid = false;
  return SDP_OK;
}

extern "C" sdp_status sdp_get_W(sdp_problem* h, double* W_dev) {
  if (!h || !W_dev || !h->have_W) return SDP_ERR_ARG;
  SDP_CK(h, cudaMemcpyAsync(W_dev, h->W, (size_t)h->n * h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  return SDP_OK;
}

extern "C" sdp_status sdp_get_solution(sdp_problem* h, double* X_host, double* y_host, double* S_host) {
  if (!h) return SDP_ERR_ARG;
  const size_t nn = (size_t)h->n * h->n;
  if (X_host) SDP_CK(h, cudaMemcpyAsync(X_host, h->X, nn * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (y_host) SDP_CK(h, cudaMemcpyAsync(y_host, h->y, h->m * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (S_host) SDP_CK(h, cudaMemcpyAsync(S_host, h->S, nn * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  SDP_CK(h, cudaStreamSynchronize(h->stream));
  return SDP_OK;
}

extern "C" sdp_status sdp_set_state(sdp_problem* h, const double* X_host, const double* y_host,
                                    const double* S_host, int iter) {
  if (!h || !X_host || !y_host || !S_host || iter < 0) return SDP_ERR_ARG;
  const size_t nn = (size_t)h->n * h->n;
  SDP_CK(h, cudaMemcpyAsync(h->X, X_host, nn * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  SDP_CK(h, cudaMemcpyAsync(h->y, y_host, h->m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  SDP_CK(h, cudaMemcpyAsync(h->S, S_host, nn * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  SDP_CK(h, cudaStreamSynchronize(h->stream));
  h->iter = iter;
  h->chol_valid = false;
  h->pc_valid = false;
  return SDP_OK;
}

extern "C" sdp_status sdp_get_state(sdp_problem* h, double* X_host, double* y_host, double* S_host, int* iter) {
  if (!h) return SDP_ERR_ARG;
  SDP_TRY(sdp_get_solution(h, X_host, y_host, S_host));
  if (iter) *iter = h->iter;
  return SDP_OK;
}

extern "C" sdp_status sdp_sizes(const sdp_problem* h, int* n, int* m, int* k, int64_t* nnzV) {
  if (!h) return SDP_ERR_ARG;
  if (n) *n = h->n;
  if (m) *m = h->m;
  if (k) *k = h->k;
  if (nnzV) *nnzV = h->nnzV;
  return SDP_OK;
}

extern "C" int64_t sdp_launch_count(const sdp_problem* h) {
  (void)h;
  return g_launches.load();
}

extern "C" sdp_status sdp_precond_info(sdp_problem* h, double* tau, int* k) {
  if (!h) return SDP_ERR_ARG;
  if (!h->pc_valid) return SDP_ERR_ARG;
  if (tau) *tau = h->tau;
  if (k) *k = h->kpc;
  return SDP_OK;
}

// ---- thin wrappers over the implementations in the other translation units
extern "C" sdp_status sdp_hessian_matvec(sdp_problem* h, const double* v_dev, double* Hv_dev, int prec) {
  if (!h || !v_dev || !Hv_dev) return SDP_ERR_ARG;
  sdp_status s = matvec_impl(h, v_dev, Hv_dev, prec);
  if (s != SDP_OK) return s;
  SDP_CK(h, cudaGetLastError());
  return SDP_OK;
}

extern "C" sdp_status sdp_precond_build(sdp_problem* h) {
  if (!h) return SDP_ERR_ARG;
  if (!h->have_W) {
    h->last_error = "precond_build: no scaling matrix W";
    return SDP_ERR_ARG;
  }
  sdp_status s = precond_build_impl(h);
  if (s != SDP_OK) return s;
  SDP_CK(h, cudaGetLastError());
  return SDP_OK;
}

extern "C" sdp_status sdp_precond_apply(sdp_problem* h, const double* r_dev, double* z_dev, int prec) {
  if (!h || !r_dev || !z_dev) return SDP_ERR_ARG;
  if (!h->pc_valid) {
    h->last_error = "precond_apply: call sdp_precond_build first";
    return SDP_ERR_ARG;
  }
  sdp_status s = precond_apply_impl(h, r_dev, z_dev, prec);
  if (s != SDP_OK) return s;
  SDP_CK(h, cudaGetLastError());
  return SDP_OK;
}

extern "C" sdp_status sdp_pcg_solve(sdp_problem* h, const double* r_dev, double* y_dev, double rtol, int maxit,
                                    int prec, int* iters, double* relres) {
  if (!h || !r_dev || !y_dev || maxit < 1 || !(rtol >= 0.0)) return SDP_ERR_ARG;
  if (!h->pc_valid) {
    sdp_status s = sdp_precond_build(h);
    if (s != SDP_OK) return s;
  }
  return pcg_impl(h, r_dev, y_dev, rtol, maxit, prec, iters, relres);
}

extern "C" sdp_status sdp_ipm_step(sdp_problem* h, sdp_ipm_info* info) {
  if (!h) return SDP_ERR_ARG;
  return ipm_step_impl(h, info);
}

extern "C" sdp_status sdp_reset(sdp_problem* h) {
  if (!h) return SDP_ERR_ARG;
  const size_t nn = (size_t)h->n * h->n;
  fill(h->stream, h->X, nn, 0.0);
  add_diag(h->stream, h->n, h->X, h->n, h->xi);
  fill(h->stream, h->S, nn, 0.0);
  add_diag(h->stream, h->n, h->S, h->n, h->xi);
  SDP_CK(h, cudaMemsetAsync(h->y, 0, h->m * sizeof(double), h->stream));
  h->iter = 0;
  h->chol_valid = false;
  h->have_W = false;
  h->pc_valid = false;
  h->W32_valid = h->W16_valid = false;
  return SDP_OK;
}
