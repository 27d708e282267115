// Event timing of one kernel class, used by the benchmark to measure the
// dominant kernel's device time inside a full solve.  Events come from a
// recycled pool; nothing is recorded unless a class is enabled.
#include "internal.cuh"

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace sdpgb {

namespace {
struct Pending {
  cudaEvent_t a, b;
  double flops, bytes;
};
std::mutex g_mu;
std::string g_cls;
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
double g_ms = 0, g_flops = 0, g_bytes = 0;
int64_t g_count = 0;

cudaEvent_t take() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void drain() {
  for (auto& p : g_pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.b);
    cudaEventElapsedTime(&ms, p.a, p.b);
    g_ms += ms;
    g_flops += p.flops;
    g_bytes += p.bytes;
    g_count++;
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}
}  // namespace

thread_local bool g_paused = false;   // per host thread: set while this thread captures a graph
bool ktimer_on(const char* cls) { return !g_paused && !g_cls.empty() && g_cls == cls; }
void ktimer_pause(bool paused) { g_paused = paused; }

// One open event per thread: launches of a class are not nested.
thread_local cudaEvent_t t_open = nullptr;

void ktimer_begin(cudaStream_t st, const char* cls) {
  if (!ktimer_on(cls)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  t_open = take();
  cudaEventRecord(t_open, st);
}

void ktimer_end(cudaStream_t st, const char* cls, double flops, double bytes) {
  if (!ktimer_on(cls) || !t_open) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take();
  cudaEventRecord(b, st);
  g_pending.push_back({t_open, b, flops, bytes});
  t_open = nullptr;
  if (g_pending.size() > 4096) drain();
}

void ktimer_set(const char* cls) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  g_cls = cls ? cls : "";
}

void ktimer_read(double* ms, int64_t* launches, double* flops, double* bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  if (ms) *ms = g_ms;
  if (launches) *launches = g_count;
  if (flops) *flops = g_flops;
  if (bytes) *bytes = g_bytes;
  g_ms = g_flops = g_bytes = 0;
  g_count = 0;
}

void allow_max_smem(const void* func) {
  static std::mutex mu;
  static std::vector<const void*> done;
  std::lock_guard<std::mutex> lk(mu);
  for (const void* f : done)
    if (f == func) return;
  int dev = 0, mx = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, func);
  // the limit covers dynamic memory only; static shared memory counts against the same per-CTA total
  cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
  cudaGetLastError();
  done.push_back(func);
}

}  // namespace sdpgb

extern "C" sdp_status sdp_timing_enable(sdp_problem* h, const char* cls) {
  if (!h) return SDP_ERR_ARG;
  sdpgb::ktimer_set(cls);
  return SDP_OK;
}

extern "C" sdp_status sdp_timing_read(sdp_problem* h, double* ms, int64_t* launches, double* flops, double* bytes) {
  if (!h) return SDP_ERR_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  sdpgb::ktimer_read(ms, launches, flops, bytes);
  return SDP_OK;
}
