// Event timing of one kernel class, used by the benchmark to measure the
// dominant kernel's device time inside a full solve.  Events come from a
// recycled pool; nothing is recorded unless a class is enabled.
#include "internal.cuh"

#include <cstring>
#include <string>
#include <vector>

namespace sdpgb {

namespace {
struct Pending {
  cudaEvent_t a, b;
  double flops, bytes;
};
std::string g_cls;
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
cudaEvent_t g_open = nullptr;
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

bool ktimer_on(const char* cls) { return !g_cls.empty() && g_cls == cls; }

void ktimer_begin(cudaStream_t st, const char* cls) {
  if (!ktimer_on(cls)) return;
  g_open = take();
  cudaEventRecord(g_open, st);
}

void ktimer_end(cudaStream_t st, const char* cls, double flops, double bytes) {
  if (!ktimer_on(cls) || !g_open) return;
  cudaEvent_t b = take();
  cudaEventRecord(b, st);
  g_pending.push_back({g_open, b, flops, bytes});
  g_open = nullptr;
  if (g_pending.size() > 4096) drain();
}

void ktimer_set(const char* cls) {
  drain();
  g_cls = cls ? cls : "";
}

void ktimer_read(double* ms, int64_t* launches, double* flops, double* bytes) {
  drain();
  if (ms) *ms = g_ms;
  if (launches) *launches = g_count;
  if (flops) *flops = g_flops;
  if (bytes) *bytes = g_bytes;
  g_ms = g_flops = g_bytes = 0;
  g_count = 0;
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
