// Event timing of one kernel class, used by the benchmark to measure the
// dominant kernel's device time inside a full solve.  Events come from a
// recycled pool; nothing is recorded unless a class is enabled.
#include "internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace sdpgb {

namespace {
struct Pending {
  cudaEvent_t a, b;
  double flops, bytes;
  const char* cls;
};
struct Acc {
  double ms = 0, flops = 0, bytes = 0;
  int64_t count = 0;
};
std::mutex g_mu;
std::string g_cls;                  // recorded class, or "*" for every class
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
std::map<std::string, Acc> g_acc;   // per class

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
    Acc& a = g_acc[p.cls];
    a.ms += ms;
    a.flops += p.flops;
    a.bytes += p.bytes;
    a.count++;
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}
}  // namespace

// per host thread: set while this thread captures a graph
thread_local bool g_paused = false;
bool ktimer_on(const char* cls) { return !g_paused && !g_cls.empty() && (g_cls == "*" || g_cls == cls); }
void ktimer_pause(bool paused) { g_paused = paused; }

// Open regions of this thread (classes may nest when every class is recorded).
thread_local std::vector<std::pair<const char*, cudaEvent_t>> t_open;

void ktimer_begin(cudaStream_t st, const char* cls) {
  if (!ktimer_on(cls)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t e = take();
  cudaEventRecord(e, st);
  t_open.push_back({cls, e});
}

void ktimer_end(cudaStream_t st, const char* cls, double flops, double bytes) {
  if (!ktimer_on(cls) || t_open.empty()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto top = t_open.back();
  t_open.pop_back();
  cudaEvent_t b = take();
  cudaEventRecord(b, st);
  g_pending.push_back({top.second, b, flops, bytes, cls});
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
  Acc t;
  for (auto& kv : g_acc) {
    if (g_cls == "*" || kv.first == g_cls) {
      t.ms += kv.second.ms;
      t.flops += kv.second.flops;
      t.bytes += kv.second.bytes;
      t.count += kv.second.count;
    }
  }
  if (ms) *ms = t.ms;
  if (launches) *launches = t.count;
  if (flops) *flops = t.flops;
  if (bytes) *bytes = t.bytes;
  g_acc.clear();
}

// "class ms launches flops bytes" per line, then clears the accumulators
size_t ktimer_report(char* buf, size_t len) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  std::string s;
  char line[256];
  for (auto& kv : g_acc) {
    snprintf(line, sizeof(line), "%s %.6f %lld %.6e %.6e\n", kv.first.c_str(), kv.second.ms,
             (long long)kv.second.count, kv.second.flops, kv.second.bytes);
    s += line;
  }
  g_acc.clear();
  if (buf && len > 0) {
    const size_t c = std::min(len - 1, s.size());
    memcpy(buf, s.data(), c);
    buf[c] = 0;
  }
  return s.size() + 1;
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

extern "C" int64_t sdp_timing_report(sdp_problem* h, char* buf, int64_t len) {
  if (!h) return -1;
  if (h->stream) cudaStreamSynchronize(h->stream);
  return (int64_t)sdpgb::ktimer_report(buf, len > 0 ? (size_t)len : 0);
}

extern "C" sdp_status sdp_timing_read(sdp_problem* h, double* ms, int64_t* launches, double* flops, double* bytes) {
  if (!h) return SDP_ERR_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  sdpgb::ktimer_read(ms, launches, flops, bytes);
  return SDP_OK;
}
