// Instrumentation (see profile.cuh) and its C-ABI.
#include "common.cuh"
#include "profile.cuh"

#include <atomic>
#include <mutex>
#include <vector>

namespace ld {

namespace {
struct Rec {
  cudaEvent_t a, b;
  int cls;
  double flops, bytes;
  bool done;
};
std::atomic<long long> g_launches{0};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void prof_count() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void prof_add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool prof_enabled() { return g_on.load(std::memory_order_relaxed); }

int prof_begin(cudaStream_t s) {
  if (!prof_enabled()) return -1;
  // A stream being captured into a graph takes no timing events.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{};
  r.a = get_event();
  r.b = get_event();
  r.done = false;
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_end(int token, KClass c, cudaStream_t s, double flops, double bytes) {
  if (token < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (token >= (int)g_recs.size()) return;
  Rec& r = g_recs[token];
  r.cls = c;
  r.flops = flops;
  r.bytes = bytes;
  r.done = true;
  cudaEventRecord(r.b, s);
}

}  // namespace ld

using namespace ld;

extern "C" {

int logdet_profile_enable(int on) {
  g_on.store(on != 0);
  return LOGDET_OK;
}

int logdet_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  return LOGDET_OK;
}

int logdet_profile_read(int32_t kclass, int64_t* launches, double* device_ms, double* flops,
                        double* bytes) {
  if (kclass < 0 || kclass >= KC_COUNT) {
    set_error("profile class %d out of range", kclass);
    return LOGDET_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t n = 0;
  double ms = 0.0, f = 0.0, b = 0.0;
  for (auto& r : g_recs) {
    if (!r.done || r.cls != kclass) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) {
      set_error("profile event synchronize failed");
      return LOGDET_ECUDA;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    ms += t;
    f += r.flops;
    b += r.bytes;
    ++n;
  }
  if (launches) *launches = n;
  if (device_ms) *device_ms = ms;
  if (flops) *flops = f;
  if (bytes) *bytes = b;
  return LOGDET_OK;
}

int64_t logdet_launch_count(void) { return g_launches.load(); }

}  // extern "C"
