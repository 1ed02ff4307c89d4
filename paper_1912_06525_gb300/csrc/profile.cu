// Launch counter and CUDA-event profiler of tagged kernels.  The profiler
// records an event pair on the launching stream around each tagged launch;
// katz_profile_read synchronises and sums the elapsed times per tag together
// with the algorithmic bytes the launcher reports.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace katz {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(); }

// Host-side fault injection: after g_fail_after more device allocations the
// next one fails (no CUDA call is made for it); -1 = off.
static std::atomic<int64_t> g_fail_after{-1};
bool alloc_fault() {
  int64_t v = g_fail_after.load();
  while (v >= 0) {
    if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}

namespace {
struct Rec {
  std::string tag;
  cudaEvent_t a, b;
  double bytes;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
cudaEvent_t g_pending = nullptr;
std::vector<cudaEvent_t> g_pool;
struct Agg {
  int64_t launches = 0;
  double ms = 0, bytes = 0;
};
std::map<std::string, Agg> g_agg;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  KATZ_CUDA(cudaEventCreate(&e));
  return e;
}

void drain() {  // fold finished records into the aggregate
  for (auto& r : g_recs) {
    KATZ_CUDA(cudaEventSynchronize(r.b));
    float ms = 0;
    KATZ_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    Agg& a = g_agg[r.tag];
    a.launches += 1;
    a.ms += ms;
    a.bytes += r.bytes;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}
}  // namespace

bool profiling() { return g_on; }

void prof_begin(cudaStream_t s) {
  if (!g_on) return;
  std::lock_guard<std::mutex> l(g_mu);
  g_pending = take_event();
  KATZ_CUDA(cudaEventRecord(g_pending, s));
}

void prof_end(const char* tag, double alg_bytes, cudaStream_t s) {
  if (!g_on) return;
  std::lock_guard<std::mutex> l(g_mu);
  cudaEvent_t b = take_event();
  KATZ_CUDA(cudaEventRecord(b, s));
  g_recs.push_back({tag, g_pending, b, alg_bytes});
  if (g_recs.size() > 4096) drain();
}

}  // namespace katz

extern "C" {

int64_t katz_launch_count(void) { return katz::launch_count(); }

int katz_fault_inject_alloc(int64_t after) {
  katz::g_fail_after.store(after < 0 ? -1 : after);
  return KATZ_OK;
}

int katz_profile_enable(int32_t on) {
  try {
    std::lock_guard<std::mutex> l(katz::g_mu);
    katz::drain();
    katz::g_agg.clear();
    katz::g_on = on != 0;
    return KATZ_OK;
  } catch (const katz::Error& e) {
    return e.code;
  }
}

int katz_profile_read(const char* tag, int64_t* launches, double* total_ms, double* alg_bytes) {
  try {
    std::lock_guard<std::mutex> l(katz::g_mu);
    katz::drain();
    auto it = katz::g_agg.find(tag ? tag : "");
    const katz::Agg a = it == katz::g_agg.end() ? katz::Agg{} : it->second;
    if (launches) *launches = a.launches;
    if (total_ms) *total_ms = a.ms;
    if (alg_bytes) *alg_bytes = a.bytes;
    return KATZ_OK;
  } catch (const katz::Error& e) {
    return e.code;
  }
}

}  // extern "C"
