// Launch counter and per-kernel event timing (see profile.cuh).
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mlip_internal.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

struct Rec {
  const char* name;
  cudaEvent_t a, b;
};

struct Profiler {
  std::mutex mu;
  std::atomic<bool> on{false};
  std::atomic<long long> launches{0};
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  std::vector<const char*> open_names;
  std::vector<cudaEvent_t> open_events;
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

Profiler& P() {
  static Profiler* p = new Profiler();
  return *p;
}

}  // namespace

void prof_begin(const char* name, cudaStream_t st) {
  Profiler& p = P();
  p.launches.fetch_add(1);
  if (!p.on.load()) return;
  std::lock_guard<std::mutex> g(p.mu);
  cudaEvent_t a = p.take();
  cudaEventRecord(a, st);
  p.open_names.push_back(name);
  p.open_events.push_back(a);
}

void prof_end(cudaStream_t st) {
  Profiler& p = P();
  if (!p.on.load()) return;
  std::lock_guard<std::mutex> g(p.mu);
  if (p.open_events.empty()) return;
  cudaEvent_t b = p.take();
  cudaEventRecord(b, st);
  p.recs.push_back({p.open_names.back(), p.open_events.back(), b});
  p.open_names.pop_back();
  p.open_events.pop_back();
}

bool prof_timing_on() { return P().on.load(); }
long long prof_launches() { return P().launches.load(); }
void prof_add_launches(long long k) { P().launches.fetch_add(k); }

}  // namespace mlip

extern "C" {

// Enable (1) or disable (0) per-kernel event timing; clears earlier records.
int mlip_profile_enable(int on) {
  using namespace mlip;
  Profiler& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  for (auto& r : p.recs) { p.pool.push_back(r.a); p.pool.push_back(r.b); }
  p.recs.clear();
  p.on.store(on != 0);
  return MLIP_OK;
}

long long mlip_launch_count(void) { return mlip::P().launches.load(); }

// JSON {"kernels": {"name": [launches, total_ms], ...}} of the records since
// the last mlip_profile_enable; synchronises on the recorded events.
int mlip_profile_report(char* buf, long long cap, long long* needed) {
  using namespace mlip;
  Profiler& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  std::map<std::string, std::pair<long long, double>> agg;
  for (auto& r : p.recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) { set_error("profile: event sync failed"); return MLIP_ERR_CUDA; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& x = agg[r.name];
    x.first += 1;
    x.second += ms;
  }
  std::string s = "{\"kernels\": {";
  bool first = true;
  for (auto& kv : agg) {
    char tmp[256];
    snprintf(tmp, sizeof(tmp), "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(), kv.second.first,
             kv.second.second);
    s += tmp;
    first = false;
  }
  s += "}}";
  if (needed) *needed = (long long)s.size() + 1;
  if (buf && cap > 0) {
    size_t n = std::min<size_t>((size_t)cap - 1, s.size());
    memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return MLIP_OK;
}

}  // extern "C"
