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
  std::map<std::string, std::pair<long long, double>> collected;  // graph replays: launches, ms
  std::vector<std::string> select;   // kernels to time (empty: all)
  std::atomic<long long> config{0};  // changes with the timing switch and the selection
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

// The graph being captured on this thread (its timing events), if any.
thread_local std::vector<ProfEvent>* t_capture = nullptr;
thread_local std::vector<cudaEvent_t> t_capture_open;

static bool selected(Profiler& p, const char* name) {
  if (p.select.empty()) return true;
  for (const auto& s : p.select)
    if (s == name) return true;
  return false;
}

bool prof_begin(const char* name, cudaStream_t st) {
  Profiler& p = P();
  p.launches.fetch_add(1);
  if (!p.on.load()) return false;
  {
    std::lock_guard<std::mutex> g(p.mu);
    if (!selected(p, name)) return false;
  }
  if (t_capture) {  // an event-record node of the graph, re-recorded at every replay
    cudaEvent_t a = nullptr;
    cudaEventCreate(&a);
    cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);
    t_capture->push_back({name, a, nullptr});
    t_capture_open.push_back(a);
    return true;
  }
  std::lock_guard<std::mutex> g(p.mu);
  cudaEvent_t a = p.take();
  cudaEventRecord(a, st);
  p.open_names.push_back(name);
  p.open_events.push_back(a);
  return true;
}

void prof_end(cudaStream_t st) {
  Profiler& p = P();
  if (!p.on.load()) return;
  if (t_capture) {
    if (t_capture_open.empty()) return;
    cudaEvent_t b = nullptr;
    cudaEventCreate(&b);
    cudaEventRecordWithFlags(b, st, cudaEventRecordExternal);
    const cudaEvent_t a = t_capture_open.back();
    t_capture_open.pop_back();
    for (auto it = t_capture->rbegin(); it != t_capture->rend(); ++it)
      if (it->a == a) { it->b = b; break; }
    return;
  }
  std::lock_guard<std::mutex> g(p.mu);
  if (p.open_events.empty()) return;
  cudaEvent_t b = p.take();
  cudaEventRecord(b, st);
  p.recs.push_back({p.open_names.back(), p.open_events.back(), b});
  p.open_names.pop_back();
  p.open_events.pop_back();
}

bool prof_timing_on() { return P().on.load(); }
long long prof_config() { return P().config.load(); }

void prof_capture_begin(std::vector<ProfEvent>* events) {
  t_capture = events;
  t_capture_open.clear();
}
void prof_capture_end() {
  t_capture = nullptr;
  t_capture_open.clear();
}
void prof_graph_collect(const std::vector<ProfEvent>& events) {
  Profiler& p = P();
  if (!p.on.load()) return;
  std::lock_guard<std::mutex> g(p.mu);
  for (const auto& e : events) {
    if (!e.a || !e.b) continue;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) != cudaSuccess) { cudaGetLastError(); continue; }
    auto& x = p.collected[e.name];
    x.first += 1;
    x.second += ms;
  }
}
void prof_events_free(std::vector<ProfEvent>& events) {
  for (auto& e : events) {
    if (e.a) cudaEventDestroy(e.a);
    if (e.b) cudaEventDestroy(e.b);
  }
  events.clear();
}
long long prof_launches() { return P().launches.load(); }
void prof_add_launches(long long k) { P().launches.fetch_add(k); }

// FP32 FMA throughput: every thread runs kFmaChains independent chains
// a <- a * m + c (m, c kernel arguments, so nothing folds), kFmaUnroll FMAs per
// chain per iteration; the sum is stored only when it equals a sentinel that
// the chains never reach, which keeps the work alive.
constexpr int kFmaChains = 8, kFmaUnroll = 16, kFmaThreads = 512;
__global__ void __launch_bounds__(kFmaThreads) fma_rate(int iters, float m, float c, float* __restrict__ sink) {
  float a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kFmaUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kFmaChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += a[k];
  if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

}  // namespace mlip

extern "C" {

// Enable (1) or disable (0) per-kernel event timing; clears earlier records.
int mlip_profile_enable(int on) {
  using namespace mlip;
  Profiler& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  for (auto& r : p.recs) { p.pool.push_back(r.a); p.pool.push_back(r.b); }
  p.recs.clear();
  p.collected.clear();
  if (p.on.load() != (on != 0)) p.config.fetch_add(1);
  p.on.store(on != 0);
  return MLIP_OK;
}

// Time only the kernels named in the comma-separated list (NULL or "": all).
int mlip_profile_select(const char* names) {
  using namespace mlip;
  Profiler& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  std::vector<std::string> sel;
  if (names) {
    std::string cur;
    for (const char* c = names;; ++c) {
      if (*c == ',' || *c == 0) {
        if (!cur.empty()) sel.push_back(cur);
        cur.clear();
        if (*c == 0) break;
      } else if (*c != ' ') {
        cur.push_back(*c);
      }
    }
  }
  if (sel != p.select) p.config.fetch_add(1);
  p.select = sel;
  return MLIP_OK;
}

long long mlip_launch_count(void) { return mlip::P().launches.load(); }

int mlip_fp32_fma_rate(int iters, double* tflops, double* ms, int* sms) {
  using namespace mlip;
  if (!tflops || iters < 1) { set_error("fp32 rate: null result or iters < 1"); return MLIP_ERR_INVALID_ARG; }
  int dev = 0, nsm = 0;
  MLIP_CUDA_TRY(cudaGetDevice(&dev));
  MLIP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int per_sm = 0;
  MLIP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate, kFmaThreads, 0));
  if (per_sm < 1) per_sm = 1;
  const int blocks = nsm * per_sm;
  float* sink = nullptr;
  MLIP_CUDA_TRY(cudaMalloc(&sink, sizeof(float) * blocks));
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  fma_rate<<<blocks, kFmaThreads>>>(iters / 8 + 1, 0.999999f, 1e-6f, sink);  // warm-up (clocks, code)
  cudaEventRecord(a);
  fma_rate<<<blocks, kFmaThreads>>>(iters, 0.999999f, 1e-6f, sink);
  cudaEventRecord(b);
  const cudaError_t e = cudaEventSynchronize(b);
  float t = 0.0f;
  if (e == cudaSuccess) cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || t <= 0.0f) {
    set_error("fp32 rate: kernel failed: %s", cudaGetErrorString(e));
    return MLIP_ERR_CUDA;
  }
  const double flop = 2.0 * kFmaChains * kFmaUnroll * (double)iters * blocks * kFmaThreads;
  *tflops = flop / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  if (sms) *sms = nsm;
  return MLIP_OK;
}

// JSON {"kernels": {"name": [launches, total_ms], ...}} of the records since
// the last mlip_profile_enable; synchronises on the recorded events.
int mlip_profile_report(char* buf, long long cap, long long* needed) {
  using namespace mlip;
  Profiler& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  std::map<std::string, std::pair<long long, double>> agg = p.collected;
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
