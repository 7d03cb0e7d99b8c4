// Launch accounting and optional per-kernel timing with CUDA events.
// Every kernel launch of the library goes through a ProfScope: it counts the
// launch and, when timing is enabled, records an event pair on the launching
// stream.  Reports aggregate (launches, total ms) per kernel name.
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace mlip {

// prof_begin returns whether the launch is timed (then prof_end closes it).
bool prof_begin(const char* name, cudaStream_t st);
void prof_end(cudaStream_t st);
// Whether per-kernel event timing is on (graph capture is skipped then: the
// timing events need eager launches).
bool prof_timing_on();
// Changes whenever timing is switched or the timed kernels are selected anew
// (a captured graph holds the timing events of the configuration it saw).
long long prof_config();
// Launch counter: its value, and launches replayed by a CUDA graph.
long long prof_launches();
void prof_add_launches(long long k);
// Timing inside CUDA graphs: while a capture on this thread is bracketed by
// prof_capture_begin/end (timing on), every timed launch adds a pair of
// event-record nodes to the graph; after a replay has completed,
// prof_graph_collect adds the pairs' durations to the report.
struct ProfEvent {
  const char* name;
  cudaEvent_t a, b;
};
void prof_capture_begin(std::vector<ProfEvent>* events);
void prof_capture_end();
void prof_graph_collect(const std::vector<ProfEvent>& events);
void prof_events_free(std::vector<ProfEvent>& events);

struct ProfScope {
  cudaStream_t st;
  bool timed;
  ProfScope(const char* name, cudaStream_t s) : st(s), timed(prof_begin(name, s)) {}
  ~ProfScope() {
    if (timed) prof_end(st);
  }
};

}  // namespace mlip

#define MLIP_PROF(name, st) ::mlip::ProfScope mlip_prof_scope__(name, st)
