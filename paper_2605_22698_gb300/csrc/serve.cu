// Serving: continuous batching of energy+forces and NVE requests on one GPU.
//
// One worker thread owns a CUDA stream.  Every iteration it
//   1. admits queued requests (FIFO) while the batch stays within max_slots
//      and the device-memory budget, and compacts the device state of the
//      running requests into a fresh arena when the membership changed
//      (one gather kernel; new requests arrive through one pinned H2D copy);
//   2. applies the first half kick and the drift to the NVE requests past
//      their first evaluation;
//   3. evaluates every running request as one graph (the disjoint union of
//      the systems' neighbour graphs); a batch of NVE requests whose members
//      stay the same keeps a skin neighbour list on the device between
//      iterations (compacted every step, rebuilt when an atom leaves its skin);
//   4. applies the second half kick, sums per-system kinetic energies, copies
//      back per-system energies and the outputs of the requests that end;
//   5. ends finished requests (t_done) and wakes their waiters.
// Latency statistics come from the host clock of each request's submit
// (t_arrive), admission (t_admit) and end (t_done).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "launchers.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

constexpr double kBoltzmann = 8.617333262e-5;  // eV/K
constexpr double kKappaMD = 9.648533212e-3;    // eV/A/amu -> A/fs^2

// SplitMix64 (Steele, Lea and Flood 2014): state advances by the golden-ratio
// increment; each output is the mixed state.  Doubles in [0,1) from the top
// 53 bits; normals by Box-Muller from pairs of uniforms.
struct SplitMix64 {
  uint64_t state;
  uint64_t next() {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  double normal() {
    const double u0 = uniform(), u1 = uniform();
    return std::sqrt(-2.0 * std::log1p(-u0)) * std::cos(2.0 * M_PI * u1);
  }
};

// Velocities (A/fs): each component N(0, kB T kappa / m), centre-of-mass
// velocity removed.
void maxwell_boltzmann(const std::vector<double>& masses, const int32_t* species, int64_t n, double T,
                       uint64_t seed, double* vel) {
  SplitMix64 rng{seed};
  double mv[3] = {0, 0, 0}, msum = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double m = masses[species[i]];
    const double sd = std::sqrt(kBoltzmann * T * kKappaMD / m);
    for (int k = 0; k < 3; ++k) {
      vel[3 * i + k] = rng.normal() * sd;
      mv[k] += m * vel[3 * i + k];
    }
    msum += m;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) vel[3 * i + k] -= mv[k] / msum;
}

// Arena compaction.  tab = off[nslot + 1], then (src, kind) per slot: atom a
// of slot k (off[k] <= a < off[k+1]) takes its state from the old arena at
// src + (a - off[k]) when kind = 1 (a running request), or its inputs from
// the incoming buffers at src + (a - off[k]) when kind = 0 (forces zero).
struct ArenaPtrs {
  double *pos, *vel, *F;
  int* species;
};

__global__ void arena_gather(int n, int nslot, const int* __restrict__ tab, ArenaPtrs src, ArenaPtrs dst,
                             const double* __restrict__ inc_pos, const double* __restrict__ inc_vel,
                             const int* __restrict__ inc_species) {
  const int* off = tab;
  const int* from = tab + nslot + 1;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
    int lo = 0, hi = nslot - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= a) lo = mid; else hi = mid - 1;
    }
    const int r = a - off[lo], s = from[2 * lo], kind = from[2 * lo + 1];
    if (kind) {  // running request: its current state
      const int q = s + r;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dst.pos[3 * a + k] = src.pos[3 * q + k];
        dst.vel[3 * a + k] = src.vel[3 * q + k];
        dst.F[3 * a + k] = src.F[3 * q + k];
      }
      dst.species[a] = src.species[q];
    } else {  // new request: its inputs
      const int q = s + r;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dst.pos[3 * a + k] = inc_pos[3 * q + k];
        dst.vel[3 * a + k] = inc_vel[3 * q + k];
        dst.F[3 * a + k] = 0.0;
      }
      dst.species[a] = inc_species[q];
    }
  }
}

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

enum class RState { Queued, Running, Done };

struct Request {
  uint64_t id = 0;
  int kind = MLIP_REQ_ENERGY_FORCES;
  int want_stress = 0;
  int64_t n = 0, n_steps = 0;
  double dt = 0.0;
  double cell[9];
  uint8_t pbc[3];
  std::vector<double> pos, vel;  // inputs, then (NVE) final state
  std::vector<int32_t> species;
  // results
  int status = MLIP_OK;
  double energy = 0.0, stress[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<double> forces, pe, ke;
  double t_arrive = 0, t_admit = 0, t_done = 0;
  RState state = RState::Queued;
  // worker-side
  int64_t step = 0;  // evaluations done
  int64_t bytes = 0; // admission estimate
  int64_t off = 0;   // first atom in the arena
};

}  // namespace
}  // namespace mlip

struct mlip_server {
  mlip_model* M = nullptr;
  mlip_serve_config cfg{};
  cudaStream_t st = nullptr;
  std::chrono::steady_clock::time_point t0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  bool dead = false;  // a device timeout or sticky CUDA error ended the server
  std::string dead_msg;
  uint64_t next_id = 1;
  std::deque<std::shared_ptr<mlip::Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<mlip::Request>> table;
  // statistics
  int64_t submitted = 0, completed = 0, failed = 0, rejected = 0;
  int64_t iterations = 0, atom_evals = 0, batch_req_sum = 0, changed_iterations = 0;
  double changed_busy_s = 0.0;
  double busy_s = 0.0;
  std::vector<double> lat_ms;
  std::vector<int64_t> lat_n;
  // worker state (worker thread only)
  std::vector<std::shared_ptr<mlip::Request>> running;
  mlip::Workspace ws;        // arenas and per-iteration buffers
  mlip::HostStage in_stage;  // new requests' inputs
  mlip::HostStage out_stage; // per-iteration outputs
  int arena = 0;             // which of the two arenas holds the state
  int64_t arena_n = 0;
  double per_atom_bytes = 0.0;
  int64_t held_bytes = 0;
  // Skin neighbour list of the running batch, kept on the device between
  // iterations while the membership stays the same (an NVE-only batch): built
  // at r_c + skin, compacted to r_c at every step, rebuilt when an atom moves
  // more than skin/2; the compaction and evaluation of a step are captured as
  // one CUDA graph and replayed.  skin_ok: the list belongs to the current
  // arena and batch.
  mlip::SkinList sl;
  bool skin_ok = false;
  int same_run = 0;  // consecutive iterations (this one included) with the same members
  std::atomic<int64_t> skin_reuses{0}, skin_builds{0};  // read by mlip_serve_stats
  cudaGraph_t sgraph = nullptr;
  cudaGraphExec_t sexec = nullptr;
  uint64_t swarm_gen = ~0ULL, sgraph_gen = ~0ULL;
  int64_t swarm_cap = -1, sgraph_cap = -1;
  long long sgraph_kernels = 0;
  void drop_skin_graph() {
    if (sexec) cudaGraphExecDestroy(sexec);
    if (sgraph) cudaGraphDestroy(sgraph);
    sexec = nullptr;
    sgraph = nullptr;
    swarm_gen = sgraph_gen = ~0ULL;
    swarm_cap = sgraph_cap = -1;
  }
};

namespace mlip {
namespace {

// Device bytes of one atom in a batch: node tensors and per-atom buffers of
// the evaluation, the neighbour build, the arenas, and the edges at the
// model's neighbour density with 50 % headroom.
double bytes_per_atom(const mlip_model* M) {
  const double DC = (double)M->D * M->C * 4.0;
  const int T = M->T;
  const double node = DC * (T + 1 + 7) + (double)T * M->C * 4.0 + 256.0 * 8.0 + 200.0 + 2 * 80.0;
  double edge = 16 + 64 + 64 + 16 + 4 + 8 + 12 + 3;
  if (M->precision == MLIP_PREC_FP32)
    edge += (double)M->H * 4 * 2 + (double)M->P * M->C * 4.0 * (T + 1);
  else
    edge += (double)M->H * 4 + 128.0 * T;
  const double deg = std::max(8.0, M->avg_nb) * 1.5;
  return 1.125 * (node + deg * edge);
}

int64_t ws_bytes(const Workspace& w) {
  int64_t b = 0;
  for (auto& kv : w.bufs) b += (int64_t)kv.second.bytes;
  return b;
}

double pct(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double x = q * (double)(v.size() - 1);
  const size_t i = (size_t)x;
  const double f = x - (double)i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

int bucket_of(const mlip_serve_config& c, int64_t n) {
  for (int b = 0; b < c.n_buckets; ++b)
    if (n <= c.bucket_edges[b]) return b;
  return c.n_buckets;
}

// Ends a request (under the server lock).
void finish(mlip_server* S, Request& r, int status) {
  r.status = status;
  r.t_done = now_s(S->t0);
  r.state = RState::Done;
  if (status == MLIP_OK) {
    ++S->completed;
    S->lat_ms.push_back(1e3 * (r.t_done - r.t_arrive));
    S->lat_n.push_back(r.n);
  } else {
    ++S->failed;
  }
}

}  // namespace
}  // namespace mlip

namespace mlip {
namespace {

using ReqPtr = std::shared_ptr<Request>;

struct Arena {
  double *pos = nullptr, *vel = nullptr, *F = nullptr;
  int* species = nullptr;
};

int get_arena(mlip_server* S, int which, int64_t n, Arena* a) {
  const std::string p = which ? "a1." : "a0.";
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  MLIP_TRY(S->ws.get(p + "pos", 3 * nn, &a->pos));
  MLIP_TRY(S->ws.get(p + "vel", 3 * nn, &a->vel));
  MLIP_TRY(S->ws.get(p + "F", 3 * nn, &a->F));
  MLIP_TRY(S->ws.get(p + "species", nn, &a->species));
  return MLIP_OK;
}

// Builds the arena of `cur` (running requests first, then the new ones) from
// the old arena and the new requests' inputs.
int compact(mlip_server* S, const std::vector<ReqPtr>& cur, size_t n_old_slots, Arena* out) {
  cudaStream_t st = S->st;
  WsStream wss(S->ws, st);
  const int nslot = (int)cur.size();
  int64_t total = 0, inc_n = 0;
  for (auto& r : cur) total += r->n;
  for (size_t k = n_old_slots; k < cur.size(); ++k) inc_n += cur[k]->n;
  Arena src, dst;
  MLIP_TRY(get_arena(S, S->arena, S->arena_n, &src));
  MLIP_TRY(get_arena(S, S->arena ^ 1, total, &dst));
  // incoming inputs and the slot table in one pinned blob
  const size_t nd = 6 * (size_t)inc_n, ni = (size_t)inc_n + (size_t)(nslot + 1) + 2 * (size_t)nslot;
  const size_t bytes = nd * sizeof(double) + ni * sizeof(int);
  void* hp = nullptr;
  MLIP_TRY(S->in_stage.get(bytes, &hp));
  double* hpos = static_cast<double*>(hp);
  double* hvel = hpos + 3 * inc_n;
  int* hspc = reinterpret_cast<int*>(hvel + 3 * inc_n);
  int* tab = hspc + inc_n;
  int64_t a = 0, q = 0;
  for (int k = 0; k < nslot; ++k) {
    Request& r = *cur[k];
    tab[k] = (int)a;
    if ((size_t)k < n_old_slots) {
      tab[nslot + 1 + 2 * k] = (int)r.off;
      tab[nslot + 1 + 2 * k + 1] = 1;
    } else {
      std::memcpy(hpos + 3 * q, r.pos.data(), sizeof(double) * 3 * r.n);
      if (r.kind == MLIP_REQ_NVE) std::memcpy(hvel + 3 * q, r.vel.data(), sizeof(double) * 3 * r.n);
      else std::memset(hvel + 3 * q, 0, sizeof(double) * 3 * r.n);
      std::memcpy(hspc + q, r.species.data(), sizeof(int) * r.n);
      tab[nslot + 1 + 2 * k] = (int)q;
      tab[nslot + 1 + 2 * k + 1] = 0;
      q += r.n;
    }
    r.off = a;
    a += r.n;
  }
  tab[nslot] = (int)a;
  unsigned char* dblob = nullptr;
  MLIP_TRY(S->ws.get("inc.blob", bytes, &dblob));
  MLIP_CUDA_TRY(cudaMemcpyAsync(dblob, hp, bytes, cudaMemcpyHostToDevice, st));
  const double* dpos = reinterpret_cast<const double*>(dblob);
  const double* dvel = dpos + 3 * inc_n;
  const int* dspc = reinterpret_cast<const int*>(dvel + 3 * inc_n);
  const int* dtab = dspc + inc_n;
  if (total > 0) {
    MLIP_PROF("arena_gather", st);
    arena_gather<<<(int)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(
        (int)total, nslot, dtab, ArenaPtrs{src.pos, src.vel, src.F, src.species},
        ArenaPtrs{dst.pos, dst.vel, dst.F, dst.species}, dpos, dvel, dspc);
    MLIP_LAUNCH_CHECK();
  }
  // the pinned blob is rewritten at the next compaction
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  S->arena ^= 1;
  S->arena_n = total;
  *out = dst;
  return MLIP_OK;
}

// Waits for the stream with the configured bound.  false: the bound ran out.
bool bounded_wait(mlip_server* S, cudaEvent_t ev) {
  const int64_t lim = S->cfg.device_poll_limit_us;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return true;
    if (e != cudaErrorNotReady) return true;  // reported by the next call
    if (lim > 0 && std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count() > lim)
      return false;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace
}  // namespace mlip

namespace mlip {
namespace {

// A failure is fatal for the server when the CUDA context no longer works.
bool context_broken() { return cudaDeviceSynchronize() != cudaSuccess; }

constexpr double kServeSkin = 2.0;  // A: candidates within r_c + skin

// Forces and energies of the batch at the arena's current positions from the
// resident skin list: compaction to r_c and the evaluation (a replayed graph
// after one eager run at the same workspace and capacity), then the skin check;
// if an atom left its skin the list is rebuilt at the current positions and
// the step evaluated again (its forces overwritten).  The results equal a
// fresh list's bit for bit.
int skin_evaluate(mlip_server* S, const SystemBatch& b, const Arena& A, double* d_E, double* d_S) {
  mlip_model* M = S->M;
  cudaStream_t st = S->st;
  Workspace& ws = M->ws;
  SkinList& sl = S->sl;
  ++M->eval_gen;
  int* flag = nullptr;
  MLIP_TRY(ws.get("chk.flag", 2, &flag));
  auto once = [&]() -> int {
    MLIP_TRY(launch_check_inputs((int)b.n, A.pos, A.species, M->S, flag, st));
    MLIP_TRY(skin_compact(ws, sl, A.pos, b, st));
    return evaluate_fused_edges(M, A.pos, A.species, b, sl.nl, sl.Edev(), flag, d_E, A.F, d_S, st);
  };
  auto reset = [&]() -> int {
    MLIP_CUDA_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
    MLIP_CUDA_TRY(cudaMemsetAsync(sl.flags, 0, 2 * sizeof(int), st));
    return MLIP_OK;
  };
  MLIP_TRY(reset());
  const bool graphs = !prof_timing_on();
  if (graphs && S->sexec && S->sgraph_gen == ws.gen && S->sgraph_cap == sl.cap) {
    MLIP_CUDA_TRY(cudaGraphLaunch(S->sexec, st));
    prof_add_launches(S->sgraph_kernels);
  } else if (graphs && S->swarm_gen == ws.gen && S->swarm_cap == sl.cap) {
    if (S->sexec) cudaGraphExecDestroy(S->sexec);
    if (S->sgraph) cudaGraphDestroy(S->sgraph);
    S->sexec = nullptr;
    S->sgraph = nullptr;
    const long long l0 = prof_launches();
    MLIP_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    const int rc = once();
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (rc != MLIP_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (rc != MLIP_OK) return rc;
      set_error("serve: graph capture failed: %s", cudaGetErrorString(ce));
      return MLIP_ERR_CUDA;
    }
    S->sgraph = g;
    MLIP_CUDA_TRY(cudaGraphInstantiate(&S->sexec, S->sgraph, 0));
    S->sgraph_kernels = prof_launches() - l0;
    S->sgraph_gen = ws.gen;
    S->sgraph_cap = sl.cap;
    MLIP_CUDA_TRY(cudaGraphLaunch(S->sexec, st));
  } else {
    MLIP_TRY(once());
    S->swarm_gen = ws.gen;
    S->swarm_cap = sl.cap;
  }
  MLIP_TRY(check_eval_flags(flag, st));
  int hs[2] = {0, 0};
  MLIP_CUDA_TRY(cudaMemcpyAsync(hs, sl.flags, sizeof(hs), cudaMemcpyDeviceToHost, st));
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  if (hs[1]) { set_error("serve: skin list: a kept edge has no kept reverse edge"); return MLIP_ERR_INVALID_ARG; }
  if (hs[0]) {  // an atom left its skin: a fresh list at the current positions, the step again
    MLIP_TRY(skin_build(ws, A.pos, b, M->rc, kServeSkin, &sl, st));
    ++S->skin_builds;
    MLIP_TRY(reset());
    MLIP_TRY(once());
    MLIP_TRY(check_eval_flags(flag, st));
  }
  ++S->skin_reuses;
  return MLIP_OK;
}

// One batched force evaluation over `cur` (arena A).  Per-request failures end
// those requests (status in the request); the return value is an error only
// when the server cannot go on (broken context, device timeout).
int iterate(mlip_server* S, std::vector<ReqPtr>& cur, const Arena& A, bool same_members, std::vector<ReqPtr>& ended) {
  mlip_model* M = S->M;
  cudaStream_t st = S->st;
  WsStream wss(S->ws, st), wsm(M->ws, st);
  const int nsys = (int)cur.size();
  SystemBatch b;
  b.nsys = nsys;
  b.atom_off.resize(nsys + 1);
  b.cell.resize(9 * (size_t)nsys);
  b.pbc.resize(3 * (size_t)nsys);
  bool any_nve = false, any_active = false, any_stress = false;
  for (int s = 0; s < nsys; ++s) {
    const Request& r = *cur[s];
    b.atom_off[s] = r.off;
    std::memcpy(&b.cell[9 * s], r.cell, sizeof(r.cell));
    std::memcpy(&b.pbc[3 * s], r.pbc, 3);
    any_nve |= r.kind == MLIP_REQ_NVE;
    any_active |= r.kind == MLIP_REQ_NVE && r.step > 0;
    any_stress |= r.want_stress != 0;
  }
  b.atom_off[nsys] = cur.back()->off + cur.back()->n;
  MLIP_TRY(upload_batch(M->ws, M->stage, b, st));
  // per-system time steps and the mask of systems that move this iteration
  double *d_dt = nullptr, *d_E = nullptr, *d_KE = nullptr, *d_S = nullptr;
  int* d_active = nullptr;
  MLIP_TRY(S->ws.get("it.dt", (size_t)nsys, &d_dt));
  MLIP_TRY(S->ws.get("it.active", (size_t)nsys, &d_active));
  MLIP_TRY(S->ws.get("it.E", (size_t)nsys, &d_E));
  MLIP_TRY(S->ws.get("it.KE", (size_t)nsys, &d_KE));
  if (any_stress) MLIP_TRY(S->ws.get("it.S", 9 * (size_t)nsys, &d_S));
  double* d_mass = nullptr;
  MLIP_TRY(S->ws.get("srv.mass", (size_t)std::max(M->S, 1), &d_mass));
  if (any_nve) {
    void* hp = nullptr;
    MLIP_TRY(S->in_stage.get(sizeof(double) * nsys + sizeof(int) * nsys, &hp));
    double* hdt = static_cast<double*>(hp);
    int* hact = reinterpret_cast<int*>(hdt + nsys);
    for (int s = 0; s < nsys; ++s) {
      hdt[s] = cur[s]->dt;
      hact[s] = (cur[s]->kind == MLIP_REQ_NVE && cur[s]->step > 0) ? 1 : 0;
    }
    MLIP_CUDA_TRY(cudaMemcpyAsync(d_dt, hdt, sizeof(double) * nsys, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(d_active, hact, sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
  }
  if (any_active) {
    MLIP_TRY(launch_vv_kick(b, A.species, d_mass, d_dt, d_active, A.F, A.vel, st));
    MLIP_TRY(launch_vv_drift(b, d_dt, d_active, A.vel, A.pos, st));
  }
  std::vector<int> slot_rc(nsys, MLIP_OK);
  if (!same_members) S->skin_ok = false;  // the arena was rebuilt: the list's atom order is gone
  S->same_run = same_members ? S->same_run + 1 : 1;
  const bool fused = M->precision != MLIP_PREC_FP32;
  int rc = MLIP_OK;
  if (fused && S->skin_ok && any_active)
    rc = skin_evaluate(S, b, A, d_E, d_S);  // the resident list, compacted to this step's positions
  else
    rc = evaluate(M, A.pos, A.species, b, d_E, A.F, d_S, st, true);  // a graph while the membership stays
  if (rc != MLIP_OK) S->skin_ok = false;
  if (rc != MLIP_OK) {
    if (context_broken()) return MLIP_ERR_CUDA;
    if (nsys == 1) {
      slot_rc[0] = rc;
    } else {  // find the request(s) at fault: each one alone on its own atoms
      for (int s = 0; s < nsys; ++s) {
        const Request& r = *cur[s];
        SystemBatch b1;
        single_system(b1, r.n, r.cell, r.pbc);
        MLIP_TRY(upload_batch(M->ws, M->stage, b1, st));
        slot_rc[s] = evaluate(M, A.pos + 3 * r.off, A.species + r.off, b1, d_E + s, A.F + 3 * r.off,
                              d_S ? d_S + 9 * s : nullptr, st);
        if (slot_rc[s] != MLIP_OK && context_broken()) return MLIP_ERR_CUDA;
      }
      MLIP_TRY(upload_batch(M->ws, M->stage, b, st));
    }
  }
  if (any_active) MLIP_TRY(launch_vv_kick(b, A.species, d_mass, d_dt, d_active, A.F, A.vel, st));
  if (any_nve) MLIP_TRY(launch_kinetic(M->ws, b, A.species, d_mass, A.vel, d_KE, st));
  // outputs: per-system energies (and kinetic energies, stress), then the
  // arrays of the requests that end with this iteration
  std::vector<char> ends(nsys, 0);
  size_t out_doubles = (size_t)nsys * (2 + (any_stress ? 9 : 0));
  for (int s = 0; s < nsys; ++s) {
    const Request& r = *cur[s];
    ends[s] = slot_rc[s] != MLIP_OK || r.kind == MLIP_REQ_ENERGY_FORCES || r.step + 1 >= r.n_steps + 1;
    if (ends[s] && slot_rc[s] == MLIP_OK) out_doubles += 3 * (size_t)r.n * (r.kind == MLIP_REQ_NVE ? 3 : 1);
  }
  void* hp = nullptr;
  MLIP_TRY(S->out_stage.get(out_doubles * sizeof(double), &hp));
  double* ho = static_cast<double*>(hp);
  double* hE = ho;
  double* hKE = ho + nsys;
  double* hS = ho + 2 * nsys;
  double* hx = hS + (any_stress ? 9 * (size_t)nsys : 0);
  MLIP_CUDA_TRY(cudaMemcpyAsync(hE, d_E, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
  if (any_nve) MLIP_CUDA_TRY(cudaMemcpyAsync(hKE, d_KE, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
  if (any_stress) MLIP_CUDA_TRY(cudaMemcpyAsync(hS, d_S, sizeof(double) * 9 * nsys, cudaMemcpyDeviceToHost, st));
  std::vector<double*> at(nsys, nullptr);
  for (int s = 0; s < nsys; ++s) {
    const Request& r = *cur[s];
    if (!ends[s] || slot_rc[s] != MLIP_OK) continue;
    at[s] = hx;
    const size_t bytes = sizeof(double) * 3 * r.n;
    MLIP_CUDA_TRY(cudaMemcpyAsync(hx, A.F + 3 * r.off, bytes, cudaMemcpyDeviceToHost, st));
    hx += 3 * r.n;
    if (r.kind == MLIP_REQ_NVE) {
      MLIP_CUDA_TRY(cudaMemcpyAsync(hx, A.pos + 3 * r.off, bytes, cudaMemcpyDeviceToHost, st));
      MLIP_CUDA_TRY(cudaMemcpyAsync(hx + 3 * r.n, A.vel + 3 * r.off, bytes, cudaMemcpyDeviceToHost, st));
      hx += 6 * r.n;
    }
  }
  // an NVE-only batch whose requests all go on keeps its members unless new
  // requests arrive: its skin list is built now, at the positions of the next
  // step's start, if it has none
  bool keep_members = fused;
  for (int s = 0; s < nsys && keep_members; ++s) keep_members = !ends[s] && cur[s]->kind == MLIP_REQ_NVE;
  // (only once the members have stayed for resident_after iterations: a list
  // built for a batch that changes again a step later costs more than it saves)
  keep_members = keep_members && S->cfg.resident_after > 0 && S->same_run >= S->cfg.resident_after;
  if (keep_members && !S->skin_ok) {
    S->drop_skin_graph();
    const int brc = skin_build(M->ws, A.pos, b, M->rc, kServeSkin, &S->sl, st);
    if (brc != MLIP_OK) {
      if (context_broken()) return MLIP_ERR_CUDA;
      cudaGetLastError();
    } else {
      S->skin_ok = true;
      ++S->skin_builds;
    }
  }
  cudaEvent_t ev;
  MLIP_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaEventRecord(ev, st);
  const bool ok = bounded_wait(S, ev);
  if (!ok) {
    cudaStreamSynchronize(st);  // leave nothing in flight behind the server's buffers
    cudaEventDestroy(ev);
    set_error("serve: an iteration's results took longer than %lld us", (long long)S->cfg.device_poll_limit_us);
    return MLIP_ERR_DEVICE_TIMEOUT;
  }
  cudaEventDestroy(ev);
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  for (int s = 0; s < nsys; ++s) {
    Request& r = *cur[s];
    if (slot_rc[s] != MLIP_OK) {
      r.status = slot_rc[s];
      ended.push_back(cur[s]);
      continue;
    }
    ++r.step;
    if (r.kind == MLIP_REQ_NVE) {
      r.pe.push_back(hE[s]);
      r.ke.push_back(hKE[s]);
    }
    if (!ends[s]) continue;
    r.energy = hE[s];
    if (r.want_stress) std::memcpy(r.stress, hS + 9 * (size_t)s, sizeof(r.stress));
    r.forces.assign(at[s], at[s] + 3 * r.n);
    if (r.kind == MLIP_REQ_NVE) {
      r.pos.assign(at[s] + 3 * r.n, at[s] + 6 * r.n);
      r.vel.assign(at[s] + 6 * r.n, at[s] + 9 * r.n);
    }
    r.status = MLIP_OK;
    ended.push_back(cur[s]);
  }
  return MLIP_OK;
}

}  // namespace
}  // namespace mlip

namespace mlip {
namespace {

void fail_all(mlip_server* S, int status) {  // under the lock
  for (auto& r : S->running)
    if (r->state != RState::Done) finish(S, *r, status);
  S->running.clear();
  for (auto& r : S->queue) finish(S, *r, status);
  S->queue.clear();
}

void worker_main(mlip_server* S) {
  cudaSetDevice(S->M->device);
  const int64_t budget = S->cfg.hbm_budget_bytes;
  const int max_slots = S->cfg.max_slots;
  bool changed = false;  // membership changed since the arena was built
  for (;;) {
    std::vector<ReqPtr> fresh;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || (!S->dead && (!S->queue.empty() || !S->running.empty())); });
      if (S->stop) break;
      int64_t bytes = 0;
      for (auto& r : S->running) bytes += r->bytes;
      const double t = now_s(S->t0);
      while (!S->queue.empty() && (int)(S->running.size() + fresh.size()) < max_slots) {
        ReqPtr r = S->queue.front();
        if (bytes + r->bytes > budget && !(S->running.empty() && fresh.empty())) break;
        bytes += r->bytes;
        r->state = RState::Running;
        r->t_admit = t;
        fresh.push_back(r);
        S->queue.pop_front();
      }
    }
    const auto t_it = std::chrono::steady_clock::now();
    std::vector<ReqPtr> cur = S->running;
    const size_t n_old = cur.size();
    cur.insert(cur.end(), fresh.begin(), fresh.end());
    if (cur.empty()) continue;
    Arena A;
    int rc = MLIP_OK;
    const bool moved = changed || !fresh.empty();
    if (moved) rc = compact(S, cur, n_old, &A);
    else rc = get_arena(S, S->arena, S->arena_n, &A);
    std::vector<ReqPtr> ended;
    if (rc == MLIP_OK) rc = iterate(S, cur, A, !moved, ended);
    const double dt_it = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_it).count();
    std::lock_guard<std::mutex> lk(S->mu);
    S->running = cur;
    if (rc != MLIP_OK) {
      // the server cannot go on: fail everything, admit nothing more
      const bool broken = rc == MLIP_ERR_CUDA || rc == MLIP_ERR_DEVICE_TIMEOUT;
      if (broken) {
        S->dead = true;
        S->dead_msg = last_error();
        fail_all(S, rc);
      } else {  // a host-side failure of this iteration (e.g. out of memory): fail its requests
        for (auto& r : cur) finish(S, *r, rc);
        S->running.clear();
      }
      changed = true;
      S->cv_done.notify_all();
      continue;
    }
    ++S->iterations;
    S->atom_evals += cur.back()->off + cur.back()->n;
    S->batch_req_sum += (int64_t)cur.size();
    S->busy_s += dt_it;
    if (moved) {
      ++S->changed_iterations;
      S->changed_busy_s += dt_it;
    }
    changed = !ended.empty();
    if (changed) {
      for (auto& r : ended) {
        finish(S, *r, r->status);
        if (r->kind != MLIP_REQ_NVE) {  // inputs no longer needed
          std::vector<double>().swap(r->pos);
          std::vector<int32_t>().swap(r->species);
        }
      }
      std::vector<ReqPtr> keep;
      for (auto& r : cur)
        if (r->state != RState::Done) keep.push_back(r);
      S->running.swap(keep);
      S->cv_done.notify_all();
    }
  }
  std::lock_guard<std::mutex> lk(S->mu);
  set_error("serve: the server was destroyed before the request ended");
  fail_all(S, MLIP_ERR_TIMEOUT);
  S->cv_done.notify_all();
}

void fill_result(const Request& r, mlip_result* out) {
  std::memset(out, 0, sizeof(*out));
  out->status = r.status;
  out->kind = r.kind;
  out->n = r.n;
  out->n_steps = r.n_steps;
  out->energy = r.energy;
  std::memcpy(out->stress, r.stress, sizeof(r.stress));
  out->forces = r.forces.empty() ? nullptr : r.forces.data();
  if (r.kind == MLIP_REQ_NVE && r.status == MLIP_OK) {
    out->pos = r.pos.data();
    out->vel = r.vel.data();
    out->pe = r.pe.data();
    out->ke = r.ke.data();
  }
  out->t_arrive = r.t_arrive;
  out->t_admit = r.t_admit;
  out->t_done = r.t_done;
}

}  // namespace
}  // namespace mlip

using namespace mlip;

extern "C" int mlip_serve_create(mlip_model* M, const mlip_serve_config* cfg, mlip_server** out) {
  if (!M || !out) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  *out = nullptr;
  mlip_serve_config c{};
  if (cfg) c = *cfg;
  if (c.max_slots < 0 || c.n_buckets < 0 || c.n_buckets > 8 || c.hbm_budget_bytes < 0 || c.device_poll_limit_us < 0) {
    set_error("serve: bad configuration");
    return MLIP_ERR_INVALID_ARG;
  }
  for (int b = 1; b < c.n_buckets; ++b)
    if (c.bucket_edges[b] <= c.bucket_edges[b - 1]) { set_error("serve: bucket edges must ascend"); return MLIP_ERR_INVALID_ARG; }
  if (c.reserved != 0) { set_error("serve: reserved configuration field must be 0"); return MLIP_ERR_INVALID_ARG; }
  if (c.max_slots == 0) c.max_slots = 512;
  if (c.resident_after == 0) c.resident_after = 3;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != M->device) { set_error("model lives on device %d, current device is %d", M->device, cur); return MLIP_ERR_INVALID_ARG; }
  if (c.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    MLIP_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    c.hbm_budget_bytes = (int64_t)(0.8 * (double)fr);
  }
  auto S = std::make_unique<mlip_server>();
  S->M = M;
  S->cfg = c;
  S->per_atom_bytes = bytes_per_atom(M);
  S->t0 = std::chrono::steady_clock::now();
  MLIP_CUDA_TRY(cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking));
  if ((int)M->masses.size() == M->S && M->S > 0) {
    double* d_mass = nullptr;
    int rc = S->ws.get("srv.mass", (size_t)M->S, &d_mass);
    if (rc == MLIP_OK) rc = cudaMemcpy(d_mass, M->masses.data(), sizeof(double) * M->S, cudaMemcpyHostToDevice) == cudaSuccess ? MLIP_OK : MLIP_ERR_CUDA;
    if (rc != MLIP_OK) { cudaStreamDestroy(S->st); return rc; }
  }
  mlip_server* raw = S.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return MLIP_OK;
}

extern "C" int mlip_serve_submit(mlip_server* S, const mlip_request* q, uint64_t* id) {
  if (!S || !q || !id) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  mlip_model* M = S->M;
  if (q->kind != MLIP_REQ_ENERGY_FORCES && q->kind != MLIP_REQ_NVE) { set_error("serve: unknown request kind %d", q->kind); return MLIP_ERR_INVALID_ARG; }
  if (q->n < 1 || q->n > (1LL << 26) || !q->pos || !q->species) { set_error("serve: bad atom count or null input"); return MLIP_ERR_INVALID_ARG; }
  const bool any_pbc = q->pbc[0] || q->pbc[1] || q->pbc[2];
  if (q->kind == MLIP_REQ_ENERGY_FORCES && q->want_stress && !(q->pbc[0] && q->pbc[1] && q->pbc[2])) {
    set_error("serve: stress needs a fully periodic cell");
    return MLIP_ERR_CELL;
  }
  if (any_pbc) {
    const double* h = q->cell;
    const double det = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) + h[2] * (h[3] * h[7] - h[4] * h[6]);
    if (!(std::fabs(det) > 1e-12) || !std::isfinite(det)) { set_error("serve: singular cell with a periodic axis"); return MLIP_ERR_CELL; }
  }
  if (q->kind == MLIP_REQ_NVE) {
    if ((int)M->masses.size() != M->S) { set_error("serve: the model has no masses (needed for MD)"); return MLIP_ERR_INVALID_ARG; }
    if (q->n_steps < 0 || q->n_steps > (1LL << 24) || !(q->dt_fs > 0) || !std::isfinite(q->dt_fs)) {
      set_error("serve: bad step count or time step");
      return MLIP_ERR_INVALID_ARG;
    }
    if (!q->vel && !(q->temperature_K >= 0 && std::isfinite(q->temperature_K))) { set_error("serve: bad temperature"); return MLIP_ERR_INVALID_ARG; }
  }
  auto r = std::make_shared<Request>();
  r->kind = q->kind;
  r->want_stress = q->kind == MLIP_REQ_ENERGY_FORCES ? (q->want_stress != 0) : 0;
  r->n = q->n;
  r->n_steps = q->kind == MLIP_REQ_NVE ? q->n_steps : 0;
  r->dt = q->dt_fs;
  std::memcpy(r->cell, q->cell, sizeof(r->cell));
  std::memcpy(r->pbc, q->pbc, 3);
  r->pos.assign(q->pos, q->pos + 3 * q->n);
  r->species.assign(q->species, q->species + q->n);
  for (int64_t i = 0; i < q->n; ++i) {
    if (r->species[i] < 0 || r->species[i] >= M->S) { set_error("serve: species[%lld] = %d out of range", (long long)i, r->species[i]); return MLIP_ERR_INVALID_ARG; }
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(r->pos[3 * i + k])) { set_error("serve: non-finite position of atom %lld", (long long)i); return MLIP_ERR_INVALID_ARG; }
  }
  if (r->kind == MLIP_REQ_NVE) {
    r->vel.resize(3 * q->n);
    if (q->vel) {
      std::memcpy(r->vel.data(), q->vel, sizeof(double) * 3 * q->n);
      for (double v : r->vel)
        if (!std::isfinite(v)) { set_error("serve: non-finite velocity"); return MLIP_ERR_INVALID_ARG; }
    } else {
      maxwell_boltzmann(M->masses, r->species.data(), q->n, q->temperature_K, q->seed, r->vel.data());
    }
    r->pe.reserve(r->n_steps + 1);
    r->ke.reserve(r->n_steps + 1);
  }
  r->bytes = (int64_t)(S->per_atom_bytes * (double)q->n);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->dead) { set_error("serve: the server stopped after: %s", S->dead_msg.c_str()); return MLIP_ERR_DEVICE_TIMEOUT; }
  if (S->stop) { set_error("serve: the server is shutting down"); return MLIP_ERR_INVALID_ARG; }
  if (r->bytes > S->cfg.hbm_budget_bytes) {
    ++S->rejected;
    set_error("serve: a request of %lld atoms needs about %lld bytes, over the budget of %lld", (long long)q->n,
              (long long)r->bytes, (long long)S->cfg.hbm_budget_bytes);
    return MLIP_ERR_BUDGET;
  }
  r->id = S->next_id++;
  r->t_arrive = now_s(S->t0);
  S->table[r->id] = r;
  S->queue.push_back(r);
  ++S->submitted;
  *id = r->id;
  S->cv_work.notify_one();
  return MLIP_OK;
}

extern "C" int mlip_serve_poll(mlip_server* S, uint64_t id, mlip_result* out) {
  if (!S || !out) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->table.find(id);
  if (it == S->table.end()) { set_error("serve: unknown request id %llu", (unsigned long long)id); return MLIP_ERR_NOT_FOUND; }
  if (it->second->state != RState::Done) return MLIP_PENDING;
  fill_result(*it->second, out);
  return MLIP_OK;
}

extern "C" int mlip_serve_wait(mlip_server* S, uint64_t id, int64_t timeout_ms, mlip_result* out) {
  if (!S || !out) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->table.find(id);
  if (it == S->table.end()) { set_error("serve: unknown request id %llu", (unsigned long long)id); return MLIP_ERR_NOT_FOUND; }
  ReqPtr r = it->second;
  auto done = [&] { return r->state == RState::Done; };
  if (timeout_ms < 0) S->cv_done.wait(lk, done);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    set_error("serve: request %llu still pending after %lld ms", (unsigned long long)id, (long long)timeout_ms);
    return MLIP_ERR_TIMEOUT;
  }
  fill_result(*r, out);
  return MLIP_OK;
}

extern "C" int mlip_serve_release(mlip_server* S, uint64_t id) {
  if (!S) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->table.find(id);
  if (it == S->table.end()) { set_error("serve: unknown request id %llu", (unsigned long long)id); return MLIP_ERR_NOT_FOUND; }
  if (it->second->state != RState::Done) return MLIP_PENDING;
  S->table.erase(it);
  return MLIP_OK;
}

extern "C" int mlip_serve_stats(mlip_server* S, mlip_serve_statistics* out) {
  if (!S || !out) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  std::memset(out, 0, sizeof(*out));
  std::lock_guard<std::mutex> lk(S->mu);
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->rejected = S->rejected;
  out->queued = (int64_t)S->queue.size();
  out->running = (int64_t)S->running.size();
  out->iterations = S->iterations;
  out->changed_iterations = S->changed_iterations;
  out->changed_busy_s = S->changed_busy_s;
  out->atom_evals = S->atom_evals;
  out->elapsed_s = now_s(S->t0);
  out->busy_s = S->busy_s;
  out->atom_steps_per_s = S->busy_s > 0 ? (double)S->atom_evals / S->busy_s : 0.0;
  out->p50_ms = pct(S->lat_ms, 0.50);
  out->p99_ms = pct(S->lat_ms, 0.99);
  double sum = 0.0, mx = 0.0;
  for (double v : S->lat_ms) { sum += v; mx = std::max(mx, v); }
  out->mean_ms = S->lat_ms.empty() ? 0.0 : sum / (double)S->lat_ms.size();
  out->max_ms = mx;
  out->mean_batch_atoms = S->iterations ? (double)S->atom_evals / (double)S->iterations : 0.0;
  out->mean_batch_requests = S->iterations ? (double)S->batch_req_sum / (double)S->iterations : 0.0;
  out->device_bytes = ws_bytes(S->ws) + ws_bytes(S->M->ws);
  out->n_buckets = S->cfg.n_buckets;
  std::vector<std::vector<double>> per(S->cfg.n_buckets + 1);
  for (size_t k = 0; k < S->lat_ms.size(); ++k) per[bucket_of(S->cfg, S->lat_n[k])].push_back(S->lat_ms[k]);
  for (int b = 0; b <= S->cfg.n_buckets; ++b) {
    out->bucket_count[b] = (int64_t)per[b].size();
    out->bucket_p50_ms[b] = pct(per[b], 0.50);
    out->bucket_p99_ms[b] = pct(per[b], 0.99);
  }
  out->skin_steps = S->skin_reuses.load();
  out->skin_builds = S->skin_builds.load();
  return MLIP_OK;
}

extern "C" int mlip_serve_destroy(mlip_server* S) {
  if (!S) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaStreamSynchronize(S->st);
  S->drop_skin_graph();
  cudaStreamDestroy(S->st);
  cudaGetLastError();
  delete S;
  return MLIP_OK;
}
