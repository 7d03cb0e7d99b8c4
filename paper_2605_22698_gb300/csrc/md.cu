// Velocity-Verlet NVE integration on the device (FP64 positions and
// velocities), the integrator of the batched MD workload:
//   v += dt/2 F/m kappa;  r += dt v;  F = F(r);  v += dt/2 F/m kappa,
// kappa = 9.648533212e-3 converts eV/A/amu to A/fs^2.  Kinetic energy
// KE = sum_i m_i v_i^2 / (2 kappa) in eV, reduced in FP64 in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "launchers.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

constexpr double kKappa = 9.648533212e-3;

// System of atom i (sys_of == nullptr: one system).
__device__ __forceinline__ int sys_index(const int* sys_of, int i) { return sys_of ? sys_of[i] : 0; }

__global__ void vv_kick(int n, const int* __restrict__ sys_of, const int* __restrict__ species,
                        const double* __restrict__ mass, const double* __restrict__ dt,
                        const int* __restrict__ active, const double* __restrict__ F, double* __restrict__ vel) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = sys_index(sys_of, i);
  if (active && !active[s]) return;
  const double a = 0.5 * dt[s] * kKappa / mass[species[i]];
#pragma unroll
  for (int k = 0; k < 3; ++k) vel[3 * i + k] += a * F[3 * i + k];
}

__global__ void vv_drift(int n, const int* __restrict__ sys_of, const double* __restrict__ dt,
                         const int* __restrict__ active, const double* __restrict__ vel, double* __restrict__ pos) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = sys_index(sys_of, i);
  if (active && !active[s]) return;
  const double h = dt[s];
#pragma unroll
  for (int k = 0; k < 3; ++k) pos[3 * i + k] += h * vel[3 * i + k];
}

// ke_atom[i] = m_i v_i^2 / (2 kappa)
__global__ void kinetic_atoms(int n, const int* __restrict__ species, const double* __restrict__ mass,
                              const double* __restrict__ vel, double* __restrict__ ke_atom) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v2 = vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] + vel[3 * i + 2] * vel[3 * i + 2];
  ke_atom[i] = 0.5 * mass[species[i]] * v2 / kKappa;
}

}  // namespace

int launch_vv_kick(const SystemBatch& b, const int* species, const double* mass, const double* dt,
                   const int* active, const double* F, double* vel, cudaStream_t st) {
  const int n = (int)b.n;
  if (n <= 0) return MLIP_OK;
  { MLIP_PROF("vv_kick", st); vv_kick<<<(n + 255) / 256, 256, 0, st>>>(n, b.d_sys_of, species, mass, dt, active, F, vel); }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_vv_drift(const SystemBatch& b, const double* dt, const int* active, const double* vel, double* pos,
                    cudaStream_t st) {
  const int n = (int)b.n;
  if (n <= 0) return MLIP_OK;
  { MLIP_PROF("vv_drift", st); vv_drift<<<(n + 255) / 256, 256, 0, st>>>(n, b.d_sys_of, dt, active, vel, pos); }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_kinetic(Workspace& ws, const SystemBatch& b, const int* species, const double* mass, const double* vel,
                   double* ke, cudaStream_t st) {
  const int n = (int)b.n;
  double* ke_atom = nullptr;
  MLIP_TRY(ws.get("md.ke_atom", (size_t)std::max(n, 1), &ke_atom));
  if (n > 0) { MLIP_PROF("kinetic", st); kinetic_atoms<<<(n + 255) / 256, 256, 0, st>>>(n, species, mass, vel, ke_atom); }
  MLIP_LAUNCH_CHECK();
  return launch_seg_sum(ws, b, 1, ke_atom, false, ke, st);
}

}  // namespace mlip

using namespace mlip;

extern "C" int mlip_md_nve(mlip_model* M, double* pos, double* vel, const int32_t* species, int64_t n,
                           const double cell[9], const uint8_t pbc[3], double dt_fs, int64_t n_steps, double* pe,
                           double* ke, int on_device, void* stream) {
  if (!M || !pos || !vel || !species || !cell || !pbc) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  if (n < 1 || n_steps < 0 || !(dt_fs > 0)) { set_error("bad atom count, step count or time step"); return MLIP_ERR_INVALID_ARG; }
  if ((int)M->masses.size() != M->S) { set_error("the model has no masses (needed for MD)"); return MLIP_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace& ws = M->ws;
  WsStream wss(ws, st);
  double *d_pos = pos, *d_vel = vel, *d_F = nullptr, *d_E = nullptr, *d_mass = nullptr, *d_pe = nullptr, *d_ke = nullptr;
  const int* d_sp = species;
  if (!on_device) {
    for (int64_t i = 0; i < n; ++i)
      if (species[i] < 0 || species[i] >= M->S) { set_error("species[%lld] out of range", (long long)i); return MLIP_ERR_INVALID_ARG; }
    int* dz = nullptr;
    MLIP_TRY(ws.get("md.pos", (size_t)3 * n, &d_pos));
    MLIP_TRY(ws.get("md.vel", (size_t)3 * n, &d_vel));
    MLIP_TRY(ws.get("md.species", (size_t)n, &dz));
    MLIP_CUDA_TRY(cudaMemcpyAsync(d_pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(d_vel, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dz, species, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    d_sp = dz;
  }
  double* d_dt = nullptr;
  MLIP_TRY(ws.get("md.F", (size_t)3 * n, &d_F));
  MLIP_TRY(ws.get("md.E", 1, &d_E));
  MLIP_TRY(ws.get("md.mass", (size_t)M->S, &d_mass));
  MLIP_TRY(ws.get("md.dt", 1, &d_dt));
  MLIP_TRY(ws.get("md.pe", (size_t)n_steps + 1, &d_pe));
  MLIP_TRY(ws.get("md.ke", (size_t)n_steps + 1, &d_ke));
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_mass, M->masses.data(), sizeof(double) * M->S, cudaMemcpyHostToDevice, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_dt, &dt_fs, sizeof(double), cudaMemcpyHostToDevice, st));
  SystemBatch b;
  single_system(b, n, cell, pbc);
  MLIP_TRY(upload_batch(ws, M->stage, b, st));
  MLIP_TRY(evaluate(M, d_pos, d_sp, b, d_pe, d_F, nullptr, st, true));
  MLIP_TRY(launch_kinetic(ws, b, d_sp, d_mass, d_vel, d_ke, st));
  for (int64_t s = 0; s < n_steps; ++s) {
    MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
    MLIP_TRY(launch_vv_drift(b, d_dt, nullptr, d_vel, d_pos, st));
    MLIP_TRY(evaluate(M, d_pos, d_sp, b, d_pe + s + 1, d_F, nullptr, st, true));
    MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
    MLIP_TRY(launch_kinetic(ws, b, d_sp, d_mass, d_vel, d_ke + s + 1, st));
  }
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (pe) MLIP_CUDA_TRY(cudaMemcpyAsync(pe, d_pe, sizeof(double) * (n_steps + 1), k, st));
  if (ke) MLIP_CUDA_TRY(cudaMemcpyAsync(ke, d_ke, sizeof(double) * (n_steps + 1), k, st));
  if (!on_device) {
    MLIP_CUDA_TRY(cudaMemcpyAsync(pos, d_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(vel, d_vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
  }
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  return MLIP_OK;
}

extern "C" int mlip_md_nve_batch(mlip_model* M, int32_t n_systems, const int64_t* atom_off, double* pos, double* vel,
                                 const int32_t* species, const double* cells, const uint8_t* pbc, double dt_fs,
                                 int64_t n_steps, double* pe, double* ke, int on_device, void* stream) {
  if (!M || !atom_off || !pos || !vel || !species || !cells || !pbc) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  if (n_systems < 1 || n_systems > (1 << 20)) { set_error("system count %d out of range", n_systems); return MLIP_ERR_INVALID_ARG; }
  if (n_steps < 0 || !(dt_fs > 0)) { set_error("bad step count or time step"); return MLIP_ERR_INVALID_ARG; }
  if ((int)M->masses.size() != M->S) { set_error("the model has no masses (needed for MD)"); return MLIP_ERR_INVALID_ARG; }
  if (atom_off[0] != 0) { set_error("atom_off[0] must be 0"); return MLIP_ERR_INVALID_ARG; }
  for (int s = 0; s < n_systems; ++s)
    if (atom_off[s + 1] <= atom_off[s]) { set_error("system %d has no atoms (atom_off must increase)", s); return MLIP_ERR_INVALID_ARG; }
  const int64_t n = atom_off[n_systems];
  if (n > (1LL << 28)) { set_error("atom count %lld out of range", (long long)n); return MLIP_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace& ws = M->ws;
  WsStream wss(ws, st);
  double *d_pos = pos, *d_vel = vel, *d_F = nullptr, *d_mass = nullptr, *d_pe = nullptr, *d_ke = nullptr,
         *d_dt = nullptr;
  const int* d_sp = species;
  if (!on_device) {
    for (int64_t i = 0; i < n; ++i)
      if (species[i] < 0 || species[i] >= M->S) { set_error("species[%lld] out of range", (long long)i); return MLIP_ERR_INVALID_ARG; }
    int* dz = nullptr;
    MLIP_TRY(ws.get("md.pos", (size_t)3 * n, &d_pos));
    MLIP_TRY(ws.get("md.vel", (size_t)3 * n, &d_vel));
    MLIP_TRY(ws.get("md.species", (size_t)n, &dz));
    MLIP_CUDA_TRY(cudaMemcpyAsync(d_pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(d_vel, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dz, species, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    d_sp = dz;
  }
  const size_t traces = (size_t)(n_steps + 1) * n_systems;
  MLIP_TRY(ws.get("md.F", (size_t)3 * n, &d_F));
  MLIP_TRY(ws.get("md.mass", (size_t)M->S, &d_mass));
  MLIP_TRY(ws.get("md.dt", (size_t)n_systems, &d_dt));
  MLIP_TRY(ws.get("md.pe", traces, &d_pe));
  MLIP_TRY(ws.get("md.ke", traces, &d_ke));
  std::vector<double> hdt((size_t)n_systems, dt_fs);
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_mass, M->masses.data(), sizeof(double) * M->S, cudaMemcpyHostToDevice, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_dt, hdt.data(), sizeof(double) * n_systems, cudaMemcpyHostToDevice, st));
  SystemBatch b;
  b.nsys = n_systems;
  b.atom_off.assign(atom_off, atom_off + n_systems + 1);
  b.cell.assign(cells, cells + 9 * (size_t)n_systems);
  b.pbc.assign(pbc, pbc + 3 * (size_t)n_systems);
  MLIP_TRY(upload_batch(ws, M->stage, b, st));
  MLIP_TRY(evaluate(M, d_pos, d_sp, b, d_pe, d_F, nullptr, st, true));
  MLIP_TRY(launch_kinetic(ws, b, d_sp, d_mass, d_vel, d_ke, st));
  for (int64_t s = 0; s < n_steps; ++s) {
    MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
    MLIP_TRY(launch_vv_drift(b, d_dt, nullptr, d_vel, d_pos, st));
    MLIP_TRY(evaluate(M, d_pos, d_sp, b, d_pe + (s + 1) * n_systems, d_F, nullptr, st, true));
    MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
    MLIP_TRY(launch_kinetic(ws, b, d_sp, d_mass, d_vel, d_ke + (s + 1) * n_systems, st));
  }
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (pe) MLIP_CUDA_TRY(cudaMemcpyAsync(pe, d_pe, sizeof(double) * traces, k, st));
  if (ke) MLIP_CUDA_TRY(cudaMemcpyAsync(ke, d_ke, sizeof(double) * traces, k, st));
  if (!on_device) {
    MLIP_CUDA_TRY(cudaMemcpyAsync(pos, d_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(vel, d_vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
  }
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  return MLIP_OK;
}

// ------------------------------------------------------- skin-list driver
namespace {

// The skin-list MD run's own stream (graph capture needs a stream other than the legacy
// default one), its graph, and the event that orders it after the caller's.
struct SkinRun {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
  ~SkinRun() {
    if (st) cudaStreamSynchronize(st);
    drop_graph();
    if (ev) cudaEventDestroy(ev);
    if (st) cudaStreamDestroy(st);
  }
};

}  // namespace

extern "C" int mlip_md_nve_skin(mlip_model* M, int32_t n_systems, const int64_t* atom_off, double* pos, double* vel,
                                const int32_t* species, const double* cells, const uint8_t* pbc, double dt_fs,
                                int64_t n_steps, const mlip_md_options* opt, double* pe, double* ke,
                                mlip_md_report* report, int on_device, void* stream) {
  if (!M || !atom_off || !pos || !vel || !species || !cells || !pbc) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  if (n_systems < 1 || n_systems > (1 << 20)) { set_error("system count %d out of range", n_systems); return MLIP_ERR_INVALID_ARG; }
  if (n_steps < 0 || !(dt_fs > 0)) { set_error("bad step count or time step"); return MLIP_ERR_INVALID_ARG; }
  if ((int)M->masses.size() != M->S) { set_error("the model has no masses (needed for MD)"); return MLIP_ERR_INVALID_ARG; }
  if (M->precision == MLIP_PREC_FP32) { set_error("the skin-list driver runs the 16-bit fused form"); return MLIP_ERR_INVALID_ARG; }
  mlip_md_options o{2.0, 10, 1};
  if (opt) o = *opt;
  if (!(o.skin > 0.0) || !(o.skin <= 100.0) || o.rebuild_every < 1) { set_error("bad skin or rebuild interval"); return MLIP_ERR_INVALID_ARG; }
  if (atom_off[0] != 0) { set_error("atom_off[0] must be 0"); return MLIP_ERR_INVALID_ARG; }
  for (int s = 0; s < n_systems; ++s)
    if (atom_off[s + 1] <= atom_off[s]) { set_error("system %d has no atoms (atom_off must increase)", s); return MLIP_ERR_INVALID_ARG; }
  const int64_t n = atom_off[n_systems];
  if (n > (1LL << 28)) { set_error("atom count %lld out of range", (long long)n); return MLIP_ERR_INVALID_ARG; }
  if (!on_device)
    for (int64_t i = 0; i < n; ++i)
      if (species[i] < 0 || species[i] >= M->S) { set_error("species[%lld] out of range", (long long)i); return MLIP_ERR_INVALID_ARG; }
  mlip_md_report rep{};
  SkinRun R;
  MLIP_CUDA_TRY(cudaStreamCreateWithFlags(&R.st, cudaStreamNonBlocking));
  MLIP_CUDA_TRY(cudaEventCreateWithFlags(&R.ev, cudaEventDisableTiming));
  MLIP_CUDA_TRY(cudaEventRecord(R.ev, static_cast<cudaStream_t>(stream)));
  MLIP_CUDA_TRY(cudaStreamWaitEvent(R.st, R.ev, 0));
  cudaStream_t st = R.st;
  Workspace& ws = M->ws;
  WsStream wss(ws, st);  // restored before the run's stream is destroyed (declared after R)
  ++M->eval_gen;         // the run writes the workspace: a saved separate forward is no longer usable
  double *d_pos = pos, *d_vel = vel, *d_F = nullptr, *d_mass = nullptr, *d_pe = nullptr, *d_ke = nullptr,
         *d_dt = nullptr;
  const int* d_sp = species;
  if (!on_device) {
    int* dz = nullptr;
    MLIP_TRY(ws.get("md.pos", (size_t)3 * n, &d_pos));
    MLIP_TRY(ws.get("md.vel", (size_t)3 * n, &d_vel));
    MLIP_TRY(ws.get("md.species", (size_t)n, &dz));
    MLIP_CUDA_TRY(cudaMemcpyAsync(d_pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(d_vel, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dz, species, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    d_sp = dz;
  }
  const int every = o.rebuild_every;
  const size_t traces = (size_t)(n_steps + 1) * n_systems, nb = (size_t)every * n_systems;
  double *blk_pe = nullptr, *blk_ke = nullptr, *pos0 = nullptr, *vel0 = nullptr, *F0 = nullptr;
  int* flag = nullptr;
  MLIP_TRY(ws.get("md.F", (size_t)3 * n, &d_F));
  MLIP_TRY(ws.get("md.mass", (size_t)M->S, &d_mass));
  MLIP_TRY(ws.get("md.dt", (size_t)n_systems, &d_dt));
  MLIP_TRY(ws.get("md.pe", traces, &d_pe));
  MLIP_TRY(ws.get("md.ke", traces, &d_ke));
  MLIP_TRY(ws.get("skin.blk_pe", nb, &blk_pe));
  MLIP_TRY(ws.get("skin.blk_ke", nb, &blk_ke));
  MLIP_TRY(ws.get("skin.pos0", (size_t)3 * n, &pos0));
  MLIP_TRY(ws.get("skin.vel0", (size_t)3 * n, &vel0));
  MLIP_TRY(ws.get("skin.F0", (size_t)3 * n, &F0));
  MLIP_TRY(ws.get("chk.flag", 2, &flag));
  std::vector<double> hdt((size_t)n_systems, dt_fs);
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_mass, M->masses.data(), sizeof(double) * M->S, cudaMemcpyHostToDevice, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_dt, hdt.data(), sizeof(double) * n_systems, cudaMemcpyHostToDevice, st));
  SystemBatch b;
  b.nsys = n_systems;
  b.atom_off.assign(atom_off, atom_off + n_systems + 1);
  b.cell.assign(cells, cells + 9 * (size_t)n_systems);
  b.pbc.assign(pbc, pbc + 3 * (size_t)n_systems);
  MLIP_TRY(upload_batch(ws, M->stage, b, st));

  SkinList sl;
  auto build = [&]() -> int {
    MLIP_TRY(skin_build(ws, d_pos, b, M->rc, o.skin, &sl, st));
    rep.builds++;
    rep.max_candidates = std::max<int64_t>(rep.max_candidates, sl.n_cand);
    return MLIP_OK;
  };
  // forces and energies at the current positions from the compacted list
  auto eval = [&](double* pe_out) -> int {
    MLIP_TRY(launch_check_inputs((int)n, d_pos, d_sp, M->S, flag, st));
    MLIP_TRY(skin_compact(ws, sl, d_pos, b, st));
    return evaluate_fused_edges(M, d_pos, d_sp, b, sl.nl, sl.Edev(), flag, pe_out, d_F, nullptr, st);
  };
  // k velocity-Verlet steps; energies to the block buffers
  auto run_block = [&](int k) -> int {
    for (int j = 0; j < k; ++j) {
      MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
      MLIP_TRY(launch_vv_drift(b, d_dt, nullptr, d_vel, d_pos, st));
      MLIP_TRY(eval(blk_pe + (size_t)j * n_systems));
      MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
      MLIP_TRY(launch_kinetic(ws, b, d_sp, d_mass, d_vel, blk_ke + (size_t)j * n_systems, st));
    }
    return MLIP_OK;
  };
  auto read_skin_flags = [&](int* hs) -> int {
    MLIP_CUDA_TRY(cudaMemcpyAsync(hs, sl.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs[1]) { set_error("skin list: a kept edge has no kept reverse edge"); return MLIP_ERR_INVALID_ARG; }
    return MLIP_OK;
  };
  auto reset_flags = [&]() -> int {
    MLIP_CUDA_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
    MLIP_CUDA_TRY(cudaMemsetAsync(sl.flags, 0, 2 * sizeof(int), st));
    return MLIP_OK;
  };

  // the start
  MLIP_TRY(build());
  MLIP_CUDA_TRY(cudaMemsetAsync(sl.dmax2, 0, sizeof(unsigned long long), st));
  MLIP_TRY(reset_flags());
  MLIP_TRY(eval(d_pe));
  MLIP_TRY(launch_kinetic(ws, b, d_sp, d_mass, d_vel, d_ke, st));
  MLIP_TRY(check_eval_flags(flag, st));
  {
    int hs[2];
    MLIP_TRY(read_skin_flags(hs));
  }

  // A graph is captured only after a block ran eagerly with the same workspace
  // addresses and capacity (so no buffer grows during the capture), and it is
  // replayed while both stay the same.
  const bool graphs = o.use_graph != 0 && !prof_timing_on();
  uint64_t warm_gen = ~0ULL, graph_gen = ~0ULL;
  int64_t warm_cap = -1, graph_cap = -1;
  long long graph_kernels = 0;
  for (int64_t s0 = 0; s0 < n_steps; s0 += every) {
    const int k = (int)std::min<int64_t>(every, n_steps - s0);
    if (s0 > 0) MLIP_TRY(build());
    MLIP_CUDA_TRY(cudaMemcpyAsync(pos0, d_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(vel0, d_vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(F0, d_F, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    MLIP_TRY(reset_flags());
    const bool full = k == every;
    if (graphs && full && R.exec && graph_gen == ws.gen && graph_cap == sl.cap) {
      MLIP_CUDA_TRY(cudaGraphLaunch(R.exec, st));
      prof_add_launches(graph_kernels);
      rep.graph_launches++;
    } else if (graphs && full && warm_gen == ws.gen && warm_cap == sl.cap) {
      R.drop_graph();
      const long long l0 = prof_launches();
      MLIP_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
      const int rc = run_block(k);
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(st, &g);
      if (rc != MLIP_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        set_error("skin driver: graph capture failed: %s", cudaGetErrorString(ce));
        return MLIP_ERR_CUDA;
      }
      R.graph = g;
      MLIP_CUDA_TRY(cudaGraphInstantiate(&R.exec, R.graph, 0));
      graph_kernels = prof_launches() - l0;
      graph_gen = ws.gen;
      graph_cap = sl.cap;
      rep.graph_captures++;
      MLIP_CUDA_TRY(cudaGraphLaunch(R.exec, st));
      rep.graph_launches++;
    } else {
      MLIP_TRY(run_block(k));
      if (full) {
        warm_gen = ws.gen;
        warm_cap = sl.cap;
      }
    }
    MLIP_TRY(check_eval_flags(flag, st));
    int hs[2];
    MLIP_TRY(read_skin_flags(hs));
    if (hs[0]) {
      // an atom left its skin: the block again with a fresh list at every step
      MLIP_CUDA_TRY(cudaMemcpyAsync(d_pos, pos0, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
      MLIP_CUDA_TRY(cudaMemcpyAsync(d_vel, vel0, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
      MLIP_CUDA_TRY(cudaMemcpyAsync(d_F, F0, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
      for (int j = 0; j < k; ++j) {
        const size_t row = (size_t)(s0 + j + 1) * n_systems;
        MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
        MLIP_TRY(launch_vv_drift(b, d_dt, nullptr, d_vel, d_pos, st));
        MLIP_TRY(evaluate(M, d_pos, d_sp, b, d_pe + row, d_F, nullptr, st));
        MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
        MLIP_TRY(launch_kinetic(ws, b, d_sp, d_mass, d_vel, d_ke + row, st));
      }
      rep.redone_blocks++;
    } else {
      const size_t row = (size_t)(s0 + 1) * n_systems, cnt = (size_t)k * n_systems;
      MLIP_CUDA_TRY(cudaMemcpyAsync(d_pe + row, blk_pe, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st));
      MLIP_CUDA_TRY(cudaMemcpyAsync(d_ke + row, blk_ke, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st));
    }
  }
  unsigned long long dm = 0;
  MLIP_CUDA_TRY(cudaMemcpyAsync(&dm, sl.dmax2, sizeof(dm), cudaMemcpyDeviceToHost, st));
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (pe) MLIP_CUDA_TRY(cudaMemcpyAsync(pe, d_pe, sizeof(double) * traces, kind, st));
  if (ke) MLIP_CUDA_TRY(cudaMemcpyAsync(ke, d_ke, sizeof(double) * traces, kind, st));
  if (!on_device) {
    MLIP_CUDA_TRY(cudaMemcpyAsync(pos, d_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(vel, d_vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
  }
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  double dmax2 = 0.0;
  std::memcpy(&dmax2, &dm, sizeof(dmax2));
  rep.max_displacement = std::sqrt(dmax2);
  if (report) *report = rep;
  return MLIP_OK;
}
