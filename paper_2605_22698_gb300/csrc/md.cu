// Velocity-Verlet NVE integration on the device (FP64 positions and
// velocities), the integrator of the batched MD workload:
//   v += dt/2 F/m kappa;  r += dt v;  F = F(r);  v += dt/2 F/m kappa,
// kappa = 9.648533212e-3 converts eV/A/amu to A/fs^2.  Kinetic energy
// KE = sum_i m_i v_i^2 / (2 kappa) in eV, reduced in FP64 in a fixed order.
#include <algorithm>

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
  MLIP_TRY(evaluate(M, d_pos, d_sp, b, d_pe, d_F, nullptr, st));
  MLIP_TRY(launch_kinetic(ws, b, d_sp, d_mass, d_vel, d_ke, st));
  for (int64_t s = 0; s < n_steps; ++s) {
    MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
    MLIP_TRY(launch_vv_drift(b, d_dt, nullptr, d_vel, d_pos, st));
    MLIP_TRY(evaluate(M, d_pos, d_sp, b, d_pe + s + 1, d_F, nullptr, st));
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
  MLIP_TRY(evaluate(M, d_pos, d_sp, b, d_pe, d_F, nullptr, st));
  MLIP_TRY(launch_kinetic(ws, b, d_sp, d_mass, d_vel, d_ke, st));
  for (int64_t s = 0; s < n_steps; ++s) {
    MLIP_TRY(launch_vv_kick(b, d_sp, d_mass, d_dt, nullptr, d_F, d_vel, st));
    MLIP_TRY(launch_vv_drift(b, d_dt, nullptr, d_vel, d_pos, st));
    MLIP_TRY(evaluate(M, d_pos, d_sp, b, d_pe + (s + 1) * n_systems, d_F, nullptr, st));
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
