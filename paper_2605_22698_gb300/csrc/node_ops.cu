// Node-level and reduction kernels shared by both compute forms:
// species embedding, readout and FP64 energy sum, dE/dh^T initialisation,
// edge gradients from dE/dY and dE/dr, forces and virial in FP64.
#include <algorithm>

#include "launchers.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

// h^0: scalars from the species embedding, l > 0 zero.
// h[i][d][c] = W_emb[z_i][c] for d = 0, else 0 (float4 stores; C a multiple of 4).
// amax (nullable): amax[2 s] = max |h| over the atoms of system s, from the
// per-species maxima emax[z] = max_c |W_emb[z][c]| (one atomic per atom)
__global__ void embed(int n, int C, int D, int S, const int* __restrict__ species, const float* __restrict__ W_emb,
                      float* __restrict__ h, const int* __restrict__ sys_of, const float* __restrict__ emax,
                      float* __restrict__ amax) {
  const int C4 = C / 4;
  const size_t total = (size_t)n * D * C4;
  float4* h4 = reinterpret_cast<float4*>(h);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const int c4 = (int)(k % C4);
    const size_t rest = k / C4;
    const int d = (int)(rest % D);
    const int i = (int)(rest / D);
    const int z = clamp_species(species[i], S);
    h4[k] = d == 0 ? reinterpret_cast<const float4*>(W_emb + (size_t)z * C)[c4] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (amax && c4 == 0 && d == 0)
      atomicMax(reinterpret_cast<unsigned*>(amax) + 2 * (sys_of ? sys_of[i] : 0), __float_as_uint(emax[z]));
  }
}

// dE/dh^T: W_out[z_i] on the scalars, zero elsewhere (float4 stores).
__global__ void grad_init(int n, int C, int D, int S, const int* __restrict__ species, const float* __restrict__ W_out,
                          float* __restrict__ G) {
  const int C4 = C / 4;
  const size_t total = (size_t)n * D * C4;
  float4* G4 = reinterpret_cast<float4*>(G);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const int c4 = (int)(k % C4);
    const size_t rest = k / C4;
    const int d = (int)(rest % D);
    const int i = (int)(rest / D);
    G4[k] = d == 0 ? reinterpret_cast<const float4*>(W_out + (size_t)clamp_species(species[i], S) * C)[c4]
                   : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// E_i = sum_c W_out[z_i][c] h_i,0[c] + E0[z_i]  (one warp per atom, FP32 dot, FP64 result)
__global__ void readout(int n, int C, int D, int S, const int* __restrict__ species, const float* __restrict__ W_out,
                        const float* __restrict__ E0, const float* __restrict__ h, double* __restrict__ atom_e) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const int z = clamp_species(species[i], S);
  float acc = 0.0f;
  for (int c = lane; c < C; c += 32) acc = fmaf(W_out[(size_t)z * C + c], h[(size_t)i * D * C + c], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) atom_e[i] = (double)acc + (double)E0[z];
}

// g_e = dr r^ + (1/r)(I - r^ r^T) grad(Y . dY)
__global__ void edge_grad(int E, const float4* __restrict__ ev, const float* __restrict__ dY,
                          const float* __restrict__ dr, float4* __restrict__ g, const int* __restrict__ Edev) {
  if (Edev) E = *Edev;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const float4 v = ev[e];
    const float ir = 1.0f / v.w;
    const float x = v.x * ir, y = v.y * ir, z = v.z * ir;
    float d[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) d[k] = dY[(size_t)e * 16 + k];
    float gx, gy, gz;
    sh3_vjp<float>(x, y, z, d, gx, gy, gz);
    const float rad = gx * x + gy * y + gz * z;
    gx = (gx - rad * x) * ir;
    gy = (gy - rad * y) * ir;
    gz = (gz - rad * z) * ir;
    const float dre = dr[e];
    g[e] = make_float4(gx + dre * x, gy + dre * y, gz + dre * z, 0.0f);
  }
}

// F_i = sum_{e in seg(i)} (g_e - g_rev(e)) in FP64; per-atom virial
// sum_{e in seg(i)} x_e (x) g_e (FP64) when vir is not null.
// One warp per atom: lane l sums the atom's edges l, l + 32, ... in order and
// a fixed butterfly combines the lanes (the order depends only on the edge's
// position in the receiver's segment, so it is the same in any batch).
__global__ void forces_virial(int n, const int* __restrict__ row_ptr, const int* __restrict__ rev,
                              const float4* __restrict__ g, const float4* __restrict__ ev,
                              double* __restrict__ forces, double* __restrict__ vir) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double f[3] = {0, 0, 0};
  const int end = row_ptr[i + 1];
  for (int e = row_ptr[i] + lane; e < end; e += 32) {
    const float4 a = g[e], b = g[rev[e]], x = ev[e];
    f[0] += (double)a.x - (double)b.x;
    f[1] += (double)a.y - (double)b.y;
    f[2] += (double)a.z - (double)b.z;
    if (vir) {
      const double xe[3] = {x.x, x.y, x.z}, ge[3] = {a.x, a.y, a.z};
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) v[3 * p + q] += xe[p] * ge[q];
    }
  }
  // components: 3 forces then 9 virial entries; lane 2c ends with component c
  double w[16];
#pragma unroll
  for (int k = 0; k < 3; ++k) w[k] = f[k];
#pragma unroll
  for (int k = 0; k < 9; ++k) w[3 + k] = v[k];
#pragma unroll
  for (int k = 12; k < 16; ++k) w[k] = 0.0;
  const double tot = warp_reduce16_f64(w);
  const int comp = lane >> 1;
  if ((lane & 1) == 0) {
    if (comp < 3) forces[3 * i + comp] = tot;
    else if (comp < 12 && vir) vir[(size_t)i * 9 + comp - 3] = tot;
  }
}

}  // namespace

int launch_embed(int n, int C, int D, int S, const int* species, const float* W_emb, float* h, cudaStream_t st,
                 const int* sys_of, const float* emax, float* amax) {
  if (n <= 0) return MLIP_OK;
  if (amax && !emax) { set_error("embed: the per-species maxima are missing"); return MLIP_ERR_INVALID_ARG; }
  if (C % 4) { set_error("embed: channels must be a multiple of 4"); return MLIP_ERR_INVALID_ARG; }
  {
    MLIP_PROF("embed", st);
    embed<<<std::min<int64_t>(((int64_t)n * D * (C / 4) + 255) / 256, 16384), 256, 0, st>>>(n, C, D, S, species, W_emb, h,
                                                                                      sys_of, emax, amax);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_grad_init(int n, int C, int D, int S, const int* species, const float* W_out, float* G, cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  if (C % 4) { set_error("grad_init: channels must be a multiple of 4"); return MLIP_ERR_INVALID_ARG; }
  {
    MLIP_PROF("grad_init", st);
    grad_init<<<std::min<int64_t>(((int64_t)n * D * (C / 4) + 255) / 256, 16384), 256, 0, st>>>(n, C, D, S, species,
                                                                                               W_out, G);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_readout(int n, int C, int D, int S, const int* species, const float* W, const float* b0, const float* h,
                   double* out, cudaStream_t st) {
  if (n > 0) { MLIP_PROF("readout", st); readout<<<(n + 7) / 8, 256, 0, st>>>(n, C, D, S, species, W, b0, h, out); }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_energy(Workspace& ws, const SystemBatch& b, int C, int D, int S, const int* species, const float* W_out,
                  const float* E0, const float* h, double* atom_e, double* energy, cudaStream_t st) {
  MLIP_TRY(launch_readout((int)b.n, C, D, S, species, W_out, E0, h, atom_e, st));
  return launch_seg_sum(ws, b, 1, atom_e, false, energy, st);
}

int launch_edge_grad(int E, const float4* ev, const float* dY, const float* dr, float4* g, cudaStream_t st,
                     const int* Edev) {
  if (E <= 0) return MLIP_OK;
  { MLIP_PROF("edge_grad", st); edge_grad<<<std::min((E + 255) / 256, 8192), 256, 0, st>>>(E, ev, dY, dr, g, Edev); }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_forces_virial(Workspace& ws, const SystemBatch& b, const int* row_ptr, const int* rev, const float4* g,
                         const float4* ev, double* forces, double* stress, cudaStream_t st) {
  const int n = (int)b.n;
  double* vir = nullptr;
  if (stress) MLIP_TRY(ws.get("fv.vir", (size_t)std::max(n, 1) * 9, &vir));
  if (n > 0) {
    MLIP_PROF("forces_virial", st);
    forces_virial<<<(n + 3) / 4, 128, 0, st>>>(n, row_ptr, rev, g, ev, forces, vir);
    MLIP_LAUNCH_CHECK();
  }
  if (stress) MLIP_TRY(launch_seg_sum(ws, b, 9, vir, true, stress, st));
  return MLIP_OK;
}

}  // namespace mlip
