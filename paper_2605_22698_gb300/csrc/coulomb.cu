// Charge head, charge correction and long-range Coulomb term for models with
// charges = 1 (Sec. "Treatment of electrostatics and long-range interactions").
//
//   q_i  = W_q[z_i] . h^T_i,0 + q0[z_i]                         charge head
//   qt_i = q_i - (sum_{j in S} q_j - Q_S) / N_S                  Eq. charge_correction
//   E_LR = k sum_{i<j in S} qt_i qt_j / chi(r_ij)                Eq. long_range_interaction
// with k = e^2 / (4 pi eps0) in eV A and PhysNet's surrogate distance
//   1/chi(r) = phi(x) / sqrt(r^2 + 1) + (1 - phi(x)) / r,  x = r / r0,
//   phi(x) = 1 - 10 x^3 + 15 x^4 - 6 x^5 (x < 1), 0 otherwise
// (equal to 1/r beyond the soft-core radius r0).  All pairs of each system
// (open systems only: no periodic images).  The adjoint: dE/dqt_i = gt_i =
// k sum_j qt_j / chi(r_ij); through the correction dE/dq_i = gt_i - mean_S(gt),
// which enters the network's adjoint as dE/dh^T_i,0 += dE/dq_i W_q[z_i]; the
// direct forces at fixed charges are added to the network's forces.
//
// coulomb_prep writes every atom's corrected charge and its coordinates as
// FP32 pairs hi + lo (hi = fp32(x), lo = fp32(x - hi)), so that the pair loop
// forms d = (hi_j - hi_i) + (lo_j - lo_i) in FP32 to within an FP32 rounding
// of the exact difference without the narrow FP64 pipe.  coulomb_pairs: one
// warp per atom i, lanes over the atoms j of its system (j - first = lane mod
// 32, so a system's sums do not depend on its batch); pair terms in FP32,
// folded into FP64 every 16 terms per lane, FP64 warp reduction.
#include <algorithm>

#include "kernels_common.cuh"
#include "launchers.cuh"
#include "mlip_internal.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

constexpr double kCoulombK = 14.3996454784;  // e^2 / (4 pi eps0), eV A

// 1/chi(r) and (d/dr 1/chi) / r, in forms without cancellation at small r:
//   (1 - phi) / r   = x^2 (10 - 15 x + 6 x^2) / r0
//   (1/chi)' / r    = -30 x (1-x)^2 / (r0^2 s) + 30 (1-x)^2 / r0^3 - phi / s^3 - (10 - 15 x + 6 x^2) / r0^3
// with s = sqrt(r^2 + 1); beyond r0: 1/r and -1/r^3.
__device__ __forceinline__ void inv_chi(float r, float r0, float& f, float& fpr) {
  if (r >= r0) {
    const float ir = 1.0f / r;
    f = ir;
    fpr = -ir * ir * ir;
    return;
  }
  const float x = r / r0, ir0 = 1.0f / r0;
  const float poly = 10.0f + x * (-15.0f + 6.0f * x);  // (1 - phi) / x^3
  const float phi = 1.0f - x * x * x * poly;
  const float is = rsqrtf(fmaf(r, r, 1.0f));
  const float om = (1.0f - x) * (1.0f - x);
  f = phi * is + x * x * poly * ir0;
  const float ir03 = ir0 * ir0 * ir0;
  fpr = -30.0f * x * om * ir0 * ir0 * is + 30.0f * om * ir03 - phi * is * is * is - poly * ir03;
}

constexpr int kCWarps = 8;

// qt_i = q_i - (qsum_s - Q_s) / N_s; hi/lo coordinates with the FP32 charge in hi.w
__global__ void coulomb_prep(int n, const double* __restrict__ pos, const double* __restrict__ q,
                             const double* __restrict__ qsum, const double* __restrict__ qtot,
                             const int* __restrict__ atom_off, const int* __restrict__ sys_of,
                             double* __restrict__ qt_out, float4* __restrict__ phi, float4* __restrict__ plo) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = sys_of ? sys_of[i] : 0;
    const double qt = q[i] - (qsum[s] - qtot[s]) / (double)(atom_off[s + 1] - atom_off[s]);
    qt_out[i] = qt;
    float h[3], l[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double x = pos[3 * i + k];
      h[k] = (float)x;
      l[k] = (float)(x - (double)h[k]);
    }
    phi[i] = make_float4(h[0], h[1], h[2], (float)qt);
    plo[i] = make_float4(l[0], l[1], l[2], 0.0f);
  }
}

// gt, e (added to atom_e), Fc [n][3] for every atom
__global__ void __launch_bounds__(32 * kCWarps) coulomb_pairs(int n, const float4* __restrict__ phi,
                                                              const float4* __restrict__ plo,
                                                              const double* __restrict__ qt,
                                                              const int* __restrict__ atom_off,
                                                              const int* __restrict__ sys_of, float r0,
                                                              double* __restrict__ gt_out, double* __restrict__ atom_e,
                                                              double* __restrict__ Fc) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kCWarps + (threadIdx.x >> 5);
  if (i >= n) return;  // uniform over the warp
  const int s = sys_of ? sys_of[i] : 0;
  const int j0 = atom_off[s], j1 = atom_off[s + 1];
  const float4 hi = phi[i], lo = plo[i];
  double g = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
  float g32 = 0.0f, fx32 = 0.0f, fy32 = 0.0f, fz32 = 0.0f;
  int cnt = 0;
  for (int j = j0 + lane; j < j1; j += 32) {
    if (j != i) {
      const float4 hj = phi[j], lj = plo[j];
      const float dx = (hj.x - hi.x) + (lj.x - lo.x), dy = (hj.y - hi.y) + (lj.y - lo.y),
                  dz = (hj.z - hi.z) + (lj.z - lo.z);
      const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
      float f, fpr;
      inv_chi(r, r0, f, fpr);
      const float qj = hj.w;
      g32 = fmaf(qj, f, g32);
      const float a = qj * fpr;
      fx32 = fmaf(a, dx, fx32);
      fy32 = fmaf(a, dy, fy32);
      fz32 = fmaf(a, dz, fz32);
    }
    if (++cnt == 16) {
      g += g32; fx += fx32; fy += fy32; fz += fz32;
      g32 = fx32 = fy32 = fz32 = 0.0f;
      cnt = 0;
    }
  }
  g += g32; fx += fx32; fy += fy32; fz += fz32;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    g += __shfl_xor_sync(0xffffffffu, g, o);
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o);
  }
  if (lane == 0) {
    const double qi = qt[i];
    const double gt = kCoulombK * g;
    gt_out[i] = gt;
    atom_e[i] += 0.5 * qi * gt;
    // F_i = -dE/dr_i = k qt_i sum_j qt_j (1/chi)'(r) / r (r_j - r_i)
    Fc[3 * i] = kCoulombK * qi * fx;
    Fc[3 * i + 1] = kCoulombK * qi * fy;
    Fc[3 * i + 2] = kCoulombK * qi * fz;
  }
}

// G[i][0][c] += (gt_i - gsum_s / N_s) W_q[z_i][c]
__global__ void charge_grad(int n, int C, int D, int S, const int* __restrict__ species, const float* __restrict__ W_q,
                            const double* __restrict__ gt, const double* __restrict__ gsum,
                            const int* __restrict__ atom_off, const int* __restrict__ sys_of, float* __restrict__ G) {
  const long long total = (long long)n * C;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k / C), c = (int)(k - (long long)i * C);
    const int s = sys_of ? sys_of[i] : 0;
    const double dq = gt[i] - gsum[s] / (double)(atom_off[s + 1] - atom_off[s]);
    G[(size_t)i * D * C + c] += (float)dq * W_q[(size_t)clamp_species(species[i], S) * C + c];
  }
}

__global__ void add_f64(long long m, const double* __restrict__ a, double* __restrict__ out) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (long long)gridDim.x * blockDim.x)
    out[k] += a[k];
}

struct Bufs {
  double *q, *qt, *gt, *Fc, *qsum, *gsum;
  float4 *phi, *plo;
};

int get_bufs(Workspace& ws, const SystemBatch& b, Bufs* B) {
  const size_t n = (size_t)std::max<int64_t>(b.n, 1), ns = (size_t)std::max(b.nsys, 1);
  MLIP_TRY(ws.get("cq.q", n, &B->q));
  MLIP_TRY(ws.get("cq.qt", n, &B->qt));
  MLIP_TRY(ws.get("cq.gt", n, &B->gt));
  MLIP_TRY(ws.get("cq.Fc", 3 * n, &B->Fc));
  MLIP_TRY(ws.get("cq.qsum", ns, &B->qsum));
  MLIP_TRY(ws.get("cq.gsum", ns, &B->gsum));
  MLIP_TRY(ws.get("cq.phi", n, &B->phi));
  MLIP_TRY(ws.get("cq.plo", n, &B->plo));
  return MLIP_OK;
}

}  // namespace

int coulomb_forward(Workspace& ws, const SystemBatch& b, const mlip_model* M, const double* d_pos,
                    const int* species, const float* hT, double* atom_e, cudaStream_t st) {
  if (b.any_pbc()) { set_error("the Coulomb term of a model with charges needs open systems"); return MLIP_ERR_CELL; }
  Bufs B;
  MLIP_TRY(get_bufs(ws, b, &B));
  const int n = (int)b.n;
  MLIP_TRY(launch_readout(n, M->C, M->D, M->S, species, M->W_q, M->q0, hT, B.q, st));
  MLIP_TRY(launch_seg_sum(ws, b, 1, B.q, false, B.qsum, st));
  if (n > 0) {
    {
      MLIP_PROF("coulomb_prep", st);
      coulomb_prep<<<std::min((n + 255) / 256, 4096), 256, 0, st>>>(n, d_pos, B.q, B.qsum, b.d_qtot, b.d_atom_off,
                                                                      b.d_sys_of, B.qt, B.phi, B.plo);
    }
    MLIP_LAUNCH_CHECK();
    MLIP_PROF("coulomb_pairs", st);
    coulomb_pairs<<<(n + kCWarps - 1) / kCWarps, 32 * kCWarps, 0, st>>>(n, B.phi, B.plo, B.qt, b.d_atom_off,
                                                                        b.d_sys_of, (float)M->r0, B.gt, atom_e, B.Fc);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int coulomb_adjoint(Workspace& ws, const SystemBatch& b, const mlip_model* M, const int* species, float* G,
                    cudaStream_t st) {
  Bufs B;
  MLIP_TRY(get_bufs(ws, b, &B));
  const int n = (int)b.n;
  MLIP_TRY(launch_seg_sum(ws, b, 1, B.gt, false, B.gsum, st));
  if (n > 0) {
    MLIP_PROF("charge_grad", st);
    const long long total = (long long)n * M->C;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    charge_grad<<<grid, 256, 0, st>>>(n, M->C, M->D, M->S, species, M->W_q, B.gt, B.gsum, b.d_atom_off, b.d_sys_of,
                                      G);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int coulomb_add_forces(Workspace& ws, const SystemBatch& b, double* forces, cudaStream_t st) {
  Bufs B;
  MLIP_TRY(get_bufs(ws, b, &B));
  const long long m = 3LL * b.n;
  if (m > 0) {
    MLIP_PROF("coulomb_add_forces", st);
    add_f64<<<(int)std::min<long long>((m + 255) / 256, 4096), 256, 0, st>>>(m, B.Fc, forces);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int coulomb_charges(Workspace& ws, const SystemBatch& b, double** q) {
  Bufs B;
  MLIP_TRY(get_bufs(ws, b, &B));
  *q = B.qt;
  return MLIP_OK;
}

}  // namespace mlip
