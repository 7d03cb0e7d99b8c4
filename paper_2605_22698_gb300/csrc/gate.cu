// Gated update with a species-dependent self-connection (NequIP's gate
// nonlinearity and self-connection on this layer's uniform natural-parity
// irreps), replacing the channel mix for models with gate = 1.  For node i of
// species z, channel c2, order l and l >= 1 gates q = (l - 1) C + c2:
//   pre_l = m_l W_l + h_l Wself[z][l]
//   g_q   = m_0 Wgate[:, q] + h_0 Wselfgate[z][:, q]
//   h'_0  = h_0 + silu(pre_0),   h'_l = h_l + sigmoid(g_l) pre_l
// and the adjoint, from G' = dE/dh':
//   dpre_0 = G'_0 silu'(pre_0),  dpre_l = G'_l sigmoid(g_l),
//   dg_l   = sigmoid'(g_l) sum_m G'_l,m pre_l,m
//   dE/dm_l = dpre_l W_l^T (+ dg Wgate^T on l = 0)
//   dE/dh_l = G'_l + dpre_l Wself[z][l]^T (+ dg Wselfgate[z]^T on l = 0)
// FP32 on the ALUs.  A block of C threads (one per output channel) takes 8
// nodes: their input rows are staged in shared memory and read by broadcast;
// each weight element is loaded once per block and used for all 8 nodes (the
// species weights once per species present in the block, masked per node).
// The adjoint reads transposed weight copies so that its loads are coalesced
// too, and stages the incoming gradient so that it can overwrite it in place.
#include <algorithm>

#include "kernels_common.cuh"
#include "launchers.cuh"
#include "mlip_internal.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

constexpr int kGN = 8;  // nodes per block

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + __expf(-x)); }

template <int L>
__global__ void __launch_bounds__(128) gate_fwd(int n, int C, int S, const int* __restrict__ species,
                                                const float* __restrict__ X, const float* __restrict__ X2,
                                                const float* __restrict__ hin, const float* __restrict__ Wm,
                                                const float* __restrict__ Ws, const float* __restrict__ Wg,
                                                const float* __restrict__ Wsg, float* __restrict__ hout,
                                                float* __restrict__ pre_out, float* __restrict__ g_out,
                                                const int* __restrict__ sys_of, float* __restrict__ out_max) {
  constexpr int D = (L + 1) * (L + 1);
  extern __shared__ __align__(16) float sm[];
  float* sM = sm;                     // [kGN][D][C] messages
  float* sH = sm + kGN * D * C;       // [kGN][D][C] features
  __shared__ int s_z[kGN];
  const int c2 = threadIdx.x, i0 = blockIdx.x * kGN;
  const int nk = min(kGN, n - i0);
  const int LC = L * C;
  for (int k = 0; k < kGN; ++k) {
    const bool live = k < nk;
    for (int r = 0; r < D; ++r) {
      const size_t o = ((size_t)(i0 + k) * D + r) * C + c2;
      sM[(k * D + r) * C + c2] = live ? X[o] + (X2 ? X2[o] : 0.0f) : 0.0f;
      sH[(k * D + r) * C + c2] = live ? hin[o] : 0.0f;
    }
  }
  if (c2 < kGN) s_z[c2] = c2 < nk ? clamp_species(species[i0 + c2], S) : -1;
  __syncthreads();
  // gates: sigmoid(g) for l = 1..L, this thread's channel
  float sg[kGN][L];
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    const int q = (l - 1) * C + c2;
    float acc[kGN];
#pragma unroll
    for (int k = 0; k < kGN; ++k) acc[k] = 0.0f;
    for (int c1 = 0; c1 < C; ++c1) {
      const float w = Wg[(size_t)c1 * LC + q];
#pragma unroll
      for (int k = 0; k < kGN; ++k) acc[k] = fmaf(sM[k * D * C + c1], w, acc[k]);
    }
    for (int z = 0; z < S; ++z) {
      bool any = false;
#pragma unroll
      for (int k = 0; k < kGN; ++k) any |= s_z[k] == z;
      if (!any) continue;  // uniform over the block
      const float* W = Wsg + (size_t)z * C * LC;
      for (int c1 = 0; c1 < C; ++c1) {
        const float w = W[(size_t)c1 * LC + q];
#pragma unroll
        for (int k = 0; k < kGN; ++k)
          if (s_z[k] == z) acc[k] = fmaf(sH[k * D * C + c1], w, acc[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kGN; ++k) {
      if (k < nk) g_out[(size_t)(i0 + k) * LC + q] = acc[k];
      sg[k][l - 1] = sigm(acc[k]);
    }
  }
  float m_run[kGN];
#pragma unroll
  for (int k = 0; k < kGN; ++k) m_run[k] = 0.0f;
  static_for<0, L + 1>([&](auto lc) {
    constexpr int l = decltype(lc)::value, R = 2 * l + 1;
    float acc[kGN][R];
#pragma unroll
    for (int k = 0; k < kGN; ++k)
#pragma unroll
      for (int mm = 0; mm < R; ++mm) acc[k][mm] = 0.0f;
    for (int c1 = 0; c1 < C; ++c1) {
      const float w = Wm[((size_t)l * C + c1) * C + c2];
#pragma unroll
      for (int k = 0; k < kGN; ++k)
#pragma unroll
        for (int mm = 0; mm < R; ++mm) acc[k][mm] = fmaf(sM[(k * D + l * l + mm) * C + c1], w, acc[k][mm]);
    }
    for (int z = 0; z < S; ++z) {
      bool any = false;
#pragma unroll
      for (int k = 0; k < kGN; ++k) any |= s_z[k] == z;
      if (!any) continue;
      const float* W = Ws + ((size_t)z * (L + 1) + l) * C * C;
      for (int c1 = 0; c1 < C; ++c1) {
        const float w = W[(size_t)c1 * C + c2];
#pragma unroll
        for (int k = 0; k < kGN; ++k)
          if (s_z[k] == z) {
#pragma unroll
            for (int mm = 0; mm < R; ++mm) acc[k][mm] = fmaf(sH[(k * D + l * l + mm) * C + c1], w, acc[k][mm]);
          }
      }
    }
#pragma unroll
    for (int k = 0; k < kGN; ++k) {
      if (k >= nk) continue;
#pragma unroll
      for (int mm = 0; mm < R; ++mm) {
        const size_t o = ((size_t)(i0 + k) * D + l * l + mm) * C + c2;
        const float p = acc[k][mm];
        pre_out[o] = p;
        float hv = sH[(k * D + l * l + mm) * C + c2];
        if constexpr (l == 0) hv += silu_f(p);
        else hv += sg[k][l - 1] * p;
        hout[o] = hv;
        m_run[k] = fmaxf(m_run[k], fabsf(hv));
      }
    }
  });
  if (out_max) {
#pragma unroll
    for (int k = 0; k < kGN; ++k)  // every lane of the warp takes node k together
      warp_sys_max(out_max, k < nk ? (sys_of ? sys_of[i0 + k] : 0) : -1, m_run[k]);
  }
}

// G (dE/dh', one or two buffers) -> Gm (dE/dm), and in place G <- dE/dh (G2 <- 0)
template <int L>
__global__ void __launch_bounds__(128) gate_bwd(int n, int C, int S, const int* __restrict__ species, float* G,
                                                float* G2, const float* __restrict__ pre, const float* __restrict__ gq,
                                                const float* __restrict__ WmT, const float* __restrict__ WsT,
                                                const float* __restrict__ WgT, const float* __restrict__ WsgT,
                                                float* __restrict__ Gm, const int* __restrict__ sys_of,
                                                float* __restrict__ out_max) {
  constexpr int D = (L + 1) * (L + 1);
  extern __shared__ __align__(16) float sm[];
  float* sP = sm;                     // [kGN][D][C] dE/dpre
  float* sG = sm + kGN * D * C;       // [kGN][D][C] dE/dh' (the residual)
  float* sDg = sm + 2 * kGN * D * C;  // [kGN][L C]  dE/dg
  __shared__ int s_z[kGN];
  const int c = threadIdx.x, i0 = blockIdx.x * kGN;
  const int nk = min(kGN, n - i0);
  const int LC = L * C;
  // phase 1: this thread's channel c as an output channel (c2)
  for (int k = 0; k < kGN; ++k) {
    const bool live = k < nk;
    float dg[L];
#pragma unroll
    for (int l = 0; l < L; ++l) dg[l] = 0.0f;
#pragma unroll
    for (int l = 0; l <= L; ++l) {
      const float s = (live && l > 0) ? sigm(gq[(size_t)(i0 + k) * LC + (l - 1) * C + c]) : 0.0f;
#pragma unroll
      for (int mm = 0; mm < 2 * l + 1; ++mm) {
        const int r = l * l + mm;
        const size_t o = ((size_t)(i0 + k) * D + r) * C + c;
        const float gv = live ? G[o] + (G2 ? G2[o] : 0.0f) : 0.0f;
        const float p = live ? pre[o] : 0.0f;
        sG[(k * D + r) * C + c] = gv;
        if (l == 0) {
          sP[(k * D + r) * C + c] = gv * silu_grad_f(p);
        } else {
          sP[(k * D + r) * C + c] = gv * s;
          dg[l - 1] = fmaf(gv, p, dg[l - 1]);
        }
      }
      if (l > 0) sDg[k * LC + (l - 1) * C + c] = dg[l - 1] * s * (1.0f - s);
    }
  }
  if (c < kGN) s_z[c] = c < nk ? clamp_species(species[i0 + c], S) : -1;
  __syncthreads();
  // phase 2: this thread's channel c as an input channel (c1)
  float m_run[kGN];
#pragma unroll
  for (int k = 0; k < kGN; ++k) m_run[k] = 0.0f;
  static_for<0, L + 1>([&](auto lc) {
    constexpr int l = decltype(lc)::value, R = 2 * l + 1;
    float am[kGN][R], ah[kGN][R];
#pragma unroll
    for (int k = 0; k < kGN; ++k)
#pragma unroll
      for (int mm = 0; mm < R; ++mm) am[k][mm] = ah[k][mm] = 0.0f;
    for (int c2 = 0; c2 < C; ++c2) {
      const float w = WmT[((size_t)l * C + c2) * C + c];
#pragma unroll
      for (int k = 0; k < kGN; ++k)
#pragma unroll
        for (int mm = 0; mm < R; ++mm) am[k][mm] = fmaf(sP[(k * D + l * l + mm) * C + c2], w, am[k][mm]);
    }
    for (int z = 0; z < S; ++z) {
      bool any = false;
#pragma unroll
      for (int k = 0; k < kGN; ++k) any |= s_z[k] == z;
      if (!any) continue;
      const float* W = WsT + ((size_t)z * (L + 1) + l) * C * C;
      for (int c2 = 0; c2 < C; ++c2) {
        const float w = W[(size_t)c2 * C + c];
#pragma unroll
        for (int k = 0; k < kGN; ++k)
          if (s_z[k] == z) {
#pragma unroll
            for (int mm = 0; mm < R; ++mm) ah[k][mm] = fmaf(sP[(k * D + l * l + mm) * C + c2], w, ah[k][mm]);
          }
      }
    }
    if constexpr (l == 0) {  // the gates feed on the scalar rows
      for (int q = 0; q < LC; ++q) {
        const float w = WgT[(size_t)q * C + c];
#pragma unroll
        for (int k = 0; k < kGN; ++k) am[k][0] = fmaf(sDg[k * LC + q], w, am[k][0]);
      }
      for (int z = 0; z < S; ++z) {
        bool any = false;
#pragma unroll
        for (int k = 0; k < kGN; ++k) any |= s_z[k] == z;
        if (!any) continue;
        const float* W = WsgT + (size_t)z * LC * C;
        for (int q = 0; q < LC; ++q) {
          const float w = W[(size_t)q * C + c];
#pragma unroll
          for (int k = 0; k < kGN; ++k)
            if (s_z[k] == z) ah[k][0] = fmaf(sDg[k * LC + q], w, ah[k][0]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kGN; ++k) {
      if (k >= nk) continue;
#pragma unroll
      for (int mm = 0; mm < R; ++mm) {
        const int r = l * l + mm;
        const size_t o = ((size_t)(i0 + k) * D + r) * C + c;
        Gm[o] = am[k][mm];
        m_run[k] = fmaxf(m_run[k], fabsf(am[k][mm]));
        G[o] = sG[(k * D + r) * C + c] + ah[k][mm];
        if (G2) G2[o] = 0.0f;
      }
    }
  });
  if (out_max) {
#pragma unroll
    for (int k = 0; k < kGN; ++k)
      warp_sys_max(out_max, k < nk ? (sys_of ? sys_of[i0 + k] : 0) : -1, m_run[k]);
  }
}

size_t fwd_smem(int L, int C) { return (size_t)2 * kGN * (L + 1) * (L + 1) * C * sizeof(float); }
size_t bwd_smem(int L, int C) { return ((size_t)2 * kGN * (L + 1) * (L + 1) * C + (size_t)kGN * L * C) * sizeof(float); }

}  // namespace

// Shared-memory limits of the kernels for a model's order (set at model
// creation, outside any stream capture), at the widest supported channel count
// so that models of different widths never lower each other's limit.
int gate_prepare(int L, int C) {
  (void)C;
  C = 128;
  if (L == 2) {
    MLIP_CUDA_TRY(cudaFuncSetAttribute(gate_fwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(2, C)));
    MLIP_CUDA_TRY(cudaFuncSetAttribute(gate_bwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem(2, C)));
  } else {
    MLIP_CUDA_TRY(cudaFuncSetAttribute(gate_fwd<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(3, C)));
    MLIP_CUDA_TRY(cudaFuncSetAttribute(gate_bwd<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem(3, C)));
  }
  return MLIP_OK;
}

int launch_gate_fwd(int L, int n, int C, int S, const int* species, const float* X, const float* X2,
                    const float* hin, const float* Wm, const float* Ws, const float* Wg, const float* Wsg,
                    float* hout, float* pre, float* g, const int* sys_of, float* out_max, cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  if (C > 128 || C % 32) { set_error("gated update: channels must be 32, 64 or 128"); return MLIP_ERR_INVALID_ARG; }
  const size_t sm = fwd_smem(L, C);
  const int grid = (n + kGN - 1) / kGN;
  MLIP_PROF("gate_fwd", st);
  if (L == 2) gate_fwd<2><<<grid, C, sm, st>>>(n, C, S, species, X, X2, hin, Wm, Ws, Wg, Wsg, hout, pre, g, sys_of, out_max);
  else gate_fwd<3><<<grid, C, sm, st>>>(n, C, S, species, X, X2, hin, Wm, Ws, Wg, Wsg, hout, pre, g, sys_of, out_max);
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_gate_bwd(int L, int n, int C, int S, const int* species, float* G, float* G2, const float* pre,
                    const float* g, const float* WmT, const float* WsT, const float* WgT, const float* WsgT,
                    float* Gm, const int* sys_of, float* out_max, cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  if (C > 128 || C % 32) { set_error("gated update: channels must be 32, 64 or 128"); return MLIP_ERR_INVALID_ARG; }
  const size_t sm = bwd_smem(L, C);
  const int grid = (n + kGN - 1) / kGN;
  MLIP_PROF("gate_bwd", st);
  if (L == 2) gate_bwd<2><<<grid, C, sm, st>>>(n, C, S, species, G, G2, pre, g, WmT, WsT, WgT, WsgT, Gm, sys_of, out_max);
  else gate_bwd<3><<<grid, C, sm, st>>>(n, C, S, species, G, G2, pre, g, WmT, WsT, WgT, WsgT, Gm, sys_of, out_max);
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace mlip
