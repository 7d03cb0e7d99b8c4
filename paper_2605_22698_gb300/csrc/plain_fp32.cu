// The plain FP32 form of the interaction layer and its adjoint.
//
// Every product runs on the FP32 ALUs; the per-edge radial weights of each
// layer (E x paths x C) are materialised in HBM by a SIMT GEMM and kept for
// the backward pass (stored intermediates).  Steps, per layer t:
//   radial_fwd   b_e = Bessel x envelope, z2 = silu(W2^T silu(W1^T b_e))    (per edge)
//   sgemm        w = z2 W3                                                  [E x P*C]
//   tp_fwd       m_i = s sum_{e: recv=i} TP(h_send, Y_e, w_e)  (segmented, no atomics)
//   mix_fwd      u = m W_l; h_0 += silu(u_0); h_l += u_l
// energy E = sum_i W_out[z_i] . h_i,0 + E0[z_i] (FP64 sum).  Adjoint, t = T..1:
//   mix_bwd      Gm = (G * silu'(u_0) | G) W_l^T
//   tp_bwd       per receiver j: G^{t-1}_j = G^t_j + s sum TP^T over its
//                reverse edges (Y(-r^) = (-1)^l2 Y(r^)); per edge dE/dw and
//                dE/dY (channel sums)
//   sgemm        dE/dz2 = (dE/dw) W3^T
//   radial_bwd   dE/dr through the MLP and the basis
// then g_e = dE/dr r^ + (1/r)(I - r^ r^T) grad_Y . dE/dY, F_i = sum_{recv=i}
// (g_e - g_rev(e)) and the virial sum_e x_e (x) g_e in FP64.
#include <algorithm>
#include <type_traits>

#include "kernels_common.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

constexpr int kNT = 32;  // edges per shared-memory sub-tile

// ------------------------------------------------------------ edge geometry
// ev[e] = edge_vector(e) (kernels_common.cuh)
__global__ void edge_geom(int E, const double* __restrict__ pos, const int* __restrict__ recv,
                          const int* __restrict__ send, const int8_t* __restrict__ shift, CellArg cell,
                          float4* __restrict__ ev, const int* __restrict__ Edev) {
  if (Edev) E = *Edev;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
    ev[e] = edge_vector(e, pos, recv, send, shift, cell);
}

// --------------------------------------------------------------- radial MLP
// One thread per edge.  z2T is [H][ldz] (edge index contiguous).
template <int H>
__global__ void radial_fwd(int E, const float4* __restrict__ ev, const float* __restrict__ W1,
                           const float* __restrict__ W2, float rc, int p, float* __restrict__ z2T, int ldz) {
  __shared__ float sW1[8 * H], sW2[H * H];
  for (int k = threadIdx.x; k < 8 * H; k += blockDim.x) sW1[k] = W1[k];
  for (int k = threadIdx.x; k < H * H; k += blockDim.x) sW2[k] = W2[k];
  __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const float r = ev[e].w;
  float b[8], db[8];
  radial_basis<8, false>(r, rc, p, b, db);
  float z1[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    float a = 0.0f;
#pragma unroll
    for (int n = 0; n < 8; ++n) a = fmaf(b[n], sW1[n * H + k], a);
    z1[k] = silu_f(a);
  }
  for (int k = 0; k < H; ++k) {
    float a = 0.0f;
#pragma unroll
    for (int q = 0; q < H; ++q) a = fmaf(z1[q], sW2[q * H + k], a);
    z2T[(size_t)k * ldz + e] = silu_f(a);
  }
}

// dE/dr through the MLP and basis: dz2 [E][H] (row-major) -> dr_tot[e] += dE/dr.
template <int H>
__global__ void radial_bwd(int E, const float4* __restrict__ ev, const float* __restrict__ W1,
                           const float* __restrict__ W2, float rc, int p, const float* __restrict__ dz2,
                           float* __restrict__ dr_tot) {
  __shared__ __align__(16) float sW1[8 * H], sW2[H * H];
  for (int k = threadIdx.x; k < 8 * H; k += blockDim.x) sW1[k] = W1[k];
  for (int k = threadIdx.x; k < H * H; k += blockDim.x) sW2[k] = W2[k];
  __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const float r = ev[e].w;
  float b[8], db[8];
  radial_basis<8, true>(r, rc, p, b, db);
  // z1 = silu(W1^T b); da2 = dz2 * silu'(W2^T z1); then per hidden unit k:
  // dz1_k = sum_q W2[k][q] da2[q], da1_k = dz1_k silu'(a1_k) (a1_k recomputed)
  float z1[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    float a = 0.0f;
#pragma unroll
    for (int n = 0; n < 8; ++n) a = fmaf(b[n], sW1[n * H + k], a);
    z1[k] = silu_f(a);
  }
  float da2[H];
#pragma unroll
  for (int q = 0; q < H; ++q) da2[q] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < H; ++k) {  // a2 = z1 W2, one 16-byte row load per four FMAs
    const float zk = z1[k];
    const float4* w4 = reinterpret_cast<const float4*>(sW2 + k * H);
#pragma unroll
    for (int q4 = 0; q4 < H / 4; ++q4) {
      const float4 w = w4[q4];
      da2[4 * q4] = fmaf(zk, w.x, da2[4 * q4]);
      da2[4 * q4 + 1] = fmaf(zk, w.y, da2[4 * q4 + 1]);
      da2[4 * q4 + 2] = fmaf(zk, w.z, da2[4 * q4 + 2]);
      da2[4 * q4 + 3] = fmaf(zk, w.w, da2[4 * q4 + 3]);
    }
  }
#pragma unroll
  for (int q = 0; q < H; ++q) da2[q] = dz2[(size_t)e * H + q] * silu_grad_f(da2[q]);
  float dr = 0.0f;
#pragma unroll 4
  for (int k = 0; k < H; ++k) {
    float a = 0.0f, bd = 0.0f;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      a = fmaf(b[n], sW1[n * H + k], a);
      bd = fmaf(sW1[n * H + k], db[n], bd);
    }
    float dz1 = 0.0f;
    const float4* w4 = reinterpret_cast<const float4*>(sW2 + k * H);
#pragma unroll
    for (int q4 = 0; q4 < H / 4; ++q4) {
      const float4 w = w4[q4];
      dz1 = fmaf(w.x, da2[4 * q4], dz1);
      dz1 = fmaf(w.y, da2[4 * q4 + 1], dz1);
      dz1 = fmaf(w.z, da2[4 * q4 + 2], dz1);
      dz1 = fmaf(w.w, da2[4 * q4 + 3], dz1);
    }
    dr = fmaf(dz1 * silu_grad_f(a), bd, dr);
  }
  dr_tot[e] += dr;
}

// ------------------------------------------------------------------- SGEMM
// C[M][N] (row-major, ldc) = A * B, FP32 SIMT, 128 x 128 tiles, 8 x 8 per thread.
// A_KM: A stored [K][M] (lda) else [M][K]; B_NK: B stored [N][K] (ldb) else [K][N].
// M is read from *M_dev when non-null (device-resident edge count).
template <bool A_KM, bool B_NK>
__global__ void __launch_bounds__(256) sgemm(int M, const int* M_dev, int N, int K, const float* __restrict__ A,
                                             int lda, const float* __restrict__ B, int ldb,
                                             float* __restrict__ C, int ldc) {
  if (M_dev) M = *M_dev;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * 128;
  if (m0 >= M) return;
  __shared__ __align__(16) float As[8][128];
  __shared__ __align__(16) float Bs[8][128];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += 8) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + q * 256;  // 0..1023
      int kk, mm;
      if (A_KM) { kk = idx >> 7; mm = idx & 127; }
      else { mm = idx >> 3; kk = idx & 7; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.0f;
      if (gm < M && gk < K) v = A_KM ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = v;
      int kb, nn;
      if (B_NK) { nn = idx >> 3; kb = idx & 7; }
      else { kb = idx >> 7; nn = idx & 127; }
      const int gn = n0 + nn, gkb = k0 + kb;
      float w = 0.0f;
      if (gn < N && gkb < K) w = B_NK ? B[(size_t)gn * ldb + gkb] : B[(size_t)gkb * ldb + gn];
      Bs[kb][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 4 + 64]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4 + 64]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + tx * 4 + (j & 3) + (j >> 2) * 64;
      if (gn < N) C[(size_t)gm * ldc + gn] = acc[i][j];
    }
  }
}

// -------------------------------------------------------- TP forward (plain)
// One block per balanced receiver range; thread c owns channel c.  Per
// sub-tile of kNT edges the per-edge products c_k Y[e2_k] of every used CG
// entry are staged in shared memory; each thread then walks the edges in
// order, gathers the sender's features for its channel, and accumulates the
// receiver's message in registers, flushed (times s) at segment ends.
// FIRST: only the l1 = 0 paths (input features are scalars).
// PAR (mixed-parity models): every triangle-valid path (CGTableP); a path with
// odd l2 reads the sender's channel of the other parity block, cx = (c + C/2) % C.
template <int L, bool FIRST, bool PAR = false>
__global__ void tp_fwd(int n, int C, const int* __restrict__ row_ptr, const int* __restrict__ recv,
                       const int* __restrict__ send, const float4* __restrict__ ev, const float* __restrict__ h,
                       const float* __restrict__ w, int PW, float s, float* __restrict__ m) {
  using Tab = std::conditional_t<PAR, CGTableP<L>, CGTable<L>>;
  using PI = PathInfo<L>;
  constexpr int D = NodeDims<L>::D;
  constexpr int NP = FIRST ? PI::P0 : Tab::P;
  constexpr int NZ = FIRST ? Tab::off[PI::P0] : Tab::NNZ;
  constexpr int NZP = (NZ + 3) & ~3;
  constexpr int DH = FIRST ? 1 : D;  // sender components read
  __shared__ __align__(16) float cY[kNT * NZP];
  __shared__ int s_send[kNT], s_recv[kNT];

  int i0, i1;
  block_receivers(row_ptr, n, blockIdx.x, gridDim.x, &i0, &i1);
  const int E0 = row_ptr[i0], E1 = row_ptr[i1];
  const int c = threadIdx.x;
  const bool active = c < C;
  float acc[D];
#pragma unroll
  for (int d = 0; d < D; ++d) acc[d] = 0.0f;
  int cur = i0;
  auto flush = [&](int i) {
    if (active) {
#pragma unroll
      for (int d = 0; d < D; ++d) m[((size_t)i * D + d) * C + c] = s * acc[d];
    }
#pragma unroll
    for (int d = 0; d < D; ++d) acc[d] = 0.0f;
  };
  for (int e0 = E0; e0 < E1; e0 += kNT) {
    const int nt = min(kNT, E1 - e0);
    __syncthreads();
    if (threadIdx.x < nt) {
      const int e = e0 + threadIdx.x;
      const float4 v = ev[e];
      const float ir = 1.0f / v.w;
      float Y[16];
      sh3<float>(v.x * ir, v.y * ir, v.z * ir, Y);
      float* dst = cY + threadIdx.x * NZP;
      static_for<0, NZ>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr float cv = Tab::ec[k];
        constexpr int i2 = Tab::e2[k];
        dst[k] = cv * Y[i2];
      });
      s_send[threadIdx.x] = send[e];
      s_recv[threadIdx.x] = recv[e];
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
      const int r = s_recv[t];
      while (cur < r) { flush(cur); ++cur; }
      const int j = s_send[t];
      float hj[DH], hx[PAR ? DH : 1], wp[NP];
#pragma unroll
      for (int d = 0; d < DH; ++d) hj[d] = active ? h[((size_t)j * D + d) * C + c] : 0.0f;
      if constexpr (PAR) {
        const int cx = (c + C / 2) % C;
#pragma unroll
        for (int d = 0; d < DH; ++d) hx[d] = active ? h[((size_t)j * D + d) * C + cx] : 0.0f;
      }
      const float* wrow = w + (size_t)(e0 + t) * PW * C;
#pragma unroll
      for (int p = 0; p < NP; ++p) wp[p] = active ? wrow[p * C + c] : 0.0f;
      const float* cy = cY + t * NZP;
      static_for<0, NP>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        constexpr int l1 = Tab::l1[p];
        constexpr bool swap = PAR && (Tab::l2[p] & 1);
        constexpr int kb = Tab::off[p], ke = Tab::off[p + 1];
        float wh[2 * l1 + 1];
#pragma unroll
        for (int q = 0; q < 2 * l1 + 1; ++q) wh[q] = wp[p] * (swap ? hx[l1 * l1 + q] : hj[l1 * l1 + q]);
        static_for<kb, ke>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          constexpr int i3 = Tab::e3[k], j1 = Tab::e1[k] - l1 * l1;
          acc[i3] = fmaf(cy[k], wh[j1], acc[i3]);
        });
      });
    }
  }
  while (cur < i1) { flush(cur); ++cur; }
}

// ------------------------------------------------------- TP backward (plain)
// Receiver-segment pass of the adjoint for one layer.  For receiver j and each
// of its edges e (sender i):
//   G^{t-1}_j[l1 m1] += s w_e[p] (-1)^{l2} C^p[m3][m1][m2] Y_e[l2 m2] Gm_i[l3 m3]   (not FIRST)
//   with Gt = s Gm_j:  T_p[m2] = sum_entries C h_i[l1 m1] Gt[l3 m3]
//   dE/dw_e[p] = sum_m2 Y_e[l2 m2] T_p[m2];   dE/dY_e[l2 m2] += sum_c w_e[p] T_p[m2]
// PAR: for a path with odd l2 the forward coupled output channel c to input
// channel cx = (c + C/2) % C, so thread c's dE/dw and dE/dY read the sender's
// cx, and its reverse-edge term for the receiver's channel c takes w and Gm of
// channel cx (the channel whose input c was).
template <int L, bool FIRST, bool PAR = false>
__global__ void tp_bwd(int n, int C, const int* __restrict__ row_ptr, const int* __restrict__ recv,
                       const int* __restrict__ send, const float4* __restrict__ ev,
                       const float* __restrict__ hprev, const float* __restrict__ Gm,
                       const float* __restrict__ w, int PW, float s, const float* __restrict__ Gin,
                       float* __restrict__ Gout, float* __restrict__ dw, float* __restrict__ dY) {
  using Tab = std::conditional_t<PAR, CGTableP<L>, CGTable<L>>;
  using PI = PathInfo<L>;
  constexpr int D = NodeDims<L>::D;
  constexpr int NP = FIRST ? PI::P0 : Tab::P;
  constexpr int NZ = FIRST ? Tab::off[PI::P0] : Tab::NNZ;
  constexpr int NZP = (NZ + 3) & ~3;
  constexpr int DH = FIRST ? 1 : D;
  __shared__ __align__(16) float cY[kNT * NZP];
  __shared__ __align__(16) float sY[kNT * 16];
  __shared__ int s_send[kNT], s_recv[kNT];
  __shared__ float red[4][kNT][16];

  int i0, i1;
  block_receivers(row_ptr, n, blockIdx.x, gridDim.x, &i0, &i1);
  const int E0 = row_ptr[i0], E1 = row_ptr[i1];
  const int c = threadIdx.x, lane = c & 31, warp = c >> 5;
  const int nwarps = blockDim.x >> 5;
  const bool active = c < C;
  float Gacc[D], Gt[D];
#pragma unroll
  for (int d = 0; d < D; ++d) { Gacc[d] = 0.0f; Gt[d] = 0.0f; }
  int cur = -1;
  auto flush = [&](int i) {
    if (!FIRST && active) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const size_t o = ((size_t)i * D + d) * C + c;
        Gout[o] = Gin[o] + Gacc[d];
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) Gacc[d] = 0.0f;
  };
  auto enter = [&](int i) {
#pragma unroll
    for (int d = 0; d < D; ++d) Gt[d] = active ? s * Gm[((size_t)i * D + d) * C + c] : 0.0f;
  };
  // receivers without edges still need G^{t-1} = G^t
  auto advance = [&](int r) {
    while (cur < r) {
      if (cur >= i0) flush(cur);
      ++cur;
      if (cur < i1) enter(cur);
    }
  };
  cur = i0 - 1;
  for (int e0 = E0; e0 < E1; e0 += kNT) {
    const int nt = min(kNT, E1 - e0);
    __syncthreads();
    if (threadIdx.x < nt) {
      const int e = e0 + threadIdx.x;
      const float4 v = ev[e];
      const float ir = 1.0f / v.w;
      float Y[16];
      sh3<float>(v.x * ir, v.y * ir, v.z * ir, Y);
#pragma unroll
      for (int k = 0; k < 16; ++k) sY[threadIdx.x * 16 + k] = Y[k];
      if (!FIRST) {
        float* dst = cY + threadIdx.x * NZP;
        static_for<0, NZ>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          constexpr float cv = ((Tab::l2[Tab::ep[k]] & 1) ? -1.0f : 1.0f) * Tab::ec[k];
          constexpr int i2 = Tab::e2[k];
          dst[k] = cv * Y[i2];
        });
      }
      s_send[threadIdx.x] = send[e];
      s_recv[threadIdx.x] = recv[e];
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
      advance(s_recv[t]);
      const int i = s_send[t];
      const int cx = PAR ? (c + C / 2) % C : c;
      float hi[DH], hix[PAR ? DH : 1], wp[NP], wpx[PAR ? NP : 1], Y[16];
#pragma unroll
      for (int d = 0; d < DH; ++d) hi[d] = active ? hprev[((size_t)i * D + d) * C + c] : 0.0f;
      const float* wrow = w + (size_t)(e0 + t) * PW * C;
#pragma unroll
      for (int p = 0; p < NP; ++p) wp[p] = active ? wrow[p * C + c] : 0.0f;
      if constexpr (PAR) {
#pragma unroll
        for (int d = 0; d < DH; ++d) hix[d] = active ? hprev[((size_t)i * D + d) * C + cx] : 0.0f;
#pragma unroll
        for (int p = 0; p < NP; ++p) wpx[p] = active ? wrow[p * C + cx] : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) Y[k] = sY[t * 16 + k];
      float dYp[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) dYp[k] = 0.0f;
      float* dwrow = dw + (size_t)(e0 + t) * PW * C;
      if (!FIRST) {
        float Gi[D], Gix[PAR ? D : 1];
#pragma unroll
        for (int d = 0; d < D; ++d) Gi[d] = active ? Gm[((size_t)i * D + d) * C + c] : 0.0f;
        if constexpr (PAR) {
#pragma unroll
          for (int d = 0; d < D; ++d) Gix[d] = active ? Gm[((size_t)i * D + d) * C + cx] : 0.0f;
        }
        const float* cy = cY + t * NZP;
        static_for<0, NP>([&](auto pc) {
          constexpr int p = decltype(pc)::value;
          constexpr int l3 = Tab::l3[p];
          constexpr bool swap = PAR && (Tab::l2[p] & 1);
          constexpr int kb = Tab::off[p], ke = Tab::off[p + 1];
          float wg[2 * l3 + 1];
#pragma unroll
          for (int q = 0; q < 2 * l3 + 1; ++q)
            wg[q] = swap ? s * wpx[p] * Gix[l3 * l3 + q] : s * wp[p] * Gi[l3 * l3 + q];
          static_for<kb, ke>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int i1 = Tab::e1[k], j3 = Tab::e3[k] - l3 * l3;
            Gacc[i1] = fmaf(cy[k], wg[j3], Gacc[i1]);
          });
        });
      }
      static_for<0, NP>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        constexpr int l2 = Tab::l2[p];
        constexpr bool swap = PAR && (l2 & 1);
        constexpr int kb = Tab::off[p], ke = Tab::off[p + 1];
        float Tp[2 * l2 + 1];
#pragma unroll
        for (int q = 0; q < 2 * l2 + 1; ++q) Tp[q] = 0.0f;
        static_for<kb, ke>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          constexpr int j2 = Tab::e2[k] - l2 * l2, i1 = FIRST ? 0 : Tab::e1[k], i3 = Tab::e3[k];
          constexpr float cv = Tab::ec[k];
          Tp[j2] = fmaf(cv, (swap ? hix[i1] : hi[i1]) * Gt[i3], Tp[j2]);
        });
        float dwp = 0.0f;
#pragma unroll
        for (int q = 0; q < 2 * l2 + 1; ++q) {
          dwp = fmaf(Y[l2 * l2 + q], Tp[q], dwp);
          dYp[l2 * l2 + q] = fmaf(wp[p], Tp[q], dYp[l2 * l2 + q]);
        }
        if (active) dwrow[p * C + c] = dwp;
      });
      const float tot = warp_reduce16(dYp);
      if ((lane & 1) == 0) red[warp][t][lane >> 1] = tot;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nt * 16; q += blockDim.x) {
      const int t = q >> 4, k = q & 15;
      float v = 0.0f;
      for (int ww = 0; ww < nwarps; ++ww) v += red[ww][t][k];
      dY[(size_t)(e0 + t) * 16 + k] += v;
    }
  }
  advance(i1);
}

// ----------------------------------------------------------- channel mixing
// Per order l, the (2l+1) N rows of node components times W_l (C x C), as a
// tiled FP32 GEMM: 64 rows x 128 output channels per block, K = C = 128 staged
// in shared memory, 8 x 8 outputs per thread.  Row r of order l is node
// r / (2l+1), component l^2 + r % (2l+1).
//   forward:  u = m W_l;  h_out = h_in + (l == 0 ? silu(u) : u);  u0 keeps u (l = 0)
//   backward: Gm = Gu W_l^T,  Gu = G silu'(u0) (l = 0) or G
// The input is X + X2 when X2 is given (the fused kernels' two partial buffers).
// Wg is W_l (forward) or W_l^T (backward), both read row-major [k][n].  All
// global traffic is in 16-byte vectors with every load of a thread issued
// before its first use; the A tile is kept row-major (rows padded to 132
// floats) and read four k at a time.
constexpr int kMixRows = 64;
constexpr int kMixAS = 132;  // A tile row stride (floats)
// parity (mixed-parity models): the scalar activation of the odd block (channels
// >= 64) is tanh instead of SiLU.
template <bool BWD>
__global__ void __launch_bounds__(128) mix_gemm(int n, int L, const float* __restrict__ X,
                                                const float* __restrict__ X2, const float* __restrict__ Wg,
                                                const float* __restrict__ hin,
                                                float* __restrict__ out, float* __restrict__ u0,
                                                const float* __restrict__ u0_in, int parity) {
  constexpr int C = 128, C4 = C / 4;
  extern __shared__ __align__(16) float sm[];
  float* Ws = sm;                   // [k][n]
  float* As = sm + C * C;           // [row][k], stride kMixAS
  const int l = blockIdx.y, R = 2 * l + 1, D = (L + 1) * (L + 1);
  const int rows = n * R;
  const int row0 = blockIdx.x * kMixRows;
  if (row0 >= rows) return;
  const float4* Wl4 = reinterpret_cast<const float4*>(Wg + (size_t)l * C * C);
  const float4* X4 = reinterpret_cast<const float4*>(X);
  const float4* X24 = reinterpret_cast<const float4*>(X2);
  const float4* U4 = reinterpret_cast<const float4*>(u0_in);
  // A tile: 64 rows x 32 float4, 16 per thread, loads first
  constexpr int NA = kMixRows * C4 / 128;
  float4 va[NA];
#pragma unroll
  for (int u = 0; u < NA; ++u) {
    const int q = threadIdx.x + u * 128, rr = q / C4, c4 = q % C4, r = row0 + rr;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < rows) {
      const int nd = r / R, mm = r % R;
      const size_t o = ((size_t)nd * D + l * l + mm) * C4 + c4;
      v = X4[o];
      if (X2) {
        const float4 w = X24[o];
        v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
      }
      if (BWD && l == 0) {
        const float4 uu = U4[(size_t)nd * C4 + c4];
        if (parity && c4 >= C4 / 2) {
          v.x *= tanh_grad_f(uu.x); v.y *= tanh_grad_f(uu.y); v.z *= tanh_grad_f(uu.z); v.w *= tanh_grad_f(uu.w);
        } else {
          v.x *= silu_grad_f(uu.x); v.y *= silu_grad_f(uu.y); v.z *= silu_grad_f(uu.z); v.w *= silu_grad_f(uu.w);
        }
      }
    }
    va[u] = v;
  }
#pragma unroll 8
  for (int k = threadIdx.x; k < C * C4; k += blockDim.x) reinterpret_cast<float4*>(Ws)[k] = Wl4[k];
#pragma unroll
  for (int u = 0; u < NA; ++u) {
    const int q = threadIdx.x + u * 128, rr = q / C4, c4 = q % C4;
    *reinterpret_cast<float4*>(&As[rr * kMixAS + 4 * c4]) = va[u];
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 column groups x 8 row groups
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll 1
  for (int k0 = 0; k0 < C; k0 += 4) {
    float4 a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = *reinterpret_cast<const float4*>(&As[(ty * 8 + i) * kMixAS + k0]);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const float4 b0 = *reinterpret_cast<const float4*>(&Ws[(k0 + kk) * C + tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Ws[(k0 + kk) * C + 64 + tx * 4]);
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float ai = kk == 0 ? a[i].x : kk == 1 ? a[i].y : kk == 2 ? a[i].z : a[i].w;
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(ai, b[j], acc[i][j]);
      }
    }
  }
  // epilogue: two float4 column groups per row (channels tx*4.. and 64+tx*4..)
  float4 hv[8][2];
  if (!BWD) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = row0 + ty * 8 + i;
      hv[i][0] = hv[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) {
        const int nd = r / R, mm = r % R;
        const float4* h4 = reinterpret_cast<const float4*>(hin + ((size_t)nd * D + l * l + mm) * C);
        hv[i][0] = h4[tx];
        hv[i][1] = h4[16 + tx];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = row0 + ty * 8 + i;
    if (r >= rows) continue;
    const int nd = r / R, mm = r % R;
    float4* o4 = reinterpret_cast<float4*>(out + ((size_t)nd * D + l * l + mm) * C);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      float4 u = make_float4(acc[i][4 * g], acc[i][4 * g + 1], acc[i][4 * g + 2], acc[i][4 * g + 3]);
      if (BWD) {
        o4[16 * g + tx] = u;
      } else if (l == 0) {
        reinterpret_cast<float4*>(u0 + (size_t)nd * C)[16 * g + tx] = u;
        const float4 h = hv[i][g];
        if (parity && g == 1)
          o4[16 * g + tx] = make_float4(h.x + tanhf(u.x), h.y + tanhf(u.y), h.z + tanhf(u.z), h.w + tanhf(u.w));
        else
          o4[16 * g + tx] = make_float4(h.x + silu_f(u.x), h.y + silu_f(u.y), h.z + silu_f(u.z), h.w + silu_f(u.w));
      } else {
        const float4 h = hv[i][g];
        o4[16 * g + tx] = make_float4(h.x + u.x, h.y + u.y, h.z + u.z, h.w + u.w);
      }
    }
  }
}

// Mixes for other channel counts (the 16-channel model): one thread per output
// channel, W_l in shared memory.
constexpr int kMixNodes = 8;
__global__ void mix_fwd(int n, int C, int L, const float* __restrict__ m, const float* __restrict__ Wmix,
                        const float* __restrict__ hin, float* __restrict__ hout, float* __restrict__ u0,
                        int parity) {
  extern __shared__ float smem[];
  const int l = blockIdx.y, D = (L + 1) * (L + 1), R = 2 * l + 1;
  float* W = smem;                 // [C][C]
  float* rows = smem + C * C;      // [kMixNodes * R][C]
  const float* Wl = Wmix + (size_t)l * C * C;
  for (int k = threadIdx.x; k < C * C; k += blockDim.x) W[k] = Wl[k];
  const int node0 = blockIdx.x * kMixNodes;
  for (int k = threadIdx.x; k < kMixNodes * R * C; k += blockDim.x) {
    const int rr = k / C, cc = k % C, nd = node0 + rr / R, mm = rr % R;
    rows[k] = nd < n ? m[((size_t)nd * D + l * l + mm) * C + cc] : 0.0f;
  }
  __syncthreads();
  const int c2 = threadIdx.x;
  if (c2 >= C) return;
  for (int rr = 0; rr < kMixNodes * R; ++rr) {
    const int nd = node0 + rr / R, mm = rr % R;
    if (nd >= n) break;
    float u = 0.0f;
    const float* row = rows + rr * C;
    for (int c1 = 0; c1 < C; ++c1) u = fmaf(row[c1], W[c1 * C + c2], u);
    const size_t o = ((size_t)nd * D + l * l + mm) * C + c2;
    if (l == 0) {
      u0[(size_t)nd * C + c2] = u;
      hout[o] = hin[o] + ((parity && c2 >= C / 2) ? tanhf(u) : silu_f(u));
    } else {
      hout[o] = hin[o] + u;
    }
  }
}

__global__ void mix_bwd(int n, int C, int L, const float* __restrict__ G, const float* __restrict__ u0,
                        const float* __restrict__ Wmix, float* __restrict__ Gm, int parity) {
  extern __shared__ float smem[];
  const int l = blockIdx.y, D = (L + 1) * (L + 1), R = 2 * l + 1;
  float* Wt = smem;                // Wt[c'][c] = W[c][c']
  float* rows = smem + C * C;
  const float* Wl = Wmix + (size_t)l * C * C;
  for (int k = threadIdx.x; k < C * C; k += blockDim.x) {
    const int a = k / C, b = k % C;  // W[a][b]
    Wt[b * C + a] = Wl[k];
  }
  const int node0 = blockIdx.x * kMixNodes;
  for (int k = threadIdx.x; k < kMixNodes * R * C; k += blockDim.x) {
    const int rr = k / C, cc = k % C, nd = node0 + rr / R, mm = rr % R;
    float v = 0.0f;
    if (nd < n) {
      v = G[((size_t)nd * D + l * l + mm) * C + cc];
      if (l == 0) {
        const float uu = u0[(size_t)nd * C + cc];
        v *= (parity && cc >= C / 2) ? tanh_grad_f(uu) : silu_grad_f(uu);
      }
    }
    rows[k] = v;
  }
  __syncthreads();
  const int c1 = threadIdx.x;
  if (c1 >= C) return;
  for (int rr = 0; rr < kMixNodes * R; ++rr) {
    const int nd = node0 + rr / R, mm = rr % R;
    if (nd >= n) break;
    float g = 0.0f;
    const float* row = rows + rr * C;
    for (int c2 = 0; c2 < C; ++c2) g = fmaf(Wt[c2 * C + c1], row[c2], g);
    Gm[((size_t)nd * D + l * l + mm) * C + c1] = g;
  }
}

}  // namespace

// Host-side launchers (declared in plain_fp32.h via extern templates below).
int launch_edge_geom(int E, const double* pos, const int* recv, const int* send, const int8_t* shift,
                     const CellArg& cell, float4* ev, cudaStream_t st, const int* Edev) {
  if (E <= 0) return MLIP_OK;
  {
    MLIP_PROF("edge_geom", st);
    edge_geom<<<std::min((E + 255) / 256, 8192), 256, 0, st>>>(E, pos, recv, send, shift, cell, ev, Edev);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_radial_fwd(int H, int E, const float4* ev, const float* W1, const float* W2, float rc, int p,
                      float* z2T, int ldz, cudaStream_t st) {
  if (E <= 0) return MLIP_OK;
  const int blocks = (E + 127) / 128;
  if (H == 64) { MLIP_PROF("radial_fwd", st); radial_fwd<64><<<blocks, 128, 0, st>>>(E, ev, W1, W2, rc, p, z2T, ldz); }
  else if (H == 32) { MLIP_PROF("radial_fwd", st); radial_fwd<32><<<blocks, 128, 0, st>>>(E, ev, W1, W2, rc, p, z2T, ldz); }
  else { set_error("radial hidden width %d unsupported", H); return MLIP_ERR_INVALID_ARG; }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_radial_bwd(int H, int E, const float4* ev, const float* W1, const float* W2, float rc, int p,
                      const float* dz2, float* dr_tot, cudaStream_t st) {
  if (E <= 0) return MLIP_OK;
  const int blocks = (E + 127) / 128;
  if (H == 64) { MLIP_PROF("radial_bwd", st); radial_bwd<64><<<blocks, 128, 0, st>>>(E, ev, W1, W2, rc, p, dz2, dr_tot); }
  else if (H == 32) { MLIP_PROF("radial_bwd", st); radial_bwd<32><<<blocks, 128, 0, st>>>(E, ev, W1, W2, rc, p, dz2, dr_tot); }
  else { set_error("radial hidden width %d unsupported", H); return MLIP_ERR_INVALID_ARG; }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_sgemm(bool a_km, bool b_nk, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                 float* C, int ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return MLIP_OK;
  dim3 grid((N + 127) / 128, (M + 127) / 128);
  if (a_km && !b_nk) { MLIP_PROF("sgemm", st); sgemm<true, false><<<grid, 256, 0, st>>>(M, nullptr, N, K, A, lda, B, ldb, C, ldc); }
  else if (!a_km && b_nk) { MLIP_PROF("sgemm", st); sgemm<false, true><<<grid, 256, 0, st>>>(M, nullptr, N, K, A, lda, B, ldb, C, ldc); }
  else if (!a_km && !b_nk) { MLIP_PROF("sgemm", st); sgemm<false, false><<<grid, 256, 0, st>>>(M, nullptr, N, K, A, lda, B, ldb, C, ldc); }
  else { MLIP_PROF("sgemm", st); sgemm<true, true><<<grid, 256, 0, st>>>(M, nullptr, N, K, A, lda, B, ldb, C, ldc); }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

static int tp_blocks(int n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(n, sms * 8));
}

int launch_tp_fwd(int L, bool first, int n, int C, const int* row_ptr, const int* recv, const int* send,
                  const float4* ev, const float* h, const float* w, int PW, float s, float* m, cudaStream_t st,
                  bool par) {
  if (n <= 0) return MLIP_OK;
  const int G = tp_blocks(n), threads = std::max(C, 32);
#define MLIP_TPF(LL, FF, PP)                                                                         \
  {                                                                                                  \
    MLIP_PROF("tp_fwd", st);                                                                         \
    tp_fwd<LL, FF, PP><<<G, threads, 0, st>>>(n, C, row_ptr, recv, send, ev, h, w, PW, s, m);        \
  }
  if (L == 2 && first) { if (par) MLIP_TPF(2, true, true) else MLIP_TPF(2, true, false) }
  else if (L == 2) { if (par) MLIP_TPF(2, false, true) else MLIP_TPF(2, false, false) }
  else if (L == 3 && first) { if (par) MLIP_TPF(3, true, true) else MLIP_TPF(3, true, false) }
  else if (L == 3) { if (par) MLIP_TPF(3, false, true) else MLIP_TPF(3, false, false) }
  else { set_error("l_max %d unsupported", L); return MLIP_ERR_INVALID_ARG; }
#undef MLIP_TPF
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_tp_bwd(int L, bool first, int n, int C, const int* row_ptr, const int* recv, const int* send,
                  const float4* ev, const float* hprev, const float* Gm, const float* w, int PW, float s,
                  const float* Gin, float* Gout, float* dw, float* dY, cudaStream_t st, bool par) {
  if (n <= 0) return MLIP_OK;
  const int G = tp_blocks(n), threads = std::max(C, 32);
  if (threads > 128) { set_error("channels %d unsupported", C); return MLIP_ERR_INVALID_ARG; }
#define MLIP_TPB(LL, FF, PP)                                                                            \
  {                                                                                                     \
    MLIP_PROF("tp_bwd", st);                                                                            \
    tp_bwd<LL, FF, PP><<<G, threads, 0, st>>>(n, C, row_ptr, recv, send, ev, hprev, Gm, w, PW, s, Gin, Gout, dw, dY); \
  }
  if (L == 2 && first) { if (par) MLIP_TPB(2, true, true) else MLIP_TPB(2, true, false) }
  else if (L == 2) { if (par) MLIP_TPB(2, false, true) else MLIP_TPB(2, false, false) }
  else if (L == 3 && first) { if (par) MLIP_TPB(3, true, true) else MLIP_TPB(3, true, false) }
  else if (L == 3) { if (par) MLIP_TPB(3, false, true) else MLIP_TPB(3, false, false) }
  else { set_error("l_max %d unsupported", L); return MLIP_ERR_INVALID_ARG; }
#undef MLIP_TPB
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_mix_fwd(int n, int C, int L, const float* m, const float* Wmix, const float* hin, float* hout,
                   float* u0, cudaStream_t st, int parity) {
  if (n <= 0) return MLIP_OK;
  if (C == 128) {
    const size_t smem = (size_t)(128 * 128 + kMixRows * kMixAS) * sizeof(float);
    MLIP_CUDA_TRY(cudaFuncSetAttribute(mix_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((n * (2 * L + 1) + kMixRows - 1) / kMixRows, L + 1);
    { MLIP_PROF("mix_fwd", st); mix_gemm<false><<<grid, 128, smem, st>>>(n, L, m, nullptr, Wmix, hin, hout, u0, nullptr, parity); }
    MLIP_LAUNCH_CHECK();
    return MLIP_OK;
  }
  const size_t smem = ((size_t)C * C + (size_t)kMixNodes * (2 * L + 1) * C) * sizeof(float);
  MLIP_CUDA_TRY(cudaFuncSetAttribute(mix_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((n + kMixNodes - 1) / kMixNodes, L + 1);
  { MLIP_PROF("mix_fwd", st); mix_fwd<<<grid, std::max(C, 32), smem, st>>>(n, C, L, m, Wmix, hin, hout, u0, parity); }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_mix_bwd(int n, int C, int L, const float* G, const float* u0, const float* Wmix, const float* WmixT,
                   float* Gm, cudaStream_t st, int parity) {
  if (n <= 0) return MLIP_OK;
  if (C == 128) {
    const size_t smem = (size_t)(128 * 128 + kMixRows * kMixAS) * sizeof(float);
    MLIP_CUDA_TRY(cudaFuncSetAttribute(mix_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((n * (2 * L + 1) + kMixRows - 1) / kMixRows, L + 1);
    { MLIP_PROF("mix_bwd", st); mix_gemm<true><<<grid, 128, smem, st>>>(n, L, G, nullptr, WmixT, nullptr, Gm, nullptr, u0, parity); }
    MLIP_LAUNCH_CHECK();
    return MLIP_OK;
  }
  const size_t smem = ((size_t)C * C + (size_t)kMixNodes * (2 * L + 1) * C) * sizeof(float);
  MLIP_CUDA_TRY(cudaFuncSetAttribute(mix_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((n + kMixNodes - 1) / kMixNodes, L + 1);
  { MLIP_PROF("mix_bwd", st); mix_bwd<<<grid, std::max(C, 32), smem, st>>>(n, C, L, G, u0, Wmix, Gm, parity); }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace mlip
