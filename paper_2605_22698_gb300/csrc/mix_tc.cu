// Per-irrep channel mixes of the fused form on the tensor cores.
//
// For every order l the (2l+1) N rows of node components are multiplied by
// the C x C weight W_l (C = 128):
//   forward:  u = m W_l;  h_out = h_in + (l == 0 ? silu(u) : u);  u0 keeps u (l = 0)
//   adjoint:  dE/dm = Gu W_l^T,  Gu = dE/dh silu'(u0) (l = 0) or dE/dh
// where m (or dE/dh) arrives as the sum of the two partial buffers of the
// message kernels.  One CTA takes 128 rows of one order: thread r loads row r,
// scales it by a power of two (largest entry in [2^13, 2^14)) and writes it
// split into FP16 hi and lo parts as the A operand (M = 128, K = 128); the
// B operand is the model's pre-split image of W_l^T (forward) or W_l
// (adjoint), bulk-copied once per CTA; the product A_hi B_hi + A_lo B_hi +
// A_hi B_lo (three tcgen05 MMA chains, FP32 accumulation, N = 128) keeps about
// 21 significant bits.  Two threads share a row (64 channels each; 8 warps per
// CTA): they load and split their halves, read their halves of the
// accumulator row back from tensor memory, remove both scales exactly and
// apply the update.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "kernels_common.cuh"
#include "launchers.cuh"
#include "profile.cuh"
#include "sm100_tc.cuh"
#include "split16.cuh"

namespace mlip {
namespace {

// smem: A_hi, A_lo, B_hi, B_lo (32 KB each), then the barriers
template <bool BWD>
__global__ void __launch_bounds__(2 * kMM) mix_tc(int n, int L, const float* __restrict__ X, const float* __restrict__ X2,
                                              const uint8_t* __restrict__ wimg, const float* __restrict__ wscale,
                                              const float* __restrict__ hin, float* __restrict__ out,
                                              float* __restrict__ u0, const float* __restrict__ u0_in,
                                              int* __restrict__ err, const int* __restrict__ sys_of,
                                              float* __restrict__ out_max) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAh = smem;
  uint8_t* sAl = smem + kMOp;
  uint8_t* sBh = smem + 2 * kMOp;
  uint8_t* sBl = smem + 3 * kMOp;
  __shared__ __align__(8) uint64_t bar_w, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_s;
  __shared__ float s_amax[2 * kMM];
  const int l = blockIdx.y, R = 2 * l + 1, D = (L + 1) * (L + 1);
  const int rows = n * R, row0 = blockIdx.x * kMM;
  if (row0 >= rows) return;  // uniform over the CTA
  const int tid = threadIdx.x, warp = tid >> 5;
  const int rt = tid & (kMM - 1), half = tid >> 7;  // row of the tile, half of the channels
  constexpr int HC = kMC / 2;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, kMC);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar_w, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::fence_mbar_init();
    abort_s = 0;
  }
  __syncthreads();
  // weight image of this order: hi then lo, 32 KB each, one bulk copy each
  const uint8_t* wl = wimg + (size_t)l * 2 * kMOp;
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&bar_w, 2 * kMOp);
    tc::bulk_g2s(sBh, wl, kMOp, &bar_w);
    tc::bulk_g2s(sBl, wl + kMOp, kMOp, &bar_w);
  }
  // this thread's half row, scaled (by the row's power of two) and split
  const int r = row0 + rt;
  const bool live = r < rows;
  const int nd = live ? r / R : 0, mm = live ? r % R : 0;
  const size_t base = ((size_t)nd * D + l * l + mm) * kMC;
  const int cq = half * (HC / 4);  // first float4 of this half
  float v[HC];
  if (live) {
    const float4* x4 = reinterpret_cast<const float4*>(X + base);
#pragma unroll
    for (int q = 0; q < HC / 4; ++q) {
      float4 a = x4[cq + q];
      if (X2) {
        const float4 b = reinterpret_cast<const float4*>(X2 + base)[cq + q];
        a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
      }
      if (BWD && l == 0) {
        const float4 u = reinterpret_cast<const float4*>(u0_in + (size_t)nd * kMC)[cq + q];
        a.x *= silu_grad_f(u.x); a.y *= silu_grad_f(u.y); a.z *= silu_grad_f(u.z); a.w *= silu_grad_f(u.w);
      }
      v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < HC; ++k) v[k] = 0.0f;
  }
  float amax = 0.0f;
#pragma unroll
  for (int k = 0; k < HC; ++k) amax = fmaxf(amax, fabsf(v[k]));
  s_amax[tid] = amax;
  __syncthreads();
  const float sc = pow2_scale(fmaxf(s_amax[rt], s_amax[rt + kMM]));
#pragma unroll
  for (int kh = 0; kh < HC / 8; ++kh) {
    const int kg = half * (HC / 8) + kh;
    split8(v + kh * 8, sc, reinterpret_cast<uint4*>(sAh + canon128(rt, kg * 8)),
           reinterpret_cast<uint4*>(sAl + canon128(rt, kg * 8)));
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  bool issued = false;
  if (tid == 0) {
    if (tc::mbar_wait(&bar_w, 0)) {
      tc::fence_after_sync();
      const uint32_t idesc = tc::idesc_16bit(kMM, kMC, false);
      const uint32_t ah = tc::smem_u32(sAh), al = tc::smem_u32(sAl), bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);
      const uint32_t as[3] = {ah, al, ah}, bs[3] = {bh, bh, bl};
#pragma unroll 1
      for (int pass = 0; pass < 3; ++pass)
#pragma unroll
        for (int kk = 0; kk < kMC / 16; ++kk) {
          const uint64_t ad = tc::desc_noswizzle(as[pass] + kk * 256, kMLBO, kMSBO);
          const uint64_t bd = tc::desc_noswizzle(bs[pass] + kk * 256, kMLBO, kMSBO);
          tc::mma_bf16(tmem_base, ad, bd, idesc, (pass | kk) ? 1u : 0u);
        }
      tc::mma_commit(&bar_mma);
      issued = true;
    } else {
      atomicOr(err, 128);
      abort_s = 1;
    }
  }
  __syncthreads();
  if (!abort_s) {
    if (!tc::mbar_wait(&bar_mma, 0)) {
      atomicOr(err, 128);
      abort_s = 1;
    }
  }
  __syncthreads();  // abort_s is uniform from here on
  tc::fence_after_sync();
  if (!abort_s) {  // every warp reads its lanes (tcgen05.ld is warp-collective)
    const float inv = 1.0f / (sc * wscale[l]);
    const uint32_t taddr = tmem_base + ((uint32_t)((warp & 3) * 32) << 16);
    float4* o4 = reinterpret_cast<float4*>(out + base);
    const float4* h4 = reinterpret_cast<const float4*>(hin + base);
    float4* u4 = reinterpret_cast<float4*>(u0 + (size_t)nd * kMC);
    float m = 0.0f;  // max |out| over this thread's half row
#pragma unroll 1
    for (int c0 = half * HC; c0 < (half + 1) * HC; c0 += 32) {
      float w[32];
#pragma unroll
      for (int c = 0; c < 32; c += 8) tc::tmem_ld8(taddr + c0 + c, w + c);
      tc::tmem_ld_wait();
      if (!live) continue;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 u = make_float4(w[4 * q] * inv, w[4 * q + 1] * inv, w[4 * q + 2] * inv, w[4 * q + 3] * inv);
        const int i4 = c0 / 4 + q;
        float4 o;
        if (BWD) {
          o = u;
        } else {
          const float4 h = h4[i4];
          if (l == 0) {
            u4[i4] = u;
            o = make_float4(h.x + silu_f(u.x), h.y + silu_f(u.y), h.z + silu_f(u.z), h.w + silu_f(u.w));
          } else {
            o = make_float4(h.x + u.x, h.y + u.y, h.z + u.z, h.w + u.w);
          }
        }
        o4[i4] = o;
        m = fmaxf(m, fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)), fmaxf(fabsf(o.z), fabsf(o.w))));
      }
    }
    if (out_max) warp_sys_max(out_max, live ? (sys_of ? sys_of[nd] : 0) : -1, m);
  }
  if (tid == 0) {
    if (abort_s && issued) tc::mbar_wait(&bar_mma, 0, 1LL << 20);  // the product in flight, bounded
    if (abort_s && !issued) tc::mbar_wait(&bar_w, 0, 1LL << 20);   // the weight copies in flight
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem_base, kMC);
}

}  // namespace

// Split FP16 images of the mix weights of one layer: per order l, for the
// forward B[n][k] = W_l[k][n] and for the adjoint B[n][k] = W_l[n][k], each as
// hi (32 KB) then lo (32 KB) in the canonical layout, times a power-of-two
// scale per order (scale[l]).  fwd/bwd receive (L+1) * 64 KB each.
void pack_mix_images(const float* W, int L, std::vector<uint8_t>& fwd, std::vector<uint8_t>& bwd,
                     std::vector<float>& scale) {
  const int C = kMC;
  fwd.assign((size_t)(L + 1) * 2 * kMOp, 0);
  bwd.assign((size_t)(L + 1) * 2 * kMOp, 0);
  scale.assign(L + 1, 1.0f);
  for (int l = 0; l <= L; ++l) {
    const float* Wl = W + (size_t)l * C * C;
    float amax = 0.0f;
    for (int q = 0; q < C * C; ++q) amax = std::max(amax, std::fabs(Wl[q]));
    const float sc = amax > 0.0f ? std::ldexp(1.0f, 13 - std::ilogb(amax)) : 1.0f;
    scale[l] = sc;
    for (int n = 0; n < C; ++n)
      for (int k = 0; k < C; ++k) {
        for (int which = 0; which < 2; ++which) {
          const float x = (which == 0 ? Wl[k * C + n] : Wl[n * C + k]) * sc;
          const __half h = __float2half_rn(x);
          const __half lo = __float2half_rn(x - __half2float(h));
          std::vector<uint8_t>& img = which == 0 ? fwd : bwd;
          uint8_t* o = img.data() + (size_t)l * 2 * kMOp + canon128(n, k);
          std::memcpy(o, &h, 2);
          std::memcpy(o + kMOp, &lo, 2);
        }
      }
  }
}

int launch_mix_tc(bool bwd, int n, int C, int L, const float* X, const float* X2, const uint8_t* wimg,
                  const float* wscale, const float* hin, float* out, float* u0, const float* u0_in, int* err,
                  cudaStream_t st, const int* sys_of, float* amax) {
  if (n <= 0) return MLIP_OK;
  if (C != kMC) { set_error("the fused form needs 128 channels"); return MLIP_ERR_INVALID_ARG; }
  const int smem = 4 * kMOp;
  dim3 grid((n * (2 * L + 1) + kMM - 1) / kMM, L + 1);
  if (bwd) {
    MLIP_CUDA_TRY(cudaFuncSetAttribute(mix_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    MLIP_PROF("mix_tc_bwd", st);
    mix_tc<true><<<grid, 2 * kMM, smem, st>>>(n, L, X, X2, wimg, wscale, hin, out, u0, u0_in, err, sys_of,
                                                           amax);
  } else {
    MLIP_CUDA_TRY(cudaFuncSetAttribute(mix_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    MLIP_PROF("mix_tc", st);
    mix_tc<false><<<grid, 2 * kMM, smem, st>>>(n, L, X, X2, wimg, wscale, hin, out, u0, u0_in, err, sys_of,
                                                           amax);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace mlip
