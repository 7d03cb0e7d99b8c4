// Radial MLP of the fused form with its 64 x 64 hidden layer on the tensor
// cores (tcgen05.mma kind::f16, FP16 operands, FP32 accumulation in tensor
// memory), for H = 64.
//
// The radial network of every edge e is  z1 = silu(e_n W1),  z2 = silu(z1 W2)
// (Bessel basis e_n times the envelope, bias-free layers).  A CTA of 256
// threads takes 128 edges at a time (one tensor-memory lane each), two threads
// per edge, each with half of the 64 hidden units:
//   forward  (radial_tc):      z1 in FP32 on the ALUs, each row scaled by a
//       power of two so that its largest entry lies in [2^13, 2^14) and written
//       as the FP16 A operand; one MMA chain (M = 128 edges, N = 64, K = 64)
//       against W2^T; the row of a2 = z1 W2 is read back, unscaled exactly,
//       and z2 = silu(a2) is written as the 16-bit operand tile of the
//       message kernels (4 KB per 32 edges, canonical K-major layout).
//   adjoint  (radial_bwd_tc):  the same product for a2, then
//       da2 = dE/dz2 * silu'(a2) (scaled per row likewise), a second MMA chain
//       dz1 = da2 W2^T against W2, and per edge
//       dE/dr += sum_k dz1_k silu'(a1_k) (W1 de/dr)_k  (the halves' partial
//       sums added in a fixed order).
// The power-of-two row scales keep FP16 away from overflow and underflow and
// are removed exactly after the product.  Each FP32 operand x is split into
// x_hi = fp16(x) and x_lo = fp16(x - x_hi) and the product is taken as
// A_hi B_hi + A_lo B_hi + A_hi B_lo (three MMA chains into one accumulator),
// which keeps about 21 significant bits: the layer stays at FP32-level
// accuracy while its flops run on the tensor pipe.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels_common.cuh"
#include "launchers.cuh"
#include "profile.cuh"
#include "sm100_tc.cuh"

namespace mlip {
namespace {

constexpr int kRH = 64;          // hidden width
constexpr int kRM = 128;         // edges per MMA tile (M)
constexpr int kZ2Tile = 32;      // edges per z2 operand tile of the message kernels
constexpr int kAOpBytes = kRM * kRH * 2;   // 16 KB
constexpr int kBOpBytes = kRH * kRH * 2;   // 8 KB
// CTAs of 256 threads per SM: forward 2 x (48 KB shared, 64 tensor-memory
// columns), adjoint 2 x (64 KB, 128 columns)
constexpr int kFwdCTAs = 2, kBwdCTAs = 2;

__device__ __forceinline__ uint16_t f16_bits(float x) {
  const __half v = __float2half_rn(x);
  return *reinterpret_cast<const uint16_t*>(&v);
}
__device__ __forceinline__ uint16_t z2_bits(float x, int use_bf16) {
  if (use_bf16) {
    const __nv_bfloat16 v = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t*>(&v);
  }
  return f16_bits(x);
}

// 2^k with max|row| * 2^k in [2^13, 2^14) (1 for an all-zero row).
__device__ __forceinline__ float row_scale(float amax) {
  if (!(amax > 0.0f)) return 1.0f;
  const int ex = ilogbf(amax);  // amax in [2^ex, 2^(ex+1))
  return exp2f((float)max(-100, min(100, 13 - ex)));
}

__device__ __forceinline__ void split16(float x, uint16_t& hi, uint16_t& lo) {
  const __half h = __float2half_rn(x);
  hi = *reinterpret_cast<const uint16_t*>(&h);
  lo = f16_bits(x - __half2float(h));
}

// Two threads per edge (row r of the tile): half h of the row holds hidden
// units [32 h, 32 h + 32).  The halves exchange their row maxima (the row's
// power-of-two scale) and partial sums through shared memory.
constexpr int kRT = 2 * kRM;  // threads per CTA
constexpr int kHH = kRH / 2;  // hidden units per thread

// Writes half h of an FP32 row (times sc) into the FP16 hi and lo A operands
// (canonical layout, K = 64).
__device__ __forceinline__ void put_half_row(uint8_t* Ahi, uint8_t* Alo, int r, int h, const float* v, float sc) {
#pragma unroll
  for (int kq = 0; kq < kHH / 8; ++kq) {
    const int kg = h * (kHH / 8) + kq;
    uint32_t ph[4], pl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint16_t h0, l0, h1, l1;
      split16(v[kq * 8 + 2 * q] * sc, h0, l0);
      split16(v[kq * 8 + 2 * q + 1] * sc, h1, l1);
      ph[q] = (uint32_t)h0 | ((uint32_t)h1 << 16);
      pl[q] = (uint32_t)l0 | ((uint32_t)l1 << 16);
    }
    *reinterpret_cast<uint4*>(Ahi + tc::canon_off(r, kg * 8)) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
    *reinterpret_cast<uint4*>(Alo + tc::canon_off(r, kg * 8)) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
  }
}

// Issues D = A_hi B_hi + A_lo B_hi + A_hi B_lo over K = 64 (12 MMAs of K = 16)
// and commits to `bar`.
__device__ __forceinline__ void mma_tile(uint32_t dtm, const uint8_t* Ahi, const uint8_t* Alo, const uint8_t* Bhi,
                                         const uint8_t* Blo, uint64_t* bar) {
  const uint32_t idesc = tc::idesc_16bit(kRM, kRH, false);
  const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
  const uint32_t as[3] = {ah, al, ah}, bs[3] = {bh, bh, bl};
#pragma unroll
  for (int pass = 0; pass < 3; ++pass)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint64_t ad = tc::desc_noswizzle(as[pass] + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
      const uint64_t bd = tc::desc_noswizzle(bs[pass] + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
      tc::mma_bf16(dtm, ad, bd, idesc, (pass | kk) ? 1u : 0u);
    }
  tc::mma_commit(bar);
}

// Reads this thread's 32 accumulator columns (its lane; columns col0..+31) times inv.
__device__ __forceinline__ void get_half_row(uint32_t taddr, float* v, float inv) {
#pragma unroll
  for (int c = 0; c < kHH / 8; ++c) tc::tmem_ld8(taddr + c * 8, v + c * 8);
  tc::tmem_ld_wait();
#pragma unroll
  for (int k = 0; k < kHH; ++k) v[k] *= inv;
}

__device__ __forceinline__ float absmax32(const float* v) {
  float m = 0.0f;
#pragma unroll
  for (int k = 0; k < kHH; ++k) m = fmaxf(m, fabsf(v[k]));
  return m;
}

// Half h of the basis functions of edge length r into sb[0..4), sdb[0..4).
template <bool GRAD>
__device__ __forceinline__ void basis_half(float r, float rc, int p, int h, float* sb, float* sdb) {
  float b[4], db[4];
  if (h == 0) radial_basis<8, GRAD, 0, 4>(r, rc, p, b, db);
  else radial_basis<8, GRAD, 4, 4>(r, rc, p, b, db);
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    sb[n] = b[n];
    if (GRAD) sdb[n] = db[n];
  }
}

// ------------------------------------------------------------- forward
__global__ void __launch_bounds__(kRT, kFwdCTAs) radial_tc(int E, int n_tiles32, const float4* __restrict__ ev,
                                                 const float* __restrict__ W1, const uint8_t* __restrict__ w2img,
                                                 float wsc, float rc, int p, int use_bf16,
                                                 uint8_t* __restrict__ z2t, const int* __restrict__ Edev,
                                                 int* __restrict__ err) {
  if (Edev) {  // edge count on the device (capacity-sized launch)
    E = *Edev;
    n_tiles32 = (E + kZ2Tile - 1) / kZ2Tile;
  }
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAh = smem;
  uint8_t* sAl = smem + kAOpBytes;
  uint8_t* sBh = smem + 2 * kAOpBytes;  // W2^T image: hi then lo
  uint8_t* sBl = sBh + kBOpBytes;
  __shared__ __align__(16) float sW1[8 * kRH];
  __shared__ float s_b[kRM][8];
  __shared__ float s_amax[kRT];
  __shared__ __align__(8) uint64_t bar, bar_w;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, rt = tid & (kRM - 1), hf = tid >> 7;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, kRH);
    tc::tmem_relinquish();
  }
  bool w_waited = false;  // thread 0: the weight image has landed
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_init(&bar_w, 1);
    tc::fence_mbar_init();
    abort_s = 0;
    tc::mbar_arrive_expect_tx(&bar_w, 2 * kBOpBytes);
    tc::bulk_g2s(sBh, w2img, 2 * kBOpBytes, &bar_w);
  }
  for (int q = tid; q < 8 * kRH; q += blockDim.x) sW1[q] = W1[q];
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // tensor-memory lanes of this warp: rows 32 (warp % 4) ..; columns of this half
  const uint32_t taddr = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + hf * kHH;
  const int n_edges = n_tiles32 * kZ2Tile;  // z2 rows to write (E rounded up to 32)
  uint32_t phase = 0;
  int issued = 0, done = 0;  // products issued / phases seen complete (thread 0)
#pragma unroll 1
  for (int base = blockIdx.x * kRM; base < n_edges; base += gridDim.x * kRM) {
    const int e = base + rt;
    const bool live = e < E;
    if (live) basis_half<false>(ev[e].w, rc, p, hf, &s_b[rt][4 * hf], nullptr);
    __syncthreads();
    float z[kHH];
    float amax = 0.0f;
    if (live) {
#pragma unroll
      for (int k = 0; k < kHH; ++k) {
        const int kk = hf * kHH + k;
        float a = 0.0f;
#pragma unroll
        for (int n = 0; n < 8; ++n) a = fmaf(s_b[rt][n], sW1[n * kRH + kk], a);
        z[k] = silu_f(a);
      }
      amax = absmax32(z);
    } else {
#pragma unroll
      for (int k = 0; k < kHH; ++k) z[k] = 0.0f;
    }
    s_amax[tid] = amax;
    __syncthreads();
    const float sc = row_scale(fmaxf(s_amax[rt], s_amax[rt + kRM]));
    put_half_row(sAh, sAl, rt, hf, z, sc);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      if (!w_waited) w_waited = tc::mbar_wait(&bar_w, 0);
      tc::fence_after_sync();
      if (w_waited) {
        mma_tile(tmem_base, sAh, sAl, sBh, sBl, &bar);
        ++issued;
      } else {
        atomicOr(err, 32);
        abort_s = 1;
        tc::mbar_arrive(&bar);  // completes the phase: nobody waits for an MMA that was not issued
      }
    }
    if (!tc::mbar_wait(&bar, phase)) {
      atomicOr(err, 32);
      abort_s = 1;
    } else if (tid == 0) {
      ++done;
    }
    phase ^= 1;
    tc::fence_after_sync();
    get_half_row(taddr, z, 1.0f / (sc * wsc));
    if (e < n_edges) {
      uint8_t* tile = z2t + (size_t)(e / kZ2Tile) * (kZ2Tile * kRH * 2);
      const int t = e % kZ2Tile;
#pragma unroll
      for (int kq = 0; kq < kHH / 8; ++kq) {
        const int kg = hf * (kHH / 8) + kq;
        uint32_t pk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int k = kq * 8 + 2 * q;
          const float v0 = live ? silu_f(z[k]) : 0.0f, v1 = live ? silu_f(z[k + 1]) : 0.0f;
          pk[q] = (uint32_t)z2_bits(v0, use_bf16) | ((uint32_t)z2_bits(v1, use_bf16) << 16);
        }
        *reinterpret_cast<uint4*>(tile + tc::canon_off(t, kg * 8)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // the next tile rewrites sA, the basis and the accumulator
    tc::fence_after_sync();
    if (abort_s) break;
  }
  if (tid == 0) {
    if (issued > done) tc::mbar_wait(&bar, done & 1, 1LL << 20);  // the product in flight, bounded
    if (!w_waited) tc::mbar_wait(&bar_w, 0, 1LL << 20);          // the weight copy in flight, bounded
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem_base, kRH);
}

// ------------------------------------------------------------- adjoint
__global__ void __launch_bounds__(kRT, kBwdCTAs) radial_bwd_tc(int E, const float4* __restrict__ ev,
                                                     const float* __restrict__ W1,
                                                     const uint8_t* __restrict__ w2img, float wsc,
                                                     float rc, int p, const float* __restrict__ dz2,
                                                     float* __restrict__ dr_tot, int init,
                                                     const int* __restrict__ Edev, int* __restrict__ err) {
  if (Edev) E = *Edev;  // edge count on the device (capacity-sized launch)
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAh = smem;
  uint8_t* sAl = smem + kAOpBytes;
  uint8_t* sBth = smem + 2 * kAOpBytes;   // W2^T: a2 = z1 W2      (the image: hi, lo,
  uint8_t* sBtl = sBth + kBOpBytes;
  uint8_t* sBnh = sBtl + kBOpBytes;       // W2:   dz1 = da2 W2^T   then hi, lo)
  uint8_t* sBnl = sBnh + kBOpBytes;
  __shared__ __align__(16) float sW1[8 * kRH];
  __shared__ float s_b[kRM][8], s_db[kRM][8];
  __shared__ float s_amax[kRT], s_dr[kRT];
  __shared__ __align__(8) uint64_t bar, bar_w;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, rt = tid & (kRM - 1), hf = tid >> 7;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 2 * kRH);
    tc::tmem_relinquish();
  }
  bool w_waited = false;  // thread 0: the weight image has landed
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_init(&bar_w, 1);
    tc::fence_mbar_init();
    abort_s = 0;
    tc::mbar_arrive_expect_tx(&bar_w, 4 * kBOpBytes);
    tc::bulk_g2s(sBth, w2img, 4 * kBOpBytes, &bar_w);
  }
  for (int q = tid; q < 8 * kRH; q += blockDim.x) sW1[q] = W1[q];
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + hf * kHH;
  uint32_t phase = 0;
  int issued = 0, done = 0;
#pragma unroll 1
  for (int base = blockIdx.x * kRM; base < E; base += gridDim.x * kRM) {
    const int e = base + rt;
    const bool live = e < E;
    if (live) basis_half<true>(ev[e].w, rc, p, hf, &s_b[rt][4 * hf], &s_db[rt][4 * hf]);
    __syncthreads();
    // first layer for this half: pre-activations a1 (kept) and z1 = silu(a1)
    float a1[kHH], z[kHH];
    float amax = 0.0f;
    if (live) {
#pragma unroll
      for (int k = 0; k < kHH; ++k) {
        const int kk = hf * kHH + k;
        float a = 0.0f;
#pragma unroll
        for (int n = 0; n < 8; ++n) a = fmaf(s_b[rt][n], sW1[n * kRH + kk], a);
        a1[k] = a;
        z[k] = silu_f(a);
      }
      amax = absmax32(z);
    } else {
#pragma unroll
      for (int k = 0; k < kHH; ++k) a1[k] = z[k] = 0.0f;
    }
    s_amax[tid] = amax;
    __syncthreads();
    const float sc1 = row_scale(fmaxf(s_amax[rt], s_amax[rt + kRM]));
    put_half_row(sAh, sAl, rt, hf, z, sc1);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      if (!w_waited) w_waited = tc::mbar_wait(&bar_w, 0);
      tc::fence_after_sync();
      if (w_waited) {
        mma_tile(tmem_base, sAh, sAl, sBth, sBtl, &bar);
        ++issued;
      } else {
        atomicOr(err, 64);
        abort_s = 1;
        tc::mbar_arrive(&bar);  // completes the phase: nobody waits for an MMA that was not issued
      }
    }
    if (!tc::mbar_wait(&bar, phase)) {
      atomicOr(err, 64);
      abort_s = 1;
    } else if (tid == 0) {
      ++done;
    }
    phase ^= 1;
    tc::fence_after_sync();
    get_half_row(taddr, z, 1.0f / (sc1 * wsc));  // a2 of this half
    // da2 = dE/dz2 silu'(a2)
    if (live) {
      const float4* g4 = reinterpret_cast<const float4*>(dz2 + (size_t)e * kRH + hf * kHH);
#pragma unroll
      for (int q4 = 0; q4 < kHH / 4; ++q4) {
        const float4 g = g4[q4];
        z[4 * q4] = g.x * silu_grad_f(z[4 * q4]);
        z[4 * q4 + 1] = g.y * silu_grad_f(z[4 * q4 + 1]);
        z[4 * q4 + 2] = g.z * silu_grad_f(z[4 * q4 + 2]);
        z[4 * q4 + 3] = g.w * silu_grad_f(z[4 * q4 + 3]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < kHH; ++k) z[k] = 0.0f;
    }
    s_amax[tid] = absmax32(z);
    __syncthreads();  // both halves' maxima; the first product (complete) no longer reads sA
    const float sc2 = row_scale(fmaxf(s_amax[rt], s_amax[rt + kRM]));
    put_half_row(sAh, sAl, rt, hf, z, sc2);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      if (!abort_s) {
        mma_tile(tmem_base + kRH, sAh, sAl, sBnh, sBnl, &bar);
        ++issued;
      } else {
        tc::mbar_arrive(&bar);
      }
    }
    if (!tc::mbar_wait(&bar, phase)) {
      atomicOr(err, 64);
      abort_s = 1;
    } else if (tid == 0) {
      ++done;
    }
    phase ^= 1;
    tc::fence_after_sync();
    get_half_row(taddr + kRH, z, 1.0f / (sc2 * wsc));  // dz1 of this half
    float dr = 0.0f;
    if (live) {
#pragma unroll
      for (int k = 0; k < kHH; ++k) {
        const int kk = hf * kHH + k;
        float bd = 0.0f;
#pragma unroll
        for (int n = 0; n < 8; ++n) bd = fmaf(sW1[n * kRH + kk], s_db[rt][n], bd);
        dr = fmaf(z[k] * silu_grad_f(a1[k]), bd, dr);
      }
    }
    s_dr[tid] = dr;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (hf == 0 && live) {
      const float d = s_dr[rt] + s_dr[rt + kRM];
      dr_tot[e] = init ? d : dr_tot[e] + d;  // the first layer processed initialises dE/dr
    }
    if (abort_s) break;
  }
  if (tid == 0) {
    if (issued > done) tc::mbar_wait(&bar, done & 1, 1LL << 20);  // the product in flight, bounded
    if (!w_waited) tc::mbar_wait(&bar_w, 0, 1LL << 20);          // the weight copy in flight, bounded
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem_base, 2 * kRH);
}

}  // namespace

// Split FP16 image of W2 for the radial kernels: the forward operand
// B[n][k] = W2[k][n] (hi 8 KB, lo 8 KB) then the adjoint's B[n][k] = W2[n][k]
// (hi, lo), canonical layout, all times the power-of-two *scale with
// max|W2| * scale in [2^13, 2^14).  32 KB.
void pack_radial_images(const float* W2, std::vector<uint8_t>& img, float* scale) {
  float amax = 0.0f;
  for (int q = 0; q < kRH * kRH; ++q) amax = std::max(amax, std::fabs(W2[q]));
  const float sc = amax > 0.0f ? std::ldexp(1.0f, std::max(-100, std::min(100, 13 - std::ilogb(amax)))) : 1.0f;
  *scale = sc;
  img.assign(4 * kBOpBytes, 0);
  for (int which = 0; which < 2; ++which)
    for (int n = 0; n < kRH; ++n)
      for (int k = 0; k < kRH; ++k) {
        const float x = (which == 0 ? W2[k * kRH + n] : W2[n * kRH + k]) * sc;
        const __half h = __float2half_rn(x);
        const __half lo = __float2half_rn(x - __half2float(h));
        uint8_t* o = img.data() + (size_t)which * 2 * kBOpBytes + tc::canon_off(n, k);
        std::memcpy(o, &h, 2);
        std::memcpy(o + kBOpBytes, &lo, 2);
      }
}

// Persistent grids: as many CTAs as fit on the device at once (the launch
// bounds' CTAs per SM: their registers, shared memory and tensor-memory
// columns fit together), at most one per tile.
static int radial_grid(int per_sm, int tiles) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(tiles, sms * per_sm));
}

int launch_radial_tc(int H, int E, int n_tiles32, const float4* ev, const float* W1, const uint8_t* w2img,
                     float wsc, float rc, int p, int use_bf16, uint8_t* z2t, int* err, cudaStream_t st,
                     const int* Edev) {
  if (n_tiles32 <= 0) return MLIP_OK;
  if (H != kRH) { set_error("the fused form needs hidden = 64"); return MLIP_ERR_INVALID_ARG; }
  const int tiles = (n_tiles32 * kZ2Tile + kRM - 1) / kRM;
  const int smem = 2 * kAOpBytes + 2 * kBOpBytes;
  MLIP_CUDA_TRY(cudaFuncSetAttribute(radial_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  {
    MLIP_PROF("radial_tc", st);
    radial_tc<<<radial_grid(kFwdCTAs, tiles), kRT, smem, st>>>(E, n_tiles32, ev, W1, w2img, wsc, rc, p,
                                                                       use_bf16, z2t, Edev, err);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_radial_bwd_tc(int H, int E, const float4* ev, const float* W1, const uint8_t* w2img, float wsc, float rc,
                         int p, const float* dz2, float* dr_tot, bool init, int* err, cudaStream_t st,
                         const int* Edev) {
  if (E <= 0) return MLIP_OK;
  if (H != kRH) { set_error("the fused form needs hidden = 64"); return MLIP_ERR_INVALID_ARG; }
  const int tiles = (E + kRM - 1) / kRM;
  const int smem = 2 * kAOpBytes + 4 * kBOpBytes;
  MLIP_CUDA_TRY(cudaFuncSetAttribute(radial_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  {
    MLIP_PROF("radial_bwd_tc", st);
    radial_bwd_tc<<<radial_grid(kBwdCTAs, tiles), kRT, smem, st>>>(E, ev, W1, w2img, wsc, rc, p, dz2,
                                                                              dr_tot, init ? 1 : 0, Edev, err);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace mlip
