// Shared pieces of the 128 x 128 split-FP16 tensor-core products (the channel
// mixes and the gated update): every FP32 operand x is scaled by a power of
// two and written as hi = fp16(x) and lo = fp16(x - hi); the products
// A_hi B_hi + A_lo B_hi + A_hi B_lo accumulate in FP32 (about 21 significant
// bits).  Operands are 128 rows x 128 K in the canonical no-swizzle K-major
// layout of tcgen05 (8-row x 16-byte core matrices).
#pragma once
#include <cstdint>

#include <cuda_fp16.h>

namespace mlip {

constexpr int kMC = 128;                      // channels (K and N of one block)
constexpr int kMM = 128;                      // rows per CTA (MMA M)
constexpr int kMOp = kMM * kMC * 2;           // one 16-bit 128 x 128 operand: 32 KB
constexpr uint32_t kMLBO = 128, kMSBO = 2048; // K-adjacent / row-group-adjacent core matrices

// Byte offset of element (row r, column k) in a canonical 128 x 128 operand.
__host__ __device__ constexpr uint32_t canon128(int r, int k) {
  return (uint32_t)((r >> 3) * kMSBO + (k >> 3) * kMLBO + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint16_t h16(float x) {
  const __half v = __float2half_rn(x);
  return *reinterpret_cast<const uint16_t*>(&v);
}

// Power of two that brings the largest magnitude amax into [2^13, 2^14).
__device__ __forceinline__ float pow2_scale(float amax) {
  if (!(amax > 0.0f)) return 1.0f;
  return exp2f((float)max(-100, min(100, 13 - ilogbf(amax))));
}

// hi and lo FP16 halves of eight scaled values, packed for one 16-byte store each.
__device__ __forceinline__ void split8(const float* v, float sc, uint4* hi, uint4* lo) {
  uint32_t ph[4], pl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint16_t hh[2], ll[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float x = v[2 * q + j] * sc;
      const __half h = __float2half_rn(x);
      hh[j] = *reinterpret_cast<const uint16_t*>(&h);
      ll[j] = h16(x - __half2float(h));
    }
    ph[q] = (uint32_t)hh[0] | ((uint32_t)hh[1] << 16);
    pl[q] = (uint32_t)ll[0] | ((uint32_t)ll[1] << 16);
  }
  *hi = make_uint4(ph[0], ph[1], ph[2], ph[3]);
  *lo = make_uint4(pl[0], pl[1], pl[2], pl[3]);
}

}  // namespace mlip
