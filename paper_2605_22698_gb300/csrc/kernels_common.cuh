// Device helpers shared by the interaction kernels.
#pragma once

#include <type_traits>

#include "mlip_internal.cuh"

namespace mlip {

template <int L>
struct NodeDims {
  static constexpr int D = (L + 1) * (L + 1);
};

// Compile-time loop: f(std::integral_constant<int, k>) for k in [B, E).
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    if constexpr (E - B == 1) {
      f(std::integral_constant<int, B>{});
    } else {
      constexpr int M = B + (E - B) / 2;
      static_for<B, M>(f);
      static_for<M, E>(f);
    }
  }
}

// Paths with l1 = 0 come first in lexicographic order.
template <int L>
struct PathInfo {
  using T = CGTable<L>;
  static constexpr int P = T::P;
  static constexpr int NNZ = T::NNZ;
  static constexpr int P0 = L + 1;                  // (0,0,0), (0,1,1), (0,2,2)[, (0,3,3)]
  static constexpr int NNZ0 = T::off[L + 1];        // entries of the l1 = 0 paths
};

// SiLU and its derivative through the logistic sigmoid 1 / (1 + exp(-x)),
// with the fast divide (2 ulp) instead of the IEEE one: exp(-x) overflowing to
// infinity gives sigmoid 0, as it should.
__device__ __forceinline__ float sigmoid_f(float x) { return __fdividef(1.0f, 1.0f + expf(-x)); }
__device__ __forceinline__ float silu_f(float x) { return x * sigmoid_f(x); }
__device__ __forceinline__ float tanh_grad_f(float x) {
  const float t = tanhf(x);
  return 1.0f - t * t;
}
__device__ __forceinline__ float silu_grad_f(float x) {
  const float s = sigmoid_f(x);
  return s * (1.0f + x * (1.0f - s));
}

// Bessel basis times the polynomial envelope, and its r-derivative.
//   e_n = sqrt(2/rc) sin(n pi r / rc) / r * u(r/rc)
//   u(x) = 1 - a x^p + b x^{p+1} - c x^{p+2},  a = (p+1)(p+2)/2, b = p(p+2), c = p(p+1)/2
// evaluated in the algebraically identical factored form
//   u(x)  = (1-x)^3 sum_{k<p} C(k+2, 2) x^k,   u'(x) = -p(p+1)(p+2)/2 x^{p-1} (1-x)^2,
// which keeps FP32 accuracy near the cutoff (the expanded form cancels there).
// (NC functions from n = N0 + 1: e[0..NC) = e_{N0+1..N0+NC}; the full set by default)
template <int NB, bool GRAD, int N0 = 0, int NC = NB>
__device__ __forceinline__ void radial_basis(float r, float rc, int p, float* e, float* de) {
  const float x = r / rc;
  float u = 0.0f, du = 0.0f;
  if (x < 1.0f) {
    const float om = 1.0f - x;
    float poly = 0.0f, xk = 1.0f, xpm1 = 1.0f;
    for (int k = 0; k < p; ++k) {
      poly = fmaf(0.5f * (float)((k + 2) * (k + 1)), xk, poly);
      if (k < p - 1) xpm1 *= x;
      xk *= x;
    }
    u = om * om * om * poly;
    du = -0.5f * (float)(p * (p + 1) * (p + 2)) * xpm1 * om * om / rc;
  }
  const float pref = sqrtf(2.0f / rc);
  const float inv_r = 1.0f / r;
#pragma unroll
  for (int n = N0 + 1; n <= N0 + NC; ++n) {
    const float k = (float)n * 3.14159265358979f / rc;
    float sn, cs;
    sincosf(k * r, &sn, &cs);
    const float B = pref * sn * inv_r;
    e[n - 1 - N0] = B * u;
    if (GRAD) {
      const float dB = pref * (k * cs * inv_r - sn * inv_r * inv_r);
      de[n - 1 - N0] = dB * u + B * du;
    }
  }
}

// Receiver range of block b out of G, balanced by edges: [first receiver with
// row_ptr >= b*E/G, first receiver with row_ptr >= (b+1)*E/G); the last block
// ends at n.
__device__ __forceinline__ int lower_bound_i32(const int* a, int n, long long v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((long long)a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ void block_receivers(const int* row_ptr, int n, int b, int G, int* i0, int* i1) {
  const long long E = row_ptr[n];
  *i0 = (b == 0) ? 0 : lower_bound_i32(row_ptr, n + 1, (E * b) / G);
  *i1 = (b == G - 1) ? n : lower_bound_i32(row_ptr, n + 1, (E * (b + 1)) / G);
  if (*i0 > n) *i0 = n;
  if (*i1 > n) *i1 = n;
}

// Sum 16 values over the 32 lanes; lane l ends with the total of component l >> 1.
__device__ __forceinline__ float warp_reduce16(const float* v) {
  const int lane = threadIdx.x & 31;
  float u[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool hi = lane & 16;
    float send = hi ? v[k] : v[k + 8];
    float keep = hi ? v[k + 8] : v[k];
    u[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool hi = lane & 8;
    float send = hi ? u[k] : u[k + 4];
    float keep = hi ? u[k + 4] : u[k];
    u[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool hi = lane & 4;
    float send = hi ? u[k] : u[k + 2];
    float keep = hi ? u[k + 2] : u[k];
    u[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool hi = lane & 2;
    float send = hi ? u[0] : u[1];
    float keep = hi ? u[1] : u[0];
    u[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  u[0] += __shfl_xor_sync(0xffffffffu, u[0], 1);
  return u[0];
}

// Species index for reading per-species weights: an index outside [0, S) is
// reported by the input check and the call fails, but it must never address
// outside the weights meanwhile.
__device__ __forceinline__ int clamp_species(int z, int S) { return min(max(z, 0), S - 1); }

// out[2 sys] = max(out[2 sys], m) for m >= 0 (float bits ordered as integers);
// one atomic per warp when all its lanes' values belong to one system (sys < 0:
// nothing to add).  Every lane of the warp calls it.
__device__ __forceinline__ void warp_sys_max(float* out, int sys, float m) {
  const int s0 = __shfl_sync(0xffffffffu, sys, 0);
  if (__all_sync(0xffffffffu, sys == s0)) {
    const unsigned mm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    if ((threadIdx.x & 31) == 0 && s0 >= 0) atomicMax(reinterpret_cast<unsigned*>(out) + 2 * s0, mm);
  } else if (sys >= 0) {
    atomicMax(reinterpret_cast<unsigned*>(out) + 2 * sys, __float_as_uint(m));
  }
}

// FP64 form of warp_reduce16: 16 values summed over the 32 lanes, lane l ends
// with the total of component l >> 1 (16 additions per lane instead of 80 for
// 16 separate butterflies; the FP64 pipe is narrow on this part).
__device__ __forceinline__ double warp_reduce16_f64(const double* v) {
  const int lane = threadIdx.x & 31;
  double u[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool hi = lane & 16;
    const double send = hi ? v[k] : v[k + 8];
    const double keep = hi ? v[k + 8] : v[k];
    u[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int w = 4; w >= 1; w >>= 1) {
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const bool hi = lane & (2 * w);
      const double send = hi ? u[k] : u[k + w];
      const double keep = hi ? u[k + w] : u[k];
      u[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * w);
    }
  }
  u[0] += __shfl_xor_sync(0xffffffffu, u[0], 1);
  return u[0];
}

// Sum 32 values over the 32 lanes; lane l ends with the total of value l.
__device__ __forceinline__ float warp_reduce32(const float* v) {
  const int lane = threadIdx.x & 31;
  float u[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const bool hi = lane & 16;
    const float send = hi ? v[k] : v[k + 16];
    const float keep = hi ? v[k + 16] : v[k];
    u[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1) {
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const bool hi = lane & w;
      const float send = hi ? u[k] : u[k + w];
      const float keep = hi ? u[k + w] : u[k];
      u[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return u[0];
}

// Lattice rows of every system of a batch on the device ([nsys][9], zero rows
// for systems without a periodic axis) and the system of each atom (nullptr
// for a batch of one).
struct CellArg {
  const double* cells;
  const int* sys_of;
  int any_pbc;
};

// x_e = (r_j - r_i) + S.h in FP64 (same operation order as the neighbour test),
// rounded to FP32; (x, y, z, |x|).  Lattice rows of the receiver's system.
__device__ __forceinline__ float4 edge_vector(int e, const double* __restrict__ pos, const int* __restrict__ recv,
                                              const int* __restrict__ send, const int8_t* __restrict__ shift,
                                              const CellArg& cell) {
  const int i = recv[e], j = send[e];
  const double S0 = shift[3 * e], S1 = shift[3 * e + 1], S2 = shift[3 * e + 2];
  const double* h = cell.cells + (cell.sys_of ? 9 * cell.sys_of[i] : 0);
  double x[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double sk = 0.0;
    if (cell.any_pbc)
      sk = __dadd_rn(__dadd_rn(__dmul_rn(S0, h[k]), __dmul_rn(S1, h[3 + k])), __dmul_rn(S2, h[6 + k]));
    x[k] = __dadd_rn(__dsub_rn(pos[3 * j + k], pos[3 * i + k]), sk);
  }
  const double r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(x[0], x[0]), __dmul_rn(x[1], x[1])), __dmul_rn(x[2], x[2])));
  return make_float4((float)x[0], (float)x[1], (float)x[2], (float)r);
}

}  // namespace mlip
