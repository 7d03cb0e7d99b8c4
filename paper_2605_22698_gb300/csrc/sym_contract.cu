// Symmetric contraction of correlation order 2 (the product basis of MACE,
// Sec. "Background and related work"; MACE table: correlation 2), applied to
// every node's aggregated messages A between the scatter-sum and the channel
// mix.  For node i of species z and channel c:
//   B[l3 m3] = w1[z][l3][c] A[l3 m3]
//            + sum_q w2[z][q][c] sum_{m1, m2} C^q[m3][m1][m2] A[l1 m1] A[l2 m2]
// over the couplings q = (l1 <= l2 <= L, l3 <= L) of natural parity (the
// generated coupling table's paths with l1 <= l2 <= L, in their order).  The
// adjoint is the product rule on both factors:
//   GA[l1 m1] += w2 C GB[l3 m3] A[l2 m2],  GA[l2 m2] += w2 C GB[l3 m3] A[l1 m1].
// One thread per (node, channel): the node's (L+1)^2 components of its channel
// are loaded (coalesced over channels), contracted in registers with the
// coupling entries as immediates, and written back.  Node-wise and HBM-bound:
// forward reads A (one or two partial buffers) and writes A (kept for the
// adjoint) and B; the adjoint reads GB and A and writes GA.  Both may run in
// place (out == in): a thread reads all its inputs before it writes.
#include <algorithm>
#include <array>

#include "kernels_common.cuh"
#include "launchers.cuh"
#include "mlip_internal.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

// The coupling table's paths used by the contraction: l1 <= l2 <= L.
template <int L>
struct ScPaths {
  using Tab = CGTable<L>;
  static constexpr int count() {
    int q = 0;
    for (int p = 0; p < Tab::P; ++p)
      if (Tab::l1[p] <= Tab::l2[p] && Tab::l2[p] <= L) ++q;
    return q;
  }
  static constexpr int Q = count();
  static constexpr std::array<int, Q> paths() {
    std::array<int, Q> a{};
    int q = 0;
    for (int p = 0; p < Tab::P; ++p)
      if (Tab::l1[p] <= Tab::l2[p] && Tab::l2[p] <= L) a[q++] = p;
    return a;
  }
};

constexpr int kScThreads = 256;

template <int L>
__global__ void __launch_bounds__(kScThreads) sc_fwd(int n, int C, int S, const float* X,
                                                     const float* __restrict__ X2, const int* __restrict__ species,
                                                     const float* __restrict__ w1, const float* __restrict__ w2,
                                                     float* __restrict__ Asave, float* out) {
  using Tab = CGTable<L>;
  using SP = ScPaths<L>;
  constexpr int D = (L + 1) * (L + 1), Q = SP::Q;
  constexpr std::array<int, Q> pq = SP::paths();
  const long long total = (long long)n * C;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / C), c = (int)(idx - (long long)i * C);
    const int z = clamp_species(species[i], S);
    const size_t base = (size_t)i * D * C + c;
    float a[D];
#pragma unroll
    for (int k = 0; k < D; ++k) a[k] = X[base + (size_t)k * C];
    if (X2) {
#pragma unroll
      for (int k = 0; k < D; ++k) a[k] += X2[base + (size_t)k * C];
    }
    float b[D];
#pragma unroll
    for (int l = 0; l <= L; ++l) {
      const float wl = w1[((size_t)z * (L + 1) + l) * C + c];
#pragma unroll
      for (int k = l * l; k < (l + 1) * (l + 1); ++k) b[k] = wl * a[k];
    }
    static_for<0, Q>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      constexpr int p = pq[q], l3 = Tab::l3[p];
      const float wq = w2[((size_t)z * Q + q) * C + c];
      float t[2 * l3 + 1];
#pragma unroll
      for (int k = 0; k < 2 * l3 + 1; ++k) t[k] = 0.0f;
      static_for<Tab::off[p], Tab::off[p + 1]>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int j3 = Tab::e3[k] - l3 * l3, i1 = Tab::e1[k], i2 = Tab::e2[k];
        constexpr float cv = Tab::ec[k];
        t[j3] = fmaf(cv, a[i1] * a[i2], t[j3]);
      });
#pragma unroll
      for (int k = 0; k < 2 * l3 + 1; ++k) b[l3 * l3 + k] = fmaf(wq, t[k], b[l3 * l3 + k]);
    });
#pragma unroll
    for (int k = 0; k < D; ++k) {
      Asave[base + (size_t)k * C] = a[k];
      out[base + (size_t)k * C] = b[k];
    }
  }
}

// out_max (nullable): per system, max |GA| (the FP16 operand scale of the
// message adjoint), at out_max[2 sys].  Each thread keeps a running maximum
// over its grid-stride elements (flushed when its system changes) and the
// warps add theirs once at the end: one atomic per warp per launch instead of
// one per warp per iteration on the same address.
template <int L>
__global__ void __launch_bounds__(kScThreads) sc_bwd(int n, int C, int S, const float* GB, const float* __restrict__ A,
                                                     const int* __restrict__ species, const float* __restrict__ w1,
                                                     const float* __restrict__ w2, float* GA,
                                                     const int* __restrict__ sys_of, float* __restrict__ out_max) {
  using Tab = CGTable<L>;
  using SP = ScPaths<L>;
  constexpr int D = (L + 1) * (L + 1), Q = SP::Q;
  constexpr std::array<int, Q> pq = SP::paths();
  const long long total = (long long)n * C;
  const long long stride = (long long)gridDim.x * blockDim.x;
  float m_run = 0.0f;
  int s_run = -1;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const int i = (int)(idx / C), c = (int)(idx - (long long)i * C);
    float m = 0.0f;
    {
      const int z = clamp_species(species[i], S);
      const size_t base = (size_t)i * D * C + c;
      float g[D], a[D], ga[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        g[k] = GB[base + (size_t)k * C];
        a[k] = A[base + (size_t)k * C];
      }
#pragma unroll
      for (int l = 0; l <= L; ++l) {
        const float wl = w1[((size_t)z * (L + 1) + l) * C + c];
#pragma unroll
        for (int k = l * l; k < (l + 1) * (l + 1); ++k) ga[k] = wl * g[k];
      }
      static_for<0, Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int p = pq[q], l3 = Tab::l3[p];
        const float wq = w2[((size_t)z * Q + q) * C + c];
        float wg[2 * l3 + 1];
#pragma unroll
        for (int k = 0; k < 2 * l3 + 1; ++k) wg[k] = wq * g[l3 * l3 + k];
        static_for<Tab::off[p], Tab::off[p + 1]>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          constexpr int i1 = Tab::e1[k], i2 = Tab::e2[k], j3 = Tab::e3[k] - l3 * l3;
          constexpr float cv = Tab::ec[k];
          const float tq = cv * wg[j3];
          ga[i1] = fmaf(tq, a[i2], ga[i1]);
          ga[i2] = fmaf(tq, a[i1], ga[i2]);
        });
      });
#pragma unroll
      for (int k = 0; k < D; ++k) {
        GA[base + (size_t)k * C] = ga[k];
        m = fmaxf(m, fabsf(ga[k]));
      }
    }
    if (out_max) {
      const int sy = sys_of ? sys_of[i] : 0;
      if (sy != s_run) {
        if (s_run >= 0) atomicMax(reinterpret_cast<unsigned*>(out_max) + 2 * s_run, __float_as_uint(m_run));
        s_run = sy;
        m_run = 0.0f;
      }
      m_run = fmaxf(m_run, m);
    }
  }
  if (out_max) warp_sys_max(out_max, s_run, m_run);  // every lane of the warp reaches this
}

int sc_grid(int n, int C) {
  const long long blocks = ((long long)n * C + kScThreads - 1) / kScThreads;
  return (int)std::max<long long>(1, std::min<long long>(blocks, 152LL * 16));
}

}  // namespace

int sc_num_paths(int L) { return L == 2 ? ScPaths<2>::Q : L == 3 ? ScPaths<3>::Q : 0; }

int launch_sym_contract(int L, int n, int C, int S, const float* X, const float* X2, const int* species, const float* w1,
                        const float* w2, float* Asave, float* out, cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  MLIP_PROF("sym_contract", st);
  if (L == 2) sc_fwd<2><<<sc_grid(n, C), kScThreads, 0, st>>>(n, C, S, X, X2, species, w1, w2, Asave, out);
  else sc_fwd<3><<<sc_grid(n, C), kScThreads, 0, st>>>(n, C, S, X, X2, species, w1, w2, Asave, out);
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_sym_contract_bwd(int L, int n, int C, int S, const float* GB, const float* A, const int* species,
                            const float* w1, const float* w2, float* GA, const int* sys_of, float* out_max,
                            cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  MLIP_PROF("sym_contract_bwd", st);
  if (L == 2) sc_bwd<2><<<sc_grid(n, C), kScThreads, 0, st>>>(n, C, S, GB, A, species, w1, w2, GA, sys_of, out_max);
  else sc_bwd<3><<<sc_grid(n, C), kScThreads, 0, st>>>(n, C, S, GB, A, species, w1, w2, GA, sys_of, out_max);
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace mlip
