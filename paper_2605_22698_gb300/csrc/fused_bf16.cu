// Fused tensor-core form of the interaction layer (16-bit operands: BF16, or
// FP16 for the tighter error bar, with FP32 accumulation in tensor memory).
//
// Per layer:
//   radial_tc     (radial_tc.cu) r -> Bessel x envelope -> z1 -> z2 per edge,
//                 z2 written as BF16 or FP16 in the tcgen05 canonical K-major layout,
//                 one 4 KB tile per kNT = 32 consecutive (receiver-sorted) edges
//   tp_fused      one launch per path group (all l1 = 0 paths for the first
//                 layer, else the paths of one output order l3).  Each CTA keeps
//                 its group's W3 slices resident in shared memory (bulk-copied
//                 once), streams the z2 tiles of its balanced receiver range
//                 through a double buffer with 1-D bulk copies, and per tile
//                 issues one tcgen05.mma (M = 128 channels, N = 32 edges,
//                 K = 64) per path: w[c][e] = W3_p^T z2 lands in tensor memory.
//                 Thread c then reads its lane (channel c) with tcgen05.ld and
//                 runs the FP32 tensor product for its channel over the tile's
//                 edges, accumulating the receiver's message in registers and
//                 flushing it at segment ends (no atomics).
// The per-edge radial weights never reach HBM.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <memory>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels_common.cuh"
#include "launchers.cuh"
#include "profile.cuh"
#include "sm100_tc.cuh"

namespace mlip {
namespace {

constexpr int kNT = 32;           // edges per tile (MMA N)

// 16-bit operand encodings (bits of a BF16 or FP16 value)
__host__ __device__ inline uint16_t to16(float x, bool bf16) {
  if (bf16) {
    const __nv_bfloat16 v = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t*>(&v);
  }
  const __half v = __float2half_rn(x);
  return *reinterpret_cast<const uint16_t*>(&v);
}
// Two FP32 values as 16-bit operands (a in the low half, b in the high half),
// round to nearest, one packed conversion.
__device__ __forceinline__ uint32_t pack16x2(float a, float b, bool bf16) {
  if (bf16) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
  }
  const __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
constexpr int kTileBytes = kNT * 64 * 2;
constexpr int kW3PathBytes = 128 * 64 * 2;

// ------------------------------------------------------------ path groups
// MODE < 0: the l1 = 0 paths (first layer, scalar inputs); MODE = l: paths with l3 = l.
template <int L, int MODE>
struct Group {
  using Tab = CGTable<L>;
  static constexpr bool sel(int p) { return MODE < 0 ? Tab::l1[p] == 0 : Tab::l3[p] == MODE; }
  static constexpr int count() {
    int n = 0;
    for (int p = 0; p < Tab::P; ++p) n += sel(p) ? 1 : 0;
    return n;
  }
  static constexpr int NP = count();
  static constexpr std::array<int, NP> make_paths() {
    std::array<int, NP> a{};
    int n = 0;
    for (int p = 0; p < Tab::P; ++p)
      if (sel(p)) a[n++] = p;
    return a;
  }
  static constexpr std::array<int, NP> paths = make_paths();
  // offset of each member path's entries in the group's entry list; every
  // path starts on a multiple of 4 (16-byte vector loads), padding entries zero
  static constexpr std::array<int, NP + 1> make_eoff() {
    std::array<int, NP + 1> a{};
    for (int s = 0; s < NP; ++s) a[s + 1] = a[s] + ((Tab::off[paths[s] + 1] - Tab::off[paths[s]] + 3) & ~3);
    return a;
  }
  static constexpr std::array<int, NP + 1> eoff = make_eoff();
  static constexpr int NZ = eoff[NP];
  static constexpr int NZP = (NZ + 3) & ~3;
  // output components written: [comp0, comp0 + NOUT)
  static constexpr int comp0 = MODE < 0 ? 0 : MODE * MODE;
  static constexpr int NOUT = MODE < 0 ? (L + 1) * (L + 1) : 2 * MODE + 1;
  static constexpr int max_l1() {
    int m = 0;
    for (int s = 0; s < NP; ++s) m = Tab::l1[paths[s]] > m ? Tab::l1[paths[s]] : m;
    return m;
  }
  static constexpr int DH = (max_l1() + 1) * (max_l1() + 1);  // sender components read
  static constexpr int tmem_cols() {
    int need = NP * kNT, c = 32;
    while (c < need) c <<= 1;
    return c;
  }
  static constexpr int NCOLS = tmem_cols();
  static constexpr size_t smem_bytes() {
    return (size_t)NP * kW3PathBytes + 2 * kTileBytes + (size_t)kNT * NZP * 4 + 2 * kNT * 4 + 64;
  }
};

// ------------------------------------------------------------ warp sets
// A CTA runs kWS warp sets of 4 warps (128 threads, one per channel and TMEM
// lane).  Every warp set writes its partial sums to an output buffer of its
// own (the next mix adds the buffers), so the warp sets never wait for each
// other inside a tile.
constexpr int kWS = 2;
constexpr int kThreads = 128 * kWS;
// Work split between the two warp sets of a CTA: every set runs all of the
// group's paths (one copy of the per-edge code for both sets, each edge's
// sender rows gathered once) on its own edges of the tile.  An edge belongs to
// set (its position within its receiver's edge segment) & 1: a receiver's
// edges alternate between the sets, so each set's share of a receiver, and the
// order in which it is summed, do not depend on where tile boundaries fall
// (a system's results do not depend on the other systems of its batch).
constexpr bool kEdgeSplit = true;
static_assert(kEdgeSplit, "the adjoint's dE/dY partial buffers hold one warp set per edge");

// Per-tile edge lists of the two sets, built by one warp (lane t = edge slot t).
__device__ __forceinline__ void build_lists(int t, bool valid, int par, int* s_list, int* s_cnt) {
  const unsigned lt = (1u << t) - 1u;
  const unsigned m0 = __ballot_sync(0xffffffffu, valid && par == 0);
  const unsigned m1 = __ballot_sync(0xffffffffu, valid && par == 1);
  if (valid) {
    if (par == 0) s_list[__popc(m0 & lt)] = t;
    else s_list[kNT + __popc(m1 & lt)] = t;
  }
  if (t == 0) {
    s_cnt[0] = __popc(m0);
    s_cnt[1] = __popc(m1);
  }
}


template <int L, int MODE, bool BWD>
struct Split {
  using G = Group<L, MODE>;
  using Tab = CGTable<L>;
  static constexpr int NP = G::NP;
  static constexpr int cost(int p) {
    const int nz = Tab::off[p + 1] - Tab::off[p];
    const int l1 = Tab::l1[p], l2 = Tab::l2[p], l3 = Tab::l3[p];
    if (!BWD) return (2 * l1 + 1) + 2 * nz;
    return (MODE < 0 ? 0 : 2 * (2 * l3 + 1) + 2 * nz) + 3 * nz + 4 * (2 * l2 + 1);
  }
  static constexpr std::array<int, NP> make() {
    std::array<int, NP> ws{};
    if (kEdgeSplit) return ws;  // every warp set runs every path, on its own edges
    std::array<bool, NP> done{};
    int load[kWS] = {};
    for (int it = 0; it < NP; ++it) {
      int best = -1;
      for (int s = 0; s < NP; ++s)
        if (!done[s] && (best < 0 || cost(G::paths[s]) > cost(G::paths[best]))) best = s;
      int w = 0;
      for (int k = 1; k < kWS; ++k)
        if (load[k] < load[w]) w = k;
      ws[best] = w;
      load[w] += cost(G::paths[best]);
      done[best] = true;
    }
    return ws;
  }
  static constexpr std::array<int, NP> ws = make();
  // harmonic components l2 m2 touched by warp set W (bit mask over 16)
  static constexpr int ymask(int W) {
    int m = 0;
    for (int s = 0; s < NP; ++s)
      if (ws[s] == W) {
        const int l2 = Tab::l2[G::paths[s]];
        for (int q = 0; q < 2 * l2 + 1; ++q) m |= 1 << (l2 * l2 + q);
      }
    return m;
  }
  static constexpr int nyv(int W) { return __builtin_popcount(ymask(W)); }
  // edges packed into one 16-value channel butterfly
  static constexpr int ypack(int W) { return nyv(W) <= 4 ? 4 : (nyv(W) <= 8 ? 2 : 1); }
  static constexpr std::array<int, 16> ylist(int W) {
    std::array<int, 16> a{};
    int n = 0;
    for (int k = 0; k < 16; ++k)
      if (ymask(W) >> k & 1) a[n++] = k;
    return a;
  }
  // sender components read by warp set W (max l1 of its paths)
  static constexpr int dh(int W) {
    int m = -1;
    for (int s = 0; s < NP; ++s)
      if (ws[s] == W && Tab::l1[G::paths[s]] > m) m = Tab::l1[G::paths[s]];
    return m < 0 ? 1 : (m + 1) * (m + 1);
  }
};

// Per-CTA copy of the group's CG entries for the per-tile products c * Y:
// coefficient (with the reverse-edge sign (-1)^l2 when SIGNED) and Y index.
template <int L, int MODE, bool SIGNED>
__device__ __forceinline__ void load_group_table(float* tab_c, uint8_t* tab_y) {
  using G = Group<L, MODE>;
  using Tab = CGTable<L>;
  const int tid = threadIdx.x;
  static_for<0, G::NP>([&](auto sc) {
    constexpr int sl = decltype(sc)::value;
    constexpr int p = G::paths[sl];
    constexpr int kb = Tab::off[p], ke = Tab::off[p + 1], gb = G::eoff[sl];
    static_for<kb, ke>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr float cv = ((SIGNED && (Tab::l2[p] & 1)) ? -1.0f : 1.0f) * Tab::ec[k];
      constexpr int i2 = Tab::e2[k];
      if (tid == gb + k - kb) {
        tab_c[gb + k - kb] = cv;
        tab_y[gb + k - kb] = (uint8_t)i2;
      }
    });
    if (tid >= gb + (ke - kb) && tid < G::eoff[sl + 1]) {  // padding up to the next path
      tab_c[tid] = 0.0f;
      tab_y[tid] = 0;
    }
  });
}

// Per tile: receiver/sender ids and harmonics (threads < kNT), then the
// products cY[t][k] = c_k Y_t[i2_k] by all threads.
// With s_dws (adjoint): s_dws[t], s_dws[kNT + t] = the scale of edge t's
// system and its inverse (dws2[system], see dw_scales).
template <int NZ, int NZP>
__device__ __forceinline__ void tile_setup(int tile, int E0, int E1, const int* __restrict__ recv,
                                           const int* __restrict__ send, const float* __restrict__ Yg, int* s_recv,
                                           int* s_send, float* sY, float* cY, const float* tab_c,
                                           const uint8_t* tab_y, const uint8_t* __restrict__ epar, int* s_list,
                                           int* s_cnt, int* s_own, const int* __restrict__ sys_of = nullptr,
                                           const float2* __restrict__ dws2 = nullptr, float* s_dws = nullptr) {
  const int tid = threadIdx.x;
  if (tid < kNT) {
    const int e = tile * kNT + tid;
    const bool valid = e >= E0 && e < E1;
    const int r = valid ? recv[e] : -1;
    const int par = valid ? epar[e] : 0;
    s_recv[tid] = r;
    s_send[tid] = valid ? send[e] : 0;
    if (s_own) s_own[tid] = valid ? par : -1;
    build_lists(tid, valid, par, s_list, s_cnt);
    if (s_dws) {
      const float2 v = valid ? dws2[sys_of ? sys_of[r] : 0] : make_float2(1.0f, 1.0f);
      s_dws[tid] = v.x;
      s_dws[kNT + tid] = v.y;
    }
  }
  for (int q = tid; q < kNT * 4; q += blockDim.x) {  // 16 floats per edge as float4
    const int t = q >> 2, e = tile * kNT + t;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e >= E0 && e < E1) v = reinterpret_cast<const float4*>(Yg)[(size_t)e * 4 + (q & 3)];
    reinterpret_cast<float4*>(sY)[q] = v;
  }
  __syncthreads();
  if (NZ > 0) {
    for (int q = tid; q < kNT * NZ; q += blockDim.x) {
      const int t = q / NZ, k = q - t * NZ;
      cY[t * NZP + k] = tab_c[k] * sY[t * 16 + tab_y[k]];
    }
  }
}

// Real harmonics of every edge direction, Y[e][16] (once per evaluation), and
// (par != nullptr) the parity of the edge's position in its receiver's
// segment (which warp set of the message kernels takes it).
// The edge vector ev[e] (edge_vector) comes first in the same pass.
__global__ void edge_sh(int E, const double* __restrict__ pos, const int* __restrict__ send,
                        const int8_t* __restrict__ shift, CellArg cell, float4* __restrict__ ev,
                        float* __restrict__ Yg, const int* __restrict__ Edev, const int* __restrict__ row_ptr,
                        const int* __restrict__ recv, uint8_t* __restrict__ par) {
  if (Edev) E = *Edev;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    if (par) par[e] = (uint8_t)((e - row_ptr[recv[e]]) & 1);
    const float4 v = edge_vector(e, pos, recv, send, shift, cell);
    ev[e] = v;
    const float ir = 1.0f / v.w;
    float Y[16];
    sh3<float>(v.x * ir, v.y * ir, v.z * ir, Y);
    float4* dst = reinterpret_cast<float4*>(Yg + (size_t)e * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_float4(Y[4 * q], Y[4 * q + 1], Y[4 * q + 2], Y[4 * q + 3]);
  }
}

// p[0 .. per * *Edev) = 0 (p 16-byte aligned)
__global__ void zero_edges(const int* __restrict__ Edev, int per, float* __restrict__ p) {
  const long long n = (long long)(*Edev) * per, n4 = n >> 2;
  float4* q = reinterpret_cast<float4*>(p);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x)
    q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (blockIdx.x == 0 && threadIdx.x < (int)(n & 3)) p[(n4 << 2) + threadIdx.x] = 0.0f;
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr));
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
}
template <int CH>
__device__ __forceinline__ void tmem_ldn(uint32_t taddr, float* v);
template <>
__device__ __forceinline__ void tmem_ldn<4>(uint32_t taddr, float* v) { tmem_ld4(taddr, v); }
template <>
__device__ __forceinline__ void tmem_ldn<8>(uint32_t taddr, float* v) { tc::tmem_ld8(taddr, v); }

// Edges per chunk of the per-warp-set loop: the sender gathers of the next
// chunk are issued before the current chunk is computed, so light groups
// (little work per edge) take longer chunks.
template <int WORK>
constexpr int chunk_edges() { return WORK <= 8 ? 8 : 4; }

__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float* v) {
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr));
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
}

// ---------------------------------------------------------------- tp_fused
// CTAs of a fused kernel that fit on one SM by shared memory (at most 2):
// the register budget per thread follows from it (128 for 2, 255 for 1).
constexpr int ctas_per_sm(size_t smem_bytes) { return (smem_bytes + 2048) * 2 <= 232448 ? 2 : 1; }

template <int L, int MODE>
struct FwdLayout {
  using G = Group<L, MODE>;
  static constexpr int NP = G::NP;
  static constexpr size_t off_z2 = (size_t)NP * kW3PathBytes;
  static constexpr size_t off_cy = off_z2 + 2 * kTileBytes;
  static constexpr size_t off_y = off_cy + (size_t)kNT * G::NZP * 4;
  static constexpr size_t off_tab = off_y + kNT * 16 * 4;
  static constexpr size_t off_taby = off_tab + (size_t)G::NZP * 4;
  static constexpr size_t off_idx = off_taby + (((size_t)G::NZP + 15) & ~(size_t)15);
  static constexpr size_t off_bar = off_idx + 2 * kNT * 4;
  static constexpr size_t bytes = off_bar + 64;
  static_assert(bytes <= 232448 - 1024, "shared memory of the forward kernel exceeds the per-block limit");
};

// N 16-byte shared-memory loads into v[4N] (src 16-byte aligned).
template <int N>
__device__ __forceinline__ void load4(const float* src, float* v) {
#pragma unroll
  for (int q = 0; q < N; ++q) {
    const float4 x = reinterpret_cast<const float4*>(src)[q];
    v[4 * q] = x.x;
    v[4 * q + 1] = x.y;
    v[4 * q + 2] = x.z;
    v[4 * q + 3] = x.w;
  }
}

template <int L, int MODE, int W>
__device__ __forceinline__ void fwd_edge(const float* wv, const float* hj, const float* cy, float* acc) {
  using G = Group<L, MODE>;
  using S = Split<L, MODE, false>;
  using Tab = CGTable<L>;
  static_for<0, G::NP>([&](auto sc) {
    constexpr int sl = decltype(sc)::value;
    if constexpr (S::ws[sl] == W) {
      constexpr int p = G::paths[sl];
      constexpr int l1 = Tab::l1[p];
      constexpr int kb = Tab::off[p], ke = Tab::off[p + 1], gb = G::eoff[sl];
      float wh[2 * l1 + 1];
#pragma unroll
      for (int q = 0; q < 2 * l1 + 1; ++q) wh[q] = wv[sl] * hj[l1 * l1 + q];
      float c4[(ke - kb + 3) & ~3];
      load4<(ke - kb + 3) / 4>(cy + gb, c4);
      static_for<kb, ke>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int o3 = Tab::e3[k] - G::comp0, j1 = Tab::e1[k] - l1 * l1;
        acc[o3] = fmaf(c4[k - kb], wh[j1], acc[o3]);
      });
    }
  });
}

// Hint: the 128-byte line at p into L1 (no register written).
__device__ __forceinline__ void prefetch_l1(const float* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// One warp set over one tile: 2-edge chunks, sender features prefetched one
// chunk ahead, partial messages flushed (times s) into this warp set's buffer.
template <int L, int MODE, int W, int CHO = 0>
__device__ __forceinline__ void fwd_tile_ws(const int* s_send, const int* s_recv, const float* cY, uint32_t taddr0,
                                            const float* __restrict__ h, int& cur, float* acc,
                                            float* __restrict__ mW, float s, const int* list, int cnt) {
  using G = Group<L, MODE>;
  using S = Split<L, MODE, false>;
  constexpr int D = NodeDims<L>::D;
  constexpr int C = 128;
  constexpr int DH = S::dh(W);
  constexpr int CH = CHO > 0 ? CHO : chunk_edges<DH>();  // edges per chunk (CHO: set by the caller)
  const int c = threadIdx.x & 127;
  if (cnt <= 0) return;  // uniform over the warp set
  auto slot = [&](int i) { return list[i < cnt ? i : cnt - 1]; };
  float hn[CH][DH];
#pragma unroll
  for (int j = 0; j < CH; ++j) {
    const int sj = s_send[slot(j)];
#pragma unroll
    for (int d = 0; d < DH; ++d) hn[j][d] = h[((size_t)sj * D + d) * C + c];
  }
#pragma unroll 1
  for (int base = 0; base < cnt; base += CH) {
    float wvc[G::NP][CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int t = slot(base + j);
      static_for<0, G::NP>([&](auto sc) {
        constexpr int sl = decltype(sc)::value;
        if constexpr (S::ws[sl] == W) wvc[sl][j] = tmem_ld1(taddr0 + sl * kNT + t);
      });
    }
    tc::tmem_ld_wait();
    float hc[CH][DH];
#pragma unroll
    for (int j = 0; j < CH; ++j)
#pragma unroll
      for (int d = 0; d < DH; ++d) hc[j][d] = hn[j][d];
    if (base + CH < cnt) {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int sj = s_send[slot(base + CH + j)];
#pragma unroll
        for (int d = 0; d < DH; ++d) hn[j][d] = h[((size_t)sj * D + d) * C + c];
      }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      if (base + j >= cnt) break;
      const int t = list[base + j];
      const int r = s_recv[t];
      while (cur < r) {
#pragma unroll
        for (int q = 0; q < G::NOUT; ++q) {
          mW[((size_t)cur * D + G::comp0 + q) * C + c] = s * acc[q];
          acc[q] = 0.0f;
        }
        ++cur;
      }
      float wv[G::NP];
#pragma unroll
      for (int sl = 0; sl < G::NP; ++sl) wv[sl] = wvc[sl][j];
      fwd_edge<L, MODE, W>(wv, hc[j], cY + t * G::NZP, acc);
    }
  }
}

template <int L, int MODE>
__global__ void __launch_bounds__(kThreads, ctas_per_sm(FwdLayout<L, MODE>::bytes)) tp_fused(int n, const int* __restrict__ row_ptr,
                                                     const int* __restrict__ recv, const int* __restrict__ send,
                                                     const float* __restrict__ Yg, const float* __restrict__ h,
                                                     const uint8_t* __restrict__ w3img,
                                                     const uint8_t* __restrict__ z2t, float s, float* __restrict__ mA,
                                                     float* __restrict__ mB, int use_bf16,
                                                     const uint8_t* __restrict__ epar, int* __restrict__ err) {
  using G = Group<L, MODE>;
  using FL = FwdLayout<L, MODE>;
  constexpr int D = NodeDims<L>::D;
  constexpr int C = 128;
  constexpr int NP = G::NP;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sW3 = smem;
  uint8_t* sZ2 = smem + FL::off_z2;
  float* cY = reinterpret_cast<float*>(smem + FL::off_cy);
  float* sY = reinterpret_cast<float*>(smem + FL::off_y);
  float* tab_c = reinterpret_cast<float*>(smem + FL::off_tab);
  uint8_t* tab_y = smem + FL::off_taby;
  int* s_send = reinterpret_cast<int*>(smem + FL::off_idx);
  int* s_recv = s_send + kNT;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + FL::off_bar);
  uint64_t* bar_w3 = bars;
  uint64_t* bar_z2 = bars + 1;  // [2]
  uint64_t* bar_mma = bars + 3;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 4);
  __shared__ int abort_s;
  __shared__ int s_list[2 * kNT], s_cnt[2];  // the warp sets' edges of the tile

  const int tid = threadIdx.x, warp = tid >> 5, c = tid & 127, wsid = warp >> 2;
  float* mW = wsid == 0 ? mA : mB;
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, G::NCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(bar_w3, 1);
    tc::mbar_init(bar_z2, 1);
    tc::mbar_init(bar_z2 + 1, 1);
    tc::mbar_init(bar_mma, 1);
    tc::fence_mbar_init();
    abort_s = 0;
  }
  load_group_table<L, MODE, false>(tab_c, tab_y);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tmem_holder;
  const uint32_t taddr0 = tbase + ((uint32_t)((warp & 3) * 32) << 16);

  int i0, i1;
  block_receivers(row_ptr, n, blockIdx.x, gridDim.x, &i0, &i1);
  const int E0 = row_ptr[i0], E1 = row_ptr[i1];
  const int t_begin = E0 / kNT, t_end = (E1 > E0) ? (E1 + kNT - 1) / kNT : t_begin;
  const int n_tiles = t_end - t_begin;

  int z2_issued[2] = {0, 0}, z2_waited[2] = {0, 0};
  bool w3_issued = false;
  if (tid == 0 && n_tiles > 0) {
    tc::mbar_arrive_expect_tx(bar_w3, NP * kW3PathBytes);
#pragma unroll 1
    for (int sl = 0; sl < NP; ++sl)
      tc::bulk_g2s(sW3 + sl * kW3PathBytes, w3img + (size_t)sl * kW3PathBytes, kW3PathBytes, bar_w3);
    w3_issued = true;
    tc::mbar_arrive_expect_tx(bar_z2, kTileBytes);
    tc::bulk_g2s(sZ2, z2t + (size_t)t_begin * kTileBytes, kTileBytes, bar_z2);
    z2_issued[0] = 1;
  }

  float acc[G::NOUT];
#pragma unroll
  for (int q = 0; q < G::NOUT; ++q) acc[q] = 0.0f;
  int cur = i0;
  const uint32_t idesc = tc::idesc_16bit(128, kNT, use_bf16 != 0);

#pragma unroll 1
  for (int it = 0; it < n_tiles; ++it) {
    const int tile = t_begin + it;
    const int buf = it & 1;
    if (tid == 0) {
      bool ok = true;
      if (it + 1 < n_tiles) {
        const int nb = buf ^ 1;
        tc::mbar_arrive_expect_tx(bar_z2 + nb, kTileBytes);
        tc::bulk_g2s(sZ2 + nb * kTileBytes, z2t + (size_t)(tile + 1) * kTileBytes, kTileBytes, bar_z2 + nb);
        z2_issued[nb]++;
      }
      if (it == 0) ok = ok && tc::mbar_wait(bar_w3, 0);
      ok = ok && tc::mbar_wait(bar_z2 + buf, (uint32_t)(z2_waited[buf] & 1));
      if (ok) {
        z2_waited[buf]++;
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(sW3), b0 = tc::smem_u32(sZ2 + buf * kTileBytes);
#pragma unroll 1
        for (int sl = 0; sl < NP; ++sl)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = tc::desc_noswizzle(a0 + sl * kW3PathBytes + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
            const uint64_t bd = tc::desc_noswizzle(b0 + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
            tc::mma_bf16(tbase + sl * kNT, ad, bd, idesc, kk > 0 ? 1u : 0u);
          }
        tc::mma_commit(bar_mma);
      } else {
        atomicOr(err, 1);
        abort_s = 1;
      }
    }
    tile_setup<G::NZ, G::NZP>(tile, E0, E1, recv, send, Yg, s_recv, s_send, sY, cY, tab_c, tab_y, epar, s_list, s_cnt,
                              nullptr);
    __syncthreads();
    if (abort_s) break;
    if (!tc::mbar_wait(bar_mma, (uint32_t)(it & 1))) {
      atomicOr(err, 2);
      abort_s = 1;
    }
    tc::fence_after_sync();
    // two CTAs per SM leave 128 registers a thread: 2-edge chunks when an edge carries the 16 sender
    // components of l1 <= 3 (4-edge chunks of them spill)
    constexpr int CHO = (ctas_per_sm(FwdLayout<L, MODE>::bytes) == 2 && Split<L, MODE, false>::dh(0) > 12) ? 2 : 0;
    fwd_tile_ws<L, MODE, 0, CHO>(s_send, s_recv, cY, taddr0, h, cur, acc, mW, s, s_list + wsid * kNT, s_cnt[wsid]);
    tc::fence_before_sync();
    __syncthreads();
    if (abort_s) break;
  }
  if (!abort_s) {
    while (cur < i1) {
#pragma unroll
      for (int q = 0; q < G::NOUT; ++q) {
        mW[((size_t)cur * D + G::comp0 + q) * C + c] = s * acc[q];
        acc[q] = 0.0f;
      }
      ++cur;
    }
  }
  if (tid == 0) {
    if (w3_issued && n_tiles > 0) tc::mbar_wait(bar_w3, 0, 1LL << 20);
    for (int b = 0; b < 2; ++b)
      while (z2_waited[b] < z2_issued[b]) {
        if (!tc::mbar_wait(bar_z2 + b, (uint32_t)(z2_waited[b] & 1), 1LL << 20)) break;
        z2_waited[b]++;
      }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, G::NCOLS);
}

// Pipelined forward for the groups that fit one CTA per SM: two producer warps
// prepare tile it + 1 (ids, edge lists, harmonics, c.Y products, the z2 copy
// and the product w = W3^T z2 into the other of two tensor-memory buffers)
// while the eight consumer warps run tile it; mbarriers full / done per buffer
// order them, so the consumers never wait at a CTA-wide barrier.
// Pipelined kernels (forward and adjoint): two warp sets of consumers, two producer warps.
constexpr int kWSConsumers = 256, kWSProducers = 64, kWSThreads = kWSConsumers + kWSProducers;
constexpr int kWSFChunk = 2;  // consumers' edges per chunk (register budget of 10 warps per SM)

template <int L, int MODE>
struct FwdLayoutWS {
  using G = Group<L, MODE>;
  static constexpr int NP = G::NP;
  static constexpr int tmem_cols() {
    int need = 2 * NP * kNT, c = 32;
    while (c < need) c <<= 1;
    return c;
  }
  static constexpr int NCOLS = tmem_cols();
  static constexpr size_t off_z2 = (size_t)NP * kW3PathBytes;
  static constexpr size_t off_cy = off_z2 + 2 * kTileBytes;
  static constexpr size_t off_y = off_cy + 2 * (size_t)kNT * G::NZP * 4;
  static constexpr size_t off_tab = off_y + 2 * kNT * 16 * 4;
  static constexpr size_t off_taby = off_tab + (size_t)G::NZP * 4;
  static constexpr size_t off_idx = off_taby + (((size_t)G::NZP + 15) & ~(size_t)15);
  static constexpr size_t off_bar = off_idx + 2 * 2 * kNT * 4;
  static constexpr size_t bytes = off_bar + 128;
  static constexpr bool fits = bytes <= 232448 - 1024 && NCOLS <= 512;
};

template <int L, int MODE>
__global__ void __launch_bounds__(kWSThreads, 1)
    tp_fused_ws(int n, const int* __restrict__ row_ptr, const int* __restrict__ recv, const int* __restrict__ send,
                const float* __restrict__ Yg, const float* __restrict__ h, const uint8_t* __restrict__ w3img,
                const uint8_t* __restrict__ z2t, float s, float* __restrict__ mA, float* __restrict__ mB,
                int use_bf16, const uint8_t* __restrict__ epar, int* __restrict__ err) {
  using G = Group<L, MODE>;
  using FL = FwdLayoutWS<L, MODE>;
  static_assert(FL::fits, "shared or tensor memory of the pipelined forward kernel exceeds the per-SM limits");
  constexpr int D = NodeDims<L>::D;
  constexpr int C = 128;
  constexpr int NP = G::NP;
  constexpr int NZ = G::NZ, NZP = G::NZP;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sW3 = smem;
  uint8_t* sZ2 = smem + FL::off_z2;
  float* cYb = reinterpret_cast<float*>(smem + FL::off_cy);
  float* sYb = reinterpret_cast<float*>(smem + FL::off_y);
  float* tab_c = reinterpret_cast<float*>(smem + FL::off_tab);
  uint8_t* tab_y = smem + FL::off_taby;
  int* idxb = reinterpret_cast<int*>(smem + FL::off_idx);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + FL::off_bar);
  uint64_t* bar_w3 = bars;
  uint64_t* bar_z2 = bars + 1;    // [2]
  uint64_t* bar_full = bars + 3;  // [2]
  uint64_t* bar_done = bars + 5;  // [2]
  uint64_t* bar_fin = bars + 7;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 8);
  __shared__ volatile int abort_s;
  __shared__ int abort_p;
  __shared__ int s_lists[2][2 * kNT], s_cnts[2][2];

  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, FL::NCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(bar_w3, 1);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(bar_z2 + b, 1);
      tc::mbar_init(bar_full + b, kWSProducers + 1);
      tc::mbar_init(bar_done + b, kWSConsumers);
    }
    tc::mbar_init(bar_fin, 1);
    tc::fence_mbar_init();
    abort_s = 0;
    abort_p = 0;
  }
  load_group_table<L, MODE, false>(tab_c, tab_y);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tmem_holder;
  const uint32_t wcol0 = 0, wcol1 = NP * kNT;

  int i0, i1;
  block_receivers(row_ptr, n, blockIdx.x, gridDim.x, &i0, &i1);
  const int E0 = row_ptr[i0], E1 = row_ptr[i1];
  const int t_begin = E0 / kNT, t_end = (E1 > E0) ? (E1 + kNT - 1) / kNT : t_begin;
  const int n_tiles = t_end - t_begin;
  const uint32_t idesc = tc::idesc_16bit(128, kNT, use_bf16 != 0);

  if (warp >= 8) {
    // ---------------------------------------------------------- producers
    const int pt = tid - kWSConsumers;  // 0..63
    const bool elect = pt == 0;
    int z2_issued[2] = {0, 0}, z2_waited[2] = {0, 0};
    bool w3_waited = false;
    if (elect && n_tiles > 0) {
      tc::mbar_arrive_expect_tx(bar_w3, NP * kW3PathBytes);
#pragma unroll 1
      for (int sl = 0; sl < NP; ++sl)
        tc::bulk_g2s(sW3 + sl * kW3PathBytes, w3img + (size_t)sl * kW3PathBytes, kW3PathBytes, bar_w3);
    }
    auto setup = [&](int it) {  // tile it into buffer b = it & 1
      const int b = it & 1, tile = t_begin + it;
      int* s_send = idxb + b * 2 * kNT;
      int* s_recv = s_send + kNT;
      float* sY = sYb + b * kNT * 16;
      float* cY = cYb + b * kNT * NZP;
      if (elect) {
        tc::mbar_arrive_expect_tx(bar_z2 + b, kTileBytes);
        tc::bulk_g2s(sZ2 + b * kTileBytes, z2t + (size_t)tile * kTileBytes, kTileBytes, bar_z2 + b);
        z2_issued[b]++;
      }
      if (pt < kNT) {  // one warp: lane = edge slot
        const int e = tile * kNT + pt;
        const bool valid = e >= E0 && e < E1;
        s_recv[pt] = valid ? recv[e] : -1;
        s_send[pt] = valid ? send[e] : 0;
        build_lists(pt, valid, valid ? epar[e] : 0, s_lists[b], s_cnts[b]);
      }
      for (int q = pt; q < kNT * 4; q += kWSProducers) {
        const int t = q >> 2, e = tile * kNT + t;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e >= E0 && e < E1) v = reinterpret_cast<const float4*>(Yg)[(size_t)e * 4 + (q & 3)];
        reinterpret_cast<float4*>(sY)[q] = v;
      }
      tc::named_bar(1, kWSProducers);
      for (int q = pt; q < kNT * NZ; q += kWSProducers) {
        const int t = q / NZ, k = q - t * NZ;
        cY[t * NZP + k] = tab_c[k] * sY[t * 16 + tab_y[k]];
      }
      if (elect) {
        bool ok = true;
        if (!w3_waited) ok = w3_waited = tc::mbar_wait(bar_w3, 0);
        ok = ok && tc::mbar_wait(bar_z2 + b, (uint32_t)(z2_waited[b] & 1));
        if (ok) {
          z2_waited[b]++;
          tc::fence_after_sync();
          const uint32_t a0 = tc::smem_u32(sW3), b0 = tc::smem_u32(sZ2 + b * kTileBytes);
          const uint32_t wcol = b ? wcol1 : wcol0;
#pragma unroll 1
          for (int sl = 0; sl < NP; ++sl)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = tc::desc_noswizzle(a0 + sl * kW3PathBytes + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
              const uint64_t bd = tc::desc_noswizzle(b0 + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
              tc::mma_bf16(tbase + wcol + sl * kNT, ad, bd, idesc, kk > 0 ? 1u : 0u);
            }
          tc::mma_commit(bar_full + b);
        } else {
          atomicOr(err, 1);
          abort_s = 1;
          tc::mbar_arrive(bar_full + b);  // completes the phase so the consumers see the abort
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(bar_full + b);
    };
    auto stop = [&]() -> bool {  // one decision for all producer threads (named barriers must not diverge)
      if (elect) abort_p = abort_s;
      tc::named_bar(1, kWSProducers);
      const bool st = abort_p != 0;
      tc::named_bar(1, kWSProducers);
      return st;
    };
    if (n_tiles > 0) setup(0);
#pragma unroll 1
    for (int it = 0; it + 1 < n_tiles; ++it) {
      if (stop()) break;
      // buffer (it + 1) & 1 was last read by the consumers' tile it - 1
      if (it >= 1 && !tc::mbar_wait_sleep(bar_done + ((it + 1) & 1), (uint32_t)(((it - 1) >> 1) & 1))) {
        atomicOr(err, 2);
        abort_s = 1;
      }
      if (stop()) break;
      tc::fence_after_sync();
      setup(it + 1);
    }
    if (elect) {
      for (int b = 0; b < 2; ++b)
        while (z2_waited[b] < z2_issued[b]) {
          if (!tc::mbar_wait(bar_z2 + b, (uint32_t)(z2_waited[b] & 1), 1LL << 20)) break;
          z2_waited[b]++;
        }
      if (n_tiles > 0 && !w3_waited) tc::mbar_wait(bar_w3, 0, 1LL << 20);
      tc::mma_commit(bar_fin);  // every product issued by this thread
    }
  } else {
    // ---------------------------------------------------------- consumers
    const int wsid = warp >> 2, c = tid & 127;
    float* mW = wsid == 0 ? mA : mB;
    const uint32_t taddr0 = tbase + ((uint32_t)((warp & 3) * 32) << 16);
    float acc[G::NOUT];
#pragma unroll
    for (int q = 0; q < G::NOUT; ++q) acc[q] = 0.0f;
    int cur = i0;
    bool aborted = false;
#pragma unroll 1
    for (int it = 0; it < n_tiles; ++it) {
      const int b = it & 1;
      if (abort_s) {
        aborted = true;
        break;
      }
      if (!tc::mbar_wait(bar_full + b, (uint32_t)((it >> 1) & 1))) {
        atomicOr(err, 2);
        abort_s = 1;
        aborted = true;
        break;
      }
      if (abort_s) {  // the producers failed on this tile: its buffers are not valid
        aborted = true;
        break;
      }
      tc::fence_after_sync();
      const int* s_send = idxb + b * 2 * kNT;
      const int* s_recv = s_send + kNT;
      const float* cY = cYb + b * kNT * NZP;
      fwd_tile_ws<L, MODE, 0, kWSFChunk>(s_send, s_recv, cY, taddr0 + (b ? wcol1 : wcol0), h, cur, acc, mW, s,
                                          s_lists[b] + wsid * kNT, s_cnts[b][wsid]);
      tc::fence_before_sync();
      tc::mbar_arrive(bar_done + b);
    }
    if (!aborted) {
      while (cur < i1) {
#pragma unroll
        for (int q = 0; q < G::NOUT; ++q) {
          mW[((size_t)cur * D + G::comp0 + q) * C + c] = s * acc[q];
          acc[q] = 0.0f;
        }
        ++cur;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) tc::mbar_wait(bar_fin, 0, 1LL << 20);  // no product in flight, bounded
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, FL::NCOLS);
}

// ------------------------------------------------------------ tp_fused_bwd
// Adjoint of one layer for one path group.  Per tile of kNT receiver-sorted
// edges: (1) w = W3_p^T z2 recomputed on the tensor cores into tensor memory;
// (2) per edge e = (j <- i) and channel c (paths split between the warp sets):
//       G^{t-1}_j[l1 m1] += s w[p] (-1)^{l2} C Y[l2 m2] Gm_i[l3 m3]        (reverse edge)
//       T_p[m2] = sum C h_i[l1 m1] Gt_j[l3 m3],   Gt = s Gm_j
//       dE/dw_e[p] = sum_m2 Y[l2 m2] T_p[m2]   -> 16-bit operand tile in shared memory
//       dE/dY_e[l2 m2] += sum_c w[p] T_p[m2]   (channel sum: warp butterfly + shared memory)
// (3) dE/dz2[k][e] = sum_{p,c} W3[k][p][c] dE/dw_e[p][c]: a second MMA with A
// read M-major from the same resident W3 image (rows 64..127 of that M = 128
// product are unused), accumulated into dz2[e][k].  Group kernels of one layer
// run one after another on the stream, so G^{t-1}, dY and dz2 are updated
// with plain read-modify-writes; G^{t-1} is kept as two buffers (one per warp
// set), the first group initialising them from G^t.
constexpr bool kMnLboIsK = true;  // descriptor assignment checked by mlip_selftest(2 / 3)

// dE/dw of a tile for the second product: one 16-bit tile (B2H bytes), or with
// SPLIT a hi tile rn16(x) followed by a lo tile rn16(x - hi), so that the
// product carries no rounding of dE/dw (about 22 significant bits with FP16
// operands, 16 with BF16): W3's own 16-bit rounding is then the only one left
// in the per-path weights and their adjoint.
template <int L, int MODE, bool SPLIT>
struct BwdLayoutT {
  using G = Group<L, MODE>;
  static constexpr int NP = G::NP;
  static constexpr bool FIRST = MODE < 0;
  static constexpr int D = NodeDims<L>::D;
  static constexpr int B2H = kNT * NP * 128 * 2;
  static constexpr int B2_BYTES = (SPLIT ? 2 : 1) * B2H;
  static constexpr int NZ = FIRST ? 0 : G::NZ;
  static constexpr int NZP = FIRST ? 4 : G::NZP;
  static constexpr int tmem_cols() {
    int need = (NP + 1) * kNT, c = 32;
    while (c < need) c <<= 1;
    return c;
  }
  static constexpr int NCOLS = tmem_cols();
  static constexpr size_t off_z2 = (size_t)NP * kW3PathBytes;
  static constexpr size_t off_b2 = off_z2 + 2 * kTileBytes;
  static constexpr size_t off_cy = off_b2 + B2_BYTES;
  static constexpr size_t off_y = off_cy + (size_t)kNT * NZP * 4;
  static constexpr size_t off_red = off_y + kNT * 16 * 4;
  // dE/dY partials [4 warps of the owning set][kNT][16]: every edge belongs to one warp set
  static constexpr size_t off_tab = off_red + (size_t)4 * kNT * 16 * 4;
  static constexpr size_t off_taby = off_tab + (size_t)NZP * 4;
  static constexpr size_t off_idx = off_taby + (((size_t)NZP + 15) & ~(size_t)15);
  static constexpr size_t off_bar = off_idx + 2 * kNT * 4;
  static constexpr size_t bytes = off_bar + 64;
  static constexpr bool fits = bytes <= 232448 - 1024;
};


// Pipelined form's buffers (see tp_fused_bwd_ws below).

template <int L, int MODE, bool SPLIT>
struct BwdLayoutWST {
  using G = Group<L, MODE>;
  static constexpr int NP = G::NP;
  static constexpr bool FIRST = MODE < 0;
  static constexpr int B2H = kNT * NP * 128 * 2;
  static constexpr int B2_BYTES = (SPLIT ? 2 : 1) * B2H;
  static constexpr int NZ = FIRST ? 0 : G::NZ;
  static constexpr int NZP = FIRST ? 4 : G::NZP;
  static constexpr int tmem_cols() {
    int need = 2 * (NP + 1) * kNT, c = 32;
    while (c < need) c <<= 1;
    return c;
  }
  static constexpr int NCOLS = tmem_cols();
  static constexpr size_t rest = 2 * kTileBytes + (size_t)2 * kNT * NZP * 4 + 2 * kNT * 16 * 4 + 8 * kNT * 16 * 4 +
                                 (size_t)NZP * 4 + (((size_t)NZP + 15) & ~(size_t)15) + 4 * kNT * 4 + 4 * kNT * 4 + 128;
  static constexpr int NB2 = (size_t)NP * kW3PathBytes + rest + 2 * (size_t)B2_BYTES <= 231424 ? 2 : 1;
  static constexpr size_t off_z2 = (size_t)NP * kW3PathBytes;
  static constexpr size_t off_b2 = off_z2 + 2 * kTileBytes;
  static constexpr size_t off_cy = off_b2 + (size_t)NB2 * B2_BYTES;   // [2][kNT][NZP]
  static constexpr size_t off_y = off_cy + (size_t)2 * kNT * NZP * 4; // [2][kNT][16]
  static constexpr size_t off_red = off_y + 2 * kNT * 16 * 4;         // [2][4 warps of the owning set][kNT][16]
  static constexpr size_t off_tab = off_red + 8 * kNT * 16 * 4;
  static constexpr size_t off_taby = off_tab + (size_t)NZP * 4;
  static constexpr size_t off_idx = off_taby + (((size_t)NZP + 15) & ~(size_t)15);  // [2][send kNT, recv kNT]
  static constexpr size_t off_dws = off_idx + 4 * kNT * 4;                          // [2][scale kNT, inverse kNT]
  static constexpr size_t off_bar = off_dws + 4 * kNT * 4;
  static constexpr size_t bytes = off_bar + 128;
  // groups whose buffers do not fit keep the single-role kernel
  static constexpr bool fits = bytes <= 232448 - 1024 && NCOLS <= 512;
};

// dE/dw is split into hi and lo tiles in every group whose adjoint buffers
// still fit: the single-role kernel's, and the pipelined kernel's where that
// kernel is used (one CTA per SM and its unsplit buffers fit).  At l <= 2 that
// is every group; at l <= 3 the groups of up to four paths.
template <int L, int MODE>
struct DwSplit {
  using N1 = BwdLayoutT<L, MODE, true>;
  static constexpr bool ws_used = ctas_per_sm(N1::bytes) == 1 && BwdLayoutWST<L, MODE, false>::fits;
  static constexpr bool value = N1::fits && (!ws_used || BwdLayoutWST<L, MODE, true>::fits);
};
template <int L, int MODE>
using BwdLayout = BwdLayoutT<L, MODE, DwSplit<L, MODE>::value>;
template <int L, int MODE>
using BwdLayoutWS = BwdLayoutWST<L, MODE, DwSplit<L, MODE>::value>;

template <int L, int MODE, int W>
__device__ __forceinline__ void bwd_edge(const float* wv, int t, const float* hi, const float* Gi, const float* Gt,
                                         const float* Y, const float* cy, float s, float dw_scale, int use_bf16,
                                         uint8_t* sB2, float* Gacc, float* dYp) {
  using G = Group<L, MODE>;
  using S = Split<L, MODE, true>;
  using Tab = CGTable<L>;
  constexpr bool FIRST = MODE < 0;
  constexpr int SBO2 = G::NP * 2048;
  const int c = threadIdx.x & 127;
  static_for<0, G::NP>([&](auto sc) {
    constexpr int sl = decltype(sc)::value;
    if constexpr (S::ws[sl] == W) {
      constexpr int p = G::paths[sl];
      constexpr int l2 = Tab::l2[p], l3 = Tab::l3[p];
      constexpr int kb = Tab::off[p], ke = Tab::off[p + 1], gb = G::eoff[sl];
      const float wp = wv[sl];
      if constexpr (!FIRST) {
        float wg[2 * l3 + 1];
#pragma unroll
        for (int q = 0; q < 2 * l3 + 1; ++q) wg[q] = s * wp * Gi[l3 * l3 + q - G::comp0];
        float c4[(ke - kb + 3) & ~3];
        load4<(ke - kb + 3) / 4>(cy + gb, c4);
        static_for<kb, ke>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          constexpr int i1 = Tab::e1[k], j3 = Tab::e3[k] - l3 * l3;
          Gacc[i1] = fmaf(c4[k - kb], wg[j3], Gacc[i1]);
        });
      }
      float Tp[2 * l2 + 1];
#pragma unroll
      for (int q = 0; q < 2 * l2 + 1; ++q) Tp[q] = 0.0f;
      static_for<kb, ke>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int j2 = Tab::e2[k] - l2 * l2, i1 = Tab::e1[k], o3 = Tab::e3[k] - G::comp0;
        constexpr float cv = Tab::ec[k];
        Tp[j2] = fmaf(cv, hi[i1] * Gt[o3], Tp[j2]);
      });
      float dwp = 0.0f;
#pragma unroll
      for (int q = 0; q < 2 * l2 + 1; ++q) {
        dwp = fmaf(Y[l2 * l2 + q], Tp[q], dwp);
        dYp[l2 * l2 + q] = fmaf(wp, Tp[q], dYp[l2 * l2 + q]);
      }
      const int kidx = sl * 128 + c;
      uint16_t* dst = reinterpret_cast<uint16_t*>(sB2 + (t >> 3) * SBO2 + (kidx >> 3) * 128 + (t & 7) * 16 +
                                                  (kidx & 7) * 2);
      const float x = dwp * dw_scale;
      if constexpr (BwdLayout<L, MODE>::B2_BYTES > BwdLayout<L, MODE>::B2H) {
        // hi and lo by Veltkamp's splitting (multiplier 2^s + 1, s = 24 - the format's significand
        // bits): hi has the format's precision, so it is exact in it, and hi + lo = x exactly; one
        // packed conversion then gives both 16-bit values, the lo tile following the hi tile
        const float t = __fmul_rn(x, use_bf16 ? 65537.0f : 8193.0f);
        const float hi = __fsub_rn(t, __fsub_rn(t, x));
        const uint32_t pk = pack16x2(hi, __fsub_rn(x, hi), use_bf16);
        dst[0] = (uint16_t)(pk & 0xFFFFu);
        dst[BwdLayout<L, MODE>::B2H / 2] = (uint16_t)(pk >> 16);
      } else {
        dst[0] = to16(x, use_bf16);
      }
    }
  });
}

template <int L, int MODE, int W>
__device__ __forceinline__ void bwd_tile_ws(int i0, int i1, const int* s_send, const int* s_recv, const float* sY,
                                            const float* cY, uint32_t taddr0, const float* __restrict__ hprev,
                                            const float* __restrict__ Gm, const float* __restrict__ GinA,
                                            const float* __restrict__ GinB, float* __restrict__ GoutW,
                                            int first_group, int& cur, float* Gacc, float* Gt, float* red,
                                            uint8_t* sB2, float s, const float* dws, int use_bf16, int wsid,
                                            const int* list, int cnt) {
  using G = Group<L, MODE>;
  using S = Split<L, MODE, true>;
  using BL = BwdLayout<L, MODE>;
  constexpr int D = NodeDims<L>::D;
  constexpr int C = 128;
  constexpr bool FIRST = MODE < 0;
  constexpr int DH = S::dh(W);
  constexpr int NG = FIRST ? 1 : G::NOUT;
  constexpr int SBO2 = G::NP * 2048;
  const int c = threadIdx.x & 127, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto flush = [&](int i) {
    if constexpr (!FIRST) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const size_t o = ((size_t)i * D + d) * C + c;
        if (!first_group) atomicAdd(&GoutW[o], Gacc[d]);
        else GoutW[o] = (wsid == 0 ? GinA[o] + GinB[o] : 0.0f) + Gacc[d];
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) Gacc[d] = 0.0f;
  };
  auto enter = [&](int i) {
#pragma unroll
    for (int q = 0; q < G::NOUT; ++q) Gt[q] = s * Gm[((size_t)i * D + G::comp0 + q) * C + c];
  };
  auto advance = [&](int r) {
    while (cur < r) {
      if (cur >= i0) flush(cur);
      ++cur;
      if (cur < i1) enter(cur);
    }
  };
  constexpr int CH = chunk_edges<DH + (FIRST ? 0 : NG)>();
  static_assert(CH % S::ypack(W) == 0, "edge packing must divide the chunk");
  float pv[16];
  // the harmonic component this lane pair reduces (fixed for the thread; -1: none)
  int my_comp = -1;
  {
    constexpr std::array<int, 16> yl = S::ylist(W);
    constexpr int NVP = 16 / S::ypack(W), NV = S::nyv(W);
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (((lane >> 1) % NVP) == k) my_comp = yl[k];
  }
  if (cnt <= 0) return;  // uniform over the warp set
  auto lslot = [&](int i) { return list[i < cnt ? i : cnt - 1]; };
  float hn[CH][DH], gn[CH][NG];
#pragma unroll
  for (int j = 0; j < CH; ++j) {
    const int si = s_send[lslot(j)];
#pragma unroll
    for (int d = 0; d < DH; ++d) hn[j][d] = hprev[((size_t)si * D + d) * C + c];
    if constexpr (!FIRST) {
#pragma unroll
      for (int q = 0; q < NG; ++q) gn[j][q] = Gm[((size_t)si * D + G::comp0 + q) * C + c];
    }
  }
#pragma unroll 1
  for (int base = 0; base < cnt; base += CH) {
    float wvc[G::NP][CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int t = lslot(base + j);
      static_for<0, G::NP>([&](auto sc) {
        constexpr int sl = decltype(sc)::value;
        if constexpr (S::ws[sl] == W) wvc[sl][j] = tmem_ld1(taddr0 + sl * kNT + t);
      });
    }
    tc::tmem_ld_wait();
    float hc[CH][DH], gc[CH][NG];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
#pragma unroll
      for (int d = 0; d < DH; ++d) hc[j][d] = hn[j][d];
#pragma unroll
      for (int q = 0; q < NG; ++q) gc[j][q] = FIRST ? 0.0f : gn[j][q];
    }
    if (base + CH < cnt) {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int si = s_send[lslot(base + CH + j)];
#pragma unroll
        for (int d = 0; d < DH; ++d) hn[j][d] = hprev[((size_t)si * D + d) * C + c];
        if constexpr (!FIRST) {
#pragma unroll
          for (int q = 0; q < NG; ++q) gn[j][q] = Gm[((size_t)si * D + G::comp0 + q) * C + c];
        }
      }
    }
    static_for<0, CH>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      const bool live = base + j < cnt;
      const int t = lslot(base + j);
      const int r = live ? s_recv[t] : -1;
      float dYp[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) dYp[k] = 0.0f;
      if (r >= 0) {
        advance(r);
        float Y[16];
        load4<4>(sY + t * 16, Y);
        float wv[G::NP];
#pragma unroll
        for (int sl = 0; sl < G::NP; ++sl) wv[sl] = wvc[sl][j];
        bwd_edge<L, MODE, W>(wv, t, hc[j], gc[j], Gt, Y, cY + t * BL::NZP, s, dws[t], use_bf16, sB2, Gacc, dYp);
      }
      // channel sums of this edge's dE/dY components, several edges per butterfly
      constexpr int PK = S::ypack(W), NVP = 16 / PK, NV = S::nyv(W);
      constexpr std::array<int, 16> yl = S::ylist(W);
      constexpr int slot = j % PK;
#pragma unroll
      for (int i = 0; i < NVP; ++i) pv[slot * NVP + i] = i < NV ? dYp[yl[i < NV ? i : 0]] : 0.0f;
      if constexpr (slot == PK - 1) {
        const float tot = warp_reduce16(pv);
        const int ie = base + j - (PK - 1) + (lane >> 1) / NVP;  // list entry of this lane pair's value
        if ((lane & 1) == 0 && my_comp >= 0 && ie < cnt) red[((warp & 3) * kNT + list[ie]) * 16 + my_comp] = tot;
      }
    });
  }
}


// Heavy groups: one copy of the per-edge body in a runtime loop over the
// tile's edges, taken in pairs (keeps the hot loop inside the instruction
// cache); the sender rows of an edge are loaded into one of two register
// buffers an edge ahead of their use, after an L1 prefetch a pair ahead.
template <int L, int MODE, int W>
__device__ __forceinline__ void bwd_tile_ws_roll(int i0, int i1, const int* s_send, const int* s_recv,
                                                 const float* sY, const float* cY, uint32_t taddr0,
                                                 const float* __restrict__ hprev, const float* __restrict__ Gm,
                                                 const float* __restrict__ GinA, const float* __restrict__ GinB,
                                                 float* __restrict__ GoutW, int first_group, int& cur, float* Gacc,
                                                 float* Gt, float* red, uint8_t* sB2, float s, const float* dws,
                                                 int use_bf16, int wsid, const int* list, int cnt) {
  using G = Group<L, MODE>;
  using S = Split<L, MODE, true>;
  using BL = BwdLayout<L, MODE>;
  constexpr int D = NodeDims<L>::D;
  constexpr int C = 128;
  constexpr bool FIRST = MODE < 0;
  constexpr int DH = S::dh(W);
  constexpr int NG = FIRST ? 1 : G::NOUT;
  constexpr int SBO2 = G::NP * 2048;
  // dE/dY: the NV components of PK consecutive edges packed into one 32-value
  // channel butterfly (PK = floor(32 / NV); the tile's last group may be short)
  constexpr int NV = S::nyv(W), PK = 32 / NV;
  constexpr std::array<int, 16> yl = S::ylist(W);
  const int c = threadIdx.x & 127, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int yl_rt[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) yl_rt[k] = yl[k];
  auto flush = [&](int i) {
    if constexpr (!FIRST) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const size_t o = ((size_t)i * D + d) * C + c;
        if (!first_group) atomicAdd(&GoutW[o], Gacc[d]);
        else GoutW[o] = (wsid == 0 ? GinA[o] + GinB[o] : 0.0f) + Gacc[d];
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) Gacc[d] = 0.0f;
  };
  auto enter = [&](int i) {
#pragma unroll
    for (int q = 0; q < G::NOUT; ++q) Gt[q] = s * Gm[((size_t)i * D + G::comp0 + q) * C + c];
  };
  auto advance = [&](int r) {
    while (cur < r) {
      if (cur >= i0) flush(cur);
      ++cur;
      if (cur < i1) enter(cur);
    }
  };
  auto gather = [&](int t, float* hv, float* gv) {
    const int si = s_send[t];
#pragma unroll
    for (int d = 0; d < DH; ++d) hv[d] = hprev[((size_t)si * D + d) * C + c];
    if constexpr (!FIRST) {
#pragma unroll
      for (int q = 0; q < NG; ++q) gv[q] = Gm[((size_t)si * D + G::comp0 + q) * C + c];
    }
  };
  float pv[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) pv[i] = 0.0f;
  // list entry i (edge slot t) of this warp set
  auto edge = [&](int i, int t, const float* hc, const float* gc, const float* wv) {
    const int r = s_recv[t];
    float dYp[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) dYp[k] = 0.0f;
    if (r >= 0) {
      advance(r);
      float Y[16];
      load4<4>(sY + t * 16, Y);
      bwd_edge<L, MODE, W>(wv, t, hc, gc, Gt, Y, cY + t * BL::NZP, s, dws[t], use_bf16, sB2, Gacc, dYp);
    }
#pragma unroll
    for (int q = 0; q < NV * (PK - 1); ++q) pv[q] = pv[q + NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) pv[NV * (PK - 1) + q] = dYp[yl[q]];
    const int slot = i % PK;
    if (slot == PK - 1 || i == cnt - 1) {
      const float tot = warp_reduce32(pv);
      // lane v holds the total of value v: list entry i - (PK - 1) + v / NV, component v % NV;
      // entries older than this group's first were written by the previous group
      const int ie = i - (PK - 1) + lane / NV;
      if (lane < PK * NV && ie >= i - slot) red[((warp & 3) * kNT + list[ie]) * 16 + yl_rt[lane % NV]] = tot;
    }
  };
  // list entries in pairs with two register buffers: the sender rows of the
  // next pair's entry load while the other entry of this pair is computed
  if (cnt <= 0) return;  // uniform over the warp set
  auto lslot = [&](int i) { return list[i < cnt ? i : cnt - 1]; };
  float hA[DH], gA[NG], hB[DH], gB[NG];
#pragma unroll
  for (int q = 0; q < NG; ++q) gA[q] = gB[q] = 0.0f;
  gather(lslot(0), hA, gA);
  gather(lslot(1), hB, gB);
#pragma unroll 1
  for (int i = 0; i < cnt; i += 2) {
    const int tA = list[i], tB = lslot(i + 1);
    {  // the next pair's sender rows into L1 (one line per lane: a warp's 32 channels of a
       // component), so that their register loads, issued after this pair's first edge, hit L1
      const int lane = threadIdx.x & 31;
#pragma unroll
      for (int q0 = 0; q0 < 2 * (DH + NG); q0 += 32) {
        const int q = q0 + lane;
        const int e = i + 2 + q / (DH + NG), d = q % (DH + NG);
        if (q < 2 * (DH + NG) && e < cnt && (!FIRST || d < DH)) {
          const int si = s_send[list[e]];
          prefetch_l1((d < DH ? hprev + ((size_t)si * D + d) * C : Gm + ((size_t)si * D + G::comp0 + d - DH) * C) +
                      (c & ~31));
        }
      }
    }
    float wA[G::NP], wB[G::NP];
    static_for<0, G::NP>([&](auto sc) {
      constexpr int sl = decltype(sc)::value;
      if constexpr (S::ws[sl] == W) {
        wA[sl] = tmem_ld1(taddr0 + sl * kNT + tA);
        wB[sl] = tmem_ld1(taddr0 + sl * kNT + tB);
      }
    });
    tc::tmem_ld_wait();
    edge(i, tA, hA, gA, wA);
    if (i + 2 < cnt) gather(list[i + 2], hA, gA);
    if (i + 1 < cnt) {
      edge(i + 1, tB, hB, gB, wB);
      if (i + 3 < cnt) gather(list[i + 3], hB, gB);
    }
  }
}

template <int L, int MODE>
__global__ void __launch_bounds__(kThreads, ctas_per_sm(BwdLayout<L, MODE>::bytes)) tp_fused_bwd(int n, const int* __restrict__ row_ptr,
                                                         const int* __restrict__ recv, const int* __restrict__ send,
                                                         const float* __restrict__ Yg,
                                                         const float* __restrict__ hprev,
                                                         const float* __restrict__ Gm,
                                                         const uint8_t* __restrict__ w3img,
                                                         const uint8_t* __restrict__ z2t, float s,
                                                         const float* __restrict__ GinA, const float* __restrict__ GinB,
                                                         float* __restrict__ GoutA, float* __restrict__ GoutB,
                                                         int first_group, float* __restrict__ dY,
                                                         float* __restrict__ dz2, int use_bf16,
                                                         const int* __restrict__ sys_of,
                                                         const float2* __restrict__ dws2,
                                                         const uint8_t* __restrict__ epar, int* __restrict__ err) {
  using G = Group<L, MODE>;
  using BL = BwdLayout<L, MODE>;
  static_assert(BL::fits, "shared memory of the adjoint kernel exceeds the per-block limit");
  constexpr int D = NodeDims<L>::D;
  constexpr int NP = G::NP;
  constexpr bool FIRST = BL::FIRST;
  constexpr int SBO2 = NP * 2048;  // B' operand: K' = NP * 128 channels
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sW3 = smem;
  uint8_t* sZ2 = smem + BL::off_z2;
  uint8_t* sB2 = smem + BL::off_b2;
  float* cY = reinterpret_cast<float*>(smem + BL::off_cy);
  float* sY = reinterpret_cast<float*>(smem + BL::off_y);
  float* red = reinterpret_cast<float*>(smem + BL::off_red);  // [4][kNT][16]
  float* tab_c = reinterpret_cast<float*>(smem + BL::off_tab);
  uint8_t* tab_y = smem + BL::off_taby;
  int* s_send = reinterpret_cast<int*>(smem + BL::off_idx);
  int* s_recv = s_send + kNT;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BL::off_bar);
  uint64_t* bar_w3 = bars;
  uint64_t* bar_z2 = bars + 1;  // [2]
  uint64_t* bar_mma = bars + 3;
  uint64_t* bar_mma2 = bars + 4;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 5);
  __shared__ int abort_s;
  __shared__ float s_dws[2 * kNT];  // per-edge scale of dE/dw in the second product, and its inverse
  __shared__ int s_list[2 * kNT], s_cnt[2], s_own[kNT];  // the warp sets' edges of the tile

  const int tid = threadIdx.x, warp = tid >> 5, wsid = warp >> 2, c = tid & 127;
  float* GoutW = wsid == 0 ? GoutA : GoutB;
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, BL::NCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(bar_w3, 1);
    tc::mbar_init(bar_z2, 1);
    tc::mbar_init(bar_z2 + 1, 1);
    tc::mbar_init(bar_mma, 1);
    tc::mbar_init(bar_mma2, 1);
    tc::fence_mbar_init();
    abort_s = 0;
  }
  if constexpr (!FIRST) load_group_table<L, MODE, true>(tab_c, tab_y);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tmem_holder;
  const uint32_t taddr0 = tbase + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t dcol = NP * kNT;  // columns of dE/dz2 in tensor memory

  int i0, i1;
  block_receivers(row_ptr, n, blockIdx.x, gridDim.x, &i0, &i1);
  const int E0 = row_ptr[i0], E1 = row_ptr[i1];
  const int t_begin = E0 / kNT, t_end = (E1 > E0) ? (E1 + kNT - 1) / kNT : t_begin;
  const int n_tiles = t_end - t_begin;

  int z2_issued[2] = {0, 0}, z2_waited[2] = {0, 0};
  bool w3_issued = false;
  if (tid == 0 && n_tiles > 0) {
    tc::mbar_arrive_expect_tx(bar_w3, NP * kW3PathBytes);
#pragma unroll 1
    for (int sl = 0; sl < NP; ++sl)
      tc::bulk_g2s(sW3 + sl * kW3PathBytes, w3img + (size_t)sl * kW3PathBytes, kW3PathBytes, bar_w3);
    w3_issued = true;
    tc::mbar_arrive_expect_tx(bar_z2, kTileBytes);
    tc::bulk_g2s(sZ2, z2t + (size_t)t_begin * kTileBytes, kTileBytes, bar_z2);
    z2_issued[0] = 1;
  }

  float Gacc[D], Gt[G::NOUT];
#pragma unroll
  for (int d = 0; d < D; ++d) Gacc[d] = 0.0f;
#pragma unroll
  for (int q = 0; q < G::NOUT; ++q) Gt[q] = 0.0f;
  int cur = i0 - 1;
  const uint32_t idesc1 = tc::idesc_16bit(128, kNT, use_bf16 != 0);
  const uint32_t idesc2 = idesc1 | (1u << 15);  // A M-major

#pragma unroll 1
  for (int it = 0; it < n_tiles; ++it) {
    const int tile = t_begin + it;
    const int buf = it & 1;
    if (tid == 0) {
      bool ok = true;
      if (it + 1 < n_tiles) {
        const int nb = buf ^ 1;
        tc::mbar_arrive_expect_tx(bar_z2 + nb, kTileBytes);
        tc::bulk_g2s(sZ2 + nb * kTileBytes, z2t + (size_t)(tile + 1) * kTileBytes, kTileBytes, bar_z2 + nb);
        z2_issued[nb]++;
      }
      if (it == 0) ok = ok && tc::mbar_wait(bar_w3, 0);
      ok = ok && tc::mbar_wait(bar_z2 + buf, (uint32_t)(z2_waited[buf] & 1));
      if (ok) {
        z2_waited[buf]++;
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(sW3), b0 = tc::smem_u32(sZ2 + buf * kTileBytes);
#pragma unroll 1
        for (int sl = 0; sl < NP; ++sl)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = tc::desc_noswizzle(a0 + sl * kW3PathBytes + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
            const uint64_t bd = tc::desc_noswizzle(b0 + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
            tc::mma_bf16(tbase + sl * kNT, ad, bd, idesc1, kk > 0 ? 1u : 0u);
          }
        tc::mma_commit(bar_mma);
      } else {
        atomicOr(err, 4);
        abort_s = 1;
      }
    }
    tile_setup<BL::NZ, BL::NZP>(tile, E0, E1, recv, send, Yg, s_recv, s_send, sY, cY, tab_c, tab_y, epar, s_list,
                                s_cnt, s_own, sys_of, dws2, s_dws);
    __syncthreads();
    if (abort_s) break;
    if (!tc::mbar_wait(bar_mma, (uint32_t)(it & 1))) {
      atomicOr(err, 8);
      abort_s = 1;
    }
    tc::fence_after_sync();
    {
      using S = Split<L, MODE, true>;
      constexpr bool heavy0 = S::dh(0) + (FIRST ? 0 : G::NOUT) > 8, heavy1 = S::dh(1) + (FIRST ? 0 : G::NOUT) > 8;
      const int* lst = s_list + wsid * kNT;
      const int cnt = s_cnt[wsid];
      if constexpr (heavy0)
        bwd_tile_ws_roll<L, MODE, 0>(i0, i1, s_send, s_recv, sY, cY, taddr0, hprev, Gm, GinA, GinB, GoutW,
                                       first_group, cur, Gacc, Gt, red, sB2, s, s_dws, use_bf16, wsid, lst, cnt);
      else
        bwd_tile_ws<L, MODE, 0>(i0, i1, s_send, s_recv, sY, cY, taddr0, hprev, Gm, GinA, GinB, GoutW, first_group,
                                  cur, Gacc, Gt, red, sB2, s, s_dws, use_bf16, wsid, lst, cnt);
    }
    // second product: dE/dz2 = W3 dE/dw over this tile
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sW3), b0 = tc::smem_u32(sB2);
      const uint32_t kstride = 1024, mstride = 128;
      const uint32_t lbo = kMnLboIsK ? kstride : mstride, sbo = kMnLboIsK ? mstride : kstride;
      constexpr int NH = BL::B2_BYTES / BL::B2H;  // dE/dw tiles: hi, and lo when split
#pragma unroll 1
      for (int q = 0; q < NH * NP; ++q) {
        const int sl = q % NP, half = q / NP;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const uint64_t ad = tc::desc_noswizzle(a0 + sl * kW3PathBytes + kk * 2 * kstride, lbo, sbo);
          const uint64_t bd = tc::desc_noswizzle(b0 + half * BL::B2H + sl * 2048 + kk * 256, 128, SBO2);
          tc::mma_bf16(tbase + dcol, ad, bd, idesc2, (q | kk) ? 1u : 0u);
        }
      }
      tc::mma_commit(bar_mma2);
    }
    // channel sums of dE/dY while the product runs
    {
      using S = Split<L, MODE, true>;
      constexpr int m0 = S::ymask(0), m1 = S::ymask(1);
      for (int q = tid; q < kNT * 16; q += blockDim.x) {
        const int t = q >> 4, k = q & 15;
        const int e = tile * kNT + t;
        if (e >= E0 && e < E1 && ((m0 | m1) >> k & 1)) {
          float v = 0.0f;  // the four warps of the set that owns edge t
#pragma unroll
          for (int w = 0; w < 4; ++w) v += red[(w * kNT + t) * 16 + k];
          atomicAdd(&dY[(size_t)e * 16 + k], v);  // one add per kernel and address: deterministic
        }
      }
    }
    if (!tc::mbar_wait(bar_mma2, (uint32_t)(it & 1))) {
      atomicOr(err, 16);
      abort_s = 1;
    }
    tc::fence_after_sync();
    if (warp < 2) {  // lanes 0..63 hold hidden units k = 0..63
#pragma unroll 1
      for (int ch = 0; ch < kNT / 8; ++ch) {
        float v[8];
        tc::tmem_ld8(taddr0 + dcol + ch * 8, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int e = tile * kNT + ch * 8 + j;
          if (e >= E0 && e < E1) {
            const float x = v[j] * s_dws[kNT + ch * 8 + j];
            if (first_group) dz2[(size_t)e * 64 + tid] = x;  // the layer's first group initialises dE/dz2
            else atomicAdd(&dz2[(size_t)e * 64 + tid], x);
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (abort_s) break;
  }
  if (!abort_s) {
    // remaining receivers of the range
    while (cur < i1) {
      if (cur >= i0 && !FIRST) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const size_t o = ((size_t)cur * D + d) * 128 + c;
          if (!first_group) atomicAdd(&GoutW[o], Gacc[d]);
          else GoutW[o] = (wsid == 0 ? GinA[o] + GinB[o] : 0.0f) + Gacc[d];
        }
      }
#pragma unroll
      for (int d = 0; d < D; ++d) Gacc[d] = 0.0f;
      ++cur;
    }
  }
  if (tid == 0) {
    if (w3_issued && n_tiles > 0) tc::mbar_wait(bar_w3, 0, 1LL << 20);
    for (int b = 0; b < 2; ++b)
      while (z2_waited[b] < z2_issued[b]) {
        if (!tc::mbar_wait(bar_z2 + b, (uint32_t)(z2_waited[b] & 1), 1LL << 20)) break;
        z2_waited[b]++;
      }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, BL::NCOLS);
}


// ------------------------------------------------- tp_fused_bwd, pipelined
// Groups that hold one CTA per SM run a warp-specialised form of the same
// adjoint: warps 0..7 (two warp sets) do only the per-edge work; warps 8 and
// 9 prepare each tile one ahead (receiver/sender ids, harmonics, per-system
// scales, c*Y products, the first product w = W3^T z2 into one of two
// tensor-memory buffers) and finish it one behind (the second product
// dE/dz2 = W3 dE/dw, the channel sums of dE/dY, and dE/dz2 read back from
// tensor-memory lanes 0..63, which warps 8 and 9 can read).  Tile buffers
// alternate by tile parity b; mbarriers order the roles:
//   full[b]   64 producer arrivals + the first product's commit
//   done[b]   256 consumer arrivals: the tile's dE/dw and dE/dY partials are written
//   mma2[b]   the second product's commit
// The producer prepares tile it + 1 before it finishes tile it, and prepares a
// buffer only after finishing the tile that last used it.  Long waits of the
// producers sleep between polls so that they leave the issue slots to the
// consumers.


template <int L, int MODE>
__global__ void __launch_bounds__(kWSThreads, 1)
    tp_fused_bwd_ws(int n, const int* __restrict__ row_ptr, const int* __restrict__ recv,
                    const int* __restrict__ send, const float* __restrict__ Yg, const float* __restrict__ hprev,
                    const float* __restrict__ Gm, const uint8_t* __restrict__ w3img, const uint8_t* __restrict__ z2t,
                    float s, const float* __restrict__ GinA, const float* __restrict__ GinB,
                    float* __restrict__ GoutA, float* __restrict__ GoutB, int first_group, float* __restrict__ dY,
                    float* __restrict__ dz2, int use_bf16, const int* __restrict__ sys_of,
                    const float2* __restrict__ dws2, const uint8_t* __restrict__ epar, int* __restrict__ err) {
  using G = Group<L, MODE>;
  using BL = BwdLayoutWS<L, MODE>;
  static_assert(BL::fits, "shared or tensor memory of the pipelined adjoint kernel exceeds the per-SM limits");
  constexpr int D = NodeDims<L>::D;
  constexpr int NP = G::NP;
  constexpr bool FIRST = BL::FIRST;
  constexpr int NZ = BL::NZ, NZP = BL::NZP;
  constexpr int SBO2 = NP * 2048;  // B' operand: K' = NP * 128 channels
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sW3 = smem;
  uint8_t* sZ2 = smem + BL::off_z2;
  uint8_t* sB2base = smem + BL::off_b2;
  float* cYb = reinterpret_cast<float*>(smem + BL::off_cy);
  float* sYb = reinterpret_cast<float*>(smem + BL::off_y);
  float* redb = reinterpret_cast<float*>(smem + BL::off_red);
  float* tab_c = reinterpret_cast<float*>(smem + BL::off_tab);
  uint8_t* tab_y = smem + BL::off_taby;
  int* idxb = reinterpret_cast<int*>(smem + BL::off_idx);
  float* dwsb = reinterpret_cast<float*>(smem + BL::off_dws);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BL::off_bar);
  uint64_t* bar_w3 = bars;
  uint64_t* bar_z2 = bars + 1;    // [2]
  uint64_t* bar_full = bars + 3;  // [2]
  uint64_t* bar_mma2 = bars + 5;  // [2]
  uint64_t* bar_done = bars + 7;  // [2]
  uint64_t* bar_fin = bars + 9;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 10);
  __shared__ volatile int abort_s;
  __shared__ int abort_p;  // producers' copy, written by the elected producer before their barrier
  __shared__ int s_lists[2][2 * kNT], s_cnts[2][2], s_owns[2][kNT];  // the warp sets' edges, per buffer

  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, BL::NCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(bar_w3, 1);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(bar_z2 + b, 1);
      tc::mbar_init(bar_full + b, kWSProducers + 1);
      tc::mbar_init(bar_mma2 + b, 1);
      tc::mbar_init(bar_done + b, kWSConsumers);
    }
    tc::mbar_init(bar_fin, 1);
    tc::fence_mbar_init();
    abort_s = 0;
    abort_p = 0;
  }
  if constexpr (!FIRST) load_group_table<L, MODE, true>(tab_c, tab_y);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tmem_holder;
  const uint32_t wcol0 = 0, wcol1 = NP * kNT, dcol0 = 2 * NP * kNT, dcol1 = 2 * NP * kNT + kNT;

  int i0, i1;
  block_receivers(row_ptr, n, blockIdx.x, gridDim.x, &i0, &i1);
  const int E0 = row_ptr[i0], E1 = row_ptr[i1];
  const int t_begin = E0 / kNT, t_end = (E1 > E0) ? (E1 + kNT - 1) / kNT : t_begin;
  const int n_tiles = t_end - t_begin;
  const uint32_t idesc1 = tc::idesc_16bit(128, kNT, use_bf16 != 0);
  const uint32_t idesc2 = idesc1 | (1u << 15);  // A M-major

  if (warp >= 8) {
    // ---------------------------------------------------------- producers
    const int pt = tid - kWSConsumers;  // 0..63
    const bool elect = pt == 0;
    int z2_issued[2] = {0, 0}, z2_waited[2] = {0, 0};
    bool w3_waited = false;
    if (elect && n_tiles > 0) {
      tc::mbar_arrive_expect_tx(bar_w3, NP * kW3PathBytes);
#pragma unroll 1
      for (int sl = 0; sl < NP; ++sl)
        tc::bulk_g2s(sW3 + sl * kW3PathBytes, w3img + (size_t)sl * kW3PathBytes, kW3PathBytes, bar_w3);
    }
    // tile it into buffer b = it & 1
    auto setup = [&](int it) {
      const int b = it & 1, tile = t_begin + it;
      int* s_send = idxb + b * 2 * kNT;
      int* s_recv = s_send + kNT;
      float* s_dws = dwsb + b * 2 * kNT;
      float* sY = sYb + b * kNT * 16;
      float* cY = cYb + b * kNT * NZP;
      if (elect) {
        tc::mbar_arrive_expect_tx(bar_z2 + b, kTileBytes);
        tc::bulk_g2s(sZ2 + b * kTileBytes, z2t + (size_t)tile * kTileBytes, kTileBytes, bar_z2 + b);
        z2_issued[b]++;
      }
      if (pt < kNT) {  // one warp: lane = edge slot
        const int e = tile * kNT + pt;
        const bool valid = e >= E0 && e < E1;
        const int r = valid ? recv[e] : -1;
        const int par = valid ? epar[e] : 0;
        s_recv[pt] = r;
        s_send[pt] = valid ? send[e] : 0;
        s_owns[b][pt] = valid ? par : -1;
        build_lists(pt, valid, par, s_lists[b], s_cnts[b]);
        const float2 v = valid ? dws2[sys_of ? sys_of[r] : 0] : make_float2(1.0f, 1.0f);
        s_dws[pt] = v.x;
        s_dws[kNT + pt] = v.y;
      }
      for (int q = pt; q < kNT * 4; q += kWSProducers) {
        const int t = q >> 2, e = tile * kNT + t;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e >= E0 && e < E1) v = reinterpret_cast<const float4*>(Yg)[(size_t)e * 4 + (q & 3)];
        reinterpret_cast<float4*>(sY)[q] = v;
      }
      tc::named_bar(1, kWSProducers);
      if constexpr (NZ > 0) {
        for (int q = pt; q < kNT * NZ; q += kWSProducers) {
          const int t = q / NZ, k = q - t * NZ;
          cY[t * NZP + k] = tab_c[k] * sY[t * 16 + tab_y[k]];
        }
      }
      if (elect) {
        bool ok = true;
        if (!w3_waited) ok = w3_waited = tc::mbar_wait(bar_w3, 0);
        ok = ok && tc::mbar_wait(bar_z2 + b, (uint32_t)(z2_waited[b] & 1));
        if (ok) {
          z2_waited[b]++;
          tc::fence_after_sync();
          const uint32_t a0 = tc::smem_u32(sW3), b0 = tc::smem_u32(sZ2 + b * kTileBytes);
          const uint32_t wcol = b ? wcol1 : wcol0;
#pragma unroll 1
          for (int sl = 0; sl < NP; ++sl)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = tc::desc_noswizzle(a0 + sl * kW3PathBytes + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
              const uint64_t bd = tc::desc_noswizzle(b0 + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
              tc::mma_bf16(tbase + wcol + sl * kNT, ad, bd, idesc1, kk > 0 ? 1u : 0u);
            }
          tc::mma_commit(bar_full + b);
        } else {
          atomicOr(err, 4);
          abort_s = 1;
          tc::mbar_arrive(bar_full + b);  // completes the phase so the consumers see the abort
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(bar_full + b);
    };
    // tile it after the consumers: the second product, the channel sums of
    // dE/dY, and dE/dz2 read back (lanes 0..63 = hidden units).  A failed wait
    // only raises the abort; the warp-collective tensor-memory loads still run
    // on every lane, and the loop stops at the next uniform check.
    auto drain = [&](int it) {
      const int b = it & 1, tile = t_begin + it;
      const float* s_dws = dwsb + b * 2 * kNT;
      const float* red = redb + b * 4 * kNT * 16;
      const uint32_t dcol = b ? dcol1 : dcol0;
      if (!tc::mbar_wait_sleep(bar_done + b, (uint32_t)((it >> 1) & 1))) {
        atomicOr(err, 8);
        abort_s = 1;
      }
      tc::fence_after_sync();
      if (elect) {
        const uint8_t* sB2 = sB2base + (BL::NB2 == 2 ? b : 0) * BL::B2_BYTES;
        const uint32_t a0 = tc::smem_u32(sW3), b0 = tc::smem_u32(sB2);
        const uint32_t kstride = 1024, mstride = 128;
        const uint32_t lbo = kMnLboIsK ? kstride : mstride, sbo = kMnLboIsK ? mstride : kstride;
        constexpr int NH = BL::B2_BYTES / BL::B2H;  // dE/dw tiles: hi, and lo when split
#pragma unroll 1
        for (int q = 0; q < NH * NP; ++q) {
          const int sl = q % NP, half = q / NP;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const uint64_t ad = tc::desc_noswizzle(a0 + sl * kW3PathBytes + kk * 2 * kstride, lbo, sbo);
            const uint64_t bd = tc::desc_noswizzle(b0 + half * BL::B2H + sl * 2048 + kk * 256, 128, SBO2);
            tc::mma_bf16(tbase + dcol, ad, bd, idesc2, (q | kk) ? 1u : 0u);
          }
        }
        tc::mma_commit(bar_mma2 + b);
      }
      {  // channel sums of dE/dY while the product runs
        using S = Split<L, MODE, true>;
        constexpr int m0 = S::ymask(0), m1 = S::ymask(1);
        for (int q = pt; q < kNT * 16; q += kWSProducers) {
          const int t = q >> 4, k = q & 15;
          const int e = tile * kNT + t;
          if (e >= E0 && e < E1 && ((m0 | m1) >> k & 1)) {
            float v = 0.0f;  // the four warps of the set that owns edge t
#pragma unroll
            for (int w = 0; w < 4; ++w) v += red[(w * kNT + t) * 16 + k];
            atomicAdd(&dY[(size_t)e * 16 + k], v);  // one add per kernel and address: deterministic
          }
        }
      }
      if (!tc::mbar_wait_sleep(bar_mma2 + b, (uint32_t)((it >> 1) & 1))) {
        atomicOr(err, 16);
        abort_s = 1;
      }
      tc::fence_after_sync();
      const uint32_t taddr = tbase + ((uint32_t)((warp & 3) * 32) << 16) + dcol;
#pragma unroll 1
      for (int ch = 0; ch < kNT / 8; ++ch) {
        float v[8];
        tc::tmem_ld8(taddr + ch * 8, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int e = tile * kNT + ch * 8 + j;
          if (e >= E0 && e < E1) {
            const float x = v[j] * s_dws[kNT + ch * 8 + j];
            if (first_group) dz2[(size_t)e * 64 + pt] = x;  // the layer's first group initialises dE/dz2
            else atomicAdd(&dz2[(size_t)e * 64 + pt], x);
          }
        }
      }
      tc::fence_before_sync();
    };
    // the same decision for all producer threads (named barriers must not diverge)
    auto stop = [&]() -> bool {
      if (elect) abort_p = abort_s;
      tc::named_bar(1, kWSProducers);
      const bool st = abort_p != 0;
      tc::named_bar(1, kWSProducers);
      return st;
    };
    if (n_tiles > 0) setup(0);
#pragma unroll 1
    for (int it = 0; it < n_tiles; ++it) {
      if (stop()) break;
      if (it + 1 < n_tiles) setup(it + 1);  // its buffer was drained at it - 1
      drain(it);
    }
    if (elect) {
      for (int b = 0; b < 2; ++b)
        while (z2_waited[b] < z2_issued[b]) {
          if (!tc::mbar_wait(bar_z2 + b, (uint32_t)(z2_waited[b] & 1), 1LL << 20)) break;
          z2_waited[b]++;
        }
      if (n_tiles > 0 && !w3_waited) tc::mbar_wait(bar_w3, 0, 1LL << 20);
      tc::mma_commit(bar_fin);  // every product issued by this thread
    }
  } else {
    // ---------------------------------------------------------- consumers
    using S = Split<L, MODE, true>;
    // the first layer's group (one sender component, every output order) also takes the rolled
    // per-edge loop: its unrolled 8-edge chunks overflow the instruction cache
    constexpr bool heavy0 = FIRST || S::dh(0) + (FIRST ? 0 : G::NOUT) > 8, heavy1 = S::dh(1) + (FIRST ? 0 : G::NOUT) > 8;
    const int wsid = warp >> 2, c = tid & 127;
    float* GoutW = wsid == 0 ? GoutA : GoutB;
    const uint32_t taddr0 = tbase + ((uint32_t)((warp & 3) * 32) << 16);
    float Gacc[D], Gt[G::NOUT];
#pragma unroll
    for (int d = 0; d < D; ++d) Gacc[d] = 0.0f;
#pragma unroll
    for (int q = 0; q < G::NOUT; ++q) Gt[q] = 0.0f;
    int cur = i0 - 1;
    bool aborted = false;
#pragma unroll 1
    for (int it = 0; it < n_tiles; ++it) {
      const int b = it & 1;
      if (abort_s) {
        aborted = true;
        break;
      }
      if (!tc::mbar_wait(bar_full + b, (uint32_t)((it >> 1) & 1))) {
        atomicOr(err, 8);
        abort_s = 1;
        aborted = true;
        break;
      }
      if constexpr (BL::NB2 == 1) {  // one dE/dw tile: the previous second product must have read it
        if (it > 0 && !tc::mbar_wait(bar_mma2 + ((it - 1) & 1), (uint32_t)(((it - 1) >> 1) & 1))) {
          atomicOr(err, 16);
          abort_s = 1;
          aborted = true;
          break;
        }
      }
      tc::fence_after_sync();
      const int* s_send = idxb + b * 2 * kNT;
      const int* s_recv = s_send + kNT;
      const float* sY = sYb + b * kNT * 16;
      const float* cY = cYb + b * kNT * NZP;
      const float* s_dws = dwsb + b * 2 * kNT;
      float* red = redb + b * 4 * kNT * 16;
      uint8_t* sB2 = sB2base + (BL::NB2 == 2 ? b : 0) * BL::B2_BYTES;
      const uint32_t tw = taddr0 + (b ? wcol1 : wcol0);
      const int* lst = s_lists[b] + wsid * kNT;
      const int cnt = s_cnts[b][wsid];
      if constexpr (heavy0)
        bwd_tile_ws_roll<L, MODE, 0>(i0, i1, s_send, s_recv, sY, cY, tw, hprev, Gm, GinA, GinB, GoutW, first_group,
                                       cur, Gacc, Gt, red, sB2, s, s_dws, use_bf16, wsid, lst, cnt);
      else
        bwd_tile_ws<L, MODE, 0>(i0, i1, s_send, s_recv, sY, cY, tw, hprev, Gm, GinA, GinB, GoutW, first_group, cur,
                                  Gacc, Gt, red, sB2, s, s_dws, use_bf16, wsid, lst, cnt);
      // dE/dw (for the second product) and the dE/dY partials are written
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      tc::mbar_arrive(bar_done + b);
    }
    if (!aborted) {
      // remaining receivers of the range
      while (cur < i1) {
        if (cur >= i0 && !FIRST) {
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const size_t o = ((size_t)cur * D + d) * 128 + c;
            if (!first_group) atomicAdd(&GoutW[o], Gacc[d]);
            else GoutW[o] = (wsid == 0 ? GinA[o] + GinB[o] : 0.0f) + Gacc[d];
          }
        }
#pragma unroll
        for (int d = 0; d < D; ++d) Gacc[d] = 0.0f;
        ++cur;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) tc::mbar_wait(bar_fin, 0, 1LL << 20);  // no product in flight, bounded
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, BL::NCOLS);
}

// Per-system scale of dE/dw in the adjoint's second product (FP16 operands)
// and its inverse: |dE/dw| <= 17 max|h| s max|Gm| (orthonormal CG rows,
// |Y| <= 1), so the power of two 2^floor(log2(2^14 / (32 max|h| s max|Gm|)))
// keeps the scaled values below 2^14.  BF16 operands: no scale.
__global__ void dw_scales(int nsys, const float* __restrict__ absmax, float s, int use_bf16,
                          float2* __restrict__ dws2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nsys) return;
  float sc = 1.0f;
  if (!use_bf16) {
    const float U = 32.0f * absmax[2 * q] * s * absmax[2 * q + 1];
    sc = U > 0.0f ? exp2f(fminf(fmaxf(floorf(log2f(16384.0f / U)), -60.0f), 60.0f)) : 1.0f;
  }
  dws2[q] = make_float2(sc, 1.0f / sc);  // powers of two: the inverse is exact
}

// ------------------------------------------------------------- self test
// One M = 128, N = 32, K = 64 tile: D = A B^T with the canonical layouts.
__global__ void umma_selftest(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ D,
                              int* __restrict__ err) {
  __shared__ __align__(1024) uint8_t sA[128 * 64 * 2];
  __shared__ __align__(1024) uint8_t sB[32 * 64 * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t holder;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int idx = tid; idx < 128 * 64; idx += blockDim.x)
    *reinterpret_cast<__nv_bfloat16*>(sA + tc::canon_off(idx / 64, idx % 64)) = __float2bfloat16_rn(A[idx]);
  for (int idx = tid; idx < 32 * 64; idx += blockDim.x)
    *reinterpret_cast<__nv_bfloat16*>(sB + tc::canon_off(idx / 64, idx % 64)) = __float2bfloat16_rn(B[idx]);
  tc::fence_proxy_async_smem();
  if (warp == 0) {
    tc::tmem_alloc(&holder, 32);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = holder;
  if (tid == 0) {
    for (int kk = 0; kk < 4; ++kk) {
      const uint64_t ad = tc::desc_noswizzle(tc::smem_u32(sA) + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
      const uint64_t bd = tc::desc_noswizzle(tc::smem_u32(sB) + kk * 256, tc::kCanonLBO, tc::kCanonSBO);
      tc::mma_bf16(tbase, ad, bd, tc::idesc_bf16(128, 32), kk > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
  }
  const bool ok = tc::mbar_wait(&bar, 0);
  if (!ok && tid == 0) atomicOr(err, 1);
  tc::fence_after_sync();
  if (ok) {
    for (int col = 0; col < 32; col += 8) {
      float v[8];
      tc::tmem_ld8(tbase + ((uint32_t)(warp * 32) << 16) + col, v);
      tc::tmem_ld_wait();
      for (int j = 0; j < 8; ++j) D[tid * 32 + col + j] = v[j];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 32);
}

// MN-major A operand check for the adjoint GEMM: A' = W^T read from the
// forward K-major image of W [128 rows (c)][64 (k)]: A'[k][c] (64 valid rows of
// an M = 128 MMA), B = X [32][128] K-major (K = 128 channels).  `variant`
// selects which descriptor offset is the K-direction stride.
__global__ void umma_selftest_mn(const float* __restrict__ W, const float* __restrict__ X, float* __restrict__ D,
                                 int variant, int* __restrict__ err) {
  __shared__ __align__(1024) uint8_t sA[32768];
  __shared__ __align__(1024) uint8_t sB[32 * 128 * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t holder;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int idx = tid; idx < 32768 / 4; idx += blockDim.x) reinterpret_cast<uint32_t*>(sA)[idx] = 0u;
  __syncthreads();
  for (int idx = tid; idx < 128 * 64; idx += blockDim.x)  // W[c][k] at canon_off(c, k)
    *reinterpret_cast<__nv_bfloat16*>(sA + tc::canon_off(idx / 64, idx % 64)) = __float2bfloat16_rn(W[idx]);
  for (int idx = tid; idx < 32 * 128; idx += blockDim.x) {  // X[e][c], K = 128
    const int e = idx / 128, c = idx % 128;
    *reinterpret_cast<__nv_bfloat16*>(sB + (e >> 3) * 2048 + (c >> 3) * 128 + (e & 7) * 16 + (c & 7) * 2) =
        __float2bfloat16_rn(X[idx]);
  }
  tc::fence_proxy_async_smem();
  if (warp == 0) {
    tc::tmem_alloc(&holder, 32);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = holder;
  if (tid == 0) {
    const uint32_t kstride = 1024, mstride = 128;  // along K' (channel groups) and M' (hidden groups)
    const uint32_t lbo = variant == 0 ? kstride : mstride, sbo = variant == 0 ? mstride : kstride;
    const uint32_t idesc = tc::idesc_bf16(128, 32) | (1u << 15);  // A MN-major
    for (int kk = 0; kk < 8; ++kk) {
      const uint64_t ad = tc::desc_noswizzle(tc::smem_u32(sA) + kk * 2 * kstride, lbo, sbo);
      const uint64_t bd = tc::desc_noswizzle(tc::smem_u32(sB) + kk * 256, 128, 2048);
      tc::mma_bf16(tbase, ad, bd, idesc, kk > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
  }
  const bool ok = tc::mbar_wait(&bar, 0);
  if (!ok && tid == 0) atomicOr(err, 1);
  tc::fence_after_sync();
  if (ok) {
    for (int col = 0; col < 32; col += 8) {
      float v[8];
      tc::tmem_ld8(tbase + ((uint32_t)(warp * 32) << 16) + col, v);
      tc::tmem_ld_wait();
      for (int j = 0; j < 8; ++j) D[tid * 32 + col + j] = v[j];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 32);
}

// CTAs of a fused kernel resident per SM: limited by registers (64K per SM),
// shared memory (228 KB per SM, 1 KB reserved per CTA) and tensor memory (512
// columns per SM); at most 2.
template <class K>
int resident_ctas(K kernel, size_t smem, int ncols) {
  cudaFuncAttributes fa{};
  int regs = 255;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) regs = fa.numRegs;
  else cudaGetLastError();
  const int by_regs = 65536 / std::max(1, ((regs + 7) & ~7) * kThreads);
  const int by_smem = (int)((228 * 1024) / (smem + 1024 + fa.sharedSizeBytes));
  return std::max(1, std::min({by_regs, by_smem, 512 / ncols, 2}));
}

template <int L, int MODE>
int launch_group(int n, const int* row_ptr, const int* recv, const int* send, const float* Yg, const float* h,
                 const uint8_t* w3img, const uint8_t* z2t, float s, float* mA, float* mB, int use_bf16,
                 const uint8_t* epar, int* err, int blocks, cudaStream_t st) {  // blocks: SM count
  if constexpr (ctas_per_sm(FwdLayout<L, MODE>::bytes) == 1 && FwdLayoutWS<L, MODE>::fits) {  // pipelined
    const size_t smem = FwdLayoutWS<L, MODE>::bytes;
    MLIP_CUDA_TRY(cudaFuncSetAttribute(tp_fused_ws<L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    blocks = std::min(n, blocks);
    {
      MLIP_PROF("tp_fused", st);
      tp_fused_ws<L, MODE><<<blocks, kWSThreads, smem, st>>>(n, row_ptr, recv, send, Yg, h, w3img, z2t, s, mA, mB,
                                                            use_bf16, epar, err);
    }
  } else {
    const size_t smem = FwdLayout<L, MODE>::bytes;
    MLIP_CUDA_TRY(cudaFuncSetAttribute(tp_fused<L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    blocks = std::min(n, blocks * resident_ctas(tp_fused<L, MODE>, smem, Group<L, MODE>::NCOLS));
    {
      MLIP_PROF("tp_fused", st);
      tp_fused<L, MODE><<<blocks, kThreads, smem, st>>>(n, row_ptr, recv, send, Yg, h, w3img, z2t, s, mA, mB,
                                                        use_bf16, epar, err);
    }
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

template <int L, int MODE>
int launch_group_bwd(int n, const int* row_ptr, const int* recv, const int* send, const float* Yg,
                     const float* hprev, const float* Gm, const uint8_t* w3img, const uint8_t* z2t, float s,
                     const float* GinA, const float* GinB, float* GoutA, float* GoutB, int first_group, float* dY,
                     float* dz2, int use_bf16, const int* sys_of, const float2* dws2, const uint8_t* epar,
                     int* err, int blocks, cudaStream_t st) {
  using BL = BwdLayout<L, MODE>;
  if constexpr (ctas_per_sm(BL::bytes) == 1 && BwdLayoutWS<L, MODE>::fits) {  // one CTA per SM: pipelined
    using BW = BwdLayoutWS<L, MODE>;
    const size_t smem = BW::bytes;
    MLIP_CUDA_TRY(cudaFuncSetAttribute(tp_fused_bwd_ws<L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    blocks = std::min(n, blocks);
    {
      MLIP_PROF("tp_fused_bwd", st);
      tp_fused_bwd_ws<L, MODE><<<blocks, kWSThreads, smem, st>>>(n, row_ptr, recv, send, Yg, hprev, Gm, w3img, z2t,
                                                                  s, GinA, GinB, GoutA, GoutB, first_group, dY, dz2,
                                                                  use_bf16, sys_of, dws2, epar, err);
    }
    MLIP_LAUNCH_CHECK();
    return MLIP_OK;
  }
  const size_t smem = BL::bytes;
  MLIP_CUDA_TRY(cudaFuncSetAttribute(tp_fused_bwd<L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  blocks = std::min(n, blocks * resident_ctas(tp_fused_bwd<L, MODE>, smem, BL::NCOLS));
  {
    MLIP_PROF("tp_fused_bwd", st);
    tp_fused_bwd<L, MODE><<<blocks, kThreads, smem, st>>>(n, row_ptr, recv, send, Yg, hprev, Gm, w3img, z2t, s, GinA,
                                                          GinB, GoutA, GoutB, first_group, dY, dz2, use_bf16, sys_of,
                                                          dws2, epar, err);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace

// Path-group layout of W3 for one layer: for each group (first layer: one group
// of the l1 = 0 paths; later layers: one group per l3 = 0..L), the BF16 A
// operands W3_p^T [128 channels][64 hidden] of its paths in the canonical
// K-major layout, concatenated.  Byte offset of each group in *group_off.
int pack_w3_groups(const mlip_model* M, int t, std::vector<uint8_t>& img, std::vector<size_t>& group_off) {
  const int P = M->P, C = M->C, H = M->H, L = M->L;
  std::vector<int> l1s, l2s, l3s;
  for (int a = 0; a <= L; ++a)
    for (int b = 0; b <= 3; ++b)
      for (int c3 = 0; c3 <= L; ++c3)
        if (c3 >= std::abs(a - b) && c3 <= a + b && (a + b + c3) % 2 == 0) { l1s.push_back(a); l2s.push_back(b); l3s.push_back(c3); }
  const float* W3 = M->host_weights.data() + (M->W3[t] - M->d_weights);
  std::vector<std::vector<int>> groups;
  if (t == 0) {
    std::vector<int> g;
    for (int p = 0; p < P; ++p) if (l1s[p] == 0) g.push_back(p);
    groups.push_back(g);
  } else {
    for (int l3 = 0; l3 <= L; ++l3) {
      std::vector<int> g;
      for (int p = 0; p < P; ++p) if (l3s[p] == l3) g.push_back(p);
      groups.push_back(g);
    }
  }
  img.clear();
  group_off.clear();
  for (auto& g : groups) {
    group_off.push_back(img.size());
    for (int p : g) {
      const size_t base = img.size();
      img.resize(base + kW3PathBytes, 0);
      for (int c = 0; c < C; ++c)
        for (int k = 0; k < H; ++k) {
          const uint16_t v = to16(W3[((size_t)k * P + p) * C + c], M->precision == MLIP_PREC_BF16);
          std::memcpy(&img[base + tc::canon_off(c, k)], &v, 2);
        }
    }
  }
  group_off.push_back(img.size());
  return MLIP_OK;
}

// Forward message pass of one layer with the fused kernels: m = mA + mB (one
// buffer per warp set), every component written.
int launch_tp_fused(int L, bool first, int n, const int* row_ptr, const int* recv, const int* send,
                    const float* Yg, const float* h, const uint8_t* w3img, const std::vector<size_t>& goff,
                    const uint8_t* z2t, float s, float* mA, float* mB, int use_bf16, const uint8_t* epar, int* err,
                    cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms;
#define MLIP_G(LL, MM, GI) \
  MLIP_TRY((launch_group<LL, MM>(n, row_ptr, recv, send, Yg, h, w3img + goff[GI], z2t, s, mA, mB, use_bf16, epar, \
                                 err, blocks, st)))
  if (L == 2) {
    if (first) { MLIP_G(2, -1, 0); }
    else { MLIP_G(2, 0, 0); MLIP_G(2, 1, 1); MLIP_G(2, 2, 2); }
  } else if (L == 3) {
    if (first) { MLIP_G(3, -1, 0); }
    else { MLIP_G(3, 0, 0); MLIP_G(3, 1, 1); MLIP_G(3, 2, 2); MLIP_G(3, 3, 3); }
  } else {
    set_error("l_max %d unsupported", L);
    return MLIP_ERR_INVALID_ARG;
  }
#undef MLIP_G
  return MLIP_OK;
}

// Adjoint message pass of one layer with the fused kernels (all groups in
// order); G^{t-1} = GoutA + GoutB.
int launch_tp_fused_bwd(int L, bool first, int n, const int* row_ptr, const int* recv, const int* send,
                        const float* Yg, const float* hprev, const float* Gm, const uint8_t* w3img,
                        const std::vector<size_t>& goff, const uint8_t* z2t, float s, const float* GinA,
                        const float* GinB, float* GoutA, float* GoutB, float* dY, float* dz2, int use_bf16,
                        const int* sys_of, const float2* dws2, const uint8_t* epar, int* err, cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms;
#define MLIP_GB(LL, MM, GI)                                                                                  \
  MLIP_TRY((launch_group_bwd<LL, MM>(n, row_ptr, recv, send, Yg, hprev, Gm, w3img + goff[GI], z2t, s, GinA, GinB, \
                                     GoutA, GoutB, GI == 0, dY, dz2, use_bf16, sys_of, dws2, epar, err, blocks, \
                                     st)))
  if (L == 2) {
    if (first) { MLIP_GB(2, -1, 0); }
    else { MLIP_GB(2, 0, 0); MLIP_GB(2, 1, 1); MLIP_GB(2, 2, 2); }
  } else if (L == 3) {
    if (first) { MLIP_GB(3, -1, 0); }
    else { MLIP_GB(3, 0, 0); MLIP_GB(3, 1, 1); MLIP_GB(3, 2, 2); MLIP_GB(3, 3, 3); }
  } else {
    set_error("l_max %d unsupported", L);
    return MLIP_ERR_INVALID_ARG;
  }
#undef MLIP_GB
  return MLIP_OK;
}

int umma_selftest_run(double* rel_err) {
  const int M = 128, N = 32, K = 64;
  std::vector<float> A(M * K), B(N * K), D(M * N, 0.0f);
  uint64_t st = 12345;
  auto rnd = [&]() {
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    return (float)((st >> 40) & 0xFFFF) / 65536.0f - 0.5f;
  };
  for (auto& a : A) a = __bfloat162float(__float2bfloat16_rn(rnd()));
  for (auto& b : B) b = __bfloat162float(__float2bfloat16_rn(rnd()));
  float *dA, *dB, *dD;
  int* derr;
  MLIP_CUDA_TRY(cudaMalloc(&dA, A.size() * 4));
  MLIP_CUDA_TRY(cudaMalloc(&dB, B.size() * 4));
  MLIP_CUDA_TRY(cudaMalloc(&dD, D.size() * 4));
  MLIP_CUDA_TRY(cudaMalloc(&derr, 4));
  MLIP_CUDA_TRY(cudaMemcpy(dA, A.data(), A.size() * 4, cudaMemcpyHostToDevice));
  MLIP_CUDA_TRY(cudaMemcpy(dB, B.data(), B.size() * 4, cudaMemcpyHostToDevice));
  MLIP_CUDA_TRY(cudaMemset(dD, 0, D.size() * 4));
  MLIP_CUDA_TRY(cudaMemset(derr, 0, 4));
  { MLIP_PROF("umma_selftest", 0); umma_selftest<<<1, 128>>>(dA, dB, dD, derr); }
  MLIP_LAUNCH_CHECK();
  MLIP_CUDA_TRY(cudaDeviceSynchronize());
  int herr = 0;
  MLIP_CUDA_TRY(cudaMemcpy(D.data(), dD, D.size() * 4, cudaMemcpyDeviceToHost));
  MLIP_CUDA_TRY(cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost));
  cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(derr);
  if (herr) { set_error("tensor-core self test: MMA completion wait timed out"); return MLIP_ERR_DEVICE_TIMEOUT; }
  double maxerr = 0, maxref = 0;
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      double ref = 0;
      for (int k = 0; k < K; ++k) ref += (double)A[i * K + k] * B[j * K + k];
      maxerr = std::max(maxerr, std::fabs(ref - D[i * N + j]));
      maxref = std::max(maxref, std::fabs(ref));
    }
  *rel_err = maxerr / std::max(maxref, 1e-30);
  return MLIP_OK;
}

int umma_selftest_mn_run(int variant, double* rel_err) {
  std::vector<float> W(128 * 64), X(32 * 128), D(128 * 32, 0.0f);
  uint64_t st = 777;
  auto rnd = [&]() {
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    return (float)((st >> 40) & 0xFFFF) / 65536.0f - 0.5f;
  };
  for (auto& a : W) a = __bfloat162float(__float2bfloat16_rn(rnd()));
  for (auto& b : X) b = __bfloat162float(__float2bfloat16_rn(rnd()));
  float *dW, *dX, *dD;
  int* derr;
  MLIP_CUDA_TRY(cudaMalloc(&dW, W.size() * 4));
  MLIP_CUDA_TRY(cudaMalloc(&dX, X.size() * 4));
  MLIP_CUDA_TRY(cudaMalloc(&dD, D.size() * 4));
  MLIP_CUDA_TRY(cudaMalloc(&derr, 4));
  MLIP_CUDA_TRY(cudaMemcpy(dW, W.data(), W.size() * 4, cudaMemcpyHostToDevice));
  MLIP_CUDA_TRY(cudaMemcpy(dX, X.data(), X.size() * 4, cudaMemcpyHostToDevice));
  MLIP_CUDA_TRY(cudaMemset(dD, 0, D.size() * 4));
  MLIP_CUDA_TRY(cudaMemset(derr, 0, 4));
  { MLIP_PROF("umma_selftest_mn", 0); umma_selftest_mn<<<1, 128>>>(dW, dX, dD, variant, derr); }
  MLIP_LAUNCH_CHECK();
  MLIP_CUDA_TRY(cudaDeviceSynchronize());
  int herr = 0;
  MLIP_CUDA_TRY(cudaMemcpy(D.data(), dD, D.size() * 4, cudaMemcpyDeviceToHost));
  MLIP_CUDA_TRY(cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost));
  cudaFree(dW); cudaFree(dX); cudaFree(dD); cudaFree(derr);
  if (herr) { set_error("tensor-core self test: MMA completion wait timed out"); return MLIP_ERR_DEVICE_TIMEOUT; }
  double maxerr = 0, maxref = 0;
  for (int k = 0; k < 64; ++k)
    for (int e = 0; e < 32; ++e) {
      double ref = 0;
      for (int c = 0; c < 128; ++c) ref += (double)W[c * 64 + k] * X[e * 128 + c];
      maxerr = std::max(maxerr, std::fabs(ref - D[k * 32 + e]));
      maxref = std::max(maxref, std::fabs(ref));
    }
  *rel_err = maxerr / std::max(maxref, 1e-30);
  return MLIP_OK;
}

// Forward half of one evaluation: edge geometry and harmonics, the layers, the
// readout and the per-system energies.  What the adjoint half reads stays in
// the model's workspace: the node features and mix pre-activations of every
// layer (the contraction's inputs and the gate's pre-activations for those
// options) and the per-system maxima that scale the adjoint's FP16 operand.
int fused_forward_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                        const NeighborList& nl, const int* Edev, int* flag, double* d_energy, cudaStream_t st) {
  Workspace& ws = M->ws;
  const int n = (int)b.n, C = M->C, D = M->D, T = M->T, L = M->L, H = M->H;
  const float s = (float)(1.0 / M->avg_nb);
  const int use_bf16 = M->precision == MLIP_PREC_BF16 ? 1 : 0;
  const int E = (int)nl.E;  // the edge count, or with Edev the capacity
  const int n_tiles = (E + kNT - 1) / kNT;
  const size_t Ec = (size_t)std::max(E, 1), ND = (size_t)std::max(n, 1) * D * C;
  CellArg ca{b.d_cell, b.d_sys_of, b.any_pbc() ? 1 : 0};
  float4* ev = nullptr;
  float *mA = nullptr, *mB = nullptr, *Yg = nullptr;
  double* atom_e = nullptr;
  MLIP_TRY(ws.get("ef.ev", Ec, &ev));
  MLIP_TRY(ws.get("fz.Y", Ec * 16, &Yg));
  MLIP_TRY(ws.get("ef.m", ND, &mA));
  MLIP_TRY(ws.get("fz.m2", ND, &mB));
  MLIP_TRY(ws.get("ef.atom_e", (size_t)std::max(n, 1), &atom_e));
  std::vector<float*> h(T + 1), u0(T), A(T, nullptr), gpre(T, nullptr), gg(T, nullptr);
  std::vector<uint8_t*> z2t(T);
  for (int t = 0; t <= T; ++t) MLIP_TRY(ws.get("ef.h" + std::to_string(t), ND, &h[t]));
  for (int t = 0; t < T; ++t) {
    MLIP_TRY(ws.get("ef.u" + std::to_string(t), (size_t)n * C, &u0[t]));
    if (M->corr == 2) MLIP_TRY(ws.get("ef.A" + std::to_string(t), ND, &A[t]));
    if (M->gate) {
      MLIP_TRY(ws.get("ef.gpre" + std::to_string(t), ND, &gpre[t]));
      MLIP_TRY(ws.get("ef.gg" + std::to_string(t), (size_t)std::max(n, 1) * L * C, &gg[t]));
    }
    MLIP_TRY(ws.get("fz.z2t" + std::to_string(t), (size_t)std::max(n_tiles, 1) * kTileBytes, &z2t[t]));
  }
  uint8_t* epar = nullptr;
  MLIP_TRY(ws.get("fz.epar", Ec, &epar));
  if (E > 0) {
    {
      MLIP_PROF("edge_sh", st);
      edge_sh<<<std::min((E + 255) / 256, 8192), 256, 0, st>>>(E, d_pos, nl.send, nl.shift, ca, ev, Yg, Edev,
                                                               nl.row_ptr, nl.recv, epar);
    }
    MLIP_LAUNCH_CHECK();
  }
  // per layer t and system: max |h^t|, max |dE/dm^t| (FP16 operand scale of the adjoint), accumulated by
  // the kernels that write those tensors
  float* absmax = nullptr;
  MLIP_TRY(ws.get("fz.absmax", 2 * (size_t)T * b.nsys, &absmax));
  if (!use_bf16) MLIP_CUDA_TRY(cudaMemsetAsync(absmax, 0, sizeof(float) * 2 * T * b.nsys, st));
  auto amax_h = [&](int t) -> float* { return use_bf16 || t >= T ? nullptr : absmax + 2 * (size_t)t * b.nsys; };
  MLIP_TRY(launch_embed(n, C, D, M->S, d_species, M->W_emb, h[0], st, b.d_sys_of, M->d_embmax, amax_h(0)));
  for (int t = 0; t < T; ++t) {
    if (!M->d_radimg) { set_error("the fused form needs hidden = 64"); return MLIP_ERR_INVALID_ARG; }
    MLIP_TRY(launch_radial_tc(H, E, n_tiles, ev, M->W1[t], M->d_radimg + (size_t)t * 32768, M->rad_scale[t],
                              (float)M->rc, M->p, use_bf16, z2t[t], flag + 1, st, Edev));
    MLIP_TRY(launch_tp_fused(L, t == 0, n, nl.row_ptr, nl.recv, nl.send, Yg, h[t], M->d_w3img + M->w3_layer_off[t],
                             M->w3_goff[t], z2t[t], s, mA, mB, use_bf16, epar, flag + 1, st));
    float* mB_mix = mB;
    if (M->corr == 2) {  // B(mA + mB) into mA; the mix reads it alone
      MLIP_TRY(launch_sym_contract(L, n, C, M->S, mA, mB, d_species, M->Wsc1[t], M->Wsc2[t], A[t], mA, st));
      mB_mix = nullptr;
    }
    if (M->gate)  // gated update with the species self-connection in place of the mix (tensor cores)
      MLIP_TRY(launch_gate_tc_fwd(L, n, M->S, d_species, mA, mB_mix, h[t], M->gate_fwd_img[t], M->gate_fwd_scale[t],
                                  h[t + 1], gpre[t], gg[t], flag + 1, b.d_sys_of, amax_h(t + 1), st));
    else
      MLIP_TRY(launch_mix_tc(false, n, C, L, mA, mB_mix, M->mix_fwd_img[t], M->mix_scale[t], h[t], h[t + 1], u0[t],
                             nullptr, flag + 1, st, b.d_sys_of, amax_h(t + 1)));
  }
  if (M->charges) {  // readout, charge head and Coulomb term, then the per-system sums
    MLIP_TRY(launch_readout(n, C, D, M->S, d_species, M->W_out, M->E0, h[T], atom_e, st));
    MLIP_TRY(coulomb_forward(ws, b, M, d_pos, d_species, h[T], atom_e, st));
    MLIP_TRY(launch_seg_sum(ws, b, 1, atom_e, false, d_energy, st));
  } else {
    MLIP_TRY(launch_energy(ws, b, C, D, M->S, d_species, M->W_out, M->E0, h[T], atom_e, d_energy, st));
  }
  return MLIP_OK;
}

// Adjoint half: forces and stress from the workspace the forward half left.
// With recompute (a separate forward call came before) the edge geometry, the
// harmonics and every layer's radial MLP output z2 are computed again from the
// positions instead of being read from the forward's per-edge buffers.
int fused_adjoint_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                         const NeighborList& nl, const int* Edev, int* flag, double* d_forces, double* d_stress,
                         bool recompute, cudaStream_t st) {
  Workspace& ws = M->ws;
  const int n = (int)b.n, C = M->C, D = M->D, T = M->T, L = M->L, H = M->H;
  const float s = (float)(1.0 / M->avg_nb);
  const int use_bf16 = M->precision == MLIP_PREC_BF16 ? 1 : 0;
  const int E = (int)nl.E;
  const int n_tiles = (E + kNT - 1) / kNT;
  const size_t Ec = (size_t)std::max(E, 1), ND = (size_t)std::max(n, 1) * D * C;
  CellArg ca{b.d_cell, b.d_sys_of, b.any_pbc() ? 1 : 0};
  float4 *ev = nullptr, *g = nullptr;
  float *Yg = nullptr, *Gm = nullptr, *dY = nullptr, *dr = nullptr, *dz2 = nullptr;
  float *GaA = nullptr, *GaB = nullptr, *GbA = nullptr, *GbB = nullptr;
  MLIP_TRY(ws.get("ef.ev", Ec, &ev));
  MLIP_TRY(ws.get("fz.Y", Ec * 16, &Yg));
  std::vector<float*> h(T + 1), u0(T), A(T, nullptr), gpre(T, nullptr), gg(T, nullptr);
  std::vector<uint8_t*> z2t(T);
  for (int t = 0; t <= T; ++t) MLIP_TRY(ws.get("ef.h" + std::to_string(t), ND, &h[t]));
  for (int t = 0; t < T; ++t) {
    MLIP_TRY(ws.get("ef.u" + std::to_string(t), (size_t)n * C, &u0[t]));
    if (M->corr == 2) MLIP_TRY(ws.get("ef.A" + std::to_string(t), ND, &A[t]));
    if (M->gate) {
      MLIP_TRY(ws.get("ef.gpre" + std::to_string(t), ND, &gpre[t]));
      MLIP_TRY(ws.get("ef.gg" + std::to_string(t), (size_t)std::max(n, 1) * L * C, &gg[t]));
    }
    MLIP_TRY(ws.get("fz.z2t" + std::to_string(t), (size_t)std::max(n_tiles, 1) * kTileBytes, &z2t[t]));
  }
  float *gdpre = nullptr, *gdg = nullptr;  // the tensor-core gate's adjoint scratch
  if (M->gate) {
    MLIP_TRY(ws.get("fz.gdpre", ND, &gdpre));
    MLIP_TRY(ws.get("fz.gdg", (size_t)std::max(n, 1) * L * C, &gdg));
  }
  uint8_t* epar = nullptr;
  MLIP_TRY(ws.get("fz.epar", Ec, &epar));
  if (recompute && E > 0) {
    {
      MLIP_PROF("edge_sh", st);
      edge_sh<<<std::min((E + 255) / 256, 8192), 256, 0, st>>>(E, d_pos, nl.send, nl.shift, ca, ev, Yg, Edev,
                                                               nl.row_ptr, nl.recv, epar);
    }
    MLIP_LAUNCH_CHECK();
  }
  auto zero = [&](float* p, int per) -> int {
    if (E <= 0) return MLIP_OK;
    if (!Edev) {
      MLIP_CUDA_TRY(cudaMemsetAsync(p, 0, (size_t)E * per * sizeof(float), st));
      return MLIP_OK;
    }
    const long long n4 = ((long long)E * per + 3) / 4;
    {
      MLIP_PROF("zero_edges", st);
      zero_edges<<<(int)std::min<long long>((n4 + 255) / 256, 8192), 256, 0, st>>>(Edev, per, p);
    }
    MLIP_LAUNCH_CHECK();
    return MLIP_OK;
  };
  float* absmax = nullptr;
  MLIP_TRY(ws.get("fz.absmax", 2 * (size_t)T * b.nsys, &absmax));
  auto amax_h = [&](int t) -> float* { return use_bf16 || t >= T ? nullptr : absmax + 2 * (size_t)t * b.nsys; };
  {
    MLIP_TRY(ws.get("ef.g", Ec, &g));
    MLIP_TRY(ws.get("ef.Gm", ND, &Gm));
    MLIP_TRY(ws.get("ef.Ga", ND, &GaA));
    MLIP_TRY(ws.get("fz.Ga2", ND, &GaB));
    MLIP_TRY(ws.get("ef.Gb", ND, &GbA));
    MLIP_TRY(ws.get("fz.Gb2", ND, &GbB));
    MLIP_TRY(ws.get("ef.dY", Ec * 16, &dY));
    MLIP_TRY(ws.get("ef.dr", Ec, &dr));
    MLIP_TRY(ws.get("fz.dz2", Ec * 64, &dz2));
    MLIP_TRY(launch_grad_init(n, C, D, M->S, d_species, M->W_out, GaA, st));
    if (M->charges) MLIP_TRY(coulomb_adjoint(ws, b, M, d_species, GaA, st));
    MLIP_CUDA_TRY(cudaMemsetAsync(GaB, 0, ND * sizeof(float), st));
    MLIP_TRY(zero(dY, 16));  // dE/dz2 and dE/dr are initialised by the first group / layer that writes them
    float2* dws2 = nullptr;  // per system: scale of dE/dw and its inverse
    MLIP_TRY(ws.get("fz.dws2", (size_t)b.nsys, &dws2));
    for (int t = T - 1; t >= 0; --t) {
      // max |dE/dm| of the message adjoint's input: from the mix, or from the contraction's adjoint
      float* gmax = use_bf16 ? nullptr : amax_h(t) + 1;
      if (M->gate)  // Gm = dE/dm; GaA <- dE/dh^t's residual part (with the self-connection), GaB <- 0
        MLIP_TRY(launch_gate_tc_bwd(L, n, M->S, d_species, GaA, GaB, gpre[t], gg[t], M->gate_bwd_img[t],
                                    M->gate_bwd_scale[t], Gm, gdpre, gdg, flag + 1, b.d_sys_of,
                                    M->corr == 2 ? nullptr : gmax, st));
      else
        MLIP_TRY(launch_mix_tc(true, n, C, L, GaA, GaB, M->mix_bwd_img[t], M->mix_scale[t], nullptr, Gm, nullptr,
                               u0[t], flag + 1, st, b.d_sys_of, M->corr == 2 ? nullptr : gmax));
      if (M->corr == 2)
        MLIP_TRY(launch_sym_contract_bwd(L, n, C, M->S, Gm, A[t], d_species, M->Wsc1[t], M->Wsc2[t], Gm, b.d_sys_of, gmax,
                                         st));
      {
        MLIP_PROF("dw_scales", st);
        dw_scales<<<(b.nsys + 127) / 128, 128, 0, st>>>(b.nsys, absmax + 2 * (size_t)t * b.nsys, s, use_bf16,
                                                        dws2);
        MLIP_LAUNCH_CHECK();
      }
      if (recompute)  // the radial weights of this layer, again from the edge lengths
        MLIP_TRY(launch_radial_tc(H, E, n_tiles, ev, M->W1[t], M->d_radimg + (size_t)t * 32768, M->rad_scale[t],
                                  (float)M->rc, M->p, use_bf16, z2t[t], flag + 1, st, Edev));
      MLIP_TRY(launch_tp_fused_bwd(L, t == 0, n, nl.row_ptr, nl.recv, nl.send, Yg, h[t], Gm,
                                   M->d_w3img + M->w3_layer_off[t], M->w3_goff[t], z2t[t], s, GaA, GaB, GbA, GbB, dY,
                                   dz2, use_bf16, b.d_sys_of, dws2, epar, flag + 1, st));
      MLIP_TRY(launch_radial_bwd_tc(H, E, ev, M->W1[t], M->d_radimg + (size_t)t * 32768, M->rad_scale[t],
                                    (float)M->rc, M->p, dz2, dr, t == T - 1, flag + 1, st, Edev));
      std::swap(GaA, GbA);
      std::swap(GaB, GbB);
    }
    MLIP_TRY(launch_edge_grad(E, ev, dY, dr, g, st, Edev));
    double* fbuf = d_forces;
    if (!fbuf) MLIP_TRY(ws.get("ef.fscratch", (size_t)3 * std::max(n, 1), &fbuf));
    MLIP_TRY(launch_forces_virial(ws, b, nl.row_ptr, nl.rev, g, ev, fbuf, d_stress, st));
    if (M->charges) MLIP_TRY(coulomb_add_forces(ws, b, fbuf, st));
  }
  return MLIP_OK;
}

int evaluate_fused_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                         const NeighborList& nl, const int* Edev, int* flag, double* d_energy, double* d_forces,
                         double* d_stress, cudaStream_t st) {
  MLIP_TRY(fused_forward_edges(M, d_pos, d_species, b, nl, Edev, flag, d_energy, st));
  if (d_forces || d_stress)
    MLIP_TRY(fused_adjoint_edges(M, d_pos, d_species, b, nl, Edev, flag, d_forces, d_stress, false, st));
  return MLIP_OK;
}

int check_eval_flags(const int* flag, cudaStream_t st) {
  int hflag[2] = {0, 0};
  MLIP_CUDA_TRY(cudaMemcpyAsync(hflag, flag, sizeof(hflag), cudaMemcpyDeviceToHost, st));
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  if (hflag[0] & 1) { set_error("species index out of range"); return MLIP_ERR_INVALID_ARG; }
  if (hflag[0] & 2) { set_error("non-finite position"); return MLIP_ERR_INVALID_ARG; }
  if (hflag[1]) { set_error("fused kernel: a bounded wait timed out (code %d)", hflag[1]); return MLIP_ERR_DEVICE_TIMEOUT; }
  return MLIP_OK;
}

// evaluate_fused; reports the edge count and the degree capacity of its build
static int evaluate_fused_exact(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                                double* d_energy, double* d_forces, double* d_stress, cudaStream_t st,
                                int64_t* E_out, int* maxdeg_out) {
  Workspace& ws = M->ws;
  int* flag = nullptr;
  MLIP_TRY(ws.get("chk.flag", 2, &flag));
  MLIP_CUDA_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
  MLIP_TRY(launch_check_inputs((int)b.n, d_pos, d_species, M->S, flag, st));
  NeighborList nl;
  MLIP_TRY(build_neighbors_batch(ws, d_pos, b, M->rc, true, st, &nl));
  if (E_out) *E_out = nl.E;
  if (maxdeg_out) *maxdeg_out = nl.maxdeg;
  MLIP_TRY(evaluate_fused_edges(M, d_pos, d_species, b, nl, nullptr, flag, d_energy, d_forces, d_stress, st));
  return check_eval_flags(flag, st);
}

int evaluate_fused(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                   double* d_energy, double* d_forces, double* d_stress, cudaStream_t st) {
  return evaluate_fused_exact(M, d_pos, d_species, b, d_energy, d_forces, d_stress, st, nullptr, nullptr);
}

// ------------------------------------------------ graph-replayed evaluation
// One cached graph per layout, a few per model (a server alternates layouts).
struct EvalGraph {
  // the layout and outputs the graph serves
  int64_t n = -1;
  int nsys = -1;
  bool forces = false, stress = false;
  long long prof = -1;  // timing configuration at the capture
  std::vector<int64_t> atom_off;
  std::vector<uint8_t> pbc;
  // capacities: from the last exact build (edge count with 25 % headroom)
  int64_t E_exact = -1, Ecap = 0;
  int maxdeg = 0;
  NlPlan plan;
  uint64_t warm_gen = ~0ULL;  // workspace generation of the last eager run of the graph's launches
  uint64_t graph_gen = ~0ULL;
  bool broken = false;        // a capture failed: this layout runs eagerly
  uint64_t last_use = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  std::vector<ProfEvent> events;
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    prof_events_free(events);
    graph_gen = ~0ULL;
  }
  ~EvalGraph() { drop_graph(); }
};

struct EvalGraphs {
  std::vector<std::unique_ptr<EvalGraph>> g;
  cudaStream_t cap = nullptr;  // capture stream (capture needs a stream other than the legacy one)
  uint64_t clock = 0;
  ~EvalGraphs() {
    g.clear();
    if (cap) cudaStreamDestroy(cap);
  }
};

void free_eval_graphs(EvalGraphs* g) { delete g; }

static constexpr size_t kMaxCachedGraphs = 24;

int evaluate_fused_graph(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                         double* d_energy, double* d_forces, double* d_stress, cudaStream_t st) {
  if (!M->egraph) M->egraph = new EvalGraphs();
  EvalGraphs& GS = *M->egraph;
  Workspace& ws = M->ws;
  const int64_t n = b.n;
  const int nsys = b.nsys;
  const bool prof = prof_timing_on();
  const long long pcfg = prof_config();
  EvalGraph* found = nullptr;
  for (auto& e : GS.g) {
    EvalGraph& G = *e;
    if (G.n == n && G.nsys == nsys && G.forces == (d_forces != nullptr) && G.stress == (d_stress != nullptr) &&
        G.prof == pcfg && G.atom_off == b.atom_off && G.pbc == b.pbc) {
      found = &G;
      break;
    }
  }
  if (!found) {
    if (GS.g.size() >= kMaxCachedGraphs) {  // the least recently used makes room
      size_t lru = 0;
      for (size_t k = 1; k < GS.g.size(); ++k)
        if (GS.g[k]->last_use < GS.g[lru]->last_use) lru = k;
      GS.g.erase(GS.g.begin() + lru);
    }
    GS.g.push_back(std::make_unique<EvalGraph>());
    found = GS.g.back().get();
    found->n = n;
    found->nsys = nsys;
    found->forces = d_forces != nullptr;
    found->stress = d_stress != nullptr;
    found->prof = pcfg;
    found->atom_off = b.atom_off;
    found->pbc = b.pbc;
  }
  EvalGraph& G = *found;
  G.last_use = ++GS.clock;
  auto exact = [&]() -> int {
    int64_t E = 0;
    int md = 0;
    G.drop_graph();
    G.warm_gen = ~0ULL;
    MLIP_TRY(evaluate_fused_exact(M, d_pos, d_species, b, d_energy, d_forces, d_stress, st, &E, &md));
    G.E_exact = E;
    G.Ecap = std::max<int64_t>(G.Ecap, E + E / 4 + 4096);
    G.maxdeg = std::max(G.maxdeg, md);
    return MLIP_OK;
  };
  if (G.broken || G.E_exact < 0) return exact();

  // graph-owned inputs, outputs and flags (eval [0..1], neighbours [2..5])
  double *gpos = nullptr, *gE = nullptr, *gF = nullptr, *gS = nullptr;
  int *gsp = nullptr, *gflags = nullptr;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  MLIP_TRY(ws.get("eg.pos", 3 * nn, &gpos));
  MLIP_TRY(ws.get("eg.sp", nn, &gsp));
  MLIP_TRY(ws.get("eg.E", (size_t)nsys, &gE));
  MLIP_TRY(ws.get("eg.F", 3 * nn, &gF));
  MLIP_TRY(ws.get("eg.S", 9 * (size_t)nsys, &gS));
  MLIP_TRY(ws.get("eg.flags", 8, &gflags));
  MLIP_TRY(nl_plan(ws, M->stage, b, M->rc, G.maxdeg, G.Ecap, st, &G.plan));
  MLIP_CUDA_TRY(cudaMemcpyAsync(gpos, d_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(gsp, d_species, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
  auto body = [&](cudaStream_t s) -> int {
    MLIP_CUDA_TRY(cudaMemsetAsync(gflags, 0, 8 * sizeof(int), s));
    MLIP_TRY(launch_check_inputs((int)n, gpos, gsp, M->S, gflags, s));
    NeighborList nl;
    MLIP_TRY(build_neighbors_nosync(ws, gpos, b, G.plan, s, &nl, gflags + 2));
    return evaluate_fused_edges(M, gpos, gsp, b, nl, nl.row_ptr + n, gflags, gE, G.forces ? gF : nullptr,
                                G.stress ? gS : nullptr, s);
  };
  bool replayed = false;
  if (G.exec && G.graph_gen == ws.gen) {
    MLIP_CUDA_TRY(cudaGraphLaunch(G.exec, st));
    prof_add_launches(G.kernels);
    replayed = true;
  } else if (G.warm_gen == ws.gen) {
    G.drop_graph();
    if (!GS.cap) MLIP_CUDA_TRY(cudaStreamCreateWithFlags(&GS.cap, cudaStreamNonBlocking));
    const long long l0 = prof_launches();
    cudaError_t ce = cudaStreamBeginCapture(GS.cap, cudaStreamCaptureModeRelaxed);
    int rc = MLIP_ERR_CUDA;
    if (ce == cudaSuccess) {
      if (prof) prof_capture_begin(&G.events);
      rc = body(GS.cap);
      if (prof) prof_capture_end();
      cudaGraph_t g = nullptr;
      ce = cudaStreamEndCapture(GS.cap, &g);
      G.graph = g;
    }
    if (rc == MLIP_OK && ce == cudaSuccess && G.graph)
      ce = cudaGraphInstantiate(&G.exec, G.graph, 0);
    if (rc != MLIP_OK || ce != cudaSuccess || !G.exec) {
      cudaGetLastError();  // a capture that cannot be made: this layout runs without a graph
      G.drop_graph();
      G.broken = true;
      return exact();
    }
    G.kernels = prof_launches() - l0;
    G.graph_gen = ws.gen;
    MLIP_CUDA_TRY(cudaGraphLaunch(G.exec, st));
    replayed = true;
  } else {
    MLIP_TRY(body(st));
    G.warm_gen = ws.gen;
  }
  int hf[8];
  MLIP_CUDA_TRY(cudaMemcpyAsync(hf, gflags, sizeof(hf), cudaMemcpyDeviceToHost, st));
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  if (replayed && prof) prof_graph_collect(G.events);
  if (hf[0] & 1) { set_error("species index out of range"); return MLIP_ERR_INVALID_ARG; }
  if (hf[0] & 2) { set_error("non-finite position"); return MLIP_ERR_INVALID_ARG; }
  if (hf[1]) { set_error("fused kernel: a bounded wait timed out (code %d)", hf[1]); return MLIP_ERR_DEVICE_TIMEOUT; }
  if (hf[2] > G.maxdeg || hf[5] || hf[3] || hf[4]) return exact();  // out of room (or an unusual list): exactly
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_energy, gE, sizeof(double) * nsys, cudaMemcpyDeviceToDevice, st));
  if (d_forces) MLIP_CUDA_TRY(cudaMemcpyAsync(d_forces, gF, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
  if (d_stress) MLIP_CUDA_TRY(cudaMemcpyAsync(d_stress, gS, sizeof(double) * 9 * nsys, cudaMemcpyDeviceToDevice, st));
  return MLIP_OK;
}

}  // namespace mlip
