// Gated update with the species self-connection on the tensor cores (fused
// form, 128 channels).  The update of one layer (node i of species z, order l,
// channel n; l >= 1 gates q = (l - 1) C + n):
//   pre_l = m_l W_l + h_l Wself[z][l]
//   g_q   = m_0 Wgate[:, q] + h_0 Wselfgate[z][:, q]
//   h'_0  = h_0 + silu(pre_0),   h'_l = h_l + sigmoid(g_l) pre_l
// and its adjoint from G' = dE/dh':
//   dpre_0 = G'_0 silu'(pre_0),  dpre_l = G'_l sigmoid(g_l),  dg_l = sigmoid'(g_l) sum_m G'_l,m pre_l,m
//   dE/dm_l = dpre_l W_l^T (+ dg Wgate^T, l = 0)
//   dE/dh_l = G'_l + dpre_l Wself[z][l]^T (+ dg Wselfgate[z]^T, l = 0)
// are sums of 128 x 128 products over the (2l + 1) N rows of order l.  One CTA
// takes 128 rows and runs a list of terms: a source A (the messages, the
// features or dE/dpre of the rows, or a block of 128 gates / gate gradients of
// the rows' nodes), optionally masked to the rows of one species, times a
// weight block B, accumulated into one 128-column output block in tensor
// memory (forward order 0: pre_0 or one of L gate blocks; later orders: pre_l;
// adjoint: dE/dm or dE/dh), one CTA per row tile, order and output block.
// The species self-connection thus costs S terms whose A rows
// of the other species are zero: tensor-core work is cheap next to the rows'
// traffic.  Operands are split FP16 (split16.cuh) with one power-of-two scale
// per row (over the sources feeding the CTA's output block) and one per output
// block of B, so the sums keep about 21 significant bits.  The epilogue applies the update
// (forward) or writes dE/dm and adds dE/dh (adjoint).  Order 0 runs first in
// the forward: the later orders read its gates.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "kernels_common.cuh"
#include "launchers.cuh"
#include "mlip_internal.cuh"
#include "profile.cuh"
#include "sm100_tc.cuh"
#include "split16.cuh"

namespace mlip {

namespace {

// One term of an order's list.  src: forward 0 = messages, 1 = features;
// adjoint 0 = dE/dpre, 1 + b = gate-gradient block b (order 0 only).
// mask: species of the rows kept (-1: all).  out: tensor-memory block.
struct GateTerm {
  int src, mask, out;
};

// Terms of order l (bwd: adjoint), grouped so that consecutive terms with the
// same source and mask share the A operand.
__host__ __device__ inline int gate_nterms(bool bwd, int l, int L, int S) {
  return l == 0 ? (1 + L) * (1 + S) : 1 + S;
}

__host__ __device__ inline GateTerm gate_term(bool bwd, int l, int L, int S, int j) {
  GateTerm t;
  if (l == 0) {
    const int m = j / (1 + L), b = j % (1 + L);  // m: 0 = no mask, 1 + s = species s
    t.mask = m - 1;
    if (!bwd) {  // A: messages (m = 0) or features of species s; out: pre_0 (b = 0) or gate block b
      t.src = m == 0 ? 0 : 1;
      t.out = b;
    } else {  // A: dE/dpre_0 (b = 0) or gate-gradient block b; out: dE/dm (m = 0) or dE/dh
      t.src = b;
      t.out = m == 0 ? 0 : 1;
    }
  } else {
    t.mask = j - 1;
    t.src = bwd ? 0 : (j == 0 ? 0 : 1);
    t.out = bwd ? (j == 0 ? 0 : 1) : 0;
  }
  return t;
}

}  // namespace

// Weight blocks of one layer for the terms above, every order in turn, each as
// a split FP16 B operand B[n][k] (n: output channel, k: input channel; hi then
// lo, 64 KB), and per (order, output block) the power of two applied to every
// block feeding it.  Wm [L+1][C][C], Ws [S][L+1][C][C], Wg [C][L C],
// Wsg [S][C][L C] (host).  img receives the blocks, scale [L+1][4].
void pack_gate_images(bool bwd, const float* Wm, const float* Ws, const float* Wg, const float* Wsg, int L, int S,
                      std::vector<uint8_t>& img, std::vector<float>& scale) {
  const int C = kMC, LC = L * C;
  // element (n, k) of the weight block of term t at order l
  auto elem = [&](int l, const GateTerm& t, int n, int k) -> float {
    if (!bwd) {
      // A row (k) times B gives output n: pre needs W[k][n], gates Wg[k][(b-1) C + n]
      const bool self = t.mask >= 0;
      if (t.out == 0) {
        return self ? Ws[(((size_t)t.mask * (L + 1) + l) * C + k) * C + n] : Wm[((size_t)l * C + k) * C + n];
      }
      const int q = (t.out - 1) * C + n;
      return self ? Wsg[((size_t)t.mask * C + k) * LC + q] : Wg[(size_t)k * LC + q];
    }
    // adjoint: output k' = n (an input channel of the forward), A column k (a forward output)
    const bool self = t.mask >= 0;
    if (t.src == 0) {  // dE/dpre_l: W[n][k]
      return self ? Ws[(((size_t)t.mask * (L + 1) + l) * C + n) * C + k] : Wm[((size_t)l * C + n) * C + k];
    }
    const int q = (t.src - 1) * C + k;  // gate-gradient block: Wg[n][q]
    return self ? Wsg[((size_t)t.mask * C + n) * LC + q] : Wg[(size_t)n * LC + q];
  };
  size_t nblk = 0;
  for (int l = 0; l <= L; ++l) nblk += gate_nterms(bwd, l, L, S);
  img.assign(nblk * 2 * kMOp, 0);
  scale.assign((size_t)(L + 1) * 4, 1.0f);
  size_t blk = 0;
  for (int l = 0; l <= L; ++l) {
    const int nt = gate_nterms(bwd, l, L, S);
    float amax[4] = {0, 0, 0, 0};
    for (int j = 0; j < nt; ++j) {
      const GateTerm t = gate_term(bwd, l, L, S, j);
      for (int n = 0; n < C; ++n)
        for (int k = 0; k < C; ++k) amax[t.out] = std::max(amax[t.out], std::fabs(elem(l, t, n, k)));
    }
    for (int b = 0; b < 4; ++b)
      scale[(size_t)l * 4 + b] = amax[b] > 0.0f ? std::ldexp(1.0f, 13 - std::ilogb(amax[b])) : 1.0f;
    for (int j = 0; j < nt; ++j, ++blk) {
      const GateTerm t = gate_term(bwd, l, L, S, j);
      const float sc = scale[(size_t)l * 4 + t.out];
      uint8_t* o = img.data() + blk * 2 * kMOp;
      for (int n = 0; n < C; ++n)
        for (int k = 0; k < C; ++k) {
          const float x = elem(l, t, n, k) * sc;
          const __half h = __float2half_rn(x);
          const __half lo = __float2half_rn(x - __half2float(h));
          std::memcpy(o + canon128(n, k), &h, 2);
          std::memcpy(o + kMOp + canon128(n, k), &lo, 2);
        }
    }
  }
}

// First block of order l in a layer's image list.
__host__ __device__ inline size_t gate_block0(bool bwd, int l, int L, int S) {
  size_t b = 0;
  for (int q = 0; q < l; ++q) b += gate_nterms(bwd, q, L, S);
  return b;
}

namespace {

// One CTA: 128 rows of order l = l_first + blockIdx.y (two threads a row, 64
// channels each), output block blockIdx.z (ncols: its tensor-memory columns).
// Forward: A0 (+ A0b) = the message buffers, A1 = the input features; writes
// pre, the gates (order 0) and the updated features.
// Adjoint: A0 = dE/dpre, A1 = dE/dg [N][L][C]; writes Gm = dE/dm and adds
// dE/dh into G (which holds dE/dh').
template <bool BWD>
__global__ void __launch_bounds__(2 * kMM) gate_tc(int n, int L, int S, int l_first, int ncols,
                                                   const int* __restrict__ species, const float* __restrict__ A0,
                                                   const float* __restrict__ A0b, const float* __restrict__ A1,
                                                   const uint8_t* __restrict__ img, const float* __restrict__ wscale,
                                                   const float* __restrict__ hin, float* __restrict__ hout,
                                                   float* __restrict__ pre, float* __restrict__ gq,
                                                   float* __restrict__ Gm, float* __restrict__ G, int* __restrict__ err,
                                                   const int* __restrict__ sys_of, float* __restrict__ out_max) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAh = smem;
  uint8_t* sAl = smem + kMOp;
  uint8_t* sBh = smem + 2 * kMOp;
  uint8_t* sBl = smem + 3 * kMOp;
  __shared__ __align__(8) uint64_t bar_w, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_s;
  __shared__ float s_amax[2 * kMM];
  const int l = l_first + blockIdx.y, R = 2 * l + 1, D = (L + 1) * (L + 1), LC = L * kMC;
  const int rows = n * R, row0 = blockIdx.x * kMM;
  if (row0 >= rows) return;  // uniform over the CTA
  const int tid = threadIdx.x, warp = tid >> 5;
  const int rt = tid & (kMM - 1), half = tid >> 7;
  constexpr int HC = kMC / 2;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, (uint32_t)ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar_w, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::fence_mbar_init();
    abort_s = 0;
  }
  const int r = row0 + rt;
  const bool live = r < rows;
  const int nd = live ? r / R : 0, mm = live ? r % R : 0;
  const int z = live ? clamp_species(species[nd], S) : -1;
  const size_t base = ((size_t)nd * D + l * l + mm) * kMC;  // this row in [N][D][C] tensors
  const int c0 = half * HC;                                   // first channel of this thread
  // half row of source src (zeros for a dead row)
  auto load = [&](int src, float* v) {
    const float* p = nullptr;
    const float* p2 = nullptr;
    if (!BWD) {
      p = src == 0 ? A0 + base : hin + base;
      if (src == 0 && A0b) p2 = A0b + base;
    } else {
      p = src == 0 ? A0 + base : A1 + ((size_t)nd * L + src - 1) * kMC;
    }
#pragma unroll
    for (int q = 0; q < HC / 4; ++q) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      if (live) {
        a = reinterpret_cast<const float4*>(p + c0)[q];
        if (p2) {
          const float4 b = reinterpret_cast<const float4*>(p2 + c0)[q];
          a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
        }
      }
      v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
    }
  };
  // this CTA's output block ob: the terms feeding it, and the row's scale over the sources they read
  const int ob = blockIdx.z;
  const int nt = gate_nterms(BWD, l, L, S);
  unsigned srcs = 0;
  for (int j = 0; j < nt; ++j) {
    const GateTerm t = gate_term(BWD, l, L, S, j);
    if (t.out == ob) srcs |= 1u << t.src;
  }
  {
    float amax = 0.0f;
    for (int src = 0; src < 4; ++src) {
      if (!((srcs >> src) & 1u)) continue;
      float v[HC];
      load(src, v);
#pragma unroll
      for (int k = 0; k < HC; ++k) amax = fmaxf(amax, fabsf(v[k]));
    }
    s_amax[tid] = amax;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const float sc = pow2_scale(fmaxf(s_amax[rt], s_amax[rt + kMM]));
  const uint8_t* blocks = img + gate_block0(BWD, l, L, S) * 2 * kMOp;
  const uint32_t idesc = tc::idesc_16bit(kMM, kMC, false);
  int prev_src = -1, prev_mask = -2;
  int k = 0;     // this CTA's products so far (the same count on every thread)
  int done = 0;  // products committed (tid 0)
#pragma unroll 1
  for (int j = 0; j < nt; ++j) {
    const GateTerm t = gate_term(BWD, l, L, S, j);
    if (t.out != ob) continue;  // uniform
    __syncthreads();
    if (abort_s) break;  // uniform
    if (k > 0 && !tc::mbar_wait(&bar_mma, (uint32_t)((k - 1) & 1))) {  // the previous product has read A and B
      atomicOr(err, 256);
      abort_s = 1;
    }
    tc::fence_after_sync();
    __syncthreads();
    if (abort_s) break;
    if (tid == 0) {
      tc::mbar_arrive_expect_tx(&bar_w, 2 * kMOp);
      tc::bulk_g2s(sBh, blocks + (size_t)j * 2 * kMOp, kMOp, &bar_w);
      tc::bulk_g2s(sBl, blocks + (size_t)j * 2 * kMOp + kMOp, kMOp, &bar_w);
    }
    if (t.src != prev_src || t.mask != prev_mask) {  // a new A operand (uniform: the list is)
      float v[HC];
      if (t.mask >= 0 && z != t.mask) {  // a row of another species: zeros, nothing to load
#pragma unroll
        for (int k = 0; k < HC; ++k) v[k] = 0.0f;
      } else {
        load(t.src, v);
      }
#pragma unroll
      for (int kh = 0; kh < HC / 8; ++kh) {
        const int kg = half * (HC / 8) + kh;
        split8(v + kh * 8, sc, reinterpret_cast<uint4*>(sAh + canon128(rt, kg * 8)),
               reinterpret_cast<uint4*>(sAl + canon128(rt, kg * 8)));
      }
      tc::fence_proxy_async_smem();
      prev_src = t.src;
      prev_mask = t.mask;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      if (tc::mbar_wait(&bar_w, (uint32_t)(k & 1))) {
        tc::fence_after_sync();
        const uint32_t ah = tc::smem_u32(sAh), al = tc::smem_u32(sAl), bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);
        const uint32_t as[3] = {ah, al, ah}, bs[3] = {bh, bh, bl};
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass)
#pragma unroll
          for (int kk = 0; kk < kMC / 16; ++kk) {
            const uint64_t ad = tc::desc_noswizzle(as[pass] + kk * 256, kMLBO, kMSBO);
            const uint64_t bd = tc::desc_noswizzle(bs[pass] + kk * 256, kMLBO, kMSBO);
            tc::mma_bf16(tbase, ad, bd, idesc, (k | pass | kk) ? 1u : 0u);
          }
        tc::mma_commit(&bar_mma);
        done = k + 1;
      } else {
        atomicOr(err, 256);
        abort_s = 1;
      }
    }
    ++k;
  }
  __syncthreads();
  if (!abort_s && k > 0 && !tc::mbar_wait(&bar_mma, (uint32_t)((k - 1) & 1))) {
    atomicOr(err, 256);
    abort_s = 1;
  }
  __syncthreads();  // abort_s is uniform from here on
  tc::fence_after_sync();
  if (!abort_s) {  // every warp reads its lanes (tcgen05.ld is warp-collective)
    const uint32_t taddr = tbase + ((uint32_t)((warp & 3) * 32) << 16);
    float m = 0.0f;
    {
      const int b = ob;
      const float inv = 1.0f / (sc * wscale[l * 4 + b]);
#pragma unroll 1
      for (int cc = c0; cc < c0 + HC; cc += 32) {
        float w[32];
#pragma unroll
        for (int c = 0; c < 32; c += 8) tc::tmem_ld8(taddr + cc + c, w + c);
        tc::tmem_ld_wait();
        if (!live) continue;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int ch = cc + 4 * q;
          const float4 u = make_float4(w[4 * q] * inv, w[4 * q + 1] * inv, w[4 * q + 2] * inv, w[4 * q + 3] * inv);
          if (!BWD) {
            if (b > 0) {  // gate block b of node nd (order 0 rows)
              reinterpret_cast<float4*>(gq + (size_t)nd * LC + (b - 1) * kMC + ch)[0] = u;
              continue;
            }
            reinterpret_cast<float4*>(pre + base + ch)[0] = u;
            const float4 h = reinterpret_cast<const float4*>(hin + base + ch)[0];
            float4 o;
            if (l == 0) {
              o = make_float4(h.x + silu_f(u.x), h.y + silu_f(u.y), h.z + silu_f(u.z), h.w + silu_f(u.w));
            } else {
              const float4 gg = reinterpret_cast<const float4*>(gq + (size_t)nd * LC + (l - 1) * kMC + ch)[0];
              o = make_float4(h.x + sigmoid_f(gg.x) * u.x, h.y + sigmoid_f(gg.y) * u.y, h.z + sigmoid_f(gg.z) * u.z,
                              h.w + sigmoid_f(gg.w) * u.w);
            }
            reinterpret_cast<float4*>(hout + base + ch)[0] = o;
            m = fmaxf(m, fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)), fmaxf(fabsf(o.z), fabsf(o.w))));
          } else if (b == 0) {  // dE/dm
            reinterpret_cast<float4*>(Gm + base + ch)[0] = u;
            m = fmaxf(m, fmaxf(fmaxf(fabsf(u.x), fabsf(u.y)), fmaxf(fabsf(u.z), fabsf(u.w))));
          } else {  // dE/dh = dE/dh' + the self-connection's part
            float4* gp = reinterpret_cast<float4*>(G + base + ch);
            float4 gv = gp[0];
            gv.x += u.x; gv.y += u.y; gv.z += u.z; gv.w += u.w;
            gp[0] = gv;
          }
        }
      }
    }
    if (out_max && ob == 0) warp_sys_max(out_max, live ? (sys_of ? sys_of[nd] : 0) : -1, m);
  }
  if (tid == 0 && abort_s) {  // bounded waits for what is still in flight
    if (done > 0) tc::mbar_wait(&bar_mma, (uint32_t)((done - 1) & 1), 1LL << 20);
    tc::mbar_wait(&bar_w, (uint32_t)((done) & 1), 1LL << 20);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, (uint32_t)ncols);
}

}  // namespace

namespace {

// Adjoint's elementwise part, one thread per (node, channel): G <- G + G2 (the
// two partial buffers of dE/dh'; G2 <- 0), dE/dpre and dE/dg for the products.
// The order is a template parameter so that every row's loads issue at once.
template <int L>
__global__ void __launch_bounds__(128) gate_tc_prep(int n, float* __restrict__ G, float* __restrict__ G2,
                                                    const float* __restrict__ pre, const float* __restrict__ gq,
                                                    float* __restrict__ dpre, float* __restrict__ dg) {
  constexpr int D = (L + 1) * (L + 1);
  const int nd = blockIdx.x, c = threadIdx.x;
  if (nd >= n) return;
  float gv[D], p[D], s[L + 1];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    const size_t o = ((size_t)nd * D + r) * kMC + c;
    gv[r] = G[o] + (G2 ? G2[o] : 0.0f);
    p[r] = pre[o];
  }
#pragma unroll
  for (int l = 1; l <= L; ++l) s[l] = sigmoid_f(gq[((size_t)nd * L + l - 1) * kMC + c]);
#pragma unroll
  for (int r = 0; r < D; ++r) {
    const size_t o = ((size_t)nd * D + r) * kMC + c;
    if (G2) {
      G[o] = gv[r];
      G2[o] = 0.0f;
    }
  }
  dpre[(size_t)nd * D * kMC + c] = gv[0] * silu_grad_f(p[0]);
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    float acc = 0.0f;
#pragma unroll
    for (int mm = 0; mm < 2 * l + 1; ++mm) {
      const int r = l * l + mm;
      dpre[((size_t)nd * D + r) * kMC + c] = gv[r] * s[l];
      acc = fmaf(gv[r], p[r], acc);
    }
    dg[((size_t)nd * L + l - 1) * kMC + c] = acc * s[l] * (1.0f - s[l]);
  }
}

constexpr int kGateSmem = 4 * kMOp;

}  // namespace

int gate_tc_prepare() {
  MLIP_CUDA_TRY(cudaFuncSetAttribute(gate_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGateSmem));
  MLIP_CUDA_TRY(cudaFuncSetAttribute(gate_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGateSmem));
  return MLIP_OK;
}

int launch_gate_tc_fwd(int L, int n, int S, const int* species, const float* X, const float* X2, const float* hin,
                       const uint8_t* img, const float* wscale, float* hout, float* pre, float* g, int* err,
                       const int* sys_of, float* out_max, cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  if (L < 1 || L > 3) { set_error("tensor-core gate: l_max must be 1, 2 or 3"); return MLIP_ERR_INVALID_ARG; }
  {  // order 0 first (the pre-activations of the scalars and every gate), then the other orders
    MLIP_PROF("gate_fwd", st);
    gate_tc<false><<<dim3((n + kMM - 1) / kMM, 1, 1 + L), 2 * kMM, kGateSmem, st>>>(
        n, L, S, 0, kMC, species, X, X2, hin, img, wscale, hin, hout, pre, g, nullptr,
        nullptr, err, sys_of, out_max);
  }
  MLIP_LAUNCH_CHECK();
  {
    MLIP_PROF("gate_fwd", st);
    gate_tc<false><<<dim3((n * (2 * L + 1) + kMM - 1) / kMM, L, 1), 2 * kMM, kGateSmem, st>>>(
        n, L, S, 1, kMC, species, X, X2, hin, img, wscale, hin, hout, pre, g, nullptr, nullptr, err, sys_of,
        out_max);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

int launch_gate_tc_bwd(int L, int n, int S, const int* species, float* G, float* G2, const float* pre, const float* g,
                       const uint8_t* img, const float* wscale, float* Gm, float* dpre, float* dg, int* err,
                       const int* sys_of, float* out_max, cudaStream_t st) {
  if (n <= 0) return MLIP_OK;
  if (L < 1 || L > 3) { set_error("tensor-core gate: l_max must be 1, 2 or 3"); return MLIP_ERR_INVALID_ARG; }
  {
    MLIP_PROF("gate_prep", st);
    if (L == 1) gate_tc_prep<1><<<n, kMC, 0, st>>>(n, G, G2, pre, g, dpre, dg);
    else if (L == 2) gate_tc_prep<2><<<n, kMC, 0, st>>>(n, G, G2, pre, g, dpre, dg);
    else gate_tc_prep<3><<<n, kMC, 0, st>>>(n, G, G2, pre, g, dpre, dg);
  }
  MLIP_LAUNCH_CHECK();
  {
    MLIP_PROF("gate_bwd", st);
    gate_tc<true><<<dim3((n * (2 * L + 1) + kMM - 1) / kMM, L + 1, 2), 2 * kMM, kGateSmem, st>>>(
        n, L, S, 0, kMC, species, dpre, nullptr, dg, img, wscale, nullptr, nullptr, nullptr, nullptr, Gm, G,
        err, sys_of, out_max);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace mlip
