// Subsampled Hessian rows (Eq. full_hessian, H_ij = d2E / dr_i dr_j = -dF_i/dr_j,
// and the rows of Eq. sampled_hessian2) by forward-over-reverse
// differentiation: the layer and its hand-written adjoint (the forces) run in
// dual numbers that carry, next to every value, its derivative along three
// tangent directions of the positions.  With the tangents e_{rho,x}, e_{rho,y},
// e_{rho,z} on one atom rho the derivative of the forces is -H e = -(rows of
// atom rho) (H is symmetric), all 3n entries of three rows in one pass.  For a
// batch of graphs the tangents sit on the row atom of every graph at once:
// graphs do not interact, so one pass gives Eq. sampled_hessian2's rows of the
// summed forces F_rho = sum_g F_{i_rho,g}, the concatenation of the graphs' rows.
//
// The kernels are plain SIMT code on FP32 duals with the model's FP32 weights
// (every precision form of a model gives the same rows): per edge the edge
// vector, harmonics and radial basis (and, in the adjoint, the basis
// derivative) and the radial MLP with its per-path weights w (stored per edge
// for the pass); per receiver and channel the tensor product with its
// segmented sum; per node the channel mixes; then the reverse chain in the
// same order as the library's FP32 form.  The nonlinear steps are written out
// generically, so the duals carry their second derivatives.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels_common.cuh"
#include "launchers.cuh"
#include "profile.cuh"
#include "sh_poly.h"

namespace mlip {
namespace {

constexpr int kNT = 3;  // tangents per pass: the three axes of the row atoms

// A value with its derivatives along kNT tangents.
struct Dn {
  float v, d[kNT];
  __host__ __device__ Dn() {}
  __host__ __device__ Dn(double c) : v((float)c) {
#pragma unroll
    for (int k = 0; k < kNT; ++k) d[k] = 0.0f;
  }
};
__device__ __forceinline__ Dn operator+(const Dn& a, const Dn& b) {
  Dn r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < kNT; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
__device__ __forceinline__ Dn operator-(const Dn& a, const Dn& b) {
  Dn r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < kNT; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
__device__ __forceinline__ Dn operator*(const Dn& a, const Dn& b) {
  Dn r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < kNT; ++k) r.d[k] = fmaf(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
__device__ __forceinline__ Dn operator*(const Dn& a, float c) {
  Dn r;
  r.v = a.v * c;
#pragma unroll
  for (int k = 0; k < kNT; ++k) r.d[k] = a.d[k] * c;
  return r;
}
__device__ __forceinline__ Dn operator*(float c, const Dn& a) { return a * c; }
__device__ __forceinline__ Dn& operator+=(Dn& a, const Dn& b) { return a = a + b; }
__device__ __forceinline__ Dn& operator-=(Dn& a, const Dn& b) { return a = a - b; }
// a + b c
__device__ __forceinline__ Dn fma_d(const Dn& b, const Dn& c, const Dn& a) {
  Dn r;
  r.v = fmaf(b.v, c.v, a.v);
#pragma unroll
  for (int k = 0; k < kNT; ++k) r.d[k] = fmaf(b.d[k], c.v, fmaf(b.v, c.d[k], a.d[k]));
  return r;
}
__device__ __forceinline__ Dn fma_c(const Dn& b, float c, const Dn& a) {  // a + b c, c a constant
  Dn r;
  r.v = fmaf(b.v, c, a.v);
#pragma unroll
  for (int k = 0; k < kNT; ++k) r.d[k] = fmaf(b.d[k], c, a.d[k]);
  return r;
}
// f(a) with f(a.v) = fv and f'(a.v) = fd (the chain rule)
__device__ __forceinline__ Dn apply(const Dn& a, float fv, float fd) {
  Dn r;
  r.v = fv;
#pragma unroll
  for (int k = 0; k < kNT; ++k) r.d[k] = fd * a.d[k];
  return r;
}
__device__ __forceinline__ Dn inv_d(const Dn& a) {
  const float iv = 1.0f / a.v;
  return apply(a, iv, -iv * iv);
}
__device__ __forceinline__ Dn sin_d(const Dn& a) { return apply(a, sinf(a.v), cosf(a.v)); }
__device__ __forceinline__ Dn cos_d(const Dn& a) { return apply(a, cosf(a.v), -sinf(a.v)); }
// the logistic sigmoid s = 1 / (1 + exp(-x)), s' = s (1 - s)
__device__ __forceinline__ Dn sigmoid_d(const Dn& a) {
  const float s = 1.0f / (1.0f + expf(-a.v));
  return apply(a, s, s * (1.0f - s));
}
// SiLU x s(x) and its derivative s (1 + x (1 - s)), both as dual expressions
__device__ __forceinline__ Dn silu_d(const Dn& x) { return x * sigmoid_d(x); }
__device__ __forceinline__ Dn silu_grad_d(const Dn& x) {
  const Dn s = sigmoid_d(x);
  return s * (Dn(1.0) + x * (Dn(1.0) - s));
}

// Bessel basis times the polynomial envelope (the layer's radial features) and
// their r-derivatives, as dual expressions of r:
//   e_n = sqrt(2/rc) sin(n pi r/rc) / r u(r/rc),  u(x) = (1-x)^3 sum_{k<p} C(k+2,2) x^k,
//   u'(x) = -p(p+1)(p+2)/2 x^(p-1) (1-x)^2 (the envelope's factored form).
__device__ __forceinline__ void basis_d(const Dn& r, float rc, int p, Dn* e, Dn* de) {
  const Dn x = r * (1.0f / rc);
  const Dn om = Dn(1.0) - x;
  Dn poly = Dn(0.0), xk = Dn(1.0);
  for (int k = 0; k < p; ++k) {
    poly = fma_c(xk, 0.5f * (float)((k + 1) * (k + 2)), poly);
    xk = xk * x;
  }
  Dn xp1 = Dn(1.0);
  for (int k = 0; k < p - 1; ++k) xp1 = xp1 * x;
  const Dn u = om * om * om * poly;
  const Dn du = (-0.5f * (float)(p * (p + 1) * (p + 2)) / rc) * xp1 * om * om;  // du/dr
  const float A = sqrtf(2.0f / rc);
  const Dn ir = inv_d(r);
  const Dn th = r * (3.14159265358979323846f / rc);
  const Dn s1 = sin_d(th), c1 = cos_d(th);
  Dn sn = s1, cn = c1;  // sin(n th), cos(n th) by the angle-addition recurrence
  for (int n = 1; n <= 8; ++n) {
    const Dn f = A * sn * ir;  // sqrt(2/rc) sin(n th) / r
    const Dn df = A * ((3.14159265358979323846f * n / rc) * cn * ir - sn * ir * ir);
    e[n - 1] = f * u;
    de[n - 1] = df * u + f * du;
    const Dn s2 = sn * c1 + cn * s1, c2 = cn * c1 - sn * s1;
    sn = s2;
    cn = c2;
  }
}

// --------------------------------------------------------------- kernels
// V [n][3] of Dn: zero, then e_axis on the row atom of every graph.
__global__ void hz_tangent(int nsys, const int64_t* __restrict__ atom_off, const int* __restrict__ rows, int R,
                           int rho, Dn* __restrict__ V) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsys) return;
  const int64_t a = atom_off[g] + rows[(size_t)g * R + rho];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) V[3 * a + ax].d[ax] = 1.0f;
}

// Per edge: the edge vector (dual), harmonics and the basis with its derivative.
__global__ void hz_edges(int E, const double* __restrict__ pos, const int* __restrict__ recv,
                         const int* __restrict__ send, const int8_t* __restrict__ shift, CellArg cell,
                         const Dn* __restrict__ V, float rc, int p, Dn* __restrict__ ev, Dn* __restrict__ Yd,
                         Dn* __restrict__ eb, Dn* __restrict__ deb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const float4 v = edge_vector(e, pos, recv, send, shift, cell);
  const int i = recv[e], j = send[e];
  Dn x[3];
  const float xv[3] = {v.x, v.y, v.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[a] = Dn(0.0);
    x[a].v = xv[a];
#pragma unroll
    for (int k = 0; k < kNT; ++k) x[a].d[k] = V[3 * j + a].d[k] - V[3 * i + a].d[k];
  }
  Dn r = Dn(0.0);
  r.v = v.w;
#pragma unroll
  for (int k = 0; k < kNT; ++k) r.d[k] = (x[0].v * x[0].d[k] + x[1].v * x[1].d[k] + x[2].v * x[2].d[k]) / v.w;
  const Dn ir = inv_d(r);
  const Dn ux = x[0] * ir, uy = x[1] * ir, uz = x[2] * ir;
  Dn Y[16];
  sh3<Dn>(ux, uy, uz, Y);
  ev[4 * (size_t)e] = x[0];
  ev[4 * (size_t)e + 1] = x[1];
  ev[4 * (size_t)e + 2] = x[2];
  ev[4 * (size_t)e + 3] = r;
#pragma unroll
  for (int k = 0; k < 16; ++k) Yd[16 * (size_t)e + k] = Y[k];
  Dn b[8], db[8];
  basis_d(r, rc, p, b, db);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    eb[8 * (size_t)e + k] = b[k];
    deb[8 * (size_t)e + k] = db[k];
  }
}

// Per edge (one block): z1 = silu(W1^T e), z2 = silu(W2^T z1) (threads < H),
// then w[p][c] = sum_k z2[k] W3[k][p C + c] for the layer's PW paths (thread c).
template <int H>
__global__ void hz_radial(int E, int C, int PW, int PC, const Dn* __restrict__ eb, const float* __restrict__ W1,
                          const float* __restrict__ W2, const float* __restrict__ W3, Dn* __restrict__ w) {
  __shared__ Dn z1[H], z2[H];
  const int e = blockIdx.x, t = threadIdx.x;
  if (t < H) {
    Dn a = Dn(0.0);
#pragma unroll
    for (int n = 0; n < 8; ++n) a = fma_c(eb[8 * (size_t)e + n], W1[n * H + t], a);
    z1[t] = silu_d(a);
  }
  __syncthreads();
  if (t < H) {
    Dn a = Dn(0.0);
    for (int q = 0; q < H; ++q) a = fma_c(z1[q], W2[q * H + t], a);
    z2[t] = silu_d(a);
  }
  __syncthreads();
  for (int c = t; c < C; c += blockDim.x)
    for (int p = 0; p < PW; ++p) {
      Dn a = Dn(0.0);
      for (int k = 0; k < H; ++k) a = fma_c(z2[k], W3[(size_t)k * PC + p * C + c], a);
      w[((size_t)e * PW + p) * C + c] = a;
    }
}

// h^0: the species embedding on the scalars, zero on l > 0 (constants).
__global__ void hz_embed(int n, int C, int D, int S, const int* __restrict__ species, const float* __restrict__ W_emb,
                         Dn* __restrict__ h) {
  const size_t total = (size_t)n * D * C;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(k % C);
    const size_t rest = k / C;
    const int d = (int)(rest % D), i = (int)(rest / D);
    h[k] = Dn(d == 0 ? W_emb[(size_t)clamp_species(species[i], S) * C + c] : 0.0f);
  }
}

// Message of receiver i (one block), channel c (one thread):
//   m[i][l3 m3][c] = s sum_{e: recv = i} sum_p w[e][p][c] sum C^p h[send][l1 m1][c] Y_e[l2 m2].
template <int L, bool FIRST>
__global__ void hz_tp_fwd(int n, int C, const int* __restrict__ row_ptr, const int* __restrict__ send,
                          const Dn* __restrict__ Yd, const Dn* __restrict__ h, const Dn* __restrict__ w, int PW,
                          float s, Dn* __restrict__ m) {
  using Tab = CGTable<L>;
  constexpr int D = NodeDims<L>::D;
  constexpr int NP = FIRST ? PathInfo<L>::P0 : Tab::P;
  const int i = blockIdx.x, c = threadIdx.x;
  if (c >= C) return;
  Dn acc[D];
#pragma unroll
  for (int d = 0; d < D; ++d) acc[d] = Dn(0.0);
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    const int j = send[e];
    const Dn* Y = Yd + 16 * (size_t)e;
    static_for<0, NP>([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      const Dn wp = w[((size_t)e * PW + p) * C + c];
      static_for<Tab::off[p], Tab::off[p + 1]>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int i1 = Tab::e1[k], i2 = Tab::e2[k], i3 = Tab::e3[k];
        constexpr float cv = Tab::ec[k];
        const Dn hv = h[((size_t)j * D + i1) * C + c];
        acc[i3] = fma_d(wp * hv, cv * Y[i2], acc[i3]);
      });
    });
  }
#pragma unroll
  for (int d = 0; d < D; ++d) m[((size_t)i * D + d) * C + c] = acc[d] * s;
}

// Channel mix and update of node i (one block), output channel c2 (thread):
//   u = m[l m] W_l;  h' = h + silu(u) (l = 0), h + u (l > 0); u0 keeps u of l = 0.
template <int L>
__global__ void hz_mix_fwd(int C, const Dn* __restrict__ m, const float* __restrict__ Wmix,
                           const Dn* __restrict__ hin, Dn* __restrict__ hout, Dn* __restrict__ u0) {
  constexpr int D = NodeDims<L>::D;
  extern __shared__ Dn sm_mix[];  // [D][C]
  const int i = blockIdx.x, c2 = threadIdx.x;
  for (int k = threadIdx.x; k < D * C; k += blockDim.x) sm_mix[k] = m[(size_t)i * D * C + k];
  __syncthreads();
  if (c2 >= C) return;
  for (int l = 0; l <= L; ++l) {
    const float* Wl = Wmix + (size_t)l * C * C;
    for (int q = 0; q < 2 * l + 1; ++q) {
      const int d = l * l + q;
      Dn u = Dn(0.0);
      for (int c1 = 0; c1 < C; ++c1) u = fma_c(sm_mix[d * C + c1], Wl[c1 * C + c2], u);
      const size_t o = ((size_t)i * D + d) * C + c2;
      if (l == 0) {
        u0[(size_t)i * C + c2] = u;
        hout[o] = hin[o] + silu_d(u);
      } else {
        hout[o] = hin[o] + u;
      }
    }
  }
}

// Adjoint seed: dE/dh^T[i][0][c] = W_out[z_i][c], zero elsewhere.
__global__ void hz_grad_init(int n, int C, int D, int S, const int* __restrict__ species,
                             const float* __restrict__ W_out, Dn* __restrict__ G) {
  const size_t total = (size_t)n * D * C;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(k % C);
    const size_t rest = k / C;
    const int d = (int)(rest % D), i = (int)(rest / D);
    G[k] = Dn(d == 0 ? W_out[(size_t)clamp_species(species[i], S) * C + c] : 0.0f);
  }
}

// Mix adjoint of node i (block), input channel c1 (thread):
//   Gm[l m][c1] = sum_c2 W_l[c1][c2] G'[l m][c2],  G' = G silu'(u0) (l = 0) or G.
template <int L>
__global__ void hz_mix_bwd(int C, const Dn* __restrict__ G, const Dn* __restrict__ u0,
                           const float* __restrict__ Wmix, Dn* __restrict__ Gm) {
  constexpr int D = NodeDims<L>::D;
  extern __shared__ Dn sm_mix[];  // [D][C]
  const int i = blockIdx.x, c1 = threadIdx.x;
  for (int k = threadIdx.x; k < D * C; k += blockDim.x) {
    Dn g = G[(size_t)i * D * C + k];
    if (k < C) g = g * silu_grad_d(u0[(size_t)i * C + k]);
    sm_mix[k] = g;
  }
  __syncthreads();
  if (c1 >= C) return;
  for (int l = 0; l <= L; ++l) {
    const float* Wl = Wmix + (size_t)l * C * C;
    for (int q = 0; q < 2 * l + 1; ++q) {
      const int d = l * l + q;
      Dn g = Dn(0.0);
      for (int c2 = 0; c2 < C; ++c2) g = fma_c(sm_mix[d * C + c2], Wl[c1 * C + c2], g);
      Gm[((size_t)i * D + d) * C + c1] = g;
    }
  }
}

// Tensor-product adjoint of receiver j (block), channel c (thread), over its
// edges e (sender i):
//   G^{t-1}_j[l1 m1] += s sum_p w[e][p] (-1)^l2 C^p Y_e[l2 m2] Gm_i[l3 m3]    (the reverse edge; not FIRST)
//   T_p[m2] = sum C^p h_i[l1 m1] s Gm_j[l3 m3];  dE/dw_e[p] = sum_m2 Y_e[l2 m2] T_p[m2]
//   dE/dY_e[l2 m2] = sum_c sum_p w[e][p] T_p[m2]   (channel sum through shared memory)
template <int L, bool FIRST>
__global__ void hz_tp_bwd(int C, const int* __restrict__ row_ptr, const int* __restrict__ send,
                          const Dn* __restrict__ Yd, const Dn* __restrict__ hprev, const Dn* __restrict__ Gm,
                          const Dn* __restrict__ w, int PW, float s, const Dn* __restrict__ Gin,
                          Dn* __restrict__ Gout, Dn* __restrict__ dw, Dn* __restrict__ dY) {
  using Tab = CGTable<L>;
  constexpr int D = NodeDims<L>::D;
  constexpr int NP = FIRST ? PathInfo<L>::P0 : Tab::P;
  __shared__ Dn red[128][16];
  const int j = blockIdx.x, c = threadIdx.x;
  const bool active = c < C;
  Dn Gacc[D], Gt[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    Gacc[d] = Dn(0.0);
    Gt[d] = active ? Gm[((size_t)j * D + d) * C + c] * s : Dn(0.0);
  }
  for (int e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
    const int i = send[e];
    const Dn* Y = Yd + 16 * (size_t)e;
    Dn dYp[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) dYp[k] = Dn(0.0);
    if (active) {
      static_for<0, NP>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        constexpr int l2 = Tab::l2[p];
        const Dn wp = w[((size_t)e * PW + p) * C + c];
        Dn Tp[2 * l2 + 1];
#pragma unroll
        for (int q = 0; q < 2 * l2 + 1; ++q) Tp[q] = Dn(0.0);
        static_for<Tab::off[p], Tab::off[p + 1]>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          constexpr float cv = Tab::ec[k];
          constexpr int i1 = Tab::e1[k], i2 = Tab::e2[k], i3 = Tab::e3[k], j2 = i2 - l2 * l2;
          if constexpr (!FIRST) {  // the reverse edge's message into j
            constexpr float sg = (l2 & 1) ? -cv : cv;
            const Dn gi = Gm[((size_t)i * D + i3) * C + c];
            Gacc[i1] = fma_d(wp * gi, (sg * s) * Y[i2], Gacc[i1]);
          }
          const Dn hi = hprev[((size_t)i * D + (FIRST ? 0 : i1)) * C + c];
          Tp[j2] = fma_d(hi * Gt[i3], Dn(cv), Tp[j2]);
        });
        Dn dwp = Dn(0.0);
#pragma unroll
        for (int q = 0; q < 2 * l2 + 1; ++q) {
          dwp = fma_d(Y[l2 * l2 + q], Tp[q], dwp);
          dYp[l2 * l2 + q] = fma_d(wp, Tp[q], dYp[l2 * l2 + q]);
        }
        dw[((size_t)e * PW + p) * C + c] = dwp;
      });
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) red[threadIdx.x][k] = dYp[k];
    __syncthreads();
    if (threadIdx.x < 16) {
      Dn tot = Dn(0.0);
      for (int q = 0; q < (int)blockDim.x; ++q) tot += red[q][threadIdx.x];
      dY[16 * (size_t)e + threadIdx.x] += tot;
    }
    __syncthreads();
  }
  if (!FIRST && active) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const size_t o = ((size_t)j * D + d) * C + c;
      Gout[o] = Gin[o] + Gacc[d];
    }
  }
}

// Radial adjoint of edge e (one block, thread k = hidden unit):
//   dz2[k] = sum_{p,c} W3[k][p C + c] dE/dw[e][p][c];  da2 = dz2 silu'(a2);
//   dz1[q] = sum_k W2[q][k] da2[k];  dE/dr += sum_q dz1[q] silu'(a1[q]) sum_n W1[n][q] de_n/dr.
template <int H>
__global__ void hz_radial_bwd(int C, int PW, int PC, const Dn* __restrict__ eb, const Dn* __restrict__ deb,
                              const float* __restrict__ W1, const float* __restrict__ W2,
                              const float* __restrict__ W3, const Dn* __restrict__ dw, Dn* __restrict__ dr) {
  __shared__ Dn z1[H], a1[H], da2[H], part[H];
  const int e = blockIdx.x, t = threadIdx.x;
  Dn a = Dn(0.0);
  for (int n = 0; n < 8; ++n) a = fma_c(eb[8 * (size_t)e + n], W1[n * H + t], a);
  a1[t] = a;
  z1[t] = silu_d(a);
  __syncthreads();
  Dn a2 = Dn(0.0);
  for (int q = 0; q < H; ++q) a2 = fma_c(z1[q], W2[q * H + t], a2);
  Dn g = Dn(0.0);
  const Dn* dwe = dw + (size_t)e * PW * C;
  for (int pc = 0; pc < PW * C; ++pc) {
    const int p = pc / C, c = pc - p * C;
    g = fma_c(dwe[pc], W3[(size_t)t * PC + p * C + c], g);
  }
  da2[t] = g * silu_grad_d(a2);
  __syncthreads();
  Dn dz1 = Dn(0.0);
  for (int k = 0; k < H; ++k) dz1 = fma_c(da2[k], W2[t * H + k], dz1);
  Dn bd = Dn(0.0);
  for (int n = 0; n < 8; ++n) bd = fma_c(deb[8 * (size_t)e + n], W1[n * H + t], bd);
  part[t] = dz1 * silu_grad_d(a1[t]) * bd;
  __syncthreads();
  if (t == 0) {
    Dn tot = Dn(0.0);
    for (int q = 0; q < H; ++q) tot += part[q];
    dr[e] += tot;
  }
}

// g_e = dE/dx_e: the harmonics' cotangent projected on the sphere, plus dE/dr along x/r.
__global__ void hz_edge_grad(int E, const Dn* __restrict__ ev, const Dn* __restrict__ dY, const Dn* __restrict__ dr,
                             Dn* __restrict__ g) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const Dn ir = inv_d(ev[4 * (size_t)e + 3]);
  const Dn x = ev[4 * (size_t)e] * ir, y = ev[4 * (size_t)e + 1] * ir, z = ev[4 * (size_t)e + 2] * ir;
  Dn d[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) d[k] = dY[16 * (size_t)e + k];
  Dn gx, gy, gz;
  sh3_vjp<Dn>(x, y, z, d, gx, gy, gz);
  const Dn rad = gx * x + gy * y + gz * z;
  const Dn dre = dr[e];
  g[3 * (size_t)e] = (gx - rad * x) * ir + dre * x;
  g[3 * (size_t)e + 1] = (gy - rad * y) * ir + dre * y;
  g[3 * (size_t)e + 2] = (gz - rad * z) * ir + dre * z;
}

// F_i = sum_{e: recv = i} (g_e - g_rev(e)); the rows are minus its tangents:
// rows[a][i][b] = -dF_ib/d(tangent a) (double).
__global__ void hz_rows(int n, const int* __restrict__ row_ptr, const int* __restrict__ rev,
                        const Dn* __restrict__ g, double* __restrict__ rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Dn F[3] = {Dn(0.0), Dn(0.0), Dn(0.0)};
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    const int r = rev[e];
#pragma unroll
    for (int b = 0; b < 3; ++b) F[b] += g[3 * (size_t)e + b] - g[3 * (size_t)r + b];
  }
#pragma unroll
  for (int a = 0; a < kNT; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) rows[((size_t)a * n + i) * 3 + b] = -(double)F[b].d[a];
}

template <int L>
int hessian_pass_l(mlip_model* M, const double* d_pos, const int* d_sp, const SystemBatch& b,
                   const NeighborList& nl, const int64_t* d_off, const int* d_rows, int R, int rho, double* d_out,
                   cudaStream_t st) {
  Workspace& ws = M->ws;
  constexpr int D = NodeDims<L>::D;
  const int n = (int)b.n, C = M->C, T = M->T, P = M->P, P0 = M->P0;
  const int E = (int)nl.E;
  const size_t Ec = (size_t)std::max(E, 1), ND = (size_t)std::max(n, 1) * D * C;
  const float s = (float)(1.0 / M->avg_nb);
  Dn *V = nullptr, *ev = nullptr, *Yd = nullptr, *eb = nullptr, *deb = nullptr, *m = nullptr, *Ga = nullptr,
     *Gb = nullptr, *Gm = nullptr, *dw = nullptr, *dY = nullptr, *dr = nullptr, *g = nullptr;
  MLIP_TRY(ws.get("hz.V", (size_t)3 * std::max(n, 1), &V));
  MLIP_TRY(ws.get("hz.ev", 4 * Ec, &ev));
  MLIP_TRY(ws.get("hz.Y", 16 * Ec, &Yd));
  MLIP_TRY(ws.get("hz.eb", 8 * Ec, &eb));
  MLIP_TRY(ws.get("hz.deb", 8 * Ec, &deb));
  MLIP_TRY(ws.get("hz.m", ND, &m));
  MLIP_TRY(ws.get("hz.Ga", ND, &Ga));
  MLIP_TRY(ws.get("hz.Gb", ND, &Gb));
  MLIP_TRY(ws.get("hz.Gm", ND, &Gm));
  MLIP_TRY(ws.get("hz.dw", Ec * P * C, &dw));
  MLIP_TRY(ws.get("hz.dY", 16 * Ec, &dY));
  MLIP_TRY(ws.get("hz.dr", Ec, &dr));
  MLIP_TRY(ws.get("hz.g", 3 * Ec, &g));
  std::vector<Dn*> h(T + 1), u0(T), w(T);
  for (int t = 0; t <= T; ++t) MLIP_TRY(ws.get("hz.h" + std::to_string(t), ND, &h[t]));
  for (int t = 0; t < T; ++t) {
    MLIP_TRY(ws.get("hz.u" + std::to_string(t), (size_t)std::max(n, 1) * C, &u0[t]));
    MLIP_TRY(ws.get("hz.w" + std::to_string(t), Ec * (t == 0 ? P0 : P) * C, &w[t]));
  }
  const CellArg ca{b.d_cell, b.d_sys_of, b.any_pbc() ? 1 : 0};
  const int threads = ((C + 31) / 32) * 32;
  const size_t mix_smem = (size_t)D * C * sizeof(Dn);
  MLIP_CUDA_TRY(cudaMemsetAsync(V, 0, sizeof(Dn) * 3 * std::max(n, 1), st));
  {
    MLIP_PROF("hz_tangent", st);
    hz_tangent<<<(b.nsys + 127) / 128, 128, 0, st>>>(b.nsys, d_off, d_rows, R, rho, V);
  }
  if (E > 0) {
    MLIP_PROF("hz_edges", st);
    hz_edges<<<(E + 127) / 128, 128, 0, st>>>(E, d_pos, nl.recv, nl.send, nl.shift, ca, V, (float)M->rc, M->p, ev,
                                              Yd, eb, deb);
  }
  {
    MLIP_PROF("hz_embed", st);
    hz_embed<<<std::min<int>((int)((ND + 255) / 256), 4096), 256, 0, st>>>(n, C, D, M->S, d_sp, M->W_emb, h[0]);
  }
  MLIP_LAUNCH_CHECK();
  MLIP_CUDA_TRY(cudaFuncSetAttribute(hz_mix_fwd<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mix_smem));
  MLIP_CUDA_TRY(cudaFuncSetAttribute(hz_mix_bwd<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mix_smem));
  for (int t = 0; t < T; ++t) {
    const int PW = t == 0 ? P0 : P;
    if (E > 0) {
      MLIP_PROF("hz_radial", st);
      hz_radial<64><<<E, 128, 0, st>>>(E, C, PW, P * C, eb, M->W1[t], M->W2[t], M->W3[t], w[t]);
    }
    {
      MLIP_PROF("hz_tp_fwd", st);
      if (t == 0) hz_tp_fwd<L, true><<<n, threads, 0, st>>>(n, C, nl.row_ptr, nl.send, Yd, h[t], w[t], PW, s, m);
      else hz_tp_fwd<L, false><<<n, threads, 0, st>>>(n, C, nl.row_ptr, nl.send, Yd, h[t], w[t], PW, s, m);
    }
    {
      MLIP_PROF("hz_mix_fwd", st);
      hz_mix_fwd<L><<<n, threads, mix_smem, st>>>(C, m, M->Wmix[t], h[t], h[t + 1], u0[t]);
    }
    MLIP_LAUNCH_CHECK();
  }
  {
    MLIP_PROF("hz_grad_init", st);
    hz_grad_init<<<std::min<int>((int)((ND + 255) / 256), 4096), 256, 0, st>>>(n, C, D, M->S, d_sp, M->W_out, Ga);
  }
  MLIP_CUDA_TRY(cudaMemsetAsync(dY, 0, sizeof(Dn) * 16 * Ec, st));
  MLIP_CUDA_TRY(cudaMemsetAsync(dr, 0, sizeof(Dn) * Ec, st));
  for (int t = T - 1; t >= 0; --t) {
    const int PW = t == 0 ? P0 : P;
    {
      MLIP_PROF("hz_mix_bwd", st);
      hz_mix_bwd<L><<<n, threads, mix_smem, st>>>(C, Ga, u0[t], M->Wmix[t], Gm);
    }
    {
      MLIP_PROF("hz_tp_bwd", st);
      if (t == 0)
        hz_tp_bwd<L, true><<<n, threads, 0, st>>>(C, nl.row_ptr, nl.send, Yd, h[t], Gm, w[t], PW, s, Ga, Gb, dw, dY);
      else
        hz_tp_bwd<L, false><<<n, threads, 0, st>>>(C, nl.row_ptr, nl.send, Yd, h[t], Gm, w[t], PW, s, Ga, Gb, dw, dY);
    }
    if (E > 0) {
      MLIP_PROF("hz_radial_bwd", st);
      hz_radial_bwd<64><<<E, 64, 0, st>>>(C, PW, P * C, eb, deb, M->W1[t], M->W2[t], M->W3[t], dw, dr);
    }
    MLIP_LAUNCH_CHECK();
    std::swap(Ga, Gb);
  }
  if (E > 0) {
    MLIP_PROF("hz_edge_grad", st);
    hz_edge_grad<<<(E + 127) / 128, 128, 0, st>>>(E, ev, dY, dr, g);
  }
  {
    MLIP_PROF("hz_rows", st);
    hz_rows<<<(n + 127) / 128, 128, 0, st>>>(n, nl.row_ptr, nl.rev, g, d_out);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace
}  // namespace mlip

extern "C" int mlip_hessian_rows(mlip_model* M, int32_t n_systems, const int64_t* atom_off, const double* pos,
                                 const int32_t* species, const double* cells, const uint8_t* pbc, int32_t R,
                                 const int32_t* row_atoms, double* rows, int on_device, void* stream) {
  using namespace mlip;
  if (!M || !atom_off || !pos || !species || !cells || !pbc || !row_atoms || !rows) {
    set_error("null argument");
    return MLIP_ERR_INVALID_ARG;
  }
  if (n_systems < 1 || n_systems > (1 << 20)) { set_error("system count %d out of range", n_systems); return MLIP_ERR_INVALID_ARG; }
  if (R < 1 || R > 4096) { set_error("row count %d out of range", R); return MLIP_ERR_INVALID_ARG; }
  if (M->corr || M->gate || M->charges || M->parity) {
    set_error("Hessian rows: the GPU path serves the base layer (no symmetric contraction, gate, charges or mixed parity)");
    return MLIP_ERR_INVALID_ARG;
  }
  if (M->H != 64 || (M->L != 2 && M->L != 3) || M->C > 128) {
    set_error("Hessian rows: the GPU path serves hidden width 64, l_max 2 or 3 and at most 128 channels");
    return MLIP_ERR_INVALID_ARG;
  }
  if (atom_off[0] != 0) { set_error("atom_off[0] must be 0"); return MLIP_ERR_INVALID_ARG; }
  for (int g = 0; g < n_systems; ++g) {
    if (atom_off[g + 1] <= atom_off[g]) { set_error("system %d has no atoms (atom_off must increase)", g); return MLIP_ERR_INVALID_ARG; }
    for (int r = 0; r < R; ++r) {
      const int a = row_atoms[(size_t)g * R + r];
      if (a < 0 || a >= atom_off[g + 1] - atom_off[g]) {
        set_error("row atom %d of system %d is outside the system", a, g);
        return MLIP_ERR_INVALID_ARG;
      }
    }
  }
  const int64_t n = atom_off[n_systems];
  if (n > (1 << 24)) { set_error("atom count %lld out of range", (long long)n); return MLIP_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != M->device) { set_error("model lives on device %d, current device is %d", M->device, cur); return MLIP_ERR_INVALID_ARG; }
  Workspace& ws = M->ws;
  WsStream wss(ws, st);
  ++M->eval_gen;
  const double* d_pos = pos;
  const int* d_sp = species;
  double* d_rows = rows;
  if (!on_device) {
    double* dp = nullptr;
    int* dz = nullptr;
    MLIP_TRY(ws.get("in.pos", (size_t)3 * n, &dp));
    MLIP_TRY(ws.get("in.species", (size_t)n, &dz));
    MLIP_TRY(ws.get("hz.rows", (size_t)R * 9 * n, &d_rows));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dp, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(dz, species, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    d_pos = dp;
    d_sp = dz;
  }
  int64_t* d_off = nullptr;
  int* d_rows_idx = nullptr;
  int* flag = nullptr;
  MLIP_TRY(ws.get("hz.off", (size_t)n_systems + 1, &d_off));
  MLIP_TRY(ws.get("hz.rowidx", (size_t)n_systems * R, &d_rows_idx));
  MLIP_TRY(ws.get("chk.flag", 2, &flag));
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_off, atom_off, sizeof(int64_t) * (n_systems + 1), cudaMemcpyHostToDevice, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(d_rows_idx, row_atoms, sizeof(int) * (size_t)n_systems * R, cudaMemcpyHostToDevice, st));
  SystemBatch b;
  b.nsys = n_systems;
  b.atom_off.assign(atom_off, atom_off + n_systems + 1);
  b.cell.assign(cells, cells + 9 * (size_t)n_systems);
  b.pbc.assign(pbc, pbc + 3 * (size_t)n_systems);
  MLIP_TRY(upload_batch(ws, M->stage, b, st));
  MLIP_CUDA_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
  MLIP_TRY(launch_check_inputs((int)n, d_pos, d_sp, M->S, flag, st));
  NeighborList nl;
  MLIP_TRY(build_neighbors_batch(ws, d_pos, b, M->rc, true, st, &nl));
  MLIP_TRY(check_eval_flags(flag, st));
  for (int rho = 0; rho < R; ++rho) {
    double* out = d_rows + (size_t)rho * 9 * n;
    if (M->L == 2) MLIP_TRY(hessian_pass_l<2>(M, d_pos, d_sp, b, nl, d_off, d_rows_idx, R, rho, out, st));
    else MLIP_TRY(hessian_pass_l<3>(M, d_pos, d_sp, b, nl, d_off, d_rows_idx, R, rho, out, st));
  }
  if (!on_device)
    MLIP_CUDA_TRY(cudaMemcpyAsync(rows, d_rows, sizeof(double) * (size_t)R * 9 * n, cudaMemcpyDeviceToHost, st));
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  return MLIP_OK;
}
