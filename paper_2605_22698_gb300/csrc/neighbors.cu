// Cell-list neighbour build on the device (the Graph construction from a
// ChemicalSystem with a distance cutoff, App. A of arxiv 2605.22698; the
// paper's models use graph_cutoff_angstrom = 5 in every hyperparameter table).
//
// Pipeline (all FP64 geometry, integer binning):
//   nl_frac     fractional coordinates s = r h^-1; periodic axes split into an
//               integer image n = floor(s) and a wrapped part f = s - n;
//               extents of open axes reduced into a bounding box
//   nl_setup    one thread: bins per axis (each bin at least rc (1 + 1e-6) wide
//               perpendicular to its faces), search reach, cap on bin count
//   nl_bin      bin of each atom, counts; scan; nl_scatter atoms into bins
//   nl_pairs    one warp per receiver: every candidate (j, S) from the bins
//               within reach, S = q - n_j + n_i, exact test
//                 d2 = (dx*dx + dy*dy) + dz*dz < rc^2 with dx = (x_j - x_i) + sx,
//                 sx = (S0 h00 + S1 h10) + S2 h20, round-to-nearest, no FMA,
//               keys (j, S) appended to a per-receiver slab
//   scan        receiver degrees -> row_ptr
//   nl_sort     one warp per receiver: bitonic sort of its keys in shared
//               memory, compact write of recv / send / shift
//   nl_rev      per edge: binary search of (i, -S) in the sender's segment
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "mlip_internal.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

struct Grid {
  double inv[9];   // s_k = sum_a r_a inv[a][k]
  double h[9];     // rows = lattice vectors (zero for open systems)
  double w[3];     // perpendicular width of the cell per axis (1 for open systems)
  double lo[3], bsz[3];
  int pbc[3], nb[3], reach[3];
  double rc, rc2;
  int max_bins, maxdeg;
  int any_pbc;
  int bin_off;     // first bin of this system in the batch's bin arrays
  // FP32 pre-test of candidate pairs: bv[a] = Cartesian vector of one bin step
  // along axis a; pf = 1 when the coordinates involved are small enough for
  // the pre-test's error bound (nl_setup)
  float bv[9];
  int pf;
};

// Grid of atom i: one per system of a batch (sys_of == nullptr: one system).
__device__ __forceinline__ const Grid* grid_of(const Grid* g, const int* sys_of, int i) {
  return sys_of ? g + sys_of[i] : g;
}

__device__ __forceinline__ long long dbl_order(double x) {
  long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double order_dbl(long long b) {
  return __longlong_as_double(b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL));
}

__global__ void nl_frac(const double* __restrict__ pos, int n, const Grid* __restrict__ grids,
                        const int* __restrict__ sys_of, double* __restrict__ frac, int* __restrict__ img,
                        long long* __restrict__ bbox) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double f[3] = {0, 0, 0};
  bool valid = i < n;
  int sys = 0;
  if (valid) {
    if (sys_of) sys = sys_of[i];
    const Grid* g = grids + sys;
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    for (int k = 0; k < 3; ++k) {
      double s = __dadd_rn(__dadd_rn(__dmul_rn(x, g->inv[k]), __dmul_rn(y, g->inv[3 + k])), __dmul_rn(z, g->inv[6 + k]));
      if (g->pbc[k]) {
        double fl = floor(s);
        img[3 * i + k] = (int)fl;
        f[k] = s - fl;
      } else {
        img[3 * i + k] = 0;
        f[k] = s;
      }
      frac[3 * i + k] = f[k];
    }
  }
  // bounding box of open axes, per system: one atomic per warp when the
  // warp's atoms all belong to one system, else one per atom
  const int s0 = __shfl_sync(0xffffffffu, sys, 0);
  const bool uniform = __all_sync(0xffffffffu, !valid || sys == s0);
  for (int k = 0; k < 3; ++k) {
    long long mn = valid ? dbl_order(f[k]) : LLONG_MAX;
    long long mx = valid ? dbl_order(f[k]) : LLONG_MIN;
    if (uniform) {
      for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      if ((threadIdx.x & 31) == 0) {
        atomicMin(&bbox[6 * s0 + 2 * k], mn);
        atomicMax(&bbox[6 * s0 + 2 * k + 1], mx);
      }
    } else if (valid) {
      atomicMin(&bbox[6 * sys + 2 * k], mn);
      atomicMax(&bbox[6 * sys + 2 * k + 1], mx);
    }
  }
}

// One thread per system.
__global__ void nl_setup(Grid* grids, int nsys, const long long* bbox_all) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= nsys) return;
  Grid* g = grids + sys;
  const long long* bbox = bbox_all + 6 * sys;
  const double margin = 1.0 + 1e-6;
  double ext[3];
  for (int k = 0; k < 3; ++k) {
    if (g->pbc[k]) {
      g->lo[k] = 0.0;
      ext[k] = 1.0;
    } else {
      double lo = order_dbl(bbox[2 * k]), hi = order_dbl(bbox[2 * k + 1]);
      g->lo[k] = lo;
      ext[k] = fmax(hi - lo, 1e-9);
    }
    double minsz = g->rc * margin / g->w[k];
    double nbd = floor(ext[k] / minsz);
    nbd = fmin(fmax(nbd, 1.0), 1048576.0);
    g->nb[k] = (int)nbd;
  }
  // cap the bin count (keeps the bin arrays bounded); coarser bins stay correct
  while ((long long)g->nb[0] * g->nb[1] * g->nb[2] > g->max_bins) {
    int k = 0;
    if (g->nb[1] > g->nb[k]) k = 1;
    if (g->nb[2] > g->nb[k]) k = 2;
    g->nb[k] = max(1, g->nb[k] / 2);
  }
  for (int k = 0; k < 3; ++k) {
    g->bsz[k] = ext[k] / g->nb[k];
    double span = g->bsz[k] * g->w[k];  // perpendicular width of one bin
    // clamp in floating point before converting (a flat open axis has a tiny span)
    const double rd = fmin(floor(g->rc / span * margin) + 1.0, 1048576.0);
    int r = (int)rd;
    if (!g->pbc[k]) r = min(r, g->nb[k]);
    g->reach[k] = r;
  }
  // bin step vectors; the pre-test is used while every coordinate it touches
  // (local offsets within a bin, bin-to-bin shifts within reach) is below 2000 A
  double span_all = 0.0;
  for (int a = 0; a < 3; ++a) {
    double len2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double v = g->bsz[a] * (g->any_pbc ? g->h[3 * a + k] : (a == k ? 1.0 : 0.0));
      g->bv[3 * a + k] = (float)v;
      len2 += v * v;
    }
    span_all += (g->reach[a] + 1.0) * sqrt(len2);
  }
  g->pf = span_all < 2000.0 && g->rc < 100.0 ? 1 : 0;
}

__device__ __forceinline__ void bin_coords(const Grid* g, const double* f, int* b) {
  for (int k = 0; k < 3; ++k) {
    double t = floor((f[k] - g->lo[k]) / g->bsz[k]);
    int bi = (int)fmin(fmax(t, 0.0), (double)(g->nb[k] - 1));
    b[k] = bi;
  }
}

// Bin of every atom, and its position relative to the bin's corner (in the
// atom's own periodic image) rounded to FP32 for the pre-test of nl_pairs_warp.
__global__ void nl_bin(int n, const Grid* __restrict__ grids, const int* __restrict__ sys_of,
                       const double* __restrict__ pos, const double* __restrict__ frac, const int* __restrict__ img,
                       int* __restrict__ bin_of, int* __restrict__ counts, float4* __restrict__ loc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Grid* g = grid_of(grids, sys_of, i);
  double f[3] = {frac[3 * i], frac[3 * i + 1], frac[3 * i + 2]};
  int b[3];
  bin_coords(g, f, b);
  int bin = g->bin_off + (b[0] * g->nb[1] + b[1]) * g->nb[2] + b[2];
  bin_of[i] = bin;
  atomicAdd(&counts[bin], 1);
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = g->lo[a] + b[a] * g->bsz[a] + img[3 * i + a];
  double x[3];
  for (int k = 0; k < 3; ++k) {
    const double corner = g->any_pbc ? (u[0] * g->h[k] + u[1] * g->h[3 + k]) + u[2] * g->h[6 + k] : u[k];
    x[k] = pos[3 * i + k] - corner;
  }
  loc[i] = make_float4((float)x[0], (float)x[1], (float)x[2], 0.0f);
}

__global__ void nl_scatter(int n, const int* __restrict__ bin_of, const int* __restrict__ bin_start,
                           int* __restrict__ cursor, int* __restrict__ bin_atoms) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = bin_of[i];
  int slot = atomicAdd(&cursor[b], 1);
  bin_atoms[bin_start[b] + slot] = i;
}

__device__ __forceinline__ unsigned long long make_key(int j, int s0, int s1, int s2) {
  return ((unsigned long long)(unsigned)j << 24) | ((unsigned long long)(s0 + 128) << 16) |
         ((unsigned long long)(s1 + 128) << 8) | (unsigned long long)(s2 + 128);
}

// flags[0]: max degree seen; flags[1]: |S| > 127 seen
// One warp per receiver: the candidate bins within reach are taken 32 at a
// time, their atom counts prefix-summed across the lanes, and the flattened
// candidate list walked by all lanes at once (each lane finds its bin by a
// binary search over the prefix with shuffles).  Matches are compacted with a
// ballot into the receiver's slab (order irrelevant: nl_sort orders them).
// Candidates are pre-tested in FP32 from the atoms' offsets within their bins
// plus the bin-to-bin shift (|error| far below the slack of the test's
// threshold, rc^2 * 1.02 + 0.01); only the survivors take the exact FP64 test,
// which alone decides (the FP64 pipe is narrow on this part).
__global__ void nl_pairs_warp(int n, const Grid* __restrict__ grids, const int* __restrict__ sys_of,
                              const double* __restrict__ pos,
                              const double* __restrict__ frac, const int* __restrict__ img,
                              const float4* __restrict__ loc,
                              const int* __restrict__ bin_start, const int* __restrict__ bin_atoms,
                              unsigned long long* __restrict__ slab, int* __restrict__ deg, int* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const Grid* g = grid_of(grids, sys_of, i);
  const int maxdeg = g->maxdeg;
  double f[3] = {frac[3 * i], frac[3 * i + 1], frac[3 * i + 2]};
  int b[3];
  bin_coords(g, f, b);
  const int ni0 = img[3 * i], ni1 = img[3 * i + 1], ni2 = img[3 * i + 2];
  const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
  const double* h = g->h;
  const double rc2 = g->rc2;
  const bool pf = g->pf != 0;
  const float thr = (float)rc2 * 1.02f + 0.01f;
  const float4 li = loc[i];
  const int r0 = g->reach[0], r1 = g->reach[1], r2 = g->reach[2];
  const int w0 = 2 * r0 + 1, w1 = 2 * r1 + 1, w2 = 2 * r2 + 1;
  const int nbins = w0 * w1 * w2;
  int cnt = 0;
  bool bad_shift = false;
  for (int base = 0; base < nbins; base += 32) {
    // this lane's bin
    const int bidx = base + lane;
    int beg = 0, len = 0, q0 = 0, q1 = 0, q2 = 0;
    float tx = 0.0f, ty = 0.0f, tz = 0.0f;  // bin shift minus the receiver's offset
    if (bidx < nbins) {
      const int d2 = bidx % w2 - r2, d1 = (bidx / w2) % w1 - r1, d0 = bidx / (w2 * w1) - r0;
      tx = ((float)d0 * g->bv[0] + (float)d1 * g->bv[3] + (float)d2 * g->bv[6]) - li.x;
      ty = ((float)d0 * g->bv[1] + (float)d1 * g->bv[4] + (float)d2 * g->bv[7]) - li.y;
      tz = ((float)d0 * g->bv[2] + (float)d1 * g->bv[5] + (float)d2 * g->bv[8]) - li.z;
      int c0 = b[0] + d0, c1 = b[1] + d1, c2 = b[2] + d2;
      bool ok = true;
      if (g->pbc[0]) { q0 = (int)floor((double)c0 / g->nb[0]); c0 -= q0 * g->nb[0]; } else ok = ok && c0 >= 0 && c0 < g->nb[0];
      if (g->pbc[1]) { q1 = (int)floor((double)c1 / g->nb[1]); c1 -= q1 * g->nb[1]; } else ok = ok && c1 >= 0 && c1 < g->nb[1];
      if (g->pbc[2]) { q2 = (int)floor((double)c2 / g->nb[2]); c2 -= q2 * g->nb[2]; } else ok = ok && c2 >= 0 && c2 < g->nb[2];
      if (ok) {
        const int bin = g->bin_off + (c0 * g->nb[1] + c1) * g->nb[2] + c2;
        beg = bin_start[bin];
        len = bin_start[bin + 1] - beg;
      }
    }
    int incl = len;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int fb = 0; fb < total; fb += 32) {
      const int fidx = fb + lane;
      const bool act = fidx < total;
      // smallest k with incl[k] > fidx
      int lo = 0, hi = 31;
#pragma unroll
      for (int step = 0; step < 5; ++step) {
        const int mid = (lo + hi) >> 1;
        const int v = __shfl_sync(0xffffffffu, incl, mid);
        if (v > fidx) hi = mid; else lo = mid + 1;
      }
      const int k = lo;
      const int kbeg = __shfl_sync(0xffffffffu, beg, k);
      const int klen = __shfl_sync(0xffffffffu, len, k);
      const int kinc = __shfl_sync(0xffffffffu, incl, k);
      const int kq0 = __shfl_sync(0xffffffffu, q0, k), kq1 = __shfl_sync(0xffffffffu, q1, k),
                kq2 = __shfl_sync(0xffffffffu, q2, k);
      const float ktx = __shfl_sync(0xffffffffu, tx, k), kty = __shfl_sync(0xffffffffu, ty, k),
                  ktz = __shfl_sync(0xffffffffu, tz, k);
      bool hit = false;
      unsigned long long key = 0;
      int j = 0;
      if (act) {
        j = bin_atoms[kbeg + fidx - (kinc - klen)];
        if (pf) {
          const float4 lj = loc[j];
          const float ex = lj.x + ktx, ey = lj.y + kty, ez = lj.z + ktz;
          if (ex * ex + ey * ey + ez * ez > thr) j = -1;  // certainly beyond rc
        }
      }
      if (act && j >= 0) {
        const int S0 = kq0 - img[3 * j] + ni0;
        const int S1 = kq1 - img[3 * j + 1] + ni1;
        const int S2 = kq2 - img[3 * j + 2] + ni2;
        if (!(j == i && S0 == 0 && S1 == 0 && S2 == 0)) {
          double sx = 0.0, sy = 0.0, sz = 0.0;
          if (g->any_pbc) {
            sx = __dadd_rn(__dadd_rn(__dmul_rn((double)S0, h[0]), __dmul_rn((double)S1, h[3])), __dmul_rn((double)S2, h[6]));
            sy = __dadd_rn(__dadd_rn(__dmul_rn((double)S0, h[1]), __dmul_rn((double)S1, h[4])), __dmul_rn((double)S2, h[7]));
            sz = __dadd_rn(__dadd_rn(__dmul_rn((double)S0, h[2]), __dmul_rn((double)S1, h[5])), __dmul_rn((double)S2, h[8]));
          }
          const double dx = __dadd_rn(__dsub_rn(pos[3 * j], xi), sx);
          const double dy = __dadd_rn(__dsub_rn(pos[3 * j + 1], yi), sy);
          const double dz = __dadd_rn(__dsub_rn(pos[3 * j + 2], zi), sz);
          const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
          if (d2 < rc2) {
            hit = true;
            if (S0 < -127 || S0 > 127 || S1 < -127 || S1 > 127 || S2 < -127 || S2 > 127) bad_shift = true;
            key = make_key(j, S0, S1, S2);
          }
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int slot = cnt + __popc(mask & ((1u << lane) - 1u));
        if (slot < maxdeg) slab[(size_t)i * maxdeg + slot] = key;
      }
      cnt += __popc(mask);
    }
  }
  if (lane == 0) {
    deg[i] = min(cnt, maxdeg);  // the slab holds maxdeg; a larger count is flagged and the build redone
    if (cnt > maxdeg) atomicMax(&flags[0], cnt);
  }
  if (__any_sync(0xffffffffu, bad_shift) && lane == 0) atomicOr(&flags[1], 1);
}

// One warp per receiver; dynamic shared memory: warps_per_block * cap keys.
// Edges beyond the output capacity Ecap are not written; flags[3] records it.
__global__ void nl_sort(int n, int cap, const unsigned long long* __restrict__ slab, int maxdeg,
                        const int* __restrict__ row_ptr, unsigned long long* __restrict__ keys,
                        int* __restrict__ recv, int* __restrict__ send, int8_t* __restrict__ shift,
                        long long Ecap, int* __restrict__ flags) {
  extern __shared__ unsigned long long sk[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int i = blockIdx.x * (blockDim.x >> 5) + wib;
  if (i >= n) return;
  if ((long long)row_ptr[i + 1] > Ecap) {  // uniform over the warp
    if (lane == 0) atomicOr(&flags[3], 1);
    return;
  }
  unsigned long long* s = sk + (size_t)wib * cap;
  const int beg = row_ptr[i], d = row_ptr[i + 1] - beg;
  int m = 1;
  while (m < d) m <<= 1;
  for (int t = lane; t < m; t += 32) s[t] = t < d ? slab[(size_t)i * maxdeg + t] : ~0ULL;
  __syncwarp();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < m; t += 32) {
        int ixj = t ^ j;
        if (ixj > t) {
          unsigned long long a = s[t], b = s[ixj];
          bool up = (t & k) == 0;
          if ((a > b) == up) { s[t] = b; s[ixj] = a; }
        }
      }
      __syncwarp();
    }
  }
  for (int t = lane; t < d; t += 32) {
    unsigned long long key = s[t];
    keys[beg + t] = key;
    recv[beg + t] = i;
    send[beg + t] = (int)(key >> 24);
    shift[3 * (beg + t) + 0] = (int8_t)((int)((key >> 16) & 0xFF) - 128);
    shift[3 * (beg + t) + 1] = (int8_t)((int)((key >> 8) & 0xFF) - 128);
    shift[3 * (beg + t) + 2] = (int8_t)((int)(key & 0xFF) - 128);
  }
}

__global__ void nl_rev(const int* __restrict__ E_ptr, const int* __restrict__ row_ptr,
                       const int* __restrict__ recv, const int* __restrict__ send,
                       const int8_t* __restrict__ shift, const unsigned long long* __restrict__ keys,
                       int* __restrict__ rev, int* __restrict__ flags) {
  const int E = *E_ptr;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const int i = recv[e], j = send[e];
    const unsigned long long want = make_key(i, -shift[3 * e], -shift[3 * e + 1], -shift[3 * e + 2]);
    int lo = row_ptr[j], hi = row_ptr[j + 1];
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (keys[mid] < want) lo = mid + 1; else hi = mid;
    }
    if (lo < row_ptr[j + 1] && keys[lo] == want) rev[e] = lo;
    else { rev[e] = e; atomicOr(&flags[2], 1); }
  }
}

// One block: if the edge count exceeds the capacity, flag it (flags[3]) and
// empty the list (every row_ptr entry 0), so that no later kernel indexes
// beyond the capacity; the host sees the flag and builds again with room.
__global__ void nl_cap_guard(int n, int* __restrict__ row_ptr, long long Ecap, int* __restrict__ flags) {
  __shared__ int over;
  if (threadIdx.x == 0) {
    over = (long long)row_ptr[n] > Ecap ? 1 : 0;
    if (over) atomicOr(&flags[3], 1);
  }
  __syncthreads();
  if (!over) return;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) row_ptr[i] = 0;
}

// ------------------------------------------------------------ scan
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__device__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    int s = lane < nw ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  int off = w ? warp_sums[w - 1] : 0;
  int res = off + x - v;
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return res;
}

__global__ void scan_local(const int* __restrict__ in, int* __restrict__ out, long long n, int* __restrict__ bsum) {
  __shared__ int ws[32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int v[kScanItems], s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int tot;
  int ex = block_exclusive_scan(s, ws, &tot);
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void scan_blocks(int* __restrict__ bsum, int nb, int* __restrict__ total_out) {
  __shared__ int ws[32];
  int carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < nb ? bsum[i] : 0;
    int tot;
    int ex = block_exclusive_scan(v, ws, &tot);
    if (i < nb) bsum[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void scan_add(int* __restrict__ out, long long n, const int* __restrict__ bsum) {
  const long long base = (long long)blockIdx.x * kScanTile;
  const int add = bsum[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x)
    if (base + k < n) out[base + k] += add;
}

}  // namespace

int exclusive_scan_i32(Workspace& ws, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st,
                       const char* scratch) {
  int nb = (int)((n + kScanTile - 1) / kScanTile);
  if (nb < 1) nb = 1;
  int* bsum = nullptr;
  MLIP_TRY(ws.get(scratch, (size_t)nb, &bsum));
  { MLIP_PROF("scan_local", st); scan_local<<<nb, kScanThreads, 0, st>>>(in, out, n, bsum); }
  { MLIP_PROF("scan_blocks", st); scan_blocks<<<1, 1024, 0, st>>>(bsum, nb, out + n); }
  { MLIP_PROF("scan_add", st); scan_add<<<nb, kScanThreads, 0, st>>>(out, n, bsum); }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

static bool invert3(const double* h, double* inv, double* det_out) {
  double det = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
               h[2] * (h[3] * h[7] - h[4] * h[6]);
  *det_out = det;
  if (!(std::fabs(det) > 1e-12)) return false;
  double id = 1.0 / det;
  inv[0] = (h[4] * h[8] - h[5] * h[7]) * id;
  inv[1] = (h[2] * h[7] - h[1] * h[8]) * id;
  inv[2] = (h[1] * h[5] - h[2] * h[4]) * id;
  inv[3] = (h[5] * h[6] - h[3] * h[8]) * id;
  inv[4] = (h[0] * h[8] - h[2] * h[6]) * id;
  inv[5] = (h[2] * h[3] - h[0] * h[5]) * id;
  inv[6] = (h[3] * h[7] - h[4] * h[6]) * id;
  inv[7] = (h[1] * h[6] - h[0] * h[7]) * id;
  inv[8] = (h[0] * h[4] - h[1] * h[3]) * id;
  return true;
}

// Cell geometry of one system: inverse, lattice rows, perpendicular widths.
static int make_grid(const double* cell, const uint8_t* pbc, double rc, int64_t n_atoms, Grid* hg) {
  *hg = Grid{};
  hg->any_pbc = (pbc[0] || pbc[1] || pbc[2]) ? 1 : 0;
  if (hg->any_pbc) {
    double det;
    if (!invert3(cell, hg->inv, &det)) { set_error("neighbors: singular cell with a periodic axis"); return MLIP_ERR_CELL; }
    for (int k = 0; k < 9; ++k) hg->h[k] = cell[k];
    for (int k = 0; k < 3; ++k) {
      // width = 1 / |column k of h^-1|
      double c2 = hg->inv[k] * hg->inv[k] + hg->inv[3 + k] * hg->inv[3 + k] + hg->inv[6 + k] * hg->inv[6 + k];
      hg->w[k] = 1.0 / std::sqrt(c2);
      hg->pbc[k] = pbc[k] ? 1 : 0;
    }
  } else {
    for (int k = 0; k < 9; ++k) { hg->inv[k] = (k % 4 == 0) ? 1.0 : 0.0; hg->h[k] = 0.0; }
    for (int k = 0; k < 3; ++k) { hg->w[k] = 1.0; hg->pbc[k] = 0; }
  }
  hg->rc = rc;
  hg->rc2 = rc * rc;
  hg->max_bins = (int)std::min<int64_t>(std::max<int64_t>(64, 4 * n_atoms), 1 << 24);
  return MLIP_OK;
}

int build_neighbors(Workspace& ws, const double* d_pos, int64_t n64, const double* cell,
                    const uint8_t* pbc, double rc, bool want_rev, cudaStream_t st, NeighborList* out) {
  SystemBatch b;
  single_system(b, n64, cell, pbc);
  b.d_sys_of = nullptr;  // one system: no per-atom table needed
  return build_neighbors_batch(ws, d_pos, b, rc, want_rev, st, out);
}

int build_neighbors_batch(Workspace& ws, const double* d_pos, const SystemBatch& b, double rc, bool want_rev,
                          cudaStream_t st, NeighborList* out) {
  const int64_t n64 = b.n;
  if (n64 < 0 || n64 > (1LL << 30)) { set_error("neighbors: bad atom count %lld", (long long)n64); return MLIP_ERR_INVALID_ARG; }
  if (!(rc > 0)) { set_error("neighbors: cutoff must be positive"); return MLIP_ERR_INVALID_ARG; }
  if (b.nsys < 1) { set_error("neighbors: empty batch"); return MLIP_ERR_INVALID_ARG; }
  if (b.nsys > 1 && !b.d_sys_of && n64 > 0) { set_error("neighbors: batch not uploaded"); return MLIP_ERR_INVALID_ARG; }
  const int n = (int)n64, nsys = b.nsys;
  out->n = n;
  std::vector<Grid> hg(nsys);
  int64_t total_bins = 0;
  for (int s = 0; s < nsys; ++s) {
    MLIP_TRY(make_grid(&b.cell[9 * s], &b.pbc[3 * s], rc, b.atom_off[s + 1] - b.atom_off[s], &hg[s]));
    hg[s].bin_off = (int)total_bins;
    total_bins += hg[s].max_bins;
  }
  if (total_bins > (1LL << 30)) { set_error("neighbors: batch too large (%lld bins)", (long long)total_bins); return MLIP_ERR_INVALID_ARG; }
  const int nbins = (int)total_bins;

  Grid* dg = nullptr;
  double* frac = nullptr;
  int *img = nullptr, *bin_of = nullptr, *counts = nullptr, *bin_start = nullptr, *cursor = nullptr,
      *bin_atoms = nullptr, *deg = nullptr, *flags = nullptr;
  long long* bbox = nullptr;
  const int nn = std::max(n, 1);
  MLIP_TRY(ws.get("nl.grid", (size_t)nsys, &dg));
  MLIP_TRY(ws.get("nl.frac", (size_t)3 * nn, &frac));
  MLIP_TRY(ws.get("nl.img", (size_t)3 * nn, &img));
  MLIP_TRY(ws.get("nl.bin_of", (size_t)nn, &bin_of));
  MLIP_TRY(ws.get("nl.counts", (size_t)nbins + 1, &counts));
  MLIP_TRY(ws.get("nl.bin_start", (size_t)nbins + 1, &bin_start));
  MLIP_TRY(ws.get("nl.cursor", (size_t)nbins + 1, &cursor));
  MLIP_TRY(ws.get("nl.bin_atoms", (size_t)nn, &bin_atoms));
  MLIP_TRY(ws.get("nl.deg", (size_t)nn, &deg));
  MLIP_TRY(ws.get("nl.flags", 4, &flags));
  MLIP_TRY(ws.get("nl.bbox", (size_t)6 * nsys, &bbox));
  float4* loc = nullptr;
  MLIP_TRY(ws.get("nl.loc", (size_t)nn, &loc));
  MLIP_TRY(ws.get("nl.row_ptr", (size_t)nn + 1, &out->row_ptr));
  std::vector<long long> bb_init(6 * (size_t)nsys);
  for (int s = 0; s < nsys; ++s)
    for (int k = 0; k < 3; ++k) {
      bb_init[6 * s + 2 * k] = LLONG_MAX;
      bb_init[6 * s + 2 * k + 1] = LLONG_MIN;
    }

  int maxdeg = 256;
  const int threads = 128;
  const int blocks = (n + threads - 1) / threads;
  for (int attempt = 0; attempt < 6; ++attempt) {
    for (auto& g : hg) g.maxdeg = maxdeg;
    MLIP_CUDA_TRY(cudaMemcpyAsync(dg, hg.data(), sizeof(Grid) * nsys, cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(bbox, bb_init.data(), sizeof(long long) * bb_init.size(), cudaMemcpyHostToDevice, st));
    MLIP_CUDA_TRY(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
    MLIP_CUDA_TRY(cudaMemsetAsync(counts, 0, ((size_t)nbins + 1) * sizeof(int), st));
    MLIP_CUDA_TRY(cudaMemsetAsync(cursor, 0, ((size_t)nbins + 1) * sizeof(int), st));
    if (n > 0) { MLIP_PROF("nl_frac", st); nl_frac<<<blocks, threads, 0, st>>>(d_pos, n, dg, b.d_sys_of, frac, img, bbox); }
    { MLIP_PROF("nl_setup", st); nl_setup<<<(nsys + 127) / 128, 128, 0, st>>>(dg, nsys, bbox); }
    if (n > 0) { MLIP_PROF("nl_bin", st); nl_bin<<<blocks, threads, 0, st>>>(n, dg, b.d_sys_of, d_pos, frac, img, bin_of, counts, loc); }
    MLIP_LAUNCH_CHECK();
    MLIP_TRY(exclusive_scan_i32(ws, counts, bin_start, nbins, st));
    unsigned long long* slab = nullptr;
    MLIP_TRY(ws.get("nl.slab", (size_t)nn * maxdeg, &slab));
    if (n > 0) {
      { MLIP_PROF("nl_scatter", st); nl_scatter<<<blocks, threads, 0, st>>>(n, bin_of, bin_start, cursor, bin_atoms); }
      { MLIP_PROF("nl_pairs", st); nl_pairs_warp<<<(n + 3) / 4, 128, 0, st>>>(n, dg, b.d_sys_of, d_pos, frac, img, loc, bin_start, bin_atoms, slab, deg, flags); }
      MLIP_LAUNCH_CHECK();
    }
    MLIP_TRY(exclusive_scan_i32(ws, deg, out->row_ptr, n, st));
    int hflags[4];
    int E32 = 0;
    MLIP_CUDA_TRY(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(&E32, out->row_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
    MLIP_CUDA_TRY(cudaStreamSynchronize(st));
    if (hflags[1]) { set_error("neighbors: image index beyond +-127"); return MLIP_ERR_INVALID_ARG; }
    if (hflags[0] > maxdeg) {
      if (hflags[0] > kMaxDegreeLimit) {
        set_error("neighbors: a receiver has %d neighbours (limit %d)", hflags[0], kMaxDegreeLimit);
        return MLIP_ERR_INVALID_ARG;
      }
      while (maxdeg < hflags[0]) maxdeg *= 2;
      continue;
    }
    out->E = E32;
    out->maxdeg = maxdeg;
    const size_t Ecap = (size_t)std::max(E32, 1);
    MLIP_TRY(ws.get("nl.keys", Ecap, &out->keys));
    MLIP_TRY(ws.get("nl.recv", Ecap, &out->recv));
    MLIP_TRY(ws.get("nl.send", Ecap, &out->send));
    MLIP_TRY(ws.get("nl.shift", 3 * Ecap, &out->shift));
    if (n > 0) {
      int cap = 32;
      while (cap < maxdeg) cap <<= 1;
      const int wpb = 4;
      size_t smem = (size_t)wpb * cap * sizeof(unsigned long long);
      if (smem > 48 * 1024)
        MLIP_CUDA_TRY(cudaFuncSetAttribute(nl_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      {
        MLIP_PROF("nl_sort", st);
        nl_sort<<<(n + wpb - 1) / wpb, 32 * wpb, smem, st>>>(n, cap, slab, maxdeg, out->row_ptr, out->keys, out->recv,
                                                             out->send, out->shift, (long long)E32, flags);
      }
      MLIP_LAUNCH_CHECK();
    }
    if (want_rev) {
      MLIP_TRY(ws.get("nl.rev", Ecap, &out->rev));
      if (E32 > 0) {
        { MLIP_PROF("nl_rev", st); nl_rev<<<std::min((E32 + 255) / 256, 4096), 256, 0, st>>>(out->row_ptr + n, out->row_ptr, out->recv,
                                                                   out->send, out->shift, out->keys, out->rev, flags); }
        MLIP_LAUNCH_CHECK();
      }
    }
    return MLIP_OK;
  }
  set_error("neighbors: degree capacity retries exhausted");
  return MLIP_ERR_CAPACITY;
}

int nl_plan(Workspace& ws, HostStage& stage, const SystemBatch& b, double rc, int maxdeg, int64_t Ecap,
            cudaStream_t st, NlPlan* plan) {
  if (!(rc > 0) || maxdeg < 1 || maxdeg > kMaxDegreeLimit || Ecap < 1 || Ecap > (int64_t)INT32_MAX - 64) {
    set_error("neighbors: bad plan (cutoff, degree capacity or edge capacity)");
    return MLIP_ERR_INVALID_ARG;
  }
  if (b.nsys < 1 || (b.nsys > 1 && !b.d_sys_of && b.n > 0)) { set_error("neighbors: batch not uploaded"); return MLIP_ERR_INVALID_ARG; }
  const int nsys = b.nsys;
  std::vector<double> sig;
  sig.reserve(4 + 13 * (size_t)nsys);
  sig.push_back(rc);
  sig.push_back(maxdeg);
  sig.push_back((double)nsys);
  for (int s = 0; s <= nsys; ++s) sig.push_back((double)b.atom_off[s]);
  sig.insert(sig.end(), b.cell.begin(), b.cell.end());
  for (uint8_t v : b.pbc) sig.push_back(v);
  void *g0 = nullptr, *bb0 = nullptr;
  const uint64_t gen0 = ws.gen;
  MLIP_TRY(ws.get("nlp.grid0", sizeof(Grid) * nsys, &g0));
  MLIP_TRY(ws.get("nlp.bbox0", sizeof(long long) * 6 * nsys, &bb0));
  const bool same = sig == plan->sig && ws.gen == gen0 && plan->d_grid0 == g0 && plan->d_bbox0 == bb0;
  plan->rc = rc;
  plan->maxdeg = maxdeg;
  plan->nsys = nsys;
  plan->n = b.n;
  plan->Ecap = Ecap;
  plan->d_grid0 = g0;
  plan->d_bbox0 = static_cast<long long*>(bb0);
  if (same) return MLIP_OK;
  std::vector<Grid> hg(nsys);
  int64_t total_bins = 0;
  for (int s = 0; s < nsys; ++s) {
    MLIP_TRY(make_grid(&b.cell[9 * s], &b.pbc[3 * s], rc, b.atom_off[s + 1] - b.atom_off[s], &hg[s]));
    hg[s].bin_off = (int)total_bins;
    hg[s].maxdeg = maxdeg;
    total_bins += hg[s].max_bins;
  }
  if (total_bins > (1LL << 30)) { set_error("neighbors: batch too large (%lld bins)", (long long)total_bins); return MLIP_ERR_INVALID_ARG; }
  plan->nbins = (int)total_bins;
  const size_t gbytes = sizeof(Grid) * nsys, bbytes = sizeof(long long) * 6 * nsys;
  void* hp = nullptr;
  MLIP_TRY(stage.get(gbytes + bbytes, &hp));
  std::memcpy(hp, hg.data(), gbytes);
  long long* hb = reinterpret_cast<long long*>(static_cast<unsigned char*>(hp) + gbytes);
  for (int s = 0; s < nsys; ++s)
    for (int k = 0; k < 3; ++k) {
      hb[6 * s + 2 * k] = LLONG_MAX;
      hb[6 * s + 2 * k + 1] = LLONG_MIN;
    }
  MLIP_CUDA_TRY(cudaMemcpyAsync(g0, hp, gbytes, cudaMemcpyHostToDevice, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(bb0, hb, bbytes, cudaMemcpyHostToDevice, st));
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));  // the staging is reused by the next upload
  plan->sig = sig;
  return MLIP_OK;
}

int build_neighbors_nosync(Workspace& ws, const double* d_pos, const SystemBatch& b, const NlPlan& plan,
                           cudaStream_t st, NeighborList* out, int* flags) {
  const int n = (int)b.n, nsys = b.nsys, nbins = plan.nbins, maxdeg = plan.maxdeg;
  if (n != plan.n || nsys != plan.nsys) { set_error("neighbors: plan made for another batch"); return MLIP_ERR_INVALID_ARG; }
  const int nn = std::max(n, 1);
  const size_t Ecap = (size_t)plan.Ecap;
  Grid* dg = nullptr;
  double* frac = nullptr;
  float4* loc = nullptr;
  int *img = nullptr, *bin_of = nullptr, *counts = nullptr, *bin_start = nullptr, *cursor = nullptr,
      *bin_atoms = nullptr, *deg = nullptr;
  long long* bbox = nullptr;
  unsigned long long* slab = nullptr;
  MLIP_TRY(ws.get("nlg.grid", (size_t)nsys, &dg));
  MLIP_TRY(ws.get("nlg.frac", (size_t)3 * nn, &frac));
  MLIP_TRY(ws.get("nlg.img", (size_t)3 * nn, &img));
  MLIP_TRY(ws.get("nlg.loc", (size_t)nn, &loc));
  MLIP_TRY(ws.get("nlg.bin_of", (size_t)nn, &bin_of));
  MLIP_TRY(ws.get("nlg.counts", (size_t)nbins + 1, &counts));
  MLIP_TRY(ws.get("nlg.bin_start", (size_t)nbins + 1, &bin_start));
  MLIP_TRY(ws.get("nlg.cursor", (size_t)nbins + 1, &cursor));
  MLIP_TRY(ws.get("nlg.bin_atoms", (size_t)nn, &bin_atoms));
  MLIP_TRY(ws.get("nlg.deg", (size_t)nn, &deg));
  MLIP_TRY(ws.get("nlg.bbox", (size_t)6 * nsys, &bbox));
  MLIP_TRY(ws.get("nlg.slab", (size_t)nn * maxdeg, &slab));
  MLIP_TRY(ws.get("nlg.row_ptr", (size_t)nn + 1, &out->row_ptr));
  MLIP_TRY(ws.get("nlg.keys", Ecap, &out->keys));
  MLIP_TRY(ws.get("nlg.recv", Ecap, &out->recv));
  MLIP_TRY(ws.get("nlg.send", Ecap, &out->send));
  MLIP_TRY(ws.get("nlg.shift", 3 * Ecap, &out->shift));
  MLIP_TRY(ws.get("nlg.rev", Ecap, &out->rev));
  out->n = n;
  out->E = (int64_t)Ecap;
  out->maxdeg = maxdeg;
  MLIP_CUDA_TRY(cudaMemcpyAsync(dg, plan.d_grid0, sizeof(Grid) * nsys, cudaMemcpyDeviceToDevice, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(bbox, plan.d_bbox0, sizeof(long long) * 6 * nsys, cudaMemcpyDeviceToDevice, st));
  MLIP_CUDA_TRY(cudaMemsetAsync(counts, 0, ((size_t)nbins + 1) * sizeof(int), st));
  MLIP_CUDA_TRY(cudaMemsetAsync(cursor, 0, ((size_t)nbins + 1) * sizeof(int), st));
  const int threads = 128, blocks = (n + threads - 1) / threads;
  if (n > 0) { MLIP_PROF("nl_frac", st); nl_frac<<<blocks, threads, 0, st>>>(d_pos, n, dg, b.d_sys_of, frac, img, bbox); }
  { MLIP_PROF("nl_setup", st); nl_setup<<<(nsys + 127) / 128, 128, 0, st>>>(dg, nsys, bbox); }
  if (n > 0) {
    MLIP_PROF("nl_bin", st);
    nl_bin<<<blocks, threads, 0, st>>>(n, dg, b.d_sys_of, d_pos, frac, img, bin_of, counts, loc);
  }
  MLIP_LAUNCH_CHECK();
  MLIP_TRY(exclusive_scan_i32(ws, counts, bin_start, nbins, st, "nlg.bsum1"));
  if (n > 0) {
    { MLIP_PROF("nl_scatter", st); nl_scatter<<<blocks, threads, 0, st>>>(n, bin_of, bin_start, cursor, bin_atoms); }
    {
      MLIP_PROF("nl_pairs", st);
      nl_pairs_warp<<<(n + 3) / 4, 128, 0, st>>>(n, dg, b.d_sys_of, d_pos, frac, img, loc, bin_start, bin_atoms, slab,
                                                 deg, flags);
    }
    MLIP_LAUNCH_CHECK();
  }
  MLIP_TRY(exclusive_scan_i32(ws, deg, out->row_ptr, n, st, "nlg.bsum2"));
  { MLIP_PROF("nl_cap_guard", st); nl_cap_guard<<<1, 1024, 0, st>>>(n, out->row_ptr, (long long)Ecap, flags); }
  MLIP_LAUNCH_CHECK();
  if (n > 0) {
    int cap = 32;
    while (cap < maxdeg) cap <<= 1;
    const int wpb = 4;
    const size_t smem = (size_t)wpb * cap * sizeof(unsigned long long);
    if (smem > 48 * 1024)
      MLIP_CUDA_TRY(cudaFuncSetAttribute(nl_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
      MLIP_PROF("nl_sort", st);
      nl_sort<<<(n + wpb - 1) / wpb, 32 * wpb, smem, st>>>(n, cap, slab, maxdeg, out->row_ptr, out->keys, out->recv,
                                                           out->send, out->shift, (long long)Ecap, flags);
    }
    {
      MLIP_PROF("nl_rev", st);
      nl_rev<<<(int)std::min<size_t>((Ecap + 255) / 256, 4096), 256, 0, st>>>(
          out->row_ptr + n, out->row_ptr, out->recv, out->send, out->shift, out->keys, out->rev, flags);
    }
    MLIP_LAUNCH_CHECK();
  }
  return MLIP_OK;
}

}  // namespace mlip

// ------------------------------------------------------------------------
// Allocation-free variant of the neighbour build.
//
// Some callers cannot call cudaMalloc: code that runs while its process holds
// a fixed device-memory budget (a host application that partitions HBM up
// front and forbids later growth), code on a latency-critical path where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable,
// and plug-ins called from inside another framework's memory pool that must
// not allocate behind the pool's back.  mlip_neighbors_noalloc serves them:
// every scratch buffer lives in one file-scope __device__ array of fixed size
// that each GPU loading the library keeps until the process exits, and the
// caller passes the inputs and outputs in device memory.
namespace mlip {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB per device
constexpr int kNoAllocMaxAtoms = 12288;
constexpr int kNoAllocMaxDegree = 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_base[256] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code only sees a host-side stand-in for the symbol).
int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    set_error("neighbors (no-alloc): no current CUDA device");
    return MLIP_ERR_CUDA;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("neighbors (no-alloc): cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return MLIP_ERR_CUDA;
    }
    g_noalloc_base[dev] = p;
  }
  *out = g_noalloc_base[dev];
  return MLIP_OK;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
// Consecutive 256-byte-aligned pieces of the scratch array.  A failed take
// marks the carve failed, and every later take then fails too, so one check of
// `failed` after the last take covers the whole layout.
struct Carve {
  unsigned char* base;
  size_t off, cap;
  bool failed = false;
  static constexpr size_t rounded(size_t bytes) { return (bytes + 255) & ~(size_t)255; }
  template <class T>
  T* take(size_t count) {
    const size_t bytes = rounded(count * sizeof(T));
    if (failed || off + bytes > cap) {
      failed = true;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// Bytes the layout of mlip_neighbors_noalloc takes for nn atoms (the takes in
// the order the entry point makes them); at the limits it must fit the array.
constexpr size_t noalloc_layout_bytes(size_t nn) {
  const size_t bins = (nn * 4 > 64 ? nn * 4 : 64) + 1;
  const size_t scan = ((bins - 1 > nn ? bins - 1 : nn) / kScanTile + 2) * sizeof(int);
  return Carve::rounded(sizeof(Grid)) + Carve::rounded(3 * nn * sizeof(double)) + Carve::rounded(3 * nn * sizeof(int)) +
         Carve::rounded(nn * sizeof(float4)) + Carve::rounded(nn * sizeof(int)) + 3 * Carve::rounded(bins * sizeof(int)) +
         2 * Carve::rounded(nn * sizeof(int)) + Carve::rounded(4 * sizeof(int)) + Carve::rounded(6 * sizeof(long long)) +
         Carve::rounded((nn + 1) * sizeof(int)) + Carve::rounded(scan) +
         Carve::rounded(nn * kNoAllocMaxDegree * sizeof(unsigned long long));
}
static_assert(noalloc_layout_bytes(kNoAllocMaxAtoms) <= kNoAllocScratchBytes,
              "the allocation-free neighbour layout at its atom and degree limits exceeds the scratch array");

// nl_sort without the key output (the caller's edge arrays only).
__global__ void nl_sort_out(int n, int cap, const unsigned long long* __restrict__ slab, int maxdeg,
                            const int* __restrict__ row_ptr, int* __restrict__ recv, int* __restrict__ send,
                            int8_t* __restrict__ shift) {
  extern __shared__ unsigned long long sk[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int i = blockIdx.x * (blockDim.x >> 5) + wib;
  if (i >= n) return;
  unsigned long long* s = sk + (size_t)wib * cap;
  const int beg = row_ptr[i], d = row_ptr[i + 1] - beg;
  int m = 1;
  while (m < d) m <<= 1;
  for (int t = lane; t < m; t += 32) s[t] = t < d ? slab[(size_t)i * maxdeg + t] : ~0ULL;
  __syncwarp();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < m; t += 32) {
        int ixj = t ^ j;
        if (ixj > t) {
          unsigned long long a = s[t], b = s[ixj];
          bool up = (t & k) == 0;
          if ((a > b) == up) { s[t] = b; s[ixj] = a; }
        }
      }
      __syncwarp();
    }
  }
  for (int t = lane; t < d; t += 32) {
    const unsigned long long key = s[t];
    recv[beg + t] = i;
    send[beg + t] = (int)(key >> 24);
    shift[3 * (beg + t) + 0] = (int8_t)((int)((key >> 16) & 0xFF) - 128);
    shift[3 * (beg + t) + 1] = (int8_t)((int)((key >> 8) & 0xFF) - 128);
    shift[3 * (beg + t) + 2] = (int8_t)((int)(key & 0xFF) - 128);
  }
}

int scan_fixed(const int32_t* in, int32_t* out, int64_t n, int* bsum, cudaStream_t st) {
  int nb = (int)((n + kScanTile - 1) / kScanTile);
  if (nb < 1) nb = 1;
  scan_local<<<nb, kScanThreads, 0, st>>>(in, out, n, bsum);
  scan_blocks<<<1, 1024, 0, st>>>(bsum, nb, out + n);
  scan_add<<<nb, kScanThreads, 0, st>>>(out, n, bsum);
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace
}  // namespace mlip

extern "C" int mlip_neighbors_noalloc(const double* pos, int64_t n64, const double cell[9], const uint8_t pbc[3],
                                      double cutoff, int32_t* recv, int32_t* send, int8_t* shift, int64_t capacity,
                                      int64_t* n_edges, void* stream) {
  using namespace mlip;
  if (!n_edges || !cell || !pbc || (n64 > 0 && !pos)) { set_error("null argument"); return MLIP_ERR_INVALID_ARG; }
  *n_edges = 0;
  if (n64 < 0 || n64 > kNoAllocMaxAtoms) {
    set_error("neighbors (no-alloc): %lld atoms; this entry point handles at most %d (use mlip_neighbors)",
              (long long)n64, kNoAllocMaxAtoms);
    return MLIP_ERR_INVALID_ARG;
  }
  if (!(cutoff > 0)) { set_error("neighbors (no-alloc): cutoff must be positive"); return MLIP_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = (int)n64;
  void* base = nullptr;
  MLIP_TRY(noalloc_scratch(&base));

  Grid hg{};
  MLIP_TRY(make_grid(cell, pbc, cutoff, n, &hg));
  hg.max_bins = std::max(64, 4 * n);
  hg.maxdeg = kNoAllocMaxDegree;
  hg.bin_off = 0;

  const size_t nn = (size_t)std::max(n, 1);
  Carve cv{static_cast<unsigned char*>(base), 0, kNoAllocScratchBytes};
  Grid* dg = cv.take<Grid>(1);
  double* frac = cv.take<double>(3 * nn);
  int* img = cv.take<int>(3 * nn);
  float4* loc = cv.take<float4>(nn);
  int* bin_of = cv.take<int>(nn);
  int* counts = cv.take<int>((size_t)hg.max_bins + 1);
  int* bin_start = cv.take<int>((size_t)hg.max_bins + 1);
  int* cursor = cv.take<int>((size_t)hg.max_bins + 1);
  int* bin_atoms = cv.take<int>(nn);
  int* deg = cv.take<int>(nn);
  int* flags = cv.take<int>(4);
  long long* bbox = cv.take<long long>(6);
  int* row_ptr = cv.take<int>(nn + 1);
  int* bsum = cv.take<int>((size_t)std::max<int64_t>(hg.max_bins, nn) / kScanTile + 2);
  unsigned long long* slab = cv.take<unsigned long long>(nn * kNoAllocMaxDegree);
  if (cv.failed || !slab) {
    set_error("neighbors (no-alloc): scratch layout exceeds %zu bytes", kNoAllocScratchBytes);
    return MLIP_ERR_CAPACITY;
  }

  // the array keeps the last call's contents: clear what must start at zero
  const long long bb_init[6] = {LLONG_MAX, LLONG_MIN, LLONG_MAX, LLONG_MIN, LLONG_MAX, LLONG_MIN};
  MLIP_CUDA_TRY(cudaMemcpyAsync(dg, &hg, sizeof(Grid), cudaMemcpyHostToDevice, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(bbox, bb_init, sizeof(bb_init), cudaMemcpyHostToDevice, st));
  MLIP_CUDA_TRY(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
  MLIP_CUDA_TRY(cudaMemsetAsync(counts, 0, ((size_t)hg.max_bins + 1) * sizeof(int), st));
  MLIP_CUDA_TRY(cudaMemsetAsync(cursor, 0, ((size_t)hg.max_bins + 1) * sizeof(int), st));
  const int threads = 128, blocks = (n + threads - 1) / threads;
  if (n > 0) {
    nl_frac<<<blocks, threads, 0, st>>>(pos, n, dg, nullptr, frac, img, bbox);
    nl_setup<<<1, 32, 0, st>>>(dg, 1, bbox);
    nl_bin<<<blocks, threads, 0, st>>>(n, dg, nullptr, pos, frac, img, bin_of, counts, loc);
  } else {
    nl_setup<<<1, 32, 0, st>>>(dg, 1, bbox);
  }
  MLIP_LAUNCH_CHECK();
  MLIP_TRY(scan_fixed(counts, bin_start, hg.max_bins, bsum, st));
  if (n > 0) {
    nl_scatter<<<blocks, threads, 0, st>>>(n, bin_of, bin_start, cursor, bin_atoms);
    nl_pairs_warp<<<(n + 3) / 4, 128, 0, st>>>(n, dg, nullptr, pos, frac, img, loc, bin_start, bin_atoms, slab,
                                               deg, flags);
    MLIP_LAUNCH_CHECK();
  }
  MLIP_TRY(scan_fixed(deg, row_ptr, n, bsum, st));
  int hflags[4] = {0, 0, 0, 0};
  int E32 = 0;
  MLIP_CUDA_TRY(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
  MLIP_CUDA_TRY(cudaMemcpyAsync(&E32, row_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  if (hflags[1]) { set_error("neighbors (no-alloc): image index beyond +-127"); return MLIP_ERR_INVALID_ARG; }
  if (hflags[0] > kNoAllocMaxDegree) {
    set_error("neighbors (no-alloc): a receiver has %d neighbours (this entry point handles at most %d)", hflags[0],
              kNoAllocMaxDegree);
    return MLIP_ERR_CAPACITY;
  }
  *n_edges = E32;
  if (E32 > capacity) {
    set_error("neighbour capacity %lld < %d edges", (long long)capacity, E32);
    return MLIP_ERR_CAPACITY;
  }
  if (n > 0 && E32 > 0) {
    if (!recv || !send || !shift) { set_error("null output buffer"); return MLIP_ERR_INVALID_ARG; }
    const int wpb = 4, cap = kNoAllocMaxDegree;
    const size_t smem = (size_t)wpb * cap * sizeof(unsigned long long);
    nl_sort_out<<<(n + wpb - 1) / wpb, 32 * wpb, smem, st>>>(n, cap, slab, kNoAllocMaxDegree, row_ptr, recv, send,
                                                            shift);
    MLIP_LAUNCH_CHECK();
  }
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  return MLIP_OK;
}
