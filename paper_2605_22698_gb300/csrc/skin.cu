// Skin neighbour list for molecular dynamics.  A candidate list of the pairs
// within rc + skin is built (the ordinary cell-list build at the larger
// cutoff) and kept for a block of steps; every step compacts it to the pairs
// within rc at the current positions, with the same FP64 distance test as the
// build (round-to-nearest, no contraction).  The candidates are in the
// canonical (recv, send, S) order, so the compacted list is in that order too,
// and while no atom has moved more than skin/2 since the build it holds
// exactly the pairs a fresh build would find: |d_now - d_build| <= 2 max|dr|.
// All launch sizes depend on the atom count and the capacity only, so a step
// can be captured in a CUDA graph and replayed after the next build.
#include <algorithm>

#include "mlip_internal.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

// ||r_j - r_i + S^T h||^2 evaluated exactly as the neighbour build does
__device__ __forceinline__ double pair_d2(const double* __restrict__ pos, int i, int j,
                                          const int8_t* __restrict__ S, const double* __restrict__ h, int any_pbc) {
  double s[3] = {0.0, 0.0, 0.0};
  if (any_pbc) {
    const double S0 = S[0], S1 = S[1], S2 = S[2];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      s[k] = __dadd_rn(__dadd_rn(__dmul_rn(S0, h[k]), __dmul_rn(S1, h[3 + k])), __dmul_rn(S2, h[6 + k]));
  }
  const double dx = __dadd_rn(__dsub_rn(pos[3 * j], pos[3 * i]), s[0]);
  const double dy = __dadd_rn(__dsub_rn(pos[3 * j + 1], pos[3 * i + 1]), s[1]);
  const double dz = __dadd_rn(__dsub_rn(pos[3 * j + 2], pos[3 * i + 2]), s[2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

constexpr int kWarpsPerBlock = 4;

// One warp per receiver: keep[e] = (d2 < rc2) over its candidates, deg[i] =
// the kept count; displacement of atom i from its position at the build.
__global__ void skin_mark(int n, const int* __restrict__ crow, const int* __restrict__ csend,
                          const int8_t* __restrict__ cshift, const double* __restrict__ pos,
                          const double* __restrict__ pos_ref, const double* __restrict__ cells,
                          const int* __restrict__ sys_of, int any_pbc, double rc2, double half2,
                          uint8_t* __restrict__ keep, int* __restrict__ deg, int* __restrict__ flags,
                          unsigned long long* __restrict__ dmax2) {
  __shared__ double s_m2[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kWarpsPerBlock + w;
  double m2 = 0.0;
  if (i < n) {
    const double* h = cells + (sys_of ? 9 * sys_of[i] : 0);
    const int beg = crow[i], end = crow[i + 1];
    int cnt = 0;
    for (int e = beg + lane; e < end; e += 32) {
      const bool k = pair_d2(pos, i, csend[e], cshift + 3 * e, h, any_pbc) < rc2;
      keep[e] = k ? 1 : 0;
      cnt += k ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) {
      deg[i] = cnt;
      const double dx = pos[3 * i] - pos_ref[3 * i], dy = pos[3 * i + 1] - pos_ref[3 * i + 1],
                   dz = pos[3 * i + 2] - pos_ref[3 * i + 2];
      m2 = dx * dx + dy * dy + dz * dz;
    }
  }
  if (lane == 0) s_m2[w] = m2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = s_m2[0];
    for (int k = 1; k < kWarpsPerBlock; ++k) m = fmax(m, s_m2[k]);
    if (!(m <= half2)) atomicOr(&flags[0], 1);  // also catches a non-finite position
    if (m > 0.0) atomicMax(dmax2, (unsigned long long)__double_as_longlong(m));  // m >= 0: bit order = value order
  }
}

// One warp per receiver: the kept candidates, in order, to the compacted list;
// newidx[e] = their new index (-1 for dropped candidates).
__global__ void skin_write(int n, const int* __restrict__ crow, const int* __restrict__ csend,
                           const int8_t* __restrict__ cshift, const uint8_t* __restrict__ keep,
                           const int* __restrict__ row_ptr, int* __restrict__ recv, int* __restrict__ send,
                           int8_t* __restrict__ shift, int* __restrict__ newidx) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (i >= n) return;
  const int beg = crow[i], end = crow[i + 1];
  int out = row_ptr[i];
  for (int base = beg; base < end; base += 32) {
    const int e = base + lane;
    const bool k = e < end && keep[e];
    const unsigned m = __ballot_sync(0xffffffffu, k);
    if (e < end) {
      if (k) {
        const int o = out + __popc(m & ((1u << lane) - 1u));
        recv[o] = i;
        send[o] = csend[e];
        shift[3 * o] = cshift[3 * e];
        shift[3 * o + 1] = cshift[3 * e + 1];
        shift[3 * o + 2] = cshift[3 * e + 2];
        newidx[e] = o;
      } else {
        newidx[e] = -1;
      }
    }
    out += __popc(m);
  }
}

// Reverse index of every kept edge.  The distance test is symmetric bit for
// bit (dx of j <- i, -S is exactly -dx), so the reverse of a kept candidate is
// kept; a missing one is flagged.
__global__ void skin_rev(const int* __restrict__ n_cand, const int* __restrict__ crev,
                         const int* __restrict__ newidx, int* __restrict__ rev, int* __restrict__ flags) {
  const int Ec = *n_cand;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ec; e += gridDim.x * blockDim.x) {
    const int o = newidx[e];
    if (o < 0) continue;
    const int r = newidx[crev[e]];
    if (r < 0) {
      atomicOr(&flags[1], 1);
      rev[o] = o;
    } else {
      rev[o] = r;
    }
  }
}

}  // namespace

int skin_build(Workspace& ws, const double* d_pos, const SystemBatch& b, double rc, double skin, SkinList* sl,
               cudaStream_t st) {
  if (!(skin > 0.0) || !(rc > 0.0)) { set_error("skin list: cutoff and skin must be positive"); return MLIP_ERR_INVALID_ARG; }
  NeighborList cand;
  MLIP_TRY(build_neighbors_batch(ws, d_pos, b, rc + skin, true, st, &cand));
  const int64_t n = b.n;
  if (cand.E > sl->cap || n != sl->n) {
    const int64_t want = std::max<int64_t>(cand.E + cand.E / 8 + 1024, sl->cap);
    if (want > (int64_t)INT32_MAX - 64) { set_error("skin list: %lld candidates exceed the index range", (long long)want); return MLIP_ERR_CAPACITY; }
    sl->cap = want;
  }
  sl->n = n;
  sl->rc = rc;
  sl->skin = skin;
  sl->n_cand = cand.E;
  const size_t cap = (size_t)sl->cap, nn = (size_t)std::max<int64_t>(n, 1);
  MLIP_TRY(ws.get("skin.crow", nn + 1, &sl->crow));
  MLIP_TRY(ws.get("skin.crecv", cap, &sl->crecv));
  MLIP_TRY(ws.get("skin.csend", cap, &sl->csend));
  MLIP_TRY(ws.get("skin.crev", cap, &sl->crev));
  MLIP_TRY(ws.get("skin.cshift", 3 * cap, &sl->cshift));
  MLIP_TRY(ws.get("skin.pos_ref", 3 * nn, &sl->pos_ref));
  MLIP_TRY(ws.get("skin.deg", nn, &sl->deg));
  MLIP_TRY(ws.get("skin.newidx", cap, &sl->newidx));
  MLIP_TRY(ws.get("skin.keep", cap, &sl->keep));
  MLIP_TRY(ws.get("skin.row_ptr", nn + 1, &sl->nl.row_ptr));
  MLIP_TRY(ws.get("skin.recv", cap, &sl->nl.recv));
  MLIP_TRY(ws.get("skin.send", cap, &sl->nl.send));
  MLIP_TRY(ws.get("skin.shift", 3 * cap, &sl->nl.shift));
  MLIP_TRY(ws.get("skin.rev", cap, &sl->nl.rev));
  MLIP_TRY(ws.get("skin.flags", 2, &sl->flags));
  MLIP_TRY(ws.get("skin.dmax2", 1, &sl->dmax2));
  sl->nl.n = n;
  sl->nl.E = sl->cap;
  sl->nl.keys = nullptr;
  const size_t E = (size_t)cand.E;
  MLIP_CUDA_TRY(cudaMemcpyAsync(sl->crow, cand.row_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, st));
  if (E > 0) {
    MLIP_CUDA_TRY(cudaMemcpyAsync(sl->crecv, cand.recv, sizeof(int) * E, cudaMemcpyDeviceToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(sl->csend, cand.send, sizeof(int) * E, cudaMemcpyDeviceToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(sl->crev, cand.rev, sizeof(int) * E, cudaMemcpyDeviceToDevice, st));
    MLIP_CUDA_TRY(cudaMemcpyAsync(sl->cshift, cand.shift, 3 * E, cudaMemcpyDeviceToDevice, st));
  }
  MLIP_CUDA_TRY(cudaMemcpyAsync(sl->pos_ref, d_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
  return MLIP_OK;
}

int skin_compact(Workspace& ws, SkinList& sl, const double* d_pos, const SystemBatch& b, cudaStream_t st) {
  const int n = (int)sl.n;
  if (n <= 0) { set_error("skin list: no atoms"); return MLIP_ERR_INVALID_ARG; }
  const double rc2 = sl.rc * sl.rc;
  // an atom may move at most skin/2 (less a margin for the rounding of the distances)
  const double half = 0.5 * sl.skin - 1e-9, half2 = half * half;
  const int blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  {
    MLIP_PROF("skin_mark", st);
    skin_mark<<<blocks, 32 * kWarpsPerBlock, 0, st>>>(n, sl.crow, sl.csend, sl.cshift, d_pos, sl.pos_ref, b.d_cell,
                                                      b.d_sys_of, b.any_pbc() ? 1 : 0, rc2, half2, sl.keep, sl.deg,
                                                      sl.flags, sl.dmax2);
  }
  MLIP_LAUNCH_CHECK();
  MLIP_TRY(exclusive_scan_i32(ws, sl.deg, sl.nl.row_ptr, n, st, "skin.bsum"));
  {
    MLIP_PROF("skin_write", st);
    skin_write<<<blocks, 32 * kWarpsPerBlock, 0, st>>>(n, sl.crow, sl.csend, sl.cshift, sl.keep, sl.nl.row_ptr,
                                                       sl.nl.recv, sl.nl.send, sl.nl.shift, sl.newidx);
  }
  MLIP_LAUNCH_CHECK();
  {
    MLIP_PROF("skin_rev", st);
    const int g = (int)std::min<int64_t>((sl.cap + 255) / 256, 8192);
    skin_rev<<<g, 256, 0, st>>>(sl.crow + n, sl.crev, sl.newidx, sl.nl.rev, sl.flags);
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}

}  // namespace mlip
