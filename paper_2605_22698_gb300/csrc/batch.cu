// Batches of independent systems evaluated as one graph (the disjoint union
// of their neighbour graphs), and the per-system reductions that go with it:
// energies, virials and kinetic energies summed in FP64 over fixed chunks of
// each system's own atoms (so a system's sums are the same whatever else is in
// its batch).
#include <algorithm>
#include <cmath>

#include "launchers.cuh"
#include "profile.cuh"

namespace mlip {
namespace {

// sys_of[i] = s with atom_off[s] <= i < atom_off[s+1]
__global__ void fill_sys_of(int n, int nsys, const int* __restrict__ atom_off, int* __restrict__ sys_of) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (atom_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    sys_of[i] = lo;
  }
}

constexpr int kSegThreads = 256;

// One block per chunk: partial[c][k] = sum over the chunk's atoms of v[i][k],
// each thread summing its atoms in order, then a fixed tree: a packed warp
// butterfly (K <= 16 components at once) and the warps' sums in warp order.
template <int K>
__global__ void seg_partial(const int* __restrict__ chunk, const double* __restrict__ v,
                            double* __restrict__ partial) {
  static_assert(K >= 1 && K <= 16, "up to 16 components");
  __shared__ double wsum[kSegThreads / 32][K];
  const int c = blockIdx.x;
  const int a0 = chunk[3 * c + 1], a1 = chunk[3 * c + 2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  for (int i = a0 + threadIdx.x; i < a1; i += kSegThreads)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += v[(size_t)i * K + k];
  if constexpr (K == 1) {
    double t = acc[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) wsum[w][0] = t;
  } else {
    const double t = warp_reduce16_f64(acc);  // lane l: component l >> 1
    if ((lane & 1) == 0 && (lane >> 1) < K) wsum[w][lane >> 1] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < K) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kSegThreads / 32; ++q) t += wsum[q][threadIdx.x];
    partial[(size_t)c * K + threadIdx.x] = t;
  }
}

// out[s][k] = scale_s * sum of the system's chunk partials, in chunk order.
template <int K>
__global__ void seg_finish(int nsys, const int* __restrict__ sys_chunk_off, const double* __restrict__ partial,
                           const double* __restrict__ scale, double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nsys * K) return;
  const int s = q / K, k = q - s * K;
  double acc = 0.0;
  for (int c = sys_chunk_off[s]; c < sys_chunk_off[s + 1]; ++c) acc += partial[(size_t)c * K + k];
  out[q] = scale ? acc * scale[s] : acc;
}


double cell_volume3(const double* h) {
  return std::fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                   h[2] * (h[3] * h[7] - h[4] * h[6]));
}

}  // namespace

void single_system(SystemBatch& b, int64_t n, const double* cell, const uint8_t* pbc) {
  b.nsys = 1;
  b.n = n;
  b.atom_off = {0, n};
  b.cell.assign(cell, cell + 9);
  b.pbc.assign(pbc, pbc + 3);
  b.qtot.clear();
}

int upload_batch(Workspace& ws, HostStage& stage, SystemBatch& b, cudaStream_t st) {
  const int nsys = b.nsys;
  if (nsys < 1 || (int)b.atom_off.size() != nsys + 1 || (int)b.cell.size() != 9 * nsys ||
      (int)b.pbc.size() != 3 * nsys || (!b.qtot.empty() && (int)b.qtot.size() != nsys)) {
    set_error("batch: inconsistent system tables");
    return MLIP_ERR_INVALID_ARG;
  }
  b.n = b.atom_off[nsys];
  if (b.n > (1LL << 30)) { set_error("batch: %lld atoms in total (limit 2^30)", (long long)b.n); return MLIP_ERR_INVALID_ARG; }
  b.chunk.clear();
  b.sys_chunk_off.assign(nsys + 1, 0);
  for (int s = 0; s < nsys; ++s) {
    b.sys_chunk_off[s] = (int)(b.chunk.size() / 3);
    for (int64_t a = b.atom_off[s]; a < b.atom_off[s + 1]; a += kSegChunk) {
      b.chunk.push_back(s);
      b.chunk.push_back((int)a);
      b.chunk.push_back((int)std::min<int64_t>(a + kSegChunk, b.atom_off[s + 1]));
    }
  }
  b.sys_chunk_off[nsys] = (int)(b.chunk.size() / 3);
  const int nch = b.nchunk();
  // one pinned blob: doubles (cells, 1/V, total charges), then ints (offsets, chunks, chunk offsets)
  const size_t nd = (size_t)11 * nsys, ni = (size_t)(nsys + 1) + 3 * (size_t)nch + (size_t)(nsys + 1);
  const size_t bytes = nd * sizeof(double) + ni * sizeof(int);
  void* hp = nullptr;
  MLIP_TRY(stage.get(bytes, &hp));
  double* hd = static_cast<double*>(hp);
  for (int s = 0; s < nsys; ++s) {
    const uint8_t* pb = &b.pbc[3 * s];
    const bool any = pb[0] || pb[1] || pb[2], all = pb[0] && pb[1] && pb[2];
    for (int k = 0; k < 9; ++k) hd[9 * s + k] = any ? b.cell[9 * s + k] : 0.0;
    const double vol = all ? cell_volume3(&b.cell[9 * s]) : 0.0;
    hd[9 * nsys + s] = vol > 0.0 ? 1.0 / vol : 0.0;
    hd[10 * nsys + s] = b.qtot.empty() ? 0.0 : b.qtot[s];
  }
  int* hi = reinterpret_cast<int*>(hd + nd);
  for (int s = 0; s <= nsys; ++s) hi[s] = (int)b.atom_off[s];
  std::copy(b.chunk.begin(), b.chunk.end(), hi + nsys + 1);
  std::copy(b.sys_chunk_off.begin(), b.sys_chunk_off.end(), hi + nsys + 1 + 3 * nch);
  unsigned char* dblob = nullptr;
  MLIP_TRY(ws.get("batch.blob", bytes, &dblob));
  b.d_sys_of = nullptr;
  if (nsys > 1 && b.n > 0) MLIP_TRY(ws.get("batch.sys_of", (size_t)b.n, &b.d_sys_of));
  b.d_cell = reinterpret_cast<double*>(dblob);
  b.d_inv_vol = b.d_cell + 9 * nsys;
  b.d_qtot = b.d_cell + 10 * nsys;
  b.d_atom_off = reinterpret_cast<int*>(b.d_cell + nd);
  b.d_chunk = b.d_atom_off + nsys + 1;
  b.d_sys_chunk_off = b.d_chunk + 3 * nch;
  // the same tables as the last upload into unchanged buffers: nothing to copy
  std::vector<double> sig;
  sig.reserve(1 + (size_t)(nsys + 1) + 13 * (size_t)nsys);
  sig.push_back((double)nsys);
  for (int s = 0; s <= nsys; ++s) sig.push_back((double)b.atom_off[s]);
  sig.insert(sig.end(), b.cell.begin(), b.cell.end());
  for (uint8_t v : b.pbc) sig.push_back(v);
  for (int s = 0; s < nsys; ++s) sig.push_back(b.qtot.empty() ? 0.0 : b.qtot[s]);
  if (sig == ws.batch_sig && ws.batch_gen == ws.gen) return MLIP_OK;
  ws.batch_sig.clear();
  MLIP_CUDA_TRY(cudaMemcpyAsync(dblob, hp, bytes, cudaMemcpyHostToDevice, st));
  if (b.d_sys_of) {
    const int n = (int)b.n;
    MLIP_PROF("fill_sys_of", st);
    fill_sys_of<<<std::min((n + 255) / 256, 4096), 256, 0, st>>>(n, nsys, b.d_atom_off, b.d_sys_of);
    MLIP_LAUNCH_CHECK();
  }
  // the pinned blob is reused by the next upload: wait for this copy
  MLIP_CUDA_TRY(cudaStreamSynchronize(st));
  ws.batch_sig = sig;
  ws.batch_gen = ws.gen;
  return MLIP_OK;
}

int launch_seg_sum(Workspace& ws, const SystemBatch& b, int K, const double* v, bool scale_inv_vol, double* out,
                   cudaStream_t st) {
  const int nch = b.nchunk();
  double* part = nullptr;
  MLIP_TRY(ws.get("seg.part", (size_t)std::max(nch, 1) * K, &part));
  if (K == 1) {
    if (nch > 0) { MLIP_PROF("seg_partial", st); seg_partial<1><<<nch, kSegThreads, 0, st>>>(b.d_chunk, v, part); }
    { MLIP_PROF("seg_finish", st); seg_finish<1><<<(b.nsys + 127) / 128, 128, 0, st>>>(b.nsys, b.d_sys_chunk_off, part, scale_inv_vol ? b.d_inv_vol : nullptr, out); }
  } else if (K == 9) {
    if (nch > 0) { MLIP_PROF("seg_partial", st); seg_partial<9><<<nch, kSegThreads, 0, st>>>(b.d_chunk, v, part); }
    { MLIP_PROF("seg_finish", st); seg_finish<9><<<(9 * b.nsys + 127) / 128, 128, 0, st>>>(b.nsys, b.d_sys_chunk_off, part, scale_inv_vol ? b.d_inv_vol : nullptr, out); }
  } else {
    set_error("seg_sum: unsupported width %d", K);
    return MLIP_ERR_INVALID_ARG;
  }
  MLIP_LAUNCH_CHECK();
  return MLIP_OK;
}


}  // namespace mlip
