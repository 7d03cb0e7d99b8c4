// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "mlip.h"
#include "sh_poly.h"

namespace mlip {

// ----------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
const char* last_error();

#define MLIP_CUDA_TRY(expr)                                                                    \
  do {                                                                                         \
    cudaError_t e__ = (expr);                                                                  \
    if (e__ != cudaSuccess) {                                                                  \
      cudaGetLastError(); /* clear a non-sticky error so later calls are not blamed */          \
      ::mlip::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e__), __FILE__, __LINE__); \
      return e__ == cudaErrorMemoryAllocation ? MLIP_ERR_OOM : MLIP_ERR_CUDA;                  \
    }                                                                                          \
  } while (0)

#define MLIP_TRY(expr)              \
  do {                              \
    int r__ = (expr);               \
    if (r__ != MLIP_OK) return r__; \
  } while (0)

#define MLIP_LAUNCH_CHECK() MLIP_CUDA_TRY(cudaGetLastError())

// ------------------------------------------------------- coupling tables
template <int L>
struct CGTable;
template <int L>
struct CGTableP;  // every triangle-valid path, both parities (mixed-parity models)
#include "cg_tables.inc"

// ------------------------------------------------------------ workspace
// Grow-only named device buffers, owned by a model (or a neighbour call).
struct Workspace {
  struct Buf { void* p = nullptr; size_t bytes = 0; };
  std::map<std::string, Buf> bufs;
  uint64_t gen = 0;  // bumped whenever a buffer is (re)allocated: device addresses may have changed
  cudaStream_t stream = nullptr;  // the stream of the caller (allocations and releases are ordered on it)
  // the batch tables last uploaded into this workspace (upload_batch skips an identical upload)
  std::vector<double> batch_sig;
  uint64_t batch_gen = ~0ULL;
  int get(const std::string& name, size_t bytes, void** out);
  template <class T>
  int get(const std::string& name, size_t count, T** out) {
    void* p = nullptr;
    int rc = get(name, count * sizeof(T) + 16, &p);
    *out = static_cast<T*>(p);
    return rc;
  }
  void release();
  ~Workspace() { release(); }
};

// Sets the workspace's stream for the scope of an entry point.
struct WsStream {
  Workspace& ws;
  cudaStream_t prev;
  WsStream(Workspace& w, cudaStream_t s) : ws(w), prev(w.stream) { w.stream = s; }
  ~WsStream() { ws.stream = prev; }
};

// Pinned host staging (grow-only).
struct HostStage {
  void* p = nullptr;
  size_t bytes = 0;
  int get(size_t need, void** out);
  ~HostStage();
};

// --------------------------------------------------------- neighbours
constexpr int kMaxDegreeLimit = 4096;

struct NeighborList {
  int64_t n = 0, E = 0;
  int32_t* row_ptr = nullptr;   // [n + 1], receiver segments
  int32_t* recv = nullptr;      // [E]
  int32_t* send = nullptr;      // [E]
  int8_t* shift = nullptr;      // [E * 3]
  int32_t* rev = nullptr;       // [E] index of the reverse edge (j <- i, -S)
  unsigned long long* keys = nullptr;  // [E] sorted (send, S) keys per segment
  int maxdeg = 0;                      // per-receiver slab capacity the build used
};

// Builds the sorted list on the device.  Synchronises `st` once to read E.
int build_neighbors(Workspace& ws, const double* d_pos, int64_t n, const double* cell,
                    const uint8_t* pbc, double rc, bool want_rev, cudaStream_t st, NeighborList* out);

struct EvalGraphs;
void free_eval_graphs(EvalGraphs* g);

// Neighbour build without host synchronisation (the launches can be captured
// in a CUDA graph): the grids of a batch are made on the host and uploaded by
// nl_plan (skipped when the batch, cell and cutoff are those of the last plan);
// build_neighbors_nosync then only launches device work, with a per-receiver
// slab of maxdeg entries and edge arrays of capacity Ecap (out->E = Ecap, the
// count is row_ptr[n] on the device).  Overflows are flagged, never written
// past: flags[0] = a receiver's count when above maxdeg (its list is cut),
// flags[1] an image index beyond +-127, flags[2] a missing reverse edge,
// flags[3] more than Ecap edges (the list is then emptied).
struct NlPlan {
  double rc = 0.0;
  int maxdeg = 0, nbins = 0, nsys = 0;
  int64_t n = -1, Ecap = 0;
  void* d_grid0 = nullptr;       // grids as made on the host (nl_setup completes a copy)
  long long* d_bbox0 = nullptr;  // initial bounding boxes [nsys][6]
  std::vector<double> sig;       // what the uploaded grids were made from
};
struct SystemBatch;
int nl_plan(Workspace& ws, HostStage& stage, const SystemBatch& b, double rc, int maxdeg, int64_t Ecap,
            cudaStream_t st, NlPlan* plan);
int build_neighbors_nosync(Workspace& ws, const double* d_pos, const SystemBatch& b, const NlPlan& plan,
                           cudaStream_t st, NeighborList* out, int* flags);

// ----------------------------------------------------- batches of systems
// Independent systems evaluated together as one graph: the disjoint union of
// their neighbour graphs (no edge joins two systems).  Atoms of system s are
// [atom_off[s], atom_off[s+1]) of the concatenated arrays.  Every per-system
// reduction (energy, virial, kinetic energy) runs over fixed chunks counted
// from the system's first atom, so a system's results do not depend on the
// other systems of its batch.
constexpr int kSegChunk = 1024;  // atoms per reduction chunk

struct SystemBatch {
  int nsys = 0;
  int64_t n = 0;                      // total atoms
  std::vector<int64_t> atom_off;      // [nsys + 1]
  std::vector<double> cell;           // [nsys * 9] lattice rows
  std::vector<uint8_t> pbc;           // [nsys * 3]
  std::vector<double> qtot;           // [nsys] total charges (empty: all zero; models with the charge head)
  std::vector<int> chunk;             // [nchunk * 3]: system, first atom, end atom
  std::vector<int> sys_chunk_off;     // [nsys + 1]: chunks of system s
  // device copies (upload_batch)
  int* d_sys_of = nullptr;            // [n] system of each atom
  int* d_atom_off = nullptr;          // [nsys + 1]
  double* d_cell = nullptr;           // [nsys * 9], zero rows for systems with no periodic axis
  double* d_inv_vol = nullptr;        // [nsys], 1/V for fully periodic systems, else 0
  double* d_qtot = nullptr;           // [nsys] total charges
  int* d_chunk = nullptr;             // [nchunk * 3]
  int* d_sys_chunk_off = nullptr;     // [nsys + 1]
  int nchunk() const { return (int)(chunk.size() / 3); }
  bool any_pbc() const {
    for (uint8_t v : pbc)
      if (v) return true;
    return false;
  }
};

// Fills the host tables of a batch (offsets, cells, pbc must be set) and
// copies them to the device through the model's pinned staging.
int upload_batch(Workspace& ws, HostStage& stage, SystemBatch& b, cudaStream_t st);
// One system as a batch of one.
void single_system(SystemBatch& b, int64_t n, const double* cell, const uint8_t* pbc);

// Neighbour list of the disjoint union.  `b` must have been uploaded.
int build_neighbors_batch(Workspace& ws, const double* d_pos, const SystemBatch& b, double rc, bool want_rev,
                          cudaStream_t st, NeighborList* out);

// Skin neighbour list for MD: candidates (recv <- send, S) within rc + skin,
// in the canonical order, built at the positions pos_ref and kept in buffers
// of fixed capacity; each step compacts them to the pairs within rc.  While no
// atom has moved more than skin/2 from pos_ref, the compacted list equals a
// fresh build at rc element for element (order, shifts and reverse indices).
struct SkinList {
  int64_t n = 0, cap = 0, n_cand = 0;  // atoms, edge capacity, candidates of the last build
  double rc = 0.0, skin = 0.0;
  int32_t *crow = nullptr, *crecv = nullptr, *csend = nullptr, *crev = nullptr;  // candidates
  int8_t* cshift = nullptr;
  double* pos_ref = nullptr;  // [n][3] positions at the build
  int32_t *deg = nullptr, *newidx = nullptr;
  uint8_t* keep = nullptr;
  NeighborList nl;                  // compacted list; nl.E = cap (capacity)
  int* flags = nullptr;             // [0] an atom moved > skin/2, [1] reverse edge missing
  unsigned long long* dmax2 = nullptr;  // largest squared displacement (bits of a double)
  const int* Edev() const { return nl.row_ptr + n; }
};
// Candidate build at b's positions (synchronises the stream once).
int skin_build(Workspace& ws, const double* d_pos, const SystemBatch& b, double rc, double skin, SkinList* sl,
               cudaStream_t st);
// Compacts the candidates to the pairs within rc at d_pos and flags atoms that
// moved more than skin/2; launch sizes depend only on n and the capacity.
int skin_compact(Workspace& ws, SkinList& sl, const double* d_pos, const SystemBatch& b, cudaStream_t st);

// exclusive scan of n int32 values into out[0..n] (out[n] = total)
// (block sums in the workspace buffer named `scratch`)
int exclusive_scan_i32(Workspace& ws, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st,
                       const char* scratch = "scan.bsum");

}  // namespace mlip

// ------------------------------------------------------------- the model
struct mlip_model {
  int S = 0, T = 0, C = 0, L = 0, Lsh = 3, NB = 8, H = 0, p = 6;
  double rc = 5.0, avg_nb = 1.0;
  int P = 0, P0 = 0, D = 0;  // paths, paths with l1 = 0, node components
  int precision = MLIP_PREC_FP32;
  std::vector<double> masses;
  std::vector<float> host_weights;
  float* d_weights = nullptr;  // one allocation
  const float* W_emb = nullptr;
  const float* W_out = nullptr;
  const float* E0 = nullptr;
  std::vector<const float*> W1, W2, W3, Wmix;
  // symmetric contraction (correlation 2; empty otherwise): w1 [S][L+1][C], w2 [S][Q][C] per layer
  int corr = 0, Q = 0;
  std::vector<const float*> Wsc1, Wsc2;
  // charge head and Coulomb term (charges = 1): q_i = W_q[z] . h_i,0 + q0[z]; soft-core radius r0
  int charges = 0;
  double r0 = 0.0;
  const float* W_q = nullptr;
  const float* q0 = nullptr;
  // gated update (gate = 1): Wself [S][L+1][C][C], Wgate [C][L C], Wselfgate [S][C][L C] per layer,
  // and their transposes for the adjoint ([S][L+1][c2][c1], [L C][C], [S][L C][C])
  int gate = 0;
  std::vector<const float*> Wself, Wgate, Wselfgate, WselfT, WgateT, WselfgateT;
  // mixed parity (parity = 1): channel blocks of even and odd parity, every triangle-valid path
  int parity = 0;
  float* d_gateT = nullptr;
  float* d_wmixT = nullptr;            // channel-mix weights transposed, per layer and order
  std::vector<const float*> WmixT;
  // fused form: split FP16 tensor-core images of the mix weights per layer
  // (forward and adjoint, (L+1) x 64 KB each) and their per-order scales
  uint8_t* d_miximg = nullptr;
  float* d_mixscale = nullptr;
  std::vector<const uint8_t*> mix_fwd_img, mix_bwd_img;
  std::vector<const float*> mix_scale;
  // fused form with the gated update: split FP16 weight blocks of the
  // tensor-core gate per layer (forward and adjoint) and their scales [L+1][4]
  uint8_t* d_gateimg = nullptr;
  float* d_gatescale = nullptr;
  std::vector<const uint8_t*> gate_fwd_img, gate_bwd_img;
  std::vector<const float*> gate_fwd_scale, gate_bwd_scale;
  // fused form: max_c |W_emb[z][c]| per species (the FP16 scale of the first adjoint layer)
  float* d_embmax = nullptr;
  // fused form: split FP16 images of the radial MLP's W2 per layer (32 KB each)
  // and their power-of-two scales
  uint8_t* d_radimg = nullptr;
  std::vector<float> rad_scale;
  // fused form: W3 of every layer as BF16 tensor-core operands, grouped by path group
  uint8_t* d_w3img = nullptr;
  std::vector<size_t> w3_layer_off;
  std::vector<std::vector<size_t>> w3_goff;
  int device = 0;
  mlip::Workspace ws;
  mlip::HostStage stage;
  mlip::EvalGraphs* egraph = nullptr;  // cached CUDA graphs of the fused evaluation (fused_bf16.cu)
  // The last separate forward evaluation (mlip_energy_forward), which
  // mlip_energy_backward differentiates: its batch and neighbour list (device
  // tables in the workspace).  Every evaluation that writes the workspace bumps
  // eval_gen; the saved forward is usable while tape_gen == eval_gen.
  uint64_t eval_gen = 0, tape_gen = 0;
  mlip::SystemBatch tape_batch;
  mlip::NeighborList tape_nl;
};
