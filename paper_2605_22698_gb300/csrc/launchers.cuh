// Host launchers of the device kernels (defined in plain_fp32.cu, node_ops.cu).
#pragma once

#include <cstdint>
#include <vector>

#include "kernels_common.cuh"

namespace mlip {

// Edge kernels take an optional device edge count Edev: when given, the launch
// is sized for E (a capacity) and the kernel processes *Edev <= E edges.
int launch_edge_geom(int E, const double* pos, const int* recv, const int* send, const int8_t* shift,
                     const CellArg& cell, float4* ev, cudaStream_t st, const int* Edev = nullptr);
int launch_radial_fwd(int H, int E, const float4* ev, const float* W1, const float* W2, float rc, int p,
                      float* z2T, int ldz, cudaStream_t st);
int launch_radial_bwd(int H, int E, const float4* ev, const float* W1, const float* W2, float rc, int p,
                      const float* dz2, float* dr_tot, cudaStream_t st);
int launch_sgemm(bool a_km, bool b_nk, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                 float* C, int ldc, cudaStream_t st);
// par: mixed-parity models (every path; odd-l2 paths couple the other parity block)
int launch_tp_fwd(int L, bool first, int n, int C, const int* row_ptr, const int* recv, const int* send,
                  const float4* ev, const float* h, const float* w, int PW, float s, float* m, cudaStream_t st,
                  bool par = false);
int launch_tp_bwd(int L, bool first, int n, int C, const int* row_ptr, const int* recv, const int* send,
                  const float4* ev, const float* hprev, const float* Gm, const float* w, int PW, float s,
                  const float* Gin, float* Gout, float* dw, float* dY, cudaStream_t st, bool par = false);
// parity: tanh instead of SiLU on the odd scalar block (channels >= C/2) of mixed-parity models
int launch_mix_fwd(int n, int C, int L, const float* m, const float* Wmix, const float* hin, float* hout,
                   float* u0, cudaStream_t st, int parity = 0);
int launch_mix_bwd(int n, int C, int L, const float* G, const float* u0, const float* Wmix, const float* WmixT,
                   float* Gm, cudaStream_t st, int parity = 0);
// amax (nullable): per-system max |h| accumulated into amax[2 s] (zeroed by the caller) from the
// per-species maxima emax[z] = max_c |W_emb[z][c]|
int launch_embed(int n, int C, int D, int S, const int* species, const float* W_emb, float* h, cudaStream_t st,
                 const int* sys_of = nullptr, const float* emax = nullptr, float* amax = nullptr);
int launch_grad_init(int n, int C, int D, int S, const int* species, const float* W_out, float* G, cudaStream_t st);
// out_i = W[z_i] . h_i,0 + b0[z_i] (FP32 dot, FP64 result)
int launch_readout(int n, int C, int D, int S, const int* species, const float* W, const float* b0, const float* h,
                   double* out, cudaStream_t st);
// per-system energies energy[nsys] (FP64)
int launch_energy(Workspace& ws, const SystemBatch& b, int C, int D, int S, const int* species, const float* W_out,
                  const float* E0, const float* h, double* atom_e, double* energy, cudaStream_t st);
int launch_edge_grad(int E, const float4* ev, const float* dY, const float* dr, float4* g, cudaStream_t st,
                     const int* Edev = nullptr);
// forces[n][3]; stress[nsys][9] = virial / V per system (zero rows for systems
// without a fully periodic cell), nullable
int launch_forces_virial(Workspace& ws, const SystemBatch& b, const int* row_ptr, const int* rev, const float4* g,
                         const float4* ev, double* forces, double* stress, cudaStream_t st);
// out[s][k] = sum over the atoms of system s of v[i][k] (K = 1 or 9), times 1/V_s if scale_inv_vol
int launch_seg_sum(Workspace& ws, const SystemBatch& b, int K, const double* v, bool scale_inv_vol, double* out,
                   cudaStream_t st);

// Radial MLP of the fused form on the tensor cores (H = 64): z2 operand tiles,
// and dE/dr accumulated from dE/dz2.  err receives the bounded-wait flags.
int launch_radial_tc(int H, int E, int n_tiles32, const float4* ev, const float* W1, const uint8_t* w2img,
                     float wsc, float rc, int p, int use_bf16, uint8_t* z2t, int* err, cudaStream_t st,
                     const int* Edev = nullptr);
// init: write dE/dr instead of adding to it
int launch_radial_bwd_tc(int H, int E, const float4* ev, const float* W1, const uint8_t* w2img, float wsc, float rc,
                         int p, const float* dz2, float* dr_tot, bool init, int* err, cudaStream_t st,
                         const int* Edev = nullptr);
// Split FP16 image of one layer's W2 for the two kernels above (32 KB) and its
// power-of-two scale.
void pack_radial_images(const float* W2, std::vector<uint8_t>& img, float* scale);

// Channel mixes of the fused form on the tensor cores (C = 128): X (+ X2) times
// the split weight images of one layer (pack_mix_images), forward or adjoint.
void pack_mix_images(const float* W, int L, std::vector<uint8_t>& fwd, std::vector<uint8_t>& bwd,
                     std::vector<float>& scale);
// amax (nullable): per-system max |out| accumulated into amax[2 s] (zeroed by the caller)
int launch_mix_tc(bool bwd, int n, int C, int L, const float* X, const float* X2, const uint8_t* wimg,
                  const float* wscale, const float* hin, float* out, float* u0, const float* u0_in, int* err,
                  cudaStream_t st, const int* sys_of = nullptr, float* amax = nullptr);

int launch_check_inputs(int n, const double* pos, const int* species, int S, int* flag, cudaStream_t st);
int pack_w3_groups(const mlip_model* M, int t, std::vector<uint8_t>& img, std::vector<size_t>& group_off);
int umma_selftest_run(double* rel_err);
int umma_selftest_mn_run(int variant, double* rel_err);

// Energy, forces and stress of a batch of systems whose positions and species
// are on the device (concatenated).  d_energy [nsys], d_forces [n][3] and
// d_stress [nsys][9] are device pointers (forces and stress nullable).  The
// batch must have been uploaded.
int evaluate_plain(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                   double* d_energy, double* d_forces, double* d_stress, cudaStream_t st);
// Fused 16-bit form (tcgen05 radial MLP and path products), same contract.
int evaluate_fused(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                   double* d_energy, double* d_forces, double* d_stress, cudaStream_t st);
// The fused form's evaluation on a given neighbour list: no build and no
// synchronisation.  With Edev, nl.E is a capacity and *Edev the edge count on
// the device (launch sizes then depend on the capacity only, so the work can be
// captured in a CUDA graph).  Input and bounded-wait errors are flagged in
// flag[0..1] (check_eval_flags).
int evaluate_fused_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                         const NeighborList& nl, const int* Edev, int* flag, double* d_energy, double* d_forces,
                         double* d_stress, cudaStream_t st);
// The two halves of evaluate_fused_edges, for the separate forward and
// backward entry points.  The forward leaves in the workspace what the adjoint
// reads (node features and pre-activations of every layer, the FP16 operand
// scales); the adjoint with recompute first computes the edge geometry, the
// harmonics and, layer by layer, the radial weights again from the positions.
int fused_forward_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                        const NeighborList& nl, const int* Edev, int* flag, double* d_energy, cudaStream_t st);
int fused_adjoint_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                        const NeighborList& nl, const int* Edev, int* flag, double* d_forces, double* d_stress,
                        bool recompute, cudaStream_t st);
// The plain form's halves on a given neighbour list (its adjoint reads the
// per-edge radial weights the forward stored: the stored-intermediate design
// of the comparator form).
int plain_forward_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                        const NeighborList& nl, double* d_energy, cudaStream_t st);
int plain_adjoint_edges(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                        const NeighborList& nl, double* d_forces, double* d_stress, cudaStream_t st);
// Synchronises st and turns the flags of evaluate_fused_edges into a status.
int check_eval_flags(const int* flag, cudaStream_t st);
// evaluate_fused for callers that repeat the same batch layout (one system
// evaluated again and again, MD steps): the evaluation, neighbour build
// included, runs without host synchronisation and is captured once as a CUDA
// graph, replayed while the layout, the requested outputs and the workspace
// stay the same.  The first call of a layout runs evaluate_fused (to learn
// the edge count), the second runs the same launches eagerly, the third
// captures.  Results equal evaluate_fused's bit for bit; capacity overflows
// are detected after the replay and the call is redone by evaluate_fused.
int evaluate_fused_graph(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b,
                         double* d_energy, double* d_forces, double* d_stress, cudaStream_t st);
// The model's form; graph: allow evaluate_fused_graph (fused forms).
int evaluate(mlip_model* M, const double* d_pos, const int* d_species, const SystemBatch& b, double* d_energy,
             double* d_forces, double* d_stress, cudaStream_t st, bool graph = false);

// Velocity Verlet on a batch: systems with active[s] != 0 move with their own
// time step dt[s] (fs); the others are left as they are.
int launch_vv_kick(const SystemBatch& b, const int* species, const double* mass, const double* dt,
                   const int* active, const double* F, double* vel, cudaStream_t st);
int launch_vv_drift(const SystemBatch& b, const double* dt, const int* active, const double* vel, double* pos,
                    cudaStream_t st);
// ke[s] = sum over system s of m v^2 / (2 kappa)  (eV)
int launch_kinetic(Workspace& ws, const SystemBatch& b, const int* species, const double* mass, const double* vel,
                   double* ke, cudaStream_t st);

// Symmetric contraction of correlation order 2 (sym_contract.cu): out = B(A)
// with A = X (+ X2), A also written to Asave; its adjoint GA from GB at A
// (out_max: per-system max |GA| at out_max[2 sys], nullable).  In place allowed.
int sc_num_paths(int L);
int launch_sym_contract(int L, int n, int C, int S, const float* X, const float* X2, const int* species, const float* w1,
                        const float* w2, float* Asave, float* out, cudaStream_t st);
int launch_sym_contract_bwd(int L, int n, int C, int S, const float* GB, const float* A, const int* species,
                            const float* w1, const float* w2, float* GA, const int* sys_of, float* out_max,
                            cudaStream_t st);

// Charge head, charge correction and Coulomb term (coulomb.cu), for models
// with charges = 1 and open systems.  Forward: from h^T and the per-atom
// readout energies in atom_e, adds the Coulomb shares to atom_e and keeps
// the corrected charges, dE/dqt and the direct forces in the workspace.
// Adjoint: adds dE/dq_i W_q[z_i] to the scalar rows of G and the direct
// forces to forces.
int coulomb_forward(Workspace& ws, const SystemBatch& b, const mlip_model* M, const double* d_pos,
                    const int* species, const float* hT, double* atom_e, cudaStream_t st);
int coulomb_adjoint(Workspace& ws, const SystemBatch& b, const mlip_model* M, const int* species, float* G,
                    cudaStream_t st);
int coulomb_add_forces(Workspace& ws, const SystemBatch& b, double* forces, cudaStream_t st);
// the corrected charges of the last coulomb_forward ([n] FP64, device)
int coulomb_charges(Workspace& ws, const SystemBatch& b, double** q);

// Gated update with the species self-connection (gate.cu), replacing the
// channel mix for models with gate = 1: forward h_out from the messages
// X (+ X2) and h_in, keeping pre [n][D][C] and the gate pre-activations
// g [n][L C]; adjoint from G (+ G2) = dE/dh': Gm = dE/dm, and in place
// G <- dE/dh (G2 <- 0).  out_max (nullable): per-system max |h_out| or |Gm|.
int gate_prepare(int L, int C);
int launch_gate_fwd(int L, int n, int C, int S, const int* species, const float* X, const float* X2,
                    const float* hin, const float* Wm, const float* Ws, const float* Wg, const float* Wsg,
                    float* hout, float* pre, float* g, const int* sys_of, float* out_max, cudaStream_t st);
int launch_gate_bwd(int L, int n, int C, int S, const int* species, float* G, float* G2, const float* pre,
                    const float* g, const float* WmT, const float* WsT, const float* WgT, const float* WsgT,
                    float* Gm, const int* sys_of, float* out_max, cudaStream_t st);
// The same on the tensor cores (gate_tc.cu; fused form, 128 channels): the
// layer's split FP16 weight blocks and scales from pack_gate_images.  The
// adjoint needs dpre [n][D][C] and dg [n][L C] as scratch.
void pack_gate_images(bool bwd, const float* Wm, const float* Ws, const float* Wg, const float* Wsg, int L, int S,
                      std::vector<uint8_t>& img, std::vector<float>& scale);
int gate_tc_prepare();
int launch_gate_tc_fwd(int L, int n, int S, const int* species, const float* X, const float* X2, const float* hin,
                       const uint8_t* img, const float* wscale, float* hout, float* pre, float* g, int* err,
                       const int* sys_of, float* out_max, cudaStream_t st);
int launch_gate_tc_bwd(int L, int n, int S, const int* species, float* G, float* G2, const float* pre, const float* g,
                       const uint8_t* img, const float* wscale, float* Gm, float* dpre, float* dg, int* err,
                       const int* sys_of, float* out_max, cudaStream_t st);

}  // namespace mlip
