// Host launchers of the device kernels (defined in plain_fp32.cu, node_ops.cu).
#pragma once

#include "kernels_common.cuh"

namespace mlip {

int launch_edge_geom(int E, const double* pos, const int* recv, const int* send, const int8_t* shift,
                     const CellArg& cell, float4* ev, cudaStream_t st);
int launch_radial_fwd(int H, int E, const float4* ev, const float* W1, const float* W2, float rc, int p,
                      float* z2T, int ldz, cudaStream_t st);
int launch_radial_bwd(int H, int E, const float4* ev, const float* W1, const float* W2, float rc, int p,
                      const float* dz2, float* dr_tot, cudaStream_t st);
int launch_sgemm(bool a_km, bool b_nk, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                 float* C, int ldc, cudaStream_t st);
int launch_tp_fwd(int L, bool first, int n, int C, const int* row_ptr, const int* recv, const int* send,
                  const float4* ev, const float* h, const float* w, int PW, float s, float* m, cudaStream_t st);
int launch_tp_bwd(int L, bool first, int n, int C, const int* row_ptr, const int* recv, const int* send,
                  const float4* ev, const float* hprev, const float* Gm, const float* w, int PW, float s,
                  const float* Gin, float* Gout, float* dw, float* dY, cudaStream_t st);
int launch_mix_fwd(int n, int C, int L, const float* m, const float* Wmix, const float* hin, float* hout,
                   float* u0, cudaStream_t st);
int launch_mix_bwd(int n, int C, int L, const float* G, const float* u0, const float* Wmix, float* Gm,
                   cudaStream_t st);
int launch_mix_fwd2(int n, int C, int L, const float* mA, const float* mB, const float* Wmix, const float* hin,
                    float* hout, float* u0, cudaStream_t st);
int launch_mix_bwd2(int n, int C, int L, const float* GA, const float* GB, const float* u0, const float* Wmix,
                    float* Gm, cudaStream_t st);
int launch_embed(int n, int C, int D, const int* species, const float* W_emb, float* h, cudaStream_t st);
int launch_grad_init(int n, int C, int D, const int* species, const float* W_out, float* G, cudaStream_t st);
int launch_energy(int n, int C, int D, const int* species, const float* W_out, const float* E0, const float* h,
                  double* atom_e, double* energy, cudaStream_t st);
int launch_edge_grad(int E, const float4* ev, const float* dY, const float* dr, float4* g, cudaStream_t st);
int launch_forces_virial(Workspace& ws, int n, const int* row_ptr, const int* rev, const float4* g,
                         const float4* ev, double* forces, double* stress, double inv_vol, cudaStream_t st);

int launch_check_inputs(int n, const double* pos, const int* species, int S, int* flag, cudaStream_t st);
int pack_w3_groups(const mlip_model* M, int t, std::vector<uint8_t>& img, std::vector<size_t>& group_off);
int umma_selftest_run(double* rel_err);
int umma_selftest_mn_run(int variant, double* rel_err);

// Plain FP32 energy/forces/stress of one system whose positions and species
// are on the device.  d_energy, d_forces (n x 3), d_stress (9) are device
// pointers (forces/stress nullable).
int energy_forces_plain(mlip_model* M, const double* d_pos, const int* d_species, int64_t n, const double* cell,
                        const uint8_t* pbc, double* d_energy, double* d_forces, double* d_stress,
                        cudaStream_t st);

// Fused BF16 form (tcgen05 radial MLP), same contract as energy_forces_plain.
int energy_forces_fused(mlip_model* M, const double* d_pos, const int* d_species, int64_t n, const double* cell,
                        const uint8_t* pbc, double* d_energy, double* d_forces, double* d_stress,
                        cudaStream_t st);

int launch_vv_kick(int n, const int* species, const double* mass, double half_dt, const double* F, double* vel,
                   cudaStream_t st);
int launch_vv_drift(int n, double dt, const double* vel, double* pos, cudaStream_t st);
int launch_kinetic(int n, const int* species, const double* mass, const double* vel, double* out, cudaStream_t st);
int energy_forces_device(mlip_model* M, const double* d_pos, const int* d_species, int64_t n, const double* cell,
                         const uint8_t* pbc, double* d_energy, double* d_forces, double* d_stress, cudaStream_t st);

}  // namespace mlip
