/*
 * mlip.h - C ABI of the GB300 equivariant interaction-layer library.
 *
 * The library evaluates an equivariant message-passing interatomic potential
 * of the NequIP/MACE family that arxiv 2605.22698 ("mlip v2") trains and
 * simulates (Sec. 2 "Background and related work"; Sec. 4 "Accelerating
 * equivariant operations with e3j"; hyperparameters of Tables
 * tbl:nequip_params and tbl:mace_params).  Energy is a per-atom readout plus
 * per-species reference energies (Eq. multihead_readout with one head);
 * forces are -dE/dr (the first derivative in Eq. full_hessian).  The model:
 *
 *   edges     all (receiver i, sender j, image S) with |r_j - r_i + S.h| < rc
 *   x_e       r_j - r_i + S.h,  r = |x_e|,  unit vector r^ = x_e / r
 *   Y_e       real spherical harmonics Y_{l m}(r^), l <= 3 (16 values)
 *   b_e[n]    sqrt(2/rc) sin(n pi r/rc)/r * u(r/rc), n = 1..8, u the p = 6
 *             polynomial envelope
 *   w_e       W3^T silu(W2^T silu(W1^T b_e))  -> one weight per path and channel
 *   m_i       (1/avg_num_neighbors) sum_{e: recv = i} sum_paths w_e[p][c]
 *             sum_{m1,m2} CG^p[m3][m1][m2] h_j[l1 m1][c] Y_e[l2 m2]
 *   update    u = m W_l per l; h_0 += silu(u_0); h_{l>0} += u_l
 *   energy    E = sum_i (W_out[z_i] . h_i,0 + E0[z_i])
 *
 * Conventions (all functions):
 *   - Return an int status: 0 = MLIP_OK, negative = error; they never abort.
 *     mlip_last_error() gives a thread-local message for the last failure.
 *     A sticky CUDA error is reported as MLIP_ERR_CUDA.
 *   - Units: positions A (double, row-major [n][3]), energies eV, forces eV/A,
 *     stress eV/A^3 (ASE sign: stress = (1/V) dE/d(strain)), time fs, mass amu.
 *   - cell: 3 x 3 row-major doubles, rows are the lattice vectors; pbc: 3 bytes.
 *     cell and pbc are always HOST pointers.  For a system with no periodic
 *     axis the cell is ignored.  Positions are never wrapped.
 *   - on_device = 0: positions, species and outputs are host pointers; the
 *     call copies them to and from device buffers it owns.  on_device = 1: they are
 *     device pointers on the current CUDA device.  stream: a cudaStream_t or
 *     NULL (legacy default stream).
 *   - The caller owns every buffer it passes.  Opaque handles are owned by the
 *     library and released with the matching _free/_destroy.  One model handle
 *     must not be used by two threads at the same time.
 *   - Species are integers 0..n_species-1.
 */
#ifndef MLIP_H
#define MLIP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MLIP_OK = 0,
  MLIP_PENDING = 1,
  MLIP_ERR_INVALID_ARG = -1,
  MLIP_ERR_CUDA = -2,
  MLIP_ERR_OOM = -3,
  MLIP_ERR_BUDGET = -4,
  MLIP_ERR_CAPACITY = -5,
  MLIP_ERR_CELL = -6,
  MLIP_ERR_DEGENERATE = -7,
  MLIP_ERR_TIMEOUT = -8,
  MLIP_ERR_DEVICE_TIMEOUT = -9,
  MLIP_ERR_NOT_FOUND = -10
} mlip_status;

/* Precision of a model's compute path.
 * MLIP_PREC_FP32: the plain FP32 form - every product on the FP32 ALUs, the
 *   per-edge radial weights materialised in HBM, stored intermediates.
 * MLIP_PREC_BF16: the fused form - the radial MLP's output layer (forward and
 *   adjoint) on tcgen05 tensor cores with BF16 operands and FP32 accumulation
 *   in tensor memory; harmonics, tensor product, mixes and reductions in FP32
 *   (FP64 for energy, virial, forces); radial weights recomputed in the
 *   adjoint, never stored.
 * MLIP_PREC_F16: the same fused form with FP16 operands (3 more mantissa bits;
 *   the adjoint operand is scaled by a power of two per layer to stay in
 *   range).  Same speed; used where BF16 rounding of the weights exceeds a
 *   2e-3 max|F| force tolerance. */
enum { MLIP_PREC_FP32 = 0, MLIP_PREC_BF16 = 1, MLIP_PREC_F16 = 2 };

typedef struct mlip_model mlip_model;

/* Hyperparameters.  Defaults of the paper's tables: n_basis 8 (num_rbf),
 * hidden 64 (radial_net_n_hidden), two hidden layers, envelope p = 6,
 * cutoff 5 A (graph_cutoff_angstrom).  Supported: channels 16 or 128 (BF16
 * form: 128), l_max 2 or 3, sh_l_max 3, n_basis 8, hidden 32 or 64.
 * correlation: 0 = the scatter-summed messages go straight to the channel
 * mix (NequIP-style layer); 2 = MACE's symmetric contraction of correlation
 * order 2 (MACE table: correlation 2) is applied to them first, per node and
 * channel with species-dependent weights:
 *   B[l3 m3] = w1[z][l3] A[l3 m3]
 *            + sum_q w2[z][q] sum C^q[m3][m1][m2] A[l1 m1] A[l2 m2]
 * over the Q couplings q = (l1 <= l2 <= l_max, l3 <= l_max), triangle rule,
 * l1 + l2 + l3 even, lexicographic (Q = 8 for l_max 2, 15 for l_max 3). */
typedef struct {
  int32_t n_species, n_layers, channels, l_max, sh_l_max, n_basis, hidden, envelope_p;
  double cutoff;             /* rc, A */
  double avg_num_neighbors;  /* message scale s = 1/avg_num_neighbors */
  const double* masses;      /* n_species masses (amu), host; may be NULL (no MD) */
  int32_t correlation;       /* 0 or 2 (see above) */
  int32_t charges;           /* 1: charge head, charge correction and Coulomb term (below) */
  double coulomb_r0;         /* soft-core radius r0 of the Coulomb term, A (charges = 1) */
  int32_t gate;              /* 1: gated update with a species self-connection (below) */
  int32_t parity;            /* 1: mixed-parity features (below) */
} mlip_model_desc;

/* parity = 1 (the mixed-parity irreps of the paper's NequIP table,
 * "0e + 0o + 1o + 1e + 2e + 2o", here with C/2 channels of each order and
 * parity): channels c < C/2 of every order form the even-parity block, c >= C/2
 * the odd block.  The paths are every triangle-valid (l1, l2, l3) in
 * lexicographic order, odd l1 + l2 + l3 (pseudotensor couplings) included
 * (18 for l_max 2, 34 for l_max 3); a path with odd l2 couples each channel to
 * the same channel of the other block (output parity = input parity x
 * (-1)^l2).  The embedding and the readout use the even scalars only, the
 * channel mixes keep the blocks (block-diagonal W_l), and the scalar update is
 * h_0 += silu(u) on even channels and tanh(u) on odd ones: the weights outside
 * those blocks are ignored (zeroed at creation).  Plain FP32 form only, without
 * correlation, charges or gate; an even channel count. */

/* gate = 1 (NequIP's gate nonlinearity and self-connection, on the uniform
 * natural-parity irreps of this layer; 32, 64 or 128 channels): the channel
 * mix and residual update become, per node of species z and channel,
 *   pre_l = m_l W_l + h_l Wself[z][l],   g_l = m_0 Wgate_l + h_0 Wselfgate[z]_l (l >= 1)
 *   h_0 += silu(pre_0),   h_l += sigmoid(g_l) pre_l   (one gate per channel and l, shared over m)
 * with weights Wself [S][L+1][C][C], Wgate [C][L C], Wselfgate [S][C][L C]
 * after each layer's W_mix (and the contraction's weights). */

/* charges = 1 (Sec. "Treatment of electrostatics and long-range
 * interactions"): per-atom charges q_i = W_q[z_i] . h^T_i,0 + q0[z_i] (weights
 * W_q [S][C], q0 [S] after E0), corrected to the system's total charge Q
 * (Eq. charge_correction: qt_i = q_i - (sum_j q_j - Q) / N), and the energy
 * gains E_LR = k sum_{i<j} qt_i qt_j / chi(r_ij) over all pairs of the system
 * (Eq. long_range_interaction; k = 14.3996454784 eV A / e^2; PhysNet's
 * surrogate distance 1/chi(r) = phi(r/r0) / sqrt(r^2 + 1) + (1 - phi(r/r0)) / r,
 * phi(x) = 1 - 10 x^3 + 15 x^4 - 6 x^5 for x < 1, else 0).  Open systems only:
 * every entry point returns MLIP_ERR_CELL for a periodic system; Q = 0 except
 * through mlip_energy_forces_charged. */

/* Thread-local text of the last error (never NULL). */
const char* mlip_last_error(void);
int mlip_version(void);

/* Number of float32 weights a model with this description takes, in the order
 *   W_emb [S][C]; per layer: W1 [8][H], W2 [H][H], W3 [H][P][C], W_mix [L+1][C][C]
 *   (with correlation 2 also w1 [S][L+1][C], w2 [S][Q][C]; with gate also Wself,
 *   Wgate, Wselfgate); W_out [S][C]; E0 [S] (with charges also W_q [S][C], q0 [S])
 * (P = number of coupling paths (l1 <= L, l2 <= 3, l3 <= L, triangle rule,
 * l1 + l2 + l3 even, lexicographic).  Errors: MLIP_ERR_INVALID_ARG. */
int mlip_model_num_weights(const mlip_model_desc* desc, int64_t* n_weights);

/* Create a model on the current device from host weights (copied).
 * Errors: MLIP_ERR_INVALID_ARG (unsupported hyperparameters, wrong count),
 * MLIP_ERR_OOM, MLIP_ERR_CUDA. */
int mlip_model_create(const mlip_model_desc* desc, const float* weights, int64_t n_weights,
                      int precision, mlip_model** out);

/* Load a parameter file: "MLIPPRM1", u32 version (1, 2 or 3), 8 x i32 (S, T,
 * C, L, Lsh, NB, H, p), versions 2 and 3: i32 correlation, i32 charges, f64
 * coulomb_r0, i32 gate; version 3: i32 parity; then 2 x f64 (rc,
 * avg_num_neighbors), S x f64 masses, i64 count,
 * count x f32 weights; little-endian.  Errors as mlip_model_create plus
 * MLIP_ERR_NOT_FOUND (unreadable file). */
int mlip_model_load(const char* params_path, int precision, mlip_model** out);

int mlip_model_free(mlip_model* model);

/* Directed neighbour list (the Graph built from a ChemicalSystem with
 * graph_cutoff_angstrom, App. A): all (recv i, send j, S) with
 *   d2 = (dx*dx + dy*dy) + dz*dz < cutoff^2,  dx = (x_j - x_i) + sx,
 *   sx = (S0*h00 + S1*h10) + S2*h20 (likewise y, z), in FP64 with no fused
 *   multiply-add,
 * excluding i == j with S = 0; S_k = 0 on open axes.  Sorted by (recv, send,
 * S0, S1, S2).  recv/send: int32[capacity]; shift: int8[capacity * 3].
 * On return *n_edges holds the number of edges; if it exceeds capacity the
 * call returns MLIP_ERR_CAPACITY and writes nothing (retry with a larger
 * buffer).  Other errors: MLIP_ERR_CELL (singular cell with a periodic axis),
 * MLIP_ERR_INVALID_ARG (|S| > 127, n < 0, cutoff <= 0, a receiver with more
 * than 4096 neighbours), MLIP_ERR_CUDA. */
int mlip_neighbors(const double* pos, int64_t n, const double cell[9], const uint8_t pbc[3],
                   double cutoff, int32_t* recv, int32_t* send, int8_t* shift, int64_t capacity,
                   int64_t* n_edges, int on_device, void* stream);

/* Allocation-free neighbour list (the paper has no counterpart; it is an
 * interface for callers that cannot allocate device memory).  Some callers
 * cannot call cudaMalloc: an application that fixes its device-memory budget
 * up front and forbids later growth, a latency-critical loop that must not
 * take the implicit device synchronisation of cudaMalloc/cudaFree, or a
 * plug-in running inside another framework's memory pool.  This call computes
 * the same list as mlip_neighbors (same definition, order and bit-identical
 * output) but allocates nothing: its scratch is one file-scope device array
 * of 32 MiB, kept by every GPU that loads the library until the process exits.
 *   pos: DEVICE pointer [n][3]; recv, send: DEVICE int32[capacity]; shift:
 *   DEVICE int8[capacity * 3]; cell, pbc: host; stream: cudaStream_t or NULL.
 * Limits: n <= 12288 atoms and at most 256 neighbours per receiver; larger
 * inputs return MLIP_ERR_INVALID_ARG (atoms) or MLIP_ERR_CAPACITY (degree)
 * with a message naming the limit.  *n_edges and MLIP_ERR_CAPACITY behave as
 * in mlip_neighbors.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) for that device.  All calls share the one
 * array: calls that overlap on
 * the GPU (two streams, two threads) race and must be serialised by the
 * caller.  The call synchronises the stream (to read the edge count). */
int mlip_neighbors_noalloc(const double* pos, int64_t n, const double cell[9], const uint8_t pbc[3],
                           double cutoff, int32_t* recv, int32_t* send, int8_t* shift, int64_t capacity,
                           int64_t* n_edges, void* stream);

/* Energy, forces and stress of one system.  energy: one double; forces:
 * double[n][3] or NULL; stress: double[9] or NULL (requires pbc all true, else
 * MLIP_ERR_CELL).  The neighbour list is built on the device inside the call.
 * Errors: MLIP_ERR_INVALID_ARG (species out of range, n < 1), MLIP_ERR_CELL,
 * MLIP_ERR_OOM, MLIP_ERR_CUDA.  The call synchronises the stream once (to size
 * the edge buffers). */
int mlip_energy_forces(mlip_model* model, const double* pos, const int32_t* species, int64_t n,
                       const double cell[9], const uint8_t pbc[3], double* energy, double* forces,
                       double* stress, int on_device, void* stream);

/* Separate forward and backward of one system's energy, for automatic
 * differentiation frameworks (the library's torch.autograd.Function uses them).
 * The paper differentiates its energy for forces (Eq. full_hessian, first
 * derivative, F = -dE/dr); this pair splits that differentiation in two calls.
 *
 * mlip_energy_forward: the energy of one system (arguments as in
 *   mlip_energy_forces; energy: one double, on the device when on_device).  It
 *   runs no adjoint kernel.  It keeps, in the model's workspace, its own copy of
 *   the positions and species, the neighbour list and the node features (and
 *   mix pre-activations) of every layer; nothing per edge is kept for the
 *   backward.  Synchronises the stream (input check, edge count).
 * mlip_energy_backward: the gradient of g E with respect to the positions of
 *   the last forward, grad_pos[i][a] = g dE/dr_ia = -g F_ia (double[n][3]),
 *   and optionally g times the stress (double[9], fully periodic cells only,
 *   else MLIP_ERR_CELL).  grad_energy points to g (one double; on the device
 *   when on_device, like grad_pos and stress).  The fused forms compute the
 *   edge geometry, harmonics and each layer's radial weights again from the
 *   saved positions and run the adjoint kernels; the plain FP32 form reads the
 *   radial weights its forward stored.  It may be called more than once for one
 *   forward.  Any other evaluation of the model after the forward (any entry
 *   point, the server, MD) overwrites what the forward kept: the backward then
 *   returns MLIP_ERR_INVALID_ARG.  Other errors: MLIP_ERR_CUDA,
 *   MLIP_ERR_DEVICE_TIMEOUT.  With on_device the backward does not synchronise
 *   (except to read the fused kernels' error flags). */
int mlip_energy_forward(mlip_model* model, const double* pos, const int32_t* species, int64_t n,
                        const double cell[9], const uint8_t pbc[3], double* energy, int on_device, void* stream);
int mlip_energy_backward(mlip_model* model, const double* grad_energy, double* grad_pos, double* stress,
                         int on_device, void* stream);

/* Subsampled Hessian rows of a batch of systems (Sec. "Training with Hessian
 * labels": Eq. full_hessian, H_ij = d2E/dr_i dr_j = -dF_i/dr_j, and the rows of
 * Eq. sampled_hessian2).  For every row index rho = 0..R-1 and every system g
 * the row atom is row_atoms[g * R + rho] (an index within system g); the
 * summed force F_rho = sum_g F_{atom(g, rho)} is differentiated with respect to
 * all positions:
 *   rows[rho][a][j][b] = -dF_rho,a / dr_jb,   a, b = x, y, z, j = 0..n-1
 * (double[R][3][n][3], n the batch's total atom count).  Systems do not
 * interact, so each row is the concatenation of the systems' own rows (zero
 * outside system g for the part of g).  Computed on the GPU by
 * forward-over-reverse differentiation of the energy and its adjoint in FP32
 * dual numbers (the model's FP32 weights, whatever its precision form).
 *   atom_off [n_systems + 1], cells [n_systems][9], pbc [n_systems][3],
 *   row_atoms [n_systems][R]: host arrays; pos [n][3], species [n] and rows:
 *   host or device (on_device).
 * Errors: MLIP_ERR_INVALID_ARG (bad sizes, a row atom outside its system,
 * species out of range, a model with the symmetric contraction, gate or
 * charges, hidden width other than 64, more than 128 channels), MLIP_ERR_CELL,
 * MLIP_ERR_OOM, MLIP_ERR_CUDA.  Synchronises the stream. */
int mlip_hessian_rows(mlip_model* model, int32_t n_systems, const int64_t* atom_off, const double* pos,
                      const int32_t* species, const double* cells, const uint8_t* pbc, int32_t R,
                      const int32_t* row_atoms, double* rows, int on_device, void* stream);

/* Energy, forces and the corrected charges of one open system of total
 * charge total_charge (e) with a model built with charges = 1 (see
 * mlip_model_desc).  pos double[n][3], species int32[n]; energy double[1];
 * forces double[n][3] or NULL; charges double[n] or NULL.  Host or device
 * arrays as for mlip_energy_forces.  Errors: MLIP_ERR_INVALID_ARG (model
 * without charges, null or out-of-range inputs), MLIP_ERR_CUDA. */
int mlip_energy_forces_charged(mlip_model* model, const double* pos, const int32_t* species, int64_t n,
                               double total_charge, double* energy, double* forces, double* charges,
                               int on_device, void* stream);

/* Energy, forces and stress of a batch of independent systems in one call
 * (the batched inference of the Introduction): the systems are evaluated
 * together as one graph, the disjoint union of their neighbour graphs, so
 * many small systems fill the GPU like one large one.  System s owns atoms
 * [atom_off[s], atom_off[s+1]) of pos (double[n][3]) and species (int32[n]),
 * n = atom_off[n_systems]; cells: double[n_systems][9] (lattice rows), pbc:
 * uint8[n_systems][3].  energy: double[n_systems]; forces: double[n][3] or
 * NULL; stress: double[n_systems][9] or NULL (every system fully periodic,
 * else MLIP_ERR_CELL).  atom_off, cells and pbc are host arrays; pos, species
 * and the outputs are host or device arrays per on_device.  Every system must
 * have at least one atom.  A system's energy, forces and stress do not depend
 * on the other systems of the batch (per-system sums run over chunks counted
 * from the system's own first atom, and the 16-bit operand scale is chosen per
 * system).  Errors as mlip_energy_forces. */
int mlip_energy_forces_batch(mlip_model* model, int32_t n_systems, const int64_t* atom_off, const double* pos,
                             const int32_t* species, const double* cells, const uint8_t* pbc, double* energy,
                             double* forces, double* stress, int on_device, void* stream);

/* Velocity-Verlet NVE trajectory of one system (the batched MD
 * engines named in the Introduction and in "NPT ensemble
 * simulations"; NVE is the integrator of the benchmark workloads):
 *   v += dt/2 F/m kappa;  r += dt v;  F = F(r);  v += dt/2 F/m kappa,
 * kappa = 9.648533212e-3 (eV/A/amu -> A/fs^2), FP64 positions and velocities,
 * masses from the model description (per species).  pos, vel: [n][3] in/out
 * (A, A/fs).  pe, ke: n_steps + 1 potential / kinetic energies (eV; the start
 * and after every step) or NULL.  The neighbour list is rebuilt at every force
 * evaluation.  Errors: MLIP_ERR_INVALID_ARG (no masses, bad sizes, species out
 * of range), the errors of mlip_energy_forces. */
int mlip_md_nve(mlip_model* model, double* pos, double* vel, const int32_t* species, int64_t n,
                const double cell[9], const uint8_t pbc[3], double dt_fs, int64_t n_steps, double* pe,
                double* ke, int on_device, void* stream);

/* Velocity-Verlet NVE trajectories of a batch of independent systems (the
 * replicas of a batched MD run) advanced together: every step evaluates all
 * systems as one graph (see mlip_energy_forces_batch) with the same time step.
 * atom_off, cells, pbc as in mlip_energy_forces_batch (host arrays); pos, vel:
 * [n][3] in/out; species [n]; pe, ke: [n_steps + 1][n_systems] (row k: after
 * step k) or NULL.  Each system's trajectory equals mlip_md_nve on that system
 * alone.  Errors as mlip_md_nve. */
int mlip_md_nve_batch(mlip_model* model, int32_t n_systems, const int64_t* atom_off, double* pos, double* vel,
                      const int32_t* species, const double* cells, const uint8_t* pbc, double dt_fs,
                      int64_t n_steps, double* pe, double* ke, int on_device, void* stream);

/* Options of the skin-list MD driver. */
typedef struct {
  double skin;            /* A added to the cutoff for the candidate list (> 0) */
  int32_t rebuild_every;  /* steps per block: the candidate list is rebuilt before every block (>= 1) */
  int32_t use_graph;      /* 1: capture the steps of a block as one CUDA graph and replay it for later
                             blocks; 0: launch them one by one (same kernels, same results) */
} mlip_md_options;

/* What the skin-list driver did. */
typedef struct {
  int64_t builds;          /* candidate-list builds */
  int64_t redone_blocks;   /* blocks run again with a fresh list at every step (an atom moved > skin/2) */
  int64_t graph_captures;  /* CUDA graphs captured */
  int64_t graph_launches;  /* graph replays */
  int64_t max_candidates;  /* largest candidate count of a build */
  double max_displacement; /* largest displacement from the positions of the last build (A) */
} mlip_md_report;

/* mlip_md_nve_batch with a skin neighbour list (the batched MD workload): the
 * pairs within rc + skin are listed before every block of rebuild_every steps
 * and compacted at every step to the pairs within rc (in the list's canonical
 * order), so no cell-list build runs inside a block and a block's launches
 * have fixed sizes, which lets them be captured as one CUDA graph.  If an atom
 * moves more than skin/2 from its position at the block's build, the block is
 * run again from its start with a fresh list at every step, so the trajectory
 * equals mlip_md_nve_batch's bit for bit in every case.  Needs a 16-bit
 * (fused) model.  opt NULL: skin 2 A, rebuild every 10 steps, graphs on.
 * report nullable.  Runs on a stream of its own ordered after `stream`;
 * returns after the trajectory is complete.  Errors as mlip_md_nve_batch, and
 * MLIP_ERR_INVALID_ARG for a 32-bit model or bad options. */
int mlip_md_nve_skin(mlip_model* model, int32_t n_systems, const int64_t* atom_off, double* pos, double* vel,
                     const int32_t* species, const double* cells, const uint8_t* pbc, double dt_fs,
                     int64_t n_steps, const mlip_md_options* opt, double* pe, double* ke, mlip_md_report* report,
                     int on_device, void* stream);

/* ------------------------------------------------------------- serving
 * Continuous batching of independent requests (the paper's batched
 * inference and MD serving, Introduction and "NPT ensemble simulations"):
 * a worker thread owns one CUDA stream and, at every iteration, evaluates
 * all running requests together as one graph (mlip_energy_forces_batch).
 * An energy+forces request runs for one iteration; an NVE request runs for
 * n_steps + 1 (the start and one per velocity-Verlet step).  After every
 * iteration finished requests leave the batch and queued requests join it
 * (first in, first out) while the batch stays within max_slots requests and
 * the device-memory budget.  A request's results do not depend on the other
 * requests it shared batches with.
 *
 * Ownership: the server uses the model exclusively while it exists (do not
 * call other functions on the model meanwhile; free the model after
 * mlip_serve_destroy).  Submit copies the inputs.  Result arrays belong to
 * the server and stay valid until mlip_serve_release of that id (or
 * destroy).  submit, poll, wait, release and stats may be called from any
 * thread. */
typedef struct mlip_server mlip_server;

enum { MLIP_REQ_ENERGY_FORCES = 0, MLIP_REQ_NVE = 1 };

typedef struct {
  int64_t hbm_budget_bytes;   /* device memory for batches (estimated per atom and
                                 edge); 0: 80 % of the free memory at create */
  int32_t max_slots;          /* most requests in one batch; 0: 512 */
  int32_t n_buckets;          /* size classes of the latency statistics, 0..8 */
  int64_t bucket_edges[8];    /* ascending upper atom counts of the classes (the
                                 last class takes every larger request) */
  int64_t device_poll_limit_us; /* longest host wait (microseconds) for one
                                 iteration's results; exceeded: the batch's
                                 requests fail with MLIP_ERR_DEVICE_TIMEOUT and
                                 the server admits nothing more.  0: no limit */
  int32_t resident_after;     /* a batch of NVE requests keeps a skin neighbour
                                 list on the device once its members have stayed
                                 the same for this many iterations (0: 3;
                                 negative: never, a fresh list every iteration) */
  int32_t reserved;           /* 0 */
} mlip_serve_config;

typedef struct {
  int32_t kind;               /* MLIP_REQ_ENERGY_FORCES or MLIP_REQ_NVE */
  int32_t want_stress;        /* energy+forces: also the stress (fully periodic cell) */
  int64_t n;                  /* atoms, >= 1 */
  const double* pos;          /* host [n][3], A */
  const int32_t* species;     /* host [n], 0..n_species-1 */
  double cell[9];             /* lattice rows (ignored without a periodic axis) */
  uint8_t pbc[3];
  const double* vel;          /* NVE: host [n][3] A/fs, or NULL: Maxwell-Boltzmann at
                                 temperature_K from seed (SplitMix64 normals by
                                 Box-Muller, centre-of-mass velocity removed) */
  double temperature_K;
  uint64_t seed;
  int64_t n_steps;            /* NVE: velocity-Verlet steps, >= 0 */
  double dt_fs;               /* NVE: time step (fs), > 0 */
} mlip_request;

typedef struct {
  int32_t status;             /* MLIP_OK or the error that ended this request */
  int32_t kind;
  int64_t n, n_steps;
  double energy;              /* energy (NVE: potential energy at the end) */
  double stress[9];           /* when requested */
  const double* forces;       /* [n][3] (NVE: at the end) */
  const double* pos;          /* NVE: final positions [n][3]; NULL otherwise */
  const double* vel;          /* NVE: final velocities [n][3] */
  const double* pe;           /* NVE: potential energy at the start and after every step [n_steps + 1] */
  const double* ke;           /* NVE: kinetic energy, same points */
  double t_arrive, t_admit, t_done;  /* seconds on the server's clock (0 = create) */
} mlip_result;

typedef struct {
  int64_t submitted, completed, failed, rejected, queued, running;
  int64_t iterations;         /* batched force evaluations */
  int64_t atom_evals;         /* sum over iterations of the atoms evaluated */
  double elapsed_s;           /* server clock now */
  double busy_s;              /* worker time inside iterations */
  double atom_steps_per_s;    /* atom_evals / busy_s */
  double p50_ms, p99_ms, mean_ms, max_ms;  /* t_done - t_arrive of completed requests */
  double mean_batch_atoms, mean_batch_requests;
  int64_t device_bytes;       /* device memory held by the server and the model's workspace */
  int32_t n_buckets;
  int64_t bucket_count[9];
  double bucket_p50_ms[9], bucket_p99_ms[9];
  int64_t skin_steps;         /* MD steps evaluated on the resident skin neighbour list (no rebuild) */
  int64_t skin_builds;        /* skin list builds: a batch of NVE requests kept its members, or an atom left its skin */
  int64_t changed_iterations; /* iterations whose membership differed from the previous one's (compaction, new layout) */
  double changed_busy_s;      /* worker time inside those iterations (busy_s includes it) */
} mlip_serve_statistics;

/* Starts the worker.  Errors: MLIP_ERR_INVALID_ARG (bad config: max_slots < 0,
 * n_buckets outside 0..8, edges not ascending), MLIP_ERR_CUDA. */
int mlip_serve_create(mlip_model* model, const mlip_serve_config* config, mlip_server** out);
/* Validates and copies a request and queues it; *id identifies it.  Errors:
 * MLIP_ERR_INVALID_ARG (sizes, species, non-finite input, NVE without masses),
 * MLIP_ERR_CELL (stress without a fully periodic cell, singular cell),
 * MLIP_ERR_BUDGET (the request alone exceeds the memory budget),
 * MLIP_ERR_DEVICE_TIMEOUT (the server stopped after a device timeout). */
int mlip_serve_submit(mlip_server* server, const mlip_request* req, uint64_t* id);
/* MLIP_OK and *out filled when the request has ended (out->status tells how);
 * MLIP_PENDING while it is queued or running; MLIP_ERR_NOT_FOUND for an
 * unknown or released id. */
int mlip_serve_poll(mlip_server* server, uint64_t id, mlip_result* out);
/* As poll, but waits up to timeout_ms (< 0: no limit) for the end; returns
 * MLIP_ERR_TIMEOUT if the request is still pending then. */
int mlip_serve_wait(mlip_server* server, uint64_t id, int64_t timeout_ms, mlip_result* out);
/* Frees an ended request's results (MLIP_PENDING if it has not ended). */
int mlip_serve_release(mlip_server* server, uint64_t id);
int mlip_serve_stats(mlip_server* server, mlip_serve_statistics* out);
/* Stops admitting, finishes the running iteration, fails queued and running
 * requests with MLIP_ERR_TIMEOUT, joins the worker and frees the server. */
int mlip_serve_destroy(mlip_server* server);

/* Self test of a hardware path (no counterpart in the paper).  which = 1: one
 * tcgen05 tile product (M = 128, N = 32, K = 64, BF16 operands in the
 * shared-memory layout the fused kernels use, FP32 accumulation in tensor
 * memory) against a host FP64 product; *result = max |error| / max |value|.
 * which = 2, 3: the transposed product of the adjoint (A read M-major from the
 * forward weight image, K = 128), with the two possible assignments of the
 * descriptor's leading/stride offsets; the kernels use the one that passes.
 * Errors: MLIP_ERR_INVALID_ARG (unknown test), MLIP_ERR_DEVICE_TIMEOUT (the
 * MMA completion wait ran out), MLIP_ERR_CUDA. */
int mlip_selftest(int which, double* result);

/* Tracing (no counterpart in the paper; used by the benchmark).
 * mlip_launch_count: number of kernels the library has launched in this
 *   process (monotone counter).
 * mlip_profile_enable(1): from now on every kernel launch records a pair of
 *   CUDA events on its stream (clears earlier records); 0 stops recording.
 *   Do not enable it while a stream is being captured into a CUDA graph.
 *   Evaluations replayed as CUDA graphs carry their event pairs as event
 *   nodes and are timed too (the graph is captured again when the timing
 *   configuration changes).
 * mlip_profile_report: writes a NUL-terminated JSON object
 *   {"kernels": {"<name>": [launches, total_ms], ...}} for the records since
 *   the last enable into buf (at most cap bytes); *needed receives the full
 *   size.  It synchronises on the recorded events.  Errors: MLIP_ERR_CUDA. */
int mlip_profile_enable(int on);
long long mlip_launch_count(void);
int mlip_profile_report(char* buf, long long cap, long long* needed);
/* mlip_profile_select("name,name"): time only the kernels with these names
 * (NULL or "": all); launches are still counted. */
int mlip_profile_select(const char* names);

/* Measured FP32 FMA throughput of the current device (no counterpart in the
 * paper; the denominator of the FP32-ALU roofline the benchmark reports).
 * Launches one grid of independent FMA chains filling every SM (the SM count
 * is read from the device) after one shorter warm-up launch, and times it with
 * CUDA events on the default stream.  iters: loop trips per thread (each 256
 * FMAs); 20000 runs for about 50 ms on a GB300.  *tflops receives 2 x FMAs /
 * seconds / 1e12; *ms (nullable) the timed duration; *sms (nullable) the SM
 * count.  It allocates and frees a small sink buffer and synchronises the
 * device's default stream.  Errors: MLIP_ERR_INVALID_ARG, MLIP_ERR_CUDA. */
int mlip_fp32_fma_rate(int iters, double* tflops, double* ms, int* sms);

#ifdef __cplusplus
}
#endif

#endif /* MLIP_H */
