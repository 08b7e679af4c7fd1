/*
 * allegro.h - C ABI of the GB300 Allegro energy/force library.
 *
 * The library evaluates the Allegro-shaped interatomic potential of
 * "Allegro-Legato" (arXiv 2303.08169) on one GPU: periodic cell-list
 * neighbour search, per-pair Bessel x envelope radial basis and real
 * spherical harmonics, channel-wise Clebsch-Gordan tensor products with
 * per-atom neighbour sums, latent and energy per-pair MLPs, the energy
 * E = sum_ij E_ij (Sec. 2.1) and the forces f_i = -dE/dr_i (Eq. 1) from
 * hand-written adjoint kernels, plus microcanonical velocity-Verlet steps
 * (Sec. 3.2) with the per-step count of force components above 5 sigma
 * (Fig. 1 caption).
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: ALLEGRO_OK (0) or one of the
 *    ALLEGRO_E_* codes below; allegro_last_error() then holds a message.
 *    No C++ exception crosses this boundary and no call aborts the process.
 *  - Units: Angstrom, eV, fs, amu.  Forces in eV/Angstrom.
 *  - Arrays marked "host or device" may be either: the library inspects the
 *    pointer (cudaPointerGetAttributes) and copies host data through its own
 *    stream.  Arrays marked "device" must be device memory of the current
 *    GPU.  The caller owns every array it passes; the library never keeps a
 *    caller pointer after a call returns.
 *  - Row-major layouts: positions/velocities/forces are N x 3 (x, y, z per
 *    atom).  cell is a host 3 x 3 matrix of lattice vectors (rows); only
 *    orthorhombic (diagonal) cells are accepted.
 *  - All GPU work is enqueued on the context's stream (allegro_set_stream,
 *    default: the legacy default stream); calls that return host values
 *    synchronise that stream before returning.
 *  - One context per host thread; contexts are independent.
 */
#ifndef ALLEGRO_GB300_H
#define ALLEGRO_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ALLEGRO_OK                 0
#define ALLEGRO_E_INVALID_ARG      1  /* null pointer, negative size, bad enum   */
#define ALLEGRO_E_MISMATCH         2  /* create() arguments disagree with blob   */
#define ALLEGRO_E_CUTOFF_TOO_LARGE 3  /* r_cut needs images beyond |n_a| <= 2    */
#define ALLEGRO_E_NONORTHO_CELL    4  /* cell has off-diagonal entries or L <= 0 */
#define ALLEGRO_E_PAIR_OVERFLOW    5  /* pair capacity exceeded (context grows;  */
                                      /* retry the call)                         */
#define ALLEGRO_E_OOM              6  /* device allocation failed                */
#define ALLEGRO_E_NONFINITE        7  /* non-finite position or force            */
#define ALLEGRO_E_TIMEOUT          8  /* a bounded device wait gave up           */
#define ALLEGRO_E_CUDA             9  /* any other CUDA runtime error            */
#define ALLEGRO_E_UNSUPPORTED     10  /* model shape outside the compiled set    */
#define ALLEGRO_E_BLOB            11  /* malformed weights blob                  */

#define ALLEGRO_FP32 0   /* every per-pair GEMM in FP32 on CUDA cores           */
#define ALLEGRO_BF16 1   /* per-pair GEMMs on tensor cores, BF16 operands,      */
                         /* FP32 accumulation (C 16, D 128, E 32, 2+ layers)    */
#define ALLEGRO_FP16 2   /* same tensor-core path with FP16 operands            */
#define ALLEGRO_FP16_SPLIT 3  /* FP16 operands; the two-body MLP and the energy   */
                         /* hidden layer with split operands x = hi + lo, three */
                         /* MMAs per product (about twice the mantissa bits)    */

typedef struct allegro_ctx allegro_ctx;

/* Library version string, static storage. */
const char* allegro_version(void);

/*
 * Create a context from an "ALW1" weights blob (layout documented in
 * synth/weights.py: header, per-species sigma_Z/mu_Z, named FP64 tensors).
 *  weights_blob, blob_bytes : host bytes; copied, the caller keeps ownership.
 *  species_mass             : host, n_species masses in amu (index = type id);
 *                             used only by the MD entry points.
 *  r_cut, l_max, n_layers   : must equal the blob header (else E_MISMATCH).
 * Supported model shapes (E_UNSUPPORTED otherwise): two species, 8 Bessel
 * functions, envelope p = 6, two latent hidden widths D = D, one energy
 * hidden width, and (l_max, C, D, E) in {(1, 8, 32, 32), (0, 16, 128, 32),
 * (1, 16, 128, 32), (2, 16, 128, 32)} (the last three: the l_max sweep of
 * Table 2 at one width, in every precision; the tensor-core precisions need
 * at least two layers).  The header's parity flag: 0 (natural-parity coupling
 * paths) or 1 (full O(3): parity-odd paths and pseudotensor features, Sec. 2.1
 * E(3) equivariance including inversion).  With at most two layers (or
 * l_max 0) the odd paths cannot reach the energy (a pseudotensor gives a true
 * scalar only through a second odd path, and no path into l = 0 is odd), so
 * the model computed is the natural-parity one and the pseudotensor mixing
 * matrices are not loaded (nor part of the weight vector); every precision
 * runs it.  From three layers on (l_max 1 or 2) the FP32 passes run the
 * full-O(3) model: features of both parities per channel, every even and odd
 * coupling path, one mixing matrix per output irrep (l, s), each with one
 * column per path of the irreps its layer receives (else E_BLOB); the
 * tensor-core precisions and training are E_UNSUPPORTED for it.  An
 * out-of-range flag is E_BLOB.
 * The paper defines only the pairwise-energy decomposition and equivariance
 * (Sec. 2.1); the layer structure follows the Allegro reading stated in the
 * oracle package.
 */
int allegro_create(const void* weights_blob, size_t blob_bytes,
                   const double* species_mass, int32_t n_species,
                   double r_cut, int32_t l_max, int32_t n_layers,
                   allegro_ctx** out);

/* Free a context and all device memory it owns.  NULL is ignored. */
void allegro_destroy(allegro_ctx* ctx);

/* Enqueue all later work on this cudaStream_t (NULL = legacy stream). */
int allegro_set_stream(allegro_ctx* ctx, void* cuda_stream);

/* Message of the last failing call on this context (static if ctx NULL). */
const char* allegro_last_error(const allegro_ctx* ctx);

/*
 * Build the periodic neighbour list (Sec. 2.4 linked-list cells + adjacency
 * list) for n_atoms positions and keep it in the context.
 *  positions : host or device, N x 3 FP64.
 *  cell      : host 3 x 3 FP64 (orthorhombic).
 *  n_pairs   : host out, number of ordered pairs (i, j, n).
 * A pair is (i, j, n) with n in Z^3, (j, n) != (i, 0), and
 * d^2 = (Dx^2 + Dy^2) + Dz^2 < r_cut^2 in FP64 without fused multiply-add,
 * where D = (w_j - w_i) + n L and w are positions wrapped into [0, L).
 * Every periodic image counts, so r_cut may exceed L/2 (up to 2 L).
 */
int allegro_build_neighbors(allegro_ctx* ctx, int64_t n_atoms,
                            const double* positions, const double* cell,
                            int64_t* n_pairs);

/*
 * Copy the last neighbour list out, in CSR form sorted by (i, j, n_x, n_y,
 * n_z).  All outputs device, caller-allocated; any may be NULL.
 *  row_ptr : N + 1 int32;  col : P int32 (j);  img : P x 3 int8 (n);
 *  rev     : P int32, index of the reverse pair (j, i, -n).
 */
int allegro_get_neighbors(allegro_ctx* ctx, int32_t* row_ptr, int32_t* col,
                          int8_t* img, int32_t* rev);

/*
 * Energy and forces (Sec. 2.1, Eq. 1): rebuilds the neighbour list, runs the
 * forward pair passes, the energy reduction (FP64) and the hand-written
 * adjoint passes.
 *  positions    : host or device, N x 3 FP64.
 *  species      : host or device, N int32 in [0, n_species).
 *  cell         : host 3 x 3 FP64 (orthorhombic).
 *  energy_out   : host, total energy E (FP64).
 *  forces_out   : host or device, N x 3 FP32 = -dE/dr (may be NULL).
 *  atom_energy  : host or device, N FP64 per-atom energies E_i (may be NULL).
 *  precision    : ALLEGRO_FP32, ALLEGRO_BF16, ALLEGRO_FP16 or
 *                 ALLEGRO_FP16_SPLIT (the tensor-core modes: E_UNSUPPORTED
 *                 unless l_max <= 2, C = 16, D = 128, E = 32, at least two
 *                 layers, and natural parity or at most two layers).
 * On ALLEGRO_E_PAIR_OVERFLOW nothing is written; the context has grown and
 * the call may simply be repeated.  The call reuses the MD state's buffers:
 * allegro_md_init again before the next allegro_md_step_* (which otherwise
 * returns ALLEGRO_E_INVALID_ARG).  The ring-polymer state is kept.
 */
int allegro_energy_forces(allegro_ctx* ctx, int64_t n_atoms,
                          const double* positions, const int32_t* species,
                          const double* cell, double* energy_out,
                          float* forces_out, double* atom_energy,
                          int32_t precision);

/*
 * Count force components above threshold * sigma, sigma^2 = mean of F_ia^2
 * over all 3N components (Fig. 1 caption, ">5 sigma" with threshold 5).
 *  forces : host or device, N x 3 FP32.   count_out : host.
 */
int allegro_outlier_count(allegro_ctx* ctx, int64_t n_atoms,
                          const float* forces, double threshold,
                          int64_t* count_out);

/*
 * Load the MD state (copied into the context).
 *  positions, velocities : host or device, N x 3 FP64 (A, A/fs).
 *  species               : host or device, N int32.
 *  cell                  : host 3 x 3 FP64 (orthorhombic).
 * Computes the initial forces with the current precision
 * (allegro_set_md_precision, default ALLEGRO_FP32).
 */
int allegro_md_init(allegro_ctx* ctx, int64_t n_atoms, const double* positions,
                    const double* velocities, const int32_t* species,
                    const double* cell);

/* Precision used by allegro_md_init / allegro_md_step_nve. */
int allegro_set_md_precision(allegro_ctx* ctx, int32_t precision);

/*
 * Verlet-skin reuse of the neighbour list in the MD steps (Sec. 3.2 runs
 * long NVT and NVE trajectories; reusing the list between rebuilds is the
 * classical way to amortise its cost).  skin_A in [0, r_cut] A, 0 (the
 * default) rebuilding every step.  With skin_A > 0 the list of the MD state
 * holds every pair within r_cut + skin_A; each step of allegro_md_step_nve /
 * _nvt rebuilds it only when some atom has moved by more than skin_A / 2
 * (minimum image) since the last build, and at the first step of every call.
 * Pairs beyond r_cut contribute exactly zero (the envelope vanishes there),
 * so results equal those of per-step rebuilds up to FP32 summation order.
 * Takes effect at the next allegro_md_init; ring-polymer steps always
 * rebuild.  ALLEGRO_E_INVALID_ARG outside the range; allegro_md_init returns
 * ALLEGRO_E_CUTOFF_TOO_LARGE when r_cut + skin exceeds twice a cell length.
 * The builds since allegro_md_init: allegro_query(ALLEGRO_Q_REBUILDS).
 */
int allegro_set_skin(allegro_ctx* ctx, double skin_A);

/*
 * n_steps microcanonical velocity-Verlet steps of dt_fs each (Eq. 1,
 * Sec. 3.2): v += dt/2 a; r += dt v; wrap; F = F(r); v += dt/2 a with
 * a = kappa F / m, kappa = 9.648533e-3 A/fs^2 per eV/(A amu), in FP64.
 * After each step the step's outlier count (> 5 sigma) and its energies are
 * recorded.  One step is captured once as a CUDA graph and replayed.
 *  outlier_counts : host or device, n_steps int64 (may be NULL).
 *  energies       : host or device, n_steps x 3 FP64 (E_pot, E_kin, E_tot),
 *                   may be NULL.
 * On ALLEGRO_E_PAIR_OVERFLOW the state is rolled back to the start of the
 * call, the capacity is grown, and the call may be repeated.
 */
int allegro_md_step_nve(allegro_ctx* ctx, double dt_fs, int32_t n_steps,
                        int64_t* outlier_counts, double* energies);

/*
 * Copy the MD state out.  positions, velocities: host or device N x 3 FP64
 * (positions wrapped into the cell); forces: host or device N x 3 FP32;
 * step: host.  Any pointer may be NULL.
 */
int allegro_md_get_state(allegro_ctx* ctx, double* positions,
                         double* velocities, float* forces, int64_t* step);

/*
 * The outlier count of allegro_outlier_count without allocating device
 * memory, for callers that cannot allocate: applications whose own allocator
 * holds all device memory (a foreign cudaMalloc fails or fragments their
 * pool), and latency-bound loops where cudaMalloc/cudaFree would synchronise
 * the device.  The paper has no counterpart; this is a deployment
 * convenience.
 *  n_atoms   : 1 .. 4,194,304 (the fixed scratch size), else
 *              ALLEGRO_E_INVALID_ARG with a message in allegro_last_error(NULL).
 *  forces    : device, N x 3 FP32.
 *  threshold : count components with |F| > threshold * sigma (5 for >5 sigma).
 *  count_out : device, one int64, written asynchronously on the stream.
 *  cuda_stream : cudaStream_t (NULL = legacy default stream); the call only
 *              enqueues kernels, synchronise before reading count_out.
 * The reduction scratch is a fixed 256 KB array in device global memory that
 * every GPU loading the library keeps until the process exits.  All calls
 * share it and it keeps the last call's contents; every kernel overwrites the
 * slots it later reads, so nothing needs clearing, but calls that overlap on
 * the GPU (different streams, or different host threads on one device) race
 * on it and must be serialised by the caller.  The first call on each device
 * (and again after the device's CUDA context changed, e.g. after
 * cudaDeviceReset) looks the array's device address up (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * A CUDA error left pending by the caller's earlier work is reported as
 * ALLEGRO_E_CUDA without being cleared, and nothing is launched.
 */
int allegro_outlier_count_noalloc(int64_t n_atoms, const float* forces, double threshold,
                                  int64_t* count_out, void* cuda_stream);

/*
 * A batch of structures for training (SAM, Eq. 3).  All arrays host.
 *  atom_offset : n_structs + 1, structure k owns atoms [off[k], off[k+1]).
 *  positions   : N_tot x 3 FP64;  species: N_tot int32;
 *  cells       : n_structs x 9 FP64 (orthorhombic, row-major 3 x 3);
 *  e_target    : n_structs FP64 target energies;  f_target: N_tot x 3 FP32.
 */
typedef struct allegro_batch {
  int32_t n_structs;
  const int64_t* atom_offset;
  const double* positions;
  const int32_t* species;
  const double* cells;
  const double* e_target;
  const float* f_target;
} allegro_batch;

/*
 * Loss and its weight gradient (FP32 passes).  Loss (per-atom MSE, Table 5,
 * weights as arguments):
 *   L = (w_energy / B) sum_b ((E_b - E*_b) / N_b)^2
 *       + (w_force / (3 sum_b N_b)) sum |F - F*|^2.
 * The gradient is the hand-written weight adjoint of the pair passes; the
 * force term's mixed derivative -d/dw (v . dE/dr), v = dL/dF, is a central
 * difference of that adjoint along v (displacement at most 0.01 A).
 *  loss_out : host (may be NULL);  grad_out: host or device, n_params FP32 in
 *  blob order (may be NULL; see ALLEGRO_Q_N_PARAMS).
 * Models of at most two layers (E_UNSUPPORTED otherwise).
 */
int allegro_loss_grad(allegro_ctx* ctx, const allegro_batch* batch, double w_energy, double w_force,
                      double* loss_out, float* grad_out);

/*
 * One sharpness-aware minimisation step (Eq. 3) with Adam as the base
 * optimizer (Table 5: beta = (0.9, 0.999), eps = 1e-8):
 *   g = grad L(w);  w' = w + rho g / ||g|| (w' = w if g = 0);
 *   g' = grad L(w');  w <- Adam(w, g') with step size lr.
 * Updates the context's weights and Adam state.  loss_out: host, L(w).
 */
int allegro_sam_train_step(allegro_ctx* ctx, const allegro_batch* batch, double rho, double lr,
                           double w_energy, double w_force, double* loss_out);

/*
 * Loss landscape around the current weights w (the sharpness of Eq. 2 and its
 * measurement in Sec. 5.4, Table 4 and Fig. 5): for k < n_points the loss of
 * the batch (as allegro_loss_grad, weights w_energy, w_force) at
 *   w_k = w + scales[k] d_k,   d_k = dirs + k dir_stride,
 * into losses_out[k].  The sharpness estimate max_k L(w + eps_k) - L(w) over
 * random eps_k of norm rho takes d_k = eps_k, scales 1 (and one point with
 * scale 0 for L(w)); the one-dimensional surface L(w + p d), p in [-1, 1],
 * takes dir_stride 0 and scales p.  The random directions are the caller's.
 * dirs: device FP32, n_params per direction; dir_stride: elements between
 * directions (0: the same direction for every point); scales, losses_out:
 * host, n_points >= 1.  One forward energy+force evaluation of the batch per
 * point (FP32 passes), no gradient.  The context's weights and Adam state
 * are unchanged on return (the MD graph is re-captured at the next step).
 * Models of at most two layers (E_UNSUPPORTED otherwise).
 */
int allegro_loss_scan(allegro_ctx* ctx, const allegro_batch* batch, const float* dirs, int64_t dir_stride,
                      const double* scales, int32_t n_points, double w_energy, double w_force, double* losses_out);

/* The trainable weights as one FP32 vector in blob order (every weight
 * matrix row-major, sigma/mu excluded); host or device, n = n_params. */
int allegro_get_weights(allegro_ctx* ctx, float* out, int64_t n);
/* Replace the weights (host or device input) and reset the Adam state (moments
 * zero, step count 0): the next SAM step is the first of a new run. */
int allegro_set_weights(allegro_ctx* ctx, const float* in, int64_t n);

/*
 * NVT steps (the paper equilibrates at 200 K before its NVE runs, Sec. 3.2;
 * its thermostat is not named: here Nose-Hoover): each step is a thermostat
 * half step (dt/2), the velocity-Verlet step of allegro_md_step_nve, and a
 * thermostat half step, in FP64, with g = 3N degrees of freedom, thermostat
 * mass Q = g kB T tau^2 and the time-reversible half step
 *   xi += (h/2) G;  v *= exp(-xi h);  eta += xi h;  xi += (h/2) G,
 *   G = (2 K - g kB T) / Q,  h = dt / 2,
 * K the kinetic energy at that point.  temperature_K > 0, tau_fs > 0 (the
 * thermostat period).  outlier_counts: host or device int64[n_steps] or
 * NULL; energies: host or device FP64[n_steps x 4] (E_pot, E_kin, E_tot, H)
 * or NULL, H = E_pot + K + Q xi^2 / 2 + g kB T eta the conserved extended
 * energy.  The thermostat state (xi, eta) persists across calls and is reset
 * to zero by allegro_md_init.  Errors and pair-capacity growth as
 * allegro_md_step_nve.
 */
int allegro_md_step_nvt(allegro_ctx* ctx, double dt_fs, int32_t n_steps, double temperature_K, double tau_fs,
                        int64_t* outlier_counts, double* energies);
/* The thermostat state (xi in 1/fs, eta) into host or device xi_eta[2]. */
int allegro_md_get_thermostat(allegro_ctx* ctx, double* xi_eta);

/*
 * Ring-polymer (path-integral) MD, the nuclear-quantum-effect workload of
 * Sec. 6 (Fig. 6): every atom is P replicas (beads) coupled by harmonic
 * springs along a closed ring, at P times the physical temperature,
 *   H_P = sum_k [ sum_i m_i |v_ik|^2 / 2 + V(q_k) ]
 *         + sum_i sum_k m_i omega_P^2 |q_ik - q_i,k+1|^2 / 2,
 *   omega_P = P kB T / hbar,  replica P + 1 = replica 1.
 * The paper states neither the equations nor the integrator; this is the
 * standard form, integrated by velocity Verlet with the spring part solved
 * exactly in the normal modes of the ring (frequencies 2 omega_P sin(k pi / P)).
 * The energies and forces of all P replicas come from ONE neighbour build and
 * ONE pass sequence over all P n atoms, in the precision set by
 * allegro_set_md_precision.
 *
 * allegro_pimd_init: n_beads in [1, 64], n_atoms >= 1; positions and
 * velocities host or device FP64[n_beads x n_atoms x 3], replica-major
 * (replica k's atom i at (k n_atoms + i) x 3), in A and A/fs; species host or
 * device int32[n_atoms] (shared by the replicas); cell host FP64[9]
 * (orthorhombic, as allegro_build_neighbors); temperature_K > 0.  Bead
 * positions are not wrapped (the neighbour build wraps them), so the springs
 * are plain differences.  Evaluates the forces once; copies the inputs.  The
 * ring state (positions, velocities, forces) lives in its own arrays and
 * survives other calls; allegro_pimd_init and allegro_pimd_step end the
 * single-system MD state (allegro_md_init again before allegro_md_step_*).
 *
 * allegro_pimd_step: n_steps >= 0 steps of dt_fs > 0 (one captured CUDA
 * graph per step: one neighbour build for all replicas, each replica its own
 * system in the common box, then the pair passes over all replicas):
 *   v += dt/2 F/m;  free ring evolution for dt;  F <- F(q);  v += dt/2 F/m,
 * energies: host or device FP64[n_steps x 3] or NULL: (mean replica energy
 * sum_k V(q_k) / P, kinetic energy of all replicas, H_P) in eV after each
 * step.  Pair-capacity overflow rolls the ring back to the start of the
 * call, grows the context and repeats (ALLEGRO_E_PAIR_OVERFLOW only if growth
 * fails); after ALLEGRO_E_NONFINITE the ring state is undefined
 * (allegro_pimd_init again).
 *
 * allegro_pimd_get_state: positions, velocities host or device
 * FP64[n_beads x n_atoms x 3] (either may be NULL).
 */
int allegro_pimd_init(allegro_ctx* ctx, int32_t n_beads, int64_t n_atoms, const double* positions,
                      const double* velocities, const int32_t* species, const double* cell, double temperature_K);
int allegro_pimd_step(allegro_ctx* ctx, double dt_fs, int32_t n_steps, double* energies);
int allegro_pimd_get_state(allegro_ctx* ctx, double* positions, double* velocities);

/* Keys of allegro_query. */
#define ALLEGRO_Q_N_PAIRS      0  /* ordered pairs of the last neighbour build   */
#define ALLEGRO_Q_CAPACITY     1  /* pair capacity currently allocated           */
#define ALLEGRO_Q_STEP_KERNELS 2  /* kernel launches in one captured MD step     */
#define ALLEGRO_Q_N_ATOMS      3  /* atoms of the current state                  */
#define ALLEGRO_Q_N_PARAMS     4  /* trainable parameters (weights vector length) */
#define ALLEGRO_Q_RP_STEP_KERNELS 5  /* kernel launches in one ring-polymer step */
#define ALLEGRO_Q_BATCH_PAIRS  6  /* ordered pairs of the last training batch     */
#define ALLEGRO_Q_REBUILDS     7  /* skin: neighbour builds since allegro_md_init  */
/* Launch shapes the autotuner chose for the FP32 pass kernels (value passes;
 * tangent passes of the training step): 4 bits per pass in the order A, B, C,
 * B^T, A^T from the lowest, each the number of waves of one block per SM
 * (1, 2, 4 or 8; 8 before the first tuning).  Tuning runs on the first FP32
 * evaluation of a context (and again when the pair capacity has more than
 * doubled); the results do not depend on the launch shape. */
#define ALLEGRO_Q_FP32_LAUNCH   8
#define ALLEGRO_Q_TANGENT_LAUNCH 9

/* Read one integer property of the context into *value (host). */
int allegro_query(allegro_ctx* ctx, int32_t what, int64_t* value);

/*
 * Instrumentation (not part of the paper's method): mean device time in ms of
 * each phase of one energy+forces evaluation at the current MD state, over
 * n_reps evaluations timed with CUDA events on the context stream:
 *   ms_out[0] neighbour build   [1] pass A (two-body)   [2] passes B (layers
 *   below the last)   [3] pass C (last layer + energy, forward and adjoint)
 *   [4] passes B^T   [5] pass A^T (+ geometry adjoint)   [6] force assembly
 *   and reductions.  With n_out >= 9, the two kernels of each forward layer
 *   pass of the tensor-core path, summed over layers: [7] B1 (tensor product
 *   + mixing)  [8] B2 (latent MLP + env); the FP32 path has one kernel per
 *   layer pass ([7] = [2], [8] = 0).  The layer adjoint B^T is one kernel in
 *   both paths.
 * ms_out: host, n_out >= 7.  The MD state is unchanged (the evaluation is
 * deterministic).  Requires allegro_md_init.
 */
int allegro_phase_times(allegro_ctx* ctx, int32_t n_reps, double* ms_out, int32_t n_out);

/*
 * Diagnostic (not part of the paper's method): one 128 x n tile GEMM
 * D = bf16(A) bf16(B)^T with FP32 accumulation, run through the same
 * tensor-core building blocks (tcgen05.mma, swizzled shared-memory operands,
 * TMEM accumulator) as the BF16 pair passes, for checking them against a
 * host reference.  a: device 128 x k FP32; b: device n x k FP32; d: device
 * 128 x n FP32 (row-major).  16 <= n <= 256, n % 16 == 0, 16 <= k <= 256,
 * k % 16 == 0, else ALLEGRO_E_INVALID_ARG; ALLEGRO_E_TIMEOUT if the bounded
 * wait for the MMA gave up.  Runs on the legacy default stream and
 * synchronises.
 */
int allegro_selftest_mma(int32_t n, int32_t k, const float* a, const float* b, float* d);

/*
 * Same diagnostic with the B-operand form selectable: mode 0 is the call
 * above; mode 1 computes d = bf16(a) (128 x k) bf16(b) (k x n, row-major),
 * reading the K-major image of b as an MN-major operand (the form the BF16
 * adjoint passes use to apply W^T without a transposed copy); mode 2 is mode 1
 * with the two descriptor strides exchanged (kept to verify which reading of
 * the descriptor the hardware follows).
 */
int allegro_selftest_mma_mode(int32_t n, int32_t k, const float* a, const float* b, float* d, int32_t mode);

/*
 * Diagnostic (not part of the paper's method): SiLU(x) = x sigmoid(x) and its
 * derivative as the tensor-core passes compute them, sigmoid(x) =
 * 1/2 + tanh(x/2)/2 with the tanh.approx.f32 instruction, for checking their
 * error against a host reference (the error model of the tensor-core tests
 * rests on it).  x: device, n FP32; y: device, 2n FP32, y[2i] = SiLU(x[i]),
 * y[2i+1] = SiLU'(x[i]).  0 <= n <= 2^30, else ALLEGRO_E_INVALID_ARG.  Runs on
 * the legacy default stream and synchronises.
 */
int allegro_selftest_silu(int64_t n, const float* x, float* y);

/*
 * Failure injection for the failure-detection tests (not part of the paper's
 * method).  Every wait of the tensor-core passes on an mbarrier is bounded;
 * when one gives up, the pass skips its remaining MMAs, frees its tensor
 * memory, returns, and the calling entry point reports ALLEGRO_E_TIMEOUT
 * (MD and ring-polymer steps first restore the state they started from).
 * enable != 0 makes the passes on the current device issue no weight copies
 * and wait at most 2^20 clock cycles for them, so that every tensor-core call
 * ends in ALLEGRO_E_TIMEOUT with no copy or MMA in flight; enable == 0
 * restores normal operation (copies issued, 2^31-cycle limit).  Process-wide
 * for the current device; synchronises the device before and after, so call
 * it between calls, never while another thread uses the library.
 * ALLEGRO_E_CUDA if the device could not be updated.
 */
int allegro_debug_inject_wait_timeout(int32_t enable);

#ifdef __cplusplus
}
#endif

#endif /* ALLEGRO_GB300_H */
