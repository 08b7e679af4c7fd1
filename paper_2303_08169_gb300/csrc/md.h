// md.h - launchers for the per-atom kernels (md.cu).
#pragma once
#include <cuda_runtime.h>

namespace al {

constexpr double kKappa = 9.648533e-3;   // 1 eV/(A amu) in A/fs^2
constexpr double kBoltzmannEv = 8.617333262e-5;   // eV/K
constexpr double kHbarEvFs = 0.6582119569;         // reduced Planck constant, eV fs
constexpr int kMaxBeads = 64;                      // replicas per atom in ring-polymer MD

struct AtomArgs {
  int n;
  const int* species;
  double sigma[2], mu[2], mass[2];
};

int atom_blocks(int n);

// F = sum_j (g_ij - g_ji); E_i; per-block partials -> stats[0] = E, stats[1] = sum F^2.
void launch_forces(const AtomArgs& a, const int* row_ptr, const int* rev, const float* G,
                   const double* epart, int tile, float* F, double* Ei, double* blk,
                   double* stats, int* flags, cudaStream_t s);

// stats[1] = sum F^2 for an external force array.
void launch_sum_f2(int n, const float* F, double* stats, cudaStream_t s);

// count |F_ia| > thr * sqrt(stats[1] / 3N) into *out.
void launch_outliers(int n, const float* F, const double* stats, double thr,
                     unsigned long long* blk, long long* out, cudaStream_t s);

void launch_kick_drift(const AtomArgs& a, double* r, double* v, const float* F, double dt,
                       const double L[3], cudaStream_t s);

void launch_kick_measure(const AtomArgs& a, double* v, const float* F, double dt,
                         const double* stats, double thr, double* blk_ke,
                         unsigned long long* blk_out, long long* step, int max_steps,
                         double* energies, long long* outliers, cudaStream_t s);

// Nose-Hoover NVT (thermostat state nh = (xi, eta, K, s), FP64):
// nh[2] = K of the velocities v
void launch_nh_set_k(const AtomArgs& a, const double* v, double* blk_ke, double* nh, cudaStream_t s);
// thermostat half step, then v = s v + dt/2 kappa F/m and r = wrap(r + dt v)
void launch_nvt_first_half(const AtomArgs& a, double* r, double* v, const float* F, double dt, const double L[3],
                           double gkt, double q, const double* blk_ke, double* nh, cudaStream_t s);
// v += dt/2 kappa F/m, thermostat half step (K from v), v = s v, record
// (E_pot, K, E_tot, H) and the outlier count of the step
void launch_nvt_second_half(const AtomArgs& a, double* v, const float* F, double dt, const double* stats,
                            double thr, double gkt, double q, double* blk_ke, unsigned long long* blk_out,
                            double* nh, long long* step, int max_steps, double* energies, long long* outliers,
                            cudaStream_t s);

// Ring-polymer MD (P replicas of n atoms, bead-major q, v, F):
// exact free ring-polymer evolution for dt (C: P x P normal modes, w: mode
// frequencies in 1/fs, both device)
void launch_rp_free(int P, int n, double* q, double* v, const double* C, const double* w, double dt, cudaStream_t s);
// v += h kappa F / m; a: one replica's atoms (n = a.n, species of one replica)
void launch_rp_kick(int P, const AtomArgs& a, double* v, const float* F, double h, cudaStream_t s);
// record (mean replica energy, kinetic energy, H_P) of the step from stats[0]
// = sum of the replica energies; blk: 2 (P n / 256 + 1) doubles
void launch_rp_record(int P, const AtomArgs& a, const double* q, const double* v, double wp, double* blk,
                      const double* stats, long long* step, int max_steps, double* energies, cudaStream_t s);

}  // namespace al
