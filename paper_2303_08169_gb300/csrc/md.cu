// md.cu - per-atom kernels: force assembly, FP64 energy reduction, the >5 sigma
// outlier count (Fig. 1 caption) and FP64 velocity-Verlet NVE (Eq. 1, Sec. 3.2).
#include "common.cuh"
#include "md.h"

namespace al {
namespace {

constexpr int kBlock = 256;

template <class T>
AL_DEV T block_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  T r = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  __syncthreads();
  return r;  // valid in thread 0
}

// F_i = sum_{pairs p of row i} (g_p - g_rev(p)), g = dE/dDelta (Delta = r_j + nL - r_i);
// E_i = sigma_Z sum_j E_ij + mu_Z from the per-(tile, atom) partial sums.
__global__ void __launch_bounds__(kBlock)
k_forces(AtomArgs a, const int* __restrict__ row_ptr, const int* __restrict__ rev,
         const float* __restrict__ G, const double* __restrict__ epart, int tile,
         float* __restrict__ F, double* __restrict__ Ei_out, double* __restrict__ blk,
         const int* __restrict__ flags) {
  __shared__ double sh[kBlock / 32];
  if (*flags & 1) return;   // pair overflow: nothing valid to assemble
  const int i = blockIdx.x * kBlock + threadIdx.x;
  double e = 0.0, f2 = 0.0;
  if (i < a.n) {
    const int r0 = row_ptr[i], r1 = row_ptr[i + 1];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int p = r0; p < r1; ++p) {
      const int q = rev[p];
      fx += G[3 * p] - G[3 * q];
      fy += G[3 * p + 1] - G[3 * q + 1];
      fz += G[3 * p + 2] - G[3 * q + 2];
    }
    F[3 * i] = fx;
    F[3 * i + 1] = fy;
    F[3 * i + 2] = fz;
    double s = 0.0;
    if (r1 > r0) {
      const int t0 = r0 / tile, t1 = (r1 - 1) / tile;
      for (int t = t0; t <= t1; ++t) s += epart[t + i];
    }
    const int z = a.species[i];
    e = a.sigma[z] * s + a.mu[z];
    if (Ei_out) Ei_out[i] = e;
    f2 = (double)fx * fx + (double)fy * fy + (double)fz * fz;
  }
  const double se = block_sum(e, sh);
  const double sf = block_sum(f2, sh);
  if (threadIdx.x == 0) {
    blk[2 * blockIdx.x] = se;
    blk[2 * blockIdx.x + 1] = sf;
  }
}

// stats[0] = E, stats[1] = sum F^2 (fixed-order sum of the block partials)
__global__ void k_finalize(const double* __restrict__ blk, int nblk, double* __restrict__ stats,
                           int* __restrict__ flags) {
  if (threadIdx.x != 0) return;
  double e = 0.0, f = 0.0;
  for (int b = 0; b < nblk; ++b) {
    e += blk[2 * b];
    f += blk[2 * b + 1];
  }
  stats[0] = e;
  stats[1] = f;
  if (!isfinite(e) || !isfinite(f)) atomicOr(flags, 2);
}

// count |F_ia| > thr * sigma, sigma^2 = sum F^2 / (3N), computed in FP64
__global__ void __launch_bounds__(kBlock)
k_outliers(int n, const float* __restrict__ F, const double* __restrict__ stats, double thr,
           unsigned long long* __restrict__ blk) {
  __shared__ unsigned long long sh[kBlock / 32];
  const int i = blockIdx.x * kBlock + threadIdx.x;
  unsigned long long c = 0;
  if (i < n && n > 0) {
    const double sigma = sqrt(stats[1] / (3.0 * n));
    const double lim = thr * sigma;
    for (int a = 0; a < 3; ++a) c += fabs((double)F[3 * i + a]) > lim ? 1ull : 0ull;
  }
  const unsigned long long s = block_sum(c, sh);
  if (threadIdx.x == 0) blk[blockIdx.x] = s;
}

__global__ void k_sum_u64(const unsigned long long* __restrict__ blk, int nblk,
                          long long* __restrict__ out) {
  if (threadIdx.x != 0) return;
  unsigned long long s = 0;
  for (int b = 0; b < nblk; ++b) s += blk[b];
  *out = (long long)s;
}

AL_DEV double wrap1(double r, double L) {
  const double q = floor(__ddiv_rn(r, L));
  double w = __dsub_rn(r, __dmul_rn(q, L));
  if (w < 0.0) w = __dadd_rn(w, L);
  if (w >= L) w = 0.0;
  return w;
}

// first half of a step: v += dt/2 kappa F/m; r = wrap(r + dt v)
__global__ void __launch_bounds__(kBlock)
k_kick_drift(AtomArgs a, double* __restrict__ r, double* __restrict__ v,
             const float* __restrict__ F, double dt, double L0, double L1, double L2) {
  const int i = blockIdx.x * kBlock + threadIdx.x;
  if (i >= a.n) return;
  const double c = 0.5 * dt * kKappa / a.mass[a.species[i]];
  const double L[3] = {L0, L1, L2};
  for (int k = 0; k < 3; ++k) {
    const double vv = v[3 * i + k] + c * (double)F[3 * i + k];
    v[3 * i + k] = vv;
    r[3 * i + k] = wrap1(r[3 * i + k] + dt * vv, L[k]);
  }
}

// second half: v += dt/2 kappa F/m, kinetic energy and outliers of the step
__global__ void __launch_bounds__(kBlock)
k_kick_measure(AtomArgs a, double* __restrict__ v, const float* __restrict__ F, double dt,
               const double* __restrict__ stats, double thr, double* __restrict__ blk_ke,
               unsigned long long* __restrict__ blk_out) {
  __shared__ double sh[kBlock / 32];
  __shared__ unsigned long long shu[kBlock / 32];
  const int i = blockIdx.x * kBlock + threadIdx.x;
  double ke = 0.0;
  unsigned long long c = 0;
  if (i < a.n) {
    const double m = a.mass[a.species[i]];
    const double cc = 0.5 * dt * kKappa / m;
    const double sigma = sqrt(stats[1] / (3.0 * a.n));
    const double lim = thr * sigma;
    for (int k = 0; k < 3; ++k) {
      const double f = (double)F[3 * i + k];
      const double vv = v[3 * i + k] + cc * f;
      v[3 * i + k] = vv;
      ke += 0.5 * m * vv * vv;
      c += fabs(f) > lim ? 1ull : 0ull;
    }
  }
  const double s = block_sum(ke, sh);
  const unsigned long long sc = block_sum(c, shu);
  if (threadIdx.x == 0) {
    blk_ke[blockIdx.x] = s / kKappa;
    blk_out[blockIdx.x] = sc;
  }
}

// energies[step] = (E_pot, E_kin, E_tot), outliers[step]; step counter advances
__global__ void k_record(const double* __restrict__ stats, const double* __restrict__ blk_ke,
                         const unsigned long long* __restrict__ blk_out, int nblk,
                         long long* __restrict__ step, int max_steps, double* __restrict__ energies,
                         long long* __restrict__ outliers) {
  if (threadIdx.x != 0) return;
  double ke = 0.0;
  unsigned long long c = 0;
  for (int b = 0; b < nblk; ++b) {
    ke += blk_ke[b];
    c += blk_out[b];
  }
  const long long s = *step;
  if (s >= 0 && s < max_steps) {
    energies[3 * s] = stats[0];
    energies[3 * s + 1] = ke;
    energies[3 * s + 2] = stats[0] + ke;
    outliers[s] = (long long)c;
  }
  *step = s + 1;
}

// ---- Nose-Hoover thermostat (NVT); state nh = (xi, eta, K, s) in FP64 ----

// K of the current velocities into nh[2] (per-block partials, then a
// fixed-order sum by k_nh_set_k)
__global__ void __launch_bounds__(kBlock)
k_ke_partials(AtomArgs a, const double* __restrict__ v, double* __restrict__ blk_ke) {
  __shared__ double sh[kBlock / 32];
  const int i = blockIdx.x * kBlock + threadIdx.x;
  double ke = 0.0;
  if (i < a.n) {
    const double m = a.mass[a.species[i]];
    for (int k = 0; k < 3; ++k) ke += 0.5 * m * v[3 * i + k] * v[3 * i + k];
  }
  const double s = block_sum(ke, sh);
  if (threadIdx.x == 0) blk_ke[blockIdx.x] = s / kKappa;
}
__global__ void k_nh_set_k(const double* __restrict__ blk_ke, int nblk, double* __restrict__ nh) {
  if (threadIdx.x != 0) return;
  double k = 0.0;
  for (int b = 0; b < nblk; ++b) k += blk_ke[b];
  nh[2] = k;
}

// thermostat half step of length h (one thread): K from the block partials of
// the current velocities (use_partials) or nh[2]; xi by (h/2) G, G = (2K -
// g kT) / Q; s = exp(-xi h) (the next kernel scales the velocities by it);
// K by s^2; eta by xi h; xi by (h/2) G
__global__ void k_nh_half(const double* __restrict__ blk_ke, int nblk, int use_partials, double h, double gkt,
                          double q, double* __restrict__ nh) {
  if (threadIdx.x != 0) return;
  double k = 0.0;
  if (use_partials) {
    for (int b = 0; b < nblk; ++b) k += blk_ke[b];
  } else {
    k = nh[2];
  }
  double xi = nh[0] + 0.5 * h * (2.0 * k - gkt) / q;
  const double s = exp(-xi * h);
  k = k * s * s;
  const double eta = nh[1] + xi * h;
  xi = xi + 0.5 * h * (2.0 * k - gkt) / q;
  nh[0] = xi;
  nh[1] = eta;
  nh[2] = k;
  nh[3] = s;
}

// v = s v (thermostat) then the first half kick and the drift
__global__ void __launch_bounds__(kBlock)
k_kick_drift_nh(AtomArgs a, double* __restrict__ r, double* __restrict__ v, const float* __restrict__ F, double dt,
                double L0, double L1, double L2, const double* __restrict__ nh) {
  const int i = blockIdx.x * kBlock + threadIdx.x;
  if (i >= a.n) return;
  const double c = 0.5 * dt * kKappa / a.mass[a.species[i]];
  const double s = nh[3];
  const double L[3] = {L0, L1, L2};
  for (int k = 0; k < 3; ++k) {
    const double vs = v[3 * i + k] * s;
    const double vv = vs + c * (double)F[3 * i + k];
    v[3 * i + k] = vv;
    r[3 * i + k] = wrap1(r[3 * i + k] + dt * vv, L[k]);
  }
}

__global__ void __launch_bounds__(kBlock) k_scale_v(int n3, double* __restrict__ v, const double* __restrict__ nh) {
  const int i = blockIdx.x * kBlock + threadIdx.x;
  if (i < n3) v[i] *= nh[3];
}

// energies[step] = (E_pot, K, E_pot + K, H), H = E_pot + K + Q xi^2 / 2 + g kT eta
__global__ void k_record_nh(const double* __restrict__ stats, const unsigned long long* __restrict__ blk_out,
                            int nblk, const double* __restrict__ nh, double gkt, double q,
                            long long* __restrict__ step, int max_steps, double* __restrict__ energies,
                            long long* __restrict__ outliers) {
  if (threadIdx.x != 0) return;
  unsigned long long c = 0;
  for (int b = 0; b < nblk; ++b) c += blk_out[b];
  const long long s = *step;
  if (s >= 0 && s < max_steps) {
    const double e = stats[0], k = nh[2];
    energies[4 * s] = e;
    energies[4 * s + 1] = k;
    energies[4 * s + 2] = e + k;
    energies[4 * s + 3] = e + k + 0.5 * q * nh[0] * nh[0] + gkt * nh[1];
    outliers[s] = (long long)c;
  }
  *step = s + 1;
}

// ---- ring-polymer MD (Sec. 6): P replicas of n atoms, bead-major arrays
// x[(k n + i) 3 + a]; C[j P + k] the orthogonal normal-mode matrix, w[k] the
// mode frequencies (1/fs) ----

// exact free ring-polymer evolution for dt, one thread per (atom, component)
__global__ void __launch_bounds__(kBlock)
k_rp_free(int P, int n, double* __restrict__ q, double* __restrict__ v, const double* __restrict__ C,
          const double* __restrict__ w, double dt) {
  const int t = blockIdx.x * kBlock + threadIdx.x;
  if (t >= 3 * n) return;
  double x[kMaxBeads], y[kMaxBeads], qm[kMaxBeads], vm[kMaxBeads];
  for (int j = 0; j < P; ++j) {
    x[j] = q[(size_t)j * 3 * n + t];
    y[j] = v[(size_t)j * 3 * n + t];
  }
  for (int k = 0; k < P; ++k) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < P; ++j) {
      a = fma(C[j * P + k], x[j], a);
      b = fma(C[j * P + k], y[j], b);
    }
    const double om = w[k];
    if (om == 0.0) {
      qm[k] = a + dt * b;
      vm[k] = b;
    } else {
      const double c = cos(om * dt), s = sin(om * dt);
      qm[k] = c * a + (s / om) * b;
      vm[k] = -om * s * a + c * b;
    }
  }
  for (int j = 0; j < P; ++j) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < P; ++k) {
      a = fma(C[j * P + k], qm[k], a);
      b = fma(C[j * P + k], vm[k], b);
    }
    q[(size_t)j * 3 * n + t] = a;
    v[(size_t)j * 3 * n + t] = b;
  }
}

// v += h kappa F/m for every replica
__global__ void __launch_bounds__(kBlock)
k_rp_kick(int P, AtomArgs a, double* __restrict__ v, const float* __restrict__ F, double h) {
  const int n = a.n;
  const long long t = (long long)blockIdx.x * kBlock + threadIdx.x;
  if (t >= 3ll * P * n) return;
  const int i = (int)((t / 3) % n);
  v[t] += h * kKappa * (double)F[t] / a.mass[a.species[i]];
}

// block partials of sum m |v|^2 / 2 and sum m wp^2 |q_k - q_k+1|^2 / 2
// (amu A^2/fs^2), one thread per (replica, atom)
__global__ void __launch_bounds__(kBlock)
k_rp_energy(int P, AtomArgs a, const double* __restrict__ q, const double* __restrict__ v, double wp,
            double* __restrict__ blk) {
  const int n = a.n;
  __shared__ double sh[kBlock / 32];
  const int t = blockIdx.x * kBlock + threadIdx.x;
  double ke = 0.0, se = 0.0;
  if (t < P * n) {
    const int k = t / n, i = t % n, k1 = (k + 1) % P;
    const double m = a.mass[a.species[i]];
    for (int c = 0; c < 3; ++c) {
      const double vv = v[(size_t)t * 3 + c];
      const double d = q[(size_t)t * 3 + c] - q[((size_t)k1 * n + i) * 3 + c];
      ke += 0.5 * m * vv * vv;
      se += 0.5 * m * wp * wp * d * d;
    }
  }
  const double sk = block_sum(ke, sh);
  const double ss = block_sum(se, sh);
  if (threadIdx.x == 0) {
    blk[2 * blockIdx.x] = sk;
    blk[2 * blockIdx.x + 1] = ss;
  }
}

// energies[step] = (sum_k V_k / P, K, K + springs + sum_k V_k) in eV
__global__ void k_rp_record(const double* __restrict__ blk, int nblk, const double* __restrict__ stats, int P,
                            long long* __restrict__ step, int max_steps, double* __restrict__ energies) {
  if (threadIdx.x != 0) return;
  double k = 0.0, s = 0.0;
  for (int b = 0; b < nblk; ++b) {
    k += blk[2 * b];
    s += blk[2 * b + 1];
  }
  k /= kKappa;
  s /= kKappa;
  const long long st = *step;
  if (st >= 0 && st < max_steps) {
    energies[3 * st] = stats[0] / P;
    energies[3 * st + 1] = k;
    energies[3 * st + 2] = k + s + stats[0];
  }
  *step = st + 1;
}

}  // namespace

void launch_rp_free(int P, int n, double* q, double* v, const double* C, const double* w, double dt, cudaStream_t s) {
  k_rp_free<<<(3 * n + kBlock - 1) / kBlock, kBlock, 0, s>>>(P, n, q, v, C, w, dt);
}

void launch_rp_kick(int P, const AtomArgs& a, double* v, const float* F, double h, cudaStream_t s) {
  const long long tot = 3ll * P * a.n;
  k_rp_kick<<<(unsigned)((tot + kBlock - 1) / kBlock), kBlock, 0, s>>>(P, a, v, F, h);
}

void launch_rp_record(int P, const AtomArgs& a, const double* q, const double* v, double wp, double* blk,
                      const double* stats, long long* step, int max_steps, double* energies, cudaStream_t s) {
  const int nb = (P * a.n + kBlock - 1) / kBlock;
  k_rp_energy<<<nb, kBlock, 0, s>>>(P, a, q, v, wp, blk);
  k_rp_record<<<1, 32, 0, s>>>(blk, nb, stats, P, step, max_steps, energies);
}

int atom_blocks(int n) { return (n + kBlock - 1) / kBlock; }

void launch_nh_set_k(const AtomArgs& a, const double* v, double* blk_ke, double* nh, cudaStream_t s) {
  const int nb = atom_blocks(a.n);
  k_ke_partials<<<nb, kBlock, 0, s>>>(a, v, blk_ke);
  k_nh_set_k<<<1, 32, 0, s>>>(blk_ke, nb, nh);
}

void launch_nvt_first_half(const AtomArgs& a, double* r, double* v, const float* F, double dt, const double L[3],
                           double gkt, double q, const double* blk_ke, double* nh, cudaStream_t s) {
  k_nh_half<<<1, 32, 0, s>>>(blk_ke, 0, 0, 0.5 * dt, gkt, q, nh);
  k_kick_drift_nh<<<atom_blocks(a.n), kBlock, 0, s>>>(a, r, v, F, dt, L[0], L[1], L[2], nh);
}

void launch_nvt_second_half(const AtomArgs& a, double* v, const float* F, double dt, const double* stats,
                            double thr, double gkt, double q, double* blk_ke, unsigned long long* blk_out,
                            double* nh, long long* step, int max_steps, double* energies, long long* outliers,
                            cudaStream_t s) {
  const int nb = atom_blocks(a.n);
  k_kick_measure<<<nb, kBlock, 0, s>>>(a, v, F, dt, stats, thr, blk_ke, blk_out);
  k_nh_half<<<1, 32, 0, s>>>(blk_ke, nb, 1, 0.5 * dt, gkt, q, nh);
  k_scale_v<<<(3 * a.n + kBlock - 1) / kBlock, kBlock, 0, s>>>(3 * a.n, v, nh);
  k_record_nh<<<1, 32, 0, s>>>(stats, blk_out, nb, nh, gkt, q, step, max_steps, energies, outliers);
}

void launch_forces(const AtomArgs& a, const int* row_ptr, const int* rev, const float* G,
                   const double* epart, int tile, float* F, double* Ei, double* blk,
                   double* stats, int* flags, cudaStream_t s) {
  const int nb = atom_blocks(a.n);
  k_forces<<<nb, kBlock, 0, s>>>(a, row_ptr, rev, G, epart, tile, F, Ei, blk, flags);
  k_finalize<<<1, 32, 0, s>>>(blk, nb, stats, flags);
}

void launch_outliers(int n, const float* F, const double* stats, double thr,
                     unsigned long long* blk, long long* out, cudaStream_t s) {
  const int nb = atom_blocks(n);
  k_outliers<<<nb, kBlock, 0, s>>>(n, F, stats, thr, blk);
  k_sum_u64<<<1, 32, 0, s>>>(blk, nb, out);
}

__global__ void k_sum_f2(int n, const float* __restrict__ F, double* __restrict__ stats) {
  // single block, fixed order: used only by the standalone outlier entry point
  __shared__ double sh[32];
  double f = 0.0;
  for (int k = threadIdx.x; k < 3 * n; k += blockDim.x) f += (double)F[k] * (double)F[k];
  for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    stats[1] = s;
  }
}

void launch_sum_f2(int n, const float* F, double* stats, cudaStream_t s) {
  k_sum_f2<<<1, 1024, 0, s>>>(n, F, stats);
}

void launch_kick_drift(const AtomArgs& a, double* r, double* v, const float* F, double dt,
                       const double L[3], cudaStream_t s) {
  k_kick_drift<<<atom_blocks(a.n), kBlock, 0, s>>>(a, r, v, F, dt, L[0], L[1], L[2]);
}

void launch_kick_measure(const AtomArgs& a, double* v, const float* F, double dt,
                         const double* stats, double thr, double* blk_ke,
                         unsigned long long* blk_out, long long* step, int max_steps,
                         double* energies, long long* outliers, cudaStream_t s) {
  const int nb = atom_blocks(a.n);
  k_kick_measure<<<nb, kBlock, 0, s>>>(a, v, F, dt, stats, thr, blk_ke, blk_out);
  k_record<<<1, 32, 0, s>>>(stats, blk_ke, blk_out, nb, step, max_steps, energies, outliers);
}

}  // namespace al
