// neighbor.cu - periodic cell-list neighbour search (the paper's linked-list
// decomposition and adjacency list, Sec. 2.4, moved onto the GPU).
//
// Pair set: (i, j, n), n in Z^3, (j, n) != (i, 0), with
//   w = wrap(r) into [0, L):  q = floor(r/L); w = r - q L; w += L if w < 0;
//                             w = 0 if w >= L          (FP64, rounded ops)
//   Delta_a = (w_j,a - w_i,a) + n_a L_a,  d^2 = (Dx Dx + Dy Dy) + Dz Dz
//   included iff d^2 < rc * rc, all in FP64 without fused multiply-add.
// GB300's FP64 rate is low, so each candidate is first tested in FP32 against
// rc^2 -/+ band; only candidates whose FP32 d^2 falls inside the band take the
// exact FP64 test above.  The band bounds the FP32 rounding error (see
// plan_grid), so membership is decided exactly as by the FP64 rule.
//
// Layout: CSR by centre atom, rows sorted by (j, n_x, n_y, n_z); per pair
// pi (centre), pj, pcode (image code) and rev (index of (j, i, -n)).
// One warp per centre atom enumerates candidates, counts with ballots, fills
// keys, rank-sorts its row and decodes it.  Deterministic: the cell-filling
// order does not matter because every row is sorted by a unique key.
//
// Several systems in one build: atoms [k nps, (k + 1) nps) form system k
// (same box); each system has its own cells (cell index k ncell + c) and its
// atoms pair only among themselves, so the result is the concatenation of
// the systems' own lists with atom indices offset by k nps.
#include <cmath>
#include <cstdio>

#include "common.cuh"
#include "kernels.h"

namespace al {

namespace {

constexpr int kWarpsPerBlock = 8;

// Verlet-skin reuse: every kernel of a build returns at once when the gate
// word says that the current list is still valid (uniform over the grid).
#define NB_GATED(gate) \
  if ((gate) && *(gate) == 0) return;

__global__ void k_wrap_bin(const double* __restrict__ pos, int n, int nps, GridInfo g,
                           double* __restrict__ wpos, float* __restrict__ wpos32,
                           int* __restrict__ atom_cell, int* __restrict__ cell_count,
                           int* __restrict__ flags, const int* __restrict__ gate) {
  NB_GATED(gate)
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3];
  bool finite = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double L = g.L[a];
    const double r = pos[3 * i + a];
    finite = finite && isfinite(r);
    const double q = floor(__ddiv_rn(r, L));
    double w = __dsub_rn(r, __dmul_rn(q, L));
    if (w < 0.0) w = __dadd_rn(w, L);
    if (w >= L) w = 0.0;
    if (!finite) w = 0.0;
    wpos[3 * i + a] = w;
    wpos32[3 * i + a] = (float)w;
    if (g.ncell[0] > 0) {
      int ci = (int)(w * (double)g.ncell[a] / L);
      c[a] = min(max(ci, 0), g.ncell[a] - 1);
    }
  }
  if (!finite) atomicOr(flags, kFlagNonfinite);
  if (g.ncell[0] > 0) {
    const int ncl = g.ncell[0] * g.ncell[1] * g.ncell[2];
    const int cell = (i / nps) * ncl + (c[0] * g.ncell[1] + c[1]) * g.ncell[2] + c[2];
    atom_cell[i] = cell;
    atomicAdd(&cell_count[cell], 1);
  }
}

__global__ void k_cell_fill(int n, const int* __restrict__ atom_cell,
                            const int* __restrict__ cell_start, int* __restrict__ cursor,
                            int* __restrict__ cell_atoms, const int* __restrict__ gate) {
  NB_GATED(gate)
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = atom_cell[i];
  int slot = atomicAdd(&cursor[c], 1);
  cell_atoms[cell_start[c] + slot] = i;
}

// Exact FP64 membership test (the defining rule).
// Not inlined: a real call is taken only by warps with a candidate in the band,
// instead of predicated FP64 work on every candidate (FP64 is slow on this part).
__device__ __noinline__ bool exact_in(const double* __restrict__ w, int i, int j, int nx, int ny, int nz,
                                     double Lx, double Ly, double Lz, double rc) {
  const double dx = __dadd_rn(__dsub_rn(w[3 * j], w[3 * i]), (double)nx * Lx);
  const double dy = __dadd_rn(__dsub_rn(w[3 * j + 1], w[3 * i + 1]), (double)ny * Ly);
  const double dz = __dadd_rn(__dsub_rn(w[3 * j + 2], w[3 * i + 2]), (double)nz * Lz);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return d2 < __dmul_rn(rc, rc);
}

// Visit every candidate (j, n) of centre i, lanes striding over candidates
// of i's own system (nps atoms per system).  f(j, n[3]) is called by the
// lane owning a candidate that is inside the cutoff; returns nothing, the
// caller ballots.
template <class F>
AL_DEV void for_each_candidate(int i, const GridInfo& g, const float* __restrict__ w32,
                               const double* __restrict__ w64, const int* __restrict__ atom_cell,
                               const int* __restrict__ cell_start,
                               const int* __restrict__ cell_atoms, int nps, F f) {
  const int lane = threadIdx.x & 31;
  const float xi = w32[3 * i], yi = w32[3 * i + 1], zi = w32[3 * i + 2];
  const float rc2 = (float)(g.rc * g.rc);
  const float lo = rc2 - g.band, hi = rc2 + g.band;
  const float Lf[3] = {(float)g.L[0], (float)g.L[1], (float)g.L[2]};
  if (g.ncell[0] > 0) {
    // lane o < 27 describes neighbour cell o (atom range, image shift); the
    // lanes then stride over the concatenation of the 27 ranges, so that a
    // warp visits ~10 candidates per cell in one pass instead of one pass per
    // cell
    const int ncl = g.ncell[0] * g.ncell[1] * g.ncell[2];
    const int sys_cell = (atom_cell[i] / ncl) * ncl;  // first cell of i's system
    const int cell = atom_cell[i] - sys_cell;
    const int cz = cell % g.ncell[2];
    const int cy = (cell / g.ncell[2]) % g.ncell[1];
    const int cx = cell / (g.ncell[2] * g.ncell[1]);
    int cb = 0, cn = 0, ccode = img_code(0, 0, 0);
    if (lane < 27) {
      const int ox = lane / 9 - 1, oy = (lane / 3) % 3 - 1, oz = lane % 3 - 1;
      int tx = cx + ox, ty = cy + oy, tz = cz + oz;
      int n[3] = {0, 0, 0};
      if (tx < 0) { tx += g.ncell[0]; n[0] = -1; } else if (tx >= g.ncell[0]) { tx -= g.ncell[0]; n[0] = 1; }
      if (ty < 0) { ty += g.ncell[1]; n[1] = -1; } else if (ty >= g.ncell[1]) { ty -= g.ncell[1]; n[1] = 1; }
      if (tz < 0) { tz += g.ncell[2]; n[2] = -1; } else if (tz >= g.ncell[2]) { tz -= g.ncell[2]; n[2] = 1; }
      const int other = sys_cell + (tx * g.ncell[1] + ty) * g.ncell[2] + tz;
      cb = cell_start[other];
      cn = cell_start[other + 1] - cb;
      ccode = img_code(n[0], n[1], n[2]);
    }
    int incl = cn;                                    // inclusive scan of the range lengths
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    const int excl = incl - cn;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int k0 = 0; k0 < total; k0 += 32) {
      const int k = k0 + lane;
      int o = 0;                                      // last range starting at or before k
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int c = o + step;
        const int ec = __shfl_sync(0xffffffffu, excl, c < 27 ? c : 26);
        if (c < 27 && ec <= k) o = c;
      }
      const int b = __shfl_sync(0xffffffffu, cb, o), e0 = __shfl_sync(0xffffffffu, excl, o);
      const int code = __shfl_sync(0xffffffffu, ccode, o);
      bool hit = false;
      int j = -1;
      int n[3];
      img_decode(code, n[0], n[1], n[2]);
      if (k < total) {
        j = cell_atoms[b + (k - e0)];
        const float dx = (w32[3 * j] - xi) + n[0] * Lf[0];
        const float dy = (w32[3 * j + 1] - yi) + n[1] * Lf[1];
        const float dz = (w32[3 * j + 2] - zi) + n[2] * Lf[2];
        const float d2 = dx * dx + dy * dy + dz * dz;
        const bool self = (j == i) && n[0] == 0 && n[1] == 0 && n[2] == 0;
        if (!self) {
          if (d2 < lo) hit = true;
          else if (d2 <= hi) hit = exact_in(w64, i, j, n[0], n[1], n[2], g.L[0], g.L[1], g.L[2], g.rc);
        }
      }
      f(hit, j, n);
    }
  } else {
    const int nx = 2 * g.nimg[0] + 1, ny = 2 * g.nimg[1] + 1, nz = 2 * g.nimg[2] + 1;
    const int nimg = nx * ny * nz;
    const int total = nps * nimg;
    const int j0 = (i / nps) * nps;                   // first atom of i's system
    for (int k0 = 0; k0 < total; k0 += 32) {
      const int k = k0 + lane;
      bool hit = false;
      int j = -1;
      int n[3] = {0, 0, 0};
      if (k < total) {
        j = j0 + k / nimg;
        const int m = k % nimg;
        n[0] = m / (ny * nz) - g.nimg[0];
        n[1] = (m / nz) % ny - g.nimg[1];
        n[2] = m % nz - g.nimg[2];
        const float dx = (w32[3 * j] - xi) + n[0] * Lf[0];
        const float dy = (w32[3 * j + 1] - yi) + n[1] * Lf[1];
        const float dz = (w32[3 * j + 2] - zi) + n[2] * Lf[2];
        const float d2 = dx * dx + dy * dy + dz * dz;
        const bool self = (j == i) && n[0] == 0 && n[1] == 0 && n[2] == 0;
        if (!self) {
          if (d2 < lo) hit = true;
          else if (d2 <= hi) hit = exact_in(w64, i, j, n[0], n[1], n[2], g.L[0], g.L[1], g.L[2], g.rc);
        }
      }
      f(hit, j, n);
    }
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_count(int n_atoms, int nps, GridInfo g, const float* __restrict__ w32, const double* __restrict__ w64,
        const int* __restrict__ atom_cell, const int* __restrict__ cell_start,
        const int* __restrict__ cell_atoms, int* __restrict__ row_cnt, const int* __restrict__ gate) {
  NB_GATED(gate)
  const int i = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (i >= n_atoms) return;
  int cnt = 0;
  for_each_candidate(i, g, w32, w64, atom_cell, cell_start, cell_atoms, nps,
                     [&](bool hit, int, const int*) { cnt += __popc(__ballot_sync(0xffffffffu, hit)); });
  if ((threadIdx.x & 31) == 0) row_cnt[i] = cnt;
}

// rows of up to kRowCap pairs are ranked in shared memory (every lane reads
// the same key at a time: broadcasts); longer rows use the global key buffer
constexpr int kRowCap = 192;

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_fill(int n_atoms, int nps, GridInfo g, const float* __restrict__ w32, const double* __restrict__ w64,
       const int* __restrict__ atom_cell, const int* __restrict__ cell_start,
       const int* __restrict__ cell_atoms, const int* __restrict__ row_ptr,
       const int* __restrict__ n_pairs, int64_t capacity, unsigned long long* __restrict__ keys,
       unsigned long long* __restrict__ skeys, int* __restrict__ pi, int* __restrict__ pj,
       int* __restrict__ pcode, int* __restrict__ flags, const int* __restrict__ gate) {
  NB_GATED(gate)
  __shared__ unsigned long long s_keys[kWarpsPerBlock][kRowCap];
  if ((int64_t)(*n_pairs) > capacity) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flags, kFlagPairOverflow);
    return;
  }
  const int i = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (i >= n_atoms) return;
  const int lane = threadIdx.x & 31;
  const int base = row_ptr[i];
  const int len = row_ptr[i + 1] - base;
  unsigned long long* kb = len <= kRowCap ? s_keys[threadIdx.x >> 5] : keys + base;
  int cnt = 0;
  for_each_candidate(i, g, w32, w64, atom_cell, cell_start, cell_atoms, nps,
                     [&](bool hit, int j, const int* n) {
                       const unsigned m = __ballot_sync(0xffffffffu, hit);
                       if (hit) {
                         const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                         if (pos < len)
                           kb[pos] = ((unsigned long long)j << 7) | (unsigned long long)img_code(n[0], n[1], n[2]);
                       }
                       cnt += __popc(m);
                     });
  __syncwarp();
  // rank sort of the row (keys are unique within a row); outputs written at
  // their rank
  for (int e = lane; e < len; e += 32) {
    const unsigned long long k = kb[e];
    int rank = 0;
    for (int t = 0; t < len; ++t) rank += kb[t] < k ? 1 : 0;
    skeys[base + rank] = k;
    pi[base + rank] = i;
    pj[base + rank] = (int)(k >> 7);
    pcode[base + rank] = (int)(k & 127ull);
  }
}

__global__ void k_reverse(const int* __restrict__ n_pairs, int64_t capacity,
                          const int* __restrict__ row_ptr, const int* __restrict__ pi,
                          const int* __restrict__ pj, const int* __restrict__ pcode,
                          const unsigned long long* __restrict__ skeys, int* __restrict__ rev,
                          int* __restrict__ flags, const int* __restrict__ gate) {
  NB_GATED(gate)
  const int P = *n_pairs;
  if ((int64_t)P > capacity) return;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const int i = pi[p], j = pj[p];
    const unsigned long long key =
        ((unsigned long long)i << 7) | (unsigned long long)img_code_neg(pcode[p]);
    const int end = row_ptr[j + 1];
    int lo = row_ptr[j], hi = end;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (skeys[mid] < key) lo = mid + 1; else hi = mid;
    }
    // Delta(j, i, -n) = -Delta(i, j, n) exactly, so the reverse pair exists;
    // if it ever did not, point at p itself (zero force contribution) and flag.
    if (lo < end && skeys[lo] == key) {
      rev[p] = lo;
    } else {
      rev[p] = p;
      atomicOr(flags, kFlagNonfinite);
    }
  }
}

// ---- exclusive scan (three phases, 1024 elements per block) ----
constexpr int kScanBlock = 1024;

__global__ void k_scan_reduce(const int* __restrict__ in, int n, int* __restrict__ bsum,
                              const int* __restrict__ gate) {
  NB_GATED(gate)
  __shared__ int sh[32];
  const int b = blockIdx.x;
  int v = 0;
  for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x) {
    const int idx = b * kScanBlock + k;
    v += idx < n ? in[idx] : 0;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) bsum[b] = v;
  }
}

__global__ void k_scan_blocks(int* __restrict__ bsum, int nb, const int* __restrict__ gate) {
  NB_GATED(gate)
  // single thread block, sequential over chunks of 1024
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < nb; c0 += 1024) {
    const int idx = c0 + threadIdx.x;
    const int v = idx < nb ? bsum[idx] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (idx < nb) bsum[idx] = carry + sh[threadIdx.x] - v;   // exclusive
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_apply(const int* __restrict__ in, int* __restrict__ out, int n,
                             const int* __restrict__ bsum, int nb, int* __restrict__ total,
                             const int* __restrict__ gate) {
  NB_GATED(gate)
  __shared__ int sh[kScanBlock];
  const int b = blockIdx.x;
  for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x) {
    const int idx = b * kScanBlock + k;
    sh[k] = idx < n ? in[idx] : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = bsum[b];
    for (int k = 0; k < kScanBlock; ++k) {
      const int v = sh[k];
      sh[k] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x) {
    const int idx = b * kScanBlock + k;
    if (idx < n) out[idx] = sh[k];
  }
  if (b == 0 && threadIdx.x == 0) {
    out[n] = bsum[nb];
    if (total) *total = bsum[nb];
  }
}

}  // namespace

void launch_scan(const int* in, int* out, int n, int* block_scratch, int* total_dev,
                 cudaStream_t s, const int* gate) {
  const int nb = (n + kScanBlock - 1) / kScanBlock;
  const int nbb = nb > 0 ? nb : 1;
  k_scan_reduce<<<nbb, 256, 0, s>>>(in, n, block_scratch, gate);
  k_scan_blocks<<<1, 1024, 0, s>>>(block_scratch, nbb, gate);
  k_scan_apply<<<nbb, 256, 0, s>>>(in, out, n, block_scratch, nbb, total_dev, gate);
}

GridInfo plan_grid(const double L[3], double rc) {
  GridInfo g{};
  bool cells = true;
  for (int a = 0; a < 3; ++a) {
    g.L[a] = L[a];
    const int nc = (int)std::floor(L[a] / (rc * (1.0 + 1e-9)));
    g.ncell[a] = nc;
    if (nc < 3) cells = false;
    g.nimg[a] = (int)std::ceil(rc / L[a]);
  }
  if (!cells) g.ncell[0] = g.ncell[1] = g.ncell[2] = 0;
  g.rc = rc;
  // FP32 pre-filter error bound: wrapped coordinates and L carry <= 2^-24
  // relative error, Delta accumulates <= 6 such roundings of magnitude
  // <= 3 Lmax, so |Delta_f32 - Delta| <= 2e-6 Lmax; with |Delta| ~ rc the
  // error on d^2 is below 2 sqrt3 rc 2e-6 Lmax + rounding of the squares.
  // The band is 16x that bound plus 1e-5 relative.
  const double Lmax = std::fmax(L[0], std::fmax(L[1], L[2]));
  g.band = (float)(16.0 * 2.0 * 1.7320508 * rc * 2e-6 * Lmax * (2 * g.nimg[0] + 1) +
                   1e-5 * rc * rc);
  return g;
}

void launch_build_neighbors(const NeighborBuffers& nb, const GridInfo& g, const double* pos,
                            int n_atoms, cudaStream_t s, int nps, const int* gate) {
  if (nps <= 0) nps = n_atoms > 0 ? n_atoms : 1;
  const int n_sys = n_atoms / nps;
  const int ncell = g.ncell[0] > 0 ? n_sys * g.ncell[0] * g.ncell[1] * g.ncell[2] : 0;
  if (ncell > 0) cudaMemsetAsync(nb.cell_count, 0, sizeof(int) * (ncell + 1), s);
  const int tb = 256;
  k_wrap_bin<<<(n_atoms + tb - 1) / tb, tb, 0, s>>>(pos, n_atoms, nps, g, nb.wpos, nb.wpos32,
                                                   nb.atom_cell, nb.cell_count, nb.flags, gate);
  if (ncell > 0) {
    launch_scan(nb.cell_count, nb.cell_start, ncell, nb.scan_blocks, nullptr, s, gate);
    // reuse cell_count as the fill cursor
    cudaMemsetAsync(nb.cell_count, 0, sizeof(int) * (ncell + 1), s);
    k_cell_fill<<<(n_atoms + tb - 1) / tb, tb, 0, s>>>(n_atoms, nb.atom_cell, nb.cell_start,
                                                      nb.cell_count, nb.cell_atoms, gate);
  }
  const int wb = (n_atoms + kWarpsPerBlock - 1) / kWarpsPerBlock;
  k_count<<<wb, kWarpsPerBlock * 32, 0, s>>>(n_atoms, nps, g, nb.wpos32, nb.wpos, nb.atom_cell,
                                             nb.cell_start, nb.cell_atoms, nb.row_cnt, gate);
  launch_scan(nb.row_cnt, nb.row_ptr, n_atoms, nb.scan_blocks, nb.n_pairs, s, gate);
  k_fill<<<wb, kWarpsPerBlock * 32, 0, s>>>(n_atoms, nps, g, nb.wpos32, nb.wpos, nb.atom_cell,
                                            nb.cell_start, nb.cell_atoms, nb.row_ptr, nb.n_pairs,
                                            nb.capacity, nb.keys, nb.skeys, nb.pi, nb.pj,
                                            nb.pcode, nb.flags, gate);
  k_reverse<<<152 * 8, 256, 0, s>>>(nb.n_pairs, nb.capacity, nb.row_ptr, nb.pi, nb.pj, nb.pcode,
                                    nb.skeys, nb.rev, nb.flags, gate);
}

// ---- Verlet skin (reuse of a list built with r_c + skin) ----
namespace {

// One block: flag[0] = flag[1] (a forced rebuild) or some atom moved more
// than skin/2 (minimum image) since the last build; flag[1] cleared.
__global__ void k_skin_check(int n, const double* __restrict__ pos, const double* __restrict__ pos_ref, double L0,
                             double L1, double L2, double half_skin2, int* __restrict__ flag) {
  const double L[3] = {L0, L1, L2};
  int far = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double d = pos[3 * i + a] - pos_ref[3 * i + a];
      d -= L[a] * rint(d / L[a]);
      d2 += d * d;
    }
    far |= d2 > half_skin2 ? 1 : 0;
  }
  const int any = __syncthreads_or(far);
  if (threadIdx.x == 0) {
    flag[0] = (any || flag[1]) ? 1 : 0;
    flag[1] = 0;
  }
}

// After the (possibly skipped) build: a rebuild records the reference
// positions (the state and its wrap); otherwise the build's wrapped positions
// are the reference wrap plus the minimum-image displacement, which keeps
// every pair's image code valid.  Counts rebuilds in flag[2].
__global__ void k_skin_commit(int n, const double* __restrict__ pos, double* __restrict__ pos_ref,
                              double* __restrict__ wpos, double* __restrict__ wpos_ref, double L0, double L1, double L2,
                              int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool rebuilt = flag[0] != 0;
  if (rebuilt && i == 0) flag[2] += 1;
  if (i >= n) return;
  const double L[3] = {L0, L1, L2};
  for (int a = 0; a < 3; ++a) {
    if (rebuilt) {
      pos_ref[3 * i + a] = pos[3 * i + a];
      wpos_ref[3 * i + a] = wpos[3 * i + a];
    } else {
      double d = pos[3 * i + a] - pos_ref[3 * i + a];
      d -= L[a] * rint(d / L[a]);
      wpos[3 * i + a] = wpos_ref[3 * i + a] + d;
    }
  }
}

}  // namespace

void launch_skin_check(int n, const double* pos, const double* pos_ref, const double L[3], double skin, int* flag,
                       cudaStream_t s) {
  k_skin_check<<<1, 1024, 0, s>>>(n, pos, pos_ref, L[0], L[1], L[2], 0.25 * skin * skin, flag);
}

void launch_skin_commit(int n, const double* pos, double* pos_ref, double* wpos, double* wpos_ref, const double L[3],
                        int* flag, cudaStream_t s) {
  k_skin_commit<<<(n + 255) / 256, 256, 0, s>>>(n, pos, pos_ref, wpos, wpos_ref, L[0], L[1], L[2], flag);
}

}  // namespace al
