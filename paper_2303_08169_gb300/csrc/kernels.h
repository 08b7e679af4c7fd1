// kernels.h - host-side launchers shared between the CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace al {

// Status flags raised by kernels (bitwise OR into a device int).
enum DevFlag : int {
  kFlagPairOverflow = 1,
  kFlagNonfinite = 2,
  kFlagTimeout = 4,
  kFlagBadSpecies = 8,
};

struct NeighborBuffers {
  // per atom
  double* wpos = nullptr;      // N x 3 wrapped FP64
  float* wpos32 = nullptr;     // N x 3 wrapped FP32 (distance pre-filter)
  int* atom_cell = nullptr;    // N
  int* cell_count = nullptr;   // ncell + 1
  int* cell_start = nullptr;   // ncell + 1
  int* cell_atoms = nullptr;   // N (atoms sorted by cell)
  int* row_cnt = nullptr;      // N + 1
  int* row_ptr = nullptr;      // N + 1
  // per pair (capacity)
  int* pi = nullptr;           // centre atom
  int* pj = nullptr;           // neighbour atom
  int* pcode = nullptr;        // image code (common.cuh)
  int* rev = nullptr;          // reverse pair index
  unsigned long long* keys = nullptr;   // scratch: unsorted row keys
  unsigned long long* skeys = nullptr;  // sorted row keys
  // scan scratch
  int* scan_blocks = nullptr;  // >= ceil((max(N, ncell)+1)/1024) + 1
  int* n_pairs = nullptr;      // device scalar
  int* flags = nullptr;        // device scalar (DevFlag bits)
  int64_t capacity = 0;
};

struct GridInfo {
  double L[3];
  int ncell[3];     // cells per axis (cell mode) or 0 (small-box mode)
  int nimg[3];      // image range per axis in small-box mode
  double rc;
  float band;       // FP32 pre-filter half-width on d^2
};

// Plan the grid: cell mode iff floor(L / (rc (1 + 1e-9))) >= 3 on every axis.
GridInfo plan_grid(const double L[3], double rc);

// Full rebuild: wrap, bin, count, scan, fill, sort, reverse.  Writes the pair
// count to nb.n_pairs and raises kFlagPairOverflow if it exceeds capacity
// (then the pair arrays are untouched beyond capacity and must not be used).
// nps > 0: n_atoms / nps independent systems of nps atoms each in the same
// box (atoms of system k at [k nps, (k + 1) nps)), paired only within their
// system; the cell arrays then hold (n_atoms / nps) ncell + 1 entries.
// gate (optional, device): when *gate == 0 every kernel of the build returns
// at once and the previous list stays (Verlet-skin reuse).
void launch_build_neighbors(const NeighborBuffers& nb, const GridInfo& g, const double* pos,
                            int n_atoms, cudaStream_t s, int nps = 0, const int* gate = nullptr);

// Exclusive scan of n ints (in -> out), out[n] = total; total also copied to
// *total_dev when non-null.
void launch_scan(const int* in, int* out, int n, int* block_scratch, int* total_dev,
                 cudaStream_t s, const int* gate = nullptr);

// Verlet skin: flag[0] = rebuild needed (flag[1] forced, or an atom moved by
// more than skin/2 since pos_ref), flag[1] cleared (one block); then, after
// the gated build, pos_ref/wpos_ref recorded on a rebuild, else wpos set to
// wpos_ref + the minimum-image displacement; flag[2] counts rebuilds.
void launch_skin_check(int n, const double* pos, const double* pos_ref, const double L[3], double skin, int* flag,
                       cudaStream_t s);
void launch_skin_commit(int n, const double* pos, double* pos_ref, double* wpos, double* wpos_ref, const double L[3],
                        int* flag, cudaStream_t s);

}  // namespace al
