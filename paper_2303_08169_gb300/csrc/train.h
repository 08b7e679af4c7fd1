// train.h - launchers of the weight-gradient and SAM kernels (train.cu).
#pragma once
#include <cuda_runtime.h>

namespace al {

// dW[n * ldw + k0 + k] += scale * sum_p dz[p * ldz + n esz] * x[p * ldx + k esx]
// (element strides 1, or 2 for one part of an array of tangent numbers),
// per-chunk partials in part (wgrad_part_floats() floats) added in a fixed
// order: bitwise reproducible
void launch_wgrad(const float* dz, int ldz, int esz, const float* x, int ldx, int esx, int P, int N, int K,
                  float scale, float* dW, int ldw, int k0, float* part, cudaStream_t s);
// Tensor-core version for N, K <= 128 (wgrad_tc_supported), both terms of the
// tangent weight gradient in one launch:
//   dW[n * ldw + k0 + k] += scale * sum_p (dza[p ldz + n] xa[p ldx + k esx]
//                                          + dzb[p ldz + n] xb[p ldx + k esx])
// BF16 x 3 split operands (24 significant bits) with FP32 accumulation in
// TMEM; per-CTA partials added in a fixed order (bitwise reproducible).  A
// bounded wait that runs out raises bit 4 of *flags (ALLEGRO_E_TIMEOUT).
void launch_wgrad_tc(const float* dza, const float* dzb, int ldz, const float* xa, const float* xb, int ldx, int esx,
                     int P, int N, int K, float scale, float* dW, int ldw, int k0, float* part, int* flags,
                     cudaStream_t s);
bool wgrad_tc_supported(int N, int K);
// Mixing matrix of order l on the tensor cores, both tangent terms:
//   dW[c' C Pl + c Pl + q] += scale sum_p sum_m (dVa[p][(c' NLM + l l + m) esv] Ta[p][c NT + toff + q (2l+1) + m]
//                                                + dVb[..] Tb[..])
// (C <= 128, C Pl <= 128), same arithmetic and reduction order as launch_wgrad_tc.
void launch_wgrad_mix_tc(const float* dVa, const float* dVb, int esv, const float* Ta, const float* Tb, int P, int C,
                         int NLM, int NT, int l, int Pl, int toff, float scale, float* dW, float* part, int* flags,
                         cudaStream_t s);
// mixing matrix of order l (see train.cu); dV element stride esv
void launch_wgrad_mix(const float* dV, int esv, const float* T, int P, int C, int NLM, int NT, int l, int Pl,
                      int toff, float scale, float* dW, float* part, cudaStream_t s);
size_t wgrad_part_floats();
void launch_sumsq(const float* g, int n, double* out, cudaStream_t s);
void launch_ascent(const float* w, const float* g, int n, double rho, const double* norm2, float* w_out,
                   cudaStream_t s);
void launch_adam(float* w, const float* g, float* m, float* v, int n, double lr, int t, cudaStream_t s);
// w_out = w + scale d (FP64 arithmetic, one rounding)
void launch_axpy(const float* w, const float* d, double scale, int n, float* w_out, cudaStream_t s);
void launch_apply(const float* flat, int rows, int cols, float scale, float* t_out, float* n_out, cudaStream_t s);
// Full-O(3) mixing block: [rows][C pl] blob columns into the [rows][C pu]
// device block, column c pl + q at c pu + q_map[q] (pl <= kMixQ).
constexpr int kMixQ = 32;
struct MixQ { int q[kMixQ]; };
void launch_apply_mix(const float* flat, int rows, int C, int pl, int pu, const int* q_map, float scale,
                      float* n_out, cudaStream_t s);

// ---- training batches: all structures in one pass sequence ----
// Append one structure's neighbour list and atoms at atom offset A0 and pair
// offset P0 of the batch arrays (indices shifted, box lengths per atom).
struct BatchArrays {
  int* pi;
  int* pj;
  int* pcode;
  int* rev;
  int* row_ptr;
  double* wpos;
  double* atomL;
  int* species;
  int* sid;
};
void launch_append(const BatchArrays& bt, int n, int np, int64_t A0, int64_t P0, int b, const int* pi, const int* pj,
                   const int* pcode, const int* rev, const int* row_ptr, const double* wpos, const int* species,
                   const double L[3], cudaStream_t s);
// Loss of Eq. 3's objective (per-atom energy MSE + force MSE) on the batch and
// the seeds of its weight gradient: dE[b] = E_b - E*_b; v = 2 cf (F - F*);
// *loss.
void launch_batch_loss(int B, int64_t N, const int64_t* off, const double* Ei, const double* e_target,
                       const float* F, const float* f_target, double w_energy, double cf, double* dE, float* v,
                       double* blk, double* loss, cudaStream_t s);
// seed_i = 2 w_E dE_b / (B N_b^2) for atom i of structure b
void launch_seed_energy(int B, int64_t N, const int64_t* off, const int* sid, const double* dE, double w_energy,
                        float* seed, cudaStream_t s);
}  // namespace al
