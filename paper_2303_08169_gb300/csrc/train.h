// train.h - launchers of the weight-gradient and SAM kernels (train.cu).
#pragma once
#include <cuda_runtime.h>

namespace al {

// dW[n * ldw + k0 + k] += scale * sum_p dz[p * ldz + n] * x[p * ldx + k]
void launch_wgrad(const float* dz, int ldz, const float* x, int ldx, int P, int N, int K, float scale, float* dW,
                  int ldw, int k0, cudaStream_t s);
// mixing matrix of order l (see train.cu)
void launch_wgrad_mix(const float* dV, const float* T, int P, int C, int NLM, int NT, int l, int Pl, int toff,
                      float scale, float* dW, cudaStream_t s);
void launch_sumsq(const float* g, int n, double* out, cudaStream_t s);
void launch_ascent(const float* w, const float* g, int n, double rho, const double* norm2, float* w_out,
                   cudaStream_t s);
void launch_adam(float* w, const float* g, float* m, float* v, int n, double lr, int t, cudaStream_t s);
void launch_apply(const float* flat, int rows, int cols, float scale, float* t_out, float* n_out, cudaStream_t s);

}  // namespace al
