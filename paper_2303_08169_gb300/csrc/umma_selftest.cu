// umma_selftest.cu - diagnostic: one tensor-core tile GEMM through the same
// building blocks (umma.cuh) the BF16 pair passes use, so that descriptor,
// swizzle, TMEM and barrier handling can be checked against a host reference.
#include "../../include/allegro.h"
#include "umma.cuh"

namespace al {
namespace {

using namespace umma;

// mode 0: D = A B^T with B [N x K] K-major.
// mode 1/2: D = A W with W [K x N] given row-major; its K-major image (K rows
// of N elements) is read as an MN-major operand (2: LBO/SBO swapped).
__global__ void __launch_bounds__(128) k_selftest(const float* __restrict__ A, const float* __restrict__ B,
                                                  int N, int K, float* __restrict__ D, int* __restrict__ err,
                                                  int mode) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  const int Kp = (K + 63) / 64 * 64;
  uint8_t* sA = sm;
  uint8_t* sB = sm + sw128_bytes(128, Kp);
  // fp32 -> bf16, written in the SW128 K-major layout (zero K padding)
  for (int idx = threadIdx.x; idx < 128 * (Kp / 8); idx += blockDim.x) {
    const int r = idx / (Kp / 8), k8 = (idx % (Kp / 8)) * 8;
    float v[8];
    for (int q = 0; q < 8; ++q) v[q] = (k8 + q < K) ? A[r * K + k8 + q] : 0.0f;
    st_bf16x8(sA, sw128_off(r, k8, 128), v);
  }
  if (mode == 0) {
    for (int idx = threadIdx.x; idx < N * (Kp / 8); idx += blockDim.x) {
      const int r = idx / (Kp / 8), k8 = (idx % (Kp / 8)) * 8;
      float v[8];
      for (int q = 0; q < 8; ++q) v[q] = (k8 + q < K) ? B[r * K + k8 + q] : 0.0f;
      st_bf16x8(sB, sw128_off(r, k8, N), v);
    }
  } else {
    const int Np = (N + 63) / 64 * 64;   // image of W: K rows, N columns
    for (int idx = threadIdx.x; idx < K * (Np / 8); idx += blockDim.x) {
      const int r = idx / (Np / 8), c8 = (idx % (Np / 8)) * 8;
      float v[8];
      for (int q = 0; q < 8; ++q) v[q] = (c8 + q < N) ? B[r * N + c8 + q] : 0.0f;
      st_bf16x8(sB, sw128_off(r, c8, K), v);
    }
  }
  fence_async_smem();
  if (threadIdx.x < 32) tmem_alloc(&tslot, 256);
  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tslot;
  if (threadIdx.x == 0) {
    if (mode == 0) mma_tile(taddr, smem_u32(sA), smem_u32(sB), N, K / 16, false);
    else mma_tile_bmn(taddr, smem_u32(sA), smem_u32(sB), N, K, K / 16, false, mode == 2);
    mma_commit(&mbar);
  }
  const bool ok = mbar_wait(&mbar, 0);
  tc_fence_after();
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(err, 1);
  } else {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(taddr + ((uint32_t)(w * 32) << 16) + (uint32_t)c0, v);
      for (int j = 0; j < 16; ++j) D[(w * 32 + lane) * N + c0 + j] = v[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tmem_dealloc(taddr, 256);
}

}  // namespace
}  // namespace al

extern "C" int allegro_selftest_mma(int32_t n, int32_t k, const float* a, const float* b, float* d) {
  return allegro_selftest_mma_mode(n, k, a, b, d, 0);
}


extern "C" int allegro_selftest_mma_mode(int32_t n, int32_t k, const float* a, const float* b, float* d,
                                         int32_t mode) {
  if (!a || !b || !d || n < 16 || n > 256 || n % 16 || k < 16 || k > 256 || k % 16 || mode < 0 || mode > 2)
    return ALLEGRO_E_INVALID_ARG;
  const int kp = (k + 63) / 64 * 64;
  const int np = (n + 63) / 64 * 64;
  const size_t smem = al::umma::sw128_bytes(128, kp) +
                      (mode == 0 ? al::umma::sw128_bytes(n, kp) : al::umma::sw128_bytes(k, np)) + 1024;
  cudaFuncSetAttribute(al::k_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return ALLEGRO_E_OOM;
  cudaMemset(err, 0, sizeof(int));
  al::k_selftest<<<1, 128, smem>>>(a, b, n, k, d, err, mode);
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (e != cudaSuccess) return ALLEGRO_E_CUDA;
  return h ? ALLEGRO_E_TIMEOUT : ALLEGRO_OK;
}
