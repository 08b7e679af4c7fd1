// noalloc.cu - the >5 sigma force-outlier count without any device
// allocation, for callers that cannot allocate device memory:
//   * applications whose own allocator owns all device memory (a framework
//     pool or a fixed memory budget), where a foreign cudaMalloc fails or
//     fragments their pool;
//   * latency-bound loops: cudaMalloc / cudaFree can synchronise the device
//     and take far longer than the count itself.
// The reduction scratch lives in one file-scope __device__ array of fixed size
// (every GPU that loads the library keeps it until the process exits); the
// caller passes the forces and a device output.  Its counterpart that
// allocates through a context is allegro_outlier_count.
#include <mutex>
#include <string>

#include "../../include/allegro.h"

namespace al {
void set_global_error(const std::string& msg);   // api.cu
}

namespace {

constexpr int kNaBlock = 256;
constexpr int64_t kNaMaxAtoms = int64_t(1) << 22;                       // 4,194,304 atoms
constexpr int kNaMaxBlocks = (int)((kNaMaxAtoms + kNaBlock - 1) / kNaBlock);
constexpr int kNaMaxDevices = 64;

// [0, kNaMaxBlocks) doubles: per-block sums of F^2;
// [kNaMaxBlocks, 2 kNaMaxBlocks) u64: per-block counts; then one double: sum F^2.
constexpr size_t kNaScratchBytes = (size_t)kNaMaxBlocks * 8 * 2 + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

std::mutex g_mu;
// per device: the scratch address and the CUDA context it was looked up in
// (a reset device or another context on the same ordinal loads the module
// again, possibly at another address)
void* g_scratch_ptr[kNaMaxDevices] = {};
void* g_scratch_ctx[kNaMaxDevices] = {};

// cuCtxGetCurrent through the runtime's driver entry point (no link-time
// dependency on the driver library); null if unavailable.
using CtxGetCurrentFn = int (*)(void**);
CtxGetCurrentFn ctx_get_current() {
  static const CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

void* current_context() {
  void* c = nullptr;
  const CtxGetCurrentFn fn = ctx_get_current();
  if (!fn || fn(&c) != 0) return nullptr;
  return c;
}

__global__ void k_na_sumsq(int n, const float* __restrict__ F, double* __restrict__ part) {
  __shared__ double sh[kNaBlock / 32];
  const int i = blockIdx.x * kNaBlock + threadIdx.x;
  double f = 0.0;
  if (i < n)
    for (int a = 0; a < 3; ++a) f += (double)F[3 * i + a] * (double)F[3 * i + a];
  for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kNaBlock / 32; ++w) s += sh[w];
    part[blockIdx.x] = s;     // every block writes its own slot: no zeroing needed
  }
}

// one block: sum F^2 over all blocks in a fixed order
__global__ void k_na_total(const double* __restrict__ part, int nblk, double* __restrict__ total) {
  __shared__ double sh[kNaBlock];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kNaBlock) s += part[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kNaBlock; ++k) t += sh[k];
    *total = t;
  }
}

__global__ void k_na_count(int n, const float* __restrict__ F, double thr, const double* __restrict__ total,
                           unsigned long long* __restrict__ cnt) {
  __shared__ unsigned long long sh[kNaBlock / 32];
  const int i = blockIdx.x * kNaBlock + threadIdx.x;
  const double lim = thr * sqrt(*total / (3.0 * n));
  unsigned long long c = 0;
  if (i < n)
    for (int a = 0; a < 3; ++a) c += fabs((double)F[3 * i + a]) > lim ? 1ull : 0ull;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < kNaBlock / 32; ++w) s += sh[w];
    cnt[blockIdx.x] = s;
  }
}

__global__ void k_na_final(const unsigned long long* __restrict__ cnt, int nblk, long long* __restrict__ out) {
  __shared__ unsigned long long sh[kNaBlock];
  unsigned long long s = 0;
  for (int b = threadIdx.x; b < nblk; b += kNaBlock) s += cnt[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < kNaBlock; ++k) t += sh[k];
    *out = (long long)t;
  }
}

// Device address of the scratch array on the current device, looked up once
// per device and context (host code may not use the symbol itself as a
// device pointer).
int scratch_ptr(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    al::set_global_error("outlier_count_noalloc: no current CUDA device");
    return ALLEGRO_E_CUDA;
  }
  if (dev < 0 || dev >= kNaMaxDevices) {
    al::set_global_error("outlier_count_noalloc: device index beyond 63");
    return ALLEGRO_E_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  void* ctx = current_context();
  if (!g_scratch_ptr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      al::set_global_error(std::string("outlier_count_noalloc: cudaGetSymbolAddress failed: ") +
                           cudaGetErrorString(e));
      return ALLEGRO_E_CUDA;
    }
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = current_context();   // the lookup made the context current if it was not
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return ALLEGRO_OK;
}

}  // namespace

extern "C" int allegro_outlier_count_noalloc(int64_t n_atoms, const float* forces, double threshold,
                                             int64_t* count_out, void* cuda_stream) {
  if (!forces || !count_out) {
    al::set_global_error("outlier_count_noalloc: forces and count_out are required");
    return ALLEGRO_E_INVALID_ARG;
  }
  if (n_atoms < 1 || n_atoms > kNaMaxAtoms) {
    al::set_global_error("outlier_count_noalloc: n_atoms must be in [1, 4194304] (fixed scratch size)");
    return ALLEGRO_E_INVALID_ARG;
  }
  // an error left by the caller's own earlier work stays the caller's: report
  // it without clearing it, and launch nothing
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) {
    al::set_global_error(std::string("outlier_count_noalloc: a CUDA error from earlier work is pending: ") +
                         cudaGetErrorString(pending));
    return ALLEGRO_E_CUDA;
  }
  unsigned char* base = nullptr;
  const int rc = scratch_ptr(&base);
  if (rc) return rc;
  double* part = reinterpret_cast<double*>(base);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + (size_t)kNaMaxBlocks * 8);
  double* total = reinterpret_cast<double*>(base + (size_t)kNaMaxBlocks * 16);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int n = (int)n_atoms;
  const int nblk = (n + kNaBlock - 1) / kNaBlock;
  k_na_sumsq<<<nblk, kNaBlock, 0, s>>>(n, forces, part);
  k_na_total<<<1, kNaBlock, 0, s>>>(part, nblk, total);
  k_na_count<<<nblk, kNaBlock, 0, s>>>(n, forces, threshold, total, cnt);
  k_na_final<<<1, kNaBlock, 0, s>>>(cnt, nblk, reinterpret_cast<long long*>(count_out));
  const cudaError_t e = cudaGetLastError();   // no error was pending before the launches: this one is ours
  if (e != cudaSuccess) {
    al::set_global_error(std::string("outlier_count_noalloc: ") + cudaGetErrorString(e));
    return ALLEGRO_E_CUDA;
  }
  return ALLEGRO_OK;
}
