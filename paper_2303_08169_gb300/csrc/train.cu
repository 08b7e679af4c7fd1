// train.cu - weight gradients and the SAM update (Eq. 3) on the GPU.
//
// dL/dW of a linear layer z = (W s) x (s = 1/sqrt(fan_in), extra factors
// folded in) is s * sum_pairs dz (x) x, reduced here from the per-pair dumps
// the FP32 passes write in training mode.  The SAM step (Eq. 3) then runs on
// the flat parameter vector (blob order): the ascent w' = w + rho g/||g||,
// and Adam (Table 5: beta = (0.9, 0.999)) with the gradient taken at w'.
#include "train.h"

#include <algorithm>

#include "umma.cuh"

namespace al {
namespace {

constexpr int kWT = 64;       // output tile (rows n, cols k) of the reduction
constexpr int kWP = 32;       // pairs staged per step

// part[z][n][k] = scale * sum_{p in chunk z} dz[p * ldz + n * esz] * x[p * ldx + k * esx]
// (element strides esz, esx: 1 for plain arrays, 2 for one part of an array
// of tangent numbers).  A 64 x 64 output tile per block over one chunk of
// pairs: 256 threads, each a 4 x 4 register tile fed by two 16-byte
// shared-memory reads per pair (the dz read is a broadcast within each half
// warp); every chunk writes its own partial, which k_chunk_sum adds in chunk
// order, so the gradient is the same bits on every run (no atomics).
__global__ void __launch_bounds__(256) k_wgrad(const float* __restrict__ dz, int ldz, int esz,
                                               const float* __restrict__ x, int ldx, int esx, int P, int N, int K,
                                               float scale, float* __restrict__ part, int chunk) {
  __shared__ __align__(16) float sz[kWP][kWT];
  __shared__ __align__(16) float sx[kWP][kWT];
  const int n0 = blockIdx.x * kWT, kb = blockIdx.y * kWT;
  const int pb = blockIdx.z * chunk, pe = min(P, pb + chunk);
  const int tn = (threadIdx.x >> 4) * 4, tk = (threadIdx.x & 15) * 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (int p0 = pb; p0 < pe; p0 += kWP) {
#pragma unroll
    for (int r = 0; r < kWP * kWT / 256; ++r) {
      const int idx = r * 256 + threadIdx.x;
      const int pp = idx / kWT, c = idx % kWT;
      const int p = p0 + pp;
      sz[pp][c] = (p < pe && n0 + c < N) ? dz[(size_t)p * ldz + (size_t)(n0 + c) * esz] : 0.0f;
      sx[pp][c] = (p < pe && kb + c < K) ? x[(size_t)p * ldx + (size_t)(kb + c) * esx] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int pp = 0; pp < kWP; ++pp) {
      const float4 a = *reinterpret_cast<const float4*>(&sz[pp][tn]);
      const float4 b = *reinterpret_cast<const float4*>(&sx[pp][tk]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* out = part + (size_t)blockIdx.z * N * K;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = n0 + tn + i;
    if (n >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (kb + tk + j < K) out[(size_t)n * K + kb + tk + j] = scale * acc[i][j];
  }
}

// dW[(o / K) * ldw + k0 + o % K] += sum over z of part[z][o], z in order
__global__ void k_chunk_sum(const float* __restrict__ part, int nz, int N, int K, float* __restrict__ dW, int ldw,
                            int k0) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= N * K) return;
  float acc = 0.0f;
  for (int z = 0; z < nz; ++z) acc += part[(size_t)z * N * K + o];
  dW[(size_t)(o / K) * ldw + k0 + o % K] += acc;
}

// Mixing of order l: part[blk][c' C Pl + c Pl + q] = scale sum_{p in chunk}
// sum_m dV[p][(c' NLM + l l + m) esv] T[p][c NT + toff + q (2l+1) + m]
// One block per chunk of pairs: the order-l parts of kMixG pairs' dV and T
// rows are staged in shared memory with contiguous loads, then every thread
// accumulates up to kMixR outputs (a pass over the chunk per kMixR x 256
// outputs) and writes the chunk's partial; k_chunk_sum adds them in order.
constexpr int kMixG = 16;
constexpr int kMixR = 4;

__global__ void __launch_bounds__(256) k_wgrad_mix(const float* __restrict__ dV, int esv,
                                                   const float* __restrict__ T, int P, int C, int NLM, int NT, int l,
                                                   int Pl, int toff, float scale, float* __restrict__ part, int chunk) {
  extern __shared__ float mix_s[];
  const int nm = 2 * l + 1;
  const int wv = C * nm, wt = C * Pl * nm;            // staged floats per pair
  float* dv_s = mix_s;                                // [kMixG][wv]
  float* t_s = mix_s + kMixG * wv;                    // [kMixG][wt]
  const int n_out = C * C * Pl;
  const int pb = blockIdx.x * chunk, pe = min(P, pb + chunk);
  for (int ob = 0; ob < n_out; ob += kMixR * 256) {
    float acc[kMixR];
    int dvo[kMixR], to[kMixR];
#pragma unroll
    for (int r = 0; r < kMixR; ++r) {
      acc[r] = 0.0f;
      const int o = min(ob + r * 256 + (int)threadIdx.x, n_out - 1);
      const int co = o / (C * Pl), c = (o / Pl) % C, q = o % Pl;
      dvo[r] = co * nm;
      to[r] = c * Pl * nm + q * nm;
    }
    for (int p0 = pb; p0 < pe; p0 += kMixG) {
      const int gn = min(kMixG, pe - p0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < gn * wv; idx += blockDim.x) {
        const int g = idx / wv, e = idx % wv, co = e / nm, m = e % nm;
        dv_s[g * wv + e] = dV[((size_t)(p0 + g) * C * NLM + co * NLM + l * l + m) * esv];
      }
      for (int idx = threadIdx.x; idx < gn * wt; idx += blockDim.x) {
        const int g = idx / wt, e = idx % wt, c = e / (Pl * nm), j = e % (Pl * nm);
        t_s[g * wt + e] = T[(size_t)(p0 + g) * C * NT + c * NT + toff + j];
      }
      __syncthreads();
      for (int g = 0; g < gn; ++g) {
        const float* dv = dv_s + g * wv;
        const float* tt = t_s + g * wt;
#pragma unroll
        for (int r = 0; r < kMixR; ++r)
          for (int m = 0; m < nm; ++m) acc[r] = fmaf(dv[dvo[r] + m], tt[to[r] + m], acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kMixR; ++r) {
      const int o = ob + r * 256 + (int)threadIdx.x;
      if (o < n_out) part[(size_t)blockIdx.x * n_out + o] = scale * acc[r];
    }
  }
}

__global__ void k_sumsq(const float* __restrict__ g, int n, double* __restrict__ out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)g[i] * (double)g[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) t += sh[k];
    *out = t;
  }
}

// w_out = w + rho g / ||g||  (w_out = w when ||g|| = 0)
__global__ void k_ascent(const float* __restrict__ w, const float* __restrict__ g, int n, double rho,
                         const double* __restrict__ norm2, float* __restrict__ w_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double nn = *norm2;
  w_out[i] = nn > 0.0 ? (float)((double)w[i] + rho * (double)g[i] / sqrt(nn)) : w[i];
}

// w + s d (the weights of one point of a loss scan), rounded once from FP64
__global__ void k_axpy(const float* __restrict__ w, const float* __restrict__ d, double s, int n,
                       float* __restrict__ w_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  w_out[i] = (float)((double)w[i] + s * (double)d[i]);
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, double lr, double b1, double b2, double eps, int t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gi = g[i];
  const double mi = b1 * (double)m[i] + (1.0 - b1) * gi;
  const double vi = b2 * (double)v[i] + (1.0 - b2) * gi * gi;
  m[i] = (float)mi;
  v[i] = (float)vi;
  const double mh = mi / (1.0 - pow(b1, (double)t));
  const double vh = vi / (1.0 - pow(b2, (double)t));
  w[i] = (float)((double)w[i] - lr * mh / (sqrt(vh) + eps));
}

// scaled FP32 copies of one tensor: t [in][out], n [out][in]
__global__ void k_apply(const float* __restrict__ flat, int rows, int cols, float scale, float* __restrict__ t_out,
                        float* __restrict__ n_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int o = i / cols, k = i % cols;
  const float v = flat[i] * scale;
  if (t_out) t_out[k * rows + o] = v;
  if (n_out) n_out[i] = v;
}

// Full-O(3) mixing: blob matrix [rows][C pl] into the device block
// [rows][C pu], column c pl + q at c pu + qm.q[q] (the other columns stay).
__global__ void k_apply_mix(const float* __restrict__ flat, int rows, int C, int pl, int pu, MixQ qm, float scale,
                            float* __restrict__ n_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * C * pl) return;
  const int o = i / (C * pl), k = i % (C * pl);
  n_out[(size_t)o * C * pu + (k / pl) * pu + qm.q[k % pl]] = flat[i] * scale;
}

__global__ void k_append(BatchArrays bt, int n, int np, int64_t A0, int64_t P0, int b,
                         const int* __restrict__ pi, const int* __restrict__ pj, const int* __restrict__ pcode,
                         const int* __restrict__ rev, const int* __restrict__ row_ptr,
                         const double* __restrict__ wpos, const int* __restrict__ species, double Lx, double Ly,
                         double Lz) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < np) {
    bt.pi[P0 + k] = pi[k] + (int)A0;
    bt.pj[P0 + k] = pj[k] + (int)A0;
    bt.pcode[P0 + k] = pcode[k];
    bt.rev[P0 + k] = rev[k] + (int)P0;
  }
  if (k <= n) bt.row_ptr[A0 + k] = row_ptr[k] + (int)P0;
  if (k < n) {
    const int64_t a = A0 + k;
    for (int d = 0; d < 3; ++d) bt.wpos[3 * a + d] = wpos[3 * k + d];
    bt.atomL[3 * a] = Lx;
    bt.atomL[3 * a + 1] = Ly;
    bt.atomL[3 * a + 2] = Lz;
    bt.species[a] = species[k];
    bt.sid[a] = b;
  }
}

// one block per structure: E_b - E*_b, atoms summed in a fixed order
__global__ void k_struct_dE(const int64_t* __restrict__ off, const double* __restrict__ Ei,
                            const double* __restrict__ e_target, double* __restrict__ dE) {
  __shared__ double sh[256];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int64_t i = off[b] + threadIdx.x; i < off[b + 1]; i += blockDim.x) s += Ei[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) t += sh[k];
    dE[b] = t - e_target[b];
  }
}

__global__ void k_force_resid(int64_t N, const float* __restrict__ F, const float* __restrict__ ft, double cf,
                              float* __restrict__ v, double* __restrict__ blk) {
  __shared__ double sh[256];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < N) {
    for (int d = 0; d < 3; ++d) {
      const double r = (double)F[3 * i + d] - (double)ft[3 * i + d];
      l += cf * r * r;
      v[3 * i + d] = (float)(2.0 * cf * r);
    }
  }
  sh[threadIdx.x] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) t += sh[k];
    blk[blockIdx.x] = t;
  }
}

__global__ void k_loss_total(int B, const int64_t* __restrict__ off, const double* __restrict__ dE, double wE,
                             const double* __restrict__ blk, int nblk, double* __restrict__ loss) {
  if (threadIdx.x != 0) return;
  double l = 0.0;
  for (int b = 0; b < B; ++b) {
    const double e = dE[b] / (double)(off[b + 1] - off[b]);
    l += wE / B * e * e;
  }
  for (int k = 0; k < nblk; ++k) l += blk[k];
  *loss = l;
}

__global__ void k_seed_energy(int B, int64_t N, const int64_t* __restrict__ off, const int* __restrict__ sid,
                              const double* __restrict__ dE, double wE, float* __restrict__ seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int b = sid[i];
  const double n = (double)(off[b + 1] - off[b]);
  seed[i] = (float)(2.0 * wE * dE[b] / ((double)B * n * n));
}

}  // namespace

void launch_append(const BatchArrays& bt, int n, int np, int64_t A0, int64_t P0, int b, const int* pi, const int* pj,
                   const int* pcode, const int* rev, const int* row_ptr, const double* wpos, const int* species,
                   const double L[3], cudaStream_t s) {
  const int m = std::max(n + 1, np);
  k_append<<<(m + 255) / 256, 256, 0, s>>>(bt, n, np, A0, P0, b, pi, pj, pcode, rev, row_ptr, wpos, species, L[0],
                                           L[1], L[2]);
}

void launch_batch_loss(int B, int64_t N, const int64_t* off, const double* Ei, const double* e_target,
                       const float* F, const float* f_target, double w_energy, double cf, double* dE, float* v,
                       double* blk, double* loss, cudaStream_t s) {
  const int nblk = (int)((N + 255) / 256);
  k_struct_dE<<<B, 256, 0, s>>>(off, Ei, e_target, dE);
  k_force_resid<<<nblk, 256, 0, s>>>(N, F, f_target, cf, v, blk);
  k_loss_total<<<1, 32, 0, s>>>(B, off, dE, w_energy, blk, nblk, loss);
}

void launch_seed_energy(int B, int64_t N, const int64_t* off, const int* sid, const double* dE, double w_energy,
                        float* seed, cudaStream_t s) {
  k_seed_energy<<<(int)((N + 255) / 256), 256, 0, s>>>(B, N, off, sid, dE, w_energy, seed);
}

// ---------------------------------------------------------------------------
// Tensor-core weight gradient: part[z] = scale * sum over CTA z's pairs of
// (R_a (x) Q_a + R_b (x) Q_b), R and Q per-pair operands of nR <= 128 and
// nQ <= 128 features, written as the [N][K] partial of the layer's dW (R the
// dz side, rows n, when r_is_n; else the x side, rows k).  The contraction
// over pairs is the MMA K dimension: a CTA walks its contiguous range of
// 64-pair chunks, term a then term b of each chunk (stage s: chunk s / 2,
// term s % 2, shared-memory buffer s % 2), and stages both operands of the
// stage as three BF16 parts, x = hi + mid + lo (hi = rn(x), mid = rn(x - hi),
// lo = rn(x - hi - mid): 24 significant bits).  Thread 0 issues the six
// products whose part orders sum to at most 2 (hi hi, hi mid, mid hi, hi lo,
// lo hi, mid mid; the dropped ones are below 2^-24 of the product) for the
// four 16-pair K-steps into an FP32 TMEM accumulator [128 x nQp] (stage s
// into accumulator s % 4, the four added at the end: the tensor pipe's FP32
// accumulation loses low bits as a chain grows, so the chains are kept four
// times shorter) and commits to the buffer's mbarrier; the next stage's
// global loads are in flight
// meanwhile, and a buffer is rewritten only after the MMAs that read it have
// completed.  Every wait is bounded; on a timeout the CTA stops issuing,
// raises bit 4 of *flags and writes nothing.  k_chunk_sum adds the partials
// in CTA order, so the gradient is the same bits on every run.
namespace wtc {
constexpr int kPairs = 64;                            // pairs per stage (one SW128 row of BF16)
constexpr int kThr = 512;
constexpr uint32_t kTileR = 128 * 128;                // bytes of one 128-row part tile
constexpr uint32_t kBuf = 6 * kTileR;                 // 3 R parts + 3 Q parts (nQp <= 128)
constexpr size_t kSmem = 1024 + 2 * (size_t)kBuf;
constexpr int kFlagTimeoutBit = 4;
// stages rotate over kAcc TMEM accumulators (128 columns each), added at the
// end: each accumulation chain is a quarter as long
constexpr int kAcc = 4;
}  // namespace wtc

// A per-pair operand.  The contraction index q runs over virtual pairs, nm
// per pair (q = pair nm + m: the m components of an order-l feature for the
// mixing matrices, nm = 1 otherwise); feature f splits as (f / fq, f % fq):
//   element (q, f) at p[(q / nm) ld + (q % nm) ms + (f / fq) es + (f % fq) fs2]
// (plain per-pair arrays: nm = 1, fq = 1, element (q, f) at p[q ld + f es]).
struct WgOp {
  const float* p;
  int ld, es;
  int nm = 1, ms = 0, fq = 1, fs2 = 0;
};

// 8 consecutive virtual pairs of feature f from q0 (zeros past P or past nf)
__device__ __forceinline__ void wtc_load8(const WgOp& o, int q0, int P, int f, int nf, float* v) {
  const size_t fo = (size_t)(f / o.fq) * o.es + (size_t)(f % o.fq) * o.fs2;
  int qp = q0 / o.nm, qm = q0 - qp * o.nm;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int q = q0 + e;
    v[e] = (q < P && f < nf) ? __ldg(o.p + (size_t)qp * o.ld + (size_t)qm * o.ms + fo) : 0.0f;
    if (++qm == o.nm) {
      qm = 0;
      ++qp;
    }
  }
}

// the three BF16 parts of v[0..7] into row f, pairs 8 g .. 8 g + 7 of the
// part tiles base + part * tile_bytes (R rows each)
__device__ __forceinline__ void wtc_store8(uint8_t* base, uint32_t tile_bytes, int R, int f, int g, const float* v) {
  uint32_t w[3][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float r0 = v[2 * q], r1 = v[2 * q + 1];
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(r0, r1);
      const float2 b = __bfloat1622float2(h);
      r0 -= b.x;
      r1 -= b.y;
      memcpy(&w[part][q], &h, 4);
    }
  }
  const uint32_t off = umma::sw128_off(f, 8 * g, R);
#pragma unroll
  for (int part = 0; part < 3; ++part)
    *reinterpret_cast<uint4*>(base + part * tile_bytes + off) = make_uint4(w[part][0], w[part][1], w[part][2], w[part][3]);
}

__global__ void __launch_bounds__(wtc::kThr, 1)
    k_wgrad_tc(WgOp Ra, WgOp Qa, WgOp Rb, WgOp Qb, int nR, int nQ, int nQp, int P, int chunks_per_cta,
               int r_is_n, int K, float scale, float* __restrict__ part, int* flags, long long wait_cycles) {
  using namespace umma;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t done[2];
  __shared__ uint32_t tslot;
  __shared__ int err;
  uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x;
  if (tid < 32) tmem_alloc(&tslot, 128 * wtc::kAcc);
  if (tid == 0) {
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    mbar_fence_init();
    err = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const int nchunks = (P + wtc::kPairs - 1) / wtc::kPairs;
  const int c0 = blockIdx.x * chunks_per_cta, c1 = min(nchunks, c0 + chunks_per_cta);
  const int nstage = 2 * max(c1 - c0, 0);
  const uint32_t tileQ = (uint32_t)nQp * 128;
  const uint32_t idesc = idesc_f16kind(128, nQp, false, 1);
  // per thread: up to two R tasks and two Q tasks of 8 pairs x 1 feature
  float va[2][8], vb[2][8];
  auto load_stage = [&](int st) {
    const int q0 = (c0 + st / 2) * wtc::kPairs;
    const WgOp R = (st & 1) ? Rb : Ra;                // copies: no address taken of the parameters
    const WgOp Q = (st & 1) ? Qb : Qa;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int t = tid + i * wtc::kThr;              // 1024 R tasks: f = t % 128, g = t / 128
      wtc_load8(R, q0 + 8 * (t >> 7), P, t & 127, nR, va[i]);
      const int tq = tid + i * wtc::kThr;             // nQp * 8 Q tasks: f = tq % nQp, g = tq / nQp
      if (tq < nQp * 8) wtc_load8(Q, q0 + 8 * (tq / nQp), P, tq % nQp, nQ, vb[i]);
    }
  };
  if (nstage > 0) load_stage(0);
  int issued = -1;                                     // last stage whose MMAs were committed (thread 0)
  for (int st = 0; st < nstage && !err; ++st) {
    const int b = st & 1;
    uint8_t* buf = sm + b * wtc::kBuf;
    if (st >= 2 && !mbar_wait(&done[b], (uint32_t)(((st >> 1) - 1) & 1), wait_cycles)) err = 1;
    __syncthreads();
    if (err) break;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int t = tid + i * wtc::kThr;
      wtc_store8(buf, wtc::kTileR, 128, t & 127, t >> 7, va[i]);
      const int tq = tid + i * wtc::kThr;
      if (tq < nQp * 8) wtc_store8(buf + 3 * wtc::kTileR, tileQ, nQp, tq % nQp, tq / nQp, vb[i]);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a = smem_u32(buf), q = smem_u32(buf + 3 * wtc::kTileR);
      const int pi[6] = {0, 0, 1, 0, 2, 1}, pj[6] = {0, 1, 0, 2, 0, 1};
      const uint32_t d = tmem + 128u * (uint32_t)(st % wtc::kAcc);   // stage st -> accumulator st % kAcc
#pragma unroll
      for (int pr = 0; pr < 6; ++pr)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(d, desc_sw128(a + pi[pr] * wtc::kTileR + kk * 32), desc_sw128(q + pj[pr] * tileQ + kk * 32),
                   idesc, (st >= wtc::kAcc || pr > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&done[b]);
      issued = st;
    }
    if (st + 1 < nstage) load_stage(st + 1);
  }
  // the last commit covers every MMA issued before it; waited for (bounded)
  // also after an error, so that no MMA is in flight when TMEM is freed
  if (tid == 0 && issued >= 0 && !mbar_wait(&done[issued & 1], (uint32_t)((issued >> 1) & 1), wait_cycles)) err = 1;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!err && tid < 128) {
    // warp w reads TMEM lanes 32 w .. 32 w + 31: accumulator row r = tid
    const int r = tid;
    float* out = part + (size_t)blockIdx.x * (r_is_n ? (size_t)nR * K : (size_t)nQ * K);
    const int nacc = min(nstage, wtc::kAcc);            // accumulators written, summed in order
    for (int q0 = 0; q0 < nQp; q0 += 16) {
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.0f;
      for (int ac = 0; ac < nacc; ++ac) {
        float u[16];
        tmem_ld16(tmem + ((uint32_t)((tid >> 5) * 32) << 16) + (uint32_t)(128 * ac + q0), u);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += u[j];
      }
      if (r < nR)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int qq = q0 + j;
          if (qq < nQ) out[r_is_n ? (size_t)r * K + qq : (size_t)qq * K + r] = scale * v[j];
        }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid < 32) tmem_dealloc(tmem, 128 * wtc::kAcc);
  if (err && tid == 0) atomicOr(flags, wtc::kFlagTimeoutBit);
}

int wgrad_chunks(int P, int N, int K) {
  // about four blocks per SM over all output tiles, chunks a multiple of the
  // staging depth
  const int tiles = ((N + kWT - 1) / kWT) * ((K + kWT - 1) / kWT);
  const int want = std::max(1, 152 * 4 / tiles);
  int chunk = (P + want - 1) / want;
  chunk = std::max(kWP * 8, (chunk + kWP - 1) / kWP * kWP);
  return chunk;
}

void launch_wgrad(const float* dz, int ldz, int esz, const float* x, int ldx, int esx, int P, int N, int K,
                  float scale, float* dW, int ldw, int k0, float* part, cudaStream_t s) {
  if (P <= 0) return;
  const int chunk = wgrad_chunks(P, N, K);
  const int nz = (P + chunk - 1) / chunk;
  dim3 grid((N + kWT - 1) / kWT, (K + kWT - 1) / kWT, nz);
  k_wgrad<<<grid, 256, 0, s>>>(dz, ldz, esz, x, ldx, esx, P, N, K, scale, part, chunk);
  k_chunk_sum<<<(N * K + 255) / 256, 256, 0, s>>>(part, nz, N, K, dW, ldw, k0);
}

void launch_wgrad_tc(const float* dza, const float* dzb, int ldz, const float* xa, const float* xb, int ldx, int esx,
                     int P, int N, int K, float scale, float* dW, int ldw, int k0, float* part, int* flags,
                     cudaStream_t s) {
  if (P <= 0) return;
  static bool init = false;
  static int sms = 0;
  if (!init) {
    cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wtc::kSmem);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    init = true;
  }
  // rows of the accumulator: the 128-wide side (dz when N >= K)
  const bool r_is_n = N >= K;
  const WgOp dA{dza, ldz, 1}, dB{dzb, ldz, 1}, xA{xa, ldx, esx}, xB{xb, ldx, esx};
  const int nR = r_is_n ? N : K, nQ = r_is_n ? K : N;
  const int nQp = (nQ + 15) / 16 * 16;
  const int nchunks = (P + wtc::kPairs - 1) / wtc::kPairs;
  const int cpc = (nchunks + std::max(sms, 1) - 1) / std::max(sms, 1);
  const int nz = (nchunks + cpc - 1) / cpc;
  k_wgrad_tc<<<nz, wtc::kThr, wtc::kSmem, s>>>(r_is_n ? dA : xA, r_is_n ? xA : dA, r_is_n ? dB : xB, r_is_n ? xB : dB,
                                              nR, nQ, nQp, P, cpc, r_is_n ? 1 : 0, K, scale, part, flags, 1ll << 31);
  k_chunk_sum<<<(N * K + 255) / 256, 256, 0, s>>>(part, nz, N, K, dW, ldw, k0);
}

bool wgrad_tc_supported(int N, int K) { return N >= 1 && K >= 1 && N <= 128 && K <= 128; }

// Mixing matrix of order l on the tensor cores: the contraction runs over
// (pair, m), m = 0 .. 2l, for both tangent terms,
//   dW[c'][c Pl + q] += scale sum_p sum_m (dVa[p][c' NLM + l l + m] Ta[p][c NT + toff + q nm + m]
//                                          + dVb[..] Tb[..]),
// dV arrays with element stride esv (tangent-number arrays: 2).
void launch_wgrad_mix_tc(const float* dVa, const float* dVb, int esv, const float* Ta, const float* Tb, int P, int C,
                         int NLM, int NT, int l, int Pl, int toff, float scale, float* dW, float* part, int* flags,
                         cudaStream_t s) {
  if (P <= 0) return;
  static bool init = false;
  static int sms = 0;
  if (!init) {
    cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wtc::kSmem);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    init = true;
  }
  const int nm = 2 * l + 1;
  const int Pv = P * nm;                               // virtual pairs (pair, m)
  // rows: the C Pl columns of dW (T side), cols: the C rows (dV side)
  WgOp tA{Ta + toff, C * NT, NT, nm, 1, Pl, nm}, tB{Tb + toff, C * NT, NT, nm, 1, Pl, nm};
  WgOp vA{dVa + (size_t)l * l * esv, C * NLM * esv, NLM * esv, nm, esv, 1, 0};
  WgOp vB{dVb + (size_t)l * l * esv, C * NLM * esv, NLM * esv, nm, esv, 1, 0};
  const int N = C, K = C * Pl;
  const int nQp = (N + 15) / 16 * 16;
  const int nchunks = (Pv + wtc::kPairs - 1) / wtc::kPairs;
  const int cpc = (nchunks + std::max(sms, 1) - 1) / std::max(sms, 1);
  const int nz = (nchunks + cpc - 1) / cpc;
  k_wgrad_tc<<<nz, wtc::kThr, wtc::kSmem, s>>>(tA, vA, tB, vB, K, N, nQp, Pv, cpc, 0, K, scale, part, flags,
                                              1ll << 31);
  k_chunk_sum<<<(N * K + 255) / 256, 256, 0, s>>>(part, nz, N, K, dW, K, 0);
}

void launch_wgrad_mix(const float* dV, int esv, const float* T, int P, int C, int NLM, int NT, int l, int Pl,
                      int toff, float scale, float* dW, float* part, cudaStream_t s) {
  if (P <= 0) return;
  // about four blocks per SM
  const int chunk = std::max(kMixG, (P + 152 * 4 - 1) / (152 * 4));
  const int nblk = (P + chunk - 1) / chunk;
  const int nm = 2 * l + 1;
  const size_t smem = sizeof(float) * kMixG * (size_t)(C * nm + C * Pl * nm);
  k_wgrad_mix<<<nblk, 256, smem, s>>>(dV, esv, T, P, C, NLM, NT, l, Pl, toff, scale, part, chunk);
  const int n_out = C * C * Pl;
  k_chunk_sum<<<(n_out + 255) / 256, 256, 0, s>>>(part, nblk, 1, n_out, dW, n_out, 0);
}

size_t wgrad_part_floats() {
  // k_wgrad: chunks x N x K <= (608 / tiles + 1) x tiles 64 x 64; k_wgrad_mix:
  // at most 608 blocks of C C P_l <= 16 x 16 x 4 outputs
  return std::max<size_t>((size_t)(152 * 4 + 8) * kWT * kWT, (size_t)(152 * 4 + 8) * 1024);
}

void launch_sumsq(const float* g, int n, double* out, cudaStream_t s) { k_sumsq<<<1, 1024, 0, s>>>(g, n, out); }

void launch_ascent(const float* w, const float* g, int n, double rho, const double* norm2, float* w_out,
                   cudaStream_t s) {
  k_ascent<<<(n + 255) / 256, 256, 0, s>>>(w, g, n, rho, norm2, w_out);
}

void launch_axpy(const float* w, const float* d, double scale, int n, float* w_out, cudaStream_t s) {
  k_axpy<<<(n + 255) / 256, 256, 0, s>>>(w, d, scale, n, w_out);
}

void launch_adam(float* w, const float* g, float* m, float* v, int n, double lr, int t, cudaStream_t s) {
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(w, g, m, v, n, lr, 0.9, 0.999, 1e-8, t);
}

void launch_apply(const float* flat, int rows, int cols, float scale, float* t_out, float* n_out, cudaStream_t s) {
  k_apply<<<(rows * cols + 255) / 256, 256, 0, s>>>(flat, rows, cols, scale, t_out, n_out);
}

void launch_apply_mix(const float* flat, int rows, int C, int pl, int pu, const int* q, float scale, float* n_out,
                      cudaStream_t s) {
  if (pl < 1 || pl > kMixQ || rows * C * pl <= 0) return;
  MixQ qm{};
  for (int k = 0; k < pl; ++k) qm.q[k] = q[k];
  k_apply_mix<<<(rows * C * pl + 255) / 256, 256, 0, s>>>(flat, rows, C, pl, pu, qm, scale, n_out);
}

}  // namespace al
