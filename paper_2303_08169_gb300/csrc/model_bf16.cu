// model_bf16.cu - BF16 tensor-core pair passes (tcgen05.mma, FP32 accumulation
// in TMEM) for the 16-channel, latent-128, energy-32 model with two or more
// layers at l_max 0, 1 or 2 (every kernel is instantiated per l_max).
//
// Same model and same pass order as the FP32 path (model_fp32.cu): forward
// passes, a fused last-layer forward + adjoint, then the adjoint passes
// (forces f = -dE/dr, Eq. 1).  Differences:
//  * tiles of 128 pairs, one persistent CTA of 512 threads per SM; thread t
//    owns tile row r = t % 128 (its TMEM lane) and column quarter t / 128;
//  * every per-pair GEMM (two-body, embedding, env, mixing, latent, energy
//    and their adjoints) runs on tcgen05.mma with BF16 operands in
//    128-byte-swizzled shared memory and FP32 accumulators in TMEM; the
//    adjoint GEMMs read the forward weight images as MN-major operands;
//  * pre-activations stay in TMEM between a GEMM and its adjoint;
//  * channel mixing is (l_max + 1)^2 MMAs, one per output component (l3, m),
//    over K-slices of one tile holding the tensor-product outputs;
//  * the forward layer-k pass is split in two (TP + mixing; latent MLP) so
//    that the weights of every kernel stay resident in shared memory; its
//    adjoint is one kernel (no per-atom sum lies between its two halves);
//  * sigmoid via tanh.approx.f32.
// Everything else (geometry, tensor products, envelope, residuals,
// reductions) is FP32 on CUDA cores.  x^k, S^k and V^k are stored in FP16
// between passes, dV in the operand type, the other gradients in FP32.
// Per-atom sums use the per-(tile, atom) partials of the FP32 path with
// 128-pair tiles, reduced per atom once per producing pass.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "model.h"
#include "tp_tables.inc"
#include "umma.cuh"

namespace al {
namespace {

using namespace umma;

// Limit of every bounded mbarrier wait (clock cycles) and the failure
// injection of the failure-detection tests: when c_no_weight_copies is set,
// no kernel issues its weight copies, so the weight barrier's wait runs out
// (nothing is in flight), the kernel skips its MMAs and raises the timeout
// flag that the host turns into ALLEGRO_E_TIMEOUT.
__constant__ long long c_wait_cycles = 1ll << 31;
__constant__ int c_no_weight_copies = 0;

constexpr int kT = 128;
// threads of a CTA: thread t owns tile row r = t % 128 (its TMEM lane) and
// column quarter h = t / 128 of every epilogue (16 warps per SM)
constexpr int kThr4 = 512;
constexpr int D = 128, C = 16, E = 32, NB = 8;
constexpr float kR2 = 0.70710678118654752f;
// odd row strides of per-row shared arrays (32 consecutive rows hit 32 banks)
constexpr int EP = C + 1, GP = 9;

__host__ __device__ constexpr int l_of(int lm) { return lm == 0 ? 0 : (lm < 4 ? 1 : 2); }

// Shapes of the passes at l_max = LM: NLM spherical components, NS = P_0
// scalar paths per channel, CL = C NLM features of V^k and Gamma, KH = D + C NS
// inputs of the first latent layer, NW0 = C (LM + 1) embedding outputs, NT
// tensor-product outputs per channel (the tables generated by gen_tp.cpp:
// path-major within each output order l, offset toff(l), P(l) paths).  The
// mixing operand holds output component j's K-slice (C P_l columns, channel
// c's paths at c P_l + p) from column slice(j).
template <int LM>
struct Tc {
  static_assert(LM >= 0 && LM <= 2, "l_max 0, 1 or 2");
  static constexpr int NLM = (LM + 1) * (LM + 1), NS = LM + 1, CL = C * NLM, KH = D + C * NS, NW0 = C * (LM + 1);
  static constexpr int NT = LM == 0 ? TP0_NT : LM == 1 ? TP1_NT : TP2_NT;
  static constexpr int CLP = CL + 1;                 // odd stride of per-row dGamma staging
  __host__ __device__ static constexpr int P(int l) { return LM == 0 ? tp0_P(l) : LM == 1 ? tp1_P(l) : tp2_P(l); }
  __host__ __device__ static constexpr int toff(int l) {
    return LM == 0 ? tp0_toff(l) : LM == 1 ? tp1_toff(l) : tp2_toff(l);
  }
  __host__ __device__ static constexpr int slice(int j) {
    int s = 0;
    for (int q = 0; q < j; ++q) s += C * P(l_of(q));
    return s;
  }
  template <class S>
  static AL_DEV void fwd(const S* V, const S* G, S* T) {
    if constexpr (LM == 0) tp0_fwd(V, G, T);
    else if constexpr (LM == 1) tp1_fwd(V, G, T);
    else tp2_fwd(V, G, T);
  }
  template <class S>
  static AL_DEV void fwd_scalar(const S* V, const S* G, S* T) {
    if constexpr (LM == 0) tp0_fwd_scalar(V, G, T);
    else if constexpr (LM == 1) tp1_fwd_scalar(V, G, T);
    else tp2_fwd_scalar(V, G, T);
  }
  template <class S>
  static AL_DEV void bwd(const S* V, const S* G, const S* dT, S* dV, S* dG) {
    if constexpr (LM == 0) tp0_bwd(V, G, dT, dV, dG);
    else if constexpr (LM == 1) tp1_bwd(V, G, dT, dV, dG);
    else tp2_bwd(V, G, dT, dV, dG);
  }
  template <class S>
  static AL_DEV void bwd_scalar(const S* V, const S* G, const S* dT, S* dV, S* dG) {
    if constexpr (LM == 0) tp0_bwd_scalar(V, G, dT, dV, dG);
    else if constexpr (LM == 1) tp1_bwd_scalar(V, G, dT, dV, dG);
    else tp2_bwd_scalar(V, G, dT, dV, dG);
  }
  static constexpr uint32_t kImgEmb = sw128_bytes(NW0, 128);
  static constexpr uint32_t kOpT = sw128_bytes(128, (C * NT + 63) / 64 * 64);
};
static_assert(Tc<2>::slice(1) == 48 && Tc<2>::slice(4) == 240 && Tc<2>::slice(9) == C * TP2_NT, "l_max 2 slices");
static_assert(Tc<1>::slice(1) == 32 && Tc<1>::slice(4) == C * TP1_NT && Tc<0>::slice(1) == C * TP0_NT,
              "l_max 0 / 1 slices");

constexpr uint32_t kImgTb0 = sw128_bytes(128, 64);
constexpr uint32_t kImgTb1 = sw128_bytes(128, 128);
constexpr uint32_t kImgE0 = sw128_bytes(32, 128);
constexpr uint32_t kImgEnv = sw128_bytes(16, 128);
constexpr uint32_t kImgLat0 = sw128_bytes(128, 192);   // KH <= 176 inputs used
constexpr uint32_t kImgLat1 = sw128_bytes(128, 128);
constexpr uint32_t kImgMix = sw128_bytes(16, 64);      // C P_l <= 64 inputs used
constexpr uint32_t kOp128 = sw128_bytes(128, 128);
constexpr uint32_t kOp64 = sw128_bytes(128, 64);
constexpr uint32_t kOpH = sw128_bytes(128, 192);

// Operand type of the tensor-core GEMMs: BF16 (the precision the method
// names for per-pair GEMMs) or FP16 (same tensor-core rate, 3 more mantissa
// bits).  Both accumulate in FP32.
template <class T> struct Op;
template <> struct Op<__nv_bfloat16> {
  static constexpr uint32_t fmt = 1;
  static AL_DEV uint16_t bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
  static AL_DEV float round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
  // (a, b) rounded into one 32-bit word, a in the low half; one conversion
  static AL_DEV uint32_t pack2(float a, float b, float2* back = nullptr) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    if (back) *back = __bfloat1622float2(h);
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
  }
};
template <> struct Op<__half> {
  static constexpr uint32_t fmt = 0;
  static AL_DEV uint16_t bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
  static AL_DEV float round(float x) { return __half2float(__float2half_rn(x)); }
  static AL_DEV uint32_t pack2(float a, float b, float2* back = nullptr) {
    const __half2 h = __floats2half2_rn(a, b);
    if (back) *back = __half22float2(h);
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
  }
};

// Split operands (the two-body MLP and the energy hidden layer in the split
// mode): x = hi + lo with hi = rn(x), lo = rn(x - hi), and a product
// A B ~ A_hi B_hi + A_lo B_hi + A_hi B_lo as three MMAs into one FP32
// accumulator, which keeps about twice the operand type's mantissa bits.

AL_DEV float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
AL_DEV float sgm(float z) { return fmaf(0.5f, tanh_fast(0.5f * z), 0.5f); }
AL_DEV float silu_b(float z) { return z * sgm(z); }
AL_DEV float dsilu_b(float z) {
  const float s = sgm(z);
  return s * (1.0f + z * (1.0f - s));
}

// y = (SiLU(x), dSiLU/dx(x)) with the tensor-core passes' own arithmetic
__global__ void k_silu_probe(int n, const float* __restrict__ x, float* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[2 * i] = silu_b(x[i]);
  y[2 * i + 1] = dsilu_b(x[i]);
}

// ---------------------------------------------------------------------------
struct Meta {
  int pi[kT], pj[kT], code[kT], seg[kT], atom[kT], sstart[kT + 1];
  int nseg, np, p0, tile;
  int wc[4];
};

// Neighbour-list entries of tile row t (threads t < 128), loaded one tile
// ahead into registers: i, j, image code, optionally the species of i, and
// for the first lane of each warp the centre atom of the row before it
struct MetaPre {
  int i, j, code, prev, zi;
};
template <bool kSpecies = false>
AL_DEV MetaPre meta_load(const PassBufs& b, int tile, int P) {
  MetaPre q{-1, 0, 62, -1, 0};
  const int t = threadIdx.x;
  if (t < kT) {
    const int p0 = tile * kT;
    const int np = min(kT, P - p0);
    if (t < np) {
      q.i = b.pi[p0 + t];
      q.j = b.pj[p0 + t];
      q.code = b.pcode[p0 + t];
      if (kSpecies) q.zi = b.species[q.i];
    }
    if ((t & 31) == 0 && t > 0 && t - 1 < np) q.prev = b.pi[p0 + t - 1];
  }
  return q;
}

AL_DEV void meta_setup(const PassBufs& b, int tile, int P, Meta& m, const MetaPre& q) {
  const int t = threadIdx.x;
  const int p0 = tile * kT;
  const int np = min(kT, P - p0);
  bool head = false;
  unsigned mask = 0u;
  int i = -1;
  // (every pass ends its tile with a barrier, so the previous tile is done with m)
  if (t < kT) {
    if (t < np) {
      i = q.i;
      m.pi[t] = i;
      m.pj[t] = q.j;
      m.code[t] = q.code;
    } else {
      m.pi[t] = 0;
      m.pj[t] = 0;
      m.code[t] = 62;
    }
    int prev = __shfl_up_sync(0xffffffffu, i, 1);
    if ((t & 31) == 0) prev = q.prev;
    head = t < np && (t == 0 || i != prev);          // first pair of a centre atom's run
    mask = __ballot_sync(0xffffffffu, head);
    if ((t & 31) == 0) m.wc[t >> 5] = __popc(mask);
  }
  __syncthreads();
  if (t < kT) {
    int base = 0;
    for (int w = 0; w < (t >> 5); ++w) base += m.wc[w];
    const unsigned below = (t & 31) == 31 ? 0xffffffffu : ((2u << (t & 31)) - 1u);
    const int sg = base + __popc(mask & below) - 1;
    m.seg[t] = t < np ? sg : 0;
    if (head) {
      m.sstart[sg] = t;
      m.atom[sg] = i;
    }
    if (t == 0) {
      const int nseg = m.wc[0] + m.wc[1] + m.wc[2] + m.wc[3];
      m.nseg = nseg;
      m.np = np;
      m.p0 = p0;
      m.tile = tile;
      m.sstart[nseg] = np;
    }
  }
  __syncthreads();
}

// part[(tile + atom) * W + x] = sum over the segment's pairs of f(p, x)
// (four interleaved partial sums in a fixed order: a quarter of the
// dependent chain)
template <class F>
AL_DEV void seg_store(float* __restrict__ part, const Meta& m, int W, F&& f) {
  for (int idx = threadIdx.x; idx < m.nseg * W; idx += blockDim.x) {
    const int s = idx / W, x = idx % W;
    const int s1 = m.sstart[s + 1];
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    int p = m.sstart[s];
    for (; p + 3 < s1; p += 4) {
      a0 += f(p, x);
      a1 += f(p + 1, x);
      a2 += f(p + 2, x);
      a3 += f(p + 3, x);
    }
    for (; p < s1; ++p) a0 += f(p, x);
    part[(size_t)(m.tile + m.atom[s]) * W + x] = (a0 + a1) + (a2 + a3);
  }
}

// Per-pair arrays of this path use a tile-SoA layout: element (pair p,
// feature f) of a W-wide array lives at ((p / 128) * W + f) * 128 + p % 128,
// so the 32 lanes of a warp (consecutive tile rows) touch consecutive floats.
// (tile from a register: with W and f known at compile time the feature
// offsets fold into the load/store immediates)
AL_DEV size_t sidx(int tile, int W, int f, int r) { return ((size_t)tile * W + f) * kT + r; }

// The forward per-pair state of these passes (x^k, S^k, V^k) is stored in
// FP16 between passes, two features per 32-bit word in tile-SoA order: word
// (tile, f / 2, r) holds features f (low half) and f + 1 (high half) of tile
// row r.  V^k is stored component-major (feature lm C + c), so that two
// neighbouring channels share a word.  Gradients stay FP32.  (The buffers are
// the FP32 path's, of which these passes use the first half.)
AL_DEV size_t hidx(int tile, int W, int f, int r) { return ((size_t)tile * (W >> 1) + (f >> 1)) * kT + r; }
// the stored value: producers that also feed an operand use it too, so that
// every consumer of x^k sees the same (FP16) value
AL_DEV float r16(float x) { return __half2float(__float2half_rn(x)); }
AL_DEV float2 ldh2(const float* a, size_t i) { return __half22float2(reinterpret_cast<const __half2*>(a)[i]); }
AL_DEV void sth2(float* a, size_t i, float x, float y) { reinterpret_cast<__half2*>(a)[i] = __floats2half2_rn(x, y); }
AL_DEV uint32_t h2word(float x, float y) {
  const __half2 v = __floats2half2_rn(x, y);
  uint32_t u;
  memcpy(&u, &v, 4);
  return u;
}
// dV^k is consumed only as the mixing-adjoint MMA operand of pass B1^T, so
// it is stored in the operand type itself (component-major, two channels per
// word, the layout of V^k): the same values the operand held when dV^k was
// FP32, at half the bytes
template <class Tin>
AL_DEV void st_opw(float* a, size_t i, float x, float y) { reinterpret_cast<uint32_t*>(a)[i] = Op<Tin>::pack2(x, y); }

// L2 prefetch of tile nt's block of a tile-SoA array (W features x 128 rows,
// contiguous) and of its slice of the neighbour list: issued by one thread
// one tile ahead, so that the next tile's loads hit L2
AL_DEV void prefetch_rows(const float* a, int W, int nt) {
  const char* p = reinterpret_cast<const char*>(a + (size_t)nt * W * kT);
  const uint32_t bytes = (uint32_t)W * kT * 4;
  for (uint32_t o = 0; o < bytes; o += 32768u) bulk_prefetch_l2(p + o, min(32768u, bytes - o));
}
// the same for an FP16-pair array (W features, W / 2 words per row)
AL_DEV void prefetch_rows_h(const float* a, int W, int nt) {
  const char* p = reinterpret_cast<const char*>(a) + (size_t)nt * (W / 2) * kT * 4;
  const uint32_t bytes = (uint32_t)(W / 2) * kT * 4;
  for (uint32_t o = 0; o < bytes; o += 32768u) bulk_prefetch_l2(p + o, min(32768u, bytes - o));
}
AL_DEV void prefetch_meta(const PassBufs& b, int nt) {
  bulk_prefetch_l2(b.pi + (size_t)nt * kT, kT * 4);
  bulk_prefetch_l2(b.pj + (size_t)nt * kT, kT * 4);
  bulk_prefetch_l2(b.pcode + (size_t)nt * kT, kT * 4);
}

// the same for columns [x0, x0 + nx) of W-wide partial rows, f(p, x - x0)
template <class F>
AL_DEV void seg_store_cols(float* __restrict__ part, const Meta& m, int W, int x0, int nx, F&& f) {
  for (int idx = threadIdx.x; idx < m.nseg * nx; idx += blockDim.x) {
    const int s = idx / nx, x = idx % nx;
    const int s1 = m.sstart[s + 1];
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    int p = m.sstart[s];
    for (; p + 3 < s1; p += 4) {
      a0 += f(p, x);
      a1 += f(p + 1, x);
      a2 += f(p + 2, x);
      a3 += f(p + 3, x);
    }
    for (; p < s1; ++p) a0 += f(p, x);
    part[(size_t)(m.tile + m.atom[s]) * W + x0 + x] = (a0 + a1) + (a2 + a3);
  }
}

// Gamma (or dGamma) per atom: k_atom_sums reduces the per-(tile, atom)
// partials of the producing pass (in tile order) into gsum[i][x]; the
// consumers copy the rows of the tile's first kSegCap centre atoms into
// shared memory, and rows of later segments read gsum directly.
constexpr int kSegCap = 8;
template <int CL>
AL_DEV void stage_g(const float* __restrict__ gsum, const Meta& m, float* s) {
  const int ns = min(m.nseg, kSegCap);
  for (int idx = threadIdx.x; idx < ns * (CL / 4); idx += blockDim.x) {
    const int sg = idx / (CL / 4), x = idx % (CL / 4);
    reinterpret_cast<float4*>(s + sg * CL)[x] = reinterpret_cast<const float4*>(gsum + (size_t)m.atom[sg] * CL)[x];
  }
}
template <int NLM>
AL_DEV void get_g(const float* s, const float* __restrict__ gsum, const Meta& m, int r, bool valid, int c, float* G) {
  constexpr int CL = C * NLM;
  if (!valid) {
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) G[lm] = 0.0f;
    return;
  }
  const int sg = m.seg[r];
  const float* g = sg < kSegCap ? s + sg * CL + c * NLM : gsum + (size_t)m.pi[r] * CL + c * NLM;
#pragma unroll
  for (int lm = 0; lm < NLM; ++lm) G[lm] = g[lm];
}

// gsum[i][x] = sum over the tiles t0..t1 that hold atom i's pairs of the
// partial row (t + i), in tile order (zero for an atom without pairs)
template <int CL>
__global__ void k_atom_sums(const float* __restrict__ part, const int* __restrict__ row_ptr, int n,
                            const int* __restrict__ flags, float* __restrict__ gsum) {
  if (*flags & 1) return;
  constexpr int nq = CL / 4;
  const int64_t total = (int64_t)n * nq;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / nq), x = (int)(idx % nq);
    const int p0 = row_ptr[i], p1 = row_ptr[i + 1];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p1 > p0)
      for (int tt = p0 / kT; tt <= (p1 - 1) / kT; ++tt) {
        const float4 v = reinterpret_cast<const float4*>(part + (size_t)(tt + i) * CL)[x];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
      }
    reinterpret_cast<float4*>(gsum + (size_t)i * CL)[x] = acc;
  }
}

template <int LM>
AL_DEV void geo_from_delta(float dx, float dy, float dz, float rc, float u[3], float& d, float& fc, float& dfc,
                           float* Y) {
  d = sqrtf(dx * dx + dy * dy + dz * dz);
  const float inv = 1.0f / d;
  u[0] = dx * inv;
  u[1] = dy * inv;
  u[2] = dz * inv;
  envelope(d, rc, fc, dfc);
  sph_harm<LM>(u[0], u[1], u[2], Y);
}

// Pass A: the pair separation in FP64 (the arithmetic that decides pair
// membership), rounded to FP32 and kept per pair (tile-SoA, 3 floats) for the
// later passes, which read it instead of gathering two FP64 positions.
template <int LM>
AL_DEV void geometry_first(const PassBufs& b, int tile, int r, float rc, int i, int j, int code, float u[3],
                           float& d, float& fc, float& dfc, float* Y) {
  Box box{{b.L[0], b.L[1], b.L[2]}};
  double dd[3];
  pair_delta(b.wpos, i, j, code, box, dd);
  const float dx = (float)dd[0], dy = (float)dd[1], dz = (float)dd[2];
  b.dR[sidx(tile, 3, 0, r)] = dx;
  b.dR[sidx(tile, 3, 1, r)] = dy;
  b.dR[sidx(tile, 3, 2, r)] = dz;
  geo_from_delta<LM>(dx, dy, dz, rc, u, d, fc, dfc, Y);
}
template <int LM>
AL_DEV void geometry(const PassBufs& b, int tile, int r, float rc, float u[3], float& d, float& fc, float& dfc,
                     float* Y) {
  geo_from_delta<LM>(b.dR[sidx(tile, 3, 0, r)], b.dR[sidx(tile, 3, 1, r)], b.dR[sidx(tile, 3, 2, r)], rc, u, d, fc,
                     dfc, Y);
}

// ---- MMA issue helpers (single thread) ----
// D[128 x N] = A[128 x K-slice from k-step kk0, nk steps] * B, B either the
// K-major image of an [N x K] matrix or (b_mn) the image of a [P x N] matrix
// read MN-major.
template <class Tin>
AL_DEV void mma_k(uint32_t d, const uint8_t* A, int kk0, const uint8_t* B, int N, int nk, bool b_mn, int P,
                  bool acc = false) {
  const uint32_t idesc = idesc_f16kind(128, N, b_mn, Op<Tin>::fmt);
  const uint32_t a = smem_u32(A), bb = smem_u32(B);
  for (int i = 0; i < nk; ++i) {
    const int kk = kk0 + i;
    const uint32_t aoff = (uint32_t)((kk >> 2) * (128 * 128) + (kk & 3) * 32);
    uint64_t bd;
    if (b_mn) bd = desc_sw128_mn(bb + (uint32_t)(i * 16 * 128), (uint32_t)(P * 128), 1024u);
    else bd = desc_sw128(bb + (uint32_t)((i >> 2) * (N * 128) + (i & 3) * 32));
    mma_bf16(d, desc_sw128(a + aoff), bd, idesc, (i > 0 || acc) ? 1u : 0u);
  }
}

struct Mma {
  uint64_t* bar;
  uint32_t phase;
  int* err;
  // all threads: publish smem operands, thread 0 issues, everyone waits
  template <class F>
  AL_DEV void run(F&& issue) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    const bool skip = *err != 0;
    if (!skip) {
      if (threadIdx.x == 0) {
        tc_fence_after();
        issue();
        mma_commit(bar);
      }
      if (!mbar_wait(bar, phase, c_wait_cycles)) *err = 1;
      phase ^= 1u;
    }
    tc_fence_after();
  }
  // all threads: publish smem operands, thread 0 issues without a commit; the
  // next run() commits these MMAs together with its own and waits for all,
  // so CUDA-core work between the two overlaps them
  template <class F>
  AL_DEV void issue(F&& f) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (*err == 0 && threadIdx.x == 0) {
      tc_fence_after();
      f();
    }
  }
  // run() in two halves: start() publishes, issues and commits; work that
  // touches neither the MMAs' operands nor their accumulator columns may run
  // before wait(), which every thread that called start() must reach
  bool live = false;
  template <class F>
  AL_DEV void start(F&& issue) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    live = *err == 0;
    if (live && threadIdx.x == 0) {
      tc_fence_after();
      issue();
      mma_commit(bar);
    }
  }
  AL_DEV void wait() {
    if (live) {
      if (!mbar_wait(bar, phase, c_wait_cycles)) *err = 1;
      phase ^= 1u;
    }
    tc_fence_after();
  }
};

AL_DEV uint32_t lanes(uint32_t tmem) { return tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16); }

// SiLU epilogue of a 128-column pre-activation z at TMEM column col0 whose
// adjoint needs SiLU'(z) later: thread (r, h) turns its 32 columns into
// SiLU(z), handed to st(r, n0, v[16]) 16 at a time, and writes SiLU'(z) back
// over z (one sigmoid for both); the adjoint epilogue reads SiLU' directly.
// The store is waited for before returning.
template <class St>
AL_DEV void epi_silu_keep_grad(uint32_t tmem, int col0, St&& st) {
  const int r = threadIdx.x & (kT - 1), h = threadIdx.x >> 7;
  const uint32_t base = lanes(tmem) + (uint32_t)(col0 + 32 * h);
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    float v[16], o[16];
    tmem_ld16(base + 16 * hf, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float z = v[q], sg = sgm(z);
      o[q] = z * sg;                                 // silu_b(z)
      v[q] = sg * (1.0f + z * (1.0f - sg));          // dsilu_b(z)
    }
    st(r, 32 * h + 16 * hf, o);
    tmem_st16(base + 16 * hf, v);
  }
  tmem_wait_st();
}

// thread (r, h) of a CTA with nq = blockDim / 128 column groups visits
// columns [h N/nq, (h+1) N/nq) of an N-wide accumulator at TMEM column col0,
// 16 at a time: f(r, n0, v[16])
template <class F>
AL_DEV void epi(uint32_t tmem, int col0, int N, F&& f) {
  const int r = threadIdx.x & (kT - 1), h = threadIdx.x >> 7;
  const int w = N / (int)(blockDim.x >> 7);
  const uint32_t base = lanes(tmem);
  if (w == 32) {                                     // one 32-column load and wait
    float v[32];
    tmem_ld32(base + (uint32_t)(col0 + 32 * h), v);
    f(r, 32 * h, v);
    f(r, 32 * h + 16, v + 16);
    return;
  }
  for (int n0 = h * w; n0 < (h + 1) * w; n0 += 16) {
    float v[16];
    tmem_ld16(base + (uint32_t)(col0 + n0), v);
    f(r, n0, v);
  }
}

template <class Tin>
AL_DEV void st8(uint8_t* A, uint32_t off, const float* v) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) w[q] = Op<Tin>::pack2(v[2 * q], v[2 * q + 1]);
  *reinterpret_cast<uint4*>(A + off) = make_uint4(w[0], w[1], w[2], w[3]);
}
// v = hi + lo: hi into Ahi at off, lo into Alo at off_lo (8 elements each)
template <class Tin>
AL_DEV void st8_split(uint8_t* Ahi, uint32_t off, uint8_t* Alo, uint32_t off_lo, const float* v) {
  uint32_t wh[4], wl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 hb;
    wh[q] = Op<Tin>::pack2(v[2 * q], v[2 * q + 1], &hb);
    wl[q] = Op<Tin>::pack2(v[2 * q] - hb.x, v[2 * q + 1] - hb.y);
  }
  *reinterpret_cast<uint4*>(Ahi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
  *reinterpret_cast<uint4*>(Alo + off_lo) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}
template <class Tin>
AL_DEV void st16(uint8_t* A, int r, int c0, const float* v) {
  st8<Tin>(A, sw128_off(r, c0, 128), v);
  st8<Tin>(A, sw128_off(r, c0 + 8, 128), v + 8);
}
// 16 FP16 operand values of row r from column c0 (c0 % 8 == 0) of a 128-row
// swizzled tile, as floats (the inverse of st16 for FP16 operands)
AL_DEV void ld16_h(const uint8_t* A, int r, int c0, float* x) {
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const uint4 u = *reinterpret_cast<const uint4*>(A + sw128_off(r, c0 + 8 * g, 128));
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __half2 h2;
      memcpy(&h2, &w[q], 4);
      const float2 f = __half22float2(h2);
      x[8 * g + 2 * q] = f.x;
      x[8 * g + 2 * q + 1] = f.y;
    }
  }
}

template <class Tin>
AL_DEV void st4(uint8_t* A, uint32_t off, const float* v) {
  const uint32_t w0 = Op<Tin>::pack2(v[0], v[1]);
  const uint32_t w1 = Op<Tin>::pack2(v[2], v[3]);
  *reinterpret_cast<uint2*>(A + off) = make_uint2(w0, w1);
}
// hi part into Ahi, lo part into Alo (same row and columns)
template <class Tin>
AL_DEV void st16_split(uint8_t* Ahi, uint8_t* Alo, int r, int c0, const float* v) {
  const uint32_t o0 = sw128_off(r, c0, 128), o1 = sw128_off(r, c0 + 8, 128);
  st8_split<Tin>(Ahi, o0, Alo, o0, v);
  st8_split<Tin>(Ahi, o1, Alo, o1, v + 8);
}
// operand store of an epilogue: hi (and lo) parts in split mode
template <class Tin, bool kSplit>
AL_DEV void st16_op(uint8_t* A, uint8_t* Alo, int r, int c0, const float* v) {
  if (kSplit) st16_split<Tin>(A, Alo, r, c0, v);
  else st16<Tin>(A, r, c0, v);
}
template <class Tin>
AL_DEV void st1(uint8_t* A, int r, int c, float v) {
  *reinterpret_cast<uint16_t*>(A + sw128_off(r, c, 128)) = Op<Tin>::bits(v);
}
// N (4, 8 or 12) consecutive operand columns from c0 (c0 % 4 == 0) of row r
// as 8- and 16-byte stores (one or two per row instead of N 2-byte ones)
template <class Tin, int N>
AL_DEV void st_cols(uint8_t* A, int r, int c0, const float* v) {
  static_assert(N == 4 || N == 8 || N == 12, "4, 8 or 12 columns");
  if constexpr (N == 4) {
    st4<Tin>(A, sw128_off(r, c0, 128), v);
  } else if constexpr (N == 8) {
    if ((c0 & 7) == 0) {
      st8<Tin>(A, sw128_off(r, c0, 128), v);
    } else {
      st4<Tin>(A, sw128_off(r, c0, 128), v);
      st4<Tin>(A, sw128_off(r, c0 + 4, 128), v + 4);
    }
  } else {
    if ((c0 & 7) == 0) {
      st8<Tin>(A, sw128_off(r, c0, 128), v);
      st4<Tin>(A, sw128_off(r, c0 + 8, 128), v + 8);
    } else {
      st4<Tin>(A, sw128_off(r, c0, 128), v);
      st8<Tin>(A, sw128_off(r, c0 + 4, 128), v + 4);
    }
  }
}

// Operand staging of FP16-pair state in two steps, so that a tile's loads
// are all issued before any of them is waited for: ld_row reads the N / 2
// words of features [f0, f0 + N) (f0 even) of tile row r of a W-wide array
// (zeros for an invalid row); st_row writes them into operand columns
// [c0, c0 + N) of row r (FP16 operands take the words as they are).
template <int N>
AL_DEV void ld_row(uint32_t* w, const float* __restrict__ g, int tile, int r, int W, int f0, bool valid) {
#pragma unroll
  for (int q = 0; q < N / 2; ++q)
    w[q] = valid ? reinterpret_cast<const uint32_t*>(g)[hidx(tile, W, f0 + 2 * q, r)] : 0u;
}
template <class Tin, int N>
AL_DEV void st_row(uint8_t* A, int r, int c0, const uint32_t* w) {
#pragma unroll
  for (int k = 0; k < N; k += 8) {
    uint32_t u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (Op<Tin>::fmt == 0) {
        u[q] = w[k / 2 + q];
      } else {
        __half2 hh;
        memcpy(&hh, &w[k / 2 + q], 4);
        const float2 f = __half22float2(hh);
        u[q] = Op<Tin>::pack2(f.x, f.y);
      }
    }
    *reinterpret_cast<uint4*>(A + sw128_off(r, c0 + k, 128)) = make_uint4(u[0], u[1], u[2], u[3]);
  }
}

AL_DEV uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// Common prologue/epilogue of every persistent pass kernel.
#define BF_PROLOGUE(WBYTES, LOADS)                                                \
  extern __shared__ uint8_t smem_raw[];                                           \
  __shared__ Meta m;                                                              \
  __shared__ uint64_t bars[2];                                                    \
  __shared__ uint32_t tslot;                                                      \
  __shared__ int err;                                                             \
  uint8_t* sm = align1024(smem_raw);                                              \
  if (threadIdx.x < 32) tmem_alloc(&tslot, 512);                                  \
  if (threadIdx.x == 0) {                                                         \
    mbar_init(&bars[0], 1);                                                       \
    mbar_init(&bars[1], 1);                                                       \
    mbar_fence_init();                                                            \
    err = 0;                                                                      \
  }                                                                               \
  tc_fence_before();                                                              \
  __syncthreads();                                                                \
  tc_fence_after();                                                               \
  const uint32_t tmem = tslot;                                                    \
  if (threadIdx.x == 0 && !c_no_weight_copies) {                                 \
    mbar_expect_tx(&bars[1], (WBYTES));                                           \
    LOADS;                                                                        \
  }                                                                               \
  if (!mbar_wait(&bars[1], 0, c_wait_cycles)) err = 1;                            \
  __syncthreads();                                                                \
  Mma mm{&bars[0], 0u, &err};                                                     \
  const int P = (int)min((int64_t)*b.n_pairs, b.capacity);                        \
  const int ntiles = (*b.flags & 1) ? 0 : (P + kT - 1) / kT;

#define BF_EPILOGUE                                                               \
  tc_fence_before();                                                              \
  __syncthreads();                                                                \
  if (threadIdx.x < 32) tmem_dealloc(tmem, 512);                                  \
  if (err && threadIdx.x == 0) atomicOr(const_cast<int*>(b.flags), kFlagTimeoutBit);

constexpr int kFlagTimeoutBit = 4;

// two-body input row (16 columns, 12 used); split mode: [hi | lo | hi]
template <class Tin, bool kSplit>
AL_DEV void st_h0(uint8_t* H0, int r, const float* h0) {
  if (kSplit) {
    float hi[16], lo[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      hi[q] = Op<Tin>::round(h0[q]);
      lo[q] = h0[q] - hi[q];
    }
    st16<Tin>(H0, r, 0, hi);                          // rounding hi again is exact
    st16<Tin>(H0, r, 16, lo);
    st16<Tin>(H0, r, 32, hi);
  } else {
    st16<Tin>(H0, r, 0, h0);
  }
}

// D = A B (one thread issues): plain, or the three split products
template <class Tin, bool kSplit>
AL_DEV void mma_split(uint32_t d, const uint8_t* A, const uint8_t* Alo, const uint8_t* B, const uint8_t* Blo, int N,
                      int nk, bool b_mn, int P) {
  mma_k<Tin>(d, A, 0, B, N, nk, b_mn, P);
  if (kSplit) {
    mma_k<Tin>(d, Alo, 0, B, N, nk, b_mn, P, true);
    mma_k<Tin>(d, A, 0, Blo, N, nk, b_mn, P, true);
  }
}

// ============================================================================
// Pass A: geometry, two-body MLP (12 -> 128 -> 128), x0, env1 -> Gamma^1.
// Split mode: the two-body MLP GEMMs take split operands.  The first one packs
// [h_hi | h_lo | h_hi] against the image [W_hi | W_hi | W_lo] along K (12
// inputs fit a 16-column K-step), the second adds the lo MMAs.
template <class Tin, bool kSplit, int LM>
__global__ void __launch_bounds__(kThr4, 1) k_bf_a(BfW w, PassBufs b) {
  constexpr int NLM = Tc<LM>::NLM, CL = Tc<LM>::CL;
  BF_PROLOGUE(kImgTb0 + (kSplit ? 2 : 1) * kImgTb1 + kImgEnv, {
    bulk_g2s(sm, w.tb0, kImgTb0, &bars[1]);
    bulk_g2s(sm + kImgTb0, w.tb1, kImgTb1, &bars[1]);
    bulk_g2s(sm + kImgTb0 + kImgTb1, w.env[0], kImgEnv, &bars[1]);
    if (kSplit) bulk_g2s(sm + kImgTb0 + kImgTb1 + kImgEnv, w.tb1_lo, kImgTb1, &bars[1]);
  })
  uint8_t* Wtb0 = sm;
  uint8_t* Wtb1 = Wtb0 + kImgTb0;
  uint8_t* Wenv = Wtb1 + kImgTb1;
  uint8_t* Wtb1lo = Wenv + kImgEnv;                      // split mode only
  uint8_t* H0 = Wtb1lo + (kSplit ? kImgTb1 : 0);
  uint8_t* A1 = H0 + kOp64;
  uint8_t* X = A1 + kOp128;
  uint8_t* A1lo = X + kOp128;                            // split mode only
  float* s_fc = reinterpret_cast<float*>(A1lo + (kSplit ? kOp128 : 0));
  float* s_Y = s_fc + kT;
  float* s_e = s_Y + kT * NLM;
  uint32_t* s_xs = reinterpret_cast<uint32_t*>(A1);   // [D/2][kT] x^0 words, from the x^0 epilogue to the env MMA
  // Two-body input row (species one-hot, Bessel basis), harmonics and
  // envelope of tile row r (threads r < 128) from its neighbour-list entry
  // q; zeros for a row past the list.  Row t of the next tile is formed
  // while the current tile's z2 MMA runs and kept in registers.
  float h0[16], Y[NLM], fc;
  auto pair_row = [&](int t, const MetaPre& q) {
    const int r = threadIdx.x;
    fc = 0.0f;
#pragma unroll
    for (int x = 0; x < 16; ++x) h0[x] = 0.0f;
#pragma unroll
    for (int x = 0; x < NLM; ++x) Y[x] = 0.0f;
    if (r < kT && q.i >= 0) {
      float u[3], d, dfc, B[NB];
      geometry_first<LM>(b, t, r, w.rc, q.i, q.j, q.code, u, d, fc, dfc, Y);
      bessel<NB>(d, w.rc, B, nullptr);
      const int zi = b.species[q.i], zj = b.species[q.j];
#pragma unroll
      for (int x = 0; x < 2; ++x) {                   // one-hot species (no dynamic register index)
        h0[x] = zi == x ? 1.0f : 0.0f;
        h0[2 + x] = zj == x ? 1.0f : 0.0f;
      }
#pragma unroll
      for (int x = 0; x < NB; ++x) h0[4 + x] = B[x];
    }
  };
  MetaPre mq = meta_load(b, blockIdx.x, P);
  pair_row(blockIdx.x, mq);
  for (int tile = blockIdx.x; tile < ntiles && !err; tile += gridDim.x) {
    meta_setup(b, tile, P, m, mq);
    if (threadIdx.x == 0 && tile + (int)gridDim.x < ntiles) {
      const int nt = tile + (int)gridDim.x;
      prefetch_meta(b, nt);
    }
    if (threadIdx.x < kT) {
      const int r = threadIdx.x;
      s_fc[r] = fc;
#pragma unroll
      for (int q = 0; q < NLM; ++q) s_Y[r * NLM + q] = Y[q];
      st_h0<Tin, kSplit>(H0, r, h0);
    }
    if (threadIdx.x == 0) bulk_wait_read();           // the previous tile's x^0 copy has read A1
    mm.run([&] { mma_k<Tin>(tmem + 0, H0, 0, Wtb0, 128, kSplit ? 3 : 1, false, 0); });
    epi(tmem, 0, 128, [&](int r, int n0, const float* v) {
      float o[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = silu_b(v[q]);
      st16_op<Tin, kSplit>(A1, A1lo, r, n0, o);
    });
    mq = meta_load(b, tile + (int)gridDim.x, P);     // (m holds this tile's entries from here on)
    mm.start([&] { mma_split<Tin, kSplit>(tmem + 128, A1, A1lo, Wtb1, Wtb1lo, 128, 8, false, 0); });
    pair_row(tile + (int)gridDim.x, mq);              // next tile's rows: registers and the dR store only
    mm.wait();
    epi(tmem, 128, 128, [&](int r, int n0, const float* v) {
      float o[16];
      const float fc = s_fc[r];
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = r16(fc * silu_b(v[q]));
      st16<Tin>(X, r, n0, o);
#pragma unroll
      for (int q = 0; q < 16; q += 2) s_xs[((n0 + q) >> 1) * kT + r] = h2word(o[q], o[q + 1]);
    });
    // env MMA; the x^0 tile (tile-SoA words, staged in A1, dead since z2)
    // leaves by one bulk copy issued with it
    mm.run([&] {
      mma_k<Tin>(tmem + 256, X, 0, Wenv, 16, 8, false, 0);
      bulk_s2g(b.X[0] + (size_t)tile * (D / 2) * kT, s_xs, (uint32_t)(D / 2 * kT * 4));
      bulk_commit();
    });
    if (threadIdx.x < kT) {
      float v[16];
      tmem_ld16(lanes(tmem) + 256, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) s_e[threadIdx.x * EP + q] = v[q];
      if ((int)threadIdx.x < m.np)                    // e^1 for pass A^T
#pragma unroll
        for (int q = 0; q < 16; ++q) b.Ek[1][sidx(tile, C, q, threadIdx.x)] = v[q];
    }
    __syncthreads();
    seg_store(b.gam[1], m, CL, [&](int p, int x) { return s_e[p * EP + x / NLM] * s_Y[p * NLM + x % NLM]; });
    __syncthreads();
  }
  if (threadIdx.x == 0) bulk_wait_all();
  BF_EPILOGUE
}

// ============================================================================
// Pass B1_k: tensor product of layer k and channel mixing -> V^k, scalars S^k.
// 512 threads: thread (r, h) owns tile row r and channels 4h..4h+3.
template <class Tin, int LM>
__global__ void __launch_bounds__(kThr4, 1) k_bf_b1(BfW w, PassBufs b, int k) {
  using Cf = Tc<LM>;
  constexpr int NLM = Cf::NLM, NS = Cf::NS, CL = Cf::CL, NW0 = Cf::NW0, NL = LM + 1;
  BF_PROLOGUE(Cf::kImgEmb + NL * kImgMix, {
    bulk_g2s(sm, w.emb, Cf::kImgEmb, &bars[1]);
    for (int l = 0; l < NL; ++l) bulk_g2s(sm + Cf::kImgEmb + l * kImgMix, w.mix[k - 1][l], kImgMix, &bars[1]);
  })
  uint8_t* Wemb = sm;
  uint8_t* Wmix = Wemb + Cf::kImgEmb;
  uint8_t* X = Wmix + NL * kImgMix;
  uint8_t* T = X + kOp128;
  float* s_Yb = reinterpret_cast<float*>(T + Cf::kOpT);   // [2][kT][NLM] harmonics (k = 1), one tile ahead
  float* s_g = s_Yb + 2 * kT * NLM;       // [kSegCap][CL]
  const int r = threadIdx.x & (kT - 1), h = threadIdx.x >> 7;
  auto y_fill = [&](int t, float* g) {               // quarter 0: harmonics of row r of tile t (0 past the list)
    float u[3], d, fc, dfc, Y[NLM];
#pragma unroll
    for (int q = 0; q < NLM; ++q) Y[q] = 0.0f;
    if (r < min(kT, P - t * kT)) geometry<LM>(b, t, r, w.rc, u, d, fc, dfc, Y);
#pragma unroll
    for (int q = 0; q < NLM; ++q) g[r * NLM + q] = Y[q];
  };
  if (k == 1 && h == 0) y_fill(blockIdx.x, s_Yb);
  int gb = 0;
  uint32_t xw[16];                                    // x^0 operand words (k = 1), one tile ahead
  ld_row<32>(xw, b.X[0], blockIdx.x, r, D, 32 * h, k == 1 && r < min(kT, P - (int)blockIdx.x * kT));
  MetaPre mq = meta_load(b, blockIdx.x, P);
  for (int tile = blockIdx.x; tile < ntiles && !err; tile += gridDim.x) {
    meta_setup(b, tile, P, m, mq);
    if (threadIdx.x == 0 && tile + (int)gridDim.x < ntiles) {
      const int nt = tile + (int)gridDim.x;
      prefetch_meta(b, nt);
      prefetch_rows(b.dR, 3, nt);
      if (k == 1) prefetch_rows_h(b.X[0], D, nt);
      else prefetch_rows_h(b.V[k - 1], CL, nt);
    }
    const bool valid = r < m.np;
    const float* s_Y = s_Yb + gb * kT * NLM;          // (the harmonics serve the embedding only)
    if (threadIdx.x == 0) bulk_wait_read();           // the previous tile's V^k copy has read T
    if (k == 1) {
      st_row<Tin, 32>(X, r, 32 * h, xw);
      stage_g<CL>(b.gsum[k], m, s_g);
      mm.start([&] { mma_k<Tin>(tmem + 0, X, 0, Wemb, NW0, 8, false, 0); });
      if (h == 0) y_fill(tile + (int)gridDim.x, s_Yb + (gb ^ 1) * kT * NLM);   // the next tile's, under the MMA
      gb ^= 1;
      mm.wait();
    } else {
      stage_g<CL>(b.gsum[k], m, s_g);
      __syncthreads();
    }
    float w0[16];                                     // w0 of channels 4h..4h+3: w0[cc NL + l]
    if (k == 1) tmem_ld16(lanes(tmem) + 4 * NL * h, w0);
    // channel pairs: for l3 >= 1 the P_l paths of channels c, c + 1 fill
    // 2 P_l consecutive columns of a mixing K-slice (one 16-byte chunk at
    // P_l = 4, 8 bytes at P_l = 2); the l3 = 0 slice is written per element
#pragma unroll
    for (int cc = 0; cc < 4; cc += 2) {
      float Tv[2][Cf::NT];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = 4 * h + cc + e;
        float V[NLM], G[NLM];
        if (k == 1) {
#pragma unroll
          for (int lm = 0; lm < NLM; ++lm) V[lm] = w0[(cc + e) * NL + l_of(lm)] * s_Y[r * NLM + lm];
        } else {
#pragma unroll
          for (int lm = 0; lm < NLM; ++lm) {
            const float2 t = valid ? ldh2(b.V[k - 1], hidx(tile, CL, lm * C + (c & ~1), r)) : make_float2(0.f, 0.f);
            V[lm] = (c & 1) ? t.y : t.x;
          }
        }
        get_g<NLM>(s_g, b.gsum[k], m, r, valid, c, G);
        Cf::fwd(V, G, Tv[e]);
#pragma unroll
        for (int q = 0; q < NS; ++q) st1<Tin>(T, r, c * NS + q, Tv[e][q]);
      }
      if (valid) {                                    // S of channels c0, c0 + 1: features NS c0 .. NS c0 + 2 NS - 1
        const int f0 = (4 * h + cc) * NS;
        float s2[2 * NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          s2[q] = Tv[0][q];
          s2[NS + q] = Tv[1][q];
        }
#pragma unroll
        for (int q = 0; q < 2 * NS; q += 2) sth2(b.S[k], hidx(tile, C * NS, f0 + q, r), s2[q], s2[q + 1]);
      }
      const int c0 = 4 * h + cc;
#pragma unroll
      for (int j = 1; j < NLM; ++j) {
        const int l3 = l_of(j), mm3 = j - l3 * l3, nm = 2 * l3 + 1, pl = Cf::P(l3);
        float v8[8];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < pl) v8[pl * e + q] = Tv[e][Cf::toff(l3) + q * nm + mm3];
        if (pl == 4) st8<Tin>(T, sw128_off(r, Cf::slice(j) + c0 * 4, 128), v8);
        else st4<Tin>(T, sw128_off(r, Cf::slice(j) + c0 * pl, 128), v8);
      }
    }
    mm.start([&] {
      // K-step-major over the NLM products: consecutive MMAs write different
      // accumulators, so none waits for the one before it (unrolled: the
      // K-slice offsets are compile-time constants on the issuing thread)
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int j = 0; j < NLM; ++j) {
          const int l3 = l_of(j);
          if (kk < C * Cf::P(l3) / 16)
            mma_k<Tin>(tmem + 64 + 16 * j, T, Cf::slice(j) / 16 + kk, Wmix + l3 * kImgMix + 32 * kk, 16, 1, false, 0,
                       kk > 0);
        }
    });
    {                                                 // next tile's loads, issued under the mixing MMAs
      const int nt = tile + (int)gridDim.x;
      ld_row<32>(xw, b.X[0], nt, r, D, 32 * h, k == 1 && r < min(kT, P - nt * kT));
      mq = meta_load(b, nt, P);
    }
    mm.wait();
    {
      // V^k leaves by one bulk copy of its tile-SoA words, staged in T (the
      // mixing MMAs have read it)
      uint32_t* s_vs = reinterpret_cast<uint32_t*>(T);
      const uint32_t base = lanes(tmem);
      for (int j = h; j < NLM; j += 4) {              // components h, h + 4, h + 8
        float v[16];
        tmem_ld16(base + 64 + 16 * j, v);
#pragma unroll
        for (int co = 0; co < C; co += 2) s_vs[((j * C + co) >> 1) * kT + r] = h2word(v[co], v[co + 1]);
      }
      fence_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) {
        bulk_s2g(b.V[k] + (size_t)tile * (CL / 2) * kT, s_vs, (uint32_t)(CL / 2 * kT * 4));
        bulk_commit();
      }
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
  BF_EPILOGUE
}

// ============================================================================
// Pass B2_k: latent MLP of layer k (x^k) and env of layer k+1 -> Gamma^{k+1}.
// 512 threads: column quarters for every epilogue.
template <class Tin, int LM>
__global__ void __launch_bounds__(kThr4, 1) k_bf_b2(BfW w, PassBufs b, int k) {
  constexpr int NLM = Tc<LM>::NLM, NS = Tc<LM>::NS, CL = Tc<LM>::CL, KH = Tc<LM>::KH;
  BF_PROLOGUE(kImgLat0 + kImgLat1 + kImgEnv, {
    bulk_g2s(sm, w.lat0[k - 1], kImgLat0, &bars[1]);
    bulk_g2s(sm + kImgLat0, w.lat1[k - 1], kImgLat1, &bars[1]);
    bulk_g2s(sm + kImgLat0 + kImgLat1, w.env[k], kImgEnv, &bars[1]);
  })
  uint8_t* Wl0 = sm;
  uint8_t* Wl1 = Wl0 + kImgLat0;
  uint8_t* Wenv = Wl1 + kImgLat1;
  uint8_t* HA = Wenv + kImgEnv;
  uint8_t* A1 = HA + kOpH;
  float* s_fc = reinterpret_cast<float*>(A1 + kOp128);
  float* s_Y = s_fc + kT;
  float* s_e = s_Y + kT * NLM;
  uint32_t* s_xs = reinterpret_cast<uint32_t*>(A1);   // [D/2][kT] x^k words, from the x^k epilogue to the env MMA
  const int r = threadIdx.x & (kT - 1), h = threadIdx.x >> 7;
  // [x^{k-1}, S^k] operand words, one tile ahead: quarter h holds x^{k-1}
  // columns 32h..32h+31 and, for 1 <= h <= NS, S^k columns 16(h-1)..
  uint32_t xw[16], sw[8];
  const bool has_s = h >= 1 && h <= NS;
  {
    const bool vt = r < min(kT, P - (int)blockIdx.x * kT);
    ld_row<32>(xw, b.X[k - 1], blockIdx.x, r, D, 32 * h, vt);
    ld_row<16>(sw, b.S[k], blockIdx.x, r, C * NS, 16 * max(h - 1, 0), vt && has_s);
  }
  // envelope and harmonics of tile row r (threads r < 128), one tile ahead:
  // the next tile's are formed while the current tile's z2 MMA runs
  float fcn, Yn[NLM];
  auto geo_row = [&](int t) {
    fcn = 0.0f;
#pragma unroll
    for (int q = 0; q < NLM; ++q) Yn[q] = 0.0f;
    if (threadIdx.x < kT && r < min(kT, P - t * kT)) {
      float u[3], d, dfc;
      geometry<LM>(b, t, r, w.rc, u, d, fcn, dfc, Yn);
    }
  };
  geo_row(blockIdx.x);
  MetaPre mq = meta_load(b, blockIdx.x, P);
  for (int tile = blockIdx.x; tile < ntiles && !err; tile += gridDim.x) {
    meta_setup(b, tile, P, m, mq);
    if (threadIdx.x == 0 && tile + (int)gridDim.x < ntiles) {
      const int nt = tile + (int)gridDim.x;
      prefetch_meta(b, nt);
      prefetch_rows(b.dR, 3, nt);
      prefetch_rows_h(b.X[k - 1], D, nt);
      prefetch_rows_h(b.S[k], C * NS, nt);
    }
    const bool valid = r < m.np;
    const float* xg = b.X[k - 1];
    if (threadIdx.x < kT) {
      s_fc[r] = fcn;
#pragma unroll
      for (int q = 0; q < NLM; ++q) s_Y[r * NLM + q] = Yn[q];
    }
    st_row<Tin, 32>(HA, r, 32 * h, xw);
    if (has_s) {
      st_row<Tin, 16>(HA, r, 128 + 16 * (h - 1), sw);
    } else if (h == 0) {
      float z[16] = {};
      st16<Tin>(HA, r, KH, z);
    }
    if (threadIdx.x == 0) bulk_wait_read();           // the previous tile's x^k copy has read A1
    mm.run([&] { mma_k<Tin>(tmem + 0, HA, 0, Wl0, 128, KH / 16, false, 0); });
    epi(tmem, 0, 128, [&](int rr, int n0, const float* v) {
      float o[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = silu_b(v[q]);
      st16<Tin>(A1, rr, n0, o);
    });
    mm.start([&] { mma_k<Tin>(tmem + 128, A1, 0, Wl1, 128, 8, false, 0); });
    geo_row(tile + (int)gridDim.x);                   // registers only (zeros past the last tile)
    mm.wait();
    epi(tmem, 128, 128, [&](int rr, int n0, const float* v) {
      float o[16], xs[16];
      const float fc = s_fc[rr];
      // FP16 operands: the operand tile holds the stored x^{k-1} itself
      if constexpr (Op<Tin>::fmt == 0) ld16_h(HA, rr, n0, xs);
#pragma unroll
      for (int q = 0; q < 16; q += 2) {
        float2 x;
        if constexpr (Op<Tin>::fmt == 0) x = make_float2(xs[q], xs[q + 1]);
        else x = valid ? ldh2(xg, hidx(tile, D, n0 + q, rr)) : make_float2(0.f, 0.f);
        o[q] = r16((x.x + fc * silu_b(v[q])) * kR2);
        o[q + 1] = r16((x.y + fc * silu_b(v[q + 1])) * kR2);
      }
      st16<Tin>(HA, rr, n0, o);
#pragma unroll
      for (int q = 0; q < 16; q += 2) s_xs[((n0 + q) >> 1) * kT + rr] = h2word(o[q], o[q + 1]);
    });
    // env MMA; the x^k tile (tile-SoA words, staged in A1, dead since z2)
    // leaves by one bulk copy issued with it
    mm.start([&] {
      mma_k<Tin>(tmem + 256, HA, 0, Wenv, 16, 8, false, 0);
      bulk_s2g(b.X[k] + (size_t)tile * (D / 2) * kT, s_xs, (uint32_t)(D / 2 * kT * 4));
      bulk_commit();
    });
    {                                                 // next tile's loads, issued under the env MMA
      const int nt = tile + (int)gridDim.x;
      const bool vt = r < min(kT, P - nt * kT);
      ld_row<32>(xw, b.X[k - 1], nt, r, D, 32 * h, vt);
      ld_row<16>(sw, b.S[k], nt, r, C * NS, 16 * max(h - 1, 0), vt && has_s);
      mq = meta_load(b, nt, P);
    }
    mm.wait();
    if (threadIdx.x < kT) {
      float v[16];
      tmem_ld16(lanes(tmem) + 256, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) s_e[r * EP + q] = v[q];
      if (valid)                                      // e^{k+1} for pass B^T of layer k
#pragma unroll
        for (int q = 0; q < 16; ++q) b.Ek[k + 1][sidx(tile, C, q, r)] = v[q];
    }
    __syncthreads();
    seg_store(b.gam[k + 1], m, CL, [&](int p, int x) { return s_e[p * EP + x / NLM] * s_Y[p * NLM + x % NLM]; });
    __syncthreads();
  }
  if (threadIdx.x == 0) bulk_wait_all();
  BF_EPILOGUE
}

// V^{L-1} words of channel pairs (4h, 4h+1), (4h+2, 4h+3) and the x^{L-1}
// operand words of pass C for tile t, thread (r, h) (zeros past the last tile)
template <int NLM>
AL_DEV void c_loads(const PassBufs& b, int L, int t, int P, int r, int h, __half2 (&vw)[2][NLM],
                    uint32_t (&xw)[16]) {
  constexpr int CL = C * NLM;
  const bool vt = r < min(kT, P - t * kT);
#pragma unroll
  for (int cp = 0; cp < 2; ++cp)
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm)
      vw[cp][lm] = vt ? reinterpret_cast<const __half2*>(b.V[L - 1])[hidx(t, CL, lm * C + 4 * h + 2 * cp, r)]
                      : __floats2half2_rn(0.f, 0.f);
  ld_row<32>(xw, b.X[L - 1], t, r, D, 32 * h, vt);
}

// ============================================================================
// Pass C: last layer + energy MLP forward, dE/dE_ij = sigma_Z, and their
// adjoint: dx^{L-1}, dV^{L-1}, dGamma^L partials, du, energy partials.
// 512 threads: thread (r, h) owns tile row r and column quarter h of every
// epilogue, channels 4h..4h+3 of the tensor products and energy hidden units
// 8h..8h+7.
// Split mode: the energy hidden layer takes split operands; the lo part of
// x^L goes to A1 (free after the second latent MMA) and dz_E keeps its hi and
// lo parts side by side in the 64 columns of AE.
template <class Tin, bool kSplit, int LM>
__global__ void __launch_bounds__(kThr4, 1) k_bf_c(BfW w, PassBufs b) {
  using Cf = Tc<LM>;
  constexpr int NLM = Cf::NLM, NS = Cf::NS, CL = Cf::CL, KH = Cf::KH, CLP = Cf::CLP;
  const int L = w.n_layers;
  BF_PROLOGUE(kImgLat0 + kImgLat1 + (kSplit ? 2 : 1) * kImgE0, {
    bulk_g2s(sm, w.lat0[L - 1], kImgLat0, &bars[1]);
    bulk_g2s(sm + kImgLat0, w.lat1[L - 1], kImgLat1, &bars[1]);
    bulk_g2s(sm + kImgLat0 + kImgLat1, w.e0, kImgE0, &bars[1]);
    if (kSplit) bulk_g2s(sm + kImgLat0 + kImgLat1 + kImgE0, w.e0_lo, kImgE0, &bars[1]);
  })
  uint8_t* Wl0 = sm;
  uint8_t* Wl1 = Wl0 + kImgLat0;
  uint8_t* We0 = Wl1 + kImgLat1;
  uint8_t* We0lo = We0 + kImgE0;                       // split mode only
  uint8_t* HA = We0lo + (kSplit ? kImgE0 : 0);
  uint8_t* A1 = HA + kOpH;
  uint8_t* AE = A1 + kOp128;
  float* s_dg = reinterpret_cast<float*>(HA);          // reuses HA + A1 after the last MMA
  float* s_fcb = reinterpret_cast<float*>(AE + kOp64);   // [2][kT] envelope; the next tile's filled under z2
  float* s_sig = s_fcb + 2 * kT;
  float* s_eq = s_sig + kT;                            // [4][kT] energy partials per quarter
  float* s_du = s_eq + 4 * kT;                         // [4][kT]
  float* s_g = s_du + 4 * kT;                          // [kSegCap][CL]
  const int r = threadIdx.x & (kT - 1), h = threadIdx.x >> 7;
  // quarter 0: envelope of row r of tile t (0 past the list); the pair
  // separation is loaded (fc_ld) well before it is used (fc_put)
  auto fc_ld = [&](int t, float* d3) -> bool {
    const bool v = r < min(kT, P - t * kT);
#pragma unroll
    for (int a = 0; a < 3; ++a) d3[a] = v ? b.dR[sidx(t, 3, a, r)] : 0.0f;
    return v;
  };
  auto fc_put = [&](bool v, const float* d3, float* g) {
    float u[3], d, fc = 0.0f, dfc, Y[NLM];
    if (v) geo_from_delta<LM>(d3[0], d3[1], d3[2], w.rc, u, d, fc, dfc, Y);
    g[r] = fc;
  };
  if (h == 0) {
    float d3[3];
    const bool v = fc_ld(blockIdx.x, d3);
    fc_put(v, d3, s_fcb);
  }
  int gb = 0;
  // V^{L-1} (one FP16 channel pair per word) and x^{L-1} operand words of a
  // tile, in registers; the next tile's are loaded during this tile's tail
  __half2 vw[2][NLM];
  uint32_t xw[16];
  c_loads(b, L, blockIdx.x, P, r, h, vw, xw);
  MetaPre mq = meta_load<true>(b, blockIdx.x, P);
  for (int tile = blockIdx.x; tile < ntiles && !err; tile += gridDim.x) {
    meta_setup(b, tile, P, m, mq);
    if (threadIdx.x == 0 && tile + (int)gridDim.x < ntiles) {
      const int nt = tile + (int)gridDim.x;
      prefetch_meta(b, nt);
      prefetch_rows(b.dR, 3, nt);
      prefetch_rows_h(b.V[L - 1], CL, nt);
      prefetch_rows_h(b.X[L - 1], D, nt);
    }
    const bool valid = r < m.np;
    const float* xg = b.X[L - 1];
    float nd[3];                                      // the next tile's pair separation (quarter 0)
    bool nv = false;
    if (h == 0) nv = fc_ld(tile + (int)gridDim.x, nd);
    const float* s_fc = s_fcb + gb * kT;
    if (h == 0) s_sig[r] = valid ? w.sigma[mq.zi] : 0.0f;
    stage_g<CL>(b.gsum[L], m, s_g);
    // z1 = [x^{L-1}, S] W_0: the x^{L-1} K-steps run while the tensor product
    // computes S
    st_row<Tin, 32>(HA, r, 32 * h, xw);
    if (h == 3) {
      float z[16] = {};
      st16<Tin>(HA, r, KH, z);
    }
    mm.issue([&] { mma_k<Tin>(tmem + 0, HA, 0, Wl0, 128, 8, false, 0); });
    {
      float S[4 * NS];                                 // columns D + 4 NS h .. D + 4 NS (h + 1) - 1
#pragma unroll
      for (int cp = 0; cp < 4; cp += 2) {             // channel pairs share the V words
        float V2[2][NLM];
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
          const float2 t = __half22float2(vw[cp / 2][lm]);
          V2[0][lm] = t.x;
          V2[1][lm] = t.y;
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          float G[NLM];
          get_g<NLM>(s_g, b.gsum[L], m, r, valid, 4 * h + cp + e, G);
          Cf::fwd_scalar(V2[e], G, S + (cp + e) * NS);
        }
      }
      st_cols<Tin, 4 * NS>(HA, r, D + 4 * NS * h, S);
    }
    mm.run([&] { mma_k<Tin>(tmem + 0, HA, 8, Wl0 + 2 * (128 * 128), 128, NS, false, 0, true); });
    epi_silu_keep_grad(tmem, 0, [&](int rr, int n0, const float* o) { st16<Tin>(A1, rr, n0, o); });   // z1
    mm.start([&] { mma_k<Tin>(tmem + 128, A1, 0, Wl1, 128, 8, false, 0); });
    if (h == 0) fc_put(nv, nd, s_fcb + (gb ^ 1) * kT);   // the next tile's, under the MMA
    gb ^= 1;
    mm.wait();
    epi(tmem, 128, 128, [&](int rr, int n0, const float* v) {
      float o[16], xs[16];
      const float fc = s_fc[rr];
      // FP16 operands: the operand tile holds the stored x^{L-1} itself
      if constexpr (Op<Tin>::fmt == 0) ld16_h(HA, rr, n0, xs);
#pragma unroll
      for (int q = 0; q < 16; q += 2) {
        float2 x;
        if constexpr (Op<Tin>::fmt == 0) x = make_float2(xs[q], xs[q + 1]);
        else x = valid ? ldh2(xg, hidx(tile, D, n0 + q, rr)) : make_float2(0.f, 0.f);
        o[q] = (x.x + fc * silu_b(v[q])) * kR2;
        o[q + 1] = (x.y + fc * silu_b(v[q + 1])) * kR2;
      }
      st16_op<Tin, kSplit>(HA, A1, rr, n0, o);
    });
    mm.run([&] { mma_split<Tin, kSplit>(tmem + 256, HA, A1, We0, We0lo, 32, 8, false, 0); });
    {
      float ze[8], dz[8];
      tmem_ld8(lanes(tmem) + 256 + 8 * h, ze);
      const float sig = s_sig[r];
      float e = 0.0f;
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const float wo = __ldg(w.eout + 8 * h + n);
        e = fmaf(wo, silu_b(ze[n]), e);
        dz[n] = sig * wo * dsilu_b(ze[n]);
      }
      s_eq[h * kT + r] = valid ? e : 0.0f;
      if (kSplit) {                                   // hi in columns 0..31, lo in 32..63
        st8_split<Tin>(AE, sw128_off(r, 8 * h, 128), AE, sw128_off(r, 32 + 8 * h, 128), dz);
      } else {
        st8<Tin>(AE, sw128_off(r, 8 * h, 128), dz);
      }
    }
    mm.run([&] {                                                                // dx^L
      mma_k<Tin>(tmem + 288, AE, 0, We0, 128, 2, true, 32);
      if (kSplit) {
        mma_k<Tin>(tmem + 288, AE, 2, We0, 128, 2, true, 32, true);
        mma_k<Tin>(tmem + 288, AE, 0, We0lo, 128, 2, true, 32, true);
      }
    });
    {
      float du = 0.0f;
      epi(tmem, 288, 128, [&](int rr, int n0, const float* dx) {
        float z2[16], o[16];
        tmem_ld16(lanes(tmem) + 128 + n0, z2);
        const float fc = s_fc[rr];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          du = fmaf(dx[q], silu_b(z2[q]), du);
          o[q] = dx[q] * fc * kR2 * dsilu_b(z2[q]);
        }
        st16<Tin>(A1, rr, n0, o);
      });
      s_du[h * kT + r] = du * kR2;
    }
    mm.run([&] { mma_k<Tin>(tmem + 128, A1, 0, Wl1, 128, 8, true, 128); });    // da1
    epi(tmem, 128, 128, [&](int rr, int n0, const float* da) {
      float g1[16], o[16];                             // SiLU'(z1), left in TMEM by the z1 epilogue
      tmem_ld16(lanes(tmem) + n0, g1);
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = da[q] * g1[q];
      st16<Tin>(HA, rr, n0, o);
    });
    mm.start([&] { mma_k<Tin>(tmem + 0, HA, 0, Wl0, KH, 8, true, 128); });     // [dx^{L-1}, ds]
#pragma unroll
    for (int cp = 0; cp < 2; ++cp)                    // again, for the tensor-product adjoint (under the MMA)
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm)
        vw[cp][lm] = valid ? reinterpret_cast<const __half2*>(b.V[L - 1])[hidx(tile, CL, lm * C + 4 * h + 2 * cp, r)]
                           : __floats2half2_rn(0.f, 0.f);
    mm.wait();
    epi(tmem, 0, 128, [&](int rr, int n0, const float* dh) {
      float dx[16];
      tmem_ld16(lanes(tmem) + 288 + n0, dx);
      if (valid)
#pragma unroll
        for (int q = 0; q < 16; ++q) b.dX[sidx(tile, D, n0 + q, rr)] = dh[q] + dx[q] * kR2;
    });
    {
      float ds[16];                                    // columns D + 4 NS h ..: ds of channels 4h..4h+3
      tmem_ld16(lanes(tmem) + 128 + 4 * NS * h, ds);
      float dVe[NLM];                                  // dV of the even channel of a pair
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = 4 * h + cc;
        float V[NLM], G[NLM], dV[NLM], dG[NLM];
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
          const float2 t = __half22float2(vw[cc / 2][lm]);
          V[lm] = (cc & 1) ? t.y : t.x;
          dV[lm] = 0.0f;
          dG[lm] = 0.0f;
        }
        get_g<NLM>(s_g, b.gsum[L], m, r, valid, c, G);
        Cf::bwd_scalar(V, G, ds + cc * NS, dV, dG);
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) s_dg[r * CLP + c * NLM + lm] = dG[lm];
        if (cc & 1) {
          if (valid)
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) st_opw<Tin>(b.dV, hidx(tile, CL, lm * C + c - 1, r), dVe[lm], dV[lm]);
        } else {
#pragma unroll
          for (int lm = 0; lm < NLM; ++lm) dVe[lm] = dV[lm];
        }
      }
    }
    c_loads(b, L, tile + (int)gridDim.x, P, r, h, vw, xw);
    mq = meta_load<true>(b, tile + (int)gridDim.x, P);
    __syncthreads();
    {
      // energy partials per (tile, centre atom), one warp per segment: lanes
      // stride the segment's pairs, then a shuffle tree (fixed order) in
      // FP32 (at most 128 pair energies; GB300's FP64 pipe is a small
      // fraction of its FP32 rate); the partial is stored in FP64 and the
      // per-atom and total sums over tiles stay FP64
      const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int sg = wid; sg < m.nseg; sg += (int)(blockDim.x >> 5)) {
        float acc = 0.0f;
        for (int p = m.sstart[sg] + lane; p < m.sstart[sg + 1]; p += 32)
          acc += (s_eq[p] + s_eq[kT + p]) + (s_eq[2 * kT + p] + s_eq[3 * kT + p]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) b.epart[m.tile + m.atom[sg]] = (double)acc;
      }
    }
    if (threadIdx.x < kT && valid) {
      b.dU[sidx(tile, 1, 0, r)] = (s_du[r] + s_du[kT + r]) + (s_du[2 * kT + r] + s_du[3 * kT + r]);
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) b.dY[sidx(tile, NLM, lm, r)] = 0.0f;
    }
    seg_store(b.dgam[L], m, CL, [&](int p, int x) { return s_dg[p * CLP + x]; });
    __syncthreads();
  }
  BF_EPILOGUE
}

// ============================================================================
// Pass B_k^T: adjoint of layer k.  First the Gamma^{k+1} scatter (with the
// env output e^{k+1} stored by pass B2) and the latent MLP (forward
// recomputed), then mixing and the tensor product, and
// for k = 1 the embedding; no per-atom sum lies between the two halves, so
// they share one kernel.  dS^k stays in TMEM and dx^{k-1} is
// accumulated in one set of TMEM columns (residual dx / sqrt 2, then
// dz1 W_0, then emb^T dw0) and written once.
// Shared memory: HA holds [x^{k-1}, S^k], dz1, the dV^k operand, then dw0,
// the dy partials and (with A1) the dx^{k-1} staging; A1 holds de, SiLU(z1),
// dz2 and during the mixing-adjoint rounds the dGamma^k staging of 8 channels.
// e^{k+1} is read from memory (stored by pass B2).
// TMEM columns: z1 [32, 160); z2 and da1 [160, 288); dx [288,
// 416); ds [416, 416 + C NS); w0 [464, 464 + NW0); in the rounds, the l3 = 0
// component of all channels [416, 416 + C NS) and components j >= 1 from
// column 32 (j - 1): at l_max 2 eight channels per round (32 columns each,
// [0, 256)); below l_max 2 all channels in the first round (C P_l <= 32
// columns each), which the second round reads again.
// 512 threads: thread (r, h) owns tile row r, column quarter h of every
// epilogue, channels 4h..4h+3 of the env adjoint and channels 8 hf + 2h + e
// of mixing-adjoint round hf.
template <int LM>
constexpr uint32_t reg_a1() {                        // A1 region: an operand tile or the round's dGamma staging
  return std::max<uint32_t>(kOp128, (4 * kT * (Tc<LM>::CL / 2 + 1) + 1023) / 1024 * 1024);
}
// 2, 4 or 6 consecutive TMEM columns (no column past the N-th is read)
template <int N>
AL_DEV void tmem_ldn(uint32_t taddr, float* v) {
  static_assert(N == 2 || N == 4 || N == 6, "2, 4 or 6 columns");
  if constexpr (N == 6) {
    tmem_ld6(taddr, v);
  } else {
    uint32_t t[4] = {0u, 0u, 0u, 0u};
    if constexpr (N == 4) tmem_ld4_raw(taddr, t);
    else tmem_ld2_raw(taddr, t);
    tmem_wait4(t);
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = __uint_as_float(t[q]);
  }
}
template <class Tin, bool kEmb, int LM>
__global__ void __launch_bounds__(kThr4, 1) k_bf_bt(BfW w, PassBufs b, int k) {
  using Cf = Tc<LM>;
  constexpr int NLM = Cf::NLM, NS = Cf::NS, CL = Cf::CL, KH = Cf::KH, NW0 = Cf::NW0, NL = LM + 1;
  constexpr int CLH = CL / 2 + 1;                    // odd stride of the half-round dGamma staging
  constexpr uint32_t kRegA1 = reg_a1<LM>();
  BF_PROLOGUE(kImgEnv + kImgLat0 + kImgLat1 + Cf::kImgEmb + NL * kImgMix, {
    bulk_g2s(sm, w.env[k], kImgEnv, &bars[1]);
    bulk_g2s(sm + kImgEnv, w.lat0[k - 1], kImgLat0, &bars[1]);
    bulk_g2s(sm + kImgEnv + kImgLat0, w.lat1[k - 1], kImgLat1, &bars[1]);
    bulk_g2s(sm + kImgEnv + kImgLat0 + kImgLat1, w.emb, Cf::kImgEmb, &bars[1]);
    for (int l = 0; l < NL; ++l)
      bulk_g2s(sm + kImgEnv + kImgLat0 + kImgLat1 + Cf::kImgEmb + l * kImgMix, w.mix[k - 1][l], kImgMix, &bars[1]);
  })
  uint8_t* Wenv = sm;
  uint8_t* Wl0 = Wenv + kImgEnv;
  uint8_t* Wl1 = Wl0 + kImgLat0;
  uint8_t* Wemb = Wl1 + kImgLat1;
  uint8_t* Wmix = Wemb + Cf::kImgEmb;
  uint8_t* HA = Wmix + NL * kImgMix;
  uint8_t* A1 = HA + kOpH;
  uint8_t* DE = A1;
  uint8_t* DVT = HA;
  uint8_t* DW0 = HA;
  float* s_dg = reinterpret_cast<float*>(A1);          // [kT][CLH], rounds only
  float* s_dy = reinterpret_cast<float*>(HA + kOp64);  // [4][kT][NLM], tile end only
  float* s_dxs = reinterpret_cast<float*>(HA);         // [D][kT] dx^{k-1} staging, tile end only
  // two geometry buffers [fc | Y] (the next tile's is filled under the
  // current tile's first MMA)
  float* s_geo = reinterpret_cast<float*>(A1 + kRegA1);
  constexpr int kGeo = kT + kT * NLM;
  float* s_du = s_geo + 2 * kGeo;                      // [4][kT]
  float* s_g = s_du + 4 * kT;                          // [kSegCap][CL]
  constexpr int kZ1 = 32, kZ2 = 160, kDX = 288, kDS = 416, kW0 = 464, kJ0 = 416, kJ = 0;
  const int r = threadIdx.x & (kT - 1), h = threadIdx.x >> 7;
  // envelope and harmonics of row r of tile t into buffer g (quarter 0; zeros
  // past the list); the pair separation is loaded (geo_ld) well before it is
  // used (geo_put)
  auto geo_ld = [&](int t, float* d3) -> bool {
    const bool v = r < min(kT, P - t * kT);
#pragma unroll
    for (int a = 0; a < 3; ++a) d3[a] = v ? b.dR[sidx(t, 3, a, r)] : 0.0f;
    return v;
  };
  auto geo_put = [&](bool v, const float* d3, float* g) {
    float u[3], d, fc = 0.0f, dfc, Y[NLM];
#pragma unroll
    for (int q = 0; q < NLM; ++q) Y[q] = 0.0f;
    if (v) geo_from_delta<LM>(d3[0], d3[1], d3[2], w.rc, u, d, fc, dfc, Y);
    g[r] = fc;
#pragma unroll
    for (int q = 0; q < NLM; ++q) g[kT + r * NLM + q] = Y[q];
  };
  if (h == 0) {
    float d3[3];
    const bool v = geo_ld(blockIdx.x, d3);
    geo_put(v, d3, s_geo);
  }
  int gb = 0;                                         // this tile's geometry buffer
  // the next tile's dV^k words (channels 4h..4h+3) and neighbour-list rows,
  // loaded during this tile's tail
  uint32_t dvw[NLM][2];
  auto ld_next = [&](int t) {
    const bool vt = r < min(kT, P - t * kT);
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm)
#pragma unroll
      for (int q = 0; q < 2; ++q)
        dvw[lm][q] = vt ? reinterpret_cast<const uint32_t*>(b.dV)[hidx(t, CL, lm * C + 4 * h + 2 * q, r)] : 0u;
  };
  ld_next(blockIdx.x);
  MetaPre mq = meta_load(b, blockIdx.x, P);
  for (int tile = blockIdx.x; tile < ntiles && !err; tile += gridDim.x) {
    meta_setup(b, tile, P, m, mq);
    if (threadIdx.x == 0 && tile + (int)gridDim.x < ntiles) {
      const int nt = tile + (int)gridDim.x;
      prefetch_meta(b, nt);
      prefetch_rows(b.dR, 3, nt);
      prefetch_rows(b.Ek[k + 1], C, nt);
      prefetch_rows_h(b.X[k - 1], D, nt);
      prefetch_rows_h(b.S[k], C * NS, nt);
      prefetch_rows_h(b.dV, CL, nt);
      prefetch_rows(b.dX, D, nt);
      prefetch_rows(b.dU, 1, nt);
      prefetch_rows(b.dY, NLM, nt);
      if (!kEmb) prefetch_rows_h(b.V[k - 1], CL, nt);
    }
    const bool valid = r < m.np;
    float nd[3];                                      // the next tile's pair separation (quarter 0)
    bool nv = false;
    if (h == 0) nv = geo_ld(tile + (int)gridDim.x, nd);
    const float* s_fc = s_geo + gb * kGeo;
    const float* s_Y = s_fc + kT;
    float ew[4];                                      // e^{k+1} of channels 4h..4h+3 (stored by pass B2)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) ew[cc] = valid ? b.Ek[k + 1][sidx(tile, C, 4 * h + cc, r)] : 0.0f;
    stage_g<CL>(b.dgsum[k + 1], m, s_g);
    if (threadIdx.x == 0) bulk_wait_read();           // the previous tile's dx^{k-1} copy has read HA
    uint32_t xw2[16], sw[8];                          // [x^{k-1}, S^k] operand, in flight during the env adjoint
    const bool has_s = h >= 1 && h <= NS;             // quarters 1..NS hold S^k columns 16 (h - 1)..
    ld_row<32>(xw2, b.X[k - 1], tile, r, D, 32 * h, valid);
    ld_row<16>(sw, b.S[k], tile, r, C * NS, 16 * max(h - 1, 0), valid && has_s);
    __syncthreads();                                  // geometry rows and staged dGamma rows
    float dy[NLM];                                    // dY of this thread's channels (env and embedding)
    {
      const float* e = ew;                            // e^{k+1} of channels 4h..4h+3
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) dy[lm] = 0.0f;
      float de[4];                                    // de of channels 4h..4h+3: one 8-byte store
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = 4 * h + cc;
        float dG[NLM];
        get_g<NLM>(s_g, b.dgsum[k + 1], m, r, valid, c, dG);
        float acc = 0.0f;
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
          acc = fmaf(dG[lm], s_Y[r * NLM + lm], acc);
          dy[lm] = fmaf(dG[lm], e[cc], dy[lm]);
        }
        de[cc] = acc;
      }
      st_cols<Tin, 4>(DE, r, 4 * h, de);
    }
    st_row<Tin, 32>(HA, r, 32 * h, xw2);
    if (has_s) {
      st_row<Tin, 16>(HA, r, 128 + 16 * (h - 1), sw);
    } else if (h == 0) {
      float z[16] = {};
      st16<Tin>(HA, r, KH, z);
    }
    mm.start([&] {
      mma_k<Tin>(tmem + kDX, DE, 0, Wenv, 128, 1, true, 16);                    // env^T de
      mma_k<Tin>(tmem + kZ1, HA, 0, Wl0, 128, KH / 16, false, 0);               // z1
      if (kEmb) mma_k<Tin>(tmem + kW0, HA, 0, Wemb, NW0, 8, false, 0);          // w0 = emb x^0
    });
    float dxo[32];                                    // dx^k from the layer above, columns 32h..32h+31
#pragma unroll
    for (int q = 0; q < 32; ++q) dxo[q] = valid ? b.dX[sidx(tile, D, 32 * h + q, r)] : 0.0f;
    if (h == 0) geo_put(nv, nd, s_geo + (gb ^ 1) * kGeo);   // the next tile's, under the MMAs
    gb ^= 1;
    mm.wait();
    epi_silu_keep_grad(tmem, kZ1, [&](int rr, int n0, const float* o) { st16<Tin>(A1, rr, n0, o); });   // z1
    mm.start([&] { mma_k<Tin>(tmem + kZ2, A1, 0, Wl1, 128, 8, false, 0); });   // z2
    {
      // dx = dx^k + env^T de; its residual part dx / sqrt 2 goes back into
      // the same TMEM columns, where the later MMAs accumulate onto it.  The
      // env^T de columns, the ds columns and dx^k are not the z2 MMA's, so
      // they are read, zeroed and added while it runs.
      float du = 0.0f;
      float dx[32];
      tmem_ld32(lanes(tmem) + kDX + 32 * h, dx);
#pragma unroll
      for (int q = 0; q < 32; ++q) dx[q] += dxo[q];
      const float z[4] = {0.f, 0.f, 0.f, 0.f};       // ds columns start from zero (exactly its C NS)
#pragma unroll
      for (int q = 0; q < 4 * NS; q += 4) tmem_st4(lanes(tmem) + kDS + 4 * NS * h + q, z);
      const float fc = s_fc[r];
      mm.wait();
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        float z2[16], o[16];
        tmem_ld16(lanes(tmem) + kZ2 + 32 * h + 16 * hf, z2);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float x = dx[16 * hf + q];
          du = fmaf(x, silu_b(z2[q]), du);
          o[q] = x * fc * kR2 * dsilu_b(z2[q]);
          dx[16 * hf + q] = x * kR2;
        }
        st16<Tin>(A1, r, 32 * h + 16 * hf, o);
      }
      tmem_st32(lanes(tmem) + kDX + 32 * h, dx);
      tmem_wait_st();
      s_du[h * kT + r] = du * kR2;
    }
    mm.run([&] { mma_k<Tin>(tmem + kZ2, A1, 0, Wl1, 128, 8, true, 128); });    // da1
    epi(tmem, kZ2, 128, [&](int rr, int n0, const float* da) {
      float g1[16], o[16];                             // SiLU'(z1), left in TMEM by the z1 epilogue
      tmem_ld16(lanes(tmem) + kZ1 + n0, g1);
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = da[q] * g1[q];
      st16<Tin>(HA, rr, n0, o);
    });
    mm.start([&] { mma_k<Tin>(tmem + kDX, HA, 0, Wl0, KH, 8, true, 128, true); });   // [dx, ds] += dz1 W
    // ---- mixing and tensor-product adjoint of layer k ----
    // ds and w0 of this thread's round channels (8 hf + 2h + e): NS and
    // LM + 1 columns each; w0 (columns past dx and ds) and the Gamma^k rows
    // are read while the MMA runs
    float dsv[2][2 * NS], w0[2][2 * NL];
    if (kEmb)
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) tmem_ldn<2 * NL>(lanes(tmem) + kW0 + NL * (8 * hf + 2 * h), w0[hf]);
    stage_g<CL>(b.gsum[k], m, s_g);
    mm.wait();
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) tmem_ldn<2 * NS>(lanes(tmem) + kDS + NS * (8 * hf + 2 * h), dsv[hf]);
    // column 16 lm + c of the operand: this thread's 4 channels of one lm
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm)
      *reinterpret_cast<uint2*>(DVT + sw128_off(r, 16 * lm + 4 * h, 128)) = make_uint2(dvw[lm][0], dvw[lm][1]);
    float dw[2][2 * NL];
#pragma unroll
    for (int q = 0; q < 2 * NL; ++q) dw[0][q] = dw[1][q] = 0.0f;
    float dVe[NLM];                                   // k >= 2: dV^{k-1} of the even channel of a pair
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      if (hf == 0 || LM == 2) {
        mm.run([&] {
          if (hf == 0) mma_k<Tin>(tmem + kJ0, DVT, 0, Wmix, C * NS, 1, true, 16);
#pragma unroll
          for (int j = 1; j < NLM; ++j) {
            const int l3 = l_of(j);
            if (LM == 2)                              // this round's eight channels
              mma_k<Tin>(tmem + kJ + 32 * (j - 1), DVT, j, Wmix + l3 * kImgMix + 64 * hf, C * Cf::P(l3) / 2, 1, true,
                         16);
            else
              mma_k<Tin>(tmem + kJ + 32 * (j - 1), DVT, j, Wmix + l3 * kImgMix, C * Cf::P(l3), 1, true, 16);
          }
        });
      } else {
        __syncthreads();                              // the first round's staging has been stored
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = 8 * hf + 2 * h + e;
        const int cr = LM == 2 ? 2 * h + e : c;       // channel within a component's TMEM block
        uint32_t t[4 * NLM];
        tmem_ld4_raw(lanes(tmem) + kJ0 + NS * c, t);                        // l3 = 0: columns NS c + q
#pragma unroll
        for (int j = 1; j < NLM; ++j)
          tmem_ld4_raw(lanes(tmem) + kJ + 32 * (j - 1) + Cf::P(l_of(j)) * cr, t + 4 * j);
#pragma unroll
        for (int g = 0; g < NLM; ++g) tmem_wait4(t + 4 * g);
        float dT[Cf::NT];
#pragma unroll
        for (int q = 0; q < NS; ++q) dT[q] = __uint_as_float(t[q]) + dsv[hf][NS * e + q];
#pragma unroll
        for (int j = 1; j < NLM; ++j) {
          const int l3 = l_of(j), mm3 = j - l3 * l3, nm = 2 * l3 + 1;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < Cf::P(l3)) dT[Cf::toff(l3) + q * nm + mm3] = __uint_as_float(t[4 * j + q]);
        }
        float V[NLM], G[NLM], dG[NLM], dVp[NLM];
        if (kEmb) {
#pragma unroll
          for (int lm = 0; lm < NLM; ++lm) V[lm] = w0[hf][NL * e + l_of(lm)] * s_Y[r * NLM + lm];
        } else {
#pragma unroll
          for (int lm = 0; lm < NLM; ++lm) {
            const float2 v2 = valid ? ldh2(b.V[k - 1], hidx(tile, CL, lm * C + (c & ~1), r)) : make_float2(0.f, 0.f);
            V[lm] = e ? v2.y : v2.x;
          }
        }
        get_g<NLM>(s_g, b.gsum[k], m, r, valid, c, G);
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) dG[lm] = dVp[lm] = 0.0f;
        Cf::bwd(V, G, dT, dVp, dG);
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) s_dg[r * CLH + (c - 8 * hf) * NLM + lm] = dG[lm];
        if (!kEmb) {                                  // dV^{k-1}: channel pairs (8 hf + 2h, + 1)
          if (e == 0) {
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) dVe[lm] = dVp[lm];
          } else if (valid) {
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) st_opw<Tin>(b.dV, hidx(tile, CL, lm * C + c - 1, r), dVe[lm], dVp[lm]);
          }
        } else {
#pragma unroll
          for (int lm = 0; lm < NLM; ++lm) {
            dw[hf][NL * e + l_of(lm)] = fmaf(dVp[lm], s_Y[r * NLM + lm], dw[hf][NL * e + l_of(lm)]);
            dy[lm] = fmaf(w0[hf][NL * e + l_of(lm)], dVp[lm], dy[lm]);
          }
        }
      }
      __syncthreads();
      seg_store_cols(b.dgam[k], m, CL, (CL / 2) * hf, CL / 2, [&](int p, int x) { return s_dg[p * CLH + x]; });
    }
    if (kEmb) {                                       // the DVT operand is dead: dw0 takes its place
#pragma unroll
      for (int hf = 0; hf < 2; ++hf)
#pragma unroll
        for (int q = 0; q < 2 * NL; ++q) st1<Tin>(DW0, r, NL * (8 * hf + 2 * h) + q, dw[hf][q]);
      mm.run([&] { mma_k<Tin>(tmem + kDX, DW0, 0, Wemb, 128, NL, true, NW0, true); });   // dx += emb^T dw0
    } else {
      __syncthreads();
    }
    float duo = 0.0f, dyo[NLM];
    if (threadIdx.x < kT) {
      duo = valid ? b.dU[sidx(tile, 1, 0, r)] : 0.0f;
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) dyo[lm] = valid ? b.dY[sidx(tile, NLM, lm, r)] : 0.0f;
    }
    float dxv[32];                                    // dx^{k-1}, columns 32h..32h+31
    tmem_ld32(lanes(tmem) + kDX + 32 * h, dxv);
    ld_next(tile + (int)gridDim.x);                   // zeros past the last tile
    mq = meta_load(b, tile + (int)gridDim.x, P);
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) s_dy[(h * kT + r) * NLM + lm] = dy[lm];
    __syncthreads();
    if (threadIdx.x < kT && valid) {
      b.dU[sidx(tile, 1, 0, r)] = duo + ((s_du[r] + s_du[kT + r]) + (s_du[2 * kT + r] + s_du[3 * kT + r]));
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm)
        b.dY[sidx(tile, NLM, lm, r)] = dyo[lm] + ((s_dy[r * NLM + lm] + s_dy[(kT + r) * NLM + lm]) +
                                                  (s_dy[(2 * kT + r) * NLM + lm] + s_dy[(3 * kT + r) * NLM + lm]));
    }
    __syncthreads();
    // dx^{k-1} leaves by one bulk copy of the tile's contiguous tile-SoA block
    // (feature-major, 128 rows per feature), staged over HA and the start of
    // A1 (both dead here); rows past the list carry values nothing reads.
    // Thread 0 waits for the copy's reads before the next tile writes there.
#pragma unroll
    for (int q = 0; q < 32; ++q) s_dxs[(32 * h + q) * kT + r] = dxv[q];
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      bulk_s2g(b.dX + (size_t)tile * D * kT, s_dxs, (uint32_t)(D * kT * 4));
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
  BF_EPILOGUE
}

// ============================================================================
// Pass A^T: adjoint of the Gamma^1 scatter (with the env output e^1 stored by
// pass A), of the two-body MLP (recomputed) and of the geometry; writes
// g_ij = dE/dDelta_ij.
// DE shares H0's buffer (H0 is dead after the first MMA).  Split mode: both
// two-body GEMMs and their adjoints take split operands; A1lo holds the lo
// part of silu(z1), then of dz2, then of dz1.  The dh0 adjoint reads the
// packed image [W_hi | W_hi | W_lo] (48 columns): dh0 = block 0 + block 2.
// 512 threads: column quarters for every epilogue; the env adjoint's
// channels are spread over the quarters.
template <class Tin, bool kSplit, int LM>
__global__ void __launch_bounds__(kThr4, 1) k_bf_at(BfW w, PassBufs b) {
  constexpr int NLM = Tc<LM>::NLM, CL = Tc<LM>::CL;
  BF_PROLOGUE(kImgTb0 + (kSplit ? 2 : 1) * kImgTb1 + kImgEnv, {
    bulk_g2s(sm, w.tb0, kImgTb0, &bars[1]);
    bulk_g2s(sm + kImgTb0, w.tb1, kImgTb1, &bars[1]);
    bulk_g2s(sm + kImgTb0 + kImgTb1, w.env[0], kImgEnv, &bars[1]);
    if (kSplit) bulk_g2s(sm + kImgTb0 + kImgTb1 + kImgEnv, w.tb1_lo, kImgTb1, &bars[1]);
  })
  uint8_t* Wtb0 = sm;
  uint8_t* Wtb1 = Wtb0 + kImgTb0;
  uint8_t* Wenv = Wtb1 + kImgTb1;
  uint8_t* Wtb1lo = Wenv + kImgEnv;                      // split mode only
  uint8_t* H0 = Wtb1lo + (kSplit ? kImgTb1 : 0);
  uint8_t* DE = H0;
  uint8_t* A1 = H0 + kOp64;
  uint8_t* X = A1 + kOp128;
  uint8_t* A1lo = X + kOp128;                            // split mode only
  float* s_geo = reinterpret_cast<float*>(A1lo + (kSplit ? kOp128 : 0));   // [kT][GP]: u, d, fc, dfc
  float* s_dB = s_geo + kT * GP;                          // [kT][GP]: dB
  float* s_Y = s_dB + kT * GP;
  float* s_dy = s_Y + kT * NLM;                           // [kT][NLM]
  float* s_du = s_dy + kT * NLM;                          // [4][kT]
  float* s_g = s_du + 4 * kT;                             // [kSegCap][CL]
  // [4][kT][NLM] per-quarter dY partials: X is free from the start of the
  // tile until the dz1 epilogue, and the partials are summed right after the
  // env1^T MMA
  float* s_dyq = reinterpret_cast<float*>(X);
  const int r = threadIdx.x & (kT - 1), h = threadIdx.x >> 7;
  MetaPre mq = meta_load(b, blockIdx.x, P);
  for (int tile = blockIdx.x; tile < ntiles && !err; tile += gridDim.x) {
    meta_setup(b, tile, P, m, mq);
    if (threadIdx.x == 0 && tile + (int)gridDim.x < ntiles) {
      const int nt = tile + (int)gridDim.x;
      prefetch_meta(b, nt);
      prefetch_rows(b.dR, 3, nt);
      prefetch_rows(b.dX, D, nt);
      prefetch_rows(b.dU, 1, nt);
      prefetch_rows(b.dY, NLM, nt);
      prefetch_rows(b.Ek[1], C, nt);
    }
    const bool valid = r < m.np;
    if (h == 0) {                                     // geometry, envelope, harmonics
      float Y[NLM], u[3] = {0.f, 0.f, 0.f}, d = 1.0f, fc = 0.0f, dfc = 0.0f;
#pragma unroll
      for (int q = 0; q < NLM; ++q) Y[q] = 0.0f;
      if (valid) geometry<LM>(b, tile, r, w.rc, u, d, fc, dfc, Y);
      float* g = s_geo + r * GP;
      g[0] = u[0]; g[1] = u[1]; g[2] = u[2]; g[3] = d; g[4] = fc; g[5] = dfc;
#pragma unroll
      for (int q = 0; q < NLM; ++q) s_Y[r * NLM + q] = Y[q];
    } else if (h == 1) {                              // two-body input row: species, Bessel basis
      float h0[16], B[NB], dB[NB];
#pragma unroll
      for (int q = 0; q < 16; ++q) h0[q] = 0.0f;
#pragma unroll
      for (int q = 0; q < NB; ++q) dB[q] = 0.0f;
      if (valid) {
        const float dx = b.dR[sidx(tile, 3, 0, r)], dy = b.dR[sidx(tile, 3, 1, r)], dz = b.dR[sidx(tile, 3, 2, r)];
        const int zi = b.species[m.pi[r]], zj = b.species[m.pj[r]];
        bessel<NB>(sqrtf(dx * dx + dy * dy + dz * dz), w.rc, B, dB);
#pragma unroll
        for (int q = 0; q < 2; ++q) {                 // one-hot species (no dynamic register index)
          h0[q] = zi == q ? 1.0f : 0.0f;
          h0[2 + q] = zj == q ? 1.0f : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) h0[4 + q] = B[q];
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) s_dB[r * GP + q] = dB[q];
      st_h0<Tin, kSplit>(H0, r, h0);
    }
    stage_g<CL>(b.dgsum[1], m, s_g);
    float e1[4];                                      // e^1 of channels 4h..4h+3 (stored by pass A)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) e1[cc] = valid ? b.Ek[1][sidx(tile, C, 4 * h + cc, r)] : 0.0f;
    mm.run([&] { mma_k<Tin>(tmem + 0, H0, 0, Wtb0, 128, kSplit ? 3 : 1, false, 0); });   // z1
    epi_silu_keep_grad(tmem, 0, [&](int rr, int n0, const float* o) { st16_op<Tin, kSplit>(A1, A1lo, rr, n0, o); });
    // z2; the env adjoint below (DE, the dY partials, Gamma rows) and the dx^0
    // loads touch neither its operands nor its accumulator, and run under it
    mm.start([&] { mma_split<Tin, kSplit>(tmem + 128, A1, A1lo, Wtb1, Wtb1lo, 128, 8, false, 0); });
    {
      float dy[NLM];
      const float* e = e1;
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) dy[lm] = 0.0f;
      float de[4];                                    // de of channels 4h..4h+3: one 8-byte store
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = 4 * h + cc;
        float dG[NLM];
        get_g<NLM>(s_g, b.dgsum[1], m, r, valid, c, dG);
        float acc = 0.0f;
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
          acc = fmaf(dG[lm], s_Y[r * NLM + lm], acc);
          dy[lm] = fmaf(dG[lm], e[cc], dy[lm]);
        }
        de[cc] = acc;
      }
      st_cols<Tin, 4>(DE, r, 4 * h, de);
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) s_dyq[(h * kT + r) * NLM + lm] = dy[lm];
    }
    float dxo[32];                                    // dx^0, columns 32h..32h+31, in flight during the MMAs
#pragma unroll
    for (int q = 0; q < 32; ++q) dxo[q] = valid ? b.dX[sidx(tile, D, 32 * h + q, r)] : 0.0f;
    mm.wait();
    mm.run([&] { mma_k<Tin>(tmem + 288, DE, 0, Wenv, 128, 1, true, 16); });    // env1^T de
    if (h == 0)
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm)
        s_dy[r * NLM + lm] = (s_dyq[r * NLM + lm] + s_dyq[(kT + r) * NLM + lm]) +
                             (s_dyq[(2 * kT + r) * NLM + lm] + s_dyq[(3 * kT + r) * NLM + lm]);
    {
      float du = 0.0f, dxe[32];
      tmem_ld32(lanes(tmem) + 288 + 32 * h, dxe);
      const float fc = s_geo[r * GP + 4];
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        float z2[16], o[16];
        tmem_ld16(lanes(tmem) + 128 + 32 * h + 16 * hf, z2);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float dx = dxe[16 * hf + q] + dxo[16 * hf + q];
          du = fmaf(dx, silu_b(z2[q]), du);
          o[q] = dx * fc * dsilu_b(z2[q]);
        }
        st16_op<Tin, kSplit>(A1, A1lo, r, 32 * h + 16 * hf, o);
      }
      s_du[h * kT + r] = du;
    }
    mm.run([&] { mma_split<Tin, kSplit>(tmem + 128, A1, A1lo, Wtb1, Wtb1lo, 128, 8, true, 128); });   // da1
    epi(tmem, 128, 128, [&](int rr, int n0, const float* da) {
      float g1[16], o[16];                             // SiLU'(z1), left in TMEM by the z1 epilogue
      tmem_ld16(lanes(tmem) + n0, g1);
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = da[q] * g1[q];
      st16_op<Tin, kSplit>(X, A1lo, rr, n0, o);
    });
    float duo = 0.0f, dyo[NLM];                       // loaded ahead of the MMA wait
    if (threadIdx.x < kT) {
      duo = valid ? b.dU[sidx(tile, 1, 0, r)] : 0.0f;
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) dyo[lm] = valid ? b.dY[sidx(tile, NLM, lm, r)] : 0.0f;
    }
    mm.run([&] {                                                                // dh0
      mma_k<Tin>(tmem + 416, X, 0, Wtb0, kSplit ? 48 : 16, 8, true, 128);
      if (kSplit) mma_k<Tin>(tmem + 416, A1lo, 0, Wtb0, 48, 8, true, 128, true);
    });
    mq = meta_load(b, tile + (int)gridDim.x, P);
    if (threadIdx.x < kT) {
      float dh[16];
      tmem_ld16(lanes(tmem) + 416, dh);
      if (kSplit) {
        float dl[16];
        tmem_ld16(lanes(tmem) + 448, dl);
#pragma unroll
        for (int q = 0; q < 16; ++q) dh[q] += dl[q];
      }
      if (valid) {
        const float* g = s_geo + r * GP;
        const float u[3] = {g[0], g[1], g[2]};
        const float d = g[3], dfc = g[5];
        const size_t pp = (size_t)(m.p0 + r);
        float gd = ((s_du[r] + s_du[kT + r]) + (s_du[2 * kT + r] + s_du[3 * kT + r]) + duo) * dfc;
#pragma unroll
        for (int n = 0; n < NB; ++n) gd = fmaf(dh[4 + n], s_dB[r * GP + n], gd);
        float dY[NLM];
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) dY[lm] = s_dy[r * NLM + lm] + dyo[lm];
        float gu[3];
        sph_harm_vjp<LM>(u[0], u[1], u[2], dY, gu);
        const float ud = gu[0] * u[0] + gu[1] * u[1] + gu[2] * u[2];
        const float inv = 1.0f / d;
#pragma unroll
        for (int a = 0; a < 3; ++a) b.G[pp * 3 + a] = gd * u[a] + (gu[a] - ud * u[a]) * inv;
      }
    }
    __syncthreads();
  }
  BF_EPILOGUE
}

// shared-memory bytes of each kernel (+1024 for the manual 1024-byte alignment)
template <int LM>
struct Smem {
  static constexpr int NLM = Tc<LM>::NLM, CL = Tc<LM>::CL, NL = LM + 1;
  static constexpr size_t a(bool split) {
    return 1024 + kImgTb0 + (split ? 2 : 1) * kImgTb1 + kImgEnv + kOp64 + (split ? 3 : 2) * kOp128 +
           4 * (kT + kT * NLM + kT * EP);
  }
  static constexpr size_t b1 = 1024 + Tc<LM>::kImgEmb + NL * kImgMix + kOp128 + Tc<LM>::kOpT +
                               4 * (2 * kT * NLM + kSegCap * CL);
  static constexpr size_t b2 = 1024 + kImgLat0 + kImgLat1 + kImgEnv + kOpH + kOp128 + 4 * (kT + kT * NLM + kT * EP);
  static constexpr size_t c(bool split) {
    return 1024 + kImgLat0 + kImgLat1 + (split ? 2 : 1) * kImgE0 + kOpH + kOp128 + kOp64 +
           4 * (11 * kT + kSegCap * CL);
  }
  static constexpr size_t bt = 1024 + kImgEnv + kImgLat0 + kImgLat1 + Tc<LM>::kImgEmb + NL * kImgMix + kOpH +
                               reg_a1<LM>() + 4 * (2 * (kT + kT * NLM) + 4 * kT + kSegCap * CL);
  static constexpr size_t at(bool split) {
    return 1024 + kImgTb0 + (split ? 2 : 1) * kImgTb1 + kImgEnv + kOp64 + (split ? 3 : 2) * kOp128 +
           4 * (2 * kT * GP + 2 * kT * NLM + 4 * kT + kSegCap * CL);
  }
  // 4 KB left for the static Meta, barriers and flags of every kernel
  static constexpr size_t kLimit = 232448 - 4096;
  static_assert(a(true) <= kLimit && b1 <= kLimit && b2 <= kLimit && c(true) <= kLimit && bt <= kLimit &&
                    at(true) <= kLimit,
                "shared memory per kernel");
  static_assert(kOpH + kOp128 >= 4 * kT * Tc<LM>::CLP, "pass C reuses HA + A1 for the dGamma contributions");
  static_assert(kOp128 >= 4 * 4 * kT * NLM, "pass A^T keeps the dY partials in X");
  static_assert(kOpH >= kOp64 + 4 * 4 * kT * NLM, "pass B^T keeps the dY partials in HA after its first 64 columns");
  static_assert(kOpH + reg_a1<LM>() >= 4 * D * kT, "pass B^T stages its dx^{k-1} tile over HA and A1");
  static_assert(kOp128 >= 2 * D * kT, "passes A and B2 stage their x tile in A1");
  static_assert(Tc<LM>::kOpT >= 2 * CL * kT, "pass B1 stages its V^k tile in T");
};
template struct Smem<0>;
template struct Smem<1>;
template struct Smem<2>;

int g_sms = 0;

template <class Tin, bool kSplit, int LM>
void run_tc(const BfW& w, const PassBufs& b, int64_t capacity, cudaStream_t s, KernelMarks* km) {
  using Sm = Smem<LM>;
  constexpr int CL = Tc<LM>::CL;
  constexpr size_t kSmA = Sm::a(kSplit), kSmC = Sm::c(kSplit), kSmAT = Sm::at(kSplit);
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(k_bf_a<Tin, kSplit, LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmA);
    cudaFuncSetAttribute(k_bf_b1<Tin, LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::b1);
    cudaFuncSetAttribute(k_bf_b2<Tin, LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::b2);
    cudaFuncSetAttribute(k_bf_c<Tin, kSplit, LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmC);
    cudaFuncSetAttribute(k_bf_bt<Tin, true, LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::bt);
    cudaFuncSetAttribute(k_bf_bt<Tin, false, LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::bt);
    cudaFuncSetAttribute(k_bf_at<Tin, kSplit, LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmAT);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    init = true;
  }
  const int64_t tiles = (capacity + kT - 1) / kT;
  const int grid = (int)std::min<int64_t>(tiles, g_sms > 0 ? g_sms : 148);
  const int L = w.n_layers;
  auto mark = [&](int k) {
    if (km) km->mark(k, s);
  };
  // per-atom sums of a pass's Gamma partials (timed with that pass)
  auto sums = [&](const float* part, float* gsum) {
    const int64_t items = (int64_t)b.n_atoms * (CL / 4);
    if (items == 0) return;
    const int blocks = (int)std::min<int64_t>((items + 255) / 256, (int64_t)(g_sms > 0 ? g_sms : 148) * 16);
    k_atom_sums<CL><<<blocks, 256, 0, s>>>(part, b.row_ptr, b.n_atoms, b.flags, gsum);
  };
  mark(kPhStart);
  k_bf_a<Tin, kSplit, LM><<<grid, kThr4, kSmA, s>>>(w, b);
  sums(b.gam[1], b.gsum[1]);
  mark(kPhA);
  for (int k = 1; k < L; ++k) {
    k_bf_b1<Tin, LM><<<grid, kThr4, Sm::b1, s>>>(w, b, k);
    mark(kPhB);
    k_bf_b2<Tin, LM><<<grid, kThr4, Sm::b2, s>>>(w, b, k);
    sums(b.gam[k + 1], b.gsum[k + 1]);
    mark(kPhB2);
  }
  k_bf_c<Tin, kSplit, LM><<<grid, kThr4, kSmC, s>>>(w, b);
  sums(b.dgam[L], b.dgsum[L]);
  mark(kPhC);
  for (int k = L - 1; k >= 1; --k) {
    if (k == 1) k_bf_bt<Tin, true, LM><<<grid, kThr4, Sm::bt, s>>>(w, b, k);
    else k_bf_bt<Tin, false, LM><<<grid, kThr4, Sm::bt, s>>>(w, b, k);
    sums(b.dgam[k], b.dgsum[k]);
    mark(kPhBT);
  }
  k_bf_at<Tin, kSplit, LM><<<grid, kThr4, kSmAT, s>>>(w, b);
  mark(kPhAT);
}

template <int LM>
void run_mode(const BfW& w, const PassBufs& b, int64_t capacity, cudaStream_t s, KernelMarks* km, TcMode mode) {
  switch (mode) {
    case TcMode::kBf16: run_tc<__nv_bfloat16, false, LM>(w, b, capacity, s, km); break;
    case TcMode::kFp16: run_tc<__half, false, LM>(w, b, capacity, s, km); break;
    case TcMode::kFp16Split: run_tc<__half, true, LM>(w, b, capacity, s, km); break;
  }
}

}  // namespace

bool bf16_supported(int lmax, int C_, int D_, int E_, int L) {
  return lmax >= 0 && lmax <= 2 && C_ == C && D_ == D && E_ == E && L >= 2 && L <= kMaxLayers;
}

int bf16_tile() { return kT; }

int bf16_silu_probe(int n, const float* x, float* y) {
  if (n <= 0) return 0;
  k_silu_probe<<<(n + 255) / 256, 256>>>(n, x, y);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}

int bf16_inject_wait_timeout(int enable) {
  const long long cycles = enable ? (1ll << 20) : (1ll << 31);
  const int skip = enable ? 1 : 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return -1;   // no pass kernel in flight
  if (cudaMemcpyToSymbol(c_wait_cycles, &cycles, sizeof(cycles)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_no_weight_copies, &skip, sizeof(skip)) != cudaSuccess) return -1;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}

void bf16_energy_forces(const BfW& w, const PassBufs& b, int64_t capacity, cudaStream_t s, KernelMarks* km,
                        TcMode mode) {
  switch (w.lmax) {
    case 0: run_mode<0>(w, b, capacity, s, km, mode); break;
    case 1: run_mode<1>(w, b, capacity, s, km, mode); break;
    default: run_mode<2>(w, b, capacity, s, km, mode); break;
  }
}

}  // namespace al
