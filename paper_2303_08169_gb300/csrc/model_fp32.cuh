// model_fp32.cuh - FP32 pair-tile kernels: forward passes and hand-written
// adjoint (forces f = -dE/dr, Eq. 1) for the Allegro-shaped model.
//
// Model (per ordered pair (i, j, n); the paper fixes only E = sum_ij E_ij and
// equivariance, Sec. 2.1; the layer reading is the one of the oracle):
//   x0 = fc(d) MLP_2b([onehot Z_i, onehot Z_j, B(d)]),  V0 = Lin(x0) (x) Y(u)
//   layer k: e = Lin_env(x^{k-1}); Gamma_i = sum_j e_ij (x) Y_ij / sqrt(nu)
//            T = CG(V^{k-1}_ij, Gamma_i); V^k = mix(T)   (k < L)
//            x^k = (x^{k-1} + fc MLP_k([x^{k-1}, T_scalars])) / sqrt2
//   E_ij = MLP_E(x^L);  E_i = sigma_Z sum_j E_ij + mu_Z
//
// Pass structure over tiles of kTile consecutive pairs of the CSR list (the
// scatter into Gamma_i is a barrier between layers):
//   A      : geometry, two-body MLP, x0 (stored), e^1 -> Gamma^1 partials
//   B_k    : TP_k + mix -> V^k (stored), latent_k -> x^k (stored),
//            e^{k+1} -> Gamma^{k+1} partials                      (k < L)
//   C      : layer L + energy MLP forward, then its adjoint at once
//            (dE/dE_ij = sigma_{Z_i} is local): dx^{L-1}, dV^{L-1},
//            dGamma^L partials, du
//   B_k^T  : adjoint of the Gamma^{k+1} scatter and of layer k (forward
//            of layer k recomputed in the tile)                   (k = L-1..1)
//   A^T    : adjoint of the Gamma^1 scatter, two-body MLP (recomputed),
//            geometry -> g_ij = dE/dDelta_ij
// Per-atom sums (Gamma, dGamma, sum_j E_ij) are written as per-(tile, atom)
// partials at index tile + atom and summed in tile order by the consumer, so
// every result is bitwise deterministic without atomics.
#pragma once
#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "model.h"
#include "tp_tables.inc"

namespace al {
namespace {

constexpr int kTile = 32;       // pairs per tile (FP32 passes)
constexpr int kTileDual = 16;   // pairs per tile (tangent passes: two floats per value)
constexpr int kThreads = 256;   // 8 (16) threads per pair in per-pair phases
constexpr float kRsqrt2 = 0.70710678118654752f;

// ----------------------------------------------------------------------------
// Weight staging: K-chunks of kKC rows of a [K][N] matrix are copied into a
// double-buffered shared-memory ring with cp.async while the previous chunk
// is consumed.
constexpr int kKC = 16;

AL_DEV void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
AL_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int n>
AL_DEV void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(n)); }

// Stage n floats (n % 4 == 0, 16-byte aligned source) into shared memory.
AL_DEV void stage(float* dst, const float* __restrict__ src, int n) {
  for (int q = threadIdx.x; q < n / 4; q += kThreads) cp_async16(dst + 4 * q, src + 4 * q);
}

template <int N, int K>
AL_DEV void load_chunk(float* wbuf, const float* __restrict__ Wt, int ch) {
  const int k0 = ch * kKC;
  const int kc = min(kKC, K - k0);
  stage(wbuf + (ch & 1) * kKC * N, Wt + (size_t)k0 * N, kc * N);
  cp_async_commit();
}


// Tensor-product tables per l_max; O3: the full-O(3) product over inputs of
// both parities (V of 2 NLM components, output blocks b = s (l_max+1) + l).
// Its true-scalar block 0 is the natural-parity scalar block, so the scalar
// functions are the natural ones (they read V's true tensors only).
template <int LMAX, bool O3 = false> struct TP;
template <> struct TP<0> {
  static constexpr int NT = TP0_NT, NS = TP0_NS;
  template <class S> static AL_DEV void fwd(const S* V, const S* G, S* T) { tp0_fwd(V, G, T); }
  template <class S> static AL_DEV void fwd_s(const S* V, const S* G, S* T) { tp0_fwd_scalar(V, G, T); }
  template <class S>
  static AL_DEV void bwd(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp0_bwd(V, G, dT, dV, dG); }
  template <class S>
  static AL_DEV void bwd_s(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp0_bwd_scalar(V, G, dT, dV, dG); }
  static constexpr AL_DEV int P(int l) { return tp0_P(l); }
  static constexpr AL_DEV int toff(int l) { return tp0_toff(l); }
};
template <> struct TP<1> {
  static constexpr int NT = TP1_NT, NS = TP1_NS;
  template <class S> static AL_DEV void fwd(const S* V, const S* G, S* T) { tp1_fwd(V, G, T); }
  template <class S> static AL_DEV void fwd_s(const S* V, const S* G, S* T) { tp1_fwd_scalar(V, G, T); }
  template <class S>
  static AL_DEV void bwd(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp1_bwd(V, G, dT, dV, dG); }
  template <class S>
  static AL_DEV void bwd_s(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp1_bwd_scalar(V, G, dT, dV, dG); }
  static constexpr AL_DEV int P(int l) { return tp1_P(l); }
  static constexpr AL_DEV int toff(int l) { return tp1_toff(l); }
};
template <> struct TP<2> {
  static constexpr int NT = TP2_NT, NS = TP2_NS;
  template <class S> static AL_DEV void fwd(const S* V, const S* G, S* T) { tp2_fwd(V, G, T); }
  template <class S> static AL_DEV void fwd_s(const S* V, const S* G, S* T) { tp2_fwd_scalar(V, G, T); }
  template <class S>
  static AL_DEV void bwd(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp2_bwd(V, G, dT, dV, dG); }
  template <class S>
  static AL_DEV void bwd_s(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp2_bwd_scalar(V, G, dT, dV, dG); }
  static constexpr AL_DEV int P(int l) { return tp2_P(l); }
  static constexpr AL_DEV int toff(int l) { return tp2_toff(l); }
};
template <> struct TP<1, true> {
  static constexpr int NT = TP1O_NT, NS = TP1O_NS;
  static_assert(TP1O_NS == TP1_NS, "true-scalar block");
  template <class S> static AL_DEV void fwd(const S* V, const S* G, S* T) { tp1o_fwd(V, G, T); }
  template <class S> static AL_DEV void fwd_s(const S* V, const S* G, S* T) { tp1_fwd_scalar(V, G, T); }
  template <class S>
  static AL_DEV void bwd(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp1o_bwd(V, G, dT, dV, dG); }
  template <class S>
  static AL_DEV void bwd_s(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp1_bwd_scalar(V, G, dT, dV, dG); }
  static constexpr AL_DEV int P(int b) { return tp1o_P(b); }
  static constexpr AL_DEV int toff(int b) { return tp1o_toff(b); }
};
template <> struct TP<2, true> {
  static constexpr int NT = TP2O_NT, NS = TP2O_NS;
  static_assert(TP2O_NS == TP2_NS, "true-scalar block");
  template <class S> static AL_DEV void fwd(const S* V, const S* G, S* T) { tp2o_fwd(V, G, T); }
  template <class S> static AL_DEV void fwd_s(const S* V, const S* G, S* T) { tp2_fwd_scalar(V, G, T); }
  template <class S>
  static AL_DEV void bwd(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp2o_bwd(V, G, dT, dV, dG); }
  template <class S>
  static AL_DEV void bwd_s(const S* V, const S* G, const S* dT, S* dV, S* dG) { tp2_bwd_scalar(V, G, dT, dV, dG); }
  static constexpr AL_DEV int P(int b) { return tp2o_P(b); }
  static constexpr AL_DEV int toff(int b) { return tp2o_toff(b); }
};

// Model shape.  NLM components per channel for the neighbour sums Gamma and
// the harmonics; NV for the features V^k: NLM (natural parity) or 2 NLM (full
// O(3), pseudotensors after the true tensors).  The channel mixing has NBLK
// output blocks, block b of order b % (l_max + 1) and parity b / (l_max + 1).
template <int LMAX_, int C_, int D_, int E_, bool O3_ = false>
struct Cfg {
  static constexpr int LMAX = LMAX_, C = C_, D = D_, E = E_;
  static constexpr bool O3 = O3_;
  using Tp = TP<LMAX, O3>;
  static constexpr int S = 2, NB = 8, H0 = 2 * S + NB, LDH0 = 16;
  static constexpr int NLM = (LMAX + 1) * (LMAX + 1);
  static constexpr int NV = O3 ? 2 * NLM : NLM;
  static constexpr int NBLK = O3 ? 2 * (LMAX + 1) : LMAX + 1;
  static constexpr int NT = Tp::NT, NS = Tp::NS;
  static constexpr int KH = D + C * NS;
  static constexpr int NW0 = C * (LMAX + 1);
  static constexpr int CL = C * NLM;   // Gamma per pair or atom
  static constexpr int CV = C * NV;    // V^k per pair
  static constexpr int LDD = D + 4;   // row strides in shared memory
  static constexpr int LDH = KH + 4;
  static constexpr int LDE = E + 4;
  static constexpr int WB = 2 * kKC * (KH > D ? KH : D);   // weight staging ring
  static constexpr int psum() {
    int n = 0;
    for (int b = 0; b < NBLK; ++b) n += Tp::P(b);
    return n;
  }
  static constexpr int MIXW = C * C * psum();   // all mixing matrices
  static_assert(NBLK <= kMaxMixBlocks, "mixing blocks");
};

AL_DEV int l_of(int lm) { return lm == 0 ? 0 : (lm < 4 ? 1 : 2); }

// Offset of mixing block b inside the concatenated shared-memory copy of the
// mixing matrices ([C][C P_b] each, b = 0 .. NBLK - 1).
template <class Cf>
AL_DEV int mix_off(int b) {
  int o = 0;
  for (int q = 0; q < b; ++q) o += Cf::C * Cf::C * Cf::Tp::P(q);
  return o;
}

template <class Cf>
AL_DEV void stage_mix(const LayerW& LW, float* s_mix) {
  for (int b = 0; b < Cf::NBLK; ++b)
    stage(s_mix + mix_off<Cf>(b), LW.mix[b], Cf::C * Cf::C * Cf::Tp::P(b));
  cp_async_commit();
}

// Tile GEMM: out[m][n] = sum_k A[m*LDA + k] * Wt[k*N + n] for m < TT, n < N.
// A in shared memory, Wt ([K][N], 16-byte aligned) staged through wbuf
// (>= 2 kKC N floats of shared memory); 256 threads with a TM x TN register
// tile each; epi(m, n, value) consumes every output once.  All threads of the
// block must call it; it begins and ends with a block barrier.
//
// Shared-memory traffic per k step of a warp (one wavefront = 128 bytes):
// with TN % 4 == 0, at least 16 row groups and rows whose 16-byte chunk
// stride is not a multiple of 4, the threads of a warp take 16 (or 32)
// consecutive row groups and 2 (or 1) column groups: their weight loads fall
// in one 64-byte run and A is read as float4 along k (rows in distinct
// chunks of a wavefront), 12 wavefronts per 4 k steps against 16 FMA issue
// cycles.  Otherwise a warp takes consecutive column groups (weights
// contiguous across the warp, A nearly broadcast) and A is read per k.
template <class T>
AL_DEV void ld4(const T* p, T* out) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else {
    static_assert(sizeof(T) == 8, "float or Dual");
    const float4 v0 = reinterpret_cast<const float4*>(p)[0], v1 = reinterpret_cast<const float4*>(p)[1];
    out[0] = T(v0.x, v0.y); out[1] = T(v0.z, v0.w); out[2] = T(v1.x, v1.y); out[3] = T(v1.z, v1.w);
  }
}

template <int N, int K, int TT, int LDA, class T, class Epi>
AL_DEV void gemm(const T* __restrict__ A, const float* __restrict__ Wt, float* wbuf, Epi&& epi) {
  constexpr int M = TT;
  constexpr int NCH = (K + kKC - 1) / kKC;
  static_assert(N % 4 == 0, "weights are staged in 16-byte units");
  __syncthreads();
  load_chunk<N, K>(wbuf, Wt, 0);
  if constexpr ((M * N) % kThreads != 0) {
    constexpr int R = (M * N + kThreads - 1) / kThreads;
    T acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0f;
    for (int ch = 0; ch < NCH; ++ch) {
      if (ch + 1 < NCH) {
        load_chunk<N, K>(wbuf, Wt, ch + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const float* wb = wbuf + (ch & 1) * kKC * N;
      const int k0 = ch * kKC, kc = min(kKC, K - k0);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int idx = threadIdx.x + r * kThreads;
        if (idx < M * N) {
          const int m = idx / N, n = idx % N;
          for (int k = 0; k < kc; ++k) acc[r] = fmaf(A[m * LDA + k0 + k], wb[k * N + n], acc[r]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int idx = threadIdx.x + r * kThreads;
      if (idx < M * N) epi(idx / N, idx % N, acc[r]);
    }
  } else {
    constexpr int OPT = M * N / kThreads;
    constexpr int TM = OPT >= 16 ? 2 : 1;
    constexpr int TN = OPT / TM;
    static_assert(N % TN == 0, "tile shape");
    constexpr int TX = N / TN;
    constexpr int TY = kThreads / TX;
    static_assert(TY * TM == M, "tile shape");
    constexpr int kChunkStride = LDA * (int)sizeof(T) / 16;
    constexpr bool kRows = TN % 4 == 0 && TY >= 16 && K % 4 == 0 && (LDA * (int)sizeof(T)) % 16 == 0 &&
                           kChunkStride % 4 != 0;
    const int tx = kRows ? (int)threadIdx.x / TY : (int)threadIdx.x % TX;
    const int ty = kRows ? (int)threadIdx.x % TY : (int)threadIdx.x / TX;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;
    for (int ch = 0; ch < NCH; ++ch) {
      if (ch + 1 < NCH) {
        load_chunk<N, K>(wbuf, Wt, ch + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const int k0 = ch * kKC;
      const T* a0 = A + ty * LDA + k0;
      if constexpr (kRows) {
        // thread tx's own TN columns, float4 groups at tx TN + 4 q
        const float* wc = wbuf + (ch & 1) * kKC * N + tx * TN;
        auto step4 = [&](int k) {
          T a[TM][4];
#pragma unroll
          for (int i = 0; i < TM; ++i) ld4(a0 + i * TY * LDA + k, a[i]);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            float b[TN];
#pragma unroll
            for (int q = 0; q < TN / 4; ++q) {
              const float4 v = *reinterpret_cast<const float4*>(wc + (k + kk) * N + 4 * q);
              b[4 * q] = v.x; b[4 * q + 1] = v.y; b[4 * q + 2] = v.z; b[4 * q + 3] = v.w;
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
              for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i][kk], b[j], acc[i][j]);
          }
        };
        if (K - k0 >= kKC) {
#pragma unroll
          for (int k = 0; k < kKC; k += 4) step4(k);
        } else {
          for (int k = 0; k < K - k0; k += 4) step4(k);
        }
      } else {
        // TN % 4 == 0: float4 group q of thread tx covers columns q TX 4 + tx 4 ..+3, so
        // that the 16-byte loads of a warp are contiguous (no bank conflicts)
        const float* wc = wbuf + (ch & 1) * kKC * N + (TN % 4 == 0 ? tx * 4 : tx * TN);
        auto step = [&](int k) {
          T a[TM];
          float b[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = a0[i * TY * LDA + k];
          if constexpr (TN % 4 == 0) {
#pragma unroll
            for (int q = 0; q < TN / 4; ++q) {
              const float4 v = *reinterpret_cast<const float4*>(wc + k * N + q * TX * 4);
              b[4 * q] = v.x; b[4 * q + 1] = v.y; b[4 * q + 2] = v.z; b[4 * q + 3] = v.w;
            }
          } else if constexpr (TN % 2 == 0) {
#pragma unroll
            for (int q = 0; q < TN / 2; ++q) {
              const float2 v = reinterpret_cast<const float2*>(wc + k * N)[q];
              b[2 * q] = v.x; b[2 * q + 1] = v.y;
            }
          } else {
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = wc[k * N + j];
          }
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        };
        if (K - k0 >= kKC) {
#pragma unroll
          for (int k = 0; k < kKC; ++k) step(k);
        } else {
          for (int k = 0; k < K - k0; ++k) step(k);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j)
        epi(ty + i * TY,
            kRows ? tx * TN + j : (TN % 4 == 0 ? (j / 4) * TX * 4 + tx * 4 + (j % 4) : tx * TN + j), acc[i][j]);
  }
}

// ----------------------------------------------------------------------------
// Tile bookkeeping: pair meta data and segments (runs of equal centre atom).
template <int TT>
struct TileMeta {
  int pi[TT], pj[TT], code[TT], seg[TT], atom[TT];
  int nseg, np, p0, tile;
};

// Tiles of the current list (0 on pair overflow: the list is incomplete).
// Every pass kernel loops over tiles tile = blockIdx.x, + gridDim.x, ...
template <int TT>
AL_DEV int num_tiles(const PassBufs& b) {
  if (*b.flags & 1) return 0;
  const int P = (int)min((int64_t)*b.n_pairs, b.capacity);
  return (P + TT - 1) / TT;
}

template <int TT>
AL_DEV void tile_setup(const PassBufs& b, TileMeta<TT>& t, int tile) {
  static_assert(TT <= 32, "one warp sets a tile up");
  const int P = (int)min((int64_t)*b.n_pairs, b.capacity);
  const int p0 = tile * TT;
  const int np = min(TT, P - p0);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int i = -1;
    if (lane < np) {
      i = b.pi[p0 + lane];
      t.pi[lane] = i;
      t.pj[lane] = b.pj[p0 + lane];
      t.code[lane] = b.pcode[p0 + lane];
    } else if (lane < TT) {
      t.pi[lane] = 0;
      t.pj[lane] = 0;
      t.code[lane] = 62;  // n = 0
    }
    const int prev = __shfl_up_sync(0xffffffffu, i, 1);
    const bool head = lane < np && (lane == 0 || i != prev);
    const unsigned m = __ballot_sync(0xffffffffu, head);
    const unsigned below = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    if (lane < TT) t.seg[lane] = lane < np ? __popc(m & below) - 1 : 0;
    if (head) t.atom[__popc(m & below) - 1] = i;
    if (lane == 0) {
      t.nseg = __popc(m);
      t.np = np;
      t.p0 = p0;
      t.tile = tile;
    }
  }
  __syncthreads();
}

// Sum of per-(tile, atom) partials of every segment's atom: out[s][x].
template <int W, int TT, class T>
AL_DEV void load_segments(const T* __restrict__ part, const int* __restrict__ row_ptr,
                          const TileMeta<TT>& t, T* out) {
  for (int idx = threadIdx.x; idx < t.nseg * W; idx += kThreads) {
    const int s = idx / W, x = idx % W;
    const int i = t.atom[s];
    const int t0 = row_ptr[i] / TT, t1 = (row_ptr[i + 1] - 1) / TT;
    T acc = 0.0f;
    for (int tt = t0; tt <= t1; ++tt) acc += part[(size_t)(tt + i) * W + x];
    out[s * W + x] = acc;
  }
}

// part[(tile + atom) * W + x] = sum over the segment's pairs of f(p, x).
template <int W, int TT, class T, class F>
AL_DEV void store_segments(T* __restrict__ part, const TileMeta<TT>& t, F&& f) {
  for (int idx = threadIdx.x; idx < t.nseg * W; idx += kThreads) {
    const int s = idx / W, x = idx % W;
    T acc = 0.0f;
    for (int p = 0; p < t.np; ++p)
      if (t.seg[p] == s) acc += f(p, x);
    part[(size_t)(t.tile + t.atom[s]) * W + x] = acc;
  }
}

// Copy a kTile x W block of a pair-major global array into shared memory
// (zero rows past the end of the list).
template <int W, int TT, class T>
AL_DEV void load_rows(const T* __restrict__ g, const TileMeta<TT>& t, T* s, int lds) {
  for (int idx = threadIdx.x; idx < TT * W; idx += kThreads) {
    const int m = idx / W, n = idx % W;
    s[m * lds + n] = m < t.np ? g[(size_t)(t.p0 + m) * W + n] : T(0.0f);
  }
}

// Geometry of one pair: unit vector, distance, envelope and SH.  Tangent
// passes: the separation moves along v_j - v_i (b.vdir, the position
// direction of the second-order adjoint).
template <class Cf, class T>
AL_DEV void geometry(const PassBufs& b, float rc, int i, int j, int code, T u[3], T& d,
                     T& fc, T& dfc, T* Y) {
  Box box{{b.L[0], b.L[1], b.L[2]}};
  if (b.atomL) box = Box{{b.atomL[3 * i], b.atomL[3 * i + 1], b.atomL[3 * i + 2]}};
  double dd[3];
  pair_delta(b.wpos, i, j, code, box, dd);
  T dx = (float)dd[0], dy = (float)dd[1], dz = (float)dd[2];
  if constexpr (is_dual<T>::value) {
    dx.t = b.vdir[3 * j] - b.vdir[3 * i];
    dy.t = b.vdir[3 * j + 1] - b.vdir[3 * i + 1];
    dz.t = b.vdir[3 * j + 2] - b.vdir[3 * i + 2];
  }
  d = sqrtf(dx * dx + dy * dy + dz * dz);
  const T inv = 1.0f / d;
  u[0] = dx * inv;
  u[1] = dy * inv;
  u[2] = dz * inv;
  envelope(d, rc, fc, dfc);
  sph_harm<Cf::LMAX>(u[0], u[1], u[2], Y);
}

// Training dumps: copy a tile x W block of shared memory (row stride lds)
// into a per-pair array (row-major [P][W]); no-op for a null array.  Tangent
// passes write the values to g and the tangents to gt.
template <int W, int TT, class T>
AL_DEV void dump_rows(float* g, float* gt, const TileMeta<TT>& t, const T* s, int lds) {
  if (!g) return;
  for (int idx = threadIdx.x; idx < t.np * W; idx += kThreads) {
    const int m = idx / W, n = idx % W;
    g[(size_t)(t.p0 + m) * W + n] = val(s[m * lds + n]);
    if constexpr (is_dual<T>::value) gt[(size_t)(t.p0 + m) * W + n] = s[m * lds + n].t;
  }
}

// A per-pair or per-(tile, atom) array of the pass buffers viewed as T
// (tangent passes: arrays of Dual, allocated at twice the floats).
template <class T>
AL_DEV T* as(float* p) { return reinterpret_cast<T*>(p); }

// Shared-memory carve-up helper (n elements of X, 16-byte aligned).
struct Carve {
  float* p;
  template <class X = float>
  AL_DEV X* take(int n) {
    X* r = reinterpret_cast<X*>(p);
    p += ((int)(n * sizeof(X) / 4) + 3) & ~3;
    return r;
  }
};

// ============================================================================
// Pass A: geometry, two-body MLP, x0, e^1 -> Gamma^1 partials.
template <class Cf, class T, int TT>
__global__ void __launch_bounds__(kThreads) k_pass_a(ModelW w, PassBufs b) {
  constexpr int D = Cf::D, C = Cf::C, NLM = Cf::NLM, LDD = Cf::LDD;
  __shared__ TileMeta<TT> t;
  constexpr int kSub = kThreads / TT;
  extern __shared__ float4 smem4[];
  const int ntiles = num_tiles<TT>(b);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  tile_setup(b, t, tile);
  Carve cv{reinterpret_cast<float*>(smem4)};
  float* s_wb = cv.take(Cf::WB);
  T* s_h0 = cv.take<T>(TT * Cf::LDH0);
  T* s_fc = cv.take<T>(TT);
  T* s_Y = cv.take<T>(TT * NLM);
  T* s_z1 = cv.take<T>(TT * LDD);
  T* s_x = cv.take<T>(TT * LDD);
  T* s_e = cv.take<T>(TT * C);
  if (threadIdx.x < TT) {
    const int p = threadIdx.x;
    T* h = s_h0 + p * Cf::LDH0;
    for (int k = 0; k < Cf::LDH0; ++k) h[k] = 0.0f;
    if (p < t.np) {
      T u[3], d, fc, dfc, Y[NLM], B[Cf::NB];
      geometry<Cf, T>(b, w.rc, t.pi[p], t.pj[p], t.code[p], u, d, fc, dfc, Y);
      bessel<Cf::NB>(d, w.rc, B, nullptr);
      h[b.species[t.pi[p]]] = 1.0f;
      h[Cf::S + b.species[t.pj[p]]] = 1.0f;
      for (int k = 0; k < Cf::NB; ++k) h[2 * Cf::S + k] = B[k];
      s_fc[p] = fc;
      for (int k = 0; k < NLM; ++k) s_Y[p * NLM + k] = Y[k];
    } else {
      s_fc[p] = 0.0f;
      for (int k = 0; k < NLM; ++k) s_Y[p * NLM + k] = 0.0f;
    }
  }
  __syncthreads();
  gemm<D, Cf::H0, TT, Cf::LDH0>(s_h0, w.tb0.t, s_wb, [&](int m, int n, T v) { s_z1[m * LDD + n] = silu(v); });
  __syncthreads();
  T* X0 = as<T>(b.X[0]);
  gemm<D, D, TT, LDD>(s_z1, w.tb1.t, s_wb, [&](int m, int n, T v) {
    const T x = s_fc[m] * silu(v);
    s_x[m * LDD + n] = x;
    if (m < t.np) X0[(size_t)(t.p0 + m) * D + n] = x;
  });
  __syncthreads();
  gemm<C, D, TT, LDD>(s_x, w.layer[0].env.t, s_wb, [&](int m, int n, T v) { s_e[m * C + n] = v; });
  __syncthreads();
  store_segments<Cf::CL>(as<T>(b.gam[1]), t, [&](int p, int x) {
    return s_e[p * C + x / NLM] * s_Y[p * NLM + x % NLM];
  });
  __syncthreads();   // the next tile reuses the shared arrays
  }
}

// V^{k-1}_c (NV components) for one pair and channel: from the stored array,
// or for k = 1 from w0 (x) Y (true tensors only: the pseudotensor part of
// V^0 is zero).
template <class Cf, int TT, class T>
AL_DEV void load_v(int k, const PassBufs& b, const TileMeta<TT>& t, int p, int c, const T* s_w0,
                   const T* s_Y, T* V) {
  constexpr int NLM = Cf::NLM, NV = Cf::NV;
  if (k == 1) {
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm)
      V[lm] = s_w0[p * Cf::NW0 + c * (Cf::LMAX + 1) + l_of(lm)] * s_Y[p * NLM + lm];
#pragma unroll
    for (int lm = NLM; lm < NV; ++lm) V[lm] = 0.0f;
  } else {
    const T* g = as<T>(b.V[k - 1]) + (size_t)(t.p0 + p) * Cf::CV + c * NV;
#pragma unroll
    for (int lm = 0; lm < NV; ++lm) V[lm] = p < t.np ? g[lm] : 0.0f;
  }
}

// ============================================================================
// Pass B_k (1 <= k < L): tensor product, mixing, latent MLP, e^{k+1} scatter.
template <class Cf, class T, int TT>
__global__ void __launch_bounds__(kThreads) k_pass_b(ModelW w, PassBufs b, int k) {
  constexpr int D = Cf::D, C = Cf::C, NLM = Cf::NLM, NT = Cf::NT, NS = Cf::NS, CL = Cf::CL;
  constexpr int NV = Cf::NV, CV = Cf::CV;
  constexpr int LDD = Cf::LDD, LDH = Cf::LDH, LMAX = Cf::LMAX;
  using Tp = typename Cf::Tp;
  __shared__ TileMeta<TT> t;
  constexpr int kSub = kThreads / TT;
  extern __shared__ float4 smem4[];
  const int ntiles = num_tiles<TT>(b);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  tile_setup(b, t, tile);
  Carve cv{reinterpret_cast<float*>(smem4)};
  float* s_wb = cv.take(Cf::WB);
  T* s_h = cv.take<T>(TT * LDH);
  T* s_z1 = cv.take<T>(TT * LDD);
  T* s_w0 = cv.take<T>(TT * Cf::NW0);
  T* s_G = cv.take<T>(TT * CL);
  T* s_T = cv.take<T>(TT * C * NT);
  T* s_fc = cv.take<T>(TT);
  T* s_Y = cv.take<T>(TT * NLM);
  T* s_e = cv.take<T>(TT * C);
  float* s_mix = cv.take(Cf::MIXW);
  const LayerW& LW = w.layer[k - 1];
  stage_mix<Cf>(LW, s_mix);
  if (threadIdx.x < TT) {
    const int p = threadIdx.x;
    T u[3], d, fc = 0.0f, dfc, Y[NLM];
    for (int q = 0; q < NLM; ++q) Y[q] = 0.0f;
    if (p < t.np) geometry<Cf, T>(b, w.rc, t.pi[p], t.pj[p], t.code[p], u, d, fc, dfc, Y);
    s_fc[p] = fc;
    for (int q = 0; q < NLM; ++q) s_Y[p * NLM + q] = Y[q];
  }
  load_rows<D>(as<T>(b.X[k - 1]), t, s_h, LDH);
  load_segments<CL>(as<T>(b.gam[k]), b.row_ptr, t, s_G);
  __syncthreads();
  if (k == 1) {
    gemm<Cf::NW0, D, TT, LDH>(s_h, w.emb.t, s_wb, [&](int m, int n, T v) { s_w0[m * Cf::NW0 + n] = v; });
    __syncthreads();
  }
  const int p = threadIdx.x / kSub, sub = threadIdx.x % kSub;
  for (int c = sub; c < C; c += kSub) {
    T V[NV], G[NLM], To[NT];
    load_v<Cf, TT>(k, b, t, p, c, s_w0, s_Y, V);
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) G[lm] = p < t.np ? s_G[t.seg[p] * CL + c * NLM + lm] : 0.0f;
    Tp::fwd(V, G, To);
#pragma unroll
    for (int o = 0; o < NT; ++o) s_T[(p * C + c) * NT + o] = To[o];
#pragma unroll
    for (int q = 0; q < NS; ++q) s_h[p * LDH + D + c * NS + q] = To[q];
  }
  cp_async_wait<0>();
  __syncthreads();
  if (b.train) {
    dump_rows<C * NS>(b.tr.s[k], b.trt.s[k], t, s_h + D, LDH);
    dump_rows<C * NT>(b.tr.T[k], b.trt.T[k], t, s_T, C * NT);
  }
  // channel mixing: V^k[c'][s3 l3 m] = sum_{c, q} mix_b[c'][c P_b + q] T[c][block b, q, m]
  // for every output block b = s3 (l_max + 1) + l3
  for (int co = sub; co < C; co += kSub) {
#pragma unroll
    for (int bk = 0; bk < Cf::NBLK; ++bk) {
      const int l3 = bk % (LMAX + 1), s3 = bk / (LMAX + 1);
      const int Pl = Tp::P(bk), off = Tp::toff(bk), nm = 2 * l3 + 1;
      const float* Wm = s_mix + mix_off<Cf>(bk) + co * (C * Pl);
      for (int m = 0; m < nm; ++m) {
        T acc = 0.0f;
        for (int c = 0; c < C; ++c)
          for (int q = 0; q < Pl; ++q)
            acc = fmaf(Wm[c * Pl + q], s_T[(p * C + c) * NT + off + q * nm + m], acc);
        if (p < t.np) as<T>(b.V[k])[(size_t)(t.p0 + p) * CV + co * NV + s3 * NLM + l3 * l3 + m] = acc;
      }
    }
  }
  gemm<D, Cf::KH, TT, LDH>(s_h, LW.lat0.t, s_wb, [&](int m, int n, T v) { s_z1[m * LDD + n] = silu(v); });
  __syncthreads();
  T* Xk = as<T>(b.X[k]);
  gemm<D, D, TT, LDD>(s_z1, LW.lat1.t, s_wb, [&](int m, int n, T v) {
    const T x = (s_h[m * LDH + n] + s_fc[m] * silu(v)) * kRsqrt2;
    s_h[m * LDH + n] = x;
    if (m < t.np) Xk[(size_t)(t.p0 + m) * D + n] = x;
  });
  __syncthreads();
  gemm<C, D, TT, LDH>(s_h, w.layer[k].env.t, s_wb, [&](int m, int n, T v) { s_e[m * C + n] = v; });
  __syncthreads();
  store_segments<CL>(as<T>(b.gam[k + 1]), t, [&](int pp, int x) {
    return s_e[pp * C + x / NLM] * s_Y[pp * NLM + x % NLM];
  });
  __syncthreads();   // the next tile reuses the shared arrays
  }
}

// Reduce a per-thread value over the kSub consecutive lanes of one pair.
template <int kSub, class T>
AL_DEV T sub_sum_(T v) {
#pragma unroll
  for (int o = kSub / 2; o > 0; o >>= 1) v += shfl_xor(0xffffffffu, v, o);
  return v;
}

// ============================================================================
// Pass C: last layer L and energy MLP forward, then their adjoint.
template <class Cf, class T, int TT>
__global__ void __launch_bounds__(kThreads) k_pass_c(ModelW w, PassBufs b) {
  constexpr int D = Cf::D, C = Cf::C, E = Cf::E, NLM = Cf::NLM, NS = Cf::NS, CL = Cf::CL;
  constexpr int NV = Cf::NV, CV = Cf::CV;
  constexpr int LDD = Cf::LDD, LDH = Cf::LDH, LDE = Cf::LDE, LMAX = Cf::LMAX;
  using Tp = typename Cf::Tp;
  __shared__ TileMeta<TT> t;
  constexpr int kSub = kThreads / TT;
  __shared__ T s_eij[TT];
  __shared__ T s_sig[TT];
  extern __shared__ float4 smem4[];
  const int ntiles = num_tiles<TT>(b);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  tile_setup(b, t, tile);
  const int L = w.n_layers;
  const LayerW& LW = w.layer[L - 1];
  Carve cv{reinterpret_cast<float*>(smem4)};
  float* s_wb = cv.take(Cf::WB);
  T* s_h = cv.take<T>(TT * LDH);
  T* s_z1 = cv.take<T>(TT * LDD);
  T* s_a1 = cv.take<T>(TT * LDD);
  T* s_z2 = cv.take<T>(TT * LDD);
  T* s_ze = cv.take<T>(TT * LDE);
  T* s_ae = cv.take<T>(TT * LDE);
  T* s_G = cv.take<T>(TT * CL);
  T* s_dg = cv.take<T>(TT * CL);
  T* s_w0 = cv.take<T>(TT * Cf::NW0);
  T* s_dw0 = cv.take<T>(TT * Cf::NW0);
  T* s_fc = cv.take<T>(TT);
  T* s_Y = cv.take<T>(TT * NLM);
  T* s_dy = cv.take<T>(TT * NLM);
  T* s_du = cv.take<T>(TT);
  if (threadIdx.x < TT) {
    const int p = threadIdx.x;
    T u[3], d, fc = 0.0f, dfc, Y[NLM];
    for (int q = 0; q < NLM; ++q) Y[q] = 0.0f;
    if (p < t.np) geometry<Cf, T>(b, w.rc, t.pi[p], t.pj[p], t.code[p], u, d, fc, dfc, Y);
    s_fc[p] = fc;
    for (int q = 0; q < NLM; ++q) {
      s_Y[p * NLM + q] = Y[q];
      s_dy[p * NLM + q] = 0.0f;
    }
    // dL/dE_ij = seed * sigma_Z; tangent passes take the seed's tangent too
    T sd = 0.0f;
    if (p < t.np) {
      sd = b.tr.seed_atom ? b.tr.seed_atom[t.pi[p]] : b.tr.seed;
      if constexpr (is_dual<T>::value) sd.t = b.tr.seed_atom_t ? b.tr.seed_atom_t[t.pi[p]] : 0.0f;
      sd = sd * w.sigma[b.species[t.pi[p]]];
    }
    s_sig[p] = sd;
  }
  load_rows<D>(as<T>(b.X[L - 1]), t, s_h, LDH);
  load_segments<CL>(as<T>(b.gam[L]), b.row_ptr, t, s_G);
  __syncthreads();
  if (L == 1) {
    gemm<Cf::NW0, D, TT, LDH>(s_h, w.emb.t, s_wb, [&](int m, int n, T v) { s_w0[m * Cf::NW0 + n] = v; });
    __syncthreads();
  }
  const int p = threadIdx.x / kSub, sub = threadIdx.x % kSub;
  for (int c = sub; c < C; c += kSub) {
    T V[NV], G[NLM], S[NS];
    load_v<Cf, TT>(L, b, t, p, c, s_w0, s_Y, V);
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) G[lm] = p < t.np ? s_G[t.seg[p] * CL + c * NLM + lm] : 0.0f;
    Tp::fwd_s(V, G, S);
#pragma unroll
    for (int q = 0; q < NS; ++q) s_h[p * LDH + D + c * NS + q] = S[q];
  }
  __syncthreads();
  if (b.train) dump_rows<C * NS>(b.tr.s[L], b.trt.s[L], t, s_h + D, LDH);
  gemm<D, Cf::KH, TT, LDH>(s_h, LW.lat0.t, s_wb, [&](int m, int n, T v) {
    s_z1[m * LDD + n] = v;
    s_a1[m * LDD + n] = silu(v);
  });
  __syncthreads();
  gemm<D, D, TT, LDD>(s_a1, LW.lat1.t, s_wb, [&](int m, int n, T v) {
    s_z2[m * LDD + n] = v;
    s_h[m * LDH + n] = (s_h[m * LDH + n] + s_fc[m] * silu(v)) * kRsqrt2;   // x^L
  });
  __syncthreads();
  gemm<E, D, TT, LDH>(s_h, w.e0.t, s_wb, [&](int m, int n, T v) {
    s_ze[m * LDE + n] = v;
    s_ae[m * LDE + n] = silu(v);
  });
  __syncthreads();
  if (b.train) {
    dump_rows<D>(b.tr.a1_l[L], b.trt.a1_l[L], t, s_a1, LDD);
    dump_rows<D>(b.tr.xL, b.trt.xL, t, s_h, LDH);
    dump_rows<E>(b.tr.ae, b.trt.ae, t, s_ae, LDE);
    dump_rows<1>(b.tr.dEij, b.trt.dEij, t, s_sig, 1);
  }
  if (threadIdx.x < TT) {
    const int q = threadIdx.x;
    T acc = 0.0f;
    for (int n = 0; n < E; ++n) acc = fmaf(__ldg(w.eout + n), s_ae[q * LDE + n], acc);
    s_eij[q] = q < t.np ? acc : 0.0f;
  }
  // adjoint of the energy MLP: dE/dE_ij = sigma_{Z_i}
  for (int idx = threadIdx.x; idx < TT * E; idx += kThreads) {
    const int m = idx / E, n = idx % E;
    s_ze[m * LDE + n] = s_sig[m] * __ldg(w.eout + n) * silu_grad(s_ze[m * LDE + n]);
  }
  __syncthreads();
  if (threadIdx.x < t.nseg) {
    const int s = threadIdx.x;
    double acc = 0.0;
    for (int q = 0; q < t.np; ++q)
      if (t.seg[q] == s) acc += (double)val(s_eij[q]);
    b.epart[t.tile + t.atom[s]] = acc;
  }
  if (b.train) dump_rows<E>(b.tr.dze, b.trt.dze, t, s_ze, LDE);
  gemm<D, E, TT, LDE>(s_ze, w.e0.n, s_wb, [&](int m, int n, T v) { s_h[m * LDH + n] = v; });  // dx^L
  __syncthreads();
  {
    T du = 0.0f;
    const T fc = s_fc[p];
    for (int n = sub; n < D; n += kSub) {
      const T dx = s_h[p * LDH + n];
      const T z2 = s_z2[p * LDD + n];
      du = fmaf(dx, silu(z2), du);
      s_z2[p * LDD + n] = dx * fc * kRsqrt2 * silu_grad(z2);
    }
    du = sub_sum_<kSub>(du);
    if (sub == 0) s_du[p] = du * kRsqrt2;
  }
  __syncthreads();
  if (b.train) dump_rows<D>(b.tr.dz2_l[L], b.trt.dz2_l[L], t, s_z2, LDD);
  gemm<D, D, TT, LDD>(s_z2, LW.lat1.n, s_wb, [&](int m, int n, T v) {
    s_z1[m * LDD + n] = v * silu_grad(s_z1[m * LDD + n]);
  });
  __syncthreads();
  if (b.train) dump_rows<D>(b.tr.dz1_l[L], b.trt.dz1_l[L], t, s_z1, LDD);
  gemm<Cf::KH, D, TT, LDD>(s_z1, LW.lat0.n, s_wb, [&](int m, int n, T v) {
    if (n < D) s_h[m * LDH + n] = v + s_h[m * LDH + n] * kRsqrt2;   // dx^{L-1}
    else s_h[m * LDH + n] = v;                                      // d(scalars)
  });
  __syncthreads();
  {
    T dyl[NLM];
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) dyl[lm] = 0.0f;
    for (int c = sub; c < C; c += kSub) {
      T V[NV], G[NLM], dS[NS], dV[NV], dG[NLM];
      load_v<Cf, TT>(L, b, t, p, c, s_w0, s_Y, V);
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) {
        G[lm] = p < t.np ? s_G[t.seg[p] * CL + c * NLM + lm] : 0.0f;
        dG[lm] = 0.0f;
      }
#pragma unroll
      for (int lm = 0; lm < NV; ++lm) dV[lm] = 0.0f;
#pragma unroll
      for (int q = 0; q < NS; ++q) dS[q] = s_h[p * LDH + D + c * NS + q];
      Tp::bwd_s(V, G, dS, dV, dG);   // true scalars: from true tensors only
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) s_dg[p * CL + c * NLM + lm] = dG[lm];
      if (L >= 2) {
        if (p < t.np) {
          T* g = as<T>(b.dV) + (size_t)(t.p0 + p) * CV + c * NV;
#pragma unroll
          for (int lm = 0; lm < NV; ++lm) g[lm] = dV[lm];
        }
      } else {
        T dw[LMAX + 1];
#pragma unroll
        for (int l = 0; l <= LMAX; ++l) dw[l] = 0.0f;
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
          dw[l_of(lm)] = fmaf(dV[lm], s_Y[p * NLM + lm], dw[l_of(lm)]);
          dyl[lm] = fmaf(s_w0[p * Cf::NW0 + c * (LMAX + 1) + l_of(lm)], dV[lm], dyl[lm]);
        }
#pragma unroll
        for (int l = 0; l <= LMAX; ++l) s_dw0[p * Cf::NW0 + c * (LMAX + 1) + l] = dw[l];
      }
    }
    if (L == 1) {
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) {
        const T v = sub_sum_<kSub>(dyl[lm]);
        if (sub == 0) s_dy[p * NLM + lm] = v;
      }
    }
  }
  __syncthreads();
  if (L == 1) {
    if (b.train) dump_rows<Cf::NW0>(b.tr.dw0, b.trt.dw0, t, s_dw0, Cf::NW0);
    gemm<D, Cf::NW0, TT, Cf::NW0>(s_dw0, w.emb.n, s_wb, [&](int m, int n, T v) { s_h[m * LDH + n] += v; });
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < t.np * D; idx += kThreads) {
    const int m = idx / D, n = idx % D;
    as<T>(b.dX)[(size_t)(t.p0 + m) * D + n] = s_h[m * LDH + n];
  }
  for (int idx = threadIdx.x; idx < t.np * NLM; idx += kThreads)
    as<T>(b.dY)[(size_t)t.p0 * NLM + idx] = s_dy[idx];
  if (threadIdx.x < t.np) as<T>(b.dU)[t.p0 + threadIdx.x] = s_du[threadIdx.x];
  store_segments<CL>(as<T>(b.dgam[L]), t, [&](int pp, int x) { return s_dg[pp * CL + x]; });
  __syncthreads();   // the next tile reuses the shared arrays
  }
}

// ============================================================================
// Pass B_k^T (k = L-1 .. 1): adjoint of the Gamma^{k+1} scatter and of layer k.
template <class Cf, class T, int TT>
__global__ void __launch_bounds__(kThreads) k_pass_b_bwd(ModelW w, PassBufs b, int k) {
  constexpr int D = Cf::D, C = Cf::C, NLM = Cf::NLM, NT = Cf::NT, NS = Cf::NS, CL = Cf::CL;
  constexpr int NV = Cf::NV, CV = Cf::CV;
  constexpr int LDD = Cf::LDD, LDH = Cf::LDH, LMAX = Cf::LMAX;
  using Tp = typename Cf::Tp;
  __shared__ TileMeta<TT> t;
  constexpr int kSub = kThreads / TT;
  extern __shared__ float4 smem4[];
  const int ntiles = num_tiles<TT>(b);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  tile_setup(b, t, tile);
  const LayerW& LW = w.layer[k - 1];
  const LayerW& LN = w.layer[k];
  Carve cv{reinterpret_cast<float*>(smem4)};
  float* s_wb = cv.take(Cf::WB);
  T* s_h = cv.take<T>(TT * LDH);
  T* s_z1 = cv.take<T>(TT * LDD);
  T* s_a1 = cv.take<T>(TT * LDD);
  T* s_z2 = cv.take<T>(TT * LDD);
  T* s_tmp = cv.take<T>(TT * (CV > LDD ? CV : LDD));
  T* s_G = cv.take<T>(TT * CL);
  T* s_dG = cv.take<T>(TT * CL);
  T* s_w0 = cv.take<T>(TT * Cf::NW0);
  T* s_dw0 = cv.take<T>(TT * Cf::NW0);
  T* s_e = cv.take<T>(TT * C);
  T* s_de = cv.take<T>(TT * C);
  T* s_fc = cv.take<T>(TT);
  T* s_Y = cv.take<T>(TT * NLM);
  T* s_dy = cv.take<T>(TT * NLM);
  T* s_du = cv.take<T>(TT);
  float* s_mix = cv.take(Cf::MIXW);
  stage_mix<Cf>(LW, s_mix);
  if (threadIdx.x < TT) {
    const int p = threadIdx.x;
    T u[3], d, fc = 0.0f, dfc, Y[NLM];
    for (int q = 0; q < NLM; ++q) Y[q] = 0.0f;
    if (p < t.np) geometry<Cf, T>(b, w.rc, t.pi[p], t.pj[p], t.code[p], u, d, fc, dfc, Y);
    s_fc[p] = fc;
    for (int q = 0; q < NLM; ++q) s_Y[p * NLM + q] = Y[q];
  }
  cp_async_wait<0>();
  load_rows<D>(as<T>(b.X[k]), t, s_z2, LDD);          // x^k (temporarily)
  load_rows<D>(as<T>(b.X[k - 1]), t, s_h, LDH);       // x^{k-1}
  load_segments<CL>(as<T>(b.gam[k]), b.row_ptr, t, s_G);
  load_segments<CL>(as<T>(b.dgam[k + 1]), b.row_ptr, t, s_dG);
  __syncthreads();
  gemm<C, D, TT, LDD>(s_z2, LN.env.t, s_wb, [&](int m, int n, T v) { s_e[m * C + n] = v; });  // e^{k+1}
  __syncthreads();
  const int p = threadIdx.x / kSub, sub = threadIdx.x % kSub;
  {
    const T* dg = s_dG + (p < t.np ? t.seg[p] : 0) * CL;
    for (int c = sub; c < C; c += kSub) {
      T acc = 0.0f;
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) acc = fmaf(dg[c * NLM + lm], s_Y[p * NLM + lm], acc);
      s_de[p * C + c] = p < t.np ? acc : 0.0f;
    }
    for (int lm = sub; lm < NLM; lm += kSub) {
      T acc = 0.0f;
      for (int c = 0; c < C; ++c) acc = fmaf(dg[c * NLM + lm], s_e[p * C + c], acc);
      s_dy[p * NLM + lm] = p < t.np ? acc : 0.0f;
    }
  }
  __syncthreads();
  if (b.train) dump_rows<C>(b.tr.de[k], b.trt.de[k], t, s_de, C);
  const T* dXg = as<T>(b.dX);
  gemm<D, C, TT, C>(s_de, LN.env.n, s_wb, [&](int m, int n, T v) {
    s_z2[m * LDD + n] = v + (m < t.np ? dXg[(size_t)(t.p0 + m) * D + n] : 0.0f);   // dx^k
  });
  __syncthreads();
  // recompute layer k forward (scalars, latent MLP)
  if (k == 1) {
    gemm<Cf::NW0, D, TT, LDH>(s_h, w.emb.t, s_wb, [&](int m, int n, T v) { s_w0[m * Cf::NW0 + n] = v; });
    __syncthreads();
  }
  for (int c = sub; c < C; c += kSub) {
    T V[NV], G[NLM], S[NS];
    load_v<Cf, TT>(k, b, t, p, c, s_w0, s_Y, V);
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) G[lm] = p < t.np ? s_G[t.seg[p] * CL + c * NLM + lm] : 0.0f;
    Tp::fwd_s(V, G, S);
#pragma unroll
    for (int q = 0; q < NS; ++q) s_h[p * LDH + D + c * NS + q] = S[q];
  }
  __syncthreads();
  gemm<D, Cf::KH, TT, LDH>(s_h, LW.lat0.t, s_wb, [&](int m, int n, T v) {
    s_z1[m * LDD + n] = v;
    s_a1[m * LDD + n] = silu(v);
  });
  __syncthreads();
  gemm<D, D, TT, LDD>(s_a1, LW.lat1.t, s_wb, [&](int m, int n, T v) { s_tmp[m * LDD + n] = v; });  // z2
  __syncthreads();
  if (b.train) dump_rows<D>(b.tr.a1_l[k], b.trt.a1_l[k], t, s_a1, LDD);
  {
    T du = 0.0f;
    const T fc = s_fc[p];
    for (int n = sub; n < D; n += kSub) {
      const T dx = s_z2[p * LDD + n];
      const T z2 = s_tmp[p * LDD + n];
      du = fmaf(dx, silu(z2), du);
      s_z2[p * LDD + n] = dx * fc * kRsqrt2 * silu_grad(z2);   // dz2
      s_h[p * LDH + n] = dx * kRsqrt2;                          // residual part of dx^{k-1}
    }
    du = sub_sum_<kSub>(du);
    if (sub == 0) s_du[p] = du * kRsqrt2;
  }
  __syncthreads();
  if (b.train) dump_rows<D>(b.tr.dz2_l[k], b.trt.dz2_l[k], t, s_z2, LDD);
  load_rows<CV>(as<T>(b.dV), t, s_tmp, CV);            // dV^k
  gemm<D, D, TT, LDD>(s_z2, LW.lat1.n, s_wb, [&](int m, int n, T v) {
    s_z1[m * LDD + n] = v * silu_grad(s_z1[m * LDD + n]);     // dz1
  });
  __syncthreads();
  if (b.train) dump_rows<D>(b.tr.dz1_l[k], b.trt.dz1_l[k], t, s_z1, LDD);
  gemm<Cf::KH, D, TT, LDD>(s_z1, LW.lat0.n, s_wb, [&](int m, int n, T v) {
    if (n < D) s_h[m * LDH + n] += v;
    else s_h[m * LDH + n] = v;
  });
  __syncthreads();
  // adjoint of mixing and of the full tensor product of layer k
  {
    T dyl[NLM];
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) dyl[lm] = 0.0f;
    for (int c = sub; c < C; c += kSub) {
      T dT[NT];
#pragma unroll
      for (int bk = 0; bk < Cf::NBLK; ++bk) {
        const int l3 = bk % (LMAX + 1), s3 = bk / (LMAX + 1);
        const int Pl = Tp::P(bk), off = Tp::toff(bk), nm = 2 * l3 + 1;
        for (int q = 0; q < Pl; ++q)
          for (int m = 0; m < nm; ++m) {
            T acc = bk == 0 ? s_h[p * LDH + D + c * NS + q] : 0.0f;
            for (int co = 0; co < C; ++co)
              acc = fmaf(s_mix[mix_off<Cf>(bk) + co * (C * Pl) + c * Pl + q],
                         s_tmp[p * CV + co * NV + s3 * NLM + l3 * l3 + m], acc);
            dT[off + q * nm + m] = acc;
          }
      }
      T V[NV], G[NLM], dV[NV], dG[NLM];
      load_v<Cf, TT>(k, b, t, p, c, s_w0, s_Y, V);
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) {
        G[lm] = p < t.np ? s_G[t.seg[p] * CL + c * NLM + lm] : 0.0f;
        dG[lm] = 0.0f;
      }
#pragma unroll
      for (int lm = 0; lm < NV; ++lm) dV[lm] = 0.0f;
      Tp::bwd(V, G, dT, dV, dG);
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) s_dG[p * CL + c * NLM + lm] = dG[lm];   // reuse
      if (k >= 2) {
        if (p < t.np) {
          T* g = as<T>(b.dV) + (size_t)(t.p0 + p) * CV + c * NV;
#pragma unroll
          for (int lm = 0; lm < NV; ++lm) g[lm] = dV[lm];
        }
      } else {
        T dw[LMAX + 1];
#pragma unroll
        for (int l = 0; l <= LMAX; ++l) dw[l] = 0.0f;
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
          dw[l_of(lm)] = fmaf(dV[lm], s_Y[p * NLM + lm], dw[l_of(lm)]);
          dyl[lm] = fmaf(s_w0[p * Cf::NW0 + c * (LMAX + 1) + l_of(lm)], dV[lm], dyl[lm]);
        }
#pragma unroll
        for (int l = 0; l <= LMAX; ++l) s_dw0[p * Cf::NW0 + c * (LMAX + 1) + l] = dw[l];
      }
    }
    if (k == 1) {
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) {
        const T v = sub_sum_<kSub>(dyl[lm]);
        if (sub == 0) s_dy[p * NLM + lm] += v;
      }
    }
  }
  __syncthreads();
  if (k == 1) {
    if (b.train) dump_rows<Cf::NW0>(b.tr.dw0, b.trt.dw0, t, s_dw0, Cf::NW0);
    gemm<D, Cf::NW0, TT, Cf::NW0>(s_dw0, w.emb.n, s_wb, [&](int m, int n, T v) { s_h[m * LDH + n] += v; });
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < t.np * D; idx += kThreads) {
    const int m = idx / D, n = idx % D;
    as<T>(b.dX)[(size_t)(t.p0 + m) * D + n] = s_h[m * LDH + n];
  }
  for (int idx = threadIdx.x; idx < t.np * NLM; idx += kThreads)
    as<T>(b.dY)[(size_t)t.p0 * NLM + idx] += s_dy[idx];
  if (threadIdx.x < t.np) as<T>(b.dU)[t.p0 + threadIdx.x] += s_du[threadIdx.x];
  store_segments<CL>(as<T>(b.dgam[k]), t, [&](int pp, int x) { return s_dG[pp * CL + x]; });
  __syncthreads();   // the next tile reuses the shared arrays
  }
}

// ============================================================================
// Pass A^T: adjoint of the Gamma^1 scatter, of the two-body MLP and of the
// geometry; writes g_ij = dE/dDelta_ij.
template <class Cf, class T, int TT>
__global__ void __launch_bounds__(kThreads) k_pass_a_bwd(ModelW w, PassBufs b) {
  constexpr int D = Cf::D, C = Cf::C, NLM = Cf::NLM, CL = Cf::CL, LDD = Cf::LDD, NB = Cf::NB;
  __shared__ TileMeta<TT> t;
  constexpr int kSub = kThreads / TT;
  extern __shared__ float4 smem4[];
  const int ntiles = num_tiles<TT>(b);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  tile_setup(b, t, tile);
  Carve cv{reinterpret_cast<float*>(smem4)};
  float* s_wb = cv.take(Cf::WB);
  T* s_h0 = cv.take<T>(TT * Cf::LDH0);
  T* s_z1 = cv.take<T>(TT * LDD);
  T* s_a1 = cv.take<T>(TT * LDD);
  T* s_z2 = cv.take<T>(TT * LDD);
  T* s_x = cv.take<T>(TT * LDD);
  T* s_dx = cv.take<T>(TT * LDD);
  T* s_dG = cv.take<T>(TT * CL);
  T* s_e = cv.take<T>(TT * C);
  T* s_de = cv.take<T>(TT * C);
  T* s_dh0 = cv.take<T>(TT * Cf::LDH0);
  T* s_geo = cv.take<T>(TT * 8);        // u[3], d, fc, dfc
  T* s_dB = cv.take<T>(TT * NB);
  T* s_Y = cv.take<T>(TT * NLM);
  T* s_dy = cv.take<T>(TT * NLM);
  T* s_du = cv.take<T>(TT);
  if (threadIdx.x < TT) {
    const int p = threadIdx.x;
    T* h = s_h0 + p * Cf::LDH0;
    for (int q = 0; q < Cf::LDH0; ++q) h[q] = 0.0f;
    T u[3] = {0.f, 0.f, 0.f}, d = 1.0f, fc = 0.0f, dfc = 0.0f, Y[NLM], B[NB], dB[NB];
    for (int q = 0; q < NLM; ++q) Y[q] = 0.0f;
    for (int q = 0; q < NB; ++q) dB[q] = 0.0f;
    if (p < t.np) {
      geometry<Cf, T>(b, w.rc, t.pi[p], t.pj[p], t.code[p], u, d, fc, dfc, Y);
      bessel<NB>(d, w.rc, B, dB);
      h[b.species[t.pi[p]]] = 1.0f;
      h[Cf::S + b.species[t.pj[p]]] = 1.0f;
      for (int q = 0; q < NB; ++q) h[2 * Cf::S + q] = B[q];
    }
    T* g = s_geo + p * 8;
    g[0] = u[0]; g[1] = u[1]; g[2] = u[2]; g[3] = d; g[4] = fc; g[5] = dfc;
    for (int q = 0; q < NB; ++q) s_dB[p * NB + q] = dB[q];
    for (int q = 0; q < NLM; ++q) s_Y[p * NLM + q] = Y[q];
  }
  load_rows<D>(as<T>(b.dX), t, s_dx, LDD);
  load_segments<CL>(as<T>(b.dgam[1]), b.row_ptr, t, s_dG);
  __syncthreads();
  gemm<D, Cf::H0, TT, Cf::LDH0>(s_h0, w.tb0.t, s_wb, [&](int m, int n, T v) {
    s_z1[m * LDD + n] = v;
    s_a1[m * LDD + n] = silu(v);
  });
  __syncthreads();
  gemm<D, D, TT, LDD>(s_a1, w.tb1.t, s_wb, [&](int m, int n, T v) {
    s_z2[m * LDD + n] = v;
    s_x[m * LDD + n] = s_geo[m * 8 + 4] * silu(v);
  });
  __syncthreads();
  if (b.train) {
    dump_rows<Cf::LDH0>(b.tr.h0, b.trt.h0, t, s_h0, Cf::LDH0);
    dump_rows<D>(b.tr.a1_tb, b.trt.a1_tb, t, s_a1, LDD);
  }
  gemm<C, D, TT, LDD>(s_x, w.layer[0].env.t, s_wb, [&](int m, int n, T v) { s_e[m * C + n] = v; });
  __syncthreads();
  const int p = threadIdx.x / kSub, sub = threadIdx.x % kSub;
  {
    const T* dg = s_dG + (p < t.np ? t.seg[p] : 0) * CL;
    for (int c = sub; c < C; c += kSub) {
      T acc = 0.0f;
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) acc = fmaf(dg[c * NLM + lm], s_Y[p * NLM + lm], acc);
      s_de[p * C + c] = p < t.np ? acc : 0.0f;
    }
    for (int lm = sub; lm < NLM; lm += kSub) {
      T acc = 0.0f;
      for (int c = 0; c < C; ++c) acc = fmaf(dg[c * NLM + lm], s_e[p * C + c], acc);
      s_dy[p * NLM + lm] = p < t.np ? acc : 0.0f;
    }
  }
  __syncthreads();
  if (b.train) dump_rows<C>(b.tr.de[0], b.trt.de[0], t, s_de, C);
  gemm<D, C, TT, C>(s_de, w.layer[0].env.n, s_wb, [&](int m, int n, T v) { s_dx[m * LDD + n] += v; });
  __syncthreads();
  {
    T du = 0.0f;
    const T fc = s_geo[p * 8 + 4];
    for (int n = sub; n < D; n += kSub) {
      const T dx = s_dx[p * LDD + n];
      const T z2 = s_z2[p * LDD + n];
      du = fmaf(dx, silu(z2), du);
      s_z2[p * LDD + n] = dx * fc * silu_grad(z2);
    }
    du = sub_sum_<kSub>(du);
    if (sub == 0) s_du[p] = du;
  }
  __syncthreads();
  if (b.train) dump_rows<D>(b.tr.dz2_tb, b.trt.dz2_tb, t, s_z2, LDD);
  gemm<D, D, TT, LDD>(s_z2, w.tb1.n, s_wb, [&](int m, int n, T v) {
    s_z1[m * LDD + n] = v * silu_grad(s_z1[m * LDD + n]);
  });
  __syncthreads();
  if (b.train) dump_rows<D>(b.tr.dz1_tb, b.trt.dz1_tb, t, s_z1, LDD);
  gemm<Cf::H0, D, TT, LDD>(s_z1, w.tb0.n, s_wb, [&](int m, int n, T v) { s_dh0[m * Cf::LDH0 + n] = v; });
  __syncthreads();
  if (threadIdx.x < t.np) {
    const int q = threadIdx.x;
    const T* g = s_geo + q * 8;
    const T u[3] = {g[0], g[1], g[2]};
    const T d = g[3], dfc = g[5];
    const size_t pp = (size_t)(t.p0 + q);
    T gd = (s_du[q] + as<T>(b.dU)[pp]) * dfc;
    for (int n = 0; n < NB; ++n) gd = fmaf(s_dh0[q * Cf::LDH0 + 2 * Cf::S + n], s_dB[q * NB + n], gd);
    T dY[NLM];
    for (int lm = 0; lm < NLM; ++lm) dY[lm] = s_dy[q * NLM + lm] + as<T>(b.dY)[pp * NLM + lm];
    T gu[3];
    sph_harm_vjp<Cf::LMAX>(u[0], u[1], u[2], dY, gu);
    const T ud = gu[0] * u[0] + gu[1] * u[1] + gu[2] * u[2];
    const T inv = 1.0f / d;
    for (int a = 0; a < 3; ++a) as<T>(b.G)[pp * 3 + a] = gd * u[a] + (gu[a] - ud * u[a]) * inv;
  }
  __syncthreads();   // the next tile reuses the shared arrays
  }
}

// ----------------------------------------------------------------------------
// Dynamic shared memory of each pass for scalar type X and tile TT (in the
// order of the kernels' carve-up; weight staging stays FP32).
template <class Cf, class X, int TT>
struct Smem {
  static constexpr int K = (int)(sizeof(X) / 4);
  static constexpr int r(int n) { return (n + 3) & ~3; }
  static constexpr int q(int n) { return r(K * n); }
  static constexpr int T = TT;
  static constexpr size_t a = 4 * (r(Cf::WB) + q(T * Cf::LDH0) + q(T) + q(T * Cf::NLM) + 2 * q(T * Cf::LDD) + q(T * Cf::C));
  static constexpr size_t b = 4 * (r(Cf::WB) + q(T * Cf::LDH) + q(T * Cf::LDD) + q(T * Cf::NW0) +
                                   q(T * Cf::CL) + q(T * Cf::C * Cf::NT) + q(T) + q(T * Cf::NLM) +
                                   q(T * Cf::C) + r(Cf::MIXW));
  static constexpr size_t c = 4 * (r(Cf::WB) + q(T * Cf::LDH) + 3 * q(T * Cf::LDD) + 2 * q(T * Cf::LDE) + 2 * q(T * Cf::CL) +
                                   2 * q(T * Cf::NW0) + q(T) + 2 * q(T * Cf::NLM) + q(T));
  static constexpr int tmpw = Cf::CV > Cf::LDD ? Cf::CV : Cf::LDD;
  static constexpr size_t bb = 4 * (r(Cf::WB) + q(T * Cf::LDH) + 3 * q(T * Cf::LDD) + q(T * tmpw) +
                                    2 * q(T * Cf::CL) + 2 * q(T * Cf::NW0) + 2 * q(T * Cf::C) + q(T) +
                                    2 * q(T * Cf::NLM) + q(T) + r(Cf::MIXW));
  static constexpr size_t ab = 4 * (r(Cf::WB) + q(T * Cf::LDH0) + 5 * q(T * Cf::LDD) + q(T * Cf::CL) + 2 * q(T * Cf::C) +
                                    q(T * Cf::LDH0) + q(T * 8) + q(T * Cf::NB) + 2 * q(T * Cf::NLM) + q(T));
  static_assert(a <= 227 * 1024 && b <= 227 * 1024 && c <= 227 * 1024 && bb <= 227 * 1024 && ab <= 227 * 1024,
                "shared memory per block");
};

int g_sms_fp32 = 0;

template <class Cf, class X, int TT>
void run(const ModelW& w, const PassBufs& b, int64_t capacity, cudaStream_t s, KernelMarks* km,
         const Fp32Launch* ls) {
  using Sm = Smem<Cf, X, TT>;
  static bool init = false;
  if (!init) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms_fp32, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_pass_a<Cf, X, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::a);
    cudaFuncSetAttribute(k_pass_b<Cf, X, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::b);
    cudaFuncSetAttribute(k_pass_c<Cf, X, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::c);
    cudaFuncSetAttribute(k_pass_b_bwd<Cf, X, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::bb);
    cudaFuncSetAttribute(k_pass_a_bwd<Cf, X, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::ab);
    init = true;
  }
  // blocks loop over the tiles of the list (the pair count is known on the
  // device only): waves[k] waves of one resident block per SM (eight by
  // default), or one block per tile of the capacity if that is fewer
  const Fp32Launch dflt;
  const Fp32Launch& sh = ls ? *ls : dflt;
  const int64_t tiles = (capacity + TT - 1) / TT;
  const int sms = g_sms_fp32 > 0 ? g_sms_fp32 : 152;
  auto grid_of = [&](int k) { return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sh.waves[k] * sms)); };
  const int L = w.n_layers;
  auto mark = [&](int k) {
    if (km) km->mark(k, s);
  };
  mark(kPhStart);
  k_pass_a<Cf, X, TT><<<grid_of(kPhA), kThreads, Sm::a, s>>>(w, b);
  mark(kPhA);
  for (int k = 1; k < L; ++k) {
    k_pass_b<Cf, X, TT><<<grid_of(kPhB), kThreads, Sm::b, s>>>(w, b, k);
    mark(kPhB);
  }
  k_pass_c<Cf, X, TT><<<grid_of(kPhC), kThreads, Sm::c, s>>>(w, b);
  mark(kPhC);
  for (int k = L - 1; k >= 1; --k) {
    k_pass_b_bwd<Cf, X, TT><<<grid_of(kPhBT), kThreads, Sm::bb, s>>>(w, b, k);
    mark(kPhBT);
  }
  k_pass_a_bwd<Cf, X, TT><<<grid_of(kPhAT), kThreads, Sm::ab, s>>>(w, b);
  mark(kPhAT);
}

}  // namespace
}  // namespace al
