// model.h - device-side model description shared by the pass kernels and the
// host orchestration.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace al {

constexpr int kMaxLayers = 4;

// One linear layer y = W x / sqrt(fan_in) stored twice, both pre-scaled:
//   t: [in][out]  (forward:  y[o] = sum_i x[i] t[i][o])
//   n: [out][in]  (adjoint: dx[i] = sum_o dy[o] n[o][i])
struct Lin {
  const float* t = nullptr;
  const float* n = nullptr;
};

// Output blocks of a layer's channel mixing: one per order l <= l_max
// (natural-parity models), or per irrep (l, s), block s (l_max + 1) + l,
// for full-O(3) models of three or more layers.
constexpr int kMaxMixBlocks = 6;

struct LayerW {
  Lin env;                    // C x D, extra factor 1/sqrt(nu)
  // [C][C P_b] per output block b (layers below the last); full O(3): the
  // columns of every block follow the paths of all input irreps (zero for
  // paths whose input irrep the layer does not receive)
  const float* mix[kMaxMixBlocks] = {};
  Lin lat0, lat1;             // (D + C P_0) -> D -> D
};

struct ModelW {
  Lin tb0, tb1;               // (2S + Nb) -> D -> D
  Lin emb;                    // D -> C (lmax + 1)
  LayerW layer[kMaxLayers];
  Lin e0;                     // D -> E
  const float* eout = nullptr;// E (scaled by 1/sqrt(E))
  float sigma[2], mu[2];
  float rc;
  int n_layers;
  int o3 = 0;                 // 1: full-O(3) features (both parities) and tables
};

// Training mode of the FP32 passes: every linear layer's input and the
// gradient of its pre-activation are written per pair (row-major [P][W]) so
// that the weight gradients dW = sum_pairs dz (x) x can be reduced afterwards.
struct TrainBufs {
  float seed = 1.0f;                  // dL/dE of this evaluation (scales sigma_Z)
  const float* seed_atom = nullptr;   // [N] per-atom dL/dE_i instead of seed (training batches)
  const float* seed_atom_t = nullptr; // [N] tangent of seed_atom (tangent passes)
  float* h0 = nullptr;                // [P][16] two-body input (12 used)
  float* a1_tb = nullptr;             // [P][D]  SiLU of the first two-body layer
  float* dz1_tb = nullptr;            // [P][D]
  float* dz2_tb = nullptr;            // [P][D]
  float* de[kMaxLayers] = {};         // [P][C]  gradient of env_{j+1}
  float* dw0 = nullptr;               // [P][C (lmax+1)] gradient of the embedding output
  float* s[kMaxLayers + 1] = {};      // [P][C P_0] tensor-product scalars of layer k
  float* T[kMaxLayers] = {};          // [P][C NT] tensor-product outputs of layer k < L
  float* a1_l[kMaxLayers + 1] = {};   // [P][D]  SiLU of latent layer k, first linear
  float* dz1_l[kMaxLayers + 1] = {};  // [P][D]
  float* dz2_l[kMaxLayers + 1] = {};  // [P][D]
  float* xL = nullptr;                // [P][D]  x^L
  float* ae = nullptr;                // [P][E]  energy-MLP hidden activation
  float* dze = nullptr;               // [P][E]
  float* dEij = nullptr;              // [P]     seed * sigma_Z
};

// Per-pass buffers (device).
struct PassBufs {
  // neighbour list
  const int* pi;
  const int* pj;
  const int* pcode;
  const int* row_ptr;
  const int* n_pairs;     // device scalar
  const int* flags;       // device status bits; passes skip all work on overflow
  int64_t capacity;       // pair capacity of every per-pair array
  const double* wpos;     // N x 3 wrapped positions
  const int* species;     // N
  int n_atoms;
  double L[3];
  const double* atomL = nullptr;  // training batches: N x 3 box lengths per atom (else L)
  // per pair state
  float* X[kMaxLayers];   // x^k, k = 0..L-1    (P x D)
  float* V[kMaxLayers];   // V^k, k = 1..L-1    (P x C NLM)
  float* dX;              // P x D
  float* dV;              // P x C NLM
  float* dU;              // P
  float* dY;              // P x NLM
  float* G;               // P x 3  (dE/dDelta)
  float* S[kMaxLayers];   // BF16 path: tensor-product scalars of layer k (P x C P_0)
  float* dR = nullptr;    // tensor-core path: pair separation in FP32 (P x 3), written by pass A
  // tensor-core path: env output e^k = env_k(x^{k-1}) of layer k in FP32 (P x C,
  // tile-SoA), written by the pass that forms Gamma^k (A for k = 1, B2 of
  // layer k - 1 otherwise) and read by the adjoint passes instead of forming
  // it again from x^{k-1}
  float* Ek[kMaxLayers + 1] = {};
  // per (tile, atom) partial sums, index (tile + atom)
  float* gam[kMaxLayers + 1];   // Gamma^k partials, k = 1..L
  float* dgam[kMaxLayers + 1];  // dGamma^k partials
  // tensor-core path: per-atom sums of those partials (N x C NLM)
  float* gsum[kMaxLayers + 1] = {};
  float* dgsum[kMaxLayers + 1] = {};
  double* epart;                // sum_j E_ij partials
  int tile;                     // pairs per tile (all passes)
  TrainBufs tr;                 // training dumps (FP32 path; tangent passes: the values)
  TrainBufs trt;                // tangent passes: the tangents of the same dumps
  int train;                    // nonzero: write the TrainBufs dumps
  const float* vdir = nullptr;  // tangent passes: N x 3 position direction v
};

// BF16 path weights: pre-scaled BF16 images in the 128-byte-swizzled K-major
// layout of the tensor-core operands (umma.cuh), one per linear layer.
struct BfW {
  const uint8_t* tb0 = nullptr;   // [128 x 64]  (12 inputs used)
  const uint8_t* tb1 = nullptr;   // [128 x 128]
  const uint8_t* emb = nullptr;   // [C (l_max + 1) x 128]
  const uint8_t* e0 = nullptr;    // [32 x 128]
  const uint8_t* env[kMaxLayers] = {};
  const uint8_t* lat0[kMaxLayers] = {};   // [128 x 192] (176 inputs used)
  const uint8_t* lat1[kMaxLayers] = {};
  const uint8_t* mix[kMaxLayers][3] = {}; // [16 x 64] (C P_l inputs used), l <= l_max
  // split mode: tb0 holds [W_hi | W_hi | W_lo] in columns 0, 16, 32; lo images
  // of twobody.1 and energy.0
  const uint8_t* tb1_lo = nullptr;
  const uint8_t* e0_lo = nullptr;
  const float* eout = nullptr;    // 32 FP32
  float sigma[2];
  float rc;
  int n_layers;
  int lmax;
};

bool bf16_supported(int lmax, int C, int D, int E, int L);
int bf16_tile();
// Failure injection for tests (current device): enable != 0 makes every
// tensor-core pass skip its weight copies and wait at most 2^20 cycles for
// them, so each pass raises the timeout flag with nothing in flight;
// enable == 0 restores the copies and the 2^31-cycle limit.  0 on success.
int bf16_inject_wait_timeout(int enable);
// SiLU and its derivative as the tensor-core passes evaluate them (sigmoid
// through tanh.approx.f32): y[2i], y[2i+1] for x[i]; device arrays; legacy
// stream, synchronises.  0 on success.
int bf16_silu_probe(int n, const float* x, float* y);
// Optional launch timing: mark(kind) records an event on the stream after a
// pass kernel, tagged with its kind; interval i lies between event i and
// event i + 1 and belongs to kind[i + 1].
enum KernelKind { kPhStart = -1, kPhA = 0, kPhB, kPhB2, kPhC, kPhBT, kPhAT, kPhCount };
struct KernelMarks {
  static constexpr int kMax = 48;
  cudaEvent_t ev[kMax];
  int kind[kMax];
  int n = 0;
  void mark(int k, cudaStream_t s) {
    if (n < kMax) {
      cudaEventRecord(ev[n], s);
      kind[n++] = k;
    }
  }
};

// Operand type of the tensor-core passes; the images in w must match
// (kFp16Split: FP16 images with the split two-body and energy layers).
enum class TcMode { kBf16, kFp16, kFp16Split };
void bf16_energy_forces(const BfW& w, const PassBufs& b, int64_t capacity, cudaStream_t s,
                        KernelMarks* km, TcMode mode);

// Launch shape of the FP32 pass kernels: pass kind k (kPhA, kPhB, kPhC,
// kPhBT, kPhAT) runs min(tiles of the capacity, waves[k] x SMs) blocks, each
// looping over tiles.  Every tile's arithmetic and its partial rows are fixed
// by the tile, so the results are the same bits for every launch shape; the
// autotuner of api.cu picks the fastest from measured times.
struct Fp32Launch {
  int waves[kPhCount] = {8, 8, 8, 8, 8, 8};
};

// FP32 path: one launcher per pass sequence; templated on the model shape in
// the .cu files, dispatched by (lmax, C, D, E) and w.o3.  Full-O(3) models
// (o3) carry features of both parities per channel, V^k of 2 (l_max+1)^2
// components (index s (l_max+1)^2 + l^2 + m + l), and run tiles of
// fp32_tile(true) pairs.
bool fp32_supported(int lmax, int C, int D, int E, bool o3 = false);
// km (optional): events recorded at the phase boundaries; ls (optional):
// launch shape (default eight waves for every pass).
void fp32_energy_forces(int lmax, int C, int D, int E, const ModelW& w, const PassBufs& b,
                        int64_t capacity, cudaStream_t s, KernelMarks* km = nullptr,
                        const Fp32Launch* ls = nullptr);
int fp32_tile(bool o3 = false);
// Tangent passes of the second-order adjoint: the FP32 pass sequence in
// tangent numbers (value and derivative along the position direction b.vdir),
// tiles of fp32_tangent_tile() pairs.  Every per-pair and per-(tile, atom)
// array of b holds Dual values (twice the floats of the FP32 passes); the
// training dumps write values to b.tr and tangents to b.trt.  Models: the
// 1-layer tiny model and the 2-layer main model.
int fp32_tangent_tile();
void fp32_tangent_passes(int lmax, int C, int D, int E, const ModelW& w, const PassBufs& b, int64_t capacity,
                         cudaStream_t s, KernelMarks* km = nullptr, const Fp32Launch* ls = nullptr);

}  // namespace al
