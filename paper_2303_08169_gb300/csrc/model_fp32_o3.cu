// model_fp32_o3.cu - FP32 pass sequences of full-O(3) models (Sec. 2.1's
// equivariance read to include inversion): features of both parities per
// channel, every even and odd coupling path (tpLo_* tables of gen_tp.cpp),
// one mixing block per output irrep (l, s).  The pass kernels are the ones of
// model_fp32.cuh, instantiated with the full-O(3) shape.
//
// Tile: 16 pairs.  The tensor-product output of a tile is held in shared
// memory for the channel mixing (TT C NT floats), and with NT = 102 at l_max
// 2 a 32-pair tile would not fit the 227 KB of a block.
#include "model_fp32.cuh"

namespace al {
namespace {

constexpr int kTileO3 = 16;
using CfgTinyO3 = Cfg<1, 8, 32, 32, true>;
using CfgMainL1O3 = Cfg<1, 16, 128, 32, true>;
using CfgMainO3 = Cfg<2, 16, 128, 32, true>;

}  // namespace

bool fp32_o3_supported(int lmax, int C, int D, int E) {
  return (lmax == 1 && C == 8 && D == 32 && E == 32) || ((lmax == 1 || lmax == 2) && C == 16 && D == 128 && E == 32);
}

int fp32_o3_tile() { return kTileO3; }

void fp32_o3_energy_forces(int lmax, int C, int D, int E, const ModelW& w, const PassBufs& b, int64_t capacity,
                           cudaStream_t s, KernelMarks* km, const Fp32Launch* ls) {
  if (lmax == 1 && C == 8 && D == 32 && E == 32) run<CfgTinyO3, float, kTileO3>(w, b, capacity, s, km, ls);
  else if (lmax == 1) run<CfgMainL1O3, float, kTileO3>(w, b, capacity, s, km, ls);
  else run<CfgMainO3, float, kTileO3>(w, b, capacity, s, km, ls);
}

}  // namespace al
