// model_fp32.cu - FP32 pass sequences of the natural-parity models (the
// kernels are in model_fp32.cuh) and the FP32 dispatch.
#include "model_fp32.cuh"

namespace al {
namespace {

using CfgTiny = Cfg<1, 8, 32, 32>;
using CfgMain = Cfg<2, 16, 128, 32>;
// the main model's widths at l_max 0 and 1 (the l_max sweep of Table 2)
using CfgMainL0 = Cfg<0, 16, 128, 32>;
using CfgMainL1 = Cfg<1, 16, 128, 32>;

}  // namespace

// full-O(3) pass sequences (model_fp32_o3.cu)
bool fp32_o3_supported(int lmax, int C, int D, int E);
int fp32_o3_tile();
void fp32_o3_energy_forces(int lmax, int C, int D, int E, const ModelW& w, const PassBufs& b, int64_t capacity,
                           cudaStream_t s, KernelMarks* km, const Fp32Launch* ls);

int fp32_tile(bool o3) { return o3 ? fp32_o3_tile() : kTile; }

bool fp32_supported(int lmax, int C, int D, int E, bool o3) {
  if (o3) return fp32_o3_supported(lmax, C, D, E);
  return (lmax == 1 && C == 8 && D == 32 && E == 32) || (lmax <= 2 && C == 16 && D == 128 && E == 32);
}

void fp32_energy_forces(int lmax, int C, int D, int E, const ModelW& w, const PassBufs& b,
                        int64_t capacity, cudaStream_t s, KernelMarks* km, const Fp32Launch* ls) {
  if (w.o3) fp32_o3_energy_forces(lmax, C, D, E, w, b, capacity, s, km, ls);
  else if (lmax == 1 && C == 8 && D == 32 && E == 32) run<CfgTiny, float, kTile>(w, b, capacity, s, km, ls);
  else if (lmax == 0) run<CfgMainL0, float, kTile>(w, b, capacity, s, km, ls);
  else if (lmax == 1) run<CfgMainL1, float, kTile>(w, b, capacity, s, km, ls);
  else run<CfgMain, float, kTile>(w, b, capacity, s, km, ls);
}

int fp32_tangent_tile() { return kTileDual; }

void fp32_tangent_passes(int lmax, int C, int D, int E, const ModelW& w, const PassBufs& b, int64_t capacity,
                         cudaStream_t s, KernelMarks* km, const Fp32Launch* ls) {
  if (lmax == 1 && C == 8 && D == 32 && E == 32) run<CfgTiny, Dual, kTileDual>(w, b, capacity, s, km, ls);
  else if (lmax == 2 && C == 16 && D == 128 && E == 32) run<CfgMain, Dual, kTileDual>(w, b, capacity, s, km, ls);
}

}  // namespace al
