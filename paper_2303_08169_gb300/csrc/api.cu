// api.cu - C ABI of the library (include/allegro.h): context, weights blob,
// device buffers, orchestration of the neighbour, pair-pass and per-atom
// kernels, and the CUDA-graph MD step.
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/allegro.h"
#include "kernels.h"
#include "md.h"
#include "model.h"
#include "tp_tables.inc"
#include "train.h"
#include "umma.cuh"

namespace {
thread_local std::string g_err;
}

namespace al {
// message returned by allegro_last_error(NULL) (entry points without a context)
void set_global_error(const std::string& msg) { g_err = msg; }
}  // namespace al

using namespace al;

namespace {

const char* kVersion = "allegro-gb300 0.1";

struct Tensor {
  std::string name;
  uint32_t rows, cols;
  const double* data;
};

struct Blob {
  uint32_t S, lmax, L, C, NB, p;
  uint32_t parity;   // 0: natural-parity paths only; 1: full O(3) (odd paths, pseudotensors)
  std::vector<uint32_t> latent, energy;
  double rc, nu;
  std::vector<double> sigma, mu;
  std::vector<Tensor> tensors;
  std::vector<unsigned char> bytes;
  const Tensor* find(const std::string& n) const {
    for (auto& t : tensors)
      if (t.name == n) return &t;
    return nullptr;
  }
};

bool rd32(const std::vector<unsigned char>& b, size_t off, uint32_t& v) {
  if (off + 4 > b.size()) return false;
  std::memcpy(&v, b.data() + off, 4);
  return true;
}
bool rd64f(const std::vector<unsigned char>& b, size_t off, double& v) {
  if (off + 8 > b.size()) return false;
  std::memcpy(&v, b.data() + off, 8);
  return true;
}

// Parse the "ALW1" layout (little-endian host assumed, as on x86-64 and aarch64).
bool parse_blob(const void* data, size_t n, Blob& B, std::string& why) {
  B.bytes.assign((const unsigned char*)data, (const unsigned char*)data + n);
  const auto& b = B.bytes;
  if (n < 48 || std::memcmp(b.data(), "ALW1", 4) != 0) { why = "bad magic"; return false; }
  uint32_t h[11];
  for (int k = 0; k < 11; ++k) rd32(b, 4 + 4 * k, h[k]);
  if (h[0] != 1) { why = "unsupported blob version"; return false; }
  B.S = h[1]; B.lmax = h[2]; B.L = h[3]; B.C = h[4]; B.NB = h[5]; B.p = h[6]; B.parity = h[10];
  if (B.parity > 1) { why = "parity flag must be 0 or 1"; return false; }
  const uint32_t nlat = h[7], nen = h[8], nt = h[9];
  if (nlat > 16 || nen > 16 || B.S > 16 || nt > 4096) { why = "implausible header"; return false; }
  size_t off = 48;
  B.latent.resize(nlat);
  B.energy.resize(nen);
  for (auto& v : B.latent) { if (!rd32(b, off, v)) { why = "truncated"; return false; } off += 4; }
  for (auto& v : B.energy) { if (!rd32(b, off, v)) { why = "truncated"; return false; } off += 4; }
  off += (8 - off % 8) % 8;
  if (!rd64f(b, off, B.rc) || !rd64f(b, off + 8, B.nu)) { why = "truncated"; return false; }
  off += 16;
  B.sigma.resize(B.S);
  B.mu.resize(B.S);
  for (auto& v : B.sigma) { if (!rd64f(b, off, v)) { why = "truncated"; return false; } off += 8; }
  for (auto& v : B.mu) { if (!rd64f(b, off, v)) { why = "truncated"; return false; } off += 8; }
  for (uint32_t t = 0; t < nt; ++t) {
    if (off + 48 > n) { why = "truncated directory"; return false; }
    char name[33];
    std::memcpy(name, b.data() + off, 32);
    name[32] = 0;
    Tensor T;
    T.name = name;
    rd32(b, off + 32, T.rows);
    rd32(b, off + 36, T.cols);
    uint64_t doff;
    std::memcpy(&doff, b.data() + off + 40, 8);
    off += 48;
    if (doff % 8 != 0 || doff + 8ull * T.rows * T.cols > n) { why = "tensor out of range: " + T.name; return false; }
    T.data = reinterpret_cast<const double*>(b.data() + doff);
    B.tensors.push_back(T);
  }
  return true;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// One trainable tensor: its slice of the flat parameter vector (blob order)
// and its pre-scaled FP32 copies ([in][out] and [out][in]) in the weights
// buffer.
struct WInfo {
  std::string name;
  int rows, cols;
  size_t flat_off;
  float scale;
  size_t t_off, n_off;   // offsets in floats inside d_w (t unused for some)
  bool has_t;
  // full-O(3) mixing (mix_pl > 0): the [C][C P_l] blob matrix sits in a
  // [C][C P_u] device block, column c P_l + q at c P_u + mix_q[q]
  int mix_pl = 0, mix_pu = 0;
  std::vector<int> mix_q;
};

// Coupling paths of the full-O(3) tables (gen_tp.cpp's tpLo_*): for output
// block b = s3 (l_max + 1) + l3, every (s1, l1, l2) in that order with
// |l1 - l2| <= l3 <= l1 + l2 and s3 = (l1 + s1 + l2 + l3) mod 2 whose input
// irrep (l1, s1) has its bit s1 (l_max + 1) + l1 set in `in`.
struct O3Path { int s1, l1, l2; };
std::vector<O3Path> o3_paths(int lmax, int b, unsigned in) {
  const int l3 = b % (lmax + 1), s3 = b / (lmax + 1);
  std::vector<O3Path> out;
  for (int s1 = 0; s1 <= 1; ++s1)
    for (int l1 = 0; l1 <= lmax; ++l1) {
      if (!(in >> (s1 * (lmax + 1) + l1) & 1u)) continue;
      for (int l2 = 0; l2 <= lmax; ++l2)
        if (std::abs(l1 - l2) <= l3 && l3 <= l1 + l2 && (l1 + s1 + l2 + l3) % 2 == s3) out.push_back({s1, l1, l2});
    }
  return out;
}

// Input irreps of layer k (bits as above): true tensors for layer 1, then
// every output irrep that some path of the previous layer reaches.
unsigned o3_layer_inputs(int lmax, int k) {
  unsigned in = (1u << (lmax + 1)) - 1u;
  for (int q = 1; q < k; ++q) {
    unsigned out = 0;
    for (int b = 0; b < 2 * (lmax + 1); ++b)
      if (!o3_paths(lmax, b, in).empty()) out |= 1u << b;
    in = out;
  }
  return in;
}

// Training batch (see build_batch): concatenated neighbour lists and atoms
// of all structures, and the per-atom / per-structure loss buffers.
struct TrainBatch {
  BatchArrays a{};
  int n_structs = 0;
  int64_t n_atoms = 0, n_pairs = 0;
  int64_t cap_atoms = 0, cap_pairs = 0;
  int cap_structs = 0;
  int* d_np = nullptr;          // device copy of n_pairs
  float* v = nullptr;           // dL/dF (N x 3): the position direction of the tangent passes
  float* seed = nullptr;        // energy-loss seeds dL/dE_i (N)
  float* f_target = nullptr;    // N x 3
  int64_t* atom_off = nullptr;  // n_structs + 1
  double* e_target = nullptr;
  double* dE = nullptr;         // E_b - E*_b
  double* loss_blk = nullptr;
  double* loss = nullptr;
};

struct allegro_ctx {
  std::string err;
  std::vector<WInfo> winfo;
  int64_t n_params = 0;
  float* d_master = nullptr;   // flat parameter vector (FP32, blob order)
  float* d_grad = nullptr;
  float* d_adam_m = nullptr;
  float* d_adam_v = nullptr;
  float* d_wtmp = nullptr;
  double* d_norm2 = nullptr;
  int adam_t = 0;
  bool tc_dirty = false;       // tensor-core images lag behind d_master
  TrainBufs tr{};
  int64_t tr_cap = 0;
  // second-order adjoint: tangent dumps (trt), the tangent passes' per-pair
  // and per-(tile, atom) arrays of Dual values, and the per-chunk partials of
  // the weight-gradient reductions
  TrainBufs trt{};
  float* tX[kMaxLayers] = {};
  float* tV[kMaxLayers] = {};
  float *tdX = nullptr, *tdV = nullptr, *tdU = nullptr, *tdY = nullptr, *tG = nullptr;
  float* tgam[kMaxLayers + 1] = {};
  float* tdgam[kMaxLayers + 1] = {};
  double* tepart = nullptr;
  float* wpart = nullptr;
  int64_t tr_rows = 0;
  // launch shapes of the FP32 passes chosen by the autotuner: [0] value
  // passes, [1] tangent passes; tuned for capacities up to fl_cap[i]
  Fp32Launch fl[2];
  int64_t fl_cap[2] = {0, 0};
  cudaStream_t stream = nullptr;
  Blob blob;
  double mass[2] = {14.007, 1.008};
  int D = 0, E = 0;
  // weights
  float* d_w = nullptr;
  ModelW w{};
  uint8_t* d_bw = nullptr;     // BF16 swizzled weight images
  BfW bw{};
  uint8_t* d_hw = nullptr;     // FP16 swizzled weight images
  BfW hw{};
  uint8_t* d_sw = nullptr;     // FP16 images with split two-body / energy layers
  BfW sw{};
  bool bf16_ok = false;
  // allocations
  std::vector<void*> allocs;
  int64_t n_atoms_alloc = 0;
  int ncell_alloc = 0;
  int64_t capacity = 0;
  int64_t part_rows = 0;
  // Per-pair arrays at the width of the FP32 passes (FP32 x^k, V^k, dV,
  // 32-pair tiles of per-atom partials) or of the tensor-core passes only
  // (FP16 pairs: half the words, 128-pair tiles): want_fp32 is set for good
  // by the first call that may run the FP32 passes, pb_fp32 says what is
  // allocated, and fp32_bad records an FP32 launch refused on narrow arrays.
  bool want_fp32 = false;
  bool pb_fp32 = false;
  bool fp32_bad = false;
  NeighborBuffers nb{};
  GridInfo grid{};
  PassBufs pb{};
  TrainBatch bt{};
  double* d_pos = nullptr;     // N x 3 input positions (device copy)
  int* d_species = nullptr;
  float* d_F = nullptr;
  double* d_Ei = nullptr;
  double* d_blk = nullptr;
  double* d_stats = nullptr;
  unsigned long long* d_blku = nullptr;
  long long* d_count = nullptr;
  int n_atoms = 0;
  // MD state
  bool md_ready = false;
  int md_precision = ALLEGRO_FP32;
  double* d_v = nullptr;
  double* d_blk_ke = nullptr;
  long long* d_step = nullptr;
  long long* d_out_rec = nullptr;
  double* d_e_rec = nullptr;
  int rec_cap = 0;
  long long step = 0;
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  int64_t graph_kernels = 0;
  // Nose-Hoover NVT: thermostat state (xi, eta, K, s) and its own step graph
  double* d_nh = nullptr;
  double* d_nh_snap = nullptr;
  cudaGraphExec_t graph_nvt = nullptr;
  double nvt_key[3] = {0.0, 0.0, 0.0};   // dt, T, tau of graph_nvt
  // ring-polymer MD: P replicas of rp_n atoms in one box (bead-major
  // positions, velocities and forces, own arrays so that other calls leave
  // the ring state intact), the normal-mode matrix and frequencies, species
  // per replica and tiled over all replicas, and the ring's step graph
  int rp_P = 0;
  int64_t rp_n = 0;
  double rp_T = 0.0;
  double rp_L[3] = {0.0, 0.0, 0.0};
  GridInfo rp_grid{};
  bool rp_ready = false;
  double* d_rp_q = nullptr;
  double* d_rp_v = nullptr;
  float* d_rp_F = nullptr;
  double* d_rp_q_snap = nullptr;
  double* d_rp_v_snap = nullptr;
  float* d_rp_F_snap = nullptr;
  int* d_rp_species = nullptr;
  int* d_rp_species_all = nullptr;
  double* d_rp_C = nullptr;
  double* d_rp_w = nullptr;
  double* d_rp_blk = nullptr;
  cudaGraphExec_t graph_rp = nullptr;
  double rp_graph_dt = 0.0;
  int64_t rp_graph_kernels = 0;
  // Verlet skin of the MD state (NVE, NVT): skin requested, skin of the
  // current MD state's list (set by allegro_md_init), reference positions and
  // their wrap at the last build, and [rebuild now, forced rebuild, rebuilds]
  double skin = 0.0;
  double md_skin = 0.0;
  double* d_pos_ref = nullptr;
  double* d_wpos_ref = nullptr;
  int* d_skin_flag = nullptr;
  // rollback snapshot
  double* d_pos_snap = nullptr;
  double* d_v_snap = nullptr;
  float* d_F_snap = nullptr;

  int fail(int code, const std::string& m) {
    err = m;
    g_err = m;
    return code;
  }
  template <class T>
  T* dalloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    allocs.push_back(p);
    return (T*)p;
  }
  void dfree(void* p) {
    if (!p) return;
    for (auto& a : allocs)
      if (a == p) { cudaFree(p); a = nullptr; }
  }
  // the captured step graphs bake in buffers, weights and precision: every
  // change of those drops them (they are re-captured at the next MD call)
  void drop_graphs() {
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_nvt) cudaGraphExecDestroy(graph_nvt);
    if (graph_rp) cudaGraphExecDestroy(graph_rp);
    graph = nullptr;
    graph_nvt = nullptr;
    graph_rp = nullptr;
  }
  ~allegro_ctx() {
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_nvt) cudaGraphExecDestroy(graph_nvt);
    if (graph_rp) cudaGraphExecDestroy(graph_rp);
    for (void* p : allocs)
      if (p) cudaFree(p);
  }
};

namespace {

int cuda_check(allegro_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return c->fail(ALLEGRO_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  if (c->fp32_bad) {
    c->fp32_bad = false;
    return c->fail(ALLEGRO_E_CUDA, std::string(where) + ": internal error, FP32 passes on tensor-core-width buffers");
  }
  return ALLEGRO_OK;
}

// Convert blob tensors into pre-scaled FP32 [in][out] and [out][in] copies.
int upload_weights(allegro_ctx* c) {
  const Blob& B = c->blob;
  std::vector<float> host;
  size_t flat = 0;
  c->winfo.clear();
  auto push = [&](const Tensor* T, double extra, Lin* lin, const float** raw_n) -> bool {
    if (!T) return false;
    const double s = extra / std::sqrt((double)T->cols);
    while (host.size() % 4) host.push_back(0.f);
    const size_t t_off = host.size();
    for (uint32_t i = 0; i < T->cols; ++i)
      for (uint32_t o = 0; o < T->rows; ++o) host.push_back((float)(T->data[o * T->cols + i] * s));
    while (host.size() % 4) host.push_back(0.f);
    const size_t n_off = host.size();
    for (uint32_t o = 0; o < T->rows; ++o)
      for (uint32_t i = 0; i < T->cols; ++i) host.push_back((float)(T->data[o * T->cols + i] * s));
    if (lin) {
      lin->t = reinterpret_cast<const float*>(t_off);
      lin->n = reinterpret_cast<const float*>(n_off);
    }
    if (raw_n) *raw_n = reinterpret_cast<const float*>(n_off);
    c->winfo.push_back(WInfo{T->name, (int)T->rows, (int)T->cols, flat, (float)s, t_off, n_off, true});
    flat += (size_t)T->rows * T->cols;
    return true;
  };
  // Full O(3): mixing block b of layer k as a [C][C P_u] matrix over the
  // paths of all input irreps (the kernels' tables), the blob's columns (the
  // paths of the irreps the layer receives) scattered into it, the rest zero.
  // A block that no path of the layer reaches has no blob tensor: all zero.
  auto push_mix_o3 = [&](uint32_t k, int b, const float** raw_n) -> bool {
    const int lm = (int)B.lmax, C = (int)B.C;
    const std::vector<O3Path> all = o3_paths(lm, b, (1u << (2 * (lm + 1))) - 1u);
    const std::vector<O3Path> mine = o3_paths(lm, b, o3_layer_inputs(lm, (int)k));
    const int pu = (int)all.size(), pl = (int)mine.size();
    while (host.size() % 4) host.push_back(0.f);
    const size_t n_off = host.size();
    host.resize(host.size() + (size_t)C * C * pu, 0.f);
    *raw_n = reinterpret_cast<const float*>(n_off);
    const std::string name = "layer" + std::to_string(k) + ".mix" + std::to_string(b % (lm + 1)) +
                             (b > lm ? "p" : "");
    const Tensor* T = B.find(name);
    if (pl == 0) return T == nullptr;
    if (!T || T->rows != (uint32_t)C || T->cols != (uint32_t)(C * pl)) return false;
    std::vector<int> q_of(pl);
    for (int q = 0, u = 0; q < pl; ++q) {
      while (all[u].s1 != mine[q].s1 || all[u].l1 != mine[q].l1 || all[u].l2 != mine[q].l2) ++u;
      q_of[q] = u;
    }
    const double sc = 1.0 / std::sqrt((double)T->cols);
    for (int o = 0; o < C; ++o)
      for (int ci = 0; ci < C; ++ci)
        for (int q = 0; q < pl; ++q)
          host[n_off + (size_t)o * C * pu + ci * pu + q_of[q]] = (float)(T->data[(size_t)o * T->cols + ci * pl + q] * sc);
    WInfo wi{T->name, (int)T->rows, (int)T->cols, flat, (float)sc, n_off, n_off, false};
    wi.mix_pl = pl;
    wi.mix_pu = pu;
    wi.mix_q = q_of;
    c->winfo.push_back(wi);
    flat += (size_t)T->rows * T->cols;
    return true;
  };
  ModelW& w = c->w;
  bool ok = push(B.find("twobody.0"), 1.0, &w.tb0, nullptr) && push(B.find("twobody.1"), 1.0, &w.tb1, nullptr) &&
            push(B.find("embed"), 1.0, &w.emb, nullptr);
  const int nblk = w.o3 ? 2 * ((int)B.lmax + 1) : (int)B.lmax + 1;
  for (uint32_t k = 1; ok && k <= B.L; ++k) {
    const std::string pre = "layer" + std::to_string(k) + ".";
    LayerW& LW = w.layer[k - 1];
    ok = ok && push(B.find(pre + "env"), 1.0 / std::sqrt(B.nu), &LW.env, nullptr);
    if (k < B.L && w.o3)
      for (int b = 0; ok && b < nblk; ++b) ok = ok && push_mix_o3(k, b, &LW.mix[b]);
    else if (k < B.L)
      for (uint32_t l = 0; ok && l <= B.lmax; ++l)
        ok = ok && push(B.find(pre + "mix" + std::to_string(l)), 1.0, nullptr, &LW.mix[l]);
    ok = ok && push(B.find(pre + "latent.0"), 1.0, &LW.lat0, nullptr) &&
         push(B.find(pre + "latent.1"), 1.0, &LW.lat1, nullptr);
  }
  const float* eout = nullptr;
  ok = ok && push(B.find("energy.0"), 1.0, &w.e0, nullptr) && push(B.find("energy.out"), 1.0, nullptr, &eout);
  if (!ok) return c->fail(ALLEGRO_E_BLOB, "weights blob lacks a tensor of the model");
  c->d_w = c->dalloc<float>(host.size());
  if (!c->d_w) return c->fail(ALLEGRO_E_OOM, "weights allocation failed");
  if (cudaMemcpy(c->d_w, host.data(), host.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_check(c, "weights upload");
  auto fix = [&](const float*& p) { if (p || true) p = c->d_w + reinterpret_cast<size_t>(p); };
  auto fixl = [&](Lin& l) { fix(l.t); fix(l.n); };
  fixl(w.tb0); fixl(w.tb1); fixl(w.emb); fixl(w.e0);
  for (uint32_t k = 1; k <= B.L; ++k) {
    LayerW& LW = w.layer[k - 1];
    fixl(LW.env); fixl(LW.lat0); fixl(LW.lat1);
    if (k < B.L)
      for (int b = 0; b < nblk; ++b) fix(LW.mix[b]);
  }
  w.eout = c->d_w + reinterpret_cast<size_t>(eout);
  c->n_params = (int64_t)flat;
  for (int s = 0; s < 2; ++s) {
    w.sigma[s] = (float)B.sigma[s];
    w.mu[s] = (float)B.mu[s];
  }
  w.rc = (float)B.rc;
  w.n_layers = (int)B.L;
  return ALLEGRO_OK;
}

uint16_t f2h(float f) { return __half_as_ushort(__float2half_rn(f)); }

uint16_t f2bf(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even (finite inputs)
  return (uint16_t)(u >> 16);
}

float bf2f(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// BF16 (or FP16) tensor-core images (layout of umma.cuh) of every linear
// layer of the main model, pre-scaled like the FP32 copies.
// Swizzled weight images of one tensor-core mode.  Split mode: FP16 images
// plus the lo parts rn(w - rn(w)) of twobody.1 and energy.0, and twobody.0
// packed as [hi | hi | lo] in columns 0, 16 and 32.
int upload_weights_bf16(allegro_ctx* c, TcMode mode) {
  const Blob& B = c->blob;
  const bool fp16 = mode != TcMode::kBf16;
  const bool split = mode == TcMode::kFp16Split;
  std::vector<uint8_t> img;
  auto cvt = [&](float x) { return fp16 ? f2h(x) : f2bf(x); };
  auto back = [&](uint16_t h) { return fp16 ? __half2float(__ushort_as_half(h)) : bf2f(h); };
  // part 0: rn(x); part 1: rn(x - rn(x)); copies at column offsets col_off
  auto add_parts = [&](const Tensor* T, double extra, int Rimg, int Kimg, std::initializer_list<int> parts,
                       std::initializer_list<int> col_off) -> size_t {
    const size_t base = (img.size() + 1023) / 1024 * 1024;
    img.resize(base + al::umma::sw128_bytes(Rimg, Kimg), 0);
    const double s = extra / std::sqrt((double)T->cols);
    for (uint32_t r = 0; r < T->rows; ++r)
      for (uint32_t k = 0; k < T->cols; ++k) {
        const float x = (float)(T->data[r * T->cols + k] * s);
        const uint16_t hi = cvt(x);
        const uint16_t lo = cvt(x - back(hi));
        auto po = parts.begin();
        for (int off : col_off) {
          const uint16_t h = *po++ == 0 ? hi : lo;
          std::memcpy(img.data() + base + al::umma::sw128_off((int)r, (int)k + off, Rimg), &h, 2);
        }
      }
    return base;
  };
  auto add = [&](const Tensor* T, double extra, int Rimg, int Kimg) {
    return add_parts(T, extra, Rimg, Kimg, {0}, {0});
  };
  size_t o_tb0 = split ? add_parts(B.find("twobody.0"), 1.0, 128, 64, {0, 0, 1}, {0, 16, 32})
                       : add(B.find("twobody.0"), 1.0, 128, 64);
  size_t o_tb1 = add(B.find("twobody.1"), 1.0, 128, 128);
  size_t o_emb = add(B.find("embed"), 1.0, (int)(B.C * (B.lmax + 1)), 128);
  size_t o_e0 = add(B.find("energy.0"), 1.0, 32, 128);
  size_t o_tb1_lo = 0, o_e0_lo = 0;
  if (split) {
    o_tb1_lo = add_parts(B.find("twobody.1"), 1.0, 128, 128, {1}, {0});
    o_e0_lo = add_parts(B.find("energy.0"), 1.0, 32, 128, {1}, {0});
  }
  size_t o_env[kMaxLayers], o_l0[kMaxLayers], o_l1[kMaxLayers], o_mix[kMaxLayers][3];
  for (uint32_t k = 1; k <= B.L; ++k) {
    const std::string pre = "layer" + std::to_string(k) + ".";
    o_env[k - 1] = add(B.find(pre + "env"), 1.0 / std::sqrt(B.nu), 16, 128);
    o_l0[k - 1] = add(B.find(pre + "latent.0"), 1.0, 128, 192);
    o_l1[k - 1] = add(B.find(pre + "latent.1"), 1.0, 128, 128);
    if (k < B.L)
      for (uint32_t l = 0; l <= B.lmax; ++l) o_mix[k - 1][l] = add(B.find(pre + "mix" + std::to_string(l)), 1.0, 16, 64);
  }
  uint8_t* dev = c->dalloc<uint8_t>(img.size());
  if (!dev) return c->fail(ALLEGRO_E_OOM, "tensor-core weights allocation failed");
  if (cudaMemcpy(dev, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_check(c, "tensor-core weights upload");
  (split ? c->d_sw : fp16 ? c->d_hw : c->d_bw) = dev;
  BfW& w = split ? c->sw : fp16 ? c->hw : c->bw;
  w.tb0 = dev + o_tb0;
  w.tb1 = dev + o_tb1;
  w.emb = dev + o_emb;
  w.e0 = dev + o_e0;
  w.tb1_lo = split ? dev + o_tb1_lo : nullptr;
  w.e0_lo = split ? dev + o_e0_lo : nullptr;
  for (uint32_t k = 1; k <= B.L; ++k) {
    w.env[k - 1] = dev + o_env[k - 1];
    w.lat0[k - 1] = dev + o_l0[k - 1];
    w.lat1[k - 1] = dev + o_l1[k - 1];
    if (k < B.L)
      for (uint32_t l = 0; l <= B.lmax; ++l) w.mix[k - 1][l] = dev + o_mix[k - 1][l];
  }
  w.eout = c->w.eout;
  for (int s = 0; s < 2; ++s) w.sigma[s] = (float)B.sigma[s];
  w.rc = (float)B.rc;
  w.n_layers = (int)B.L;
  w.lmax = (int)B.lmax;
  return ALLEGRO_OK;
}

int check_cell(allegro_ctx* c, const double* cell, double L[3]) {
  if (!cell) return c->fail(ALLEGRO_E_INVALID_ARG, "cell is NULL");
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (a != b && cell[3 * a + b] != 0.0) return c->fail(ALLEGRO_E_NONORTHO_CELL, "only orthorhombic cells are supported");
  for (int a = 0; a < 3; ++a) {
    L[a] = cell[4 * a];
    if (!(L[a] > 0.0) || !std::isfinite(L[a])) return c->fail(ALLEGRO_E_NONORTHO_CELL, "cell lengths must be positive");
    if (c->blob.rc > 2.0 * L[a]) return c->fail(ALLEGRO_E_CUTOFF_TOO_LARGE, "r_cut exceeds twice the cell length");
  }
  return ALLEGRO_OK;
}

int ensure_atoms(allegro_ctx* c, int64_t n, int ncell) {
  if (n > c->n_atoms_alloc) {
    const int64_t na = std::max<int64_t>(n, c->n_atoms_alloc * 5 / 4);
    for (void* p : {(void*)c->d_pos, (void*)c->d_species, (void*)c->d_F, (void*)c->d_Ei, (void*)c->d_blk,
                    (void*)c->d_blku, (void*)c->nb.wpos, (void*)c->nb.wpos32, (void*)c->nb.atom_cell,
                    (void*)c->nb.cell_atoms, (void*)c->nb.row_cnt, (void*)c->nb.row_ptr, (void*)c->nb.scan_blocks,
                    (void*)c->d_v, (void*)c->d_blk_ke, (void*)c->d_pos_snap, (void*)c->d_v_snap,
                    (void*)c->d_F_snap, (void*)c->d_pos_ref, (void*)c->d_wpos_ref})
      c->dfree(p);
    c->d_pos = c->dalloc<double>(3 * na);
    c->d_species = c->dalloc<int>(na);
    c->d_F = c->dalloc<float>(3 * na);
    c->d_Ei = c->dalloc<double>(na);
    c->d_blk = c->dalloc<double>(2 * (na / 256 + 2));
    c->d_blku = c->dalloc<unsigned long long>(na / 256 + 2);
    c->nb.wpos = c->dalloc<double>(3 * na);
    c->nb.wpos32 = c->dalloc<float>(3 * na);
    c->nb.atom_cell = c->dalloc<int>(na);
    c->nb.cell_atoms = c->dalloc<int>(na);
    c->nb.row_cnt = c->dalloc<int>(na + 1);
    c->nb.row_ptr = c->dalloc<int>(na + 1);
    c->nb.scan_blocks = c->dalloc<int>((std::max<int64_t>(na, 1 << 22) + 1) / 1024 + 4);
    c->d_v = c->dalloc<double>(3 * na);
    c->d_blk_ke = c->dalloc<double>(na / 256 + 2);
    c->d_pos_snap = c->dalloc<double>(3 * na);
    c->d_v_snap = c->dalloc<double>(3 * na);
    c->d_F_snap = c->dalloc<float>(3 * na);
    c->d_pos_ref = c->dalloc<double>(3 * na);
    c->d_wpos_ref = c->dalloc<double>(3 * na);
    if (!c->d_pos || !c->d_species || !c->d_F || !c->d_Ei || !c->d_blk || !c->d_blku || !c->nb.wpos ||
        !c->nb.wpos32 || !c->nb.atom_cell || !c->nb.cell_atoms || !c->nb.row_cnt || !c->nb.row_ptr ||
        !c->nb.scan_blocks || !c->d_v || !c->d_blk_ke || !c->d_pos_snap || !c->d_v_snap || !c->d_F_snap ||
        !c->d_pos_ref || !c->d_wpos_ref)
      return c->fail(ALLEGRO_E_OOM, "per-atom allocation failed");
    c->n_atoms_alloc = na;
    c->part_rows = 0;   // partial buffers depend on N
    c->drop_graphs();   // the step graphs hold the old per-atom buffers
  }
  if (!c->d_stats) {
    c->d_stats = c->dalloc<double>(8);
    c->d_count = c->dalloc<long long>(2);
    c->nb.n_pairs = c->dalloc<int>(1);
    c->nb.flags = c->dalloc<int>(1);
    c->d_step = c->dalloc<long long>(1);
    c->d_skin_flag = c->dalloc<int>(4);
    c->d_nh = c->dalloc<double>(4);
    c->d_nh_snap = c->dalloc<double>(4);
    if (!c->d_stats || !c->d_count || !c->nb.n_pairs || !c->nb.flags || !c->d_step || !c->d_nh || !c->d_nh_snap)
      return c->fail(ALLEGRO_E_OOM, "allocation failed");
    cudaMemset(c->nb.flags, 0, sizeof(int));
  }
  if (ncell + 1 > c->ncell_alloc) {
    c->dfree(c->nb.cell_count);
    c->dfree(c->nb.cell_start);
    c->nb.cell_count = c->dalloc<int>(ncell + 2);
    c->nb.cell_start = c->dalloc<int>(ncell + 2);
    if (!c->nb.cell_count || !c->nb.cell_start) return c->fail(ALLEGRO_E_OOM, "cell allocation failed");
    c->ncell_alloc = ncell + 2;
    c->drop_graphs();
  }
  return ALLEGRO_OK;
}

int ensure_pairs(allegro_ctx* c, int64_t cap) {
  const Blob& B = c->blob;
  const int NLM = (B.lmax + 1) * (B.lmax + 1);
  const int CL = B.C * NLM;
  const int CV = c->w.o3 ? 2 * CL : CL;   // V^k per pair (full O(3): both parities)
  const bool full = c->want_fp32 || !c->bf16_ok;
  const int tile = full ? fp32_tile(c->w.o3) : bf16_tile();
  const int64_t rows_needed = cap / tile + 2 + c->n_atoms_alloc;
  if (cap <= c->capacity && rows_needed <= c->part_rows && (c->pb_fp32 || !full)) return ALLEGRO_OK;
  if (cap > (int64_t)0x7fffffff - 1024) return c->fail(ALLEGRO_E_UNSUPPORTED, "more than 2^31 pairs");
  PassBufs& pb = c->pb;
  for (void* p : {(void*)c->nb.pi, (void*)c->nb.pj, (void*)c->nb.pcode, (void*)c->nb.rev, (void*)c->nb.keys,
                  (void*)c->nb.skeys, (void*)pb.dX, (void*)pb.dV, (void*)pb.dU, (void*)pb.dY, (void*)pb.G,
                  (void*)pb.epart})
    c->dfree(p);
  for (int k = 0; k < kMaxLayers; ++k) {
    c->dfree(pb.X[k]);
    c->dfree(pb.V[k]);
    pb.X[k] = pb.V[k] = nullptr;
  }
  for (int k = 0; k <= kMaxLayers; ++k) {
    c->dfree(pb.gam[k]);
    c->dfree(pb.dgam[k]);
    c->dfree(pb.gsum[k]);
    c->dfree(pb.dgsum[k]);
    pb.gam[k] = pb.dgam[k] = pb.gsum[k] = pb.dgsum[k] = nullptr;
  }
  // per-pair arrays of the tensor-core path are tile-SoA over 128-pair tiles;
  // every per-pair array holds whole tiles (the passes prefetch the next
  // tile's slices into L2)
  const int64_t capr = (cap + 127) / 128 * 128;
  c->nb.pi = c->dalloc<int>(capr);
  c->nb.pj = c->dalloc<int>(capr);
  c->nb.pcode = c->dalloc<int>(capr);
  c->nb.rev = c->dalloc<int>(capr);
  c->nb.keys = c->dalloc<unsigned long long>(capr);
  c->nb.skeys = c->dalloc<unsigned long long>(capr);
  bool ok = c->nb.pi && c->nb.pj && c->nb.pcode && c->nb.rev && c->nb.keys && c->nb.skeys;
  // x^k, V^k and dV: FP32 rows for the FP32 passes, FP16 (or 16-bit operand)
  // pairs, half the words, for the tensor-core passes
  const size_t xw = full ? (size_t)c->D : (size_t)c->D / 2;
  const size_t vw = full ? (size_t)CV : (size_t)CL / 2;
  for (uint32_t k = 0; k < B.L && ok; ++k) {
    pb.X[k] = c->dalloc<float>((size_t)capr * xw);
    ok = ok && pb.X[k];
    if (k >= 1) {
      pb.V[k] = c->dalloc<float>((size_t)capr * vw);
      ok = ok && pb.V[k];
    }
  }
  pb.dX = c->dalloc<float>((size_t)capr * c->D);
  pb.dV = c->dalloc<float>((size_t)capr * vw);
  pb.dU = c->dalloc<float>(capr);
  pb.dY = c->dalloc<float>((size_t)capr * NLM);
  pb.G = c->dalloc<float>((size_t)capr * 3);
  for (int k = 0; k < kMaxLayers; ++k) {
    c->dfree(pb.S[k]);
    pb.S[k] = nullptr;
  }
  c->dfree(pb.dR);
  pb.dR = nullptr;
  for (int k = 0; k <= kMaxLayers; ++k) {
    c->dfree(pb.Ek[k]);
    pb.Ek[k] = nullptr;
  }
  if (c->bf16_ok) {
    for (uint32_t k = 1; k <= B.L && ok; ++k) {       // env outputs, FP32
      pb.Ek[k] = c->dalloc<float>((size_t)capr * B.C);
      ok = ok && pb.Ek[k];
    }
    const int NSC = B.C * (B.lmax + 1);               // layer scalars (P_0 = l_max + 1 per channel), FP16 pairs
    for (uint32_t k = 1; k < B.L && ok; ++k) {
      pb.S[k] = c->dalloc<float>((size_t)capr * (NSC / 2));
      ok = ok && pb.S[k];
    }
    pb.dR = c->dalloc<float>((size_t)capr * 3);
    ok = ok && pb.dR;
  }
  const int64_t rows = rows_needed;
  pb.epart = c->dalloc<double>(rows);
  ok = ok && pb.dX && pb.dV && pb.dU && pb.dY && pb.G && pb.epart;
  for (uint32_t k = 1; k <= B.L && ok; ++k) {
    pb.gam[k] = c->dalloc<float>((size_t)rows * CL);
    pb.dgam[k] = c->dalloc<float>((size_t)rows * CL);
    ok = ok && pb.gam[k] && pb.dgam[k];
    if (c->bf16_ok && ok) {
      pb.gsum[k] = c->dalloc<float>((size_t)std::max<int64_t>(c->n_atoms_alloc, 1) * CL);
      pb.dgsum[k] = c->dalloc<float>((size_t)std::max<int64_t>(c->n_atoms_alloc, 1) * CL);
      ok = pb.gsum[k] && pb.dgsum[k];
    }
  }
  if (!ok) {
    c->capacity = 0;
    return c->fail(ALLEGRO_E_OOM, "pair buffers allocation failed (capacity " + std::to_string(cap) + ")");
  }
  c->capacity = cap;
  c->nb.capacity = cap;
  c->part_rows = rows;
  c->pb_fp32 = full;
  c->drop_graphs();
  return ALLEGRO_OK;
}

// Called by every entry point that may run the FP32 passes, before it
// allocates: from now on the per-pair arrays are allocated at FP32 width
// (reallocated now if they exist at tensor-core width).
int require_fp32(allegro_ctx* c) {
  c->want_fp32 = true;
  if (c->capacity > 0 && !c->pb_fp32) return ensure_pairs(c, c->capacity);
  return ALLEGRO_OK;
}

void fill_passbufs(allegro_ctx* c, const double L[3]) {
  PassBufs& pb = c->pb;
  pb.pi = c->nb.pi;
  pb.pj = c->nb.pj;
  pb.pcode = c->nb.pcode;
  pb.row_ptr = c->nb.row_ptr;
  pb.n_pairs = c->nb.n_pairs;
  pb.flags = c->nb.flags;
  pb.capacity = c->capacity;
  pb.wpos = c->nb.wpos;
  pb.species = c->d_species;
  pb.n_atoms = c->n_atoms;
  for (int a = 0; a < 3; ++a) pb.L[a] = L[a];
  pb.atomL = nullptr;
  pb.tile = fp32_tile(c->w.o3);
}

AtomArgs atom_args(allegro_ctx* c) {
  AtomArgs a;
  a.n = c->n_atoms;
  a.species = c->d_species;
  for (int s = 0; s < 2; ++s) {
    a.sigma[s] = c->blob.sigma[s];
    a.mu[s] = c->blob.mu[s];
    a.mass[s] = c->mass[s];
  }
  return a;
}

__global__ void k_check_species(int n, const int* __restrict__ sp, int S, int* __restrict__ flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (sp[i] < 0 || sp[i] >= S)) atomicOr(flags, kFlagBadSpecies);
}

// Neighbour build into the current capacity; grows and rebuilds once on
// overflow.  Leaves n_pairs on the host in *np_host.
int build_with_growth(allegro_ctx* c, const double* d_positions, int64_t n, int64_t* np_host) {
  for (int attempt = 0; attempt < 3; ++attempt) {
    launch_build_neighbors(c->nb, c->grid, d_positions, (int)n, c->stream);
    int np = 0, flags = 0;
    cudaMemcpyAsync(&np, c->nb.n_pairs, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&flags, c->nb.flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "neighbour build");
    if (flags & kFlagNonfinite) return c->fail(ALLEGRO_E_NONFINITE, "non-finite position");
    if (flags & kFlagBadSpecies) return c->fail(ALLEGRO_E_INVALID_ARG, "species id out of range");
    if (!(flags & kFlagPairOverflow)) {
      *np_host = np;
      return ALLEGRO_OK;
    }
    const int rc = ensure_pairs(c, (int64_t)np + np / 4 + 1024);
    if (rc) return rc;
    // every other bit returned above, so clearing the word on the library
    // stream orders the clear before the rebuild's atomicOr
    cudaMemsetAsync(c->nb.flags, 0, sizeof(int), c->stream);
  }
  return c->fail(ALLEGRO_E_PAIR_OVERFLOW, "pair capacity could not be grown");
}

// skin > 0 (MD with Verlet-skin reuse): the list holds every pair within
// r_cut + skin.
int prepare(allegro_ctx* c, int64_t n, const double* positions, const int32_t* species,
            const double* cell, double L[3], double skin = 0.0) {
  if (n <= 0 || n > (1 << 30)) return c->fail(ALLEGRO_E_INVALID_ARG, "n_atoms out of range");
  if (!positions) return c->fail(ALLEGRO_E_INVALID_ARG, "positions is NULL");
  int rc = check_cell(c, cell, L);
  if (rc) return rc;
  for (int a = 0; a < 3; ++a)
    if (c->blob.rc + skin > 2.0 * L[a])
      return c->fail(ALLEGRO_E_CUTOFF_TOO_LARGE, "r_cut + skin exceeds twice the cell length");
  c->md_ready = false;   // the per-atom buffers now hold this call's system
  c->grid = plan_grid(L, c->blob.rc + skin);
  const int ncell = c->grid.ncell[0] > 0 ? c->grid.ncell[0] * c->grid.ncell[1] * c->grid.ncell[2] : 0;
  rc = ensure_atoms(c, n, ncell);
  if (rc) return rc;
  c->n_atoms = (int)n;
  cudaMemsetAsync(c->nb.flags, 0, sizeof(int), c->stream);
  const cudaMemcpyKind kp = is_device_ptr(positions) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyAsync(c->d_pos, positions, sizeof(double) * 3 * n, kp, c->stream);
  if (species) {
    const cudaMemcpyKind ks = is_device_ptr(species) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaMemcpyAsync(c->d_species, species, sizeof(int) * n, ks, c->stream);
    k_check_species<<<(int)((n + 255) / 256), 256, 0, c->stream>>>((int)n, c->d_species, (int)c->blob.S,
                                                                   c->nb.flags);
  }
  if (c->capacity == 0) {
    const double vol = L[0] * L[1] * L[2];
    const double rc3 = c->blob.rc * c->blob.rc * c->blob.rc;
    const double est = (double)n * (4.18879 * rc3 * (double)n / vol) * 1.3 + 4096.0;
    rc = ensure_pairs(c, (int64_t)std::min(est, 2.0e9));
    if (rc) return rc;
  } else {
    rc = ensure_pairs(c, c->capacity);               // partial rows follow N (no-op when nothing changed)
    if (rc) return rc;
  }
  return cuda_check(c, "prepare");
}

bool valid_precision(int32_t p) {
  return p == ALLEGRO_FP32 || p == ALLEGRO_BF16 || p == ALLEGRO_FP16 || p == ALLEGRO_FP16_SPLIT;
}

// Launch-shape autotuner of the FP32 pass kernels (value passes: which = 0,
// tangent passes: which = 1).  run(ls, km) enqueues one whole pass sequence
// with launch shape ls and phase marks km.  For each candidate (1, 2, 4 or 8
// waves of one block per SM for every pass) the sequence runs twice; each
// pass takes the candidate of its shortest measured time.  The passes write
// the same bits for every launch shape (every tile's work is fixed), so the
// tuning runs leave the sequence's outputs as one run would; tuned again when
// the pair capacity has grown past twice the tuned one.  Not called while a
// stream is being captured (it synchronises).
template <class Run>
int autotune_fp32(allegro_ctx* c, int which, Run&& run) {
  if (c->fl_cap[which] > 0 && c->capacity <= 2 * c->fl_cap[which]) return ALLEGRO_OK;
  static const int kCand[4] = {1, 2, 4, 8};
  KernelMarks km;
  for (auto& e : km.ev) cudaEventCreate(&e);
  double best[kPhCount];
  int pick[kPhCount];
  for (int k = 0; k < kPhCount; ++k) {
    best[k] = 1e30;
    pick[k] = 8;
  }
  int rc = ALLEGRO_OK;
  for (int rep = 0; rep < 2 && !rc; ++rep)
    for (int ci = 0; ci < 4 && !rc; ++ci) {
      Fp32Launch ls;
      for (int k = 0; k < kPhCount; ++k) ls.waves[k] = kCand[ci];
      km.n = 0;
      run(&ls, &km);
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        rc = cuda_check(c, "launch-shape tuning");
        break;
      }
      double ms_k[kPhCount] = {};
      for (int i = 0; i + 1 < km.n; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, km.ev[i], km.ev[i + 1]);
        const int kd = km.kind[i + 1];
        if (kd >= 0 && kd < kPhCount) ms_k[kd] += ms;
      }
      for (int k = 0; k < kPhCount; ++k)
        if (ms_k[k] > 0.0 && ms_k[k] < best[k]) {
          best[k] = ms_k[k];
          pick[k] = kCand[ci];
        }
    }
  for (auto& e : km.ev) cudaEventDestroy(e);
  if (rc) return rc;
  for (int k = 0; k < kPhCount; ++k) c->fl[which].waves[k] = pick[k];
  c->fl_cap[which] = std::max<int64_t>(c->capacity, 1);
  return ALLEGRO_OK;
}

// Pair passes of the requested precision followed by force assembly.
void launch_model(allegro_ctx* c, int32_t precision, cudaStream_t s, KernelMarks* km) {
  const Blob& B = c->blob;
  int tile;
  if (precision == ALLEGRO_BF16) {
    bf16_energy_forces(c->bw, c->pb, c->capacity, s, km, TcMode::kBf16);
    tile = bf16_tile();
  } else if (precision == ALLEGRO_FP16) {
    bf16_energy_forces(c->hw, c->pb, c->capacity, s, km, TcMode::kFp16);
    tile = bf16_tile();
  } else if (precision == ALLEGRO_FP16_SPLIT) {
    bf16_energy_forces(c->sw, c->pb, c->capacity, s, km, TcMode::kFp16Split);
    tile = bf16_tile();
  } else {
    if (c->pb_fp32) fp32_energy_forces((int)B.lmax, (int)B.C, c->D, c->E, c->w, c->pb, c->capacity, s, km, &c->fl[0]);
    else c->fp32_bad = true;
    tile = fp32_tile(c->w.o3);
  }
  launch_forces(atom_args(c), c->nb.row_ptr, c->nb.rev, c->pb.G, c->pb.epart, tile, c->d_F, c->d_Ei, c->d_blk,
                c->d_stats, c->nb.flags, s);
}

int refresh_tc(allegro_ctx* c);

int run_model(allegro_ctx* c, int32_t precision, const double L[3]) {
  if (!valid_precision(precision))
    return c->fail(ALLEGRO_E_INVALID_ARG,
                   "precision must be ALLEGRO_FP32, ALLEGRO_BF16, ALLEGRO_FP16 or ALLEGRO_FP16_SPLIT");
  if (precision != ALLEGRO_FP32 && !c->bf16_ok)
    return c->fail(ALLEGRO_E_UNSUPPORTED, "the tensor-core path is built for the 16-channel, latent-128 model with 2+ layers and l_max <= 2 (natural parity, or full O(3) with two layers) only");
  if (precision != ALLEGRO_FP32) {
    const int rc = refresh_tc(c);
    if (rc) return rc;
  }
  fill_passbufs(c, L);
  if (precision == ALLEGRO_FP32 && c->pb_fp32) {
    const Blob& B = c->blob;
    const int rc = autotune_fp32(c, 0, [&](const Fp32Launch* ls, KernelMarks* km) {
      fp32_energy_forces((int)B.lmax, (int)B.C, c->D, c->E, c->w, c->pb, c->capacity, c->stream, km, ls);
    });
    if (rc) return rc;
  }
  launch_model(c, precision, c->stream, nullptr);
  return cuda_check(c, "model launch");
}

int copy_out(allegro_ctx* c, void* dst, const void* src, size_t bytes) {
  if (!dst) return ALLEGRO_OK;
  const cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (cudaMemcpyAsync(dst, src, bytes, k, c->stream) != cudaSuccess) return cuda_check(c, "copy out");
  return ALLEGRO_OK;
}


// ---------------------------------------------------------------------------
// Training (SAM, Eq. 3): master weights, weight gradients, Adam.

int init_master(allegro_ctx* c) {
  if (c->d_master) return ALLEGRO_OK;
  const size_t n = (size_t)c->n_params;
  std::vector<float> h(n);
  size_t off = 0;
  for (const auto& wi : c->winfo) {
    const Tensor* T = c->blob.find(wi.name);
    for (size_t q = 0; q < (size_t)wi.rows * wi.cols; ++q) h[off + q] = (float)T->data[q];
    off += (size_t)wi.rows * wi.cols;
  }
  c->d_master = c->dalloc<float>(n);
  c->d_grad = c->dalloc<float>(n);
  c->d_adam_m = c->dalloc<float>(n);
  c->d_adam_v = c->dalloc<float>(n);
  c->d_wtmp = c->dalloc<float>(n);
  c->d_norm2 = c->dalloc<double>(1);
  if (!c->d_master || !c->d_grad || !c->d_adam_m || !c->d_adam_v || !c->d_wtmp || !c->d_norm2)
    return c->fail(ALLEGRO_E_OOM, "training buffers allocation failed");
  cudaMemcpy(c->d_master, h.data(), n * 4, cudaMemcpyHostToDevice);
  cudaMemset(c->d_adam_m, 0, n * 4);
  cudaMemset(c->d_adam_v, 0, n * 4);
  c->adam_t = 0;
  return cuda_check(c, "init master weights");
}

// FP32 pass weights <- flat vector (pre-scaled copies of every tensor)
void apply_flat(allegro_ctx* c, const float* flat) {
  for (const auto& wi : c->winfo) {
    if (wi.mix_pl > 0)
      launch_apply_mix(flat + wi.flat_off, wi.rows, wi.cols / wi.mix_pl, wi.mix_pl, wi.mix_pu, wi.mix_q.data(),
                       wi.scale, c->d_w + wi.n_off, c->stream);
    else
      launch_apply(flat + wi.flat_off, wi.rows, wi.cols, wi.scale, c->d_w + wi.t_off, c->d_w + wi.n_off, c->stream);
  }
  c->tc_dirty = true;
}

// Tensor-core images <- d_master (through the blob's FP64 tensor storage).
int refresh_tc(allegro_ctx* c) {
  if (!c->tc_dirty || !c->bf16_ok || !c->d_master) return ALLEGRO_OK;
  std::vector<float> h((size_t)c->n_params);
  if (cudaMemcpy(h.data(), c->d_master, h.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_check(c, "download weights");
  for (const auto& wi : c->winfo) {
    double* dst = const_cast<double*>(c->blob.find(wi.name)->data);
    for (size_t q = 0; q < (size_t)wi.rows * wi.cols; ++q) dst[q] = h[wi.flat_off + q];
  }
  c->dfree(c->d_bw);
  c->dfree(c->d_hw);
  c->dfree(c->d_sw);
  int rc = upload_weights_bf16(c, TcMode::kBf16);
  if (!rc) rc = upload_weights_bf16(c, TcMode::kFp16);
  if (!rc) rc = upload_weights_bf16(c, TcMode::kFp16Split);
  if (!rc) c->tc_dirty = false;
  return rc;
}

const WInfo* winfo(allegro_ctx* c, const std::string& name) {
  for (const auto& wi : c->winfo)
    if (wi.name == name) return &wi;
  return nullptr;
}

// tensor-product table sizes of the model's l_max (0, 1 or 2)
int tp_ns(int lmax) { return lmax == 0 ? TP0_NS : lmax == 1 ? TP1_NS : TP2_NS; }
int tp_nt(int lmax) { return lmax == 0 ? TP0_NT : lmax == 1 ? TP1_NT : TP2_NT; }
int tp_pl(int lmax, int l) { return lmax == 0 ? tp0_P(l) : lmax == 1 ? tp1_P(l) : tp2_P(l); }
int tp_toff(int lmax, int l) { return lmax == 0 ? tp0_toff(l) : lmax == 1 ? tp1_toff(l) : tp2_toff(l); }

int ensure_train(allegro_ctx* c) {
  const int64_t cap = c->capacity;
  const int64_t rows = cap / fp32_tangent_tile() + 2 + c->n_atoms_alloc;
  if (cap <= c->tr_cap && rows <= c->tr_rows) return ALLEGRO_OK;
  const Blob& B = c->blob;
  const int D = c->D, C = (int)B.C, E = c->E, L = (int)B.L;
  const int NS = tp_ns((int)B.lmax), NT = tp_nt((int)B.lmax);
  const int NW0 = C * ((int)B.lmax + 1);
  const int NLM = ((int)B.lmax + 1) * ((int)B.lmax + 1), CL = C * NLM;
  auto re = [&](float*& p, size_t n) {
    c->dfree(p);
    p = c->dalloc<float>(n);
    return p != nullptr;
  };
  bool ok = true;
  for (TrainBufs* t : {&c->tr, &c->trt}) {          // values and tangents of the dumps
    ok = ok && re(t->h0, cap * 16) && re(t->a1_tb, cap * D) && re(t->dz1_tb, cap * D) && re(t->dz2_tb, cap * D) &&
         re(t->dw0, cap * NW0) && re(t->xL, cap * D) && re(t->ae, cap * E) && re(t->dze, cap * E) &&
         re(t->dEij, cap);
    for (int j = 0; j < L && ok; ++j) ok = re(t->de[j], cap * C);
    for (int k = 1; k <= L && ok; ++k)
      ok = re(t->s[k], cap * C * NS) && re(t->a1_l[k], cap * D) && re(t->dz1_l[k], cap * D) &&
           re(t->dz2_l[k], cap * D) && (k == L || re(t->T[k], cap * C * NT));
  }
  // tangent passes: every array holds Dual values (two floats each)
  for (int k = 0; k < L && ok; ++k) ok = re(c->tX[k], 2 * cap * D) && (k == 0 || re(c->tV[k], 2 * cap * CL));
  ok = ok && re(c->tdX, 2 * cap * D) && re(c->tdV, 2 * cap * CL) && re(c->tdU, 2 * cap) &&
       re(c->tdY, 2 * cap * NLM) && re(c->tG, 2 * cap * 3);
  for (int k = 1; k <= L && ok; ++k) ok = re(c->tgam[k], 2 * rows * CL) && re(c->tdgam[k], 2 * rows * CL);
  if (ok) {
    c->dfree(c->tepart);
    c->tepart = c->dalloc<double>((size_t)rows);
    ok = c->tepart != nullptr;
  }
  ok = ok && (c->wpart || re(c->wpart, wgrad_part_floats()));
  if (!ok) {
    c->tr_cap = c->tr_rows = 0;
    return c->fail(ALLEGRO_E_OOM, "training buffer allocation failed");
  }
  c->tr_cap = cap;
  c->tr_rows = rows;
  return ALLEGRO_OK;
}

// Weight gradient of the last tangent pass sequence (P pairs), added into
// d_grad.  For every linear layer z = (W s) x the passes dumped the value and
// the tangent of its pre-activation gradient dz and of its input x (from
// per-pair Dual arrays: element stride 2, tangent at offset 1); with the
// tangent passes seeded by (-1, dL/dE_i) and directed along v = dL/dF,
//     tangent of s sum_p dz (x) x = s sum_p (dz.t (x) x.v + dz.v (x) x.t)
// is the loss gradient: the energy term sum_i dL/dE_i dE_i/dw plus the force
// term -d/dw (v . dE/dr).
int reduce_wgrad_tangent(allegro_ctx* c, int P) {
  const Blob& B = c->blob;
  const int D = c->D, C = (int)B.C, E = c->E, Lz = (int)B.L;
  const int NS = tp_ns((int)B.lmax), NT = tp_nt((int)B.lmax);
  const int NLM = ((int)B.lmax + 1) * ((int)B.lmax + 1), NW0 = C * ((int)B.lmax + 1), KH = D + C * NS;
  const TrainBufs& v = c->tr;
  const TrainBufs& t = c->trt;
  cudaStream_t s = c->stream;
  float* part = c->wpart;
  auto g = [&](const std::string& name) { return c->d_grad + winfo(c, name)->flat_off; };
  // a per-pair input: value and tangent views (plane arrays: stride 1;
  // Dual arrays: stride 2, tangent at offset 1)
  struct In {
    const float* v;
    const float* t;
    int es;
  };
  auto plane = [](const float* pv, const float* pt) { return In{pv, pt, 1}; };
  auto dual = [](const float* p) { return In{p, p + 1, 2}; };
  // both terms on the tensor cores (BF16 x 3 split operands, FP32 accumulation)
  auto wg = [&](const float* dzv, const float* dzt, int ldz, In x, int ldx, int N, int K, float scale, float* dW,
                int ldw, int k0) {
    if (wgrad_tc_supported(N, K)) {
      launch_wgrad_tc(dzt, dzv, ldz, x.v, x.t, ldx * x.es, x.es, P, N, K, scale, dW, ldw, k0, part, c->nb.flags, s);
    } else {
      launch_wgrad(dzt, ldz, 1, x.v, ldx * x.es, x.es, P, N, K, scale, dW, ldw, k0, part, s);
      launch_wgrad(dzv, ldz, 1, x.t, ldx * x.es, x.es, P, N, K, scale, dW, ldw, k0, part, s);
    }
  };
  const float isD = 1.0f / std::sqrt((float)D);
  const int H0 = 2 * (int)B.S + 8;
  wg(v.dz1_tb, t.dz1_tb, D, plane(v.h0, t.h0), 16, D, H0, 1.0f / std::sqrt((float)H0), g("twobody.0"), H0, 0);
  wg(v.dz2_tb, t.dz2_tb, D, plane(v.a1_tb, t.a1_tb), D, D, D, isD, g("twobody.1"), D, 0);
  wg(v.dw0, t.dw0, NW0, dual(c->tX[0]), D, NW0, D, isD, g("embed"), D, 0);
  for (int j = 0; j < Lz; ++j)
    wg(v.de[j], t.de[j], C, dual(c->tX[j]), D, C, D, isD / (float)std::sqrt(B.nu),
       g("layer" + std::to_string(j + 1) + ".env"), D, 0);
  for (int k = 1; k <= Lz; ++k) {
    const std::string pre = "layer" + std::to_string(k) + ".";
    const float sh = 1.0f / std::sqrt((float)KH);
    wg(v.dz1_l[k], t.dz1_l[k], D, dual(c->tX[k - 1]), D, D, D, sh, g(pre + "latent.0"), KH, 0);
    wg(v.dz1_l[k], t.dz1_l[k], D, plane(v.s[k], t.s[k]), C * NS, D, C * NS, sh, g(pre + "latent.0"), KH, D);
    wg(v.dz2_l[k], t.dz2_l[k], D, plane(v.a1_l[k], t.a1_l[k]), D, D, D, isD, g(pre + "latent.1"), D, 0);
    if (k < Lz)
      for (int l = 0; l <= (int)B.lmax; ++l) {
        const int Pl = tp_pl((int)B.lmax, l), toff = tp_toff((int)B.lmax, l);
        const float sc = 1.0f / std::sqrt((float)(C * Pl));
        float* dW = g(pre + "mix" + std::to_string(l));
        if (wgrad_tc_supported(C, C * Pl) && (int64_t)P * (2 * l + 1) < (1ll << 31) - 1024) {
          // dV.t (x) T.v + dV.v (x) T.t on the tensor cores, over (pair, m)
          launch_wgrad_mix_tc(c->tdV + 1, c->tdV, 2, v.T[k], t.T[k], P, C, NLM, NT, l, Pl, toff, sc, dW, part,
                              c->nb.flags, s);
        } else {
          launch_wgrad_mix(c->tdV + 1, 2, v.T[k], P, C, NLM, NT, l, Pl, toff, sc, dW, part, s);   // dV.t (x) T.v
          launch_wgrad_mix(c->tdV, 2, t.T[k], P, C, NLM, NT, l, Pl, toff, sc, dW, part, s);       // dV.v (x) T.t
        }
      }
  }
  wg(v.dze, t.dze, E, plane(v.xL, t.xL), D, E, D, isD, g("energy.0"), D, 0);
  wg(v.dEij, t.dEij, 1, plane(v.ae, t.ae), E, 1, E, 1.0f / std::sqrt((float)E), g("energy.out"), E, 0);
  return cuda_check(c, "weight gradient");
}

// ---- training batches ----
// Every structure's neighbour list, built with its own box, is appended to
// one list (atom and pair indices offset) with per-atom box lengths, so that
// one pass sequence evaluates the whole batch.
template <class T>
int bt_grow(allegro_ctx* c, T*& p, int64_t n_new, int64_t n_keep) {
  T* q = c->dalloc<T>((size_t)n_new);
  if (!q) return c->fail(ALLEGRO_E_OOM, "training batch allocation failed");
  if (p && n_keep > 0) cudaMemcpyAsync(q, p, sizeof(T) * (size_t)n_keep, cudaMemcpyDeviceToDevice, c->stream);
  c->dfree(p);
  p = q;
  return ALLEGRO_OK;
}

int bt_reserve(allegro_ctx* c, int64_t atoms, int64_t pairs, int structs, int64_t keep_atoms, int64_t keep_pairs) {
  TrainBatch& t = c->bt;
  int rc = ALLEGRO_OK;
  if (atoms > t.cap_atoms) {
    const int64_t na = std::max<int64_t>(atoms, t.cap_atoms * 5 / 4);
    rc = bt_grow(c, t.a.row_ptr, na + 1, keep_atoms + 1);
    if (!rc) rc = bt_grow(c, t.a.wpos, 3 * na, 3 * keep_atoms);
    if (!rc) rc = bt_grow(c, t.a.atomL, 3 * na, 3 * keep_atoms);
    if (!rc) rc = bt_grow(c, t.a.species, na, keep_atoms);
    if (!rc) rc = bt_grow(c, t.a.sid, na, keep_atoms);
    if (!rc) rc = bt_grow(c, t.v, 3 * na, 0);
    if (!rc) rc = bt_grow(c, t.seed, na, 0);
    if (!rc) rc = bt_grow(c, t.f_target, 3 * na, 0);
    if (!rc) rc = bt_grow(c, t.loss_blk, na / 256 + 2, 0);
    if (rc) return rc;
    t.cap_atoms = na;
  }
  if (pairs > t.cap_pairs) {
    const int64_t np = std::max<int64_t>(pairs, t.cap_pairs * 5 / 4);
    rc = bt_grow(c, t.a.pi, np, keep_pairs);
    if (!rc) rc = bt_grow(c, t.a.pj, np, keep_pairs);
    if (!rc) rc = bt_grow(c, t.a.pcode, np, keep_pairs);
    if (!rc) rc = bt_grow(c, t.a.rev, np, keep_pairs);
    if (rc) return rc;
    t.cap_pairs = np;
  }
  if (structs > t.cap_structs) {
    rc = bt_grow(c, t.atom_off, structs + 1, 0);
    if (!rc) rc = bt_grow(c, t.e_target, structs, 0);
    if (!rc) rc = bt_grow(c, t.dE, structs, 0);
    if (!rc && !t.d_np) t.d_np = c->dalloc<int>(1);
    if (!rc && !t.loss) t.loss = c->dalloc<double>(1);
    if (rc || !t.d_np || !t.loss) return rc ? rc : c->fail(ALLEGRO_E_OOM, "training batch allocation failed");
    t.cap_structs = structs;
  }
  return ALLEGRO_OK;
}

int build_batch(allegro_ctx* c, const allegro_batch* b) {
  int rc0 = require_fp32(c);                           // training runs the FP32 passes
  if (rc0) return rc0;
  TrainBatch& t = c->bt;
  const int nb = b->n_structs;
  const int64_t base = b->atom_offset[0];
  const int64_t N = b->atom_offset[nb] - base;
  // a training batch replaces the single-system state
  c->md_ready = false;
  c->drop_graphs();
  int rc = bt_reserve(c, N, std::max<int64_t>(t.cap_pairs, 64 * N), nb, 0, 0);
  if (rc) return rc;
  int64_t P0 = 0;
  for (int k = 0; k < nb; ++k) {
    const int64_t a0 = b->atom_offset[k] - base, n = b->atom_offset[k + 1] - b->atom_offset[k];
    double L[3];
    rc = prepare(c, n, b->positions + 3 * (b->atom_offset[k]), b->species + b->atom_offset[k], b->cells + 9 * k, L);
    int64_t np = 0;
    if (!rc) rc = build_with_growth(c, c->d_pos, n, &np);
    if (!rc) rc = bt_reserve(c, N, P0 + np, nb, N, P0);
    if (rc) return rc;
    launch_append(t.a, (int)n, (int)np, a0, P0, k, c->nb.pi, c->nb.pj, c->nb.pcode, c->nb.rev, c->nb.row_ptr,
                  c->nb.wpos, c->d_species, L, c->stream);
    P0 += np;
  }
  if (P0 > 0x7ffffff0) return c->fail(ALLEGRO_E_UNSUPPORTED, "more than 2^31 pairs in a training batch");
  t.n_structs = nb;
  t.n_atoms = N;
  t.n_pairs = P0;
  std::vector<int64_t> off(nb + 1);
  for (int k = 0; k <= nb; ++k) off[k] = b->atom_offset[k] - base;
  const int np32 = (int)P0;
  cudaMemcpyAsync(t.atom_off, off.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(t.e_target, b->e_target, sizeof(double) * nb,
                  is_device_ptr(b->e_target) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(t.f_target, b->f_target + 3 * base, sizeof(float) * 3 * N,
                  is_device_ptr(b->f_target) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(t.d_np, &np32, sizeof(int), cudaMemcpyHostToDevice, c->stream);
  // per-atom outputs and per-pair state for the whole batch
  rc = ensure_atoms(c, N, 0);
  if (!rc) rc = ensure_pairs(c, std::max<int64_t>(P0, c->capacity));
  if (!rc) rc = ensure_train(c);
  if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = cuda_check(c, "training batch");
  return rc;
}

// pass buffers of the batch with positions wpos (wrapped or displaced)
void fill_batch_passbufs(allegro_ctx* c, const double* wpos) {
  const TrainBatch& t = c->bt;
  PassBufs& pb = c->pb;
  pb.pi = t.a.pi;
  pb.pj = t.a.pj;
  pb.pcode = t.a.pcode;
  pb.row_ptr = t.a.row_ptr;
  pb.n_pairs = t.d_np;
  pb.flags = c->nb.flags;
  pb.capacity = c->capacity;
  pb.wpos = wpos;
  pb.species = t.a.species;
  pb.n_atoms = (int)t.n_atoms;
  pb.atomL = t.a.atomL;
  for (int a = 0; a < 3; ++a) pb.L[a] = 0.0;
  pb.tile = fp32_tile(c->w.o3);
}

// Tangent pass sequence over the batch (positions moving along v = dL/dF,
// seeds (-1, dL/dE_i)), then the weight-gradient reductions into d_grad.
int batch_tangent_eval(allegro_ctx* c) {
  const Blob& B = c->blob;
  TrainBatch& t = c->bt;
  fill_batch_passbufs(c, t.a.wpos);
  PassBufs pb = c->pb;
  for (int k = 0; k < kMaxLayers; ++k) {
    pb.X[k] = c->tX[k];
    pb.V[k] = c->tV[k];
  }
  pb.dX = c->tdX;
  pb.dV = c->tdV;
  pb.dU = c->tdU;
  pb.dY = c->tdY;
  pb.G = c->tG;
  for (int k = 0; k <= kMaxLayers; ++k) {
    pb.gam[k] = c->tgam[k];
    pb.dgam[k] = c->tdgam[k];
  }
  pb.epart = c->tepart;
  pb.tile = fp32_tangent_tile();
  pb.tr = c->tr;
  pb.tr.seed = -1.0f;
  pb.tr.seed_atom = nullptr;
  pb.tr.seed_atom_t = t.seed;
  pb.trt = c->trt;
  pb.train = 1;
  pb.vdir = t.v;
  int rc = autotune_fp32(c, 1, [&](const Fp32Launch* ls, KernelMarks* km) {
    fp32_tangent_passes((int)B.lmax, (int)B.C, c->D, c->E, c->w, pb, c->capacity, c->stream, km, ls);
  });
  if (rc) return rc;
  fp32_tangent_passes((int)B.lmax, (int)B.C, c->D, c->E, c->w, pb, c->capacity, c->stream, nullptr, &c->fl[1]);
  c->pb.atomL = nullptr;
  return reduce_wgrad_tangent(c, (int)t.n_pairs);
}

// Enqueue the forward evaluation of the built batch at the current weights:
// forces, per-atom energies and the loss (Eq. 3's objective) into t.loss,
// with the seeds of its weight gradient (dE, v).
void batch_forward_loss(allegro_ctx* c, double w_energy, double w_force) {
  const Blob& B = c->blob;
  TrainBatch& t = c->bt;
  cudaStream_t s = c->stream;
  const int64_t N = t.n_atoms;
  const double cf = w_force / (3.0 * (double)N);
  fill_batch_passbufs(c, t.a.wpos);
  if (c->pb_fp32) {
    autotune_fp32(c, 0, [&](const Fp32Launch* ls, KernelMarks* km) {
      fp32_energy_forces((int)B.lmax, (int)B.C, c->D, c->E, c->w, c->pb, c->capacity, s, km, ls);
    });
    fp32_energy_forces((int)B.lmax, (int)B.C, c->D, c->E, c->w, c->pb, c->capacity, s, nullptr, &c->fl[0]);
  } else {
    c->fp32_bad = true;
  }
  AtomArgs aa = atom_args(c);
  aa.n = (int)N;
  aa.species = t.a.species;
  launch_forces(aa, t.a.row_ptr, t.a.rev, c->pb.G, c->pb.epart, fp32_tile(c->w.o3), c->d_F, c->d_Ei, c->d_blk, c->d_stats,
                c->nb.flags, s);
  c->pb.atomL = nullptr;
  launch_batch_loss((int)t.n_structs, N, t.atom_off, c->d_Ei, t.e_target, c->d_F, t.f_target, w_energy, cf, t.dE,
                    t.v, t.loss_blk, t.loss, s);
}

// Loss (per-atom MSE, energy:force weights) of the built batch and its weight
// gradient into d_grad, all structures at once.  The force term's gradient
// -d/dw sum_i v_i . dE/dr_i (v = 2 c (F - F*), c = w_force / (3 N)) is the
// derivative along v of the hand-written weight adjoint, taken exactly by the
// tangent passes (forward-mode differentiation of the FP32 pass kernels).
int loss_grad_impl(allegro_ctx* c, double w_energy, double w_force, double* loss_out) {
  const Blob& B = c->blob;
  if (B.L > 2) return c->fail(ALLEGRO_E_UNSUPPORTED, "training is built for models of at most two layers");
  int rc = init_master(c);
  if (rc) return rc;
  TrainBatch& t = c->bt;
  cudaStream_t s = c->stream;
  cudaMemsetAsync(c->d_grad, 0, sizeof(float) * c->n_params, s);
  cudaMemsetAsync(c->nb.flags, 0, sizeof(int), s);
  const int nbk = (int)t.n_structs;
  const int64_t N = t.n_atoms;
  // forward over the batch: forces, per-atom energies, loss, v = dL/dF
  batch_forward_loss(c, w_energy, w_force);
  // energy-loss seeds, then one tangent pass sequence along v: the energy
  // term and the force term's -d/dw (v . dE/dr) of Eq. 3's loss at once
  launch_seed_energy(nbk, N, t.atom_off, t.a.sid, t.dE, w_energy, t.seed, s);
  rc = batch_tangent_eval(c);
  if (rc) return rc;
  double loss = 0.0;
  int flags = 0;
  cudaMemcpyAsync(&loss, t.loss, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&flags, c->nb.flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "loss gradient");
  if (flags & kFlagTimeout) return c->fail(ALLEGRO_E_TIMEOUT, "a pass gave up a bounded wait");
  if (flags & kFlagPairOverflow) return c->fail(ALLEGRO_E_PAIR_OVERFLOW, "training batch exceeds the pair capacity");
  if (loss_out) *loss_out = loss;
  return ALLEGRO_OK;
}

int check_batch(allegro_ctx* c, const allegro_batch* b) {
  if (!b || b->n_structs < 1 || !b->atom_offset || !b->positions || !b->species || !b->cells || !b->e_target ||
      !b->f_target)
    return c->fail(ALLEGRO_E_INVALID_ARG, "incomplete batch");
  for (int k = 0; k < b->n_structs; ++k)
    if (b->atom_offset[k + 1] <= b->atom_offset[k]) return c->fail(ALLEGRO_E_INVALID_ARG, "empty structure in batch");
  return ALLEGRO_OK;
}

}  // namespace

extern "C" {

const char* allegro_version(void) { return kVersion; }

const char* allegro_last_error(const allegro_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int allegro_create(const void* weights_blob, size_t blob_bytes, const double* species_mass, int32_t n_species,
                   double r_cut, int32_t l_max, int32_t n_layers, allegro_ctx** out) {
  if (!out || !weights_blob || !species_mass) {
    g_err = "NULL argument";
    return ALLEGRO_E_INVALID_ARG;
  }
  *out = nullptr;
  allegro_ctx* c = new (std::nothrow) allegro_ctx();
  if (!c) {
    g_err = "host allocation failed";
    return ALLEGRO_E_OOM;
  }
  std::string why;
  if (!parse_blob(weights_blob, blob_bytes, c->blob, why)) {
    g_err = "weights blob: " + why;
    delete c;
    return ALLEGRO_E_BLOB;
  }
  const Blob& B = c->blob;
  if ((int)B.S != n_species || B.rc != r_cut || (int)B.lmax != l_max || (int)B.L != n_layers) {
    g_err = "create() arguments disagree with the weights blob header";
    delete c;
    return ALLEGRO_E_MISMATCH;
  }
  // Full O(3): a pseudotensor made by an odd path of layer k reaches a true
  // scalar (0e) only through a further odd path, which no l3 = 0 output has
  // (l1 = l2 there), so it first changes the energy through the mixing of
  // layer k + 1 into a layer k + 2.  With at most two layers (or l_max 0,
  // where no path is odd) the full-O(3) model therefore is the natural-parity
  // model (its pseudotensor mixing matrices, layer{k}.mix{l}p, have no effect
  // and are not loaded) and runs on every pass implementation; from three
  // layers on it runs the full-O(3) FP32 passes (features of both parities,
  // every odd path).
  c->w.o3 = (B.parity == 1 && B.L >= 3 && B.lmax >= 1) ? 1 : 0;
  const bool shape_ok = B.S == 2 && B.NB == 8 && B.p == 6 && B.latent.size() == 2 && B.latent[0] == B.latent[1] &&
                        B.energy.size() == 1 && B.L >= 1 && B.L <= (uint32_t)kMaxLayers &&
                        fp32_supported((int)B.lmax, (int)B.C, (int)B.latent[0], (int)B.energy[0], c->w.o3 != 0);
  if (!shape_ok) {
    g_err = "model shape not compiled into this library";
    delete c;
    return ALLEGRO_E_UNSUPPORTED;
  }
  c->D = (int)B.latent[0];
  c->E = (int)B.energy[0];
  for (int s = 0; s < 2; ++s) c->mass[s] = species_mass[s];
  int rc = upload_weights(c);
  c->bf16_ok = !c->w.o3 && bf16_supported((int)B.lmax, (int)B.C, c->D, c->E, (int)B.L);
  if (!rc && c->bf16_ok) rc = upload_weights_bf16(c, TcMode::kBf16);
  if (!rc && c->bf16_ok) rc = upload_weights_bf16(c, TcMode::kFp16);
  if (!rc && c->bf16_ok) rc = upload_weights_bf16(c, TcMode::kFp16Split);
  if (rc) {
    g_err = c->err;
    delete c;
    return rc;
  }
  *out = c;
  return ALLEGRO_OK;
}

void allegro_destroy(allegro_ctx* ctx) { delete ctx; }

int allegro_set_stream(allegro_ctx* ctx, void* s) {
  if (!ctx) return ALLEGRO_E_INVALID_ARG;
  ctx->stream = (cudaStream_t)s;
  ctx->drop_graphs();
  return ALLEGRO_OK;
}

int allegro_build_neighbors(allegro_ctx* ctx, int64_t n_atoms, const double* positions, const double* cell,
                            int64_t* n_pairs) {
  if (!ctx) return ALLEGRO_E_INVALID_ARG;
  double L[3];
  int rc = prepare(ctx, n_atoms, positions, nullptr, cell, L);
  if (rc) return rc;
  int64_t np = 0;
  rc = build_with_growth(ctx, ctx->d_pos, n_atoms, &np);
  if (rc) return rc;
  if (n_pairs) *n_pairs = np;
  return ALLEGRO_OK;
}

int allegro_get_neighbors(allegro_ctx* ctx, int32_t* row_ptr, int32_t* col, int8_t* img, int32_t* rev) {
  if (!ctx || ctx->n_atoms <= 0) return ALLEGRO_E_INVALID_ARG;
  int np = 0;
  cudaMemcpyAsync(&np, ctx->nb.n_pairs, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  int rc = copy_out(ctx, row_ptr, ctx->nb.row_ptr, sizeof(int) * (ctx->n_atoms + 1));
  if (!rc) rc = copy_out(ctx, col, ctx->nb.pj, sizeof(int) * np);
  if (!rc) rc = copy_out(ctx, rev, ctx->nb.rev, sizeof(int) * np);
  if (!rc && img) {
    std::vector<int> code(np);
    std::vector<int8_t> out(3 * (size_t)np);
    cudaMemcpyAsync(code.data(), ctx->nb.pcode, sizeof(int) * np, cudaMemcpyDeviceToHost, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    for (int p = 0; p < np; ++p) {
      out[3 * p] = (int8_t)(code[p] / 25 - 2);
      out[3 * p + 1] = (int8_t)((code[p] / 5) % 5 - 2);
      out[3 * p + 2] = (int8_t)(code[p] % 5 - 2);
    }
    const cudaMemcpyKind k = is_device_ptr(img) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    cudaMemcpyAsync(img, out.data(), out.size(), k, ctx->stream);
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "get_neighbors");
  return rc;
}

int allegro_energy_forces(allegro_ctx* ctx, int64_t n_atoms, const double* positions, const int32_t* species,
                          const double* cell, double* energy_out, float* forces_out, double* atom_energy,
                          int32_t precision) {
  if (!ctx) return ALLEGRO_E_INVALID_ARG;
  if (!species || !energy_out) return ctx->fail(ALLEGRO_E_INVALID_ARG, "species and energy_out are required");
  double L[3];
  int rc = precision == ALLEGRO_FP32 ? require_fp32(ctx) : ALLEGRO_OK;
  if (!rc) rc = prepare(ctx, n_atoms, positions, species, cell, L);
  if (rc) return rc;
  int64_t np = 0;
  rc = build_with_growth(ctx, ctx->d_pos, n_atoms, &np);
  if (rc) return rc;
  rc = run_model(ctx, precision, L);
  if (rc) return rc;
  double stats[2];
  int flags = 0;
  cudaMemcpyAsync(stats, ctx->d_stats, sizeof(stats), cudaMemcpyDeviceToHost, ctx->stream);
  cudaMemcpyAsync(&flags, ctx->nb.flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  rc = copy_out(ctx, forces_out, ctx->d_F, sizeof(float) * 3 * n_atoms);
  if (!rc) rc = copy_out(ctx, atom_energy, ctx->d_Ei, sizeof(double) * n_atoms);
  if (rc) return rc;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "energy_forces");
  if (flags & kFlagTimeout) return ctx->fail(ALLEGRO_E_TIMEOUT, "a tensor-core pass gave up a bounded wait");
  if (flags & kFlagNonfinite) return ctx->fail(ALLEGRO_E_NONFINITE, "non-finite energy or force");
  *energy_out = stats[0];
  return ALLEGRO_OK;
}

int allegro_outlier_count(allegro_ctx* ctx, int64_t n_atoms, const float* forces, double threshold,
                          int64_t* count_out) {
  if (!ctx || !forces || !count_out || n_atoms <= 0) return ALLEGRO_E_INVALID_ARG;
  int rc = ensure_atoms(ctx, n_atoms, 0);
  if (rc) return rc;
  const cudaMemcpyKind k = is_device_ptr(forces) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyAsync(ctx->d_F_snap, forces, sizeof(float) * 3 * n_atoms, k, ctx->stream);
  launch_sum_f2((int)n_atoms, ctx->d_F_snap, ctx->d_stats + 4, ctx->stream);
  launch_outliers((int)n_atoms, ctx->d_F_snap, ctx->d_stats + 4, threshold, ctx->d_blku, ctx->d_count,
                  ctx->stream);
  long long cnt = 0;
  cudaMemcpyAsync(&cnt, ctx->d_count, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "outlier_count");
  *count_out = cnt;
  return ALLEGRO_OK;
}

int allegro_set_skin(allegro_ctx* ctx, double skin_A) {
  if (!ctx) return ALLEGRO_E_INVALID_ARG;
  if (!(skin_A >= 0.0) || !std::isfinite(skin_A) || skin_A > ctx->blob.rc)
    return ctx->fail(ALLEGRO_E_INVALID_ARG, "skin must be in [0, r_cut]");
  ctx->skin = skin_A;
  return ALLEGRO_OK;
}

int allegro_set_md_precision(allegro_ctx* ctx, int32_t precision) {
  if (!ctx || !valid_precision(precision)) return ALLEGRO_E_INVALID_ARG;
  if (precision != ALLEGRO_FP32 && !ctx->bf16_ok)
    return ctx->fail(ALLEGRO_E_UNSUPPORTED, "the tensor-core path is built for the 16-channel, latent-128 model with 2+ layers and l_max <= 2 (natural parity, or full O(3) with two layers) only");
  if (precision == ALLEGRO_FP32) {
    const int rc = require_fp32(ctx);
    if (rc) return rc;
  }
  if (precision != ctx->md_precision) ctx->drop_graphs();
  ctx->md_precision = precision;
  return ALLEGRO_OK;
}

int allegro_md_init(allegro_ctx* ctx, int64_t n_atoms, const double* positions, const double* velocities,
                    const int32_t* species, const double* cell) {
  if (!ctx) return ALLEGRO_E_INVALID_ARG;
  if (!velocities || !species) return ctx->fail(ALLEGRO_E_INVALID_ARG, "velocities and species are required");
  double L[3];
  ctx->md_ready = false;
  int rc = ctx->md_precision == ALLEGRO_FP32 ? require_fp32(ctx) : ALLEGRO_OK;
  if (!rc) rc = prepare(ctx, n_atoms, positions, species, cell, L, ctx->skin);
  ctx->md_skin = ctx->skin;
  if (rc) return rc;
  const cudaMemcpyKind kv = is_device_ptr(velocities) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyAsync(ctx->d_v, velocities, sizeof(double) * 3 * n_atoms, kv, ctx->stream);
  int64_t np = 0;
  rc = build_with_growth(ctx, ctx->d_pos, n_atoms, &np);
  if (rc) return rc;
  // keep a little headroom for density fluctuations during the trajectory
  if (ctx->capacity < np + np / 8 + 1024) {
    rc = ensure_pairs(ctx, np + np / 4 + 1024);
    if (rc) return rc;
    rc = build_with_growth(ctx, ctx->d_pos, n_atoms, &np);
    if (rc) return rc;
  }
  rc = run_model(ctx, ctx->md_precision, L);
  if (rc) return rc;
  // state positions are the wrapped ones; they are also the skin's reference
  cudaMemcpyAsync(ctx->d_pos, ctx->nb.wpos, sizeof(double) * 3 * n_atoms, cudaMemcpyDeviceToDevice, ctx->stream);
  cudaMemcpyAsync(ctx->d_pos_ref, ctx->nb.wpos, sizeof(double) * 3 * n_atoms, cudaMemcpyDeviceToDevice, ctx->stream);
  cudaMemcpyAsync(ctx->d_wpos_ref, ctx->nb.wpos, sizeof(double) * 3 * n_atoms, cudaMemcpyDeviceToDevice,
                  ctx->stream);
  cudaMemsetAsync(ctx->d_skin_flag, 0, sizeof(int) * 4, ctx->stream);
  cudaMemsetAsync(ctx->d_nh, 0, sizeof(double) * 4, ctx->stream);   // thermostat at rest (xi = eta = 0)
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "md_init");
  ctx->drop_graphs();
  ctx->step = 0;
  ctx->md_ready = true;
  return ALLEGRO_OK;
}

namespace {

// per-step records (energies, 4 values a step, and outlier counts) for
// n_steps steps; the step graphs bake the pointers in
int ensure_records(allegro_ctx* c, int n_steps) {
  if (n_steps <= c->rec_cap) return ALLEGRO_OK;
  c->dfree(c->d_e_rec);
  c->dfree(c->d_out_rec);
  const int cap = std::max(n_steps, 1024);
  c->d_e_rec = c->dalloc<double>(4 * (size_t)cap);
  c->d_out_rec = c->dalloc<long long>(cap);
  if (!c->d_e_rec || !c->d_out_rec) return c->fail(ALLEGRO_E_OOM, "record allocation failed");
  c->rec_cap = cap;
  c->drop_graphs();
  return ALLEGRO_OK;
}

// end a capture on cs, count its kernels and instantiate it into *out
int finish_capture(allegro_ctx* c, cudaStream_t cs, bool own, cudaGraphExec_t* out, int64_t* kernels) {
  cudaGraph_t g;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (e != cudaSuccess) {
    if (own) cudaStreamDestroy(cs);
    return cuda_check(c, "end capture");
  }
  size_t n_nodes = 0;
  cudaGraphGetNodes(g, nullptr, &n_nodes);
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  cudaGraphGetNodes(g, nodes.data(), &n_nodes);
  *kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++*kernels;
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (own) cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_check(c, "graph instantiate");
  return ALLEGRO_OK;
}

// Neighbour list of one MD step: rebuilt every step without a skin; with a
// skin, the build runs only when an atom has moved by more than skin/2 since
// the last one (or a rebuild was forced), otherwise the list stays and the
// wrapped positions follow the atoms from the reference wrap.
void launch_md_neighbors(allegro_ctx* c, const double L[3], cudaStream_t cs) {
  if (c->md_skin <= 0.0) {
    launch_build_neighbors(c->nb, c->grid, c->d_pos, c->n_atoms, cs);
    return;
  }
  launch_skin_check(c->n_atoms, c->d_pos, c->d_pos_ref, L, c->md_skin, c->d_skin_flag, cs);
  launch_build_neighbors(c->nb, c->grid, c->d_pos, c->n_atoms, cs, 0, c->d_skin_flag);
  launch_skin_commit(c->n_atoms, c->d_pos, c->d_pos_ref, c->nb.wpos, c->d_wpos_ref, L, c->d_skin_flag, cs);
}

// one NVT step as a graph: thermostat half step, kick, drift, neighbour
// list, energy and forces, kick, thermostat half step, record
int capture_step_nvt(allegro_ctx* c, double dt, double temperature, double tau) {
  if (c->graph_nvt) {
    cudaGraphExecDestroy(c->graph_nvt);
    c->graph_nvt = nullptr;
  }
  double L[3] = {c->grid.L[0], c->grid.L[1], c->grid.L[2]};
  fill_passbufs(c, L);
  cudaStream_t cs = c->stream;
  bool own = false;
  if (!cs) {
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cuda_check(c, "stream");
    own = true;
  }
  const double gkt = 3.0 * (double)c->n_atoms * kBoltzmannEv * temperature;
  const double q = gkt * tau * tau;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_check(c, "capture");
  const AtomArgs a = atom_args(c);
  launch_nvt_first_half(a, c->d_pos, c->d_v, c->d_F, dt, L, gkt, q, c->d_blk_ke, c->d_nh, cs);
  launch_md_neighbors(c, L, cs);
  launch_model(c, c->md_precision, cs, nullptr);
  launch_nvt_second_half(a, c->d_v, c->d_F, dt, c->d_stats, 5.0, gkt, q, c->d_blk_ke, c->d_blku, c->d_nh,
                         c->d_step, c->rec_cap, c->d_e_rec, c->d_out_rec, cs);
  int64_t kernels = 0;
  const int rc = finish_capture(c, cs, own, &c->graph_nvt, &kernels);
  if (rc) return rc;
  c->nvt_key[0] = dt;
  c->nvt_key[1] = temperature;
  c->nvt_key[2] = tau;
  return ALLEGRO_OK;
}

// MD calls that overflow the pair capacity roll back to their first step,
// grow the capacity by half and run again, up to this many times (a long call
// on a heating system may outgrow several capacities).
constexpr int kMdAttempts = 6;

int capture_step(allegro_ctx* c, double dt) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  double L[3] = {c->grid.L[0], c->grid.L[1], c->grid.L[2]};
  fill_passbufs(c, L);
  cudaStream_t cs = c->stream;
  bool own = false;
  if (!cs) {
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cuda_check(c, "stream");
    own = true;
  }
  cudaGraph_t g;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_check(c, "capture");
  const AtomArgs a = atom_args(c);
  launch_kick_drift(a, c->d_pos, c->d_v, c->d_F, dt, L, cs);
  launch_md_neighbors(c, L, cs);
  launch_model(c, c->md_precision, cs, nullptr);
  launch_kick_measure(a, c->d_v, c->d_F, dt, c->d_stats, 5.0, c->d_blk_ke, c->d_blku, c->d_step, c->rec_cap,
                      c->d_e_rec, c->d_out_rec, cs);
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (e != cudaSuccess) {
    if (own) cudaStreamDestroy(cs);
    return cuda_check(c, "end capture");
  }
  size_t n_nodes = 0;
  cudaGraphGetNodes(g, nullptr, &n_nodes);
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  cudaGraphGetNodes(g, nodes.data(), &n_nodes);
  c->graph_kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) c->graph_kernels++;
  }
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (own) cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_check(c, "graph instantiate");
  c->graph_dt = dt;
  return ALLEGRO_OK;
}

}  // namespace

int allegro_md_step_nve(allegro_ctx* ctx, double dt_fs, int32_t n_steps, int64_t* outlier_counts,
                        double* energies) {
  if (!ctx || !ctx->md_ready) return ctx ? ctx->fail(ALLEGRO_E_INVALID_ARG, "md_init first") : ALLEGRO_E_INVALID_ARG;
  if (n_steps < 0 || !(dt_fs > 0.0) || !std::isfinite(dt_fs)) return ctx->fail(ALLEGRO_E_INVALID_ARG, "bad dt or n_steps");
  if (n_steps == 0) return ALLEGRO_OK;
  int rc0 = ensure_records(ctx, n_steps);
  if (rc0) return rc0;
  const size_t n3 = 3 * (size_t)ctx->n_atoms;
  for (int attempt = 0; attempt < kMdAttempts; ++attempt) {
    if (!ctx->graph || ctx->graph_dt != dt_fs) {
      int rc = capture_step(ctx, dt_fs);
      if (rc) return rc;
    }
    cudaMemcpyAsync(ctx->d_pos_snap, ctx->d_pos, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_v_snap, ctx->d_v, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_F_snap, ctx->d_F, sizeof(float) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemsetAsync(ctx->nb.flags, 0, sizeof(int), ctx->stream);
    cudaMemsetAsync(ctx->d_step, 0, sizeof(long long), ctx->stream);
    cudaMemsetAsync(ctx->d_skin_flag + 1, 1, sizeof(int), ctx->stream);   // skin: rebuild at the first step
    for (int s = 0; s < n_steps; ++s)
      if (cudaGraphLaunch(ctx->graph, ctx->stream) != cudaSuccess) return cuda_check(ctx, "graph launch");
    int flags = 0, np = 0;
    cudaMemcpyAsync(&flags, ctx->nb.flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(&np, ctx->nb.n_pairs, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "md steps");
    if (flags & (kFlagPairOverflow | kFlagTimeout)) {
      cudaMemcpyAsync(ctx->d_pos, ctx->d_pos_snap, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaMemcpyAsync(ctx->d_v, ctx->d_v_snap, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaMemcpyAsync(ctx->d_F, ctx->d_F_snap, sizeof(float) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      if (flags & kFlagTimeout) return ctx->fail(ALLEGRO_E_TIMEOUT, "a tensor-core pass gave up a bounded wait (state rolled back)");
      const int64_t grow = std::max<int64_t>((int64_t)np, ctx->capacity) * 3 / 2 + 1024;
      int rc = ensure_pairs(ctx, grow);
      if (rc) return rc;
      continue;
    }
    if (flags & kFlagNonfinite) return ctx->fail(ALLEGRO_E_NONFINITE, "non-finite energy or force during MD");
    ctx->step += n_steps;
    int rc = copy_out(ctx, outlier_counts, ctx->d_out_rec, sizeof(long long) * n_steps);
    if (!rc) rc = copy_out(ctx, energies, ctx->d_e_rec, sizeof(double) * 3 * n_steps);
    if (rc) return rc;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "md record copy");
    return ALLEGRO_OK;
  }
  return ctx->fail(ALLEGRO_E_PAIR_OVERFLOW, "pair capacity could not be grown during MD");
}

int allegro_md_step_nvt(allegro_ctx* ctx, double dt_fs, int32_t n_steps, double temperature_K, double tau_fs,
                        int64_t* outlier_counts, double* energies) {
  if (!ctx || !ctx->md_ready) return ctx ? ctx->fail(ALLEGRO_E_INVALID_ARG, "md_init first") : ALLEGRO_E_INVALID_ARG;
  if (n_steps < 0 || !(dt_fs > 0.0) || !std::isfinite(dt_fs)) return ctx->fail(ALLEGRO_E_INVALID_ARG, "bad dt or n_steps");
  if (!(temperature_K > 0.0) || !std::isfinite(temperature_K) || !(tau_fs > 0.0) || !std::isfinite(tau_fs))
    return ctx->fail(ALLEGRO_E_INVALID_ARG, "temperature and tau must be positive");
  if (n_steps == 0) return ALLEGRO_OK;
  int rc = ensure_records(ctx, n_steps);
  if (rc) return rc;
  const size_t n3 = 3 * (size_t)ctx->n_atoms;
  const AtomArgs a = atom_args(ctx);
  for (int attempt = 0; attempt < kMdAttempts; ++attempt) {
    if (!ctx->graph_nvt || ctx->nvt_key[0] != dt_fs || ctx->nvt_key[1] != temperature_K || ctx->nvt_key[2] != tau_fs) {
      rc = capture_step_nvt(ctx, dt_fs, temperature_K, tau_fs);
      if (rc) return rc;
    }
    cudaMemcpyAsync(ctx->d_pos_snap, ctx->d_pos, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_v_snap, ctx->d_v, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_F_snap, ctx->d_F, sizeof(float) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_nh_snap, ctx->d_nh, sizeof(double) * 4, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemsetAsync(ctx->nb.flags, 0, sizeof(int), ctx->stream);
    cudaMemsetAsync(ctx->d_step, 0, sizeof(long long), ctx->stream);
    cudaMemsetAsync(ctx->d_skin_flag + 1, 1, sizeof(int), ctx->stream);   // skin: rebuild at the first step
    launch_nh_set_k(a, ctx->d_v, ctx->d_blk_ke, ctx->d_nh, ctx->stream);   // K of the current velocities
    for (int s = 0; s < n_steps; ++s)
      if (cudaGraphLaunch(ctx->graph_nvt, ctx->stream) != cudaSuccess) return cuda_check(ctx, "graph launch");
    int flags = 0, np = 0;
    cudaMemcpyAsync(&flags, ctx->nb.flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(&np, ctx->nb.n_pairs, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "nvt steps");
    if (flags & (kFlagPairOverflow | kFlagTimeout)) {
      cudaMemcpyAsync(ctx->d_pos, ctx->d_pos_snap, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaMemcpyAsync(ctx->d_v, ctx->d_v_snap, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaMemcpyAsync(ctx->d_F, ctx->d_F_snap, sizeof(float) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaMemcpyAsync(ctx->d_nh, ctx->d_nh_snap, sizeof(double) * 4, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      if (flags & kFlagTimeout) return ctx->fail(ALLEGRO_E_TIMEOUT, "a tensor-core pass gave up a bounded wait (state rolled back)");
      const int64_t grow = std::max<int64_t>((int64_t)np, ctx->capacity) * 3 / 2 + 1024;
      rc = ensure_pairs(ctx, grow);
      if (rc) return rc;
      continue;
    }
    if (flags & kFlagNonfinite) return ctx->fail(ALLEGRO_E_NONFINITE, "non-finite energy or force during MD");
    ctx->step += n_steps;
    rc = copy_out(ctx, outlier_counts, ctx->d_out_rec, sizeof(long long) * n_steps);
    if (!rc) rc = copy_out(ctx, energies, ctx->d_e_rec, sizeof(double) * 4 * n_steps);
    if (rc) return rc;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "nvt record copy");
    return ALLEGRO_OK;
  }
  return ctx->fail(ALLEGRO_E_PAIR_OVERFLOW, "pair capacity could not be grown during MD");
}

int allegro_md_get_thermostat(allegro_ctx* ctx, double* xi_eta) {
  if (!ctx || !xi_eta) return ALLEGRO_E_INVALID_ARG;
  if (!ctx->md_ready) return ctx->fail(ALLEGRO_E_INVALID_ARG, "md_init first");
  const int rc = copy_out(ctx, xi_eta, ctx->d_nh, sizeof(double) * 2);
  if (rc) return rc;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "thermostat state");
  return ALLEGRO_OK;
}

namespace {

// Energies and forces of every replica at the current bead positions, into
// d_rp_F, with stats[0] = the sum of the replica energies.  One neighbour
// build covers all replicas (each replica its own system in the common box),
// then one pass sequence of the MD precision runs over all P n atoms.  Only
// launches: usable inside a stream capture; a pair-capacity overflow raises
// the device flag and the pass kernels skip their work.
void rp_launch_forces(allegro_ctx* c, cudaStream_t s) {
  const int64_t PN = (int64_t)c->rp_P * c->rp_n;
  c->grid = c->rp_grid;
  c->n_atoms = (int)PN;
  launch_build_neighbors(c->nb, c->rp_grid, c->d_rp_q, (int)PN, s, (int)c->rp_n);
  fill_passbufs(c, c->rp_L);
  c->pb.species = c->d_rp_species_all;
  int tile;
  const int prec = c->md_precision;
  if (prec == ALLEGRO_FP32) {
    if (c->pb_fp32) fp32_energy_forces((int)c->blob.lmax, (int)c->blob.C, c->D, c->E, c->w, c->pb, c->capacity, s);
    else c->fp32_bad = true;
    tile = fp32_tile(c->w.o3);
  } else {
    const TcMode mode = prec == ALLEGRO_BF16 ? TcMode::kBf16 : prec == ALLEGRO_FP16 ? TcMode::kFp16 : TcMode::kFp16Split;
    bf16_energy_forces(prec == ALLEGRO_BF16 ? c->bw : prec == ALLEGRO_FP16 ? c->hw : c->sw, c->pb, c->capacity, s,
                       nullptr, mode);
    tile = bf16_tile();
  }
  AtomArgs aa = atom_args(c);
  aa.n = (int)PN;
  aa.species = c->d_rp_species_all;
  launch_forces(aa, c->nb.row_ptr, c->nb.rev, c->pb.G, c->pb.epart, tile, c->d_rp_F, c->d_Ei, c->d_blk, c->d_stats,
                c->nb.flags, s);
}

AtomArgs rp_atom_args(allegro_ctx* c) {
  AtomArgs a = atom_args(c);
  a.n = (int)c->rp_n;
  a.species = c->d_rp_species;
  return a;
}

// the per-atom, cell and pair buffers for P n atoms in the ring's box
int rp_reserve(allegro_ctx* c) {
  const int64_t PN = (int64_t)c->rp_P * c->rp_n;
  const GridInfo& g = c->rp_grid;
  const int64_t ncell = g.ncell[0] > 0 ? (int64_t)c->rp_P * g.ncell[0] * g.ncell[1] * g.ncell[2] : 0;
  if (ncell > std::max<int64_t>(PN, 1 << 22)) return c->fail(ALLEGRO_E_UNSUPPORTED, "too many cells for the ring");
  int rc = ensure_atoms(c, PN, (int)ncell);
  if (rc) return rc;
  const double vol = c->rp_L[0] * c->rp_L[1] * c->rp_L[2];
  const double rc3 = c->blob.rc * c->blob.rc * c->blob.rc;
  const double est = (double)PN * (4.18879 * rc3 * (double)c->rp_n / vol) * 1.3 + 4096.0;
  if (c->capacity < (int64_t)std::min(est, 2.0e9)) return ensure_pairs(c, (int64_t)std::min(est, 2.0e9));
  return ensure_pairs(c, c->capacity);
}

// one ring-polymer step as a graph: kick, free ring evolution, neighbour
// list and forces of all replicas, kick, record
int capture_step_rp(allegro_ctx* c, double dt) {
  if (c->graph_rp) {
    cudaGraphExecDestroy(c->graph_rp);
    c->graph_rp = nullptr;
  }
  cudaStream_t cs = c->stream;
  bool own = false;
  if (!cs) {
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cuda_check(c, "stream");
    own = true;
  }
  const int P = c->rp_P;
  const double wp = P * kBoltzmannEv * c->rp_T / kHbarEvFs;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_check(c, "capture");
  const AtomArgs a = rp_atom_args(c);
  launch_rp_kick(P, a, c->d_rp_v, c->d_rp_F, 0.5 * dt, cs);
  launch_rp_free(P, (int)c->rp_n, c->d_rp_q, c->d_rp_v, c->d_rp_C, c->d_rp_w, dt, cs);
  rp_launch_forces(c, cs);
  launch_rp_kick(P, a, c->d_rp_v, c->d_rp_F, 0.5 * dt, cs);
  launch_rp_record(P, a, c->d_rp_q, c->d_rp_v, wp, c->d_rp_blk, c->d_stats, c->d_step, c->rec_cap, c->d_e_rec, cs);
  const int rc = finish_capture(c, cs, own, &c->graph_rp, &c->rp_graph_kernels);
  if (rc) return rc;
  c->rp_graph_dt = dt;
  return ALLEGRO_OK;
}

}  // namespace

int allegro_pimd_init(allegro_ctx* ctx, int32_t n_beads, int64_t n_atoms, const double* positions,
                      const double* velocities, const int32_t* species, const double* cell, double temperature_K) {
  if (!ctx) return ALLEGRO_E_INVALID_ARG;
  if (n_beads < 1 || n_beads > kMaxBeads) return ctx->fail(ALLEGRO_E_INVALID_ARG, "n_beads must be in [1, 64]");
  if (n_atoms < 1 || (int64_t)n_beads * n_atoms > (1 << 30))
    return ctx->fail(ALLEGRO_E_INVALID_ARG, "n_atoms out of range");
  if (!positions || !velocities || !species || !cell)
    return ctx->fail(ALLEGRO_E_INVALID_ARG, "positions, velocities, species and cell are required");
  if (!(temperature_K > 0.0) || !std::isfinite(temperature_K))
    return ctx->fail(ALLEGRO_E_INVALID_ARG, "temperature must be positive");
  double L[3];
  int rc = check_cell(ctx, cell, L);
  if (!rc && ctx->md_precision == ALLEGRO_FP32) rc = require_fp32(ctx);
  if (rc) return rc;
  ctx->rp_ready = false;
  ctx->md_ready = false;
  ctx->drop_graphs();
  const int P = n_beads;
  const int64_t PN = (int64_t)P * n_atoms;
  for (void* p : {(void*)ctx->d_rp_q, (void*)ctx->d_rp_v, (void*)ctx->d_rp_F, (void*)ctx->d_rp_q_snap,
                  (void*)ctx->d_rp_v_snap, (void*)ctx->d_rp_F_snap, (void*)ctx->d_rp_species,
                  (void*)ctx->d_rp_species_all, (void*)ctx->d_rp_C, (void*)ctx->d_rp_w, (void*)ctx->d_rp_blk})
    ctx->dfree(p);
  ctx->d_rp_q = ctx->dalloc<double>(3 * (size_t)PN);
  ctx->d_rp_v = ctx->dalloc<double>(3 * (size_t)PN);
  ctx->d_rp_F = ctx->dalloc<float>(3 * (size_t)PN);
  ctx->d_rp_q_snap = ctx->dalloc<double>(3 * (size_t)PN);
  ctx->d_rp_v_snap = ctx->dalloc<double>(3 * (size_t)PN);
  ctx->d_rp_F_snap = ctx->dalloc<float>(3 * (size_t)PN);
  ctx->d_rp_species = ctx->dalloc<int>((size_t)n_atoms);
  ctx->d_rp_species_all = ctx->dalloc<int>((size_t)PN);
  ctx->d_rp_C = ctx->dalloc<double>((size_t)P * P);
  ctx->d_rp_w = ctx->dalloc<double>((size_t)P);
  ctx->d_rp_blk = ctx->dalloc<double>(2 * ((size_t)PN / 256 + 2));
  if (!ctx->d_rp_q || !ctx->d_rp_v || !ctx->d_rp_F || !ctx->d_rp_q_snap || !ctx->d_rp_v_snap ||
      !ctx->d_rp_F_snap || !ctx->d_rp_species || !ctx->d_rp_species_all || !ctx->d_rp_C || !ctx->d_rp_w ||
      !ctx->d_rp_blk)
    return ctx->fail(ALLEGRO_E_OOM, "replica allocation failed");
  cudaStream_t s = ctx->stream;
  const cudaMemcpyKind kq = is_device_ptr(positions) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kv = is_device_ptr(velocities) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind ks = is_device_ptr(species) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyAsync(ctx->d_rp_q, positions, sizeof(double) * 3 * PN, kq, s);
  cudaMemcpyAsync(ctx->d_rp_v, velocities, sizeof(double) * 3 * PN, kv, s);
  cudaMemcpyAsync(ctx->d_rp_species, species, sizeof(int) * n_atoms, ks, s);
  for (int k = 0; k < P; ++k)
    cudaMemcpyAsync(ctx->d_rp_species_all + (size_t)k * n_atoms, ctx->d_rp_species, sizeof(int) * n_atoms,
                    cudaMemcpyDeviceToDevice, s);
  // normal modes of the ring: C[j P + k], frequencies omega_k = 2 omega_P sin(k' pi / P)
  const double wp = P * kBoltzmannEv * temperature_K / kHbarEvFs;
  std::vector<double> C((size_t)P * P), w(P);
  for (int k = 0; k < P; ++k) {
    for (int j = 0; j < P; ++j) {
      double cjk;
      if (k == 0) cjk = 1.0 / std::sqrt((double)P);
      else if (2 * k < P) cjk = std::sqrt(2.0 / P) * std::cos(2.0 * M_PI * j * k / P);
      else if (2 * k == P) cjk = ((j & 1) ? -1.0 : 1.0) / std::sqrt((double)P);
      else cjk = std::sqrt(2.0 / P) * std::sin(2.0 * M_PI * j * k / P);
      C[(size_t)j * P + k] = cjk;
    }
    const int kk = 2 * k <= P ? k : P - k;
    w[k] = 2.0 * wp * std::sin(kk * M_PI / P);
  }
  cudaMemcpyAsync(ctx->d_rp_C, C.data(), sizeof(double) * P * P, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(ctx->d_rp_w, w.data(), sizeof(double) * P, cudaMemcpyHostToDevice, s);
  for (int a = 0; a < 3; ++a) ctx->rp_L[a] = L[a];
  ctx->rp_grid = plan_grid(L, ctx->blob.rc);
  ctx->rp_P = P;
  ctx->rp_n = n_atoms;
  ctx->rp_T = temperature_K;
  rc = rp_reserve(ctx);
  if (rc) return rc;
  if (ctx->md_precision != ALLEGRO_FP32) {
    rc = refresh_tc(ctx);
    if (rc) return rc;
  }
  // species check, then the forces of the initial beads (growing the pair
  // capacity if the estimate was short)
  cudaMemsetAsync(ctx->nb.flags, 0, sizeof(int), s);
  k_check_species<<<(int)((n_atoms + 255) / 256), 256, 0, s>>>((int)n_atoms, ctx->d_rp_species, (int)ctx->blob.S,
                                                               ctx->nb.flags);
  for (int attempt = 0; attempt < 3; ++attempt) {
    rp_launch_forces(ctx, s);
    int flags = 0, np = 0;
    cudaMemcpyAsync(&flags, ctx->nb.flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&np, ctx->nb.n_pairs, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(ctx, "pimd_init");
    if (flags & kFlagTimeout) return ctx->fail(ALLEGRO_E_TIMEOUT, "a tensor-core pass gave up a bounded wait");
    if (flags & kFlagBadSpecies) return ctx->fail(ALLEGRO_E_INVALID_ARG, "species id out of range");
    if (flags & kFlagNonfinite) return ctx->fail(ALLEGRO_E_NONFINITE, "non-finite bead position or force");
    if (!(flags & kFlagPairOverflow)) {
      ctx->rp_ready = true;
      return ALLEGRO_OK;
    }
    rc = ensure_pairs(ctx, std::max<int64_t>((int64_t)np, ctx->capacity) * 5 / 4 + 1024);
    if (rc) return rc;
    cudaMemsetAsync(ctx->nb.flags, 0, sizeof(int), s);
  }
  return ctx->fail(ALLEGRO_E_PAIR_OVERFLOW, "pair capacity could not be grown for the ring");
}

int allegro_pimd_step(allegro_ctx* ctx, double dt_fs, int32_t n_steps, double* energies) {
  if (!ctx || !ctx->rp_ready) return ctx ? ctx->fail(ALLEGRO_E_INVALID_ARG, "pimd_init first") : ALLEGRO_E_INVALID_ARG;
  if (n_steps < 0 || !(dt_fs > 0.0) || !std::isfinite(dt_fs)) return ctx->fail(ALLEGRO_E_INVALID_ARG, "bad dt or n_steps");
  if (n_steps == 0) return ALLEGRO_OK;
  ctx->md_ready = false;                             // the shared buffers now hold the ring
  int rc = ensure_records(ctx, n_steps);
  if (!rc) rc = rp_reserve(ctx);                     // other calls may have moved the shared buffers
  if (!rc && ctx->md_precision != ALLEGRO_FP32) rc = refresh_tc(ctx);
  if (rc) return rc;
  const size_t n3 = 3 * (size_t)ctx->rp_P * (size_t)ctx->rp_n;
  cudaStream_t s = ctx->stream;
  for (int attempt = 0; attempt < kMdAttempts; ++attempt) {
    if (!ctx->graph_rp || ctx->rp_graph_dt != dt_fs) {
      rc = capture_step_rp(ctx, dt_fs);
      if (rc) return rc;
    }
    cudaMemcpyAsync(ctx->d_rp_q_snap, ctx->d_rp_q, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(ctx->d_rp_v_snap, ctx->d_rp_v, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(ctx->d_rp_F_snap, ctx->d_rp_F, sizeof(float) * n3, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(ctx->nb.flags, 0, sizeof(int), s);
    cudaMemsetAsync(ctx->d_step, 0, sizeof(long long), s);
    for (int k = 0; k < n_steps; ++k)
      if (cudaGraphLaunch(ctx->graph_rp, s) != cudaSuccess) return cuda_check(ctx, "graph launch");
    int flags = 0, np = 0;
    cudaMemcpyAsync(&flags, ctx->nb.flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&np, ctx->nb.n_pairs, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(ctx, "pimd steps");
    if (flags & (kFlagPairOverflow | kFlagTimeout)) {
      cudaMemcpyAsync(ctx->d_rp_q, ctx->d_rp_q_snap, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(ctx->d_rp_v, ctx->d_rp_v_snap, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(ctx->d_rp_F, ctx->d_rp_F_snap, sizeof(float) * n3, cudaMemcpyDeviceToDevice, s);
      cudaStreamSynchronize(s);
      if (flags & kFlagTimeout) return ctx->fail(ALLEGRO_E_TIMEOUT, "a tensor-core pass gave up a bounded wait (state rolled back)");
      rc = ensure_pairs(ctx, std::max<int64_t>((int64_t)np, ctx->capacity) * 3 / 2 + 1024);
      if (rc) return rc;
      continue;
    }
    if (flags & kFlagNonfinite) {
      ctx->rp_ready = false;                         // the ring state is no longer meaningful
      return ctx->fail(ALLEGRO_E_NONFINITE, "non-finite bead position or force");
    }
    rc = copy_out(ctx, energies, ctx->d_e_rec, sizeof(double) * 3 * n_steps);
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = cuda_check(ctx, "pimd records");
    return rc;
  }
  return ctx->fail(ALLEGRO_E_PAIR_OVERFLOW, "pair capacity could not be grown during ring-polymer MD");
}

int allegro_pimd_get_state(allegro_ctx* ctx, double* positions, double* velocities) {
  if (!ctx || !ctx->rp_ready) return ctx ? ctx->fail(ALLEGRO_E_INVALID_ARG, "pimd_init first") : ALLEGRO_E_INVALID_ARG;
  const size_t bytes = sizeof(double) * 3 * (size_t)ctx->rp_P * (size_t)ctx->rp_n;
  int rc = copy_out(ctx, positions, ctx->d_rp_q, bytes);
  if (!rc) rc = copy_out(ctx, velocities, ctx->d_rp_v, bytes);
  if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = cuda_check(ctx, "pimd state");
  return rc;
}

int allegro_query(allegro_ctx* ctx, int32_t what, int64_t* value) {
  if (!ctx || !value) return ALLEGRO_E_INVALID_ARG;
  switch (what) {
    case ALLEGRO_Q_N_PAIRS: {
      int np = 0;
      if (ctx->nb.n_pairs) {
        cudaMemcpyAsync(&np, ctx->nb.n_pairs, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "query");
      }
      *value = np;
      return ALLEGRO_OK;
    }
    case ALLEGRO_Q_CAPACITY: *value = ctx->capacity; return ALLEGRO_OK;
    case ALLEGRO_Q_STEP_KERNELS: *value = ctx->graph_kernels; return ALLEGRO_OK;
    case ALLEGRO_Q_RP_STEP_KERNELS: *value = ctx->rp_graph_kernels; return ALLEGRO_OK;
    case ALLEGRO_Q_N_ATOMS: *value = ctx->n_atoms; return ALLEGRO_OK;
    case ALLEGRO_Q_N_PARAMS: *value = ctx->n_params; return ALLEGRO_OK;
    case ALLEGRO_Q_BATCH_PAIRS: *value = ctx->bt.n_pairs; return ALLEGRO_OK;
    case ALLEGRO_Q_FP32_LAUNCH:
    case ALLEGRO_Q_TANGENT_LAUNCH: {
      const Fp32Launch& f = ctx->fl[what == ALLEGRO_Q_FP32_LAUNCH ? 0 : 1];
      const int kinds[5] = {kPhA, kPhB, kPhC, kPhBT, kPhAT};
      int64_t v = 0;
      for (int q = 0; q < 5; ++q) v |= (int64_t)f.waves[kinds[q]] << (4 * q);
      *value = v;
      return ALLEGRO_OK;
    }
    case ALLEGRO_Q_REBUILDS: {
      int f[4] = {0, 0, 0, 0};
      if (ctx->d_skin_flag) {
        cudaMemcpyAsync(f, ctx->d_skin_flag, sizeof(f), cudaMemcpyDeviceToHost, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "query");
      }
      *value = f[2];
      return ALLEGRO_OK;
    }
    default: return ctx->fail(ALLEGRO_E_INVALID_ARG, "unknown query key");
  }
}

int allegro_phase_times(allegro_ctx* ctx, int32_t n_reps, double* ms_out, int32_t n_out) {
  if (!ctx || !ms_out || n_out < 7 || n_reps < 1) return ALLEGRO_E_INVALID_ARG;
  if (!ctx->md_ready) return ctx->fail(ALLEGRO_E_INVALID_ARG, "md_init first");
  KernelMarks km;
  for (auto& e : km.ev) cudaEventCreate(&e);
  cudaEvent_t e_begin, e_end;
  cudaEventCreate(&e_begin);
  cudaEventCreate(&e_end);
  double kind_ms[kPhCount] = {}, nb_ms = 0.0, f_ms = 0.0;
  double L[3] = {ctx->grid.L[0], ctx->grid.L[1], ctx->grid.L[2]};
  fill_passbufs(ctx, L);
  int rc = ALLEGRO_OK;
  for (int r = 0; r < n_reps && !rc; ++r) {
    km.n = 0;
    cudaEventRecord(e_begin, ctx->stream);
    launch_build_neighbors(ctx->nb, ctx->grid, ctx->d_pos, ctx->n_atoms, ctx->stream);
    launch_model(ctx, ctx->md_precision, ctx->stream, &km);
    cudaEventRecord(e_end, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
      rc = cuda_check(ctx, "phase times");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e_begin, km.ev[0]);
    nb_ms += ms;
    for (int i = 0; i + 1 < km.n; ++i) {
      cudaEventElapsedTime(&ms, km.ev[i], km.ev[i + 1]);
      const int kd = km.kind[i + 1];
      if (kd >= 0 && kd < kPhCount) kind_ms[kd] += ms;
    }
    cudaEventElapsedTime(&ms, km.ev[km.n - 1], e_end);
    f_ms += ms;
  }
  for (auto& e : km.ev) cudaEventDestroy(e);
  cudaEventDestroy(e_begin);
  cudaEventDestroy(e_end);
  if (rc) return rc;
  const double n = n_reps;
  const double out[9] = {nb_ms / n,
                         kind_ms[kPhA] / n,
                         (kind_ms[kPhB] + kind_ms[kPhB2]) / n,
                         kind_ms[kPhC] / n,
                         kind_ms[kPhBT] / n,
                         kind_ms[kPhAT] / n,
                         f_ms / n,
                         kind_ms[kPhB] / n,
                         kind_ms[kPhB2] / n};
  for (int k = 0; k < std::min(n_out, 9); ++k) ms_out[k] = out[k];
  return ALLEGRO_OK;
}

int allegro_md_get_state(allegro_ctx* ctx, double* positions, double* velocities, float* forces, int64_t* step) {
  if (!ctx || !ctx->md_ready) return ALLEGRO_E_INVALID_ARG;
  const size_t n3 = 3 * (size_t)ctx->n_atoms;
  int rc = copy_out(ctx, positions, ctx->d_pos, sizeof(double) * n3);
  if (!rc) rc = copy_out(ctx, velocities, ctx->d_v, sizeof(double) * n3);
  if (!rc) rc = copy_out(ctx, forces, ctx->d_F, sizeof(float) * n3);
  if (rc) return rc;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "get_state");
  if (step) *step = ctx->step;
  return ALLEGRO_OK;
}

int allegro_loss_grad(allegro_ctx* ctx, const allegro_batch* batch, double w_energy, double w_force,
                      double* loss_out, float* grad_out) {
  if (!ctx) return ALLEGRO_E_INVALID_ARG;
  int rc = check_batch(ctx, batch);
  if (!rc) rc = build_batch(ctx, batch);
  if (!rc) rc = loss_grad_impl(ctx, w_energy, w_force, loss_out);
  if (!rc) rc = copy_out(ctx, grad_out, ctx->d_grad, sizeof(float) * ctx->n_params);
  if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = cuda_check(ctx, "loss_grad");
  return rc;
}

int allegro_sam_train_step(allegro_ctx* ctx, const allegro_batch* batch, double rho, double lr, double w_energy,
                           double w_force, double* loss_out) {
  if (!ctx) return ALLEGRO_E_INVALID_ARG;
  if (!(rho >= 0.0) || !(lr >= 0.0)) return ctx->fail(ALLEGRO_E_INVALID_ARG, "rho and lr must be >= 0");
  int rc = check_batch(ctx, batch);
  if (!rc) rc = build_batch(ctx, batch);
  if (!rc) rc = loss_grad_impl(ctx, w_energy, w_force, loss_out);            // g at w
  if (rc) return rc;
  const int n = (int)ctx->n_params;
  launch_sumsq(ctx->d_grad, n, ctx->d_norm2, ctx->stream);
  launch_ascent(ctx->d_master, ctx->d_grad, n, rho, ctx->d_norm2, ctx->d_wtmp, ctx->stream);   // w' = w + rho g/|g|
  apply_flat(ctx, ctx->d_wtmp);
  rc = loss_grad_impl(ctx, w_energy, w_force, nullptr);                       // g' at w' (same batch)
  if (rc) {
    apply_flat(ctx, ctx->d_master);
    return rc;
  }
  ctx->adam_t += 1;
  launch_adam(ctx->d_master, ctx->d_grad, ctx->d_adam_m, ctx->d_adam_v, n, lr, ctx->adam_t, ctx->stream);
  apply_flat(ctx, ctx->d_master);
  ctx->drop_graphs();
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "sam step");
  return ALLEGRO_OK;
}

int allegro_loss_scan(allegro_ctx* ctx, const allegro_batch* batch, const float* dirs, int64_t dir_stride,
                      const double* scales, int32_t n_points, double w_energy, double w_force, double* losses_out) {
  if (!ctx) return ALLEGRO_E_INVALID_ARG;
  if (!dirs || !scales || !losses_out || n_points < 1 || dir_stride < 0)
    return ctx->fail(ALLEGRO_E_INVALID_ARG, "loss_scan: dirs, scales, losses_out and n_points >= 1 are required");
  if (!is_device_ptr(dirs)) return ctx->fail(ALLEGRO_E_INVALID_ARG, "loss_scan: dirs must be device memory");
  if (ctx->blob.L > 2) return ctx->fail(ALLEGRO_E_UNSUPPORTED, "training is built for models of at most two layers");
  int rc = check_batch(ctx, batch);
  if (!rc) rc = build_batch(ctx, batch);
  if (!rc) rc = init_master(ctx);
  if (rc) return rc;
  const int n = (int)ctx->n_params;
  cudaStream_t s = ctx->stream;
  cudaMemsetAsync(ctx->nb.flags, 0, sizeof(int), s);
  for (int k = 0; k < n_points && !rc; ++k) {
    launch_axpy(ctx->d_master, dirs + (size_t)k * (size_t)dir_stride, scales[k], n, ctx->d_wtmp, s);
    apply_flat(ctx, ctx->d_wtmp);
    batch_forward_loss(ctx, w_energy, w_force);
    cudaMemcpyAsync(&losses_out[k], ctx->bt.loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = cuda_check(ctx, "loss_scan");
  }
  apply_flat(ctx, ctx->d_master);                      // the context's weights are unchanged
  ctx->drop_graphs();
  int flags = 0;
  cudaMemcpyAsync(&flags, ctx->nb.flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return rc ? rc : cuda_check(ctx, "loss_scan");
  if (rc) return rc;
  if (flags & kFlagTimeout) return ctx->fail(ALLEGRO_E_TIMEOUT, "a pass gave up a bounded wait");
  if (flags & kFlagPairOverflow) return ctx->fail(ALLEGRO_E_PAIR_OVERFLOW, "training batch exceeds the pair capacity");
  return ALLEGRO_OK;
}

int allegro_get_weights(allegro_ctx* ctx, float* out, int64_t n) {
  if (!ctx || !out) return ALLEGRO_E_INVALID_ARG;
  if (n != ctx->n_params) return ctx->fail(ALLEGRO_E_INVALID_ARG, "n must equal the parameter count");
  int rc = init_master(ctx);
  if (!rc) rc = copy_out(ctx, out, ctx->d_master, sizeof(float) * n);
  if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = cuda_check(ctx, "get_weights");
  return rc;
}

int allegro_set_weights(allegro_ctx* ctx, const float* in, int64_t n) {
  if (!ctx || !in) return ALLEGRO_E_INVALID_ARG;
  if (n != ctx->n_params) return ctx->fail(ALLEGRO_E_INVALID_ARG, "n must equal the parameter count");
  int rc = init_master(ctx);
  if (rc) return rc;
  const cudaMemcpyKind k = is_device_ptr(in) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyAsync(ctx->d_master, in, sizeof(float) * n, k, ctx->stream);
  cudaMemsetAsync(ctx->d_adam_m, 0, sizeof(float) * n, ctx->stream);     // new start: fresh Adam moments
  cudaMemsetAsync(ctx->d_adam_v, 0, sizeof(float) * n, ctx->stream);
  ctx->adam_t = 0;
  apply_flat(ctx, ctx->d_master);
  ctx->drop_graphs();
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check(ctx, "set_weights");
  return ALLEGRO_OK;
}

int allegro_selftest_silu(int64_t n, const float* x, float* y) {
  if (n < 0 || n > (int64_t)1 << 30 || (n > 0 && (!x || !y))) return ALLEGRO_E_INVALID_ARG;
  return al::bf16_silu_probe((int)n, x, y) == 0 ? ALLEGRO_OK : ALLEGRO_E_CUDA;
}

int allegro_debug_inject_wait_timeout(int32_t enable) {
  return al::bf16_inject_wait_timeout(enable) == 0 ? ALLEGRO_OK : ALLEGRO_E_CUDA;
}

}  // extern "C"
