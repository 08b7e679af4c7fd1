// umma.cuh - Blackwell (sm_100 family) tensor-core building blocks in inline
// PTX: tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation in TMEM),
// shared-memory matrix descriptors for K-major 128-byte-swizzled tiles,
// TMEM allocation and loads, mbarriers with bounded waits, and 1-D bulk
// copies (cp.async.bulk) from global to shared memory and back.
//
// Operand layout ("SW128 K-major"): a [R x K] bf16 tile (R % 8 == 0) is split
// into K-blocks of 64 elements (128 bytes per row); block b occupies R * 128
// bytes; inside it row r lives at (r / 8) * 1024 + (r % 8) * 128 and its 16-byte
// chunk c is stored at chunk position c ^ (r % 8).  Tiles start on 1024-byte
// boundaries.  One MMA consumes 16 K-elements (32 bytes), i.e. a quarter of a
// block row; successive MMAs advance the descriptor start address by 32 bytes
// inside a block and by R * 128 bytes across blocks.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#define UM_DEV __device__ __forceinline__

namespace al {
namespace umma {

UM_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) in an SW128 K-major bf16 tile with R rows.
__host__ __device__ inline uint32_t sw128_off(int r, int k, int R) {
  const int kb = k >> 6, kk = k & 63;
  const int chunk = kk >> 3;
  return (uint32_t)(kb * (R * 128) + (r >> 3) * 1024 + (r & 7) * 128 + ((chunk ^ (r & 7)) << 4) +
                    ((kk & 7) << 1));
}

// Bytes of an SW128 tile with R rows and K columns (K rounded up to 64).
__host__ __device__ constexpr uint32_t sw128_bytes(int R, int K) {
  return (uint32_t)(((K + 63) / 64) * R * 128);
}

// Shared-memory matrix descriptor: start address, leading-byte offset 16
// (unused for swizzled K-major), stride-byte offset 1024 (8 rows x 128 B),
// descriptor version 1, layout SWIZZLE_128B (2).
UM_DEV uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Descriptor of an SW128 tile used as an MN-major operand: the K-major image
// of a [P x Q] matrix (rows P, 128-byte rows along Q) read as an operand whose
// MN dimension is Q and K dimension is P.  Swizzle atoms are 8 rows (K) x 64
// elements (MN); lbo = byte stride between atoms along MN (one 64-column
// block of the image, P * 128 bytes), sbo = 1024 between atoms along K.
UM_DEV uint64_t desc_sw128_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A BF16 (bits 7-9
// = 1), B BF16 (bits 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
// Same with the operand type selectable: fmt 1 = BF16, 0 = FP16 (both
// operands alike, as kind::f16 requires).
__host__ __device__ constexpr uint32_t idesc_f16kind(int M, int N, bool b_mn_major, uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (b_mn_major ? (1u << 16) : 0u) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool b_mn_major = false) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (b_mn_major ? (1u << 16) : 0u) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

UM_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
UM_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
UM_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// ---- TMEM (one warp executes alloc / dealloc) ----
UM_DEV void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
UM_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- mbarriers ----
UM_DEV void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
UM_DEV void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
UM_DEV void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(m)), "r"(bytes)
               : "memory");
}
UM_DEV bool mbar_try_wait(uint64_t* m, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Bounded wait (by default about 2^31 clock cycles, ~1 s): returns false and
// leaves the barrier alone if the phase never completes; the caller records
// an error.
UM_DEV bool mbar_wait(uint64_t* m, uint32_t phase, long long limit = 1ll << 31) {
  const long long t0 = clock64();
  while (!mbar_try_wait(m, phase)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// ---- bulk copy global -> shared (16-byte aligned, size % 16 == 0) ----
UM_DEV void bulk_g2s(void* smem, const void* gmem, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(smem)),
      "l"(gmem), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

// ---- bulk copy shared -> global (16-byte aligned, size % 16 == 0) ----
// Completion through bulk groups: commit after the copies, then wait until
// their shared-memory sources have been read (the source may be rewritten)
// or until the writes are done.  Neither wait depends on another thread.
UM_DEV void bulk_s2g(void* gmem, const void* smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gmem), "r"(smem_u32(smem)),
               "r"(bytes)
               : "memory");
}
UM_DEV void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
UM_DEV void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
UM_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// Hint only: bring [gmem, gmem + bytes) into L2 (16-byte aligned, bytes a
// multiple of 16); nothing waits for it.
UM_DEV void bulk_prefetch_l2(const void* gmem, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}

// ---- MMA ----
UM_DEV void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
      : "memory");
}
UM_DEV void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

// Issue D[128 x N] (+)= A[128 x K] * B[N x K]^T for K = 16 * nk (single thread).
UM_DEV void mma_tile(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int N, int nk, bool accumulate) {
  const uint32_t idesc = idesc_bf16(128, N);
  for (int k = 0; k < nk; ++k) {
    const uint32_t aoff = (uint32_t)((k >> 2) * (128 * 128) + (k & 3) * 32);
    const uint32_t boff = (uint32_t)((k >> 2) * (N * 128) + (k & 3) * 32);
    mma_bf16(d_tmem, desc_sw128(a_saddr + aoff), desc_sw128(b_saddr + boff), idesc,
             (accumulate || k > 0) ? 1u : 0u);
  }
}

// Issue D[128 x N] (+)= A[128 x K] * W[K x N] where the B operand is the
// K-major image of W^T... i.e. the image of a [K x N] matrix W stored with K
// rows of N elements (the forward image of a layer whose output dim is K):
// MN-major B, N = number of image columns, K = number of image rows (P).
UM_DEV void mma_tile_bmn(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int N, int P, int nk,
                         bool accumulate, bool swap_lbo_sbo) {
  const uint32_t idesc = idesc_bf16(128, N, true);
  const uint32_t lbo = swap_lbo_sbo ? 1024u : (uint32_t)(P * 128);
  const uint32_t sbo = swap_lbo_sbo ? (uint32_t)(P * 128) : 1024u;
  for (int k = 0; k < nk; ++k) {
    const uint32_t aoff = (uint32_t)((k >> 2) * (128 * 128) + (k & 3) * 32);
    const uint32_t boff = (uint32_t)(k * 16 * 128);   // 16 image rows per MMA
    mma_bf16(d_tmem, desc_sw128(a_saddr + aoff), desc_sw128_mn(b_saddr + boff, lbo, sbo), idesc,
             (accumulate || k > 0) ? 1u : 0u);
  }
}

// tcgen05.wait::ld with the loaded registers tied to it (in/out operands): no
// use of them can be scheduled before the wait.  TMEM loads touch no generic
// memory, so the wait carries no memory clobber and ordinary loads and stores
// may be scheduled across it.
template <int N>
UM_DEV void tmem_wait_tied(uint32_t* r) {
  static_assert(N % 8 == 0, "groups of 8");
#pragma unroll
  for (int g = 0; g < N; g += 8) {
    if (g == 0)
      asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                   : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
    else
      asm volatile("" : "+r"(r[g]), "+r"(r[g + 1]), "+r"(r[g + 2]), "+r"(r[g + 3]), "+r"(r[g + 4]), "+r"(r[g + 5]),
                   "+r"(r[g + 6]), "+r"(r[g + 7]));
  }
}

// ---- TMEM -> registers: 32 lanes x 32 columns (thread t of the warp gets
// lane base + t, registers = consecutive columns) ----
UM_DEV void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  tmem_wait_tied<32>(r);
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

UM_DEV void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  tmem_wait_tied<16>(r);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 4 columns without waiting: the caller issues several loads and then calls
// tmem_wait4 on each group; the first wait waits for all of them, and tying
// the registers to it keeps every use of them after the wait.
UM_DEV void tmem_ld4_raw(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
UM_DEV void tmem_ld2_raw(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
}
// 6 consecutive columns (x4 + x2, so that no column past the 6th is read)
UM_DEV void tmem_ld6(uint32_t taddr, float* v) {
  uint32_t r[6];
  tmem_ld4_raw(taddr, r);
  tmem_ld2_raw(taddr + 4, r + 4);
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]));
#pragma unroll
  for (int j = 0; j < 6; ++j) v[j] = __uint_as_float(r[j]);
}
UM_DEV void tmem_wait4(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]));
}

UM_DEV void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
  tmem_wait_tied<8>(r);
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// registers -> TMEM (thread t of the warp writes lane base + t); the caller
// waits with tmem_wait_st before the columns are read by an MMA
UM_DEV void tmem_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
      "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
      "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31]));
}
UM_DEV void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]));
}
UM_DEV void tmem_st4(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(taddr), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]));
}
UM_DEV void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// Pack 8 floats as bf16 (round to nearest even) and store 16 bytes.
UM_DEV void st_bf16x8(uint8_t* tile, uint32_t off, const float* v) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t lo = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * q]));
    const uint32_t hi = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * q + 1]));
    w[q] = lo | (hi << 16);
  }
  *reinterpret_cast<uint4*>(tile + off) = make_uint4(w[0], w[1], w[2], w[3]);
}

}  // namespace umma
}  // namespace al
