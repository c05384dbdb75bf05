// Exact integer matrix product on the tensor cores: the engine of the block algorithm
// (Algorithm 2, "T = (E_s A_s)(B_s F_s) -- matrix product over Z", Section IV-A).
//
// Operands arrive as balanced base-256 digit planes: X = sum_t 256^t X_t with X_t in [-128, 127],
// stored as BF16 (every such integer is exact in BF16).  The product is
//
//     T = sum_d 256^d D_d,    D_d = sum_{j + l = d} X_j Y_l          ("diagonal" d),
//
// and every digit product is exact.  One CTA owns a 128 x 128 output tile and a contiguous range of
// diagonals.  For each diagonal it runs tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 in TMEM) over
// the pairs (j, l) and the inner dimension in chains of at most 256 products, so every partial sum
// is an integer of magnitude <= 2^22 and exact in FP32.  Each finished chain is drained from TMEM:
// adding 1.5 * 2^23 maps the FP32 integer x (|x| <= 2^22) to a float whose bit pattern is
// 0x4B400000 + x, so one FADD and one IADD move it into a per-output int32 running sum R.  At the end
// of diagonal d the low byte of R is digit d of T (written to global memory) and R >>= 8 carries the
// rest into diagonal d + 1; |R| stays below 2^29, so int32 never overflows.  The CTA finally writes
// R, the carry into its first diagonal past the range.
//
// Roles (320 threads): warp 0 issues TMA loads into a 6-stage shared-memory ring, warp 1 issues the
// MMAs (one elected lane) and owns the TMEM allocation (two 128-column FP32 accumulators, so one
// chain drains while the next accumulates), warps 2..9 drain (each thread one TMEM lane = one output
// row, 64 of the tile's 128 columns).  Every wait on an mbarrier gives up after ~2 s of wall time,
// sets ARBGPU_ERR_TIMEOUT and makes the CTA leave cleanly.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace arbgpu {

constexpr int TG_BM = 128;
constexpr int TG_BN = 128;
constexpr int TG_BK = 64;  // BF16 elements per k-block: one 128-byte swizzle row
constexpr int TG_STAGES = 6;
constexpr int TG_CHAIN_KB = 4;  // 4 k-blocks = 256 products per accumulation chain
constexpr int TG_EPI_WARPS = 8;
constexpr int TG_THREADS = 32 * (2 + TG_EPI_WARPS);
constexpr int TG_MAXG = 96;
constexpr int TG_TILE_BYTES = TG_BM * TG_BK * 2;  // 16 KiB per operand tile
constexpr int TG_TMEM_COLS = 256;
constexpr uint32_t TG_MAGIC_BITS = 0x4B400000u;   // bit pattern of 1.5 * 2^23
constexpr float TG_MAGIC = 12582912.0f;
constexpr size_t TG_SMEM_BYTES = 1024 + (size_t)TG_STAGES * 2 * TG_TILE_BYTES + 256;

struct DigitGemmParams {
  int M, N, Kp;   // Kp: inner dimension, a multiple of TG_BK (zero padded)
  int SA, SB;     // digit counts of the two operands
  int ND;         // SA + SB - 1 diagonals
  int tiles_m, tiles_n, groups;
  int dstart[TG_MAXG + 1];  // diagonal range of group g: [dstart[g], dstart[g+1])
  uint8_t *digits;          // [ND][Mp][Np] digit bytes of T
  int32_t *carries;         // [groups][Mp][Np] carry out of each group's last diagonal
  int64_t Mp, Np;           // padded leading sizes (multiples of the tile)
  int batch;                // independent products: item b uses planes [b*SA, (b+1)*SA) of A,
                            // [b*SB, (b+1)*SB) of B, and its own digits / carries
  int ipc;                  // batch items per CTA (consecutive, run back to back)
  int *status;
  // Multimodular mode (2 x 2 digits, one group): instead of digits and carries, item b writes
  // P_b mod m_b of its exact product P_b to zout[b][Mp][Np] (uint16).
  uint16_t *zout;
  int nz;                   // items [0, nz) are reduced; items [nz, batch) write P itself to zraw
  int64_t *zraw;            // [batch - nz][Mp][Np]
  const uint32_t *ztab;     // [batch][4]: m_b, m_b and 1 / m_b as float bits, unused
  const uint64_t *zinv;     // [batch]: floor((2^64 - 1) / m_b)
};

// Tensor map for TMA stores into BF16 planes [planes][rows][Kp] (no swizzle), box
// box_k x box_rows x box_planes (box_k * 2 bytes a multiple of 16, every box side <= 256).
bool make_residue_store_map(CUtensorMap *tm, void *base, int64_t Kp, int64_t rows, int64_t planes,
                            int box_k, int box_rows, int box_planes);

// Tensor map for TMA loads of 16-bit residue planes [planes][Mp][Np]: box 128 x 1 x box_planes
// (128 consecutive columns of one row, every plane).
bool make_z_load_map(CUtensorMap *tm, const void *base, int64_t Np, int64_t Mp, int64_t planes,
                     int box_planes);

// ------------------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `bar` with parity `parity`; false after ~2 s or when *abort is set.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (*abort) return false;
      if (global_ns() - t0 > 2000000000ull) return false;
    }
  }
}

// try_wait with a suspend-time hint: the thread may sleep up to `ns` nanoseconds for the phase.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// mbar_wait for waits that are often long: each poll sleeps up to 20 us (the thread wakes when
// the phase completes), so waiting warps take few issue slots.  False after ~2 s.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait_hint(bar, parity, 20000u)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait_hint(bar, parity, 20000u)) return true;
    if (global_ns() - t0 > 2000000000ull) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)tm) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulator.
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on `bar` once every previously issued MMA of this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with 128-byte swizzling:
// rows of 128 bytes, 8-row atoms of 1024 bytes (stride byte offset), version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

}  // namespace arbgpu
