// Host side of the tensor-core digit GEMM: TMA descriptors, diagonal-group schedule, launch.
#include <cstdio>
#include <mutex>

#include "internal.h"
#include <cstdlib>
#include <cstring>

#include "tc_gemm.cuh"

namespace arbgpu {

// ------------------------------------------------------------------------------ the kernel

struct TgShared {
  uint64_t full[TG_STAGES];
  uint64_t empty[TG_STAGES];
  uint64_t accf[2];
  uint64_t acce[2];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

__global__ void __launch_bounds__(TG_THREADS, 1)
    digit_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ DigitGemmParams P) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *tiles = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = tiles;
  uint8_t *sB = tiles + (size_t)TG_STAGES * TG_TILE_BYTES;
  TgShared *sh = (TgShared *)(tiles + (size_t)TG_STAGES * 2 * TG_TILE_BYTES);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int ntiles = P.tiles_m * P.tiles_n;
  const int tile = blockIdx.x % ntiles;
  const int group = (blockIdx.x / ntiles) % P.groups;
  // batch items [b_first, b_last) run one after the other in this CTA, their pipelines back to back
  const int bchunk = blockIdx.x / (ntiles * P.groups);
  const int b_first = bchunk * P.ipc;
  const int b_last = min(P.batch, b_first + P.ipc);
  const int mt = tile / P.tiles_n, nt = tile % P.tiles_n;
  const int m0 = mt * TG_BM, n0 = nt * TG_BN;
  const int d0 = P.dstart[group], d1 = P.dstart[group + 1];
  const int nkb = P.Kp / TG_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TG_STAGES; ++s) {
      mbar_init(&sh->full[s], 1);
      mbar_init(&sh->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh->accf[b], 1);
      mbar_init(&sh->acce[b], TG_EPI_WARPS);
    }
    mbar_init(&sh->done, 1);
    sh->abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&sh->tmem_base, TG_TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;
  volatile int *abort = &sh->abort;

  auto give_up = [&]() {
    *abort = 1;
    set_status(P.status, ARBGPU_ERR_TIMEOUT);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      uint32_t item = 0;
      bool ok = true;
      for (int bi = b_first; bi < b_last && ok; ++bi)
      for (int d = d0; d < d1 && ok; ++d) {
        const int zA = bi * P.SA, zB = bi * P.SB;  // the item's first digit planes
        const int jlo = max(0, d - (P.SB - 1)), jhi = min(d, P.SA - 1);
        for (int j = jlo; j <= jhi && ok; ++j) {
          const int l = d - j;
          for (int kb = 0; kb < nkb; ++kb, ++item) {
            const int s = item % TG_STAGES;
            const uint32_t ph = (item / TG_STAGES) & 1;
            if (!mbar_wait(&sh->empty[s], ph ^ 1, abort)) {
              give_up();
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&sh->full[s], 2 * TG_TILE_BYTES);
            tma_load_3d(sA + (size_t)s * TG_TILE_BYTES, &tmA, &sh->full[s], kb * TG_BK, m0,
                        zA + j);
            tma_load_3d(sB + (size_t)s * TG_TILE_BYTES, &tmB, &sh->full[s], kb * TG_BK, n0,
                        zB + l);
          }
        }
      }
      // before leaving, let every load this thread issued land (bounded)
      const uint32_t first = item > (uint32_t)TG_STAGES ? item - TG_STAGES : 0;
      for (uint32_t it = first; it < item; ++it)
        mbar_wait(&sh->full[it % TG_STAGES], (it / TG_STAGES) & 1, abort);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(TG_BM, TG_BN);
      uint32_t item = 0, chain = 0;
      bool ok = true;
      for (int bi = b_first; bi < b_last && ok; ++bi)
      for (int d = d0; d < d1 && ok; ++d) {
        const int jlo = max(0, d - (P.SB - 1)), jhi = min(d, P.SA - 1);
        int kbc = 0;
        for (int j = jlo; j <= jhi && ok; ++j) {
          for (int kb = 0; kb < nkb; ++kb, ++item) {
            const uint32_t buf = chain & 1;
            if (kbc == 0) {  // start of a chain: the accumulator must have been drained
              if (!mbar_wait(&sh->acce[buf], ((chain >> 1) & 1) ^ 1, abort)) {
                give_up();
                ok = false;
                break;
              }
              tc_fence_after();
            }
            const int s = item % TG_STAGES;
            if (!mbar_wait(&sh->full[s], (item / TG_STAGES) & 1, abort)) {
              give_up();
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t ad = sw128_desc(smem_u32(sA + (size_t)s * TG_TILE_BYTES));
            const uint64_t bd = sw128_desc(smem_u32(sB + (size_t)s * TG_TILE_BYTES));
#pragma unroll
            for (int kk = 0; kk < TG_BK / 16; ++kk)
              umma_bf16(tmem + buf * TG_BN, ad + 2 * kk, bd + 2 * kk, idesc,
                        (kbc > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&sh->empty[s]);
            ++kbc;
            const bool diag_end = (j == jhi) && (kb == nkb - 1);
            if (kbc == TG_CHAIN_KB || diag_end) {
              umma_commit(&sh->accf[buf]);
              ++chain;
              kbc = 0;
            }
          }
        }
      }
      umma_commit(&sh->done);
      mbar_wait(&sh->done, 0, abort);
    }
  } else {
    // ------------------------------------------------------------ drain / carry epilogue
    const int q = warp & 3;             // TMEM lane quadrant this warp may access
    const int half = (warp - 2) >> 2;   // which 64 of the tile's 128 columns
    const int row = 32 * q + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(half * 64);
    const int64_t gm = m0 + row;
    const int64_t gcol = n0 + half * 64;
    uint32_t chain = 0;
    bool ok = true;
    const bool zmode = P.zout != nullptr;  // d0 = 0, d1 = 3 in this mode
    for (int bi = b_first; bi < b_last && ok; ++bi) {
    uint8_t *const out_digits = P.digits + (int64_t)bi * P.ND * P.Mp * P.Np;
    int32_t *const out_carries = P.carries + (int64_t)bi * P.groups * P.Mp * P.Np;
    int32_t R[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) R[c] = 0;
    uint32_t zp[3][16];                     // its three digit bytes per column, packed
    for (int d = d0; d < d1 && ok; ++d) {
      const int jlo = max(0, d - (P.SB - 1)), jhi = min(d, P.SA - 1);
      const int nchains_d = ((jhi - jlo + 1) * nkb + TG_CHAIN_KB - 1) / TG_CHAIN_KB;
      // chains never straddle a pair boundary when nkb is a multiple of TG_CHAIN_KB; in general a
      // chain ends every TG_CHAIN_KB k-blocks or at the end of the diagonal
      for (int cc = 0; cc < nchains_d; ++cc, ++chain) {
        const uint32_t buf = chain & 1;
        // every lane waits, then the warp agrees, so the .sync.aligned TMEM loads run converged
        const bool got = __all_sync(0xffffffffu, mbar_wait(&sh->accf[buf], (chain >> 1) & 1, abort));
        if (!got) {
          if (lane == 0) give_up();
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t v[32];
        tmem_ld32(lane_addr + buf * TG_BN, v);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; ++c)
          R[c] += (int32_t)(__float_as_uint(__uint_as_float(v[c]) + TG_MAGIC) - TG_MAGIC_BITS);
        tmem_ld32(lane_addr + buf * TG_BN + 32, v);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; ++c)
          R[32 + c] +=
              (int32_t)(__float_as_uint(__uint_as_float(v[c]) + TG_MAGIC) - TG_MAGIC_BITS);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh->acce[buf]);
      }
      if (!ok) break;
      // digit d of T: the low byte of R; carry the rest
      uint32_t packed[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        packed[c] = ((uint32_t)(R[4 * c] & 255)) | ((uint32_t)(R[4 * c + 1] & 255) << 8) |
                    ((uint32_t)(R[4 * c + 2] & 255) << 16) | ((uint32_t)(R[4 * c + 3] & 255) << 24);
      }
#pragma unroll
      for (int c = 0; c < 64; ++c) R[c] >>= 8;
      if (zmode) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          if (d == 0) zp[0][c] = packed[c];
          if (d == 1) zp[1][c] = packed[c];
          if (d == 2) zp[2][c] = packed[c];
        }
        continue;
      }
      uint4 *dst = (uint4 *)(out_digits + ((int64_t)d * P.Mp + gm) * P.Np + gcol);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        dst[c] = make_uint4(packed[4 * c], packed[4 * c + 1], packed[4 * c + 2], packed[4 * c + 3]);
    }
    if (zmode) {
      if (ok) {
        // P = bytes + R 2^24 exactly; |P| <= Kp (m / 2)^2 < 2^50, so P + m 2^35 is in (0, 2^52)
        const uint32_t m = __ldg(P.ztab + 4 * bi);
        const uint64_t i64 = __ldg(P.zinv + bi);
        uint32_t zz[32];
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int sh = 8 * (c & 3);
          const int64_t pv = (int64_t)((zp[0][c >> 2] >> sh) & 255u) |
                             ((int64_t)((zp[1][c >> 2] >> sh) & 255u) << 8) |
                             ((int64_t)((zp[2][c >> 2] >> sh) & 255u) << 16) |
                             ((int64_t)R[c] * (int64_t)(1 << 24));
          const uint64_t x = (uint64_t)(pv + ((int64_t)m << 35));
          uint64_t r = x - __umul64hi(x, i64) * m;
          while (r >= m) r -= m;
          const uint32_t z = (uint32_t)r;
          if (c & 1)
            zz[c >> 1] |= z << 16;
          else
            zz[c >> 1] = z;
        }
        uint4 *zdst = (uint4 *)(P.zout + ((int64_t)bi * P.Mp + gm) * P.Np + gcol);
#pragma unroll
        for (int c = 0; c < 8; ++c)
          zdst[c] = make_uint4(zz[4 * c], zz[4 * c + 1], zz[4 * c + 2], zz[4 * c + 3]);
      }
    } else if (ok) {
      int4 *cdst = (int4 *)(out_carries + ((int64_t)group * P.Mp + gm) * P.Np + gcol);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        cdst[c] = make_int4(R[4 * c], R[4 * c + 1], R[4 * c + 2], R[4 * c + 3]);
    }
    }  // batch items
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, TG_TMEM_COLS);
  }
}

// ------------------------------------------------------------------------ multimodular kernel
//
// The residue products of the multimodular engine (2 x 2 balanced digits per modulus, K <= 1024).
// A work item is one modulus and one 128 x 64 output tile.  Every k-block stage holds A0, A1 (the
// two digit planes of the left residues, 128 rows) and B0 | B1 (64 rows each) stacked into one
// 128-row operand, and two MMAs of 128 x 128 x 16 per k-step write A0 B0 | A0 B1 | A1 B0 | A1 B1
// into four 64-column quarters of one of two 256-column TMEM accumulators, so the drain of an
// item overlaps the MMAs of the next (one chain over the whole K: |sum| <= K 2^14 <= 2^24 stays
// exact in FP32).  Sixteen drain warps (4 lane quadrants x 4 groups of 16 columns) form
// P = D0 + 2^8 D1 + 2^16 D2 exactly and write P mod m per entry, as the general kernel's
// multimodular mode does; items of the raw kind write P itself.

constexpr int CG_STAGES = 4;
constexpr int CG_BN = 64;                              // output columns per item
constexpr int CG_B_TILE = CG_BN * TG_BK * 2;           // 8 KiB: one B digit plane of a k-block
constexpr int CG_STAGE_BYTES = 2 * TG_TILE_BYTES + 2 * CG_B_TILE;  // A0, A1, B0, B1
constexpr size_t CG_SMEM_BYTES = 1024 + (size_t)CG_STAGES * CG_STAGE_BYTES + 256;
constexpr int CG_ACC_COLS = 4 * CG_BN;                 // one accumulator: four quarters
constexpr int CG_TMEM_COLS = 2 * CG_ACC_COLS;
constexpr int CG_MAX_KP = 1024;
constexpr int CG_EPI_WARPS = 16;  // 4 lane quadrants x 4 groups of 16 columns
constexpr int CG_THREADS = 32 * (2 + CG_EPI_WARPS);

struct CgShared {
  uint64_t full[CG_STAGES];
  uint64_t empty[CG_STAGES];
  uint64_t accf[2], acce[2], done;
  uint32_t tmem_base;
  int abort;
};

__global__ void __launch_bounds__(CG_THREADS, 1)
    crt_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ DigitGemmParams P) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *stages = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  CgShared *sh = (CgShared *)(stages + (size_t)CG_STAGES * CG_STAGE_BYTES);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // persistent: work item w = (modulus w / ntiles, output tile w % ntiles), a grid stride apart
  const int tiles_n = (int)(P.Np / CG_BN);
  const int ntiles = P.tiles_m * tiles_n;
  const int nitems = ntiles * P.batch;
  const int nkb = P.Kp / TG_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < CG_STAGES; ++s) {
      mbar_init(&sh->full[s], 1);
      mbar_init(&sh->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh->accf[b], 1);
      mbar_init(&sh->acce[b], CG_EPI_WARPS);
    }
    mbar_init(&sh->done, 1);
    sh->abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&sh->tmem_base, CG_TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // the residue planes come from the kernels before this one
  const uint32_t tmem = sh->tmem_base;
  volatile int *abort = &sh->abort;
  auto give_up = [&]() {
    *abort = 1;
    set_status(P.status, ARBGPU_ERR_TIMEOUT);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      uint32_t it = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
        const int bi = w / ntiles, tile = w - bi * ntiles;
        const int m0 = (tile / tiles_n) * TG_BM, n0 = (tile % tiles_n) * CG_BN;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % CG_STAGES;
          if (!mbar_wait(&sh->empty[s], ((it / CG_STAGES) & 1) ^ 1, abort)) {
            give_up();
            ok = false;
            break;
          }
          uint8_t *st = stages + (size_t)s * CG_STAGE_BYTES;
          mbar_arrive_expect_tx(&sh->full[s], CG_STAGE_BYTES);
          tma_load_3d(st, &tmA, &sh->full[s], kb * TG_BK, m0, 2 * bi);
          tma_load_3d(st + TG_TILE_BYTES, &tmA, &sh->full[s], kb * TG_BK, m0, 2 * bi + 1);
          tma_load_3d(st + 2 * TG_TILE_BYTES, &tmB, &sh->full[s], kb * TG_BK, n0, 2 * bi);
          tma_load_3d(st + 2 * TG_TILE_BYTES + CG_B_TILE, &tmB, &sh->full[s], kb * TG_BK, n0,
                      2 * bi + 1);
        }
      }
      // before leaving, let every load this thread issued land (bounded)
      const uint32_t first = it > (uint32_t)CG_STAGES ? it - CG_STAGES : 0;
      for (uint32_t q = first; q < it; ++q)
        mbar_wait(&sh->full[q % CG_STAGES], (q / CG_STAGES) & 1, abort);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(TG_BM, 2 * CG_BN);
      uint32_t it = 0;
      bool ok = true;
      for (int w = blockIdx.x, ii = 0; w < nitems && ok; w += gridDim.x, ++ii) {
        const int b = ii & 1;
        // the drain must have read this accumulator's previous item
        if (!mbar_wait(&sh->acce[b], ((ii >> 1) & 1) ^ 1, abort)) {
          give_up();
          break;
        }
        tc_fence_after();
        const uint32_t acc_cols = tmem + (uint32_t)(b * CG_ACC_COLS);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % CG_STAGES;
          if (!mbar_wait(&sh->full[s], (it / CG_STAGES) & 1, abort)) {
            give_up();
            ok = false;
            break;
          }
          tc_fence_after();
          uint8_t *st = stages + (size_t)s * CG_STAGE_BYTES;
          const uint64_t a0 = sw128_desc(smem_u32(st));
          const uint64_t a1 = sw128_desc(smem_u32(st + TG_TILE_BYTES));
          const uint64_t bd = sw128_desc(smem_u32(st + 2 * TG_TILE_BYTES));
#pragma unroll
          for (int kk = 0; kk < TG_BK / 16; ++kk) {
            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
            umma_bf16(acc_cols, a0 + 2 * kk, bd + 2 * kk, idesc, acc);               // A0 B0 | A0 B1
            umma_bf16(acc_cols + 2 * CG_BN, a1 + 2 * kk, bd + 2 * kk, idesc, acc);   // A1 B0 | A1 B1
          }
          umma_commit(&sh->empty[s]);
        }
        if (ok) umma_commit(&sh->accf[b]);
      }
      umma_commit(&sh->done);
      mbar_wait(&sh->done, 0, abort);
    }
  } else {
    // ------------------------------------------------------------ drain: P mod m per entry
    const int q = warp & 3;                           // TMEM lane quadrant this warp may access
    const int col0 = 16 * ((warp - 2) >> 2);          // its 16 of the item's 64 columns
    const int row = 32 * q + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col0;
    for (int w = blockIdx.x, ii = 0; w < nitems; w += gridDim.x, ++ii) {
      const int bi = w / ntiles, tile = w - bi * ntiles;
      const int b = ii & 1;
      const int64_t gm = (tile / tiles_n) * TG_BM + row;
      const int64_t gcol = (tile % tiles_n) * CG_BN + col0;
      const bool got = __all_sync(0xffffffffu, mbar_wait(&sh->accf[b], (ii >> 1) & 1, abort));
      if (!got) {
        if (lane == 0) give_up();
        break;
      }
      tc_fence_after();
      // P = D0 + 2^8 (D1a + D1b) + 2^16 D2 from the quarters A0 B0 | A0 B1 | A1 B0 | A1 B1
      const uint32_t base = lane_addr + (uint32_t)(b * CG_ACC_COLS);
      uint32_t v0[16], v1[16], v2[16], v3[16];
      tmem_ld16(base, v0);
      tmem_ld16(base + CG_BN, v1);
      tmem_ld16(base + 2 * CG_BN, v2);
      tmem_ld16(base + 3 * CG_BN, v3);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh->acce[b]);
      if (bi >= P.nz) {  // a raw item: P itself
        longlong2 *rdst =
            (longlong2 *)(P.zraw + ((int64_t)(bi - P.nz) * P.Mp + gm) * P.Np + gcol);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          int64_t pc[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int cc = 2 * c + u;
            const int64_t d1 = (int64_t)__float2int_rn(__uint_as_float(v1[cc])) +
                               __float2int_rn(__uint_as_float(v2[cc]));
            pc[u] = (int64_t)__float2int_rn(__uint_as_float(v0[cc])) + d1 * 256 +
                    (int64_t)__float2int_rn(__uint_as_float(v3[cc])) * 65536;
          }
          rdst[c] = make_longlong2(pc[0], pc[1]);
        }
        continue;
      }
      // P mod m by Horner's rule in FP32, every step exact: the quarters D0, D1a, D1b, D2 are
      // exact integers of magnitude <= Kp 2^14 <= 2^24; bal(x) = x - m rint(x / m) has
      // |bal(x)| <= m / 2 + 2 (the quotient from x (1 / m) can miss a half-way point by one);
      // then u = bal(bal(D2) 256 + bal(D1a) + bal(D1b)) and z = bal(u 256 + bal(D0)) stay below
      // 2^24 in every intermediate, and z = P mod m in balanced form.
      const float mf = __uint_as_float(__ldg(P.ztab + 4 * bi + 1));    // m as a float
      const float rinv = __uint_as_float(__ldg(P.ztab + 4 * bi + 2));  // 1 / m rounded
      const int mi = (int)__ldg(P.ztab + 4 * bi);
      auto bal = [&](float x) {
        const float q = __fadd_rn(__fmaf_rn(x, rinv, TG_MAGIC), -TG_MAGIC);
        return __fmaf_rn(-q, mf, x);
      };
      uint4 *zdst = (uint4 *)(P.zout + ((int64_t)bi * P.Mp + gm) * P.Np + gcol);
#pragma unroll
      for (int c8 = 0; c8 < 2; ++c8) {
        uint32_t zz[4];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int cc = 8 * c8 + u;
          const float d1 = __fadd_rn(bal(__uint_as_float(v1[cc])), bal(__uint_as_float(v2[cc])));
          const float hi = bal(__fmaf_rn(bal(__uint_as_float(v3[cc])), 256.0f, d1));
          const float z = bal(__fmaf_rn(hi, 256.0f, bal(__uint_as_float(v0[cc]))));
          int r = (int)(__float_as_uint(__fadd_rn(z, TG_MAGIC)) - TG_MAGIC_BITS);
          r += r < 0 ? mi : 0;
          if (u & 1)
            zz[u >> 1] |= (uint32_t)r << 16;
          else
            zz[u >> 1] = (uint32_t)r;
        }
        zdst[c8] = make_uint4(zz[0], zz[1], zz[2], zz[3]);
      }
    }
  }

  pdl_trigger();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, CG_TMEM_COLS);
  }
}

typedef CUresult (*PFN_tmapEncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                        const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                        const cuuint32_t *, CUtensorMapInterleave,
                                        CUtensorMapSwizzle, CUtensorMapL2promotion,
                                        CUtensorMapFloatOOBfill);

static PFN_tmapEncodeTiled encode_fn() {
  static PFN_tmapEncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_tmapEncodeTiled)p;
  });
  return fn;
}

// 3-D map over digit planes [planes][rows][Kp] of BF16, box = 64 (k) x box_rows x 1 plane.
static bool make_plane_map(CUtensorMap *tm, const void *base, int64_t Kp, int64_t rows,
                           int64_t planes, int box_rows = TG_BM) {
  PFN_tmapEncodeTiled enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(Kp * 2 * rows)};
  cuuint32_t box[3] = {(cuuint32_t)TG_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_residue_store_map(CUtensorMap *tm, void *base, int64_t Kp, int64_t rows, int64_t planes,
                            int box_k, int box_rows, int box_planes) {
  PFN_tmapEncodeTiled enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(Kp * 2 * rows)};
  cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_z_load_map(CUtensorMap *tm, const void *base, int64_t Np, int64_t Mp, int64_t planes,
                     int box_planes) {
  PFN_tmapEncodeTiled enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Np, (cuuint64_t)Mp, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(Np * 2), (cuuint64_t)(Np * 2 * Mp)};
  cuuint32_t box[3] = {128u, 1u, (cuuint32_t)box_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void *>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int digit_gemm_groups(arbgpu_ctx *ctx, int M, int N, int ND) {
  int tiles = ((M + TG_BM - 1) / TG_BM) * ((N + TG_BN - 1) / TG_BN);
  if (tiles < 1) tiles = 1;  // empty products (M or N zero) still get a valid layout
  int g = ctx->sm_count / tiles;  // one wave of CTAs (one CTA per SM)
  if (g < 1) g = 1;
  if (g > ND) g = ND;
  if (g > TG_MAXG) g = TG_MAXG;
  return g;
}

// Largest |running sum| bound of the drain: pairs * Kp * 2^14 plus the carried part.
bool digit_gemm_fits(int SA, int SB, int64_t Kp) {
  const int64_t pairs = SA < SB ? SA : SB;
  return pairs * Kp * 16384 + (1 << 24) < ((int64_t)1 << 31);
}

// Split the SA + SB - 1 diagonals into `groups` contiguous ranges of about equal pair counts (every
// range non-empty); ends[g] is the first diagonal after range g.
void digit_gemm_group_ends(int SA, int SB, int groups, int *ends) {
  const int ND = SA + SB - 1;
  auto pairs = [&](int d) {
    const int jlo = d - (SB - 1) > 0 ? d - (SB - 1) : 0;
    const int jhi = d < SA - 1 ? d : SA - 1;
    return (int64_t)(jhi - jlo + 1);
  };
  int64_t total = 0;
  for (int d = 0; d < ND; ++d) total += pairs(d);
  int64_t acc = 0;
  int g = 0;
  for (int d = 0; d < ND && g + 1 < groups; ++d) {
    acc += pairs(d);
    const int rest_d = ND - (d + 1), rest_g = groups - (g + 1);
    if (acc * groups >= total * (int64_t)(g + 1) || rest_d == rest_g) ends[g++] = d + 1;
  }
  ends[groups - 1] = ND;
}

bool crt_gemm_one_chain(int64_t Kp) { return Kp <= CG_MAX_KP; }

arbgpu_status launch_digit_gemm(arbgpu_ctx *ctx, const DigitGemmArgs &a, cudaStream_t stream) {
  if (a.M <= 0 || a.N <= 0 || a.Kp <= 0 || (a.Kp % TG_BK) != 0 || a.SA < 1 || a.SB < 1)
    return ARBGPU_ERR_INVALID;
  if (!digit_gemm_fits(a.SA, a.SB, a.Kp)) return ARBGPU_ERR_LIMIT;
  DigitGemmParams P{};
  P.M = a.M;
  P.N = a.N;
  P.Kp = a.Kp;
  P.SA = a.SA;
  P.SB = a.SB;
  P.ND = a.SA + a.SB - 1;
  P.tiles_m = (a.M + TG_BM - 1) / TG_BM;
  P.tiles_n = (a.N + TG_BN - 1) / TG_BN;
  P.Mp = (int64_t)P.tiles_m * TG_BM;
  P.Np = (int64_t)P.tiles_n * TG_BN;
  P.digits = a.digits;
  P.carries = a.carries;
  P.batch = a.batch > 0 ? a.batch : 1;
  P.status = ctx->status;
  P.zout = a.zout;
  P.ztab = a.ztab;
  P.zinv = a.zinv;
  P.zraw = a.zraw;
  P.nz = a.zraw ? a.nz : P.batch;
  if (a.zraw && (a.Kp > CG_MAX_KP || a.nz < 0 || a.nz > P.batch)) return ARBGPU_ERR_INVALID;
  if (a.zout && (a.SA != 2 || a.SB != 2 || a.groups != 1 || !a.ztab || !a.zinv))
    return ARBGPU_ERR_INVALID;
  const int G = a.groups;
  if (G < 1 || G > TG_MAXG || G > P.ND) return ARBGPU_ERR_INVALID;
  P.groups = G;
  int ends[TG_MAXG];
  digit_gemm_group_ends(a.SA, a.SB, G, ends);
  P.dstart[0] = 0;
  for (int t = 0; t < G; ++t) P.dstart[t + 1] = ends[t];
  for (int t = 0; t < G; ++t)
    if (P.dstart[t + 1] <= P.dstart[t]) return ARBGPU_ERR_INVALID;

  CUtensorMap tmA, tmB;
  if (!make_plane_map(&tmA, a.A, a.Kp, a.M, (int64_t)a.SA * P.batch) ||
      !make_plane_map(&tmB, a.B, a.Kp, a.N, (int64_t)a.SB * P.batch))
    return ARBGPU_ERR_CUDA;
  static bool attr_set[256] = {};
  const int dev = ctx->device & 255;
  if (!attr_set[dev]) {  // per device: the attribute applies to the current device
    if (cudaFuncSetAttribute(digit_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TG_SMEM_BYTES) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
    attr_set[dev] = true;
  }
  // batch items per CTA: the fewest waves x items over the SMs (items of a CTA run back to back)
  {
    const int64_t per = (int64_t)P.tiles_m * P.tiles_n * G;
    int best = 1;
    int64_t best_cost = INT64_MAX;
    for (int ipc = 1; ipc <= P.batch; ++ipc) {
      const int64_t ctas = per * ((P.batch + ipc - 1) / ipc);
      const int64_t cost = (ctas + ctx->sm_count - 1) / ctx->sm_count * ipc;
      if (cost < best_cost) {
        best_cost = cost;
        best = ipc;
      }
    }
    P.ipc = best;
  }
  const int64_t grid = (int64_t)P.tiles_m * P.tiles_n * G * ((P.batch + P.ipc - 1) / P.ipc);
  if (a.zout && a.Kp <= CG_MAX_KP) {
    static bool cg_attr[256] = {};
    if (!cg_attr[dev]) {
      if (cudaFuncSetAttribute(crt_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)CG_SMEM_BYTES) != cudaSuccess)
        return ARBGPU_ERR_CUDA;
      cg_attr[dev] = true;
    }
    if (grid > 0x7fffffff) return ARBGPU_ERR_LIMIT;
    LaunchScope scope(ctx, stream, a.name ? a.name : "crt_gemm",
                      (int64_t)(a.SA) * a.SB * (int64_t)a.M * a.N * a.Kp * P.batch);
    if (!make_plane_map(&tmB, a.B, a.Kp, a.N, (int64_t)a.SB * P.batch, CG_BN))
      return ARBGPU_ERR_CUDA;
    const int64_t items = (int64_t)P.tiles_m * (P.Np / CG_BN) * P.batch;
    const int64_t cgrid = items < ctx->sm_count ? items : ctx->sm_count;
    launch_pdl(crt_gemm_kernel, dim3((unsigned)cgrid), dim3(CG_THREADS), CG_SMEM_BYTES, stream,
               tmA, tmB, P);
    return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
  }
  if (grid > 0x7fffffff) return ARBGPU_ERR_LIMIT;
  LaunchScope scope(ctx, stream, a.name ? a.name : "digit_gemm",
                    (int64_t)(a.SA) * a.SB * (int64_t)a.M * a.N * a.Kp * P.batch);
  digit_gemm_kernel<<<(unsigned)grid, TG_THREADS, TG_SMEM_BYTES, stream>>>(tmA, tmB, P);
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

}  // namespace arbgpu
