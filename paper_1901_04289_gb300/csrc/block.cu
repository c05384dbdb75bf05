// The block algorithm for ball matrix products (Algorithm 2, Section IV-A) around the tensor-core
// integer engine:
//
//   scan   per row of A / column of B: largest exponent (top), exponent of the lowest set bit
//          (bottom), largest radius exponent; global p_A, p_B and the largest heights.
//   plan   h = 1.25 min(p, max(p_A, p_B)) + 192 (Algorithm 2's height bound); the product is one block when
//          every row of A and column of B scales to integers of height <= h (the common case the
//          paper describes: uniformly scaled inputs need a single block).
//   split  E A and B F with the minimal-height scalings e_i = -bottom_i, f_j = -bottom_j (Fig. 2),
//          written as balanced base-256 digits; the radius operands |A|, R_A, R_B, |B| + R_B become
//          nonnegative integers rounded UP in 13-bit windows under each row's / column's top.
//   gemm   T = (E A)(B F) exactly on the tensor cores; P1 = U(|A|) V(R_B), P2 = U(R_A) V(|B|+R_B).
//   round  C_ij = RNE_p(T_ij 2^(-e_i - f_j)) (one rounding of the exact entry) and
//          R_ij >= eps_round + P1 2^(...) + P2 2^(...), rounded up to a 30-bit radius.
#include <algorithm>
#include <thread>
#include <chrono>
#include <atomic>
#include <functional>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "inner_order.cuh"
#include "internal.h"
#include "round_regs.cuh"
#include "tc_gemm.cuh"

namespace arbgpu {

constexpr int BL_W = 13;          // radius window bits: operands rounded up to <= 2^13
constexpr int BL_SR = 2;          // digits per radius operand (2^13 fits two balanced digits)
constexpr int BL_MAX_NL = 32;     // input limbs the block path accepts
constexpr int BL_BASECASE = 30;   // Algorithm 2: blocks shorter than this go to dot products


__device__ __forceinline__ void atomic_max_i64(int64_t *p, int64_t v) {
  atomicMax((long long *)p, (long long)v);
}
__device__ __forceinline__ void atomic_min_i64(int64_t *p, int64_t v) {
  atomicMin((long long *)p, (long long)v);
}

// Per-entry quantities of the scan.
struct EntryScan {
  bool nz, special;
  int64_t top, bot;  // |m| < 2^top, lowest set bit at 2^bot
  bool rad;
  int64_t rexp;      // r < 2^rexp
};

__device__ __forceinline__ EntryScan scan_entry(const BallsView &v, int64_t idx) {
  EntryScan s;
  const uint32_t fl = __ldg(v.flags + idx);
  const int64_t e = __ldg(v.exp + idx);
  const uint32_t rm = __ldg(v.rad_man + idx);
  const int64_t re = __ldg(v.rad_exp + idx);
  const uint64_t limb0 = __ldg(v.limbs + idx);  // the lowest limb when all limbs are significant
  s.special = (fl & SPECIAL_MASK) != 0;
  s.nz = !(fl & ARBGPU_FLAG_ZERO) && !s.special;
  s.rad = rm != 0 && !s.special;
  s.top = e;
  s.rexp = re;
  s.bot = 0;
  if (s.nz) {
    if (e >= EXP_LIMIT || e <= -EXP_LIMIT) s.special = true;
    int ns = (int)nsig_of(fl);
    if (ns < 1) ns = 1;
    if (ns > v.nlimbs) ns = v.nlimbs;
    const uint64_t low =
        ns == v.nlimbs ? limb0 : __ldg(v.limbs + (int64_t)(v.nlimbs - ns) * v.stride + idx);
    s.bot = e - 64LL * ns + (low ? __ffsll((long long)low) - 1 : 0);
  }
  if (s.rad && (re >= EXP_LIMIT || re <= -EXP_LIMIT)) s.special = true;
  return s;
}

// Inner-dimension range of scan launch row blockIdx.y: the whole of [0, K) when `blocks` is null,
// else block blockIdx.y of the plan ([start, stop, basecase] triples).  Returns false for a
// basecase block (nothing to scan).
__device__ __forceinline__ bool scan_range(const int32_t *blocks, int64_t K, int64_t &k0,
                                           int64_t &k1) {
  if (!blocks) {
    k0 = 0;
    k1 = K;
    return true;
  }
  const int b = blockIdx.y;
  k0 = blocks[3 * b];
  k1 = blocks[3 * b + 1];
  return blocks[3 * b + 2] == 0;
}

// The scans run in three launches: the line statistics start at their identities, chunks of the
// inner dimension fold their entries in with atomics (many warps per line), and a last pass derives
// the per-line quantities that need the finished values (heights, |B| + R_B exponents).

// rtop/rrad = INT64_MIN, rbot = INT64_MAX for `nr` rows (and the same for `nc` columns).
__global__ void scan_init_kernel(int64_t *rtop, int64_t *rbot, int64_t *rrad, int64_t nr,
                                 int64_t *ctop, int64_t *cbot, int64_t *crad, int64_t nc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nr) {
    rtop[idx] = INT64_MIN;
    rbot[idx] = INT64_MAX;
    rrad[idx] = INT64_MIN;
  } else if (idx < nr + nc) {
    const int64_t j = idx - nr;
    ctop[j] = INT64_MIN;
    cbot[j] = INT64_MAX;
    crad[j] = INT64_MIN;
  }
}

// Chunk blockIdx.z of the scan range, of `chunk` indices.
__device__ __forceinline__ bool scan_chunk(const int32_t *blocks, int64_t K, int64_t chunk,
                                           int64_t &k0, int64_t &k1) {
  int64_t b0, b1;
  if (!scan_range(blocks, K, b0, b1)) return false;
  k0 = b0 + (int64_t)blockIdx.z * chunk;
  k1 = k0 + chunk < b1 ? k0 + chunk : b1;
  return k0 < k1;
}

// One warp per (row of A, chunk of k): row top / bottom / radius top folded into the row's values.
__global__ void scan_rows_kernel(const BallsView A, int64_t M, int64_t K, int64_t lda,
                                 const int32_t *blocks, int64_t chunk, int64_t *rtop,
                                 int64_t *rbot, int64_t *rrad, BlockStats *st) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t k0, k1;
  if (i >= M || !scan_chunk(blocks, K, chunk, k0, k1)) return;
  const int64_t ob = (int64_t)blockIdx.y * M;
  st += blockIdx.y;
  int64_t top = INT64_MIN, bot = INT64_MAX, rad = INT64_MIN, pm = 0;
  bool special = false, anyrad = false;
  for (int64_t k = k0 + lane; k < k1; k += 32) {
    EntryScan e = scan_entry(A, i * lda + k);
    special |= e.special;
    if (e.nz) {
      top = max((long long)top, (long long)e.top);
      bot = min((long long)bot, (long long)e.bot);
      pm = max((long long)pm, (long long)(e.top - e.bot));
    }
    if (e.rad) {
      anyrad = true;
      rad = max((long long)rad, (long long)e.rexp);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    top = max((long long)top, (long long)__shfl_xor_sync(0xffffffffu, top, o));
    bot = min((long long)bot, (long long)__shfl_xor_sync(0xffffffffu, bot, o));
    rad = max((long long)rad, (long long)__shfl_xor_sync(0xffffffffu, rad, o));
    pm = max((long long)pm, (long long)__shfl_xor_sync(0xffffffffu, pm, o));
  }
  special = __any_sync(0xffffffffu, special);
  anyrad = __any_sync(0xffffffffu, anyrad);
  if (lane == 0) {
    if (top != INT64_MIN) {
      atomic_max_i64(rtop + ob + i, top);
      atomic_min_i64(rbot + ob + i, bot);
    }
    if (rad != INT64_MIN) atomic_max_i64(rrad + ob + i, rad);
    if (pm) atomic_max_i64(&st->pA, pm);
    if (special) atomicOr(&st->special, 1);
    if (anyrad) atomicOr(&st->radA, 1);
  }
}

// Columns of B: block (32 columns) x (8 k-slices) over chunk blockIdx.z of k; reads coalesced
// along the row, folded into the columns' values.
__global__ void scan_cols_kernel(const BallsView B, int64_t K, int64_t N, int64_t ldb,
                                 const int32_t *blocks, int64_t chunk, int64_t *ctop,
                                 int64_t *cbot, int64_t *crad, BlockStats *st) {
  __shared__ int64_t s_top[8][33], s_bot[8][33], s_rad[8][33], s_pm[8][33];
  __shared__ int s_flags[8][33];
  int64_t k0, k1;
  if (!scan_chunk(blocks, K, chunk, k0, k1)) return;  // uniform over the CTA
  const int64_t ob = (int64_t)blockIdx.y * N;
  st += blockIdx.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t j = (int64_t)blockIdx.x * 32 + tx;
  int64_t top = INT64_MIN, bot = INT64_MAX, rad = INT64_MIN, pm = 0;
  int flags = 0;
  if (j < N) {
    for (int64_t k = k0 + ty; k < k1; k += 8) {
      EntryScan e = scan_entry(B, k * ldb + j);
      if (e.special) flags |= 1;
      if (e.nz) {
        top = max((long long)top, (long long)e.top);
        bot = min((long long)bot, (long long)e.bot);
        pm = max((long long)pm, (long long)(e.top - e.bot));
      }
      if (e.rad) {
        flags |= 2;
        rad = max((long long)rad, (long long)e.rexp);
      }
    }
  }
  s_top[ty][tx] = top;
  s_bot[ty][tx] = bot;
  s_rad[ty][tx] = rad;
  s_pm[ty][tx] = pm;
  s_flags[ty][tx] = flags;
  __syncthreads();
  if (ty == 0 && j < N) {
    for (int y = 1; y < 8; ++y) {
      top = max((long long)top, (long long)s_top[y][tx]);
      bot = min((long long)bot, (long long)s_bot[y][tx]);
      rad = max((long long)rad, (long long)s_rad[y][tx]);
      pm = max((long long)pm, (long long)s_pm[y][tx]);
      flags |= s_flags[y][tx];
    }
    if (top != INT64_MIN) {
      atomic_max_i64(ctop + ob + j, top);
      atomic_min_i64(cbot + ob + j, bot);
    }
    if (rad != INT64_MIN) atomic_max_i64(crad + ob + j, rad);
    if (pm) atomic_max_i64(&st->pB, pm);
    if (flags & 1) atomicOr(&st->special, 1);
    if (flags & 2) atomicOr(&st->radB, 1);
  }
}

// Row / column heights into the statistics, and cplus = exponent bound of |b| + r_b per column
// (|b| + r_b < 2^(max(top, rexp) + 1)).  Rows [0, M) then columns [0, N) of each of the
// gridDim.y scan ranges.
__global__ void scan_finish_kernel(const int64_t *rtop, const int64_t *rbot, int64_t M,
                                   const int64_t *ctop, const int64_t *cbot, const int64_t *crad,
                                   int64_t *cplus, int64_t N, BlockStats *st_rows,
                                   BlockStats *st_cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (idx < M) {
    const int64_t o = (int64_t)b * M + idx;
    if (rtop[o] != INT64_MIN) atomic_max_i64(&st_rows[b].hA, rtop[o] - rbot[o]);
  } else if (idx < M + N) {
    const int64_t o = (int64_t)b * N + (idx - M);
    const int64_t top = ctop[o], rad = crad[o];
    if (top != INT64_MIN) atomic_max_i64(&st_cols[b].hB, top - cbot[o]);
    if (cplus) {
      const int64_t mx = top > rad ? top : rad;
      cplus[o] = mx == INT64_MIN ? INT64_MIN : mx + 1;
    }
  }
}

// Inner-dimension chunk of the scans so that about `lines_target` warps or CTAs cover a range of
// `len` indices for `lines` lines.
static int64_t scan_chunk_len(int64_t len, int64_t lines, int64_t target, int64_t minchunk) {
  int64_t z = target / (lines > 0 ? lines : 1);
  if (z < 1) z = 1;
  int64_t chunk = (len + z - 1) / z;
  if (chunk < minchunk) chunk = minchunk;
  return chunk;
}

// Whole-range scans, one CTA per line group and no atomics on the line values.

struct LineAcc {
  int64_t top, bot, rad, pm;
  int flags;  // 1: special value, 2: nonzero radius
};

__device__ __forceinline__ void line_fold(LineAcc &a, const EntryScan &e) {
  if (e.special) a.flags |= 1;
  if (e.nz) {
    a.top = max((long long)a.top, (long long)e.top);
    a.bot = min((long long)a.bot, (long long)e.bot);
    a.pm = max((long long)a.pm, (long long)(e.top - e.bot));
  }
  if (e.rad) {
    a.flags |= 2;
    a.rad = max((long long)a.rad, (long long)e.rexp);
  }
}

__device__ __forceinline__ void line_merge(LineAcc &a, const LineAcc &b) {
  a.top = max((long long)a.top, (long long)b.top);
  a.bot = min((long long)a.bot, (long long)b.bot);
  a.rad = max((long long)a.rad, (long long)b.rad);
  a.pm = max((long long)a.pm, (long long)b.pm);
  a.flags |= b.flags;
}

__device__ __forceinline__ LineAcc line_shfl_xor(const LineAcc &a, int o) {
  LineAcc b;
  b.top = __shfl_xor_sync(0xffffffffu, a.top, o);
  b.bot = __shfl_xor_sync(0xffffffffu, a.bot, o);
  b.rad = __shfl_xor_sync(0xffffffffu, a.rad, o);
  b.pm = __shfl_xor_sync(0xffffffffu, a.pm, o);
  b.flags = __shfl_xor_sync(0xffffffffu, a.flags, o);
  return b;
}

// Both whole-range scans in one launch of 1024-thread CTAs: CTAs [0, ceil(M / 8)) take eight rows
// of A (128 threads along each row), the others eight columns of B (128 k-slices; a warp reads
// four rows of eight neighbouring entries).  Each CTA finishes its lines.  (At N = 512 the 128
// CTAs run in one wave, each thread with four entries' loads in flight.)
// Publication of the statistics to the host: the last CTA of the launch to finish copies `n`
// BlockStats from `src` into mapped pinned host memory `dst` (as 32-bit words), then writes `seq`
// into the word after them (system-scope fences between), so that the host can poll for `seq`
// instead of synchronising the stream.  `done` counts the finished CTAs (zeroed beforehand).
struct StatsPublish {
  const BlockStats *src;
  int n;
  uint32_t *dst;
  unsigned *done;
  uint32_t seq;
};

__device__ __forceinline__ void publish_stats(const StatsPublish &pub, bool wrote) {
  __shared__ bool s_last;
  if (wrote) __threadfence();  // this thread's statistics updates are visible device-wide
  __syncthreads();             // every line of this CTA is finished
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(pub.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int words = pub.n * (int)(sizeof(BlockStats) / 4);
  const volatile uint32_t *src = (const volatile uint32_t *)pub.src;
  for (int q = threadIdx.x; q < words; q += blockDim.x) pub.dst[q] = src[q];
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) {
    *(volatile uint32_t *)(pub.dst + words) = pub.seq;
    __threadfence_system();
  }
}

__global__ void __launch_bounds__(1024) scan_full_kernel(
    const BallsView A, const BallsView B, int64_t M, int64_t K, int64_t N, int64_t lda,
    int64_t ldb, int64_t *rtop, int64_t *rbot, int64_t *rrad, BlockStats *st_rows, int64_t *ctop,
    int64_t *cbot, int64_t *crad, int64_t *cplus, BlockStats *st_cols, const StatsPublish pub) {
  __shared__ LineAcc s_acc[32][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row_ctas = (M + 7) / 8;
  LineAcc a{INT64_MIN, INT64_MAX, INT64_MIN, 0, 0};
  if ((int64_t)blockIdx.x < row_ctas) {
    const int r = threadIdx.x >> 7, tk = threadIdx.x & 127;  // row of the group, k-slice
    const int64_t i = (int64_t)blockIdx.x * 8 + r;
    if (i < M)
      for (int64_t k = tk; k < K; k += 128) line_fold(a, scan_entry(A, i * lda + k));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) line_merge(a, line_shfl_xor(a, o));
    if (lane == 0) s_acc[warp][0] = a;
    __syncthreads();
    if (tk == 0 && i < M) {  // warps 4r .. 4r + 3 hold row r
      for (int w = 1; w < 4; ++w) line_merge(a, s_acc[4 * r + w][0]);
      rtop[i] = a.top;
      rbot[i] = a.bot;
      rrad[i] = a.rad;
      if (a.top != INT64_MIN) atomic_max_i64(&st_rows->hA, a.top - a.bot);
      if (a.pm) atomic_max_i64(&st_rows->pA, a.pm);
      if (a.flags & 1) atomicOr(&st_rows->special, 1);
      if (a.flags & 2) atomicOr(&st_rows->radA, 1);
    }
    if (pub.dst) publish_stats(pub, tk == 0);
    return;
  }
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;  // column of the group, k-slice
  const int64_t j = ((int64_t)blockIdx.x - row_ctas) * 8 + tx;
  if (j < N)
    for (int64_t k = ty; k < K; k += 128) line_fold(a, scan_entry(B, k * ldb + j));
  // lanes 8 apart hold the same column
  line_merge(a, line_shfl_xor(a, 8));
  line_merge(a, line_shfl_xor(a, 16));
  if (lane < 8) s_acc[warp][lane] = a;
  __syncthreads();
  if (threadIdx.x < 8 && j < N) {
    for (int w = 1; w < 32; ++w) line_merge(a, s_acc[w][tx]);
    ctop[j] = a.top;
    cbot[j] = a.bot;
    crad[j] = a.rad;
    const int64_t mx = a.top > a.rad ? a.top : a.rad;  // |b| + r_b < 2^(max(top, rexp) + 1)
    cplus[j] = mx == INT64_MIN ? INT64_MIN : mx + 1;
    if (a.top != INT64_MIN) atomic_max_i64(&st_cols->hB, a.top - a.bot);
    if (a.pm) atomic_max_i64(&st_cols->pB, a.pm);
    if (a.flags & 1) atomicOr(&st_cols->special, 1);
    if (a.flags & 2) atomicOr(&st_cols->radB, 1);
  }
  if (pub.dst) publish_stats(pub, threadIdx.x < 8);
}

// Scans of the rows of X (M x K) and the columns of Y (K x N) over the whole inner range
// (blocks = null, nb = 1) or over each of the nb ranges of a plan: the line statistics and the
// per-range BlockStats (rows into st_rows, columns into st_cols; both must hold their identities).
static arbgpu_status run_scans(arbgpu_ctx *ctx, cudaStream_t s, const BallsView &Xv, int64_t M,
                               int64_t K, int64_t ldx, const BallsView &Yv, int64_t N,
                               int64_t ldy, const int32_t *blocks, int nb, int64_t kmax,
                               int64_t *rtop, int64_t *rbot, int64_t *rrad, int64_t *ctop,
                               int64_t *cbot, int64_t *crad, int64_t *cplus,
                               BlockStats *st_rows, BlockStats *st_cols) {
  {
    const int64_t n = (M + N) * nb;
    LaunchScope sc(ctx, s, "scan_init", n);
    scan_init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rtop, rbot, rrad, M * nb, ctop,
                                                                 cbot, crad, N * nb);
  }
  const int64_t rchunk = scan_chunk_len(kmax, M * nb, 8192, 64);
  const int64_t cchunk = scan_chunk_len(kmax, (N + 31) / 32 * nb, 1024, 32);
  {
    LaunchScope sc(ctx, s, "scan_rows", M * K);
    scan_rows_kernel<<<dim3((unsigned)((M * 32 + 255) / 256), (unsigned)nb,
                            (unsigned)((kmax + rchunk - 1) / rchunk)),
                       256, 0, s>>>(Xv, M, K, ldx, blocks, rchunk, rtop, rbot, rrad, st_rows);
  }
  {
    LaunchScope sc(ctx, s, "scan_cols", K * N);
    scan_cols_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)nb,
                            (unsigned)((kmax + cchunk - 1) / cchunk)),
                       dim3(32, 8), 0, s>>>(Yv, K, N, ldy, blocks, cchunk, ctop, cbot, crad,
                                            st_cols);
  }
  {
    LaunchScope sc(ctx, s, "scan_finish", (M + N) * nb);
    scan_finish_kernel<<<dim3((unsigned)((M + N + 255) / 256), (unsigned)nb), 256, 0, s>>>(
        rtop, rbot, M, ctop, cbot, crad, cplus, N, st_rows, st_cols);
  }
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

// Balanced base-256 digits of X = (-1)^neg * L * 2^sh, L the midpoint's limb integer (nl limbs,
// only the top `ns` nonzero).  sh >= -(bit position of L's lowest set bit), so X is an integer.
__device__ __forceinline__ void split_mid_digits(const BallsView &v, int64_t idx, int64_t sh,
                                                 bool neg, int S, __nv_bfloat16 *dst,
                                                 int64_t plane) {
  uint64_t L[BL_MAX_NL];
  const int nl = v.nlimbs;
  for (int k = 0; k < nl; ++k) L[k] = __ldg(v.limbs + (int64_t)k * v.stride + idx);
  int carry = 0;
  for (int t = 0; t < S; ++t) {
    // bits [8t - sh, 8t - sh + 8) of L
    const int64_t pos = 8LL * t - sh;
    uint32_t byte = 0;
    if (pos > -8 && pos < 64LL * nl) {
      if (pos >= 0) {
        const int li = (int)(pos >> 6), bi = (int)(pos & 63);
        uint64_t w = L[li] >> bi;
        if (bi > 56 && li + 1 < nl) w |= L[li + 1] << (64 - bi);
        byte = (uint32_t)(w & 255u);
      } else {
        byte = (uint32_t)((L[0] << (-pos)) & 255u);
      }
    }
    int vv = (neg ? -(int)byte : (int)byte) + carry;
    if (vv >= 128) {
      vv -= 256;
      carry = 1;
    } else if (vv < -128) {
      vv += 256;
      carry = -1;
    } else {
      carry = 0;
    }
    dst[(int64_t)t * plane] = __int2bfloat16_rn(vv);
  }
}

// ceil(v * 2^(W - F)) for a 30-bit mag v = man * 2^(e - 30) <= 2^F, as an integer in [0, 2^W].
__device__ __forceinline__ uint32_t window_up(uint32_t man, int64_t e, int64_t F) {
  if (man == 0 || F == INT64_MIN) return 0;
  const int64_t sh = e - 30 + BL_W - F;  // <= BL_W - 30 < 0
  if (sh >= 0) return man << sh;         // (not reached: e <= F)
  const int64_t r = -sh;
  if (r >= 40) return 1;
  return (uint32_t)(((uint64_t)man + ((((uint64_t)1) << r) - 1)) >> r);
}

__device__ __forceinline__ void put_small_digits(uint32_t u, __nv_bfloat16 *dst, int64_t plane) {
  // u <= 2^13: two balanced digits
  int d0 = (int)(u & 255u), c = 0;
  if (d0 >= 128) {
    d0 -= 256;
    c = 1;
  }
  const int d1 = (int)(u >> 8) + c;
  dst[0] = __int2bfloat16_rn(d0);
  dst[plane] = __int2bfloat16_rn(d1);
}

// 30-bit upper bound of |m|: top 30 bits of the top limb plus one (Section III-E).
__device__ __forceinline__ Mag mid_upper(const BallsView &v, int64_t idx, int64_t e) {
  const uint64_t top = __ldg(v.limbs + (int64_t)(v.nlimbs - 1) * v.stride + idx);
  uint64_t b = (top >> 34) + 1;
  int64_t ee = e;
  if (b == ((uint64_t)1 << 30)) {
    b >>= 1;
    ee += 1;
  }
  return Mag{(uint32_t)b, ee};
}

struct SplitOut {
  __nv_bfloat16 *mid;  // [S][rows][Kp]
  __nv_bfloat16 *r1;   // [2][rows][Kp] first radius operand (or null)
  __nv_bfloat16 *r2;   // [2][rows][Kp] second radius operand (or null)
};

// Split A (rows = M, row-major lda) or B (rows = N, read transposed from K x N, ldb).
//   A: mid = E A; r1 = U(|A|) under rowtop; r2 = U(R_A) under rowrad.
//   B: mid = B F; r1 = V(R_B) under colrad; r2 = V(|B| + R_B) under colplus.
//   Columns [k0, k0 + K) of the operand form the block; columns K..Kp of the planes are zero.
//   trunc (or null): per line, the exponent below which the line's bits were dropped (INT64_MIN:
//   none); every nonzero entry of such a line carries 2^trunc more radius.
__global__ void split_kernel(const BallsView X, bool is_b, int64_t rows, int64_t k0, int64_t K,
                             int64_t Kp, int64_t ld, int S, const int64_t *bot, const int64_t *top,
                             const int64_t *radtop, const int64_t *plustop, SplitOut o,
                             const int64_t *trunc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * Kp) return;
  const int64_t r = idx / Kp, k = idx - (idx / Kp) * Kp;
  const int64_t plane = rows * Kp;
  const int64_t off = r * Kp + k;
  const __nv_bfloat16 z = __int2bfloat16_rn(0);
  if (k >= K) {
    for (int t = 0; t < S; ++t) o.mid[(int64_t)t * plane + off] = z;
    if (o.r1) o.r1[off] = o.r1[plane + off] = z;
    if (o.r2) o.r2[off] = o.r2[plane + off] = z;
    return;
  }
  const int64_t e = is_b ? ((k0 + k) * ld + r) : (r * ld + k0 + k);
  const uint32_t fl = __ldg(X.flags + e);
  const bool nz = !(fl & (ARBGPU_FLAG_ZERO | SPECIAL_MASK));
  const int64_t ex = __ldg(X.exp + e);
  if (nz) {
    const int64_t sh = ex - 64LL * X.nlimbs - bot[r];
    split_mid_digits(X, e, sh, (fl & ARBGPU_FLAG_SIGN) != 0, S, o.mid + off, plane);
  } else {
    for (int t = 0; t < S; ++t) o.mid[(int64_t)t * plane + off] = z;
  }
  Mag rad{__ldg(X.rad_man + e), __ldg(X.rad_exp + e)};
  if (trunc && nz && trunc[r] != INT64_MIN) rad = mag_add_up(rad, Mag{1u << 29, trunc[r] + 1});
  const Mag absm = nz ? mid_upper(X, e, ex) : Mag{0u, 0};
  if (!is_b) {
    if (o.r1) put_small_digits(window_up(absm.man, absm.exp, top[r]), o.r1 + off, plane);
    if (o.r2) put_small_digits(window_up(rad.man, rad.exp, radtop[r]), o.r2 + off, plane);
  } else {
    if (o.r1) put_small_digits(window_up(rad.man, rad.exp, radtop[r]), o.r1 + off, plane);
    if (o.r2) {
      const Mag plus = mag_add_up(absm, rad);
      put_small_digits(window_up(plus.man, plus.exp, plustop[r]), o.r2 + off, plane);
    }
  }
}

// ------------------------------------------------------------------------- rounding epilogue

struct Ends {
  int e[TG_MAXG];
};

// Per-modulus constants (the first CRT_MAX_MODULI primes below 2^16), loaded once per device:
// m_t, floor((2^64 - 1) / m_t), floor(2^32 / m_t) and 2^32 mod m_t.
__constant__ uint32_t c_mods[CRT_MAX_MODULI];
__constant__ uint64_t c_inv[CRT_MAX_MODULI];
__constant__ uint32_t c_inv32[CRT_MAX_MODULI];  // floor(2^32 / m_t)
__constant__ uint32_t c_pow32m[CRT_MAX_MODULI];  // 2^32 mod m_t

// Device copies of the tables of one modulus count (in the workspace).
struct CrtTables {
  const uint32_t *Q32;   // [NM][NW32P]: M / m_t in 32-bit limbs
  const uint32_t *M32;   // [NW32P]: M
  const uint32_t *y;     // [NM]: (M / m_t)^-1 mod m_t
  const float *rinv;     // [NM]: 1 / m_t
  int NM, NMW, NW32P;
  const uint16_t *wtab;  // reconstruction on the tensor cores: [NQP][128] BF16 weights
  const float *mbytes;   // [NQ] balanced bytes of M
  int NQ, NQP;
  // reconstruction on the 8-bit warp-level MMA: [NQ8][K8] balanced bytes of the Q_t
  const int8_t *w8 = nullptr;
  int K8 = 0, NQ8 = 0;
  const uint32_t *c32 = nullptr;  // [2 NMW + 2] words of 32896 sum_t Q_t
};

// One exact integer product.  kind 0: digit + carry form of T itself.  kind 1 (multimodular): for
// every modulus t, z_t = P_t mod m_t ([t][Mp][Np] uint16 in `digits`) of the exact residue product
// P_t = sum_k r_ik (s_kj y_t mod m_t), from which T follows by the Chinese remainder theorem.
// kind 2: T itself as int64 [Mp][Np] in `digits` (a radius product, 0 <= T < 2^63).
struct IntProduct {
  const uint8_t *digits;
  const int32_t *carries;
  int ND, groups;
  Ends ends;
  int kind;
  CrtTables crt;
};

constexpr int RD_MAXW = 48;  // limbs of the assembled product (ND <= 8 * 46)

// x mod m for x < 2^63 with inv = floor((2^64 - 1) / m) (Barrett reduction).
__device__ __forceinline__ uint32_t barrett_mod(uint64_t x, uint32_t m, uint64_t inv) {
  const uint64_t q = __umul64hi(x, inv);
  uint64_t r = x - q * m;
  while (r >= m) r -= m;
  return (uint32_t)r;
}

// z_t = P_t y_t mod m_t of entry o, written by the residue-product GEMM (uint16 planes [NM][Mp][Np]
// in place of digits; the right-hand residues carry the factor y_t).
__device__ __forceinline__ uint32_t crt_z(const IntProduct &p, int t, int64_t pl, int64_t o) {
  return __ldg((const uint16_t *)p.digits + (int64_t)t * pl + o);
}

// T_ij from its residues (Chinese remainder theorem): T = sum_t z_t Q_t - q M with
// q = round(sum_t z_t / m_t), a two's-complement integer of nw = NMW + 1 limbs.  The sum is formed
// in 32-bit limbs, sixteen at a time in 64-bit register accumulators (each < NM 2^48).
__device__ int crt_assemble(const IntProduct &p, int64_t i, int64_t j, int64_t Mp, int64_t Np,
                            uint64_t *T) {
  const CrtTables &c = p.crt;
  const int nw = c.NMW + 1;
  const int64_t pl = Mp * Np, o = i * Np + j;
  uint16_t zz[CRT_MAX_MODULI];
  float qs = 0.f;
  for (int t = 0; t < c.NM; ++t) {
    const uint32_t z = crt_z(p, t, pl, o);
    zz[t] = (uint16_t)z;
    qs = fmaf((float)z, __ldg(c.rinv + t), qs);
  }
  const int64_t q = (int64_t)rintf(qs);
  int64_t carry = 0;
  for (int l0 = 0; l0 < 2 * nw; l0 += 16) {
    uint64_t acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = 0;
    for (int t = 0; t < c.NM; ++t) {
      const uint64_t z = zz[t];
      const uint32_t *row = c.Q32 + (int64_t)t * c.NW32P;
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (l0 + u < c.NW32P) mad_wide(acc[u], (uint32_t)z, __ldg(row + l0 + u));
    }
#pragma unroll
    for (int u = 0; u < 16; u += 2) {
      const int l = l0 + u;
      const int64_t m0 = l < c.NW32P ? __ldg(c.M32 + l) : 0;
      const int64_t m1 = l + 1 < c.NW32P ? __ldg(c.M32 + l + 1) : 0;
      const int64_t v0 = (int64_t)acc[u] - q * m0 + carry;
      carry = v0 >> 32;
      const int64_t v1 = (int64_t)acc[u + 1] - q * m1 + carry;
      carry = v1 >> 32;
      const int k = l >> 1;
      if (k < nw) T[k] = (uint64_t)(uint32_t)v0 | ((uint64_t)(uint32_t)v1 << 32);
    }
  }
  return nw;
}

// Assemble T_ij (two's complement, nw limbs) from its digits and carries.
__device__ __forceinline__ int assemble(const IntProduct &p, int64_t i, int64_t j, int64_t Mp,
                                        int64_t Np, uint64_t *acc) {
  if (p.kind == 1) return crt_assemble(p, i, j, Mp, Np, acc);
  const int nw = (8 * p.ND + 32 + 63) / 64 + 1;
  for (int k = 0; k < nw; ++k) acc[k] = 0;
  const uint8_t *dp = p.digits + i * Np + j;
  const int64_t pl = Mp * Np;
  for (int d = 0; d < p.ND; ++d) acc[d >> 3] |= (uint64_t)dp[(int64_t)d * pl] << (8 * (d & 7));
  for (int g = 0; g < p.groups; ++g) {
    const int64_t c = p.carries[((int64_t)g * Mp + i) * Np + j];
    if (c == 0) continue;
    const int pos = 8 * p.ends.e[g];
    const int li = pos >> 6, bi = pos & 63;
    const uint64_t lo = (uint64_t)c << bi;
    const uint64_t hi = bi ? (uint64_t)(c >> (64 - bi)) : (uint64_t)(c < 0 ? -1 : 0);
    const uint64_t ext = c < 0 ? ~(uint64_t)0 : 0;
    u128 s = 0;
    for (int k = li; k < nw; ++k) {
      const uint64_t add = (k == li) ? lo : (k == li + 1 ? hi : ext);
      s += (u128)acc[k] + add;
      acc[k] = (uint64_t)s;
      s >>= 64;
    }
  }
  return nw;
}

// Residues of the scaled integers for the multimodular engine: X = (-1)^neg L 2^sh (as in the
// digit split), r_t = X mod m_t in balanced form, split into two balanced bytes r_t = 256 h + l,
// written to planes [2t] (l) and [2t + 1] (h) of [2 NM][rows][Kp].  |X| is cut into NCH 32-bit
// chunks (a template bound, so they stay in registers); r_t = sum_c chunk_c (2^(32c) mod m_t)
// reduced once (the sum is below NCH 2^48).

// Bits [32c, 32c + 32) of L 2^sh for c = 0..NCH-1 (zero outside L).
template <int NCH>
__device__ __forceinline__ void residue_chunks32(const BallsView &X, int64_t e, int64_t sh,
                                                 uint32_t (&ch)[NCH]) {
  const int nl = X.nlimbs;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int64_t pos = 32LL * c - sh;  // bit of L at bit 32c of X
    uint32_t v = 0;
    if (pos > -32 && pos < 64LL * nl) {
      if (pos >= 0) {
        const int li = (int)(pos >> 6), bi = (int)(pos & 63);
        uint64_t w = __ldg(X.limbs + (int64_t)li * X.stride + e) >> bi;
        if (bi > 32 && li + 1 < nl) w |= __ldg(X.limbs + (int64_t)(li + 1) * X.stride + e) << (64 - bi);
        v = (uint32_t)w;
      } else {
        v = (uint32_t)(__ldg(X.limbs + e) << (-pos));
      }
    }
    ch[c] = v;
  }
}

template <int NCH, int RE>
__global__ void __launch_bounds__(128) residue_split_kernel(
    const BallsView X, bool is_b, int64_t rows, int64_t k0, int64_t K, int64_t Kp, int64_t ld,
    const int64_t *bot, int NM, const uint32_t *pw32, int pw_stride, const uint32_t *ymul,
    __nv_bfloat16 *out, SplitOut ro, const int64_t *top, const int64_t *radtop,
    const int64_t *plustop) {
  constexpr int NC4 = (NCH + 3) / 4 * 4;  // table row in shared memory, padded for 16-byte loads
  extern __shared__ uint4 s_pw4[];
  uint32_t *s_pw = (uint32_t *)s_pw4;
  for (int q = threadIdx.x; q < NM * NC4; q += blockDim.x) {
    const int t = q / NC4, c = q - t * NC4;
    s_pw[q] = c < NCH ? __ldg(pw32 + (int64_t)t * pw_stride + c) : 0u;
  }
  __syncthreads();
  // thread idx takes entries k = k_lo + u * (Kp / RE), u < RE, of one row: each of the RE
  // sub-ranges is walked by consecutive threads, so loads and stores stay coalesced
  const int64_t kq = Kp / RE;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * kq) return;
  const int64_t r = idx / kq, k_lo = idx - r * kq;
  const int64_t plane = rows * Kp;
  __nv_bfloat16 *o = out + r * Kp + k_lo;
  uint32_t ch[RE][NCH];
  bool live[RE], neg[RE];
  bool any = false;
#pragma unroll
  for (int u = 0; u < RE; ++u) {
    const int64_t k = k_lo + u * kq;
    live[u] = neg[u] = false;
#pragma unroll
    for (int c = 0; c < NCH; ++c) ch[u][c] = 0;
    Mag absm{0u, 0}, rad{0u, 0};
    if (k < K) {
      const int64_t e = is_b ? ((k0 + k) * ld + r) : (r * ld + k0 + k);
      const uint32_t fl = __ldg(X.flags + e);
      const int64_t ex = __ldg(X.exp + e);
      if (!(fl & (ARBGPU_FLAG_ZERO | SPECIAL_MASK))) {
        live[u] = true;
        neg[u] = (fl & ARBGPU_FLAG_SIGN) != 0;
        const int64_t sh = ex - 64LL * X.nlimbs - bot[r];
        residue_chunks32<NCH>(X, e, sh, ch[u]);
        if (ro.r1 || ro.r2) absm = mid_upper(X, e, ex);
      }
      if (ro.r1 || ro.r2) rad = Mag{__ldg(X.rad_man + e), __ldg(X.rad_exp + e)};
    }
    // the radius operands of this entry (zero in the padding), as the split kernel writes them
    if (ro.r1 || ro.r2) {
      const int64_t off = r * Kp + k;
      if (!is_b) {
        if (ro.r1) put_small_digits(window_up(absm.man, absm.exp, top[r]), ro.r1 + off, plane);
        if (ro.r2) put_small_digits(window_up(rad.man, rad.exp, radtop[r]), ro.r2 + off, plane);
      } else {
        if (ro.r1) put_small_digits(window_up(rad.man, rad.exp, radtop[r]), ro.r1 + off, plane);
        if (ro.r2) {
          const Mag plus = mag_add_up(absm, rad);
          put_small_digits(window_up(plus.man, plus.exp, plustop[r]), ro.r2 + off, plane);
        }
      }
    }
    any |= live[u];
  }
  const __nv_bfloat16 z = __int2bfloat16_rn(0);
  if (!__any_sync(__activemask(), any)) {
    for (int t = 0; t < 2 * NM; ++t)
#pragma unroll
      for (int u = 0; u < RE; ++u) o[(int64_t)t * plane + u * kq] = z;
    return;
  }
  for (int t = 0; t < NM; ++t) {
    const uint4 *pw = (const uint4 *)(s_pw + t * NC4);  // the same row for every thread
    uint64_t acc[RE];
#pragma unroll
    for (int u = 0; u < RE; ++u) acc[u] = 0;
#pragma unroll
    for (int c4 = 0; c4 < NC4 / 4; ++c4) {
      const uint4 w = pw[c4];
#pragma unroll
      for (int u = 0; u < RE; ++u) {
        if (4 * c4 + 0 < NCH) acc[u] += (uint64_t)ch[u][4 * c4 + 0] * w.x;
        if (4 * c4 + 1 < NCH) acc[u] += (uint64_t)ch[u][4 * c4 + 1] * w.y;
        if (4 * c4 + 2 < NCH) acc[u] += (uint64_t)ch[u][4 * c4 + 2] * w.z;
        if (4 * c4 + 3 < NCH) acc[u] += (uint64_t)ch[u][4 * c4 + 3] * w.w;
      }
    }
    const uint32_t m = c_mods[t];
    const uint32_t yt = ymul ? __ldg(ymul + t) : 1u;
    const uint32_t i32 = c_inv32[t];
    const uint32_t c32 = c_pow32m[t];  // 2^32 mod m
#pragma unroll
    for (int u = 0; u < RE; ++u) {
      // acc = ah 2^32 + al (ah < 2^20): ((ah mod m) c32 + al) mod m in 32-bit Barrett steps
      const uint32_t ah = (uint32_t)(acc[u] >> 32), al = (uint32_t)acc[u];
      uint32_t r1 = ah - __umulhi(ah, i32) * m;
      if (r1 >= m) r1 -= m;
      const uint32_t x1 = r1 * c32;  // < 2^32
      uint32_t r2 = x1 - __umulhi(x1, i32) * m;
      if (r2 >= m) r2 -= m;
      uint32_t r3 = al - __umulhi(al, i32) * m;
      if (r3 >= m) r3 -= m;
      uint32_t rs = r2 + r3;
      if (rs >= m) rs -= m;
      int32_t res = (int32_t)rs;
      if (ymul) {  // res y < 2^32: one 32-bit Barrett step and one correction
        const uint32_t x = (uint32_t)res * yt;
        uint32_t r2 = x - __umulhi(x, i32) * m;
        if (r2 >= m) r2 -= m;
        res = (int32_t)r2;
      }
      if (res > (int32_t)(m >> 1)) res -= (int32_t)m;
      if (neg[u]) res = -res;
      if (!live[u]) res = 0;
      const int32_t lo = ((res + 128) & 255) - 128;
      const int32_t hi = (res - lo) >> 8;
      o[(int64_t)(2 * t) * plane + u * kq] = __int2bfloat16_rn(lo);
      o[(int64_t)(2 * t + 1) * plane + u * kq] = __int2bfloat16_rn(hi);
    }
  }
}

// nch: 32-bit chunks of the largest |X| of the operand.
static void launch_residues(int nch, int64_t n, cudaStream_t s, const BallsView &X, bool is_b,
                            int64_t rows, int64_t k0, int64_t K, int64_t Kp, int64_t ld,
                            const int64_t *bot, int NM, const uint32_t *pw32, int pw_stride,
                            const uint32_t *ymul, __nv_bfloat16 *out, const SplitOut &ro,
                            const int64_t *top, const int64_t *radtop, const int64_t *plustop) {
#define ARB_RES(NCH_, RE_)                                                                    \
  residue_split_kernel<NCH_, RE_><<<(unsigned)((n / RE_ + 127) / 128), 128,                   \
                                    (size_t)NM * ((NCH_ + 3) / 4 * 4) * 4, s>>>(              \
      X, is_b, rows, k0, K, Kp, ld, bot, NM, pw32, pw_stride, ymul, out, ro, top, radtop,     \
      plustop)
  if (nch <= 4) ARB_RES(4, 2);
  else if (nch <= 6) ARB_RES(6, 2);
  else if (nch <= 8) ARB_RES(8, 2);
  else if (nch <= 11) ARB_RES(11, 2);
  else if (nch <= 14) ARB_RES(14, 2);
  else if (nch <= 18) ARB_RES(18, 1);
  else if (nch <= 24) ARB_RES(24, 1);
  else if (nch <= 34) ARB_RES(34, 1);
  else if (nch <= 40) ARB_RES(40, 1);
  else ARB_RES(CRT_MAX_CHUNKS32, 1);
#undef ARB_RES
}

// ---- Residues on the 8-bit warp-level MMA, for operands beyond the tensor-core residue kernel
// (more moduli, chunks or shared memory than it takes).  With the bytes x_d of the scaled |X|
// (d < 32 KS, zero past |X|) and the unsigned bytes l, h of w_{t,d} = 2^(8d) mod m_t (times y_t
// for B), X mod m_t = (S_l + 256 S_h) mod m_t with S_b = sum_d x_d (byte b of w_{t,d}): an
// unsigned byte product on mma.sync m16n8k32 whose s32 sums are exact (|S| <= 224 255 255).  A
// warp takes 32 consecutive entries of the [rows][Kp] layout: each lane cuts its entry into
// 32-bit chunks (residue_chunks32) and writes its radius operands as residue_split_kernel does,
// the chunks reach the A fragments through shared memory, and each lane reduces the column pairs
// (2t, 2t + 1) it holds for two rows to balanced residues and stores their bytes.
constexpr int RQ_WARPS = 8;
constexpr size_t RQ_SMEM_MAX = 227 * 1024;  // opt-in shared memory of one CTA
constexpr float RQ_MAGIC = 12582912.0f;     // 1.5 * 2^23: adding it rounds |v| < 2^22 to an integer

__device__ __forceinline__ void mma_u8u8(int32_t (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm("mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int NCH>
constexpr int rq_ks() {
  return (4 * NCH + 31) / 32;
}

// Shared-memory bytes of residue_mma_kernel<NCH> for NM moduli.
template <int NCH>
static size_t rq_smem_bytes(int NM) {
  constexpr int KS = rq_ks<NCH>();
  const size_t N2 = (size_t)(2 * NM + 31) / 32 * 32;
  return N2 * (32 * KS + 16) + (size_t)(NM + 3) / 4 * 32 +
         (size_t)RQ_WARPS * 32 * (8 * KS + 1) * 4 + (size_t)RQ_WARPS * 32 * 4;
}

template <int NCH>
__global__ void __launch_bounds__(32 * RQ_WARPS) residue_mma_kernel(
    const BallsView X, bool is_b, int64_t rows, int64_t k0, int64_t K, int64_t Kp, int64_t ld,
    const int64_t *bot, int NM, const uint8_t *w8r, int KR, const float *rinv,
    __nv_bfloat16 *out, SplitOut ro, const int64_t *top, const int64_t *radtop,
    const int64_t *plustop) {
  constexpr int KS = rq_ks<NCH>();
  constexpr int CW = 8 * KS + 1;  // chunk row stride in words (odd: conflict-free columns)
  const int N2 = (2 * NM + 31) / 32 * 32, WS = 32 * KS + 16;
  extern __shared__ uint4 smem_u4[];
  uint8_t *sW = (uint8_t *)smem_u4;                           // [N2][WS] weight bytes
  uint32_t *sMod = (uint32_t *)(sW + (size_t)N2 * WS);        // [NM] m_t
  float *sR = (float *)(sMod + (NM + 3) / 4 * 4);             // [NM] 1 / m_t
  uint32_t *sCh = (uint32_t *)(sR + (NM + 3) / 4 * 4);        // [warps][32][CW] chunks
  uint32_t *sFl = sCh + RQ_WARPS * 32 * CW;                   // [warps][32] 1: live, 2: negative
  {
    const int c16 = 2 * KS;  // 16-byte pieces of a row's 32 KS bytes
    for (int q = threadIdx.x; q < N2 * c16; q += blockDim.x) {
      const int n = q / c16, u = q - n * c16;
      *(uint4 *)(sW + (size_t)n * WS + 16 * u) = __ldg((const uint4 *)(w8r + (size_t)n * KR) + u);
    }
    for (int t = threadIdx.x; t < NM; t += blockDim.x) {
      sMod[t] = c_mods[t];
      sR[t] = __ldg(rinv + t);
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  uint32_t *sChw = sCh + warp * 32 * CW;
  uint32_t *sFlw = sFl + warp * 32;
  const int64_t n = rows * Kp, plane = rows * Kp, ntile = (n + 31) / 32;
  const int nchunks = N2 / 32;
  for (int64_t tile = (int64_t)blockIdx.x * RQ_WARPS + warp; tile < ntile;
       tile += (int64_t)gridDim.x * RQ_WARPS) {
    // this lane's entry: chunks, sign, radius operands
    {
      const int64_t L = 32 * tile + lane;
      uint32_t ch[NCH];
#pragma unroll
      for (int c = 0; c < NCH; ++c) ch[c] = 0;
      uint32_t fl_out = 0;
      if (L < n) {
        const int64_t r = L / Kp, k = L - r * Kp;
        Mag absm{0u, 0}, rad{0u, 0};
        if (k < K) {
          const int64_t e = is_b ? ((k0 + k) * ld + r) : (r * ld + k0 + k);
          const uint32_t fl = __ldg(X.flags + e);
          const int64_t ex = __ldg(X.exp + e);
          if (!(fl & (ARBGPU_FLAG_ZERO | SPECIAL_MASK))) {
            fl_out = 1u | ((fl & ARBGPU_FLAG_SIGN) ? 2u : 0u);
            const int64_t sh = ex - 64LL * X.nlimbs - bot[r];
            residue_chunks32<NCH>(X, e, sh, ch);
            if (ro.r1 || ro.r2) absm = mid_upper(X, e, ex);
          }
          if (ro.r1 || ro.r2) rad = Mag{__ldg(X.rad_man + e), __ldg(X.rad_exp + e)};
        }
        if (ro.r1 || ro.r2) {
          const int64_t off = r * Kp + k;
          if (!is_b) {
            if (ro.r1) put_small_digits(window_up(absm.man, absm.exp, top[r]), ro.r1 + off, plane);
            if (ro.r2) put_small_digits(window_up(rad.man, rad.exp, radtop[r]), ro.r2 + off, plane);
          } else {
            if (ro.r1) put_small_digits(window_up(rad.man, rad.exp, radtop[r]), ro.r1 + off, plane);
            if (ro.r2) {
              const Mag plus = mag_add_up(absm, rad);
              put_small_digits(window_up(plus.man, plus.exp, plustop[r]), ro.r2 + off, plane);
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 8 * KS; ++c) sChw[lane * CW + c] = (c < NCH && (fl_out & 1u)) ? ch[c] : 0u;
      sFlw[lane] = fl_out;
    }
    __syncwarp();
    // A fragments: register r of row tile mt holds chunk 8 ks + tig + 4 (r >> 1) (bytes
    // 32 ks + 4 tig .. (+16)) of row 16 mt + g + 8 (r & 1)
    uint32_t af[KS][2][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < 4; ++r)
          af[ks][mt][r] = sChw[(16 * mt + g + 8 * (r & 1)) * CW + 8 * ks + tig + 4 * (r >> 1)];
    uint32_t rfl[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) rfl[mt][h] = sFlw[16 * mt + 8 * h + g];
    __syncwarp();
    for (int nc = 0; nc < nchunks; ++nc) {
      int32_t acc[2][4][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const uint8_t *wrow = sW + (size_t)(32 * nc + 8 * nt + g) * WS + 32 * ks + 4 * tig;
          const uint32_t b0 = *(const uint32_t *)wrow, b1 = *(const uint32_t *)(wrow + 16);
          mma_u8u8(acc[0][nt], af[ks][0], b0, b1);
          mma_u8u8(acc[1][nt], af[ks][1], b0, b1);
        }
      // columns 2t, 2t + 1 of rows 16 mt + g (+ 8): t = 16 nc + 4 nt + tig.  With 0 <= S_b <
      // 2^24 (exact in FP32): r_h = S_h mod m (|r_h| <= m, one FMA, exact), x = 256 r_h + S_l
      // (|x| < 2^25), then x mod m from a float quotient off by at most one, balanced.
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int t = 16 * nc + 4 * nt + tig;
        if (t >= NM) continue;
        const int32_t m = (int32_t)sMod[t], hm = m >> 1;
        const float mf = (float)m, rm = sR[t];
        __nv_bfloat16 *o0 = out + (int64_t)(2 * t) * plane + 32 * tile;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int row = 16 * mt + 8 * h + g;
            if (32 * tile + row >= n) continue;
            const float fh = (float)acc[mt][nt][2 * h + 1];
            const float qh = __fadd_rn(__fmaf_rn(fh, rm, RQ_MAGIC), -RQ_MAGIC);
            const int32_t x = 256 * (int32_t)__fmaf_rn(-qh, mf, fh) + acc[mt][nt][2 * h];
            const float q = __fadd_rn(__fmaf_rn((float)x, rm, RQ_MAGIC), -RQ_MAGIC);
            int32_t res = x - (int32_t)q * m;
            if (res > hm) res -= m;
            if (res > hm) res -= m;
            if (res < -hm) res += m;
            if (res < -hm) res += m;
            if (rfl[mt][h] & 2u) res = -res;
            if (!(rfl[mt][h] & 1u)) res = 0;
            const int32_t lo = ((res + 128) & 255) - 128;
            const int32_t hi = (res - lo) >> 8;
            o0[row] = __float2bfloat16_rn((float)lo);
            o0[plane + row] = __float2bfloat16_rn((float)hi);
          }
      }
    }
  }
}

// The MMA residue kernel for nch chunks; false when it does not take the operand
// (ARBGPU_RESIDUE_MMA=0 also declines).
static bool launch_residues_mma(arbgpu_ctx *ctx, int nch, cudaStream_t s, const BallsView &X,
                                bool is_b, int64_t rows, int64_t k0, int64_t K, int64_t Kp,
                                int64_t ld, const int64_t *bot, int NM, const uint8_t *w8r, int KR,
                                const float *rinv, __nv_bfloat16 *out, const SplitOut &ro,
                                const int64_t *top, const int64_t *radtop,
                                const int64_t *plustop) {
  const char *e = getenv("ARBGPU_RESIDUE_MMA");
  if ((e && !strcmp(e, "0")) || !w8r || NM < 1 || NM > CRT_MAX_MODULI || nch > CRT_MAX_CHUNKS32)
    return false;
  const int64_t ntile = (rows * Kp + 31) / 32;
  int64_t grid = (ntile + RQ_WARPS - 1) / RQ_WARPS;
  if (grid > 2LL * ctx->sm_count) grid = 2LL * ctx->sm_count;
  if (grid < 1) return true;
  const int dev = ctx->device & 255;
#define ARB_RQ(NCH_)                                                                          \
  do {                                                                                        \
    if (32 * rq_ks<NCH_>() > KR) return false;                                                \
    const size_t smem = rq_smem_bytes<NCH_>(NM);                                              \
    if (smem > RQ_SMEM_MAX) return false;                                                     \
    static bool attr_done[256] = {};                                                          \
    if (!attr_done[dev]) {                                                                    \
      if (cudaFuncSetAttribute(residue_mma_kernel<NCH_>,                                      \
                               cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                               (int)RQ_SMEM_MAX) != cudaSuccess)                              \
        return false;                                                                         \
      attr_done[dev] = true;                                                                  \
    }                                                                                         \
    residue_mma_kernel<NCH_><<<(unsigned)grid, 32 * RQ_WARPS, smem, s>>>(                     \
        X, is_b, rows, k0, K, Kp, ld, bot, NM, w8r, KR, rinv, out, ro, top, radtop, plustop); \
  } while (0)
  if (nch <= 24)
    ARB_RQ(24);
  else if (nch <= 32)
    ARB_RQ(32);
  else if (nch <= 40)
    ARB_RQ(40);
  else
    ARB_RQ(CRT_MAX_CHUNKS32);
#undef ARB_RQ
  return true;
}

// ---- Residues on the tensor cores.  With the signed base-256 digits x_d = ±(byte d of |X|)
// (d < 4 NCH, the sign of X on every digit),
//
//     X mod m_t = (sum_d x_d w_{t,d}) mod m_t,   w_{t,d} = 2^(8d) mod m_t (times y_t for B),
//
// is a product of a digit matrix [entries][digits] and a weight table [digits][(t, byte)]: the
// balanced weight w (|w| < m_t / 2) is written as 256 h + l with l, h in [-128, 128], column 2t
// holding l and 2t + 1 holding h.  Every product is at most 255 * 128 in magnitude and at most 128
// of them are summed, so each FP32 sum S is an integer with |S| < 2^22: exact.  The drain reduces
// x = S_l + 256 S_h (|x| < 2^31) in FP32 without rounding error: q = rint(x / m) from a rounded x
// is off by at most one for |x / m| < 2^16, r = (256 S_h - q m) + S_l is exact (every partial
// result is an integer below 2^24), and one more rint(r / m) step balances r.
//
// Roles of a CTA (one per SM, persistent over tiles of 128 entries): two producer warpgroups
// (alternate tiles) write each entry's digits into a ring of shared-memory tiles, one warp issues the MMAs into a ring of
// TMEM accumulators, and ND drain warpgroups take the tiles in turn, reduce them, stage the
// residue planes in shared memory and write them with a TMA store.  Every wait on an mbarrier
// gives up after ~2 s, sets ARBGPU_ERR_TIMEOUT and leaves the loop.
constexpr int RT_ROWS = 128;            // entries per tile: the MMA's M
constexpr int RT_TILE = RT_ROWS * 128;  // bytes of one 64-digit slab of a tile (SW128, K-major)
constexpr int RT_MAX_ND = 3;            // drain warpgroups
constexpr int RT_MAX_NS = 4;            // digit tiles in flight
constexpr int RT_NP = 2;      // producer warpgroups (tiles i = p mod RT_NP go to producer p)
constexpr int RT_MAX_THREADS = 32 * (4 * RT_MAX_ND + 4 * RT_NP + 1);
constexpr float RT_MAGIC = 12582912.0f; // 1.5 * 2^23: adding it rounds |v| < 2^22 to an integer
// Dynamic shared memory of at least this much keeps one CTA per SM, so the CTA's 512 TMEM columns
// are always free when it starts.
constexpr size_t RT_SMEM_MIN = 120 * 1024;
constexpr size_t RT_SMEM_MAX = 227 * 1024;

struct RtShared {
  uint64_t a_full[RT_MAX_NS], a_empty[RT_MAX_NS];        // digit tiles
  uint64_t t_full[RT_MAX_ND + 1], t_empty[RT_MAX_ND + 1];  // TMEM accumulators
  uint32_t tmem_base;
  int never;  // an abort flag nothing sets
  uint32_t info[RT_MAX_NS][RT_ROWS];  // radius operands u1 | u2 << 14 of each tile row
};

__device__ __forceinline__ void named_bar(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// A barrier of n threads that also returns whether any of them passed `p` true.
__device__ __forceinline__ bool named_bar_or(int id, int n, bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, %2, %3, q;\n"
      " selp.u32 %0, 1, 0, o;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *tm, const void *src, int c0, int c1,
                                             int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
          (uint64_t)tm),
      "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void cp_async(void *dst, const void *src, int bytes) {
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_pending() {  // at most N groups still in flight
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Top limbs of an entry the residue step can need: |X| = L 2^sh < 2^(32 NCH) and L's top bit is
// bit 64 nl - 1, so the nonzero bits of L that reach X lie in its top ceil(NCH / 2) + 1 limbs.
template <int NCH>
constexpr int rt_top_limbs() {
  return (NCH + 1) / 2 + 1;
}
// Per producer thread, the raw fields of its entries of its next RT_PD tiles, staged by cp.async:
// words [0] exp, [1] bot, [2] flags | rad_man << 32, [3] rad_exp, [4] and [5] the two radius
// windows, [6] the line's omission exponent, [7 ...] the top limbs (word 7 + i = limb
// nl - NLW + i).  Layout [RT_NP][RT_PD][128][SW].
constexpr int RT_SLOT_FIXED = 7;
constexpr int RT_PD = 2;  // tiles staged ahead by each producer thread

// The float sg * b for byte b of `w` (exact): sg (2^23 + b) + sgb with sgb = -sg 2^23.
__device__ __forceinline__ float signed_byte(uint32_t w, int b, float sg, float sgb) {
  return __fmaf_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)b)), sg, sgb);
}
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *(const uint32_t *)&p;
}

// One operand of the residue step: A (rows of A, tiles of 2 rows x 64 inner positions) or B
// (columns of B, tiles of 4 columns x 32 inner positions).
struct RtSide {
  BallsView X;
  int64_t rows, ld;
  const int64_t *bot;    // scan: per-line lowest exponent
  const int64_t *top, *radtop, *plustop;  // the radius windows' exponents (plustop: B only)
  SplitOut ro;           // radius operands written directly (when not part of the staged planes)
  const uint16_t *wtab;  // [NPAD][128] BF16 weight table of this operand
  // negligible-limb omission: per line, the exponent tau below which the line's bits were
  // dropped (INT64_MIN: none); every nonzero entry of such a line carries 2^tau more radius
  const int64_t *trunc = nullptr;
};

struct RtArgs {
  RtSide side[2];  // 0: A, 1: B
  int64_t k0, K, Kp;
  int NM, NPAD, NS, ND, wg_cols, NPL;  // NPL: staged planes per tile (2 NM, plus 4 radius planes)
  uint32_t tcols;
  const float *rinv;  // [NM] 1 / m_t
  int *status;
};

template <bool IS_B>
struct RtGeom {
  static constexpr int JT = IS_B ? 4 : 2;  // operand lines per tile
  static constexpr int KT = RT_ROWS / JT;  // inner positions per tile (a divisor of Kp)
  // producer thread pt's entry (pj, pk): for B, the four threads of a 32-byte sector of a row of
  // B take consecutive columns, and the eight threads of a quarter warp fill tile rows with
  // distinct (row mod 8), so their swizzled 16-byte stores hit distinct banks
  __device__ static int pj(int pt) { return IS_B ? ((pt >> 3) & 3) : (pt >> 6); }
  __device__ static int pk(int pt) { return IS_B ? ((pt & 7) + 8 * (pt >> 5)) : (pt & 63); }
};

// Stage the raw fields of producer thread pt's entry of tile (tr, tk) of one side into `slot`.
template <int NCH, bool IS_B>
__device__ __forceinline__ void rt_prefetch(const RtArgs &a, const RtSide &sd, uint64_t *slot,
                                            int pt, int tr, int tk, bool want_rad, bool w1,
                                            bool w2) {
  using G = RtGeom<IS_B>;
  constexpr int NLW = rt_top_limbs<NCH>();
  const int64_t r = (int64_t)tr * G::JT + G::pj(pt), k = (int64_t)tk * G::KT + G::pk(pt);
  if (r >= sd.rows || k >= a.K) return;
  const BallsView &X = sd.X;
  const int lbase = X.nlimbs - NLW;
  const int64_t e = IS_B ? ((a.k0 + k) * sd.ld + r) : (r * sd.ld + a.k0 + k);
  cp_async(slot, X.exp + e, 8);
  cp_async(slot + 1, sd.bot + r, 8);
  cp_async(slot + 2, X.flags + e, 4);
  if (want_rad) {
    cp_async((uint32_t *)(slot + 2) + 1, X.rad_man + e, 4);
    cp_async(slot + 3, X.rad_exp + e, 8);
    if (w1) cp_async(slot + 4, (IS_B ? sd.radtop : sd.top) + r, 8);
    if (w2) cp_async(slot + 5, (IS_B ? sd.plustop : sd.radtop) + r, 8);
    if (sd.trunc) cp_async(slot + 6, sd.trunc + r, 8);
  }
#pragma unroll
  for (int i = 0; i < NLW; ++i)
    if (lbase + i >= 0)
      cp_async(slot + RT_SLOT_FIXED + i, X.limbs + (int64_t)(lbase + i) * X.stride + e, 8);
}

// The 32-bit chunks of |X| (scaled), the sign and the radius operands of producer thread pt's
// entry of tile (tr, tk), from its staged fields.
template <int NCH, bool IS_B>
__device__ __forceinline__ void rt_entry(const RtArgs &a, const RtSide &sd, const uint64_t *slot,
                                         int pt, int tr, int tk, bool want_rad, bool w1, bool w2,
                                         uint32_t (&ch)[NCH], float &sg, uint32_t &info) {
  using G = RtGeom<IS_B>;
  constexpr int NLW = rt_top_limbs<NCH>();
  const int64_t r = (int64_t)tr * G::JT + G::pj(pt), k = (int64_t)tk * G::KT + G::pk(pt);
  if (r >= sd.rows || k >= a.K) return;
  const int nl = sd.X.nlimbs;
  const int lbase = nl - NLW;  // limb index of the slot's first limb (lower ones are not read)
  const int jlo = lbase < 0 ? -2 * lbase : 0;  // first 32-bit limb word that exists
  const uint32_t *Wd = (const uint32_t *)(slot + RT_SLOT_FIXED);
  const int64_t ex = (int64_t)slot[0];
  const uint64_t w2f = slot[2];
  const uint32_t fl = (uint32_t)w2f;
  Mag absm{0u, 0};
  if (!(fl & (ARBGPU_FLAG_ZERO | SPECIAL_MASK))) {
    if (fl & ARBGPU_FLAG_SIGN) sg = -1.0f;
    // chunk c = bits [32c - sh, 32c - sh + 32) of L: a funnel shift of the slot's words q0 + c
    // and q0 + c + 1 by b, with 32 q0 + b = -sh - 64 lbase
    const int64_t p0 = -(ex - 64LL * nl - (int64_t)slot[1]) - 64LL * lbase;
    if (p0 > -32LL * (NCH + 1) && p0 < 64LL * NLW) {
      const int q0 = (int)(p0 >> 5), b = (int)(p0 & 31);
      uint32_t wv[NCH + 1];
#pragma unroll
      for (int c = 0; c <= NCH; ++c) {
        const int j = q0 + c;
        wv[c] = ((unsigned)(j - jlo) < (unsigned)(2 * NLW - jlo)) ? Wd[j] : 0u;
      }
#pragma unroll
      for (int c = 0; c < NCH; ++c) ch[c] = __funnelshift_r(wv[c], wv[c + 1], b);
    }
    if (want_rad) {
      const uint64_t top = slot[RT_SLOT_FIXED + NLW - 1];  // limb nl - 1
      uint64_t bm = (top >> 34) + 1;  // 30-bit upper bound of |m| (Section III-E)
      int64_t ee = ex;
      if (bm == ((uint64_t)1 << 30)) {
        bm >>= 1;
        ee += 1;
      }
      absm = Mag{(uint32_t)bm, ee};
    }
  }
  if (want_rad) {
    Mag rad{(uint32_t)(w2f >> 32), (int64_t)slot[3]};
    if (sd.trunc && !(fl & (ARBGPU_FLAG_ZERO | SPECIAL_MASK))) {
      const int64_t t = (int64_t)slot[6];  // bits below 2^t were dropped from this line
      if (t != INT64_MIN) rad = mag_add_up(rad, Mag{1u << 29, t + 1});
    }
    uint32_t u1 = 0, u2 = 0;
    const int64_t f1 = (int64_t)slot[4], f2 = (int64_t)slot[5];
    if (!IS_B) {
      if (w1) u1 = window_up(absm.man, absm.exp, f1);
      if (w2) u2 = window_up(rad.man, rad.exp, f2);
    } else {
      if (w1) u1 = window_up(rad.man, rad.exp, f1);
      if (w2) {
        const Mag plus = mag_add_up(absm, rad);
        u2 = window_up(plus.man, plus.exp, f2);
      }
    }
    info = u1 | (u2 << 14);
  }
}

// Tiles [0, nTA) are those of A, the rest those of B; (side, tile row, tile column) of a tile.
struct RtTiles {
  int nTA, ntkA, ntkB;
  __device__ void locate(int tile, int &side, int &tr, int &tk) const {
    side = tile >= nTA;
    const int l = side ? tile - nTA : tile, ntk = side ? ntkB : ntkA;
    tr = l / ntk;
    tk = l - tr * ntk;
  }
};

// Both operands in one launch (the tiles of A, then those of B).  The producer thread reads the
// entry (pj, pk) of its side's tile (consecutive threads take consecutive elements of the operand
// in memory) and fills tile row pj KT + pk; the drain thread t reads TMEM lane t, i.e. the entry
// (t / KT, t % KT), and stages its residues at [plane][t], the layout of the TMA store's box
// {KT, JT, planes}.
template <int NCH>
__global__ void __launch_bounds__(RT_MAX_THREADS, 1)
    residue_tc_kernel(const __grid_constant__ CUtensorMap tmoA,
                      const __grid_constant__ CUtensorMap tmoB, const __grid_constant__ RtArgs a) {
  constexpr int KD = (4 * NCH + 63) / 64;  // 64-digit slabs
  constexpr int NLW = rt_top_limbs<NCH>();
  constexpr int SW = RT_SLOT_FIXED + NLW;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const int NS = a.NS, ND = a.ND, NB = a.ND + 1;
  const size_t wside = (size_t)KD * a.NPAD * 128;  // one side's weight slabs
  uint8_t *sW = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = sW + 2 * wside;
  uint16_t *sO = (uint16_t *)(sA + (size_t)NS * KD * RT_TILE);
  uint64_t *sSlot = (uint64_t *)(sO + (size_t)ND * a.NPL * RT_ROWS);
  float2 *sMod = (float2 *)(sSlot + (size_t)RT_NP * RT_PD * SW * RT_ROWS);
  RtShared *sh = (RtShared *)(sMod + a.NPAD / 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mma_warp = 4 * ND + 4 * RT_NP;

  if (threadIdx.x == 0) {
    for (int q = 0; q < NS; ++q) {
      mbar_init(&sh->a_full[q], RT_ROWS);
      mbar_init(&sh->a_empty[q], RT_ROWS);
    }
    for (int q = 0; q < NB; ++q) {
      mbar_init(&sh->t_full[q], 1);
      mbar_init(&sh->t_empty[q], RT_ROWS);
    }
    sh->never = 0;
    fence_mbar_init();
  }
  if (warp == mma_warp) {
    tmem_alloc(&sh->tmem_base, a.tcols);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    tma_prefetch_desc(&tmoA);
    tma_prefetch_desc(&tmoB);
  }
  // both weight tables into K-major slabs of 64 columns with the 128-byte swizzle
  for (int q = threadIdx.x; q < 2 * a.NPAD * 8 * KD; q += blockDim.x) {
    const int sd = q / (a.NPAD * 8 * KD), qq = q - sd * a.NPAD * 8 * KD;
    const int n = qq / (8 * KD), c = qq - n * 8 * KD;
    const uint4 v = __ldg((const uint4 *)(a.side[sd].wtab + (size_t)n * 128) + c);
    *(uint4 *)(sW + sd * wside + (size_t)(c >> 3) * a.NPAD * 128 + (size_t)n * 128 +
               (((c & 7) ^ (n & 7)) << 4)) = v;
  }
  for (int q = threadIdx.x; q < a.NPAD / 2; q += blockDim.x)
    sMod[q] = q < a.NM ? make_float2((float)c_mods[q], __ldg(a.rinv + q)) : make_float2(1.0f, 1.0f);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // the operands and scan results come from earlier kernels

  RtTiles tl;
  tl.ntkA = (int)(a.Kp / RtGeom<false>::KT);
  tl.ntkB = (int)(a.Kp / RtGeom<true>::KT);
  tl.nTA = (int)((a.side[0].rows + 1) / 2) * tl.ntkA;
  const int nT = tl.nTA + (int)((a.side[1].rows + 3) / 4) * tl.ntkB;  // below 2^30 (host)
  // this CTA's tiles: blockIdx.x + i gridDim.x, i = 0, 1, ...
  const int ntiles = nT > (int)blockIdx.x ? (nT - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const bool rad_box = a.NPL > 2 * a.NM;

  if (warp >= 4 * ND && warp < mma_warp) {
    // ------------------------------------------------ producers: digits of 128 entries per tile
    const int p = (warp - 4 * ND) >> 2, pt = threadIdx.x - 128 * (ND + p);
    uint64_t *pslots = sSlot + (size_t)p * RT_PD * RT_ROWS * SW;
    bool want[2], w1[2], w2[2];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      w1[sd] = rad_box || a.side[sd].ro.r1;
      w2[sd] = rad_box || a.side[sd].ro.r2;
      want[sd] = w1[sd] || w2[sd];
    }
    // staged copies of this producer's j-th tile (the CTA's tile i = p + j RT_NP) into slot
    // j mod RT_PD; one commit group per call, empty past the last tile
    int fj = 0;
    auto prefetch = [&]() {
      const int j = fj++;
      const int i = p + j * RT_NP;
      if (i < ntiles) {
        uint64_t *slot = pslots + ((size_t)(j % RT_PD) * RT_ROWS + pt) * SW;
        int sd, tr, tk;
        tl.locate((int)blockIdx.x + i * (int)gridDim.x, sd, tr, tk);
        if (sd)
          rt_prefetch<NCH, true>(a, a.side[1], slot, pt, tr, tk, want[1], w1[1], w2[1]);
        else
          rt_prefetch<NCH, false>(a, a.side[0], slot, pt, tr, tk, want[0], w1[0], w2[0]);
      }
      cp_async_commit();
    };
    for (int j = 0; j < RT_PD; ++j) prefetch();
    for (int j = 0, i = p; i < ntiles; ++j, i += RT_NP) {
      const uint64_t *slot = pslots + ((size_t)(j % RT_PD) * RT_ROWS + pt) * SW;
      const int s = i % NS;
      int sd, tr, tk;
      tl.locate((int)blockIdx.x + i * (int)gridDim.x, sd, tr, tk);
      uint32_t ch[NCH];
#pragma unroll
      for (int c = 0; c < NCH; ++c) ch[c] = 0;
      uint32_t info = 0;
      float sg = 1.0f;
      cp_async_wait_pending<RT_PD - 1>();  // the groups of the later RT_PD - 1 tiles may fly
      int prow;
      if (sd) {
        rt_entry<NCH, true>(a, a.side[1], slot, pt, tr, tk, want[1], w1[1], w2[1], ch, sg, info);
        prow = RtGeom<true>::pj(pt) * RtGeom<true>::KT + RtGeom<true>::pk(pt);
      } else {
        rt_entry<NCH, false>(a, a.side[0], slot, pt, tr, tk, want[0], w1[0], w2[0], ch, sg, info);
        prow = RtGeom<false>::pj(pt) * RtGeom<false>::KT + RtGeom<false>::pk(pt);
      }
      // every slot value is in registers now: stage tile j + RT_PD into the same slot
      prefetch();
      // the digit tile s is free once the drain of the tile that used it has read its info
      if (!mbar_wait_sleep(&sh->a_empty[s], ((i / NS) & 1) ^ 1)) {
        set_status(a.status, ARBGPU_ERR_TIMEOUT);
        break;
      }
      sh->info[s][prow] = info;
      const float sgb = -8388608.0f * sg;
      uint8_t *row = sA + (size_t)s * KD * RT_TILE + (size_t)prow * 128;
#pragma unroll
      for (int sl = 0; sl < KD; ++sl) {
#pragma unroll
        for (int c16 = 0; c16 < 8; ++c16) {
          const int c = 16 * sl + 2 * c16;  // first of the two 32-bit chunks of these 16 bytes
          uint32_t wv[4] = {0u, 0u, 0u, 0u};
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (c + h < NCH) {
              const uint32_t x = ch[c + h];
              wv[2 * h] = bf16x2_bits(signed_byte(x, 0, sg, sgb), signed_byte(x, 1, sg, sgb));
              wv[2 * h + 1] =
                  bf16x2_bits(signed_byte(x, 2, sg, sgb), signed_byte(x, 3, sg, sgb));
            }
          }
          *(uint4 *)(row + (size_t)sl * RT_TILE + ((c16 ^ (prow & 7)) << 4)) =
              make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
      }
      fence_async_smem();
      mbar_arrive(&sh->a_full[s]);
    }
    cp_async_wait_all();
  } else if (warp == mma_warp) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(RT_ROWS, a.NPAD);
      for (int i = 0; i < ntiles; ++i) {
        const int s = i % NS, b = i % NB;
        const int sd = (int)blockIdx.x + i * (int)gridDim.x >= tl.nTA;
        if (!mbar_wait_sleep(&sh->a_full[s], (i / NS) & 1) ||
            !mbar_wait_sleep(&sh->t_empty[b], ((i / NB) & 1) ^ 1)) {
          set_status(a.status, ARBGPU_ERR_TIMEOUT);
          break;
        }
        tc_fence_after();
        const uint32_t tm = sh->tmem_base + (uint32_t)(b * a.wg_cols);
#pragma unroll
        for (int sl = 0; sl < KD; ++sl) {
          const uint64_t ad = sw128_desc(smem_u32(sA + ((size_t)s * KD + sl) * RT_TILE));
          const uint64_t bd = sw128_desc(smem_u32(sW + sd * wside + (size_t)sl * a.NPAD * 128));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            umma_bf16(tm, ad + 2 * kk, bd + 2 * kk, idesc, (sl > 0 || kk > 0) ? 1u : 0u);
        }
        umma_commit(&sh->t_full[b]);
      }
    }
  } else {
    // ------------------------------------------------ drain warpgroup d: tiles i = d (mod ND)
    const int d = warp >> 2, t = threadIdx.x & 127, wq = warp & 3;
    uint16_t *so = sO + (size_t)d * a.NPL * RT_ROWS + t;  // plane p of this row at so[p * 128]
    for (int i = d; i < ntiles; i += ND) {
      int sd, tr, tk;
      tl.locate((int)blockIdx.x + i * (int)gridDim.x, sd, tr, tk);
      const int JT = sd ? RtGeom<true>::JT : RtGeom<false>::JT, KT = RT_ROWS / JT;
      const int s = i % NS, b = i % NB;
      // (the wait on a_full, complete by then, orders the producer's info writes before the
      // reads below)
      const bool got = mbar_wait_sleep(&sh->t_full[b], (i / NB) & 1) &&
                       mbar_wait_sleep(&sh->a_full[s], (i / NS) & 1);
      if (t == 0) tma_store_wait_read();  // this warpgroup's previous store has read its staging
      if (named_bar_or(1 + d, RT_ROWS, !got)) {
        if (t == 0) set_status(a.status, ARBGPU_ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      const uint32_t info = sh->info[s][t];
      mbar_arrive(&sh->a_empty[s]);
      const uint32_t tm_lane =
          sh->tmem_base + (uint32_t)(b * a.wg_cols) + ((uint32_t)(32 * wq) << 16);
      for (int c0 = 0; c0 < 2 * a.NM; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tm_lane + (uint32_t)c0, v);
        tmem_wait_ld();
        // eight moduli at once (sMod is padded to a multiple of eight), then the stores of the
        // real ones
        uint32_t bits[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float2 mi = sMod[(c0 >> 1) + u];  // m_t, 1 / m_t
          const float sl = __uint_as_float(v[2 * u]), sh_ = __uint_as_float(v[2 * u + 1]);
          const float xf = __fmaf_rn(sh_, 256.0f, sl);
          const float q = __fadd_rn(__fmaf_rn(xf, mi.y, RT_MAGIC), -RT_MAGIC);
          float rr = __fadd_rn(__fmaf_rn(-q, mi.x, sh_ * 256.0f), sl);
          const float q2 = __fadd_rn(__fmaf_rn(rr, mi.y, RT_MAGIC), -RT_MAGIC);
          rr = __fmaf_rn(-q2, mi.x, rr);  // balanced: |rr| <= (m - 1) / 2
          // rr = 256 h + l with l in [-128, 127]: h = rint(rr / 256 + 1 / 512)
          const float hi = __fadd_rn(
              __fadd_rn(__fmaf_rn(rr, 0.00390625f, 0.001953125f), RT_MAGIC), -RT_MAGIC);
          const float lo = __fmaf_rn(hi, -256.0f, rr);
          bits[u] = bf16x2_bits(lo, hi);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int tt = (c0 >> 1) + u;
          if (tt < a.NM) {
            so[(2 * tt) * RT_ROWS] = (uint16_t)bits[u];
            so[(2 * tt + 1) * RT_ROWS] = (uint16_t)(bits[u] >> 16);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&sh->t_empty[b]);
      if (rad_box) {
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          const uint32_t u = (info >> (14 * w)) & 0x3FFFu;  // u <= 2^13: two balanced digits
          const float d0 = (float)(((int)(u & 255u) ^ 128) - 128);
          const float d1 = (float)(((int)u - (int)d0) >> 8);
          const uint32_t bits = bf16x2_bits(d0, d1);
          so[(2 * a.NM + 2 * w) * RT_ROWS] = (uint16_t)bits;
          so[(2 * a.NM + 2 * w + 1) * RT_ROWS] = (uint16_t)(bits >> 16);
        }
      } else {
        const RtSide &side = a.side[sd];
        const int64_t r = (int64_t)tr * JT + t / KT, k = (int64_t)tk * KT + t % KT;
        if (r < side.rows && (side.ro.r1 || side.ro.r2)) {
          const int64_t plane = side.rows * a.Kp, off = r * a.Kp + k;
          if (side.ro.r1) put_small_digits(info & 0x3FFFu, side.ro.r1 + off, plane);
          if (side.ro.r2) put_small_digits((info >> 14) & 0x3FFFu, side.ro.r2 + off, plane);
        }
      }
      fence_async_smem();
      named_bar(1 + d, RT_ROWS);
      if (t == 0)
        tma_store_3d(sd ? &tmoB : &tmoA, sO + (size_t)d * a.NPL * RT_ROWS, tk * KT, tr * JT, 0);
    }
    if (t == 0) tma_store_wait_all();
  }
  pdl_trigger();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == mma_warp) tmem_dealloc(sh->tmem_base, a.tcols);
}

struct RtLayout {
  int KD, NPAD, NS, ND, wg_cols, NPL, SW;
  size_t smem;
};

static size_t residue_tc_smem_for(int KD, int NPAD, int NS, int ND, int NPL, int NM, int SW) {
  return 1024 + (size_t)2 * KD * NPAD * 128 + (size_t)NS * KD * RT_TILE +
         (size_t)ND * NPL * RT_ROWS * 2 + (size_t)RT_NP * RT_PD * SW * RT_ROWS * 8 +
         (size_t)NPAD / 2 * 8 + sizeof(RtShared);
}

// The kernel's shape for operands of at most `nch` 32-bit chunks and NM moduli; false when it
// does not fit (the CUDA-core residue kernel then runs).
static bool residue_tc_layout(int nch, int NM, bool rad_box, int64_t entries, RtLayout *L) {
  if (nch > 32 || NM > 128 || entries > ((int64_t)1 << 36)) return false;
  L->KD = (4 * nch + 63) / 64;
  L->NPAD = (2 * NM + 15) / 16 * 16;
  L->wg_cols = L->NPAD <= 128 ? 128 : 256;
  L->NPL = 2 * NM + (rad_box ? 4 : 0);
  const int ncls = nch <= 4 ? 4 : nch <= 8 ? 8 : nch <= 11 ? 11 : nch <= 16 ? 16 : nch <= 24 ? 24 : 32;
  L->SW = RT_SLOT_FIXED + (ncls + 1) / 2 + 1;
  if (L->NPL > 256) return false;
  const int nd_max = 512 / L->wg_cols - 1 < RT_MAX_ND ? 512 / L->wg_cols - 1 : RT_MAX_ND;
  for (int nd = nd_max; nd >= 1; --nd)
    for (int ns = RT_MAX_NS; ns >= 2; --ns) {
      const size_t s = residue_tc_smem_for(L->KD, L->NPAD, ns, nd, L->NPL, NM, L->SW);
      if (s <= RT_SMEM_MAX) {
        L->ND = nd;
        L->NS = ns;
        L->smem = s < RT_SMEM_MIN ? RT_SMEM_MIN : s;
        return true;
      }
    }
  return false;
}

// Residues of both operands in one launch; outA / outB: the [NPL][rows][Kp] planes of each side.
static arbgpu_status launch_residues_tc(arbgpu_ctx *ctx, const RtLayout &L, int nch,
                                        cudaStream_t s, RtArgs a, __nv_bfloat16 *outA,
                                        __nv_bfloat16 *outB) {
  a.NPAD = L.NPAD;
  a.NS = L.NS;
  a.ND = L.ND;
  a.wg_cols = L.wg_cols;
  a.NPL = L.NPL;
  a.tcols = 32;  // a power of two covering the ND + 1 accumulators
  while (a.tcols < (uint32_t)((L.ND + 1) * L.wg_cols)) a.tcols *= 2;
  a.status = ctx->status;
  const int64_t nT = ((a.side[0].rows + 1) / 2) * (a.Kp / 64) + ((a.side[1].rows + 3) / 4) * (a.Kp / 32);
  int64_t grid = nT;
  if (grid > ctx->sm_count) grid = ctx->sm_count;
  if (grid < 1) return ARBGPU_OK;
  CUtensorMap tmA, tmB;
  if (!make_residue_store_map(&tmA, outA, a.Kp, a.side[0].rows, L.NPL, 64, 2, L.NPL) ||
      !make_residue_store_map(&tmB, outB, a.Kp, a.side[1].rows, L.NPL, 32, 4, L.NPL))
    return ARBGPU_ERR_CUDA;
  const int dev = ctx->device & 255;
  const unsigned threads = 32u * (unsigned)(4 * L.ND + 4 * RT_NP + 1);
#define ARB_RTC(NCH_)                                                                      \
  do {                                                                                     \
    static bool attr_done[256] = {};                                                       \
    if (!attr_done[dev]) {                                                                 \
      if (cudaFuncSetAttribute(residue_tc_kernel<NCH_>,                                    \
                               cudaFuncAttributeMaxDynamicSharedMemorySize,                \
                               (int)RT_SMEM_MAX) != cudaSuccess)                           \
        return ARBGPU_ERR_CUDA;                                                            \
      attr_done[dev] = true;                                                               \
    }                                                                                      \
    launch_pdl(residue_tc_kernel<NCH_>, dim3((unsigned)grid), dim3(threads), L.smem, s,    \
               tmA, tmB, a);                                                               \
  } while (0)
  if (nch <= 4) ARB_RTC(4);
  else if (nch <= 8) ARB_RTC(8);
  else if (nch <= 11) ARB_RTC(11);
  else if (nch <= 16) ARB_RTC(16);
  else if (nch <= 24) ARB_RTC(24);
  else ARB_RTC(32);
#undef ARB_RTC
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

// Load the per-modulus constants into this device's constant memory (once per device).
static arbgpu_status ensure_crt_constants(int device) {
  static bool done[256] = {};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (done[device & 255]) return ARBGPU_OK;
  const CrtPlan *full = crt_plan(CRT_MAX_MODULI);
  if (!full) return ARBGPU_ERR_CUDA;
  std::vector<uint32_t> inv32(CRT_MAX_MODULI), p32(CRT_MAX_MODULI);
  for (int t = 0; t < CRT_MAX_MODULI; ++t) {
    inv32[t] = (uint32_t)((((uint64_t)1) << 32) / full->mods[t]);
    p32[t] = (uint32_t)((((uint64_t)1) << 32) % full->mods[t]);
  }
  if (cudaMemcpyToSymbol(c_mods, full->mods.data(), 4 * CRT_MAX_MODULI) != cudaSuccess ||
      cudaMemcpyToSymbol(c_inv, full->inv.data(), 8 * CRT_MAX_MODULI) != cudaSuccess ||
      cudaMemcpyToSymbol(c_inv32, inv32.data(), 4 * CRT_MAX_MODULI) != cudaSuccess ||
      cudaMemcpyToSymbol(c_pow32m, p32.data(), 4 * CRT_MAX_MODULI) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  done[device & 255] = true;
  return ARBGPU_OK;
}

// Per-entry windowed accumulator over several blocks, Algorithm 1 style: nacc limbs of two's
// complement at 2^base with base = top_i + top_j + bc(K) + 2 - 64 nacc (so the sum of all blocks
// fits), a count of ulps lost below the window, and a 30-bit radius.
struct AccView {
  uint64_t *acc;  // [nacc][M*N]
  uint32_t *err;  // [M*N]
  uint32_t *rman;
  int64_t *rexp;
  int nacc;
  int bcK;                                  // bit length bound of the number of summed products
  const int64_t *ftop_r[2], *ftop_c[2];     // whole-range row / column tops of the products summed
  // when set: per entry, max over the summed products and inner indices k of top(a_ik) + top(b_kj)
  // (INT64_MIN when every product is zero there), the tighter exponent bound (maxplus_top_kernel)
  const int64_t *etop = nullptr;
  int64_t ncols = 0;  // N, the row length of etop
};

// Exponent bound of the accumulated sum at (i, j); false when every product is zero there.
__device__ __forceinline__ bool acc_top(const AccView &v, int64_t i, int64_t j, int64_t &top) {
  if (v.etop) {
    top = v.etop[i * (v.ncols) + j];
    return top != INT64_MIN;
  }
  bool live = false;
  top = INT64_MIN;
  for (int q = 0; q < 2; ++q) {
    if (!v.ftop_r[q]) continue;
    const int64_t a = v.ftop_r[q][i], b = v.ftop_c[q][j];
    if (a == INT64_MIN || b == INT64_MIN) continue;
    live = true;
    top = a + b > top ? a + b : top;
  }
  return live;
}

__device__ __forceinline__ int64_t acc_base_of(const AccView &v, int64_t top) {
  return top + v.bcK + 2 - 64LL * v.nacc;
}

// Adds (-1)^negate T 2^sigma (T: nw two's-complement limbs, destroyed) into the window of entry
// idx: the bits of |T| below the window are dropped (truncated toward zero) and counted as one
// lost ulp.  top: the entry's exponent bound (acc_top).
__device__ __forceinline__ void acc_add_T(const AccView &v, int64_t idx, int64_t MN, uint64_t *T,
                                          int nw, int64_t sigma, int64_t top, bool negate) {
  const bool tneg = (T[nw - 1] >> 63) != 0;
  const bool neg = tneg != negate;
  if (tneg) {
    u128 c = 1;
    for (int k = 0; k < nw; ++k) {
      c += (u128)(~T[k]);
      T[k] = (uint64_t)c;
      c >>= 64;
    }
  }
  const int64_t sh = sigma - acc_base_of(v, top);  // T's bit 0 at bit sh of the window
  uint64_t W[24];
  bool lost = false;
  for (int q = 0; q < v.nacc; ++q) {
    // bits [64q - sh, 64q - sh + 64) of |T|
    const int64_t lo = 64LL * q - sh;
    const int64_t li = lo >= 0 ? (lo >> 6) : -((-lo + 63) >> 6);
    const int bi = (int)(lo - li * 64);
    const uint64_t w0 = (li >= 0 && li < nw) ? T[li] : 0;
    const uint64_t w1 = (li + 1 >= 0 && li + 1 < nw) ? T[li + 1] : 0;
    W[q] = bi ? ((w0 >> bi) | (w1 << (64 - bi))) : w0;
  }
  if (sh < 0) {  // bits of |T| below the window
    const int64_t cut = -sh;
    for (int64_t w = 0; w < (cut >> 6) && w < nw && !lost; ++w) lost = T[w] != 0;
    if (!lost && (cut & 63) && (cut >> 6) < nw)
      lost = (T[cut >> 6] & ((((uint64_t)1) << (cut & 63)) - 1)) != 0;
  }
  const uint64_t flip = neg ? ~(uint64_t)0 : 0;
  u128 c = neg ? 1 : 0;
  for (int q = 0; q < v.nacc; ++q) {
    const int64_t o = (int64_t)q * MN + idx;
    c += (u128)v.acc[o] + (W[q] ^ flip);
    v.acc[o] = (uint64_t)c;
    c >>= 64;
  }
  if (lost) v.err[idx] += 1;
}

// rad(idx) += r, rounded up.
__device__ __forceinline__ void acc_add_radius(const AccView &v, int64_t idx, Mag r) {
  if (!r.man) return;
  const Mag cur{v.rman[idx], v.rexp[idx]};
  const Mag nr = mag_add_up(cur, r);
  v.rman[idx] = nr.man;
  v.rexp[idx] = nr.exp;
}

struct RoundArgs {
  IntProduct mid;
  IntProduct rp1, rp2;  // radius products (ND = 0 when absent)
  const int64_t *rtop, *rbot, *rrad;            // rows of A
  const int64_t *ctop, *cbot, *crad, *cplus;    // columns of B
  BallsOut C;
  int64_t M, N, ldc, Mp, Np;
  int prec;
  // optional radius bound added to every entry ([M][N], index i N + j; null when absent): the
  // radius products of the complex product by eq. 2, summed beforehand
  const uint32_t *xrman;
  const int64_t *xrexp;
  // accumulate mode (crt_round_tc_kernel<.., .., true>): (-1)^negate T 2^sigma goes into this
  // window accumulator and the block's radius bound into its radius, instead of a rounding into C
  AccView acc;
  int negate;
};

__device__ __forceinline__ Mag with_extra_radius(const RoundArgs &a, int64_t i, int64_t j, Mag r) {
  if (!a.xrman) return r;
  const int64_t o = i * a.N + j;
  const Mag x{__ldg(a.xrman + o), __ldg(a.xrexp + o)};
  return x.man ? mag_add_up(r, x) : r;
}

__device__ __forceinline__ Mag product_mag(const IntProduct &p, int64_t i, int64_t j, int64_t Mp,
                                           int64_t Np, int64_t base) {
  if (p.ND == 0) return Mag{0u, 0};
  if (p.kind == 2) return mag_from_u64((uint64_t)__ldg((const int64_t *)p.digits + i * Np + j), base);
  uint64_t acc[4];
  assemble(p, i, j, Mp, Np, acc);  // nonnegative and < 2^64 (13+13+log2 K + 2 bits)
  return mag_from_u64(acc[0], base);
}

// Round the two's-complement integer T[0..nw) times 2^sigma to p bits (nearest, ties to even) and
// store it into entry oi of C with radius >= |rounded - T 2^sigma| + extra * 2^sigma + rad.
// T is clobbered.
__device__ void round_store(uint64_t *T, int nw, int64_t sigma, uint64_t extra, Mag rad, int prec,
                            const BallsOut &C, int64_t oi) {
  const bool neg = (T[nw - 1] >> 63) != 0;
  if (neg) {
    u128 c = 1;
    for (int k = 0; k < nw; ++k) {
      c += (u128)(~T[k]);
      T[k] = (uint64_t)c;
      c >>= 64;
    }
  }
  int top = -1;
  for (int k = nw - 1; k >= 0; --k)
    if (T[k]) {
      top = k;
      break;
    }
  const int nl = C.nlimbs;
  uint64_t E[RD_MAXW + 1];
  for (int k = 0; k <= nw; ++k) E[k] = 0;
  uint32_t fl = ARBGPU_FLAG_ZERO;
  int64_t oexp = 0;
  if (top >= 0) {
    int64_t L = 64LL * top + bitlen64(T[top]);
    const int64_t k = L > prec ? L - prec : 0;
    if (k > 0) {
      // round at bit k; E = |rounded - T|
      auto bit = [&](int64_t pos) -> bool {
        return pos >= 0 && pos < 64LL * nw && ((T[pos >> 6] >> (pos & 63)) & 1);
      };
      bool sticky = false;
      for (int64_t w = 0; w < ((k - 1) >> 6) && !sticky; ++w) sticky = T[w] != 0;
      if (!sticky && ((k - 1) & 63))
        sticky = (T[(k - 1) >> 6] & ((((uint64_t)1) << ((k - 1) & 63)) - 1)) != 0;
      const bool up = bit(k - 1) && (sticky || bit(k));
      uint64_t rem[RD_MAXW];
      for (int w = 0; w < nw; ++w) {
        const int64_t lo = 64LL * w;
        rem[w] = (lo + 64 <= k) ? T[w] : (lo < k ? (T[w] & ((((uint64_t)1) << (k - lo)) - 1)) : 0);
        T[w] ^= rem[w];
      }
      if (up) {
        E[k >> 6] = ((uint64_t)1) << (k & 63);
        uint64_t borrow = 0;
        for (int w = 0; w < nw; ++w) {
          u128 d = (u128)E[w] - rem[w] - borrow;
          E[w] = (uint64_t)d;
          borrow = (uint64_t)(d >> 64) & 1;
        }
        u128 cc = ((u128)1) << (k & 63);
        for (int w = (int)(k >> 6); w < nw; ++w) {
          cc += T[w];
          T[w] = (uint64_t)cc;
          cc >>= 64;
        }
        if (bit(L)) L += 1;
      } else {
        for (int w = 0; w < nw; ++w) E[w] = rem[w];
      }
    }
    // field = T * 2^(64 nl - L), top-aligned in nl limbs
    int nsig = 0;
    for (int q = 0; q < nl; ++q) {
      const int64_t lo = 64LL * q + (L - 64LL * nl);
      const int64_t li = lo >= 0 ? (lo >> 6) : -((-lo + 63) >> 6);
      const int bi = (int)(lo - li * 64);
      const uint64_t w0 = (li >= 0 && li < nw) ? T[li] : 0;
      const uint64_t w1 = (li + 1 >= 0 && li + 1 < nw) ? T[li + 1] : 0;
      const uint64_t f = bi ? ((w0 >> bi) | (w1 << (64 - bi))) : w0;
      C.limbs[(int64_t)q * C.stride + oi] = f;
      if (f && nsig == 0) nsig = nl - q;  // lowest nonzero limb fixes the limb count
    }
    oexp = sigma + L;
    fl = (neg ? ARBGPU_FLAG_SIGN : 0u) | ((uint32_t)nsig << ARBGPU_NSIG_SHIFT);
  } else {
    for (int q = 0; q < nl; ++q) C.limbs[(int64_t)q * C.stride + oi] = 0;
  }
  C.exp[oi] = oexp;
  C.flags[oi] = fl;
  // E += extra
  {
    u128 c = extra;
    for (int w = 0; w <= nw && c; ++w) {
      c += E[w];
      E[w] = (uint64_t)c;
      c >>= 64;
    }
  }
  const Mag r = mag_add_up(mag_from_limbs(E, nw + 1, sigma), rad);
  C.rad_man[oi] = r.man;
  C.rad_exp[oi] = r.man ? r.exp : 0;
}

// Radius bound of one block product at entry (i, j): P1 2^(top_i + crad_j - 2W) and
// P2 2^(rrad_i + cplus_j - 2W), each rounded up, summed rounded up.
__device__ __forceinline__ Mag block_radius(const IntProduct &rp1, const IntProduct &rp2,
                                            const int64_t *rtop, const int64_t *rrad,
                                            const int64_t *crad, const int64_t *cplus, int64_t i,
                                            int64_t j, int64_t Mp, int64_t Np) {
  Mag r{0u, 0};
  if (rp1.ND && rtop[i] != INT64_MIN && crad[j] != INT64_MIN)
    r = mag_add_up(r, product_mag(rp1, i, j, Mp, Np, rtop[i] + crad[j] - 2 * BL_W));
  if (rp2.ND && rrad[i] != INT64_MIN && cplus[j] != INT64_MIN)
    r = mag_add_up(r, product_mag(rp2, i, j, Mp, Np, rrad[i] + cplus[j] - 2 * BL_W));
  return r;
}

__global__ void block_round_kernel(const RoundArgs a) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.M * a.N) return;
  const int64_t i = idx / a.N, j = idx - (idx / a.N) * a.N;
  uint64_t T[RD_MAXW];
  const int nw = assemble(a.mid, i, j, a.Mp, a.Np, T);
  const bool rowz = a.rtop[i] == INT64_MIN, colz = a.ctop[j] == INT64_MIN;
  const int64_t sigma = (rowz ? 0 : a.rbot[i]) + (colz ? 0 : a.cbot[j]);  // T * 2^sigma
  const Mag rad = with_extra_radius(
      a, i, j, block_radius(a.rp1, a.rp2, a.rtop, a.rrad, a.crad, a.cplus, i, j, a.Mp, a.Np));
  round_store(T, nw, sigma, 0, rad, a.prec, a.C, i * a.ldc + j);
}

// ------------------------------------------------------------------------- register epilogue
//
// The same epilogue for products of at most NW limbs, with every limb array in registers (compile-
// time sizes, runtime positions) and, for the multimodular engine, the Chinese-remainder weights
// W_t and M in shared memory.

// T (two's complement over NW limbs) from its digits and group carries.
template <int NW>
__device__ __forceinline__ void digit_assemble_regs(const IntProduct &p, int64_t i, int64_t j,
                                                    int64_t Mp, int64_t Np, uint64_t (&T)[NW]) {
  const uint8_t *dp = p.digits + i * Np + j;
  const int64_t pl = Mp * Np;
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    uint64_t w = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if (8 * k + b < p.ND) w |= (uint64_t)__ldg(dp + (int64_t)(8 * k + b) * pl) << (8 * b);
    T[k] = w;
  }
  for (int g = 0; g < p.groups; ++g) {
    const int64_t c = __ldg(p.carries + ((int64_t)g * Mp + i) * Np + j);
    if (c == 0) continue;
    const int pos = 8 * p.ends.e[g];
    const int li = pos >> 6, bi = pos & 63;
    const uint64_t lo = (uint64_t)c << bi;
    const uint64_t hi = bi ? (uint64_t)(c >> (64 - bi)) : (uint64_t)(c < 0 ? -1 : 0);
    const uint64_t ext = c < 0 ? ~(uint64_t)0 : 0;
    u128 sum = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const uint64_t add = k < li ? 0 : (k == li ? lo : (k == li + 1 ? hi : ext));
      sum += (u128)T[k] + add;
      T[k] = (uint64_t)sum;
      sum >>= 64;
    }
  }
}

// T from its residues (the multimodular engine) as a two's-complement integer over NW limbs:
// T = sum_t z_t Q_t - q M.  sQ: Q32 rows of 2 NW limbs (zero padded), sM: M in 2 NW limbs, sr:
// 1 / m_t (shared memory).
template <int NW>
__device__ __forceinline__ void crt_assemble_regs(const IntProduct &p, int64_t i, int64_t j,
                                                  int64_t Mp, int64_t Np, const uint32_t *sQ,
                                                  const uint32_t *sM, const float *sr,
                                                  uint64_t (&T)[NW]) {
  constexpr int L32 = 2 * NW;
  const int64_t pl = Mp * Np, o = i * Np + j;
  uint64_t acc[L32];
#pragma unroll
  for (int l = 0; l < L32; ++l) acc[l] = 0;
  float qs = 0.f;
  const int NM = p.crt.NM;
  for (int t0 = 0; t0 < NM; t0 += 8) {
    // the residues of eight moduli are requested together
    uint32_t zb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) zb[u] = t0 + u < NM ? crt_z(p, t0 + u, pl, o) : 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (t0 + u >= NM) break;
      const int t = t0 + u;
      const uint32_t z = zb[u];
      qs = fmaf((float)z, sr[t], qs);
      const uint4 *w4 = (const uint4 *)(sQ + t * L32);
#pragma unroll
      for (int q4 = 0; q4 < L32 / 4; ++q4) {
        const uint4 w = w4[q4];
        acc[4 * q4 + 0] += (uint64_t)z * w.x;
        acc[4 * q4 + 1] += (uint64_t)z * w.y;
        acc[4 * q4 + 2] += (uint64_t)z * w.z;
        acc[4 * q4 + 3] += (uint64_t)z * w.w;
      }
    }
  }
  const int64_t q = (int64_t)rintf(qs);
  int64_t carry = 0;
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const int64_t v0 = (int64_t)acc[2 * k] - q * (int64_t)sM[2 * k] + carry;
    carry = v0 >> 32;
    const int64_t v1 = (int64_t)acc[2 * k + 1] - q * (int64_t)sM[2 * k + 1] + carry;
    carry = v1 >> 32;
    T[k] = (uint64_t)(uint32_t)v0 | ((uint64_t)(uint32_t)v1 << 32);
  }
}

// Round T (two's complement over NW limbs) times 2^sigma to p bits and store it into entry oi of
// C with radius >= |rounded - T 2^sigma| + extra 2^sigma + rad.
template <int NW>
__device__ __forceinline__ void round_store_regs(const uint64_t (&T)[NW], int64_t sigma,
                                                 uint64_t extra, Mag rad, int prec,
                                                 const BallsOut &C, int64_t oi) {
  const bool neg = (T[NW - 1] >> 63) != 0;
  uint64_t a[NW];
  {
    const uint64_t flip = neg ? ~(uint64_t)0 : 0;
    u128 cc = neg ? 1 : 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      cc += (u128)(T[k] ^ flip);
      a[k] = (uint64_t)cc;
      cc >>= 64;
    }
  }
  int L = limbs_bitlen<NW>(a);
  const bool zero = L == 0;
  uint64_t ta[NW + 1];
  Mag r1{0u, 0};
  if (!zero)
    round_abs_regs<NW>(a, L, prec, extra, sigma, ta, r1);
  else
    r1 = mag_from_u64(extra, sigma);
  store_rounded<NW + 1, 1>(C, oi, 0, zero, neg, ta, sigma + L, mag_add_up(r1, rad));
}

// round_store_regs for a long T and a short precision: only the top NWIN limbs of |T| (64 NWIN >=
// prec + 66 bits) take part in the rounding.  The bits below that window enter as a sticky bit
// OR-ed into the window's lowest bit, which keeps round-to-nearest exact (the round bit and the
// sticky condition are unchanged), and as one more unit of the window's last place in the error
// bound, which keeps the radius an upper bound of |rounded - T 2^sigma|.
template <int NW, int NWIN>
__device__ __forceinline__ void round_store_window(const uint64_t (&T)[NW], int64_t sigma, Mag rad,
                                                   int prec, const BallsOut &C, int64_t oi) {
  const bool neg = (T[NW - 1] >> 63) != 0;
  uint64_t a[NW];
  {
    const uint64_t flip = neg ? ~(uint64_t)0 : 0;
    u128 cc = neg ? 1 : 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      cc += (u128)(T[k] ^ flip);
      a[k] = (uint64_t)cc;
      cc >>= 64;
    }
  }
  const int L = limbs_bitlen<NW>(a);
  uint64_t ta[NWIN + 1];
  Mag r1{0u, 0};
  if (L == 0) {
#pragma unroll
    for (int k = 0; k <= NWIN; ++k) ta[k] = 0;
    store_rounded<NWIN + 1, 1>(C, oi, 0, true, neg, ta, sigma, rad);
    return;
  }
  uint64_t w[NWIN];
  int sh = L - 64 * NWIN;  // the window is a >> sh (sh <= 0: all of a)
  bool sticky = false;
  if (sh <= 0) {
    sh = 0;
#pragma unroll
    for (int k = 0; k < NWIN; ++k) w[k] = k < NW ? a[k] : 0;
  } else {
    const int q = sh >> 6, r = sh & 63;
    const uint64_t lowmask = (((uint64_t)1) << r) - 1;
#pragma unroll
    for (int k = 0; k < NW; ++k) sticky |= (k < q ? a[k] : (k == q ? (a[k] & lowmask) : 0)) != 0;
    // a >>= 64 q (a barrel shifter over limbs), then the bit shift r into the window
#pragma unroll
    for (int bb = 1; bb < NW; bb <<= 1) {
      const bool on = (q & bb) != 0;
#pragma unroll
      for (int j = 0; j < NW; ++j) a[j] = on ? (j + bb < NW ? a[j + bb] : 0) : a[j];
    }
#pragma unroll
    for (int k = 0; k < NWIN; ++k) {
      const uint64_t hi = k + 1 < NW ? a[k + 1] : 0;
      w[k] = r ? ((a[k] >> r) | (hi << (64 - r))) : a[k];
    }
    w[0] |= sticky ? 1u : 0u;
  }
  int LW = L - sh;
  round_abs_regs<NWIN>(w, LW, prec, sticky ? 1u : 0u, sigma + sh, ta, r1);
  store_rounded<NWIN + 1, 1>(C, oi, 0, false, neg, ta, sigma + sh + LW, mag_add_up(r1, rad));
}

// Radius bound of one block product from its two radius products (values < 2^64).
__device__ __forceinline__ Mag product_mag_regs(const IntProduct &p, int64_t i, int64_t j,
                                                int64_t Mp, int64_t Np, int64_t base) {
  if (p.ND == 0) return Mag{0u, 0};
  if (p.kind == 2) return mag_from_u64((uint64_t)__ldg((const int64_t *)p.digits + i * Np + j), base);
  uint64_t acc[2];
  digit_assemble_regs<2>(p, i, j, Mp, Np, acc);  // nonnegative and < 2^64
  return mag_from_u64(acc[0], base);
}

__device__ __forceinline__ Mag block_radius_regs(const IntProduct &rp1, const IntProduct &rp2,
                                                 const int64_t *rtop, const int64_t *rrad,
                                                 const int64_t *crad, const int64_t *cplus,
                                                 int64_t i, int64_t j, int64_t Mp, int64_t Np) {
  Mag r{0u, 0};
  if (rp1.ND && rtop[i] != INT64_MIN && crad[j] != INT64_MIN)
    r = mag_add_up(r, product_mag_regs(rp1, i, j, Mp, Np, rtop[i] + crad[j] - 2 * BL_W));
  if (rp2.ND && rrad[i] != INT64_MIN && cplus[j] != INT64_MIN)
    r = mag_add_up(r, product_mag_regs(rp2, i, j, Mp, Np, rrad[i] + cplus[j] - 2 * BL_W));
  return r;
}

// Shared-memory bytes of the register epilogue's tables for NW limbs.
static size_t crt_smem_bytes(const IntProduct &p, int NW) {
  if (p.kind != 1) return 0;
  return ((size_t)p.crt.NM + 1) * 2 * NW * 4 + (size_t)p.crt.NM * 4;
}

template <int NW>
__global__ void __launch_bounds__(128, 6) block_round_regs_kernel(const RoundArgs a) {
  constexpr int L32 = 2 * NW;
  extern __shared__ uint4 smem_u4[];
  uint32_t *sQ = (uint32_t *)smem_u4;
  uint32_t *sM = nullptr;
  float *sr = nullptr;
  if (a.mid.kind == 1) {
    const CrtTables &c = a.mid.crt;
    sM = sQ + c.NM * L32;
    sr = (float *)(sM + L32);
    for (int k = threadIdx.x; k < (c.NM + 1) * L32; k += blockDim.x) {
      const int t = k / L32, l = k - t * L32;
      const uint32_t *src = t < c.NM ? c.Q32 + (int64_t)t * c.NW32P : c.M32;
      sQ[k] = l < c.NW32P ? __ldg(src + l) : 0u;
    }
    for (int k = threadIdx.x; k < c.NM; k += blockDim.x) sr[k] = __ldg(c.rinv + k);
    __syncthreads();
  }
  pdl_wait();  // the block products come from the GEMM kernel before this one
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.M * a.N) return;
  const int64_t i = idx / a.N, j = idx - i * a.N;
  uint64_t T[NW];
  if (a.mid.kind == 1)
    crt_assemble_regs<NW>(a.mid, i, j, a.Mp, a.Np, sQ, sM, sr, T);
  else
    digit_assemble_regs<NW>(a.mid, i, j, a.Mp, a.Np, T);
  const bool rowz = a.rtop[i] == INT64_MIN, colz = a.ctop[j] == INT64_MIN;
  const int64_t sigma = (rowz ? 0 : a.rbot[i]) + (colz ? 0 : a.cbot[j]);  // T * 2^sigma
  const Mag rad = with_extra_radius(
      a, i, j, block_radius_regs(a.rp1, a.rp2, a.rtop, a.rrad, a.crad, a.cplus, i, j, a.Mp, a.Np));
  round_store_regs<NW>(T, sigma, 0, rad, a.prec, a.C, i * a.ldc + j);
}

// ------------------------------------------------------------------------- wide epilogue
//
// The epilogue for products too long for the register kernels (p >= 512: T of 20 to 48 limbs),
// one entry per thread on the CUDA cores.  The multimodular engine's Chinese-remainder sum
// T = sum_t z_t Q_t - q M is formed sixteen 32-bit words at a time in 64-bit register
// accumulators, every thread of the CTA reading the same row of Q from shared memory (a
// broadcast) for its own z_t; the limbs of T go to shared memory, limb-major ([k][thread], so a
// warp's accesses are conflict-free); the rounding then reads only the NWIN limbs at the top of
// |T| plus a sticky bit, as round_store_window does in registers.
constexpr int RW_ROWS = 128;  // entries (threads) per CTA

// Shared-memory bytes of the wide epilogue: the Q rows and M padded to L32P words, 1 / m_t, and
// the limbs of T.
__host__ __device__ inline int rw_l32p(int nw) { return (2 * nw + 15) / 16 * 16; }
static size_t rw_smem_bytes(const IntProduct &p, int nw) {
  size_t b = (size_t)nw * RW_ROWS * 8;
  if (p.kind == 1) b += ((size_t)p.crt.NM + 1) * rw_l32p(nw) * 4 + (size_t)p.crt.NM * 4;
  return b;
}

// Round T (two's complement, nw limbs at sT[k RS]) times 2^sigma to p bits and store it into
// entry oi of C with radius >= |rounded - T 2^sigma| + rad; prec + 66 <= 64 NWIN.  T is clobbered
// (replaced by |T|).
template <int NWIN, int RS = RW_ROWS>
__device__ __forceinline__ void round_store_smem(uint64_t *sT, int nw, int64_t sigma, Mag rad,
                                                 int prec, const BallsOut &C, int64_t oi) {
  const bool neg = (sT[(nw - 1) * RS] >> 63) != 0;
  int top = -1;
  {
    const uint64_t flip = neg ? ~(uint64_t)0 : 0;
    u128 cc = neg ? 1 : 0;
    for (int k = 0; k < nw; ++k) {
      cc += (u128)(sT[k * RS] ^ flip);
      const uint64_t v = (uint64_t)cc;
      cc >>= 64;
      sT[k * RS] = v;
      if (v) top = k;
    }
  }
  uint64_t ta[NWIN + 1];
  if (top < 0) {
#pragma unroll
    for (int k = 0; k <= NWIN; ++k) ta[k] = 0;
    store_rounded<NWIN + 1, 1>(C, oi, 0, true, neg, ta, sigma, rad);
    return;
  }
  const int L = 64 * top + bitlen64(sT[top * RS]);
  uint64_t w[NWIN];
  int sh = L - 64 * NWIN;  // the window is |T| >> sh (sh <= 0: all of |T|)
  bool sticky = false;
  if (sh <= 0) {
    sh = 0;
#pragma unroll
    for (int k = 0; k < NWIN; ++k) w[k] = k <= top ? sT[k * RS] : 0;
  } else {
    const int q = sh >> 6, r = sh & 63;  // q + NWIN - 1 <= top
    for (int k = 0; k < q; ++k) sticky |= sT[k * RS] != 0;
    sticky |= (sT[q * RS] & ((((uint64_t)1) << r) - 1)) != 0;
#pragma unroll
    for (int k = 0; k < NWIN; ++k) {
      const uint64_t lo = sT[(q + k) * RS];
      const uint64_t hi = q + k + 1 <= top ? sT[(q + k + 1) * RS] : 0;
      w[k] = r ? ((lo >> r) | (hi << (64 - r))) : lo;
    }
    w[0] |= sticky ? 1u : 0u;
  }
  int LW = L - sh;
  Mag r1{0u, 0};
  round_abs_regs<NWIN>(w, LW, prec, sticky ? 1u : 0u, sigma + sh, ta, r1);
  store_rounded<NWIN + 1, 1>(C, oi, 0, false, neg, ta, sigma + sh + LW, mag_add_up(r1, rad));
}

template <int NWIN>
__global__ void __launch_bounds__(RW_ROWS) block_round_wide_kernel(const RoundArgs a, int nw) {
  extern __shared__ uint4 smem_u4[];
  uint64_t *sT = (uint64_t *)smem_u4 + threadIdx.x;  // limb k at sT[k RW_ROWS]
  const int L32P = rw_l32p(nw);
  uint32_t *sQ = (uint32_t *)((uint64_t *)smem_u4 + (size_t)nw * RW_ROWS);
  const IntProduct &p = a.mid;
  if (p.kind == 1) {
    const CrtTables &c = p.crt;
    for (int k = threadIdx.x; k < (c.NM + 1) * L32P; k += blockDim.x) {
      const int t = k / L32P, l = k - t * L32P;
      const uint32_t *src = t < c.NM ? c.Q32 + (int64_t)t * c.NW32P : c.M32;
      sQ[k] = l < c.NW32P ? __ldg(src + l) : 0u;
    }
    float *sr = (float *)(sQ + (size_t)(c.NM + 1) * L32P);
    for (int k = threadIdx.x; k < c.NM; k += blockDim.x) sr[k] = __ldg(c.rinv + k);
    __syncthreads();
  }
  pdl_wait();  // the block products come from the GEMM kernel before this one
  const int64_t idx = (int64_t)blockIdx.x * RW_ROWS + threadIdx.x;
  if (idx >= a.M * a.N) return;
  const int64_t i = idx / a.N, j = idx - i * a.N;
  const int64_t pl = a.Mp * a.Np, o = i * a.Np + j;
  if (p.kind == 1) {
    // T = sum_t z_t Q_t - q M, q = rint(sum_t z_t / m_t)
    const CrtTables &c = p.crt;
    const int NM = c.NM;
    const uint32_t *sM = sQ + (size_t)NM * L32P;
    const float *sr = (const float *)(sM + L32P);
    const uint16_t *zp = (const uint16_t *)p.digits + o;
    float qs = 0.f;
    for (int t = 0; t < NM; ++t) qs = fmaf((float)__ldg(zp + (int64_t)t * pl), sr[t], qs);
    const int64_t q = (int64_t)rintf(qs);
    int64_t carry = 0;
    for (int l0 = 0; l0 < 2 * nw; l0 += 16) {
      uint64_t acc[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) acc[u] = 0;
      const uint4 *qrow = (const uint4 *)(sQ + l0);
      for (int t0 = 0; t0 < NM; t0 += 8) {
        // the residues of eight moduli are requested together
        uint32_t zb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) zb[u] = t0 + u < NM ? __ldg(zp + (int64_t)(t0 + u) * pl) : 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (t0 + u >= NM) break;
          const uint32_t z = zb[u];
          const uint4 *w4 = qrow + (size_t)(t0 + u) * (L32P / 4);
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const uint4 w = w4[q4];
            mad_wide(acc[4 * q4 + 0], z, w.x);
            mad_wide(acc[4 * q4 + 1], z, w.y);
            mad_wide(acc[4 * q4 + 2], z, w.z);
            mad_wide(acc[4 * q4 + 3], z, w.w);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 16; u += 2) {
        const int l = l0 + u;
        const int64_t v0 = (int64_t)acc[u] - q * (int64_t)sM[l] + carry;
        carry = v0 >> 32;
        const int64_t v1 = (int64_t)acc[u + 1] - q * (int64_t)sM[l + 1] + carry;
        carry = v1 >> 32;
        if ((l >> 1) < nw)
          sT[(l >> 1) * RW_ROWS] = (uint64_t)(uint32_t)v0 | ((uint64_t)(uint32_t)v1 << 32);
      }
    }
  } else {
    // T from its digits (eight per limb) and the carries of the digit groups
    const uint8_t *dp = p.digits + o;
    for (int k = 0; k < nw; ++k) {
      uint64_t w = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b)
        if (8 * k + b < p.ND) w |= (uint64_t)__ldg(dp + (int64_t)(8 * k + b) * pl) << (8 * b);
      sT[k * RW_ROWS] = w;
    }
    for (int g = 0; g < p.groups; ++g) {
      const int64_t cg = __ldg(p.carries + ((int64_t)g * a.Mp + i) * a.Np + j);
      if (cg == 0) continue;
      const int pos = 8 * p.ends.e[g];
      const int li = pos >> 6, bi = pos & 63;
      const uint64_t lo = (uint64_t)cg << bi;
      const uint64_t hi = bi ? (uint64_t)(cg >> (64 - bi)) : (uint64_t)(cg < 0 ? -1 : 0);
      const uint64_t ext = cg < 0 ? ~(uint64_t)0 : 0;
      u128 s = 0;
      for (int k = li; k < nw; ++k) {
        const uint64_t add = k == li ? lo : (k == li + 1 ? hi : ext);
        s += (u128)sT[k * RW_ROWS] + add;
        sT[k * RW_ROWS] = (uint64_t)s;
        s >>= 64;
      }
    }
  }
  const bool rowz = a.rtop[i] == INT64_MIN, colz = a.ctop[j] == INT64_MIN;
  const int64_t sigma = (rowz ? 0 : a.rbot[i]) + (colz ? 0 : a.cbot[j]);  // T * 2^sigma
  const Mag rad = with_extra_radius(
      a, i, j, block_radius_regs(a.rp1, a.rp2, a.rtop, a.rrad, a.crad, a.cplus, i, j, a.Mp, a.Np));
  round_store_smem<NWIN>(sT, nw, sigma, rad, a.prec, a.C, i * a.ldc + j);
}

// ------------------------------------------------------------------------- MMA epilogue
//
// The Chinese-remainder sum of the multimodular engine on the 8-bit warp-level MMA
// (mma.sync m16n8k32, signed bytes into s32), for products beyond the TMEM epilogue (more than
// 64 moduli or 16 limbs).  With z_t = l_t + 256 h_t (bytes l, h), l' = l - 128, h' = h - 128 and
// Q_t = sum_n q_{t,n} 256^n (balanced bytes),
//
//     sum_t z_t Q_t = sum_n 256^n S_n + 32896 sum_t Q_t,   S_n = sum_t (l'_t q_{t,n} + h'_t q_{t,n-1}),
//
// S the product of the signed byte matrix [entries][2 NM] and the table w8 [2 NM][NQ]; |S_n| <=
// 2 NM 128 128 < 2^31, so the s32 sums are exact.  A warp takes 32 entries (two row tiles of 16) and the
// columns 32 at a time; the sums pass through shared memory to the lane of their entry, which
// carries them into the 32-bit words of T = sum_n 256^n S_n - q M (q = rint(sum_t z_t / m_t), as
// in crt_assemble).  The limbs of T go to shared memory and round_store_smem rounds them.
constexpr int RM_MAX_KS = 12;  // k-steps of 32 bytes: NM <= 192

__device__ __forceinline__ void mma_s8s8(int32_t (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory bytes of the MMA epilogue with `warps` warps: the limbs of T, the column staging,
// M and the offset term in 32-bit words, 1 / m_t and the byte table (rows padded by 16 bytes).
static size_t rm_smem_bytes(const CrtTables &c, int nw, int warps) {
  const size_t rows = 32 * (size_t)warps;
  return (size_t)nw * rows * 8 + (size_t)warps * 32 * 33 * 4 + (size_t)(2 * nw + 3) / 4 * 32 +
         (size_t)(c.NM + 3) / 4 * 16 + (size_t)c.NQ8 * (c.K8 + 16);
}

template <int NWIN, int WARPS, int KSM>
__global__ void __launch_bounds__(32 * WARPS) crt_round_mma_kernel(const RoundArgs a, int nw) {
  constexpr int ROWS = 32 * WARPS;
  extern __shared__ uint4 smem_u4[];
  const CrtTables &c = a.mid.crt;
  const int NM = c.NM, KS = c.K8 / 32, WS = c.K8 + 16, L32 = 2 * nw;
  uint64_t *sT = (uint64_t *)smem_u4;                                  // [nw][ROWS]
  int32_t *sC = (int32_t *)(sT + (size_t)nw * ROWS);                     // [WARPS][32][33]
  uint32_t *sM = (uint32_t *)(sC + WARPS * 32 * 33);                     // [L32] words of M
  uint32_t *sO = sM + (L32 + 3) / 4 * 4;                                 // [L32] offset term
  float *sr = (float *)(sO + (L32 + 3) / 4 * 4);                         // [NM] 1 / m_t
  uint8_t *sW = (uint8_t *)(sr + (NM + 3) / 4 * 4);                      // [NQ8][WS] bytes
  for (int q = threadIdx.x; q < L32; q += blockDim.x) {
    sM[q] = q < c.NW32P ? __ldg(c.M32 + q) : 0u;
    sO[q] = __ldg(c.c32 + q);  // (2 NMW + 2 = L32 words)
  }
  for (int q = threadIdx.x; q < NM; q += blockDim.x) sr[q] = __ldg(c.rinv + q);
  {
    const int c16 = c.K8 / 16;
    for (int q = threadIdx.x; q < c.NQ8 * c16; q += blockDim.x) {
      const int n = q / c16, u = q - n * c16;
      *(uint4 *)(sW + (size_t)n * WS + 16 * u) = __ldg((const uint4 *)(c.w8 + (size_t)n * c.K8) + u);
    }
  }
  __syncthreads();
  pdl_wait();  // the residues z come from the GEMM kernel before this one
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  const int64_t MN = a.M * a.N, pl = a.Mp * a.Np, ntile = (MN + 31) / 32;
  const uint16_t *zbase = (const uint16_t *)a.mid.digits;
  auto z_off = [&](int64_t e) -> int64_t {  // offset of entry e in a residue plane, -1 past MN
    if (e >= MN) return -1;
    const int64_t i = e / a.N;
    return i * a.Np + (e - i * a.N);
  };
  int32_t *sCw = sC + warp * 32 * 33;
  uint32_t *sT32 = (uint32_t *)(sT + threadIdx.x);  // word w of T at sT32[(w >> 1) 2 ROWS + (w & 1)]
  const int nchunks = c.NQ8 / 32;
  // persistent: every warp takes tiles of 32 consecutive entries, a grid's warps apart
  for (int64_t tile = (int64_t)blockIdx.x * WARPS + warp; tile < ntile;
       tile += (int64_t)gridDim.x * WARPS) {
    const int64_t e0 = 32 * tile;
    // A fragments of the tile's two row tiles for every k-step: register r of row tile mt holds
    // the bytes of z_t, z_(t+1) (t = 16 ks + 8 (r >> 1) + 2 tig) of row 16 mt + g + 8 (r & 1)
    uint32_t af[KSM][2][4];
    {
      int64_t orow[2][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) orow[mt][h] = z_off(e0 + 16 * mt + 8 * h + g);
#pragma unroll
      for (int ks = 0; ks < KSM; ++ks)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            uint32_t v = 0;
            const int t = 16 * ks + 8 * (r >> 1) + 2 * tig;
            const int64_t o = orow[mt][r & 1];
            if (ks < KS && o >= 0) {
              if (t < NM) v = __ldg(zbase + (int64_t)t * pl + o);
              if (t + 1 < NM) v |= (uint32_t)__ldg(zbase + (int64_t)(t + 1) * pl + o) << 16;
            }
            af[ks][mt][r] = v;
          }
    }
    // q = rint(sum_t z_t / m_t) of the lane's entry (row `lane` of the tile): partial sums over
    // this lane's moduli for its four rows, summed over the four lanes of its group (the same
    // value in each), then fetched from the group that holds the row
    float qp[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int ks = 0; ks < KSM; ++ks)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int t = 16 * ks + 8 * (r >> 1) + 2 * tig;
          if (ks < KS && t < NM) {
            const uint32_t v = af[ks][mt][r];
            float s = qp[mt][r & 1];
            s = fmaf((float)(v & 0xFFFFu), sr[t], s);
            if (t + 1 < NM) s = fmaf((float)(v >> 16), sr[t + 1], s);
            qp[mt][r & 1] = s;
          }
        }
    float qs = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v = qp[mt][h];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v = __shfl_sync(0xffffffffu, v, 4 * (lane & 7));
        if ((lane >> 4) == mt && ((lane >> 3) & 1) == h) qs = v;
      }
    const int64_t q = (int64_t)rintf(qs);
    // the bytes as signed bytes offset by -128
#pragma unroll
    for (int ks = 0; ks < KSM; ++ks)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < 4; ++r) af[ks][mt][r] ^= 0x80808080u;
    int64_t carry = 0;
    for (int nc = 0; nc < nchunks; ++nc) {
      int32_t acc[2][4][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0;
#pragma unroll
      for (int ks = 0; ks < KSM; ++ks) {
        if (ks < KS) {
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const uint8_t *wrow = sW + (size_t)(32 * nc + 8 * nt + g) * WS + 32 * ks + 4 * tig;
            const uint32_t b0 = *(const uint32_t *)wrow, b1 = *(const uint32_t *)(wrow + 16);
            mma_s8s8(acc[0][nt], af[ks][0], b0, b1);
            mma_s8s8(acc[1][nt], af[ks][1], b0, b1);
          }
        }
      }
      // column sums of rows 16 mt + g (+ 8) to the staging rows, then each lane carries its row
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          int32_t *r0 = sCw + (16 * mt + g) * 33 + 8 * nt + 2 * tig;
          r0[0] = acc[mt][nt][0];
          r0[1] = acc[mt][nt][1];
          r0[8 * 33] = acc[mt][nt][2];
          r0[8 * 33 + 1] = acc[mt][nt][3];
        }
      __syncwarp();
      const int32_t *mine = sCw + lane * 33;
#pragma unroll
      for (int wq = 0; wq < 8; ++wq) {
        const int w = 8 * nc + wq;
        const int64_t v = (int64_t)mine[4 * wq] + (int64_t)mine[4 * wq + 1] * 256 +
                          (int64_t)mine[4 * wq + 2] * 65536 +
                          (int64_t)mine[4 * wq + 3] * 16777216 + carry +
                          (w < L32 ? (int64_t)sO[w] - q * (int64_t)sM[w] : 0);
        carry = v >> 32;
        if (w < L32) sT32[(size_t)(w >> 1) * 2 * ROWS + (w & 1)] = (uint32_t)v;
      }
      __syncwarp();
    }
    for (int w = 8 * nchunks; w < L32; ++w) {  // words past the table's columns: M's and the sign
      const int64_t v = carry + (int64_t)sO[w] - q * (int64_t)sM[w];
      carry = v >> 32;
      sT32[(size_t)(w >> 1) * 2 * ROWS + (w & 1)] = (uint32_t)v;
    }
    const int64_t e = e0 + lane;
    if (e < MN) {
      const int64_t i = e / a.N, j = e - i * a.N;
      const bool rowz = a.rtop[i] == INT64_MIN, colz = a.ctop[j] == INT64_MIN;
      const int64_t sigma = (rowz ? 0 : a.rbot[i]) + (colz ? 0 : a.cbot[j]);  // T * 2^sigma
      const Mag rad = with_extra_radius(a, i, j,
                                        block_radius_regs(a.rp1, a.rp2, a.rtop, a.rrad, a.crad,
                                                          a.cplus, i, j, a.Mp, a.Np));
      round_store_smem<NWIN, ROWS>(sT + threadIdx.x, nw, sigma, rad, a.prec, a.C,
                                   i * a.ldc + j);
    }
    __syncwarp();
  }
}

// Limbs of the assembled product of `p` (two's complement, including the sign).
static int product_limbs(const IntProduct &p) {
  return p.kind == 1 ? p.crt.NMW + 1 : (8 * p.ND + 32 + 63) / 64 + 1;
}

// ---- The reconstruction on the tensor cores.  For one entry, with z_t = l_t + 256 h_t (bytes),
//
//     sum_t z_t Q_t = sum_n 256^n S_n,   S_n = sum_t (l_t q_{t,n} + h_t q_{t,n-1}),
//
// with q_{t,n} the balanced bytes of Q_t = M / m_t: a product of the byte matrix
// [entries][(t, byte)] and the table [(t, byte)][n].  |S_n| < 2^22 (at most 128 products of
// magnitude <= 255 * 128), so the FP32 sums are exact.  One more column weighs the bytes with
// 1/m_t and 256/m_t rounded to BF16 (the second is exactly 256 times the first): its sum is
// sum_t z_t / m_t with error below sum_t m_t |bf16(1/m_t) - 1/m_t| < NM 2^-8 <= 1/4 (0.118 for
// the 64 largest primes below 2^16), and since sum_t z_t / m_t = q + T / M with |T / M| < 1/8,
// the total stays below 1/2 and its rint is the q of T = sum_t z_t Q_t - q M.  The drain forms T = sum_n 256^n (S_n - q M_n), M_n the balanced bytes
// of M, with carries between 32-bit words, then rounds it as block_round does.
//
// Roles (one CTA per SM, persistent over tiles of 128 consecutive entries of a row of C): one
// producer warpgroup loads the tile's residues z with TMA and writes the byte rows, one warp
// issues the MMAs, ND drain warpgroups take the tiles in turn.  Waits give up after ~2 s.
constexpr int CR_MAX_ND = 3;
constexpr int CR_NS = 3;  // byte tiles in flight
constexpr int CR_NZ = 3;  // residue tiles in flight
constexpr int CR_THREADS = 32 * (4 * CR_MAX_ND + 5);

struct CrShared {
  uint64_t z_full[CR_NZ];
  uint64_t a_full[CR_NS], a_empty[CR_NS];
  uint64_t t_full[CR_MAX_ND + 1], t_empty[CR_MAX_ND + 1];
  uint32_t tmem_base;
};

struct CrArgs {
  RoundArgs ra;
  int NM, NQ, NQP, ND, wg_cols;
  uint32_t tcols;
  const uint16_t *wtab;  // [NQP][128] BF16
  const float *mbytes;   // [NQ]
  int *status;
};

static size_t crt_tc_smem(int NM, int NQ, int NQP) {
  return 1024 + (size_t)2 * NQP * 128 + (size_t)CR_NS * 2 * RT_TILE + (size_t)CR_NZ * NM * 256 +
         (size_t)((NQ + 15) & ~15) * 4 + sizeof(CrShared);
}

template <int NW, int NWIN, bool ACC>
__global__ void __launch_bounds__(CR_THREADS, 1)
    crt_round_tc_kernel(const __grid_constant__ CUtensorMap tmz, const __grid_constant__ CrArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const RoundArgs &ra = a.ra;
  const int ND = a.ND, NB = a.ND + 1, NM = a.NM;
  uint8_t *sW = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);  // 2 slabs [NQP][64]
  uint8_t *sA = sW + (size_t)2 * a.NQP * 128;                                   // CR_NS x 2 slabs
  uint16_t *sZ = (uint16_t *)(sA + (size_t)CR_NS * 2 * RT_TILE);               // CR_NZ x [NM][128]
  float *sMb = (float *)(sZ + (size_t)CR_NZ * NM * 128);
  CrShared *sh = (CrShared *)(sMb + ((a.NQ + 15) & ~15));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mma_warp = 4 * ND + 4;

  if (threadIdx.x == 0) {
    for (int q = 0; q < CR_NZ; ++q) mbar_init(&sh->z_full[q], 1);
    for (int q = 0; q < CR_NS; ++q) {
      mbar_init(&sh->a_full[q], RT_ROWS);
      mbar_init(&sh->a_empty[q], 1);
    }
    for (int q = 0; q < NB; ++q) {
      mbar_init(&sh->t_full[q], 1);
      mbar_init(&sh->t_empty[q], RT_ROWS);
    }
    fence_mbar_init();
  }
  if (warp == mma_warp) {
    tmem_alloc(&sh->tmem_base, a.tcols);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) tma_prefetch_desc(&tmz);
  for (int q = threadIdx.x; q < a.NQP * 16; q += blockDim.x) {  // weights, 128-byte swizzle
    const int n = q >> 4, c = q & 15;
    const uint4 v = __ldg((const uint4 *)(a.wtab + (size_t)n * 128) + c);
    *(uint4 *)(sW + (size_t)(c >> 3) * a.NQP * 128 + (size_t)n * 128 + (((c & 7) ^ (n & 7)) << 4)) =
        v;
  }
  for (int q = threadIdx.x; q < ((a.NQ + 15) & ~15); q += blockDim.x)  // zero past NQ
    sMb[q] = q < a.NQ ? __ldg(a.mbytes + q) : 0.0f;
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // the residues z come from the GEMM kernel before this one

  const int ntj = (int)((ra.N + RT_ROWS - 1) / RT_ROWS);
  const int nT = (int)ra.M * ntj;  // the host keeps this below 2^30
  const int ntiles = nT > (int)blockIdx.x ? (nT - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp >= 4 * ND && warp < mma_warp) {
    // ------------------------------------------------ producer: byte rows of the residues
    const int pt = threadIdx.x - 128 * ND;
    auto zload = [&](int k) {  // residues of this CTA's k-th tile into stage k mod CR_NZ
      const int tile = (int)blockIdx.x + k * (int)gridDim.x;
      const int i = tile / ntj, jb = tile - i * ntj;
      const int st = k % CR_NZ;
      mbar_arrive_expect_tx(&sh->z_full[st], (uint32_t)NM * RT_ROWS * 2);
      tma_load_3d(sZ + (size_t)st * NM * RT_ROWS, &tmz, &sh->z_full[st], jb * RT_ROWS, i, 0);
    };
    if (pt == 0)
      for (int k = 0; k < CR_NZ && k < ntiles; ++k) zload(k);
    const int nch = (2 * NM + 7) / 8;  // 16-byte chunks of a byte row that hold residues
    for (int k = 0; k < ntiles; ++k) {
      const int zs = k % CR_NZ, s = k % CR_NS;
      const bool ok = mbar_wait_sleep(&sh->z_full[zs], (k / CR_NZ) & 1) &&
                      mbar_wait_sleep(&sh->a_empty[s], ((k / CR_NS) & 1) ^ 1);
      // (also: every thread has read the residues of tile k - 1, so its stage can be refilled)
      if (named_bar_or(1 + ND, RT_ROWS, !ok)) {
        if (pt == 0) set_status(a.status, ARBGPU_ERR_TIMEOUT);
        break;
      }
      if (pt == 0 && k >= 1 && k - 1 + CR_NZ < ntiles) zload(k - 1 + CR_NZ);
      const uint16_t *zr = sZ + (size_t)zs * NM * RT_ROWS + pt;
      uint8_t *row = sA + (size_t)s * 2 * RT_TILE + (size_t)pt * 128;
#pragma unroll 4
      for (int c = 0; c < 16; ++c) {  // chunk c: moduli 4c .. 4c + 3 (low byte, high byte)
        uint32_t wv[4] = {0u, 0u, 0u, 0u};
        if (c < nch) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = 4 * c + u;
            if (t < NM) {
              const uint32_t z = zr[t * RT_ROWS];
              const float lo = __uint_as_float(__byte_perm(z, 0x4B000000u, 0x7540u)) - 8388608.0f;
              const float hi = __uint_as_float(__byte_perm(z, 0x4B000000u, 0x7541u)) - 8388608.0f;
              wv[u] = bf16x2_bits(lo, hi);
            }
          }
        }
        *(uint4 *)(row + (size_t)(c >> 3) * RT_TILE + (((c & 7) ^ (pt & 7)) << 4)) =
            make_uint4(wv[0], wv[1], wv[2], wv[3]);
      }
      fence_async_smem();
      mbar_arrive(&sh->a_full[s]);
    }
  } else if (warp == mma_warp) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(RT_ROWS, a.NQP);
      const int nks = (2 * NM + 15) / 16;  // K steps of 16 that hold residue bytes
      for (int k = 0; k < ntiles; ++k) {
        const int s = k % CR_NS, b = k % NB;
        if (!mbar_wait_sleep(&sh->a_full[s], (k / CR_NS) & 1) ||
            !mbar_wait_sleep(&sh->t_empty[b], ((k / NB) & 1) ^ 1)) {
          set_status(a.status, ARBGPU_ERR_TIMEOUT);
          break;
        }
        tc_fence_after();
        const uint32_t tm = sh->tmem_base + (uint32_t)(b * a.wg_cols);
        for (int ks = 0; ks < nks; ++ks) {
          const int sl = ks >> 2, sub = ks & 3;
          const uint64_t ad = sw128_desc(smem_u32(sA + ((size_t)s * 2 + sl) * RT_TILE));
          const uint64_t bd = sw128_desc(smem_u32(sW + (size_t)sl * a.NQP * 128));
          umma_bf16(tm, ad + 2 * sub, bd + 2 * sub, idesc, ks > 0 ? 1u : 0u);
        }
        umma_commit(&sh->t_full[b]);
        umma_commit(&sh->a_empty[s]);
      }
    }
  } else {
    // ------------------------------------------------ drain warpgroup d: tiles k = d (mod ND)
    const int d = warp >> 2, t = threadIdx.x & 127, wq = warp & 3;
    for (int k = d; k < ntiles; k += ND) {
      const int tile = (int)blockIdx.x + k * (int)gridDim.x;
      const int64_t i = tile / ntj, j = (int64_t)(tile - (int)i * ntj) * RT_ROWS + t;
      const int b = k % NB;
      if (!__all_sync(0xffffffffu, mbar_wait_sleep(&sh->t_full[b], (k / NB) & 1))) {
        if (lane == 0) set_status(a.status, ARBGPU_ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      const uint32_t tm =
          sh->tmem_base + (uint32_t)(b * a.wg_cols) + ((uint32_t)(32 * wq) << 16);
      float qf;
      {
        uint32_t v[16];
        tmem_ld16(tm + (uint32_t)(a.NQ & ~15), v);
        tmem_wait_ld();
        float sq = 0.0f;
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c == (a.NQ & 15)) sq = __uint_as_float(v[c]);
        qf = __fadd_rn(__fadd_rn(sq, RT_MAGIC), -RT_MAGIC);  // q = rint(sum_t z_t / m_t)
      }
      // T = sum_n 256^n (S_n - q M_n), four columns per 32-bit word: each biased column
      // S_n - q M_n + 1.5 2^23 has the bit pattern 0x4B400000 + (S_n - q M_n)
      uint64_t T[NW];
      int64_t carry = 0;
#pragma unroll
      for (int g = 0; g < NW / 2; ++g) {  // columns 16g .. 16g + 15 = limbs 2g, 2g + 1
        if (16 * g < a.NQ) {
          uint32_t v[16];
          tmem_ld16(tm + (uint32_t)(16 * g), v);
          tmem_wait_ld();
          uint32_t wd[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const float4 mb = *(const float4 *)(sMb + 16 * g + 4 * w);  // zero past NQ
            const float mbv[4] = {mb.x, mb.y, mb.z, mb.w};
            int64_t acc = carry - (int64_t)0x4B400000 * 0x01010101LL;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int n = 16 * g + 4 * w + c;
              const float col = n < a.NQ ? __uint_as_float(v[4 * w + c]) : 0.0f;
              const uint32_t bits =
                  __float_as_uint(__fadd_rn(__fmaf_rn(-qf, mbv[c], col), RT_MAGIC));
              acc += (int64_t)bits << (8 * c);
            }
            wd[w] = (uint32_t)acc;
            carry = acc >> 32;
          }
          T[2 * g] = (uint64_t)wd[0] | ((uint64_t)wd[1] << 32);
          T[2 * g + 1] = (uint64_t)wd[2] | ((uint64_t)wd[3] << 32);
        } else {
          const uint64_t ext = carry < 0 ? ~(uint64_t)0 : 0;  // the sign of T
          T[2 * g] = ext;
          T[2 * g + 1] = ext;
        }
      }
      tc_fence_before();
      mbar_arrive(&sh->t_empty[b]);
      if (ACC && j < ra.N) {
        // accumulate mode: add (-1)^negate T 2^sigma into the entry's window, the radius bound
        // into its radius
        const int64_t idx = i * ra.N + j;
        int64_t vtop;
        if (ra.rtop[i] != INT64_MIN && ra.ctop[j] != INT64_MIN && acc_top(ra.acc, i, j, vtop))
          acc_add_T(ra.acc, idx, ra.M * ra.N, T, NW, ra.rbot[i] + ra.cbot[j], vtop,
                    ra.negate != 0);
        acc_add_radius(ra.acc, idx,
                       block_radius_regs(ra.rp1, ra.rp2, ra.rtop, ra.rrad, ra.crad, ra.cplus, i,
                                         j, ra.Mp, ra.Np));
      } else if (j < ra.N) {
        const bool rowz = ra.rtop[i] == INT64_MIN, colz = ra.ctop[j] == INT64_MIN;
        const int64_t sigma = (rowz ? 0 : ra.rbot[i]) + (colz ? 0 : ra.cbot[j]);
        const Mag rad = with_extra_radius(ra, i, j,
                                          block_radius_regs(ra.rp1, ra.rp2, ra.rtop, ra.rrad,
                                                            ra.crad, ra.cplus, i, j, ra.Mp, ra.Np));
        if (NWIN > 0)
          round_store_window<NW, (NWIN > 0 ? NWIN : 1)>(T, sigma, rad, ra.prec, ra.C,
                                                        i * ra.ldc + j);
        else
          round_store_regs<NW>(T, sigma, 0, rad, ra.prec, ra.C, i * ra.ldc + j);
      }
    }
  }
  pdl_trigger();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == mma_warp) tmem_dealloc(sh->tmem_base, a.tcols);
}

// The reconstruction and rounding on the tensor cores, when the product is multimodular with
// NM <= 64 and fits one of the register sizes; false otherwise (block_round then runs).
static bool launch_crt_round_tc(arbgpu_ctx *ctx, const RoundArgs &ra, cudaStream_t s,
                                arbgpu_status *st, bool acc = false) {
  const CrtTables &c = ra.mid.crt;
  if (ra.mid.kind != 1 || c.NM > 64 || !c.wtab || c.NQP > 256 || c.NQP < 16) return false;
  const int nw = product_limbs(ra.mid);
  int NW = 0;
  if (ra.prec < 64 * 8 && nw <= 8 && c.NQ <= 64) NW = 8;
  else if (ra.prec < 64 * 12 && nw <= 12 && c.NQ <= 96) NW = 12;
  else if (ra.prec < 64 * 16 && nw <= 16 && c.NQ <= 128) NW = 16;
  if (!NW) return false;
  const int64_t ntj = (ra.N + RT_ROWS - 1) / RT_ROWS, nT = ra.M * ntj;
  if (nT > ((int64_t)1 << 30)) return false;
  CrArgs a{};
  a.ra = ra;
  a.NM = c.NM;
  a.NQ = c.NQ;
  a.NQP = c.NQP;
  a.wg_cols = c.NQP <= 128 ? 128 : 256;
  a.ND = c.NQP <= 128 ? 3 : 1;
  a.tcols = 512;
  a.wtab = c.wtab;
  a.mbytes = c.mbytes;
  a.status = ctx->status;
  size_t smem = crt_tc_smem(c.NM, c.NQ, c.NQP);
  if (smem > RT_SMEM_MAX) return false;
  if (smem < RT_SMEM_MIN) smem = RT_SMEM_MIN;
  CUtensorMap tm;
  if (!make_z_load_map(&tm, ra.mid.digits, ra.Np, ra.Mp, c.NM, c.NM)) return false;
  int64_t grid = nT < ctx->sm_count ? nT : ctx->sm_count;
  const unsigned threads = 32u * (unsigned)(4 * a.ND + 5);
  const int dev = ctx->device & 255;
#define ARB_CRT(NW_, NWIN_, ACC_)                                                             \
  do {                                                                                        \
    static bool attr_done[256] = {};                                                          \
    if (!attr_done[dev]) {                                                                    \
      if (cudaFuncSetAttribute(crt_round_tc_kernel<NW_, NWIN_, ACC_>,                         \
                               cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                               (int)RT_SMEM_MAX) != cudaSuccess) {                            \
        *st = ARBGPU_ERR_CUDA;                                                                \
        return true;                                                                          \
      }                                                                                       \
      attr_done[dev] = true;                                                                  \
    }                                                                                         \
    launch_pdl(crt_round_tc_kernel<NW_, NWIN_, ACC_>, dim3((unsigned)grid), dim3(threads),    \
               smem, s,                                                                       \
               tm, a);                                                                        \
  } while (0)
  // a 6-limb rounding window when it holds prec + 66 bits and T is longer
  const bool win6 = ra.prec + 66 <= 64 * 6;
  if (acc) {
    if (NW == 8) ARB_CRT(8, 0, true);
    else if (NW == 12) ARB_CRT(12, 0, true);
    else ARB_CRT(16, 0, true);
  } else if (NW == 8) {
    if (win6) ARB_CRT(8, 6, false);
    else ARB_CRT(8, 0, false);
  } else if (NW == 12) {
    if (win6) ARB_CRT(12, 6, false);
    else ARB_CRT(12, 0, false);
  } else {
    if (win6) ARB_CRT(16, 6, false);
    else ARB_CRT(16, 0, false);
  }
#undef ARB_CRT
  *st = cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
  return true;
}

// The wide epilogue with the smallest rounding window that holds prec + 66 bits; false when the
// product or the precision is beyond it (ARBGPU_ROUND_WIDE=0 also declines).
static bool launch_block_round_wide(arbgpu_ctx *ctx, const RoundArgs &ra, int nw, unsigned blocks,
                                    cudaStream_t s) {
  const char *e = getenv("ARBGPU_ROUND_WIDE");
  if ((e && !strcmp(e, "0")) || ra.mid.kind > 1 || nw < 1 || nw > RD_MAXW) return false;
  const size_t smem = rw_smem_bytes(ra.mid, nw);
  if (smem > RT_SMEM_MAX) return false;
  const int dev = ctx->device & 255;
#define ARB_RW(NWIN_)                                                                         \
  do {                                                                                        \
    static bool attr_done[256] = {};                                                          \
    if (!attr_done[dev]) {                                                                    \
      if (cudaFuncSetAttribute(block_round_wide_kernel<NWIN_>,                                \
                               cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                               (int)RT_SMEM_MAX) != cudaSuccess)                              \
        return false;                                                                         \
      attr_done[dev] = true;                                                                  \
    }                                                                                         \
    launch_pdl(block_round_wide_kernel<NWIN_>, dim3(blocks), dim3(RW_ROWS), smem, s, ra, nw); \
  } while (0)
  if (ra.prec + 66 <= 64 * 6)
    ARB_RW(6);
  else if (ra.prec + 66 <= 64 * 10)
    ARB_RW(10);
  else if (ra.prec + 66 <= 64 * 18)
    ARB_RW(18);
  else
    return false;
#undef ARB_RW
  return true;
}

// The MMA epilogue (multimodular products): persistent CTAs of eight warps, one per SM, the
// fragment set sized for at most 6 or 12 k-steps; false when the product or its tables are beyond
// it (ARBGPU_ROUND_MMA=0 also declines).
static bool launch_crt_round_mma(arbgpu_ctx *ctx, const RoundArgs &ra, int nw, cudaStream_t s) {
  const char *e = getenv("ARBGPU_ROUND_MMA");
  if (e && !strcmp(e, "0")) return false;
  const CrtTables &c = ra.mid.crt;
  if (ra.mid.kind != 1 || !c.w8 || !c.c32 || c.K8 < 32 || c.K8 > 32 * RM_MAX_KS || c.NQ8 < 32 || nw < 1 ||
      nw > RD_MAXW)
    return false;
  constexpr int W = 8;
  const size_t smem = rm_smem_bytes(c, nw, W);
  if (smem > RT_SMEM_MAX) return false;
  const int64_t ntile = (ra.M * ra.N + 31) / 32;
  const bool small = c.K8 <= 32 * 6;
  int64_t grid = (ntile + W - 1) / W;
  if (grid > (int64_t)ctx->sm_count) grid = ctx->sm_count;
  if (grid < 1) return true;
  const int dev = ctx->device & 255;
#define ARB_RM(NWIN_, KSM_)                                                                   \
  do {                                                                                        \
    static bool attr_done[256] = {};                                                          \
    if (!attr_done[dev]) {                                                                    \
      if (cudaFuncSetAttribute(crt_round_mma_kernel<NWIN_, W, KSM_>,                          \
                               cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                               (int)RT_SMEM_MAX) != cudaSuccess)                              \
        return false;                                                                         \
      attr_done[dev] = true;                                                                  \
    }                                                                                         \
    launch_pdl(crt_round_mma_kernel<NWIN_, W, KSM_>, dim3((unsigned)grid), dim3(32 * W), smem, \
               s, ra, nw);                                                                    \
  } while (0)
#define ARB_RM_K(NWIN_)  \
  do {                   \
    if (small)           \
      ARB_RM(NWIN_, 6);  \
    else                 \
      ARB_RM(NWIN_, 12); \
  } while (0)
  if (ra.prec + 66 <= 64 * 6)
    ARB_RM_K(6);
  else if (ra.prec + 66 <= 64 * 10)
    ARB_RM_K(10);
  else if (ra.prec + 66 <= 64 * 18)
    ARB_RM_K(18);
  else
    return false;
#undef ARB_RM_K
#undef ARB_RM
  return true;
}

// The rounding epilogue of one block: the register kernel of the smallest size that holds the
// product, else the MMA kernel, else the wide kernel, else the general one.
static void launch_block_round(arbgpu_ctx *ctx, const RoundArgs &ra, cudaStream_t s) {
  arbgpu_status tc_st;
  if (launch_crt_round_tc(ctx, ra, s, &tc_st)) return;  // (launch errors surface at the caller)
  const int nw = product_limbs(ra.mid);
  const unsigned blocks = (unsigned)((ra.M * ra.N + 127) / 128);
  if (crt_smem_bytes(ra.mid, 8) <= 48 * 1024 && ra.prec < 64 * 8 && nw <= 8)
    launch_pdl(block_round_regs_kernel<8>, dim3(blocks), dim3(128), crt_smem_bytes(ra.mid, 8), s,
               ra);
  else if (crt_smem_bytes(ra.mid, 12) <= 48 * 1024 && ra.prec < 64 * 12 && nw <= 12)
    launch_pdl(block_round_regs_kernel<12>, dim3(blocks), dim3(128), crt_smem_bytes(ra.mid, 12),
               s, ra);
  else if (crt_smem_bytes(ra.mid, 16) <= 48 * 1024 && ra.prec < 64 * 16 && nw <= 16)
    launch_pdl(block_round_regs_kernel<16>, dim3(blocks), dim3(128), crt_smem_bytes(ra.mid, 16),
               s, ra);
  else if (!launch_crt_round_mma(ctx, ra, nw, s) &&
           !launch_block_round_wide(ctx, ra, nw, blocks, s))
    block_round_kernel<<<blocks, 128, 0, s>>>(ra);
}

// ------------------------------------------------------------------------- several blocks

// Per-entry top / bottom exponents (INT64_MIN / INT64_MAX for zeros) for the planner.  With
// `merge`, the larger top and the smaller bottom of this operand's and the values already in
// top / bot (the other part of a complex operand: both parts of an entry share one scaling).
__global__ void entry_tb_kernel(const BallsView X, int64_t rows, int64_t cols, int64_t ld,
                                int64_t *top, int64_t *bot, int merge) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t r = idx / cols, c = idx - (idx / cols) * cols;
  EntryScan e = scan_entry(X, r * ld + c);
  int64_t t = e.nz ? e.top : INT64_MIN, b = e.nz ? e.bot : INT64_MAX;
  if (merge) {
    t = max((long long)t, (long long)top[idx]);
    b = min((long long)b, (long long)bot[idx]);
  }
  top[idx] = t;
  bot[idx] = b;
}

// The same per-entry exponents of a K x N operand, written transposed ([N][K]: column j of the
// operand is row j of the output) through a 32 x 32 shared-memory tile, so that every line the
// planner walks -- a row of A or a column of B -- is contiguous.
__global__ void __launch_bounds__(256) entry_tb_t_kernel(const BallsView X, int64_t K, int64_t N,
                                                         int64_t ld, int64_t *topT,
                                                         int64_t *botT, int merge) {
  __shared__ int64_t st[32][33], sb[32][33];
  const int64_t tiles_n = (N + 31) / 32;
  const int64_t k0 = ((int64_t)blockIdx.x / tiles_n) * 32, j0 = ((int64_t)blockIdx.x % tiles_n) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int64_t k = k0 + r, j = j0 + tx;
    int64_t t = INT64_MIN, b = INT64_MAX;
    if (k < K && j < N) {
      const EntryScan e = scan_entry(X, k * ld + j);
      if (e.nz) {
        t = e.top;
        b = e.bot;
      }
    }
    st[r][tx] = t;
    sb[r][tx] = b;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t j = j0 + r, k = k0 + tx;
    if (j < N && k < K) {
      int64_t t = st[tx][r], b = sb[tx][r];
      if (merge) {
        t = max((long long)t, (long long)topT[j * K + k]);
        b = min((long long)b, (long long)botT[j * K + k]);
      }
      topT[j * K + k] = t;
      botT[j * K + k] = b;
    }
  }
}

// Bounded grid barrier of a cooperative launch (every CTA is resident): the last CTA to arrive
// resets the count and bumps the generation; the others wait for the bump, giving up after about
// two seconds (then *failed is set and the caller leaves).  bar[0] = count, bar[1] = generation.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *failed) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_ok = 1;
    volatile unsigned *gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*gen == g) {
        if (*(volatile int *)failed || global_ns() - t0 > 2000000000ull) {
          atomicExch(failed, 1);
          s_ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

// Greedy extraction of Algorithm 2 as one cooperative launch: from the current start, one warp
// per line (a row of A in tA/bA [M][K], a column of B in tBT/bBT [N][K]) scans 32 indices at a
// time with prefix max / min across the lanes and records the first index at which the line's
// height (max top - min bottom over its nonzero entries) would exceed h; the block ends there
// (the minimum over the lines; a block holds at least one index).  Blocks shorter than the basecase
// size are widened to min(30, remaining) and marked for dot products.  CTA 0 writes the
// [start, stop, basecase] triples and their count; state[0] = start, state[1] = end of the block
// being found, bar = the barrier words (zeroed by the host), failed = the give-up flag (zeroed).
__global__ void __launch_bounds__(256) plan_coop_kernel(const int64_t *tA, const int64_t *bA,
                                                        const int64_t *tBT, const int64_t *bBT,
                                                        int64_t M, int64_t K, int64_t N, int64_t h,
                                                        int32_t *blocks, int32_t *nblocks,
                                                        int maxb, int *state, unsigned *bar,
                                                        int *failed, int *status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t lines = M + N;
  volatile int *vstate = state;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    state[0] = 0;
    state[1] = (int)K;
    *nblocks = 0;
  }
  if (!grid_barrier(bar, failed)) goto fail;
  for (int iter = 0;; ++iter) {
    const int start = vstate[0];
    if (start >= K || iter > maxb) break;
    for (int64_t L = warp; L < lines; L += nwarps) {
      const int64_t *tp = L < M ? tA + L * K : tBT + (L - M) * K;
      const int64_t *bp = L < M ? bA + L * K : bBT + (L - M) * K;
      long long hi = INT64_MIN, lo = INT64_MAX;
      // the current end, read by lane 0 and broadcast so that the loop stays warp-uniform
      int lim = __shfl_sync(0xffffffffu, lane == 0 ? vstate[1] : 0, 0);
      for (int64_t k0 = start; k0 < K && k0 < lim; k0 += 32) {
        const int64_t k = k0 + lane;
        long long t = k < K ? tp[k] : INT64_MIN;
        long long b = k < K ? bp[k] : INT64_MAX;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {  // inclusive prefix max of tops, min of bottoms
          const long long ut = __shfl_up_sync(0xffffffffu, t, o);
          const long long ub = __shfl_up_sync(0xffffffffu, b, o);
          if (lane >= o) {
            t = max(t, ut);
            b = min(b, ub);
          }
        }
        t = max(t, hi);
        b = min(b, lo);
        const bool bad = t != INT64_MIN && t - b > h;
        const unsigned m = __ballot_sync(0xffffffffu, bad);
        if (m) {
          if (lane == 0) atomicMin(state + 1, (int)(k0 + __ffs(m) - 1));
          break;
        }
        hi = __shfl_sync(0xffffffffu, t, 31);
        lo = __shfl_sync(0xffffffffu, b, 31);
        lim = __shfl_sync(0xffffffffu, lane == 0 ? vstate[1] : 0, 0);
      }
    }
    if (!grid_barrier(bar, failed)) goto fail;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      int end = state[1];
      if (end <= start) end = start + 1;
      int base = 0;
      if (end - start < BL_BASECASE) {
        end = start + (int)min((int64_t)BL_BASECASE, K - start);
        base = 1;
      }
      const int b = *nblocks;
      if (b < maxb) {
        blocks[3 * b] = start;
        blocks[3 * b + 1] = end;
        blocks[3 * b + 2] = base;
      }
      *nblocks = b + 1;
      state[0] = end;
      state[1] = (int)K;
    }
    if (!grid_barrier(bar, failed)) goto fail;
  }
  return;
fail:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *nblocks = 0;
    set_status(status, ARBGPU_ERR_TIMEOUT);
  }
}

// CTAs of plan_coop_kernel that fit on the device at once (a cooperative launch needs them all
// resident), per device.
static int plan_coop_grid(int device, int64_t lines) {
  static std::mutex mu;
  static std::vector<int> per_device;
  int cap;
  {
    std::lock_guard<std::mutex> lock(mu);
    if ((int)per_device.size() <= device) per_device.resize(device + 1, 0);
    if (!per_device[device]) {
      int per_sm = 0, sms = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_coop_kernel, 256, 0) !=
              cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
      per_device[device] = per_sm * sms;
    }
    cap = per_device[device];
  }
  const int64_t want = (lines + 7) / 8;  // eight warps (lines) per CTA
  return (int)(want < cap ? want : cap);
}

// a[k] = max over rows r of m[r][k] (INT64_MIN when every row holds INT64_MIN there): the column
// maxima of a row-major rows x K matrix, 32 columns per CTA, 8 row groups reduced in shared memory.
__global__ void __launch_bounds__(256) colmax_kernel(const int64_t *m, int64_t rows, int64_t K,
                                                     int64_t *a) {
  __shared__ long long s[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t k = (int64_t)blockIdx.x * 32 + tx;
  long long v = INT64_MIN;
  if (k < K)
    for (int64_t r = ty; r < rows; r += 8) v = max(v, (long long)m[r * K + k]);
  s[ty][tx] = v;
  __syncthreads();
  if (ty == 0 && k < K) {
    for (int q = 1; q < 8; ++q) v = max(v, s[q][tx]);
    a[k] = v;
  }
}

struct AccArgs {
  IntProduct mid, rp1, rp2;
  const int64_t *rtop, *rbot, *rrad, *ctop, *cbot, *crad, *cplus;  // this block's lines
  AccView v;
  int64_t M, N, Mp, Np;
  int negate;    // subtract the product (the -B D part of a complex real part)
  int skip_mid;  // add only the radius bound (the complex product by eq. 2)
  int skip_rad;  // add only the product (the complex product by eq. 2)
};

constexpr int ACC_MAX = 24;

// The exponent bound that places the accumulator window (the per-entry counterpart of
// Algorithm 1's e_max): etop[i][j] = max(etop[i][j], max_k top(x_ik) + top(y_kj)) over the nonzero
// entries, so |sum_k x_ik y_kj| < K 2^etop.  A max-plus matrix product, computed in int32 relative
// to each row's top rt_i and each column's top ct_j: d = top - rt_i (or - ct_j) <= 0, clamped
// below at -2^30 (a clamp only raises the bound, which stays an upper bound; a zero entry takes the
// clamp value).  rel_tops_kernel writes the relative tops once per operand; maxplus_top_kernel
// computes 128 x 128 outputs per CTA of 256 threads (8 x 8 each), the inner index in chunks of 32
// through shared memory, the next chunk's loads in flight while the current one is consumed.
constexpr int MP_T = 128, MP_K = 32, MP_PAD = 4;
constexpr int32_t MP_FLOOR = -(1 << 30);

// The same product on 16-bit halves (maxplus16_top_kernel), two outputs per instruction, when
// every nonzero entry of both operands lies within 2^13 - 1 of its line's top: live relative tops
// are then in [-8191, 0], zeros take -16384, so a sum with a zero (<= -16384) stays below every
// sum of two live entries (>= -16382) and no sum leaves int16.  The live maxima, hence the bound
// of every entry with a nonzero product, are those of the int32 kernel.
constexpr int32_t MP16_LIVE = 8191, MP16_ZERO = -16384;

// rel[r * cols + c] = top(X[r * ld + c]) - ref, ref = rt[r] (by_row) or rt[c], clamped; zeros and
// empty lines give the floor.  *wide is set when a nonzero entry lies below -MP16_LIVE.
__global__ void rel_tops_kernel(const BallsView X, int64_t ld, int64_t rows, int64_t cols,
                                const int64_t *rt, bool by_row, int32_t *rel, int *wide) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t r = idx / cols, c = idx - (idx / cols) * cols;
  const int64_t e = r * ld + c;
  const int64_t ref = by_row ? rt[r] : rt[c];
  const uint32_t fl = __ldg(X.flags + e);
  int32_t v = MP_FLOOR;
  if (!(fl & ARBGPU_FLAG_ZERO) && ref != INT64_MIN) {
    const int64_t d = __ldg(X.exp + e) - ref;
    v = d < MP_FLOOR ? MP_FLOOR : (int32_t)d;
    if (d < -MP16_LIVE) atomicOr(wide, 1);
  }
  rel[idx] = v;
}

// One operand value as the 16-bit half of maxplus16_top_kernel.
__device__ __forceinline__ uint32_t mp16_half(int32_t v) {
  return (uint32_t)(uint16_t)(int16_t)(v == MP_FLOOR ? MP16_ZERO : v);
}

// maxplus_top_kernel on 16-bit halves: the same tiles, A staged as (a, a) and B as (b_j, b_j+1)
// pairs, each __viaddmax_s16x2 giving max(a + b, acc) for two columns.  Returns at once when
// either operand's `wide` flag is set (the int32 kernel then runs).
__global__ void __launch_bounds__(256) maxplus16_top_kernel(
    const int32_t *dX, const int32_t *dY, const int *wideX, const int *wideY, const int64_t *rt,
    const int64_t *ct, int64_t M, int64_t K, int64_t N, int64_t *etop, int first) {
  if (*wideX | *wideY) return;
  __shared__ __align__(16) uint32_t sa[MP_K][MP_T + MP_PAD];
  __shared__ __align__(16) uint32_t sb[MP_K][MP_T / 2 + MP_PAD];
  const int64_t i0 = (int64_t)blockIdx.y * MP_T, j0 = (int64_t)blockIdx.x * MP_T;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  uint32_t acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0x80008000u;  // -32768 in both halves
  // this thread's 16 loads of each tile: A rows r = t / 32 (kk = t % 32); B column c = t % 128
  // (the same for every u), rows kb = t / 128
  int32_t ra[16], rb[16];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int t = threadIdx.x + 256 * u;
      const int kk = t % MP_K, r = t / MP_K;
      const int64_t i = i0 + r, k = k0 + kk;
      ra[u] = (i < M && k < K) ? __ldg(dX + i * K + k) : MP_FLOOR;
      const int c = t % MP_T, kb = t / MP_T;
      const int64_t j = j0 + c, k2 = k0 + kb;
      rb[u] = (j < N && k2 < K) ? __ldg(dY + k2 * N + j) : MP_FLOOR;
    }
  };
  load(0);
  const int c = threadIdx.x % MP_T;  // this thread's B column in the tile (even: it packs a pair)
  for (int64_t k0 = 0; k0 < K; k0 += MP_K) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int t = threadIdx.x + 256 * u;
      const uint32_t ha = mp16_half(ra[u]);
      sa[t % MP_K][t / MP_K] = ha | (ha << 16);
      const uint32_t hb = mp16_half(rb[u]);
      const uint32_t hn = __shfl_xor_sync(0xffffffffu, hb, 1);  // column c ^ 1
      if (!(c & 1)) sb[t / MP_T][c >> 1] = hb | (hn << 16);
    }
    __syncthreads();
    if (k0 + MP_K < K) load(k0 + MP_K);
#pragma unroll 4
    for (int kk = 0; kk < MP_K; ++kk) {
      const uint4 a0 = *(const uint4 *)&sa[kk][8 * ty], a1 = *(const uint4 *)&sa[kk][8 * ty + 4];
      const uint4 b0 = *(const uint4 *)&sb[kk][4 * tx];
      const uint32_t av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const uint32_t bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = __viaddmax_s16x2(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t i = i0 + 8 * ty + a;
    if (i >= M) continue;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int64_t j = j0 + 8 * tx + b;
      if (j >= N) continue;
      const int32_t v = (int32_t)(int16_t)(uint16_t)(acc[a][b >> 1] >> (16 * (b & 1)));
      const bool live = rt[i] != INT64_MIN && ct[j] != INT64_MIN;
      const int64_t e = live ? rt[i] + ct[j] + (int64_t)v : INT64_MIN;
      int64_t *o = etop + i * N + j;
      if (first || e > *o) *o = e;
    }
  }
}

// (wideX / wideY null: always runs; otherwise only when one of the flags is set)
__global__ void __launch_bounds__(256) maxplus_top_kernel(const int32_t *dX, const int32_t *dY,
                                                          const int *wideX, const int *wideY,
                                                          const int64_t *rt, const int64_t *ct,
                                                          int64_t M, int64_t K, int64_t N,
                                                          int64_t *etop, int first) {
  if (wideX && !(*wideX | *wideY)) return;
  __shared__ __align__(16) int32_t sa[MP_K][MP_T + MP_PAD];
  __shared__ __align__(16) int32_t sb[MP_K][MP_T + MP_PAD];
  const int64_t i0 = (int64_t)blockIdx.y * MP_T, j0 = (int64_t)blockIdx.x * MP_T;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int32_t acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = INT32_MIN;
  // this thread's 16 loads of each tile: A rows r = t / 32 (kk = t % 32), B rows kb = t / 128
  int32_t ra[16], rb[16];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int t = threadIdx.x + 256 * u;
      const int kk = t % MP_K, r = t / MP_K;
      const int64_t i = i0 + r, k = k0 + kk;
      ra[u] = (i < M && k < K) ? __ldg(dX + i * K + k) : MP_FLOOR;
      const int c = t % MP_T, kb = t / MP_T;
      const int64_t j = j0 + c, k2 = k0 + kb;
      rb[u] = (j < N && k2 < K) ? __ldg(dY + k2 * N + j) : MP_FLOOR;
    }
  };
  load(0);
  for (int64_t k0 = 0; k0 < K; k0 += MP_K) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int t = threadIdx.x + 256 * u;
      sa[t % MP_K][t / MP_K] = ra[u];
      sb[t / MP_T][t % MP_T] = rb[u];
    }
    __syncthreads();
    if (k0 + MP_K < K) load(k0 + MP_K);
#pragma unroll 4
    for (int kk = 0; kk < MP_K; ++kk) {
      const int4 a0 = *(const int4 *)&sa[kk][8 * ty], a1 = *(const int4 *)&sa[kk][8 * ty + 4];
      const int4 b0 = *(const int4 *)&sb[kk][8 * tx], b1 = *(const int4 *)&sb[kk][8 * tx + 4];
      const int32_t av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const int32_t bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = max(acc[a][b], av[a] + bv[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t i = i0 + 8 * ty + a;
    if (i >= M) continue;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int64_t j = j0 + 8 * tx + b;
      if (j >= N) continue;
      const bool live = rt[i] != INT64_MIN && ct[j] != INT64_MIN;
      const int64_t e = live ? rt[i] + ct[j] + (int64_t)acc[a][b] : INT64_MIN;
      int64_t *o = etop + i * N + j;
      if (first || e > *o) *o = e;
    }
  }
}

// The max-plus bound of X Y into E (first: overwrite, else raise): the 16-bit kernel, and the
// int32 kernel for operands whose `wide` flag rel_tops_kernel set (each returns at once where the
// other applies).  ARBGPU_MAXPLUS16=0 keeps the int32 kernel alone.
static void launch_maxplus(arbgpu_ctx *ctx, cudaStream_t s, const int32_t *dX, const int32_t *dY,
                           const int *wideX, const int *wideY, const int64_t *rt,
                           const int64_t *ct, int64_t M, int64_t K, int64_t N, int64_t *E,
                           int first) {
  const char *env16 = getenv("ARBGPU_MAXPLUS16");
  const bool use16 = !(env16 && !strcmp(env16, "0"));
  LaunchScope sc(ctx, s, "maxplus_top", M * K * N);
  const dim3 grid((unsigned)((N + MP_T - 1) / MP_T), (unsigned)((M + MP_T - 1) / MP_T));
  if (!use16) {
    maxplus_top_kernel<<<grid, 256, 0, s>>>(dX, dY, nullptr, nullptr, rt, ct, M, K, N, E, first);
    return;
  }
  maxplus16_top_kernel<<<grid, 256, 0, s>>>(dX, dY, wideX, wideY, rt, ct, M, K, N, E, first);
  maxplus_top_kernel<<<grid, 256, 0, s>>>(dX, dY, wideX, wideY, rt, ct, M, K, N, E, first);
}

// The window bound of an output part from its products' bounds: out = max(a, b) entry by entry
// (b null: a copy); INT64_MIN marks an entry without a nonzero product.
__global__ void etop_max_kernel(const int64_t *a, const int64_t *b, int64_t *out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long v = a[i];
  out[i] = b ? max(v, (long long)b[i]) : v;
}

// acc += T_s 2^sigma_s (bits below the window truncated toward zero, one ulp each time),
// rad += this block's radius bound.
__global__ void accumulate_kernel(const AccArgs a) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.M * a.N) return;
  const int64_t i = idx / a.N, j = idx - (idx / a.N) * a.N;
  const int64_t MN = a.M * a.N;
  const AccView &v = a.v;
  int64_t vtop;
  if (!a.skip_mid && a.rtop[i] != INT64_MIN && a.ctop[j] != INT64_MIN &&
      acc_top(v, i, j, vtop)) {
    uint64_t T[RD_MAXW];
    const int nw = assemble(a.mid, i, j, a.Mp, a.Np, T);
    acc_add_T(v, idx, MN, T, nw, a.rbot[i] + a.cbot[j], vtop, a.negate != 0);
  }
  if (a.skip_rad) return;
  acc_add_radius(v, idx,
                 block_radius(a.rp1, a.rp2, a.rtop, a.rrad, a.crad, a.cplus, i, j, a.Mp, a.Np));
}

// Final rounding of the accumulator (no basecase blocks).
__global__ void acc_round_kernel(const AccView v, BallsOut C, int64_t M, int64_t N, int64_t ldc,
                                 int prec) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int64_t i = idx / N, j = idx - (idx / N) * N;
  uint64_t T[RD_MAXW];
  const int64_t MN = M * N;
  for (int q = 0; q < v.nacc; ++q) T[q] = v.acc[(int64_t)q * MN + idx];
  T[v.nacc] = (T[v.nacc - 1] >> 63) ? ~(uint64_t)0 : 0;  // one limb of sign extension
  int64_t vtop;
  const bool live = acc_top(v, i, j, vtop);
  const int64_t base = live ? acc_base_of(v, vtop) : 0;
  round_store(T, v.nacc + 1, base, live ? v.err[idx] : 0, Mag{v.rman[idx], v.rexp[idx]}, prec, C,
              i * ldc + j);
}

// Accumulator -> an exact ball (nacc + 1 limbs, radius = lost ulps + block radii): the `initial`
// term of the dot products that finish the basecase blocks.
__global__ void acc_to_ball_kernel(const AccView v, BallsOut I, int64_t M, int64_t N) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int64_t i = idx / N, j = idx - (idx / N) * N;
  const int64_t MN = M * N;
  const int nw = v.nacc;
  uint64_t T[ACC_MAX];
  for (int q = 0; q < nw; ++q) T[q] = v.acc[(int64_t)q * MN + idx];
  const bool neg = (T[nw - 1] >> 63) != 0;
  if (neg) {
    u128 c = 1;
    for (int k = 0; k < nw; ++k) {
      c += (u128)(~T[k]);
      T[k] = (uint64_t)c;
      c >>= 64;
    }
  }
  int top = -1;
  for (int k = nw - 1; k >= 0; --k)
    if (T[k]) {
      top = k;
      break;
    }
  int64_t vtop;
  const bool live = acc_top(v, i, j, vtop);
  const int64_t base = live ? acc_base_of(v, vtop) : 0;
  const int nl = I.nlimbs;  // nacc + 1
  if (top < 0) {
    for (int q = 0; q < nl; ++q) I.limbs[(int64_t)q * I.stride + idx] = 0;
    I.exp[idx] = 0;
    I.flags[idx] = ARBGPU_FLAG_ZERO;
  } else {
    const int64_t L = 64LL * top + bitlen64(T[top]);
    int nsig = 0;
    for (int q = 0; q < nl; ++q) {
      const int64_t lo = 64LL * q + (L - 64LL * nl);
      const int64_t li = lo >= 0 ? (lo >> 6) : -((-lo + 63) >> 6);
      const int bi = (int)(lo - li * 64);
      const uint64_t w0 = (li >= 0 && li < nw) ? T[li] : 0;
      const uint64_t w1 = (li + 1 >= 0 && li + 1 < nw) ? T[li + 1] : 0;
      const uint64_t f = bi ? ((w0 >> bi) | (w1 << (64 - bi))) : w0;
      I.limbs[(int64_t)q * I.stride + idx] = f;
      if (f && nsig == 0) nsig = nl - q;
    }
    I.exp[idx] = base + L;
    I.flags[idx] = (neg ? ARBGPU_FLAG_SIGN : 0u) | ((uint32_t)nsig << ARBGPU_NSIG_SHIFT);
  }
  Mag r{v.rman[idx], v.rexp[idx]};
  if (live && v.err[idx]) r = mag_add_up(r, mag_from_u64(v.err[idx], base));
  I.rad_man[idx] = r.man;
  I.rad_exp[idx] = r.man ? r.exp : 0;
}

// ------------------------------------------------------------------------- complex product by eq. 2

// The shared scaling of a complex operand's two parts: eq. 2 forms X_re + X_im, so both parts of a
// row of A (a column of B) take one exponent.  Line tops are the larger, bottoms the smaller of
// the parts' (an empty line has top INT64_MIN and bottom INT64_MAX); st receives the largest row
// height (hA) and column height (hB), INT64_MIN when every line is empty.  One CTA per block of a
// plan: CTA b merges the lines of block b (rows at b M, columns at b N) into st[b].
__global__ void __launch_bounds__(1024) merge_parts_kernel(
    const int64_t *rtop0, const int64_t *rbot0, const int64_t *rtop1, const int64_t *rbot1,
    int64_t M, int64_t *rtop, int64_t *rbot, const int64_t *ctop0, const int64_t *cbot0,
    const int64_t *ctop1, const int64_t *cbot1, int64_t N, int64_t *ctop, int64_t *cbot,
    BlockStats *st) {
  const int64_t oM = (int64_t)blockIdx.x * M, oN = (int64_t)blockIdx.x * N;
  rtop0 += oM, rbot0 += oM, rtop1 += oM, rbot1 += oM, rtop += oM, rbot += oM;
  ctop0 += oN, cbot0 += oN, ctop1 += oN, cbot1 += oN, ctop += oN, cbot += oN;
  st += blockIdx.x;
  __shared__ long long s_h[2];
  if (threadIdx.x < 2) s_h[threadIdx.x] = INT64_MIN;
  __syncthreads();
  long long hA = INT64_MIN, hB = INT64_MIN;
  for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
    const long long t = max((long long)rtop0[i], (long long)rtop1[i]);
    const long long b = min((long long)rbot0[i], (long long)rbot1[i]);
    rtop[i] = t;
    rbot[i] = b;
    if (t != INT64_MIN) hA = max(hA, t - b);
  }
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
    const long long t = max((long long)ctop0[j], (long long)ctop1[j]);
    const long long b = min((long long)cbot0[j], (long long)cbot1[j]);
    ctop[j] = t;
    cbot[j] = b;
    if (t != INT64_MIN) hB = max(hB, t - b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    hA = max(hA, __shfl_xor_sync(0xffffffffu, hA, o));
    hB = max(hB, __shfl_xor_sync(0xffffffffu, hB, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&s_h[0], hA);
    atomicMax(&s_h[1], hB);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    BlockStats m{};
    m.hA = s_h[0];
    m.hB = s_h[1];
    *st = m;
  }
}

// Residues of X_re + X_im from those of the parts (the residue of a sum is the sum of the
// residues): r = r_re + r_im, brought back to the balanced range |r| <= (m_t - 1) / 2 and split
// again into the balanced bytes r = 256 h + l, l in [-128, 127], that the residue kernels write
// (planes [2t] = l and [2t + 1] = h of [2 NM][plane]).  Vectors [0, nvA) are those of A (planes
// of planeA entries), the rest those of B; eight entries per vector (planes are multiples of 8).
__global__ void residue_sum_kernel(const __nv_bfloat16 *reA, const __nv_bfloat16 *imA,
                                   __nv_bfloat16 *sumA, int64_t planeA,
                                   const __nv_bfloat16 *reB, const __nv_bfloat16 *imB,
                                   __nv_bfloat16 *sumB, int64_t planeB, int NM) {
  const int64_t nvA = (int64_t)NM * (planeA / 8), nvB = (int64_t)NM * (planeB / 8);
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvA + nvB) return;
  const bool is_b = v >= nvA;
  if (is_b) v -= nvA;
  const int64_t plane = is_b ? planeB : planeA, pv = plane / 8;
  const __nv_bfloat16 *re = is_b ? reB : reA, *im = is_b ? imB : imA;
  __nv_bfloat16 *sum = is_b ? sumB : sumA;
  const int t = (int)(v / pv);
  const int64_t lo = (int64_t)2 * t * plane + (v - (int64_t)t * pv) * 8, hi = lo + plane;
  const int m = (int)c_mods[t], half = (m - 1) / 2;
  uint4 q[4] = {*(const uint4 *)(re + lo), *(const uint4 *)(re + hi), *(const uint4 *)(im + lo),
                *(const uint4 *)(im + hi)};
  const __nv_bfloat16 *e = (const __nv_bfloat16 *)q;
  uint4 out[2];
  __nv_bfloat16 *o = (__nv_bfloat16 *)out;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    int r = (int)__bfloat162float(e[u]) + 256 * (int)__bfloat162float(e[8 + u]) +
            (int)__bfloat162float(e[16 + u]) + 256 * (int)__bfloat162float(e[24 + u]);
    if (r > half)
      r -= m;
    else if (r < -half)
      r += m;
    const int l = ((r + 128) & 255) - 128;
    o[u] = __int2bfloat16_rn(l);
    o[8 + u] = __int2bfloat16_rn((r - l) / 256);
  }
  *(uint4 *)(sum + lo) = out[0];
  *(uint4 *)(sum + hi) = out[1];
}

// Eq. 2 on the residue products, modulus by modulus (values in [0, m_t)): z_re = z_1 - z_2 and
// z_im = z_3 - z_1 - z_2 mod m_t, with z_1, z_2, z_3 those of X_re Y_re, X_im Y_im and
// (X_re + X_im)(Y_re + Y_im) in planes [0, NM), [NM, 2 NM), [2 NM, 3 NM) of `z`.  In place: z_re
// over z_1, z_im over z_2.  Eight entries per thread (plane is a multiple of 8).
__global__ void z3m_kernel(uint16_t *z, int NM, int64_t plane) {
  const int64_t pv = plane / 8;
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (int64_t)NM * pv) return;
  const int t = (int)(v / pv);
  const int64_t o1 = (int64_t)t * plane + (v - (int64_t)t * pv) * 8;
  const int64_t o2 = o1 + (int64_t)NM * plane, o3 = o2 + (int64_t)NM * plane;
  const int m = (int)c_mods[t];
  uint4 q[3] = {*(const uint4 *)(z + o1), *(const uint4 *)(z + o2), *(const uint4 *)(z + o3)};
  const uint16_t *e = (const uint16_t *)q;
  uint4 out[2];
  uint16_t *w = (uint16_t *)out;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int a = e[u], b = e[8 + u], c = e[16 + u];
    int re = a - b, im = c - a - b;
    if (re < 0) re += m;
    if (im < 0) im += m;
    if (im < 0) im += m;
    w[u] = (uint16_t)re;
    w[8 + u] = (uint16_t)im;
  }
  *(uint4 *)(z + o1) = out[0];
  *(uint4 *)(z + o2) = out[1];
}

// ------------------------------------------------------------------------- inner ordering
//
// Section IV-B suggests an inner scaling G_s G_s^-1 of the columns of A_s against the rows of B_s,
// combined with permutations.  Reading (the paper leaves the strategy open): a_k and b_k are the
// largest tops of column k of A and row k of B; g_k = floor((b_k - a_k) / 2) multiplies column k
// of A by 2^g_k and row k of B by 2^-g_k, which leaves A B unchanged and brings both tops to within
// one of (a_k + b_k) / 2; the indices are ordered by a_k + b_k (ties by index), and those whose
// column of A or row of B has only zero midpoints come last with g_k = 0 (their radii may still
// count).  The greedy extraction of Section IV-A then runs over that order, on copies of the
// operands permuted and scaled so (`gather_inner_kernel`); the basecase dots read the original
// operands at the original indices.  On by default for products that need several blocks;
// ARBGPU_INNER_ORDER=0 turns it off.

static bool inner_order_enabled() {
  const char *e = getenv("ARBGPU_INNER_ORDER");
  return !(e && !strcmp(e, "0"));
}

// Bytes of a ball array of `count` entries with `nl` limb planes (256-byte aligned parts).
static size_t ball_array_bytes(int64_t count, int nl) {
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t c = (size_t)(count > 0 ? count : 1);
  return al(8 * c * nl) + al(8 * c) + al(4 * c) + al(4 * c) + al(8 * c);
}

static BallsOut ball_array_at(uint8_t *base, int64_t count, int nl) {
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t c = (size_t)(count > 0 ? count : 1);
  BallsOut b{};
  b.limbs = (uint64_t *)base;
  b.stride = (int64_t)c;
  b.nlimbs = nl;
  size_t o = al(8 * c * nl);
  b.exp = (int64_t *)(base + o);
  o += al(8 * c);
  b.flags = (uint32_t *)(base + o);
  o += al(4 * c);
  b.rad_man = (uint32_t *)(base + o);
  o += al(4 * c);
  b.rad_exp = (int64_t *)(base + o);
  return b;
}

// Reordered, scaled copy of an operand (gather_inner_entry, inner_order.cuh), one thread per
// entry of the copy.
__global__ void gather_inner_kernel(const BallsView X, int64_t ld, bool is_b, int64_t rows,
                                    int64_t K, int64_t cols, const int32_t *ord, const int64_t *g,
                                    BallsOut Y, int *out_of_range) {
  const int64_t n = is_b ? K * cols : rows * K;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  if (gather_inner_entry(X, ld, is_b, K, cols, ord, g, Y, idx)) atomicOr(out_of_range, 1);
}

// ------------------------------------------------------------------------- workspace and driver

struct BlockWs {
  // whole-range scans of the operand parts: rows of A_re / A_im, columns of B_re / B_im
  size_t scan;  // the whole-range scans' region (block_scan_bytes)
  // operands and products of one block
  size_t dA, dB, rA1, rB1, mdig, mcar, r1dig, r1car, r2dig, r2car;
  // several blocks: planner input, plan, per-block line statistics
  size_t tA, bA, tB, bB, blocks, nblocks, bstats;
  size_t brtop, brbot, brrad, bctop, bcbot, bcrad, bcplus;
  // per output part: accumulator, initial balls, basecase index list
  size_t acc[2], err[2], rman[2], rexp[2], ilimbs[2], iexp[2], iflags[2], irman[2], irexp[2], bk[2];
  size_t etop[2];  // per-entry exponent bound of the accumulated products (maxplus_top_kernel)
  size_t relA[2], relB[2];  // tops of A's and B's parts relative to their lines (int32)
  size_t relwide;           // their `wide` flags (A0, A1, B0, B1): see maxplus16_top_kernel
  // negligible-limb omission: one product's E, its truncated lines and their statistics
  size_t eprod /* [products][M N] */, om_rbot, om_rrad, om_rtrunc, om_cbot, om_crad, om_cplus, om_ctrunc, om_stats;
  // multimodular engine: residue planes, residue products, tables
  size_t resA, resB, cdig, ccar, craw;
  // complex product by eq. 2: residue planes of the parts and their sum, three residue products;
  // over several blocks, the imaginary parts' per-block lines (the real parts' take the
  // b* arrays), the lines shared by both parts, the per-block statistics of the imaginary parts
  // and of the shared lines, and (inner order) the reordered imaginary parts
  size_t r3A, r3B, z3;
  size_t e2rtop, e2rbot, e2rrad, e2ctop, e2cbot, e2crad, e2cplus;
  size_t e2srtop, e2srbot, e2sctop, e2scbot, e2stats, e2mstats, oA2, oB2;
  // inner ordering (Section IV-B): per-index tops, the order and scaling, the reordered operands,
  // the range flag of the scaled exponents
  size_t ia, ib, iord, ig, oA, oB, irange;
  size_t total;
  int Smax, NDmax, Gmax, Gr, maxb, nacc, NMmax, NMWmax;
  int64_t Kp, Mp, Np;
};

static BlockWs block_ws(arbgpu_ctx *ctx, int64_t M, int64_t K, int64_t N, int prec, bool cplx,
                        bool m3, int nlA, int nlB) {
  BlockWs w{};
  const int64_t hmax = (5LL * prec) / 4 + 192;
  w.Smax = (int)((hmax + 2 + 7) / 8);
  w.NDmax = 2 * w.Smax - 1;
  w.Kp = (K + TG_BK - 1) / TG_BK * TG_BK;
  w.Mp = (M + TG_BM - 1) / TG_BM * TG_BM;
  w.Np = (N + TG_BN - 1) / TG_BN * TG_BN;
  w.Gmax = digit_gemm_groups(ctx, (int)M, (int)N, w.NDmax);
  w.Gr = digit_gemm_groups(ctx, (int)M, (int)N, 2 * BL_SR - 1);
  w.maxb = (int)(K / BL_BASECASE) + 2;  // every block but the last holds >= 30 indices
  w.nacc = (prec + 63) / 64 + 3;
  {
    int bk = 0;
    for (int64_t v = K; v > 0; v >>= 1) ++bk;
    w.NMmax = crt_moduli_for_bits((int)(2 * (hmax + 1) + bk + 2));
    w.NMWmax = (16 * w.NMmax + 63) / 64 + 1;
  }
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += al(bytes);
    return o;
  };
  const size_t MN = (size_t)M * N;
  const int parts = cplx ? 2 : 1;
  w.scan = take(block_scan_bytes(M, N, cplx));
  w.dA = take((size_t)w.Smax * M * w.Kp * 2);
  w.dB = take((size_t)w.Smax * N * w.Kp * 2);
  // the two radius products' operands and results are adjacent, so both run as one batch
  w.rA1 = take((size_t)2 * BL_SR * M * w.Kp * 2);  // both radius operands of A
  w.rB1 = take((size_t)2 * BL_SR * N * w.Kp * 2);
  w.mdig = take((size_t)w.NDmax * w.Mp * w.Np);
  w.mcar = take((size_t)w.Gmax * w.Mp * w.Np * 4);
  w.r1dig = take((size_t)2 * (2 * BL_SR - 1) * w.Mp * w.Np);
  w.r2dig = w.r1dig + (size_t)(2 * BL_SR - 1) * w.Mp * w.Np;
  w.r1car = take((size_t)2 * w.Gr * w.Mp * w.Np * 4);
  w.r2car = w.r1car + (size_t)w.Gr * w.Mp * w.Np * 4;
  w.tA = take(8 * (size_t)M * K);
  w.bA = take(8 * (size_t)M * K);
  w.tB = take(8 * (size_t)K * N);
  w.bB = take(8 * (size_t)K * N);
  w.blocks = take(12 * (size_t)w.maxb);
  w.nblocks = take(64);  // block count, planner state (2 ints), barrier words (2), give-up flag
  w.bstats = take(sizeof(BlockStats) * (size_t)w.maxb);
  w.brtop = take(8 * (size_t)w.maxb * M);
  w.brbot = take(8 * (size_t)w.maxb * M);
  w.brrad = take(8 * (size_t)w.maxb * M);
  w.bctop = take(8 * (size_t)w.maxb * N);
  w.bcbot = take(8 * (size_t)w.maxb * N);
  w.bcrad = take(8 * (size_t)w.maxb * N);
  w.bcplus = take(8 * (size_t)w.maxb * N);
  for (int q = 0; q < parts; ++q) {
    w.acc[q] = take(8 * (size_t)w.nacc * MN);
    w.err[q] = take(4 * MN);
    w.rman[q] = take(4 * MN);
    w.rexp[q] = take(8 * MN);
    w.ilimbs[q] = take(8 * (size_t)(w.nacc + 1) * MN);
    w.iexp[q] = take(8 * MN);
    w.iflags[q] = take(4 * MN);
    w.irman[q] = take(4 * MN);
    w.irexp[q] = take(8 * MN);
    w.bk[q] = take(4 * 2 * (size_t)K);
    w.etop[q] = take(8 * MN);
    w.relA[q] = take(4 * (size_t)M * K);
    w.relB[q] = take(4 * (size_t)K * N);
  }
  w.relwide = take(4 * sizeof(int));
  w.eprod = take(8 * MN * (size_t)(cplx ? 4 : 1));  // E of each real product
  w.om_rbot = take(8 * (size_t)M);
  w.om_rrad = take(8 * (size_t)M);
  w.om_rtrunc = take(8 * (size_t)M);
  w.om_cbot = take(8 * (size_t)N);
  w.om_crad = take(8 * (size_t)N);
  w.om_cplus = take(8 * (size_t)N);
  w.om_ctrunc = take(8 * (size_t)N);
  w.om_stats = take(sizeof(BlockStats));
  // residue planes, then the two radius products' operand planes (batch items NM and NM + 1)
  w.resA = take((size_t)2 * (w.NMmax + 2) * M * w.Kp * 2);
  w.resB = take((size_t)2 * (w.NMmax + 2) * N * w.Kp * 2);
  w.cdig = take((size_t)3 * w.NMmax * w.Mp * w.Np);
  w.craw = take((size_t)2 * 8 * w.Mp * w.Np);  // the two radius products as int64
  w.ccar = take(256);  // the multimodular GEMM writes no carries
  if (inner_order_enabled()) {
    w.ia = take(8 * (size_t)K);
    w.ib = take(8 * (size_t)K);
    w.iord = take(4 * (size_t)K);
    w.ig = take(8 * (size_t)K);
    // the reordered copies keep the operands' limb counts
    w.oA = take(ball_array_bytes(M * K, nlA < 1 || nlA > BL_MAX_NL ? BL_MAX_NL : nlA));
    w.oB = take(ball_array_bytes(K * N, nlB < 1 || nlB > BL_MAX_NL ? BL_MAX_NL : nlB));
    w.irange = take(4);
  }
  if (cplx && m3) {
    w.r3A = take((size_t)3 * 2 * w.NMmax * M * w.Kp * 2);
    w.r3B = take((size_t)3 * 2 * w.NMmax * N * w.Kp * 2);
    w.z3 = take((size_t)3 * w.NMmax * w.Mp * w.Np * 2);
    const size_t bm = 8 * (size_t)w.maxb * M, bn = 8 * (size_t)w.maxb * N;
    w.e2rtop = take(bm);
    w.e2rbot = take(bm);
    w.e2rrad = take(bm);
    w.e2ctop = take(bn);
    w.e2cbot = take(bn);
    w.e2crad = take(bn);
    w.e2cplus = take(bn);
    w.e2srtop = take(bm);
    w.e2srbot = take(bm);
    w.e2sctop = take(bn);
    w.e2scbot = take(bn);
    w.e2stats = take(sizeof(BlockStats) * (size_t)w.maxb);
    w.e2mstats = take(sizeof(BlockStats) * (size_t)w.maxb);
    if (w.oA) {
      w.oA2 = take(ball_array_bytes(M * K, nlA < 1 || nlA > BL_MAX_NL ? BL_MAX_NL : nlA));
      w.oB2 = take(ball_array_bytes(K * N, nlB < 1 || nlB > BL_MAX_NL ? BL_MAX_NL : nlB));
    }
  }
  w.total = off;
  return w;
}

// Every multimodular table a product at precision <= max_prec with an inner dimension <=
// max_inner can use, on the device now (so that later calls allocate nothing).
arbgpu_status block_reserve(arbgpu_ctx *ctx, int max_prec, int64_t max_inner) {
  if (ensure_crt_constants(ctx->device) != ARBGPU_OK) return ARBGPU_ERR_CUDA;
  const int64_t hmax = (5LL * max_prec) / 4 + 192;
  int bk = 0;
  for (int64_t v = max_inner; v > 0; v >>= 1) ++bk;
  int top = crt_moduli_for_bits((int)(2 * (hmax + 1) + bk + 2));
  if (top > CRT_MAX_MODULI) top = CRT_MAX_MODULI;
  for (int nm = 1; nm <= top; ++nm) {
    const CrtPlan *plan = crt_plan(nm);
    if (!plan) continue;
    CrtDevTables dt{};
    if (crt_device_tables(ctx, plan, &dt) != ARBGPU_OK) return ARBGPU_ERR_CUDA;
  }
  return ARBGPU_OK;
}

size_t block_workspace_size(arbgpu_ctx *ctx, int64_t M, int64_t K, int64_t N, int prec,
                            bool cplx, bool m3, int nlA, int nlB) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  return block_ws(ctx, M, K, N, prec, cplx, m3, nlA, nlB).total;
}

// Line statistics of one block (pointers into the whole-range or the per-block arrays).
struct Lines {
  const int64_t *rtop, *rbot, *rrad, *ctop, *cbot, *crad, *cplus;
  // negligible-limb omission (omit_product): the per-line exponents below which bits were dropped
  const int64_t *rtrunc = nullptr, *ctrunc = nullptr;
};

static int digits_for_height(int64_t h) { return h < 0 ? 1 : (int)((h + 2 + 7) / 8); }

static int bit_length(int64_t v) {
  int b = 0;
  while (v > 0) {
    ++b;
    v >>= 1;
  }
  return b;
}

// The integer engine for a block: digits (S_A x S_B digit products) or multimodular (NM residue
// products of 2 x 2 digits each, then the Chinese remainder theorem).  ARBGPU_ENGINE=digits|crt
// forces one; otherwise the cheaper by a cost model whose constants are the measured costs of the
// kernels on GB300: a tensor-core digit multiply-add, a 32-bit multiply-add of the CRT epilogue
// (per output entry), a 16-bit multiply-add of the residue kernel (per input entry), and a digit
// byte of the digit epilogue (per output entry).
static bool choose_crt(int SA, int SB, int NM, int64_t M, int64_t N, int64_t Kp, int64_t hA,
                       int64_t hB, int engine = -1) {
  const char *e = getenv("ARBGPU_ENGINE");
  if (e && !strcmp(e, "digits")) return false;
  if (e && !strcmp(e, "crt")) return true;
  if (engine >= 0) return engine == 1;  // the autotuner's choice
  // seconds per unit, measured on a GB300 (N = 512, p = 256; and N = 388, p = 1024 for the
  // reconstruction above 64 moduli, on the 8-bit warp MMA: 0.344 ms for 1.58e9 units)
  const double t_mma = 2.6e-15, t_crt = NM <= 64 ? 2.1e-13 : 2.2e-13, t_res = 2.4e-13,
               t_dig = 4e-12;
  const double MN = (double)M * (double)N;
  const double nw32 = 2.0 * ((16.0 * NM + 63) / 64 + 1);
  const double nch = (double)((hA > hB ? hA : hB) + 2) / 32 + 1;
  const double digits = t_mma * SA * SB * (double)Kp * MN + t_dig * (SA + SB) * MN;
  const double crt = t_mma * 4.0 * NM * (double)Kp * MN + t_crt * NM * nw32 * MN +
                     t_res * NM * nch * (double)Kp * (double)(M + N);
  return crt < digits;
}

// The radius products of a block on the digit engine, from the operands the split wrote at rA1 /
// rB1 (the second operands follow at this block's Kp): P1 = U(|A|) V(R_B) when B has radii,
// P2 = U(R_A) V(|B| + R_B) when A has radii, one launch when both are needed.
static arbgpu_status radius_gemm(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws, int64_t M,
                                 int64_t N, int64_t Kp, bool radA, bool radB, cudaStream_t s,
                                 IntProduct *rp1, IntProduct *rp2) {
  const int NDr = 2 * BL_SR - 1;
  *rp1 = IntProduct{};
  *rp2 = IntProduct{};
  if (!radA && !radB) return ARBGPU_OK;
  __nv_bfloat16 *rA1 = (__nv_bfloat16 *)(ws + w.rA1), *rA2 = rA1 + (size_t)BL_SR * M * Kp;
  __nv_bfloat16 *rB1 = (__nv_bfloat16 *)(ws + w.rB1), *rB2 = rB1 + (size_t)BL_SR * N * Kp;
  const bool both = radA && radB;
  DigitGemmArgs g{radB ? rA1 : rA2, radB ? rB1 : rB2, (int)M, (int)N, Kp, BL_SR, BL_SR, w.Gr,
                  ws + (radB ? w.r1dig : w.r2dig),
                  (int32_t *)(ws + (radB ? w.r1car : w.r2car)), "digit_gemm_rad",
                  both ? 2 : 1};
  arbgpu_status stg = launch_digit_gemm(ctx, g, s);
  if (stg != ARBGPU_OK) return stg;
  if (radB) {
    *rp1 = IntProduct{ws + w.r1dig, (int32_t *)(ws + w.r1car), NDr, w.Gr, {}, 0, {}};
    digit_gemm_group_ends(BL_SR, BL_SR, w.Gr, rp1->ends.e);
  }
  if (radA) {
    *rp2 = IntProduct{ws + w.r2dig, (int32_t *)(ws + w.r2car), NDr, w.Gr, {}, 0, {}};
    digit_gemm_group_ends(BL_SR, BL_SR, w.Gr, rp2->ends.e);
  }
  return ARBGPU_OK;
}

// Split the block [k0, k0 + Kb) and run its products: T = (E A)(B F), and the radius products
// P1 = U(|A|) V(R_B) (when B has radii), P2 = U(R_A) V(|B| + R_B) (when A has radii).  hA, hB: the
// largest row / column heights in the block.
// Which engines can take a block product of heights hA, hB over Kb inner indices.
static void block_engines(const BlockWs &w, int64_t Kb, int64_t hA, int64_t hB, bool *crt_ok,
                          bool *digits_ok) {
  const int64_t Kp = (Kb + TG_BK - 1) / TG_BK * TG_BK;
  const int SA = digits_for_height(hA), SB = digits_for_height(hB);
  const int NM = crt_moduli_for_bits((int)((hA > 0 ? hA : 0) + (hB > 0 ? hB : 0) +
                                           bit_length(Kb) + 2));
  const int nch32 = (int)(((hA > hB ? hA : hB) + 2 + 31) / 32) + 1;
  const size_t res_smem = (size_t)NM * ((nch32 + 3) / 4 * 4) * 4;
  const CrtPlan *plan = NM <= w.NMmax && res_smem <= 48 * 1024 ? crt_plan(NM) : nullptr;
  *crt_ok = plan && plan->NMW + 1 <= RD_MAXW;
  *digits_ok = SA <= w.Smax && SB <= w.Smax && digit_gemm_fits(SA, SB, Kp);
}

// engine: -1 lets the cost model choose, 0 asks for the digit engine, 1 for the multimodular one
// (when it can take the product).
static arbgpu_status run_block_engine(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws,
                                      const BallsView &Av, const BallsView &Bv, int64_t M,
                                      int64_t N, int64_t lda, int64_t ldb, int64_t k0, int64_t Kb,
                                      int64_t hA, int64_t hB, bool radA, bool radB,
                                      const Lines &ln, cudaStream_t s, IntProduct *mid,
                                      IntProduct *rp1, IntProduct *rp2, int engine) {
  const int64_t Kp = (Kb + TG_BK - 1) / TG_BK * TG_BK;
  const int SA = digits_for_height(hA), SB = digits_for_height(hB);
  const int NM = crt_moduli_for_bits((int)((hA > 0 ? hA : 0) + (hB > 0 ? hB : 0) +
                                           bit_length(Kb) + 2));
  const CrtPlan *plan = nullptr;
  const int nch32 = (int)(((hA > hB ? hA : hB) + 2 + 31) / 32) + 1;
  const size_t res_smem = (size_t)NM * ((nch32 + 3) / 4 * 4) * 4;  // residue kernel's table
  const bool omitted = ln.rtrunc || ln.ctrunc;  // only the tensor-core residue kernel adds the
                                                 // omission's radius
  if ((omitted || choose_crt(SA, SB, NM, M, N, Kp, hA, hB, engine)) && NM <= w.NMmax &&
      res_smem <= 48 * 1024) {
    plan = crt_plan(NM);
    if (plan && plan->NMW + 1 > RD_MAXW) plan = nullptr;
  }
  if (omitted && !plan) return ARBGPU_ERR_LIMIT;
  if (!plan && (SA > w.Smax || SB > w.Smax || !digit_gemm_fits(SA, SB, Kp)))
    return ARBGPU_ERR_LIMIT;
  __nv_bfloat16 *dA = (__nv_bfloat16 *)(ws + w.dA), *dB = (__nv_bfloat16 *)(ws + w.dB);
  // the second radius product's planes follow the first's at this block's Kp (one batched GEMM)
  __nv_bfloat16 *rA1 = (__nv_bfloat16 *)(ws + w.rA1), *rA2 = rA1 + (size_t)BL_SR * M * Kp;
  __nv_bfloat16 *rB1 = (__nv_bfloat16 *)(ws + w.rB1), *rB2 = rB1 + (size_t)BL_SR * N * Kp;
  // radius operands (and the digit planes when the digit engine runs)
  // the digit engine's planes and radius operands (the multimodular residue kernels write the
  // radius operands themselves)
  if (!plan) {
    const int64_t n = M * Kp;
    SplitOut o{dA, radB ? rA1 : nullptr, radA ? rA2 : nullptr};
    LaunchScope sc(ctx, s, "split_a", n);
    split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Av, false, M, k0, Kb, Kp, lda,
                                                             plan ? 0 : SA, ln.rbot, ln.rtop,
                                                             ln.rrad, nullptr, o, ln.rtrunc);
  }
  if (!plan) {
    const int64_t n = N * Kp;
    SplitOut o{dB, radB ? rB1 : nullptr, radA ? rB2 : nullptr};
    LaunchScope sc(ctx, s, "split_b", n);
    split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Bv, true, N, k0, Kb, Kp, ldb,
                                                             plan ? 0 : SB, ln.cbot, ln.ctop,
                                                             ln.crad, ln.cplus, o, ln.ctrunc);
  }
  if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  if (plan) {
    // ---- multimodular: residues, NM batched residue products, CRT in the consumer
    if (ensure_crt_constants(ctx->device) != ARBGPU_OK) return ARBGPU_ERR_CUDA;
    CrtDevTables dt{};
    if (crt_device_tables(ctx, plan, &dt) != ARBGPU_OK) return ARBGPU_ERR_CUDA;
    CrtTables ct{dt.Q32,         dt.M32,     dt.y,      dt.rinv,  plan->NM, plan->NMW,
                 plan->NW32P,    dt.crt_wtab, dt.mbytes, plan->NQ, plan->NQP};
    if (plan->NM > 64) ct.wtab = nullptr;  // (the table is built for NM <= 64 only)
    ct.w8 = dt.w8;
    ct.K8 = plan->K8;
    ct.NQ8 = plan->NQ8;
    ct.c32 = dt.c32;
    __nv_bfloat16 *resA = (__nv_bfloat16 *)(ws + w.resA), *resB = (__nv_bfloat16 *)(ws + w.resB);
    // with radii, the two radius products ride in the same GEMM as items NM and NM + 1: their
    // operand planes follow the residue planes, and their exact values come out as int64
    const bool fold = (radA || radB) && crt_gemm_one_chain(Kp);
    __nv_bfloat16 *fA1 = resA + (size_t)2 * NM * M * Kp, *fA2 = fA1 + (size_t)2 * M * Kp;
    __nv_bfloat16 *fB1 = resB + (size_t)2 * NM * N * Kp, *fB2 = fB1 + (size_t)2 * N * Kp;
    // the right-hand residues carry the factor y_t = (M / m_t)^-1 mod m_t of the reconstruction,
    // so the residue products are already z_t = P_t y_t mod m_t
    const SplitOut roA = fold ? SplitOut{nullptr, fA1, fA2}
                              : SplitOut{nullptr, radB ? rA1 : nullptr, radA ? rA2 : nullptr};
    const SplitOut roB = fold ? SplitOut{nullptr, fB1, fB2}
                              : SplitOut{nullptr, radB ? rB1 : nullptr, radA ? rB2 : nullptr};
    const int nchA = (int)((hA + 2 + 31) / 32) + 1, nchB = (int)((hB + 2 + 31) / 32) + 1;
    const int nch = nchA > nchB ? nchA : nchB;
    RtLayout L;
    if (residue_tc_layout(nch, NM, fold, (M > N ? M : N) * Kp, &L)) {
      // work units: algorithmic bytes (every operand entry read once, every residue and radius
      // operand plane written once)
      LaunchScope sc(ctx, s, "residues",
                     (M * (8 * (int64_t)Av.nlimbs + 24) + N * (8 * (int64_t)Bv.nlimbs + 24)) * Kb +
                         (int64_t)L.NPL * (M + N) * Kp * 2);
      RtArgs ra{};
      ra.side[0] = RtSide{Av, M, lda, ln.rbot, ln.rtop, ln.rrad, nullptr,
                          fold ? SplitOut{} : roA, dt.wtab, ln.rtrunc};
      ra.side[1] = RtSide{Bv, N, ldb, ln.cbot, ln.ctop, ln.crad, ln.cplus,
                          fold ? SplitOut{} : roB, dt.wtab + (size_t)plan->NPAD * 128,
                          ln.ctrunc};
      ra.k0 = k0, ra.K = Kb, ra.Kp = Kp, ra.NM = NM, ra.rinv = dt.rinv;
      const arbgpu_status st = launch_residues_tc(ctx, L, nch, s, ra, resA, resB);
      if (st != ARBGPU_OK) return st;
    } else {
      if (omitted) return ARBGPU_ERR_LIMIT;
      {
        LaunchScope sc(ctx, s, "residues_a", M * Kp * NM * nchA);
        if (!launch_residues_mma(ctx, nchA, s, Av, false, M, k0, Kb, Kp, lda, ln.rbot, NM,
                                 dt.w8r, plan->KR, dt.rinv, resA, roA, ln.rtop, ln.rrad,
                                 nullptr))
          launch_residues(nchA, M * Kp, s, Av, false, M, k0, Kb, Kp, lda, ln.rbot, NM, dt.pow32,
                          plan->NCHP, nullptr, resA, roA, ln.rtop, ln.rrad, nullptr);
      }
      {
        LaunchScope sc(ctx, s, "residues_b", N * Kp * NM * nchB);
        if (!launch_residues_mma(ctx, nchB, s, Bv, true, N, k0, Kb, Kp, ldb, ln.cbot, NM,
                                 dt.w8r + (size_t)plan->N2 * plan->KR, plan->KR, dt.rinv, resB,
                                 roB, ln.ctop, ln.crad, ln.cplus))
          launch_residues(nchB, N * Kp, s, Bv, true, N, k0, Kb, Kp, ldb, ln.cbot, NM, dt.pow32,
                          plan->NCHP, dt.y, resB, roB, ln.ctop, ln.crad, ln.cplus);
      }
    }
    if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
    DigitGemmArgs g{resA, resB, (int)M, (int)N, Kp, 2, 2, 1, ws + w.cdig,
                    (int32_t *)(ws + w.ccar), "crt_gemm", NM + (fold ? 2 : 0)};
    g.zout = (uint16_t *)(ws + w.cdig);
    g.ztab = dt.ztab;
    g.zinv = dt.inv;
    if (fold) {
      g.nz = NM;
      g.zraw = (int64_t *)(ws + w.craw);
    }
    arbgpu_status stg = launch_digit_gemm(ctx, g, s);
    if (stg != ARBGPU_OK) return stg;
    *mid = IntProduct{ws + w.cdig, nullptr, 3, 1, {}, 1, ct};
    mid->ends.e[0] = 3;
    if (fold) {
      *rp1 = radB ? IntProduct{ws + w.craw, nullptr, 1, 1, {}, 2, {}} : IntProduct{};
      *rp2 = radA ? IntProduct{ws + w.craw + (size_t)8 * w.Mp * w.Np, nullptr, 1, 1, {}, 2, {}}
                  : IntProduct{};
      return ARBGPU_OK;
    }
  } else {
    const int ND = SA + SB - 1;
    const int G = digit_gemm_groups(ctx, (int)M, (int)N, ND);
    if (G > w.Gmax) return ARBGPU_ERR_LIMIT;
    DigitGemmArgs g{dA, dB, (int)M, (int)N, Kp, SA, SB, G, ws + w.mdig, (int32_t *)(ws + w.mcar),
                    "digit_gemm_mid"};
    arbgpu_status stg = launch_digit_gemm(ctx, g, s);
    if (stg != ARBGPU_OK) return stg;
    *mid = IntProduct{ws + w.mdig, (int32_t *)(ws + w.mcar), ND, G, {}, 0, {}};
    digit_gemm_group_ends(SA, SB, G, mid->ends.e);
  }
  return radius_gemm(ctx, w, ws, M, N, Kp, radA, radB, s, rp1, rp2);
}

// The integer product of one block (Section IV-A) on the engine the cost model picks, or, with
// the context's autotuner on, on the engine measured faster for the product's size bucket: the
// first product of a bucket that both engines can take runs on both (once untimed, then timed
// with CUDA events, the stream synchronised; never while it is being captured), the faster is
// kept for the bucket, and the product is left as the faster engine computed it.  Both engines
// give the same integers.
static int ceil_log2(int64_t v) {
  int b = 0;
  while (((int64_t)1 << b) < v && b < 62) ++b;
  return b;
}

static arbgpu_status run_block(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws, const BallsView &Av,
                               const BallsView &Bv, int64_t M, int64_t N, int64_t lda,
                               int64_t ldb, int64_t k0, int64_t Kb, int64_t hA, int64_t hB,
                               bool radA, bool radB, const Lines &ln, cudaStream_t s,
                               IntProduct *mid, IntProduct *rp1, IntProduct *rp2) {
  auto run = [&](int engine) {
    return run_block_engine(ctx, w, ws, Av, Bv, M, N, lda, ldb, k0, Kb, hA, hB, radA, radB, ln, s,
                            mid, rp1, rp2, engine);
  };
  if (!ctx->autotune || getenv("ARBGPU_ENGINE") || ln.rtrunc || ln.ctrunc) return run(-1);
  bool crt_ok = false, digits_ok = false;
  block_engines(w, Kb, hA, hB, &crt_ok, &digits_ok);
  if (!crt_ok || !digits_ok) return run(-1);
  const int64_t Kp = (Kb + TG_BK - 1) / TG_BK * TG_BK;
  const uint64_t SA = (uint64_t)digits_for_height(hA), SB = (uint64_t)digits_for_height(hB);
  const uint64_t NM = (uint64_t)crt_moduli_for_bits((int)((hA > 0 ? hA : 0) +
                                                          (hB > 0 ? hB : 0) + bit_length(Kb) + 2));
  const uint64_t key = (SA & 1023) | (SB & 1023) << 10 | (NM & 1023) << 20 |
                       (uint64_t)ceil_log2(M) << 30 | (uint64_t)ceil_log2(N) << 36 |
                       (uint64_t)ceil_log2(Kp) << 42;
  const auto it = ctx->engine_tuned.find(key);
  if (it != ctx->engine_tuned.end()) return run(it->second ? 1 : 0);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return run(-1);
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (auto &f : ev)
        if (f) cudaEventDestroy(f);
      return run(-1);
    }
  // one untimed run of each engine first: first-use work (table uploads, kernel attributes)
  // stays out of the timings
  arbgpu_status st = run(1);
  if (st == ARBGPU_OK) st = run(0);
  float t_crt = 0.f, t_dig = 0.f;
  if (st == ARBGPU_OK && cudaEventRecord(ev[0], s) != cudaSuccess) st = ARBGPU_ERR_CUDA;
  if (st == ARBGPU_OK) st = run(1);
  if (st == ARBGPU_OK && cudaEventRecord(ev[1], s) != cudaSuccess) st = ARBGPU_ERR_CUDA;
  if (st == ARBGPU_OK) st = run(0);
  if (st == ARBGPU_OK && (cudaEventRecord(ev[2], s) != cudaSuccess ||
                          cudaEventSynchronize(ev[2]) != cudaSuccess ||
                          cudaEventElapsedTime(&t_crt, ev[0], ev[1]) != cudaSuccess ||
                          cudaEventElapsedTime(&t_dig, ev[1], ev[2]) != cudaSuccess))
    st = ARBGPU_ERR_CUDA;
  for (auto &e : ev) cudaEventDestroy(e);
  if (st != ARBGPU_OK) return st;
  ctx->tune_runs += 4;
  const bool crt_faster = t_crt < t_dig;
  ctx->engine_tuned[key] = crt_faster;
  // the digit engine ran last: its product is the one in the workspace
  return crt_faster ? run(1) : ARBGPU_OK;
}

// Radius products alone (their operands by the digit split, then radius_gemm): those of the
// block [k0, k0 + Kb) of X Y under the lines `ln`.
static arbgpu_status run_radius(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws,
                                const BallsView &Av, const BallsView &Bv, int64_t M, int64_t N,
                                int64_t lda, int64_t ldb, int64_t k0, int64_t Kb, bool radA,
                                bool radB, const Lines &ln, cudaStream_t s, IntProduct *rp1,
                                IntProduct *rp2) {
  const int64_t Kp = (Kb + TG_BK - 1) / TG_BK * TG_BK;
  *rp1 = IntProduct{};
  *rp2 = IntProduct{};
  if (!radA && !radB) return ARBGPU_OK;
  __nv_bfloat16 *rA1 = (__nv_bfloat16 *)(ws + w.rA1), *rA2 = rA1 + (size_t)BL_SR * M * Kp;
  __nv_bfloat16 *rB1 = (__nv_bfloat16 *)(ws + w.rB1), *rB2 = rB1 + (size_t)BL_SR * N * Kp;
  {
    const int64_t n = M * Kp;
    SplitOut o{nullptr, radB ? rA1 : nullptr, radA ? rA2 : nullptr};
    LaunchScope sc(ctx, s, "split_a", n);
    split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Av, false, M, k0, Kb, Kp, lda, 0,
                                                             ln.rbot, ln.rtop, ln.rrad, nullptr, o,
                                                             ln.rtrunc);
  }
  {
    const int64_t n = N * Kp;
    SplitOut o{nullptr, radB ? rB1 : nullptr, radA ? rB2 : nullptr};
    LaunchScope sc(ctx, s, "split_b", n);
    split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Bv, true, N, k0, Kb, Kp, ldb, 0,
                                                             ln.cbot, ln.ctop, ln.crad, ln.cplus,
                                                             o, ln.ctrunc);
  }
  if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  return radius_gemm(ctx, w, ws, M, N, Kp, radA, radB, s, rp1, rp2);
}

// Statistics of one real product X * Y from the whole-range scans of its parts.
static BlockStats merge_stats(const BlockStats &rows, const BlockStats &cols) {
  BlockStats m{};
  m.pA = rows.pA;
  m.hA = rows.hA;
  m.radA = rows.radA;
  m.pB = cols.pB;
  m.hB = cols.hB;
  m.radB = cols.radB;
  m.special = rows.special | cols.special;
  return m;
}

static int64_t height_bound(int prec, const BlockStats &hs) {
  const int64_t pmax = hs.pA > hs.pB ? hs.pA : hs.pB;
  return (5 * (prec < pmax ? (int64_t)prec : pmax)) / 4 + 192;
}

// Per-entry tops and bottoms of X (M x K, rows in tA / bA) and of Y (K x N, columns in the rows of
// tBT / bBT) for the planner and the inner ordering.
static arbgpu_status entry_tops(arbgpu_ctx *ctx, const BallsView &Xv, const BallsView &Yv,
                                int64_t M, int64_t K, int64_t N, int64_t ldx, int64_t ldy,
                                int64_t *tA, int64_t *bA, int64_t *tBT, int64_t *bBT,
                                cudaStream_t s, bool merge = false) {
  LaunchScope sc(ctx, s, "entry_tb", M * K + K * N);
  entry_tb_kernel<<<(unsigned)((M * K + 255) / 256), 256, 0, s>>>(Xv, M, K, ldx, tA, bA,
                                                                    merge ? 1 : 0);
  const int64_t tiles = ((K + 31) / 32) * ((N + 31) / 32);
  entry_tb_t_kernel<<<(unsigned)tiles, 256, 0, s>>>(Yv, K, N, ldy, tBT, bBT, merge ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

// Append one plan record to ctx->plan_log: kind (0 contiguous, 1 over the inner order, 2 one
// block shared by both parts of a complex product by eq. 2), h, K, the block count, then the
// [start, stop, basecase] triples.
static void log_plan(arbgpu_ctx *ctx, int kind, int64_t h, int64_t K,
                     const std::vector<int32_t> &triples) {
  std::vector<int64_t> &L = ctx->plan_log;
  L.push_back(kind);
  L.push_back(h);
  L.push_back(K);
  L.push_back((int64_t)(triples.size() / 3));
  for (int32_t v : triples) L.push_back(v);
}

// ---- negligible-limb omission (Section IV-B's last paragraph: Algorithm 2 uses every input bit,
// where Algorithm 1 omits negligible limbs).  Reading: with E_ij = max_k top(x_ik) + top(y_kj)
// (maxplus_top_kernel), the bits of row i of X below tau_i = min_j (E_ij - ctop_j) - p - G and of
// column j of Y below sigma_j = min_i (E_ij - rtop_i) - p - G, G = bc(K) + 8 (minima over the
// entries with a nonzero product), are dropped toward zero: the scaled integers then start at
// max(bottom, tau).  The product changes by less than 3 K 2^(E_ij - p - G) <= (3/64) 2^-p
// sum_k |x_ik y_kj|, and every nonzero entry of a truncated line carries 2^tau (2^sigma) more
// radius (the tensor-core residue kernel adds it), so the ball stays rigorous.  A line without a
// nonzero product is left as it is.

// Rows: one warp per row of X.  Writes the truncated row lines and tau (INT64_MIN: none) and
// folds the row heights and radius flags into st.
__global__ void __launch_bounds__(256) omission_rows_kernel(
    const int64_t *E, int64_t M, int64_t N, const int64_t *rtop, const int64_t *rbot,
    const int64_t *rrad, const int64_t *ctop, int64_t off, int64_t *obot, int64_t *orad,
    int64_t *otrunc, BlockStats *st) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= M) return;
  long long m = INT64_MAX;
  for (int64_t j = lane; j < N; j += 32) {
    const int64_t e = E[i * N + j];
    if (e != INT64_MIN) m = min(m, (long long)(e - ctop[j]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane != 0) return;
  int64_t bot = rbot[i], rr = rrad[i], t = INT64_MIN;
  if (m != INT64_MAX && rtop[i] != INT64_MIN && bot < m - off) {
    t = m - off;
    bot = t;
    rr = rr > t + 1 ? rr : t + 1;
  }
  obot[i] = bot;
  orad[i] = rr;
  otrunc[i] = t;
  if (rtop[i] != INT64_MIN) atomic_max_i64(&st->hA, rtop[i] - bot);
  if (rr != INT64_MIN) atomicOr(&st->radA, 1);
}

// Columns: 32 columns x 8 row slices per CTA, the slices' minima combined in shared memory.
__global__ void __launch_bounds__(256) omission_cols_kernel(
    const int64_t *E, int64_t M, int64_t N, const int64_t *rtop, const int64_t *ctop,
    const int64_t *cbot, const int64_t *crad, int64_t off, int64_t *obot, int64_t *orad,
    int64_t *oplus, int64_t *otrunc, BlockStats *st) {
  __shared__ long long s_m[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + tx;
  long long m = INT64_MAX;
  if (j < N)
    for (int64_t i = ty; i < M; i += 8) {
      const int64_t e = E[i * N + j];
      if (e != INT64_MIN) m = min(m, (long long)(e - rtop[i]));
    }
  s_m[ty][tx] = m;
  __syncthreads();
  if (ty != 0 || j >= N) return;
  for (int q = 1; q < 8; ++q) m = min(m, s_m[q][tx]);
  int64_t bot = cbot[j], rr = crad[j], t = INT64_MIN;
  if (m != INT64_MAX && ctop[j] != INT64_MIN && bot < m - off) {
    t = m - off;
    bot = t;
    rr = rr > t + 1 ? rr : t + 1;
  }
  obot[j] = bot;
  orad[j] = rr;
  otrunc[j] = t;
  const int64_t mx = ctop[j] > rr ? ctop[j] : rr;  // |y| + r_y < 2^(max(top, rexp) + 1)
  oplus[j] = mx == INT64_MIN ? INT64_MIN : mx + 1;
  if (ctop[j] != INT64_MIN) atomic_max_i64(&st->hB, ctop[j] - bot);
  if (rr != INT64_MIN) atomicOr(&st->radB, 1);
}

static bool omission_enabled() {
  const char *e = getenv("ARBGPU_OMIT");
  return !(e && !strcmp(e, "0"));
}

// Whether the omission is worth trying for a product with these statistics: it needs several
// blocks as it is, and some line is more than 32 bits taller than p + G needs.  (For a product
// that already fits one block the saved moduli did not repay the extra passes and the statistics
// read-back: the grouped workload of 256 products ran 77 -> 94 ms with it.)
static bool omission_wanted(int prec, int64_t K, const BlockStats &hs, bool one_block) {
  if (!omission_enabled() || one_block) return false;
  int bk = 0;
  for (int64_t v = K; v > 0; v >>= 1) ++bk;
  const int64_t lim = (int64_t)prec + bk + 8 + 32;
  return hs.hA > lim || hs.hB > lim;
}

struct Omitted {
  bool ok;
  Lines lines;
  BlockStats hs;
};

// The omission for X Y under the whole-range lines `full`, from E = its max-plus bound
// (launch_maxplus): the thresholds, the truncated lines in the workspace and their statistics
// (one read-back).  ok when the truncated operands fit one
// block of height <= h (h of the untruncated operands' precisions) and the tensor-core residue
// kernel takes them; otherwise nothing is used.
static arbgpu_status omit_product(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws,
                                  const int64_t *E, int64_t M, int64_t K, int64_t N, int prec,
                                  const Lines &full, const BlockStats &hs, cudaStream_t s,
                                  Omitted *out) {
  out->ok = false;
  int bk = 0;
  for (int64_t v = K; v > 0; v >>= 1) ++bk;
  const int64_t off = (int64_t)prec + bk + 8;
  int64_t *rb = (int64_t *)(ws + w.om_rbot), *rr = (int64_t *)(ws + w.om_rrad);
  int64_t *rt = (int64_t *)(ws + w.om_rtrunc);
  int64_t *cb = (int64_t *)(ws + w.om_cbot), *cr = (int64_t *)(ws + w.om_crad);
  int64_t *cp = (int64_t *)(ws + w.om_cplus), *ct = (int64_t *)(ws + w.om_ctrunc);
  BlockStats *st = (BlockStats *)(ws + w.om_stats);
  if (cudaMemsetAsync(st, 0, sizeof(BlockStats), s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  {
    LaunchScope sc(ctx, s, "omission", M * N);
    omission_rows_kernel<<<(unsigned)((M + 7) / 8), 256, 0, s>>>(
        E, M, N, full.rtop, full.rbot, full.rrad, full.ctop, off, rb, rr, rt, st);
    omission_cols_kernel<<<(unsigned)((N + 31) / 32), 256, 0, s>>>(
        E, M, N, full.rtop, full.ctop, full.cbot, full.crad, off, cb, cr, cp, ct, st);
    if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  }
  BlockStats os{};
  const arbgpu_status rs = read_stats(ctx, st, &os, 1, s);
  if (rs != ARBGPU_OK) return rs;
  os.pA = hs.pA;
  os.pB = hs.pB;
  os.special = hs.special;
  const int64_t h = height_bound(prec, hs);
  if (os.hA > h || os.hB > h) return ARBGPU_OK;
  // the tensor-core residue kernel must take the truncated operands (it adds their radius)
  const int NM = crt_moduli_for_bits((int)((os.hA > 0 ? os.hA : 0) + (os.hB > 0 ? os.hB : 0) +
                                           bk + 2));
  const int nch = (int)(((os.hA > os.hB ? os.hA : os.hB) + 2 + 31) / 32) + 1;
  if (NM > w.NMmax || NM > 128 || nch > 32) return ARBGPU_OK;
  {
    RtLayout L;  // (with the radius planes: the larger of the two shapes)
    if (!residue_tc_layout(nch, NM, true, (M > N ? M : N) * w.Kp, &L)) return ARBGPU_OK;
    const CrtPlan *plan = crt_plan(NM);
    if (!plan || plan->NMW + 1 > RD_MAXW) return ARBGPU_OK;
  }
  out->lines = Lines{full.rtop, rb, rr, full.ctop, cb, cr, cp, rt, ct};
  out->hs = os;
  out->ok = true;
  return ARBGPU_OK;
}

// ---- the omission for eq. 2 (Section IV-B's last paragraph under Section IV-C's shared scaling).
// Reading: both parts of a row of A (a column of B) drop their bits below one threshold, so the
// truncated parts keep one scaling per line shared by both parts.  With E_q the per-entry bound
// of output part q (its two real products, maxplus_top_kernel) and the shared line tops,
// tau_i = min_{q, j} (E_q,ij - ctop_j) - p - G and sigma_j = min_{q, i} (E_q,ij - rtop_i) - p - G,
// G = bc(K) + 9: part q changes by less than 4 K 2^(E_q,ij - p - G) <= (1/32) 2^-p times the sum
// of |a b| over its terms.  Every nonzero entry of a truncated line, in either part, carries
// 2^tau (2^sigma) more radius (split_kernel adds it to the radius operands).

// Rows: one warp per row of A.  Writes the shared truncated bottoms and tau (INT64_MIN: none), each
// part's radius line (rrad_q raised to tau + 1 where part q's row is nonzero), and folds the shared
// row heights into st[0].hA and each part's radius flag into st[1 + q].radA.
__global__ void __launch_bounds__(256) omission_eq2_rows_kernel(
    const int64_t *E0, const int64_t *E1, int64_t M, int64_t N, const int64_t *rtop,
    const int64_t *rbot, const int64_t *ctop, const int64_t *rtop0, const int64_t *rtop1,
    const int64_t *rrad0, const int64_t *rrad1, int64_t off, int64_t *obot, int64_t *otrunc,
    int64_t *orad0, int64_t *orad1, BlockStats *st) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= M) return;
  long long m = INT64_MAX;
  for (int64_t j = lane; j < N; j += 32) {
    const int64_t e0 = E0[i * N + j], e1 = E1[i * N + j];
    if (e0 != INT64_MIN) m = min(m, (long long)(e0 - ctop[j]));
    if (e1 != INT64_MIN) m = min(m, (long long)(e1 - ctop[j]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane != 0) return;
  int64_t bot = rbot[i], t = INT64_MIN;
  if (m != INT64_MAX && rtop[i] != INT64_MIN && bot < m - off) {
    t = m - off;
    bot = t;
  }
  obot[i] = bot;
  otrunc[i] = t;
  const int64_t *pt[2] = {rtop0, rtop1}, *pr[2] = {rrad0, rrad1};
  int64_t *po[2] = {orad0, orad1};
  for (int q = 0; q < 2; ++q) {
    int64_t rr = pr[q][i];
    if (t != INT64_MIN && pt[q][i] != INT64_MIN) rr = rr > t + 1 ? rr : t + 1;
    po[q][i] = rr;
    if (rr != INT64_MIN) atomicOr(&st[1 + q].radA, 1);
  }
  if (rtop[i] != INT64_MIN) atomic_max_i64(&st[0].hA, rtop[i] - bot);
}

// Columns: 32 columns x 8 row slices per CTA, the slices' minima combined in shared memory; the
// same outputs for the columns of B (radius and |y| + r_y lines of each part, flags in radB).
__global__ void __launch_bounds__(256) omission_eq2_cols_kernel(
    const int64_t *E0, const int64_t *E1, int64_t M, int64_t N, const int64_t *rtop,
    const int64_t *ctop, const int64_t *cbot, const int64_t *ctop0, const int64_t *ctop1,
    const int64_t *crad0, const int64_t *crad1, int64_t off, int64_t *obot, int64_t *otrunc,
    int64_t *orad0, int64_t *orad1, int64_t *oplus0, int64_t *oplus1, BlockStats *st) {
  __shared__ long long s_m[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + tx;
  long long m = INT64_MAX;
  if (j < N)
    for (int64_t i = ty; i < M; i += 8) {
      const int64_t e0 = E0[i * N + j], e1 = E1[i * N + j];
      if (e0 != INT64_MIN) m = min(m, (long long)(e0 - rtop[i]));
      if (e1 != INT64_MIN) m = min(m, (long long)(e1 - rtop[i]));
    }
  s_m[ty][tx] = m;
  __syncthreads();
  if (ty != 0 || j >= N) return;
  for (int q = 1; q < 8; ++q) m = min(m, s_m[q][tx]);
  int64_t bot = cbot[j], t = INT64_MIN;
  if (m != INT64_MAX && ctop[j] != INT64_MIN && bot < m - off) {
    t = m - off;
    bot = t;
  }
  obot[j] = bot;
  otrunc[j] = t;
  const int64_t *pt[2] = {ctop0, ctop1}, *pr[2] = {crad0, crad1};
  int64_t *po[2] = {orad0, orad1}, *pp[2] = {oplus0, oplus1};
  for (int q = 0; q < 2; ++q) {
    int64_t rr = pr[q][j];
    if (t != INT64_MIN && pt[q][j] != INT64_MIN) rr = rr > t + 1 ? rr : t + 1;
    po[q][j] = rr;
    const int64_t mx = pt[q][j] > rr ? pt[q][j] : rr;  // |y| + r_y < 2^(max(top, rexp) + 1)
    pp[q][j] = mx == INT64_MIN ? INT64_MIN : mx + 1;
    if (rr != INT64_MIN) atomicOr(&st[1 + q].radB, 1);
  }
  if (ctop[j] != INT64_MIN) atomic_max_i64(&st[0].hB, ctop[j] - bot);
}

// Output of a real product that may be rounded straight from one exact block.
struct DirectRound {
  BallsOut C;
  int64_t ldc;
};

// The greedy extraction of Algorithm 2 on the per-entry tops and bottoms in the workspace (tA / bA
// for the rows of X, tB / bB for the columns of Y, from entry_tops): one cooperative launch, then
// the [start, stop, basecase] triples read back into hb (the plan stays at w.blocks).
static arbgpu_status plan_blocks(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws, int64_t M,
                                 int64_t K, int64_t N, int64_t h, cudaStream_t s,
                                 std::vector<int32_t> &hb) {
  int64_t *tA = (int64_t *)(ws + w.tA), *bA = (int64_t *)(ws + w.bA);
  int64_t *tBT = (int64_t *)(ws + w.tB), *bBT = (int64_t *)(ws + w.bB);
  int32_t *blocks = (int32_t *)(ws + w.blocks), *nblocks = (int32_t *)(ws + w.nblocks);
  {
    int *state = (int *)(nblocks + 2);
    unsigned *bar = (unsigned *)(nblocks + 4);
    int *failed = (int *)(nblocks + 6);
    int64_t hh = h;
    int maxb = w.maxb;
    int *status = ctx->status;
    void *args[] = {&tA, &bA, &tBT, &bBT, &M, &K, &N, &hh, &blocks, &nblocks, &maxb,
                    &state, &bar, &failed, &status};
    const int grid = plan_coop_grid(ctx->device, M + N);
    if (grid < 1 || cudaMemsetAsync(nblocks, 0, 32, s) != cudaSuccess) return ARBGPU_ERR_CUDA;
    LaunchScope sc(ctx, s, "plan", M + N);
    if (cudaLaunchCooperativeKernel((const void *)plan_coop_kernel, dim3(grid), dim3(256), args,
                                    0, s) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
  }
  int32_t nb = 0;
  if (cudaMemcpyAsync(&nb, nblocks, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  if (nb < 1 || nb > w.maxb) return ARBGPU_ERR_LIMIT;
  hb.assign(3 * (size_t)nb, 0);
  if (cudaMemcpyAsync(hb.data(), blocks, 12 * (size_t)nb, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return ARBGPU_ERR_CUDA;
  return ARBGPU_OK;
}

// Add (-1)^negate X Y to the accumulator by Algorithm 2: plan the blocks of this product, run the
// products of the full blocks and accumulate them; append the basecase indices, tagged with
// `combo`, to `basek`.
static arbgpu_status accumulate_product(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws,
                                        const BallsView &Xv, const BallsView &Yv, int64_t M,
                                        int64_t K, int64_t N, int64_t ldx, int64_t ldy, int prec,
                                        const Lines &full, const BlockStats &hs, bool negate,
                                        int combo, const AccView &av, cudaStream_t s,
                                        std::vector<int32_t> &basek,
                                        const std::vector<int32_t> *kmap = nullptr,
                                        const DirectRound *direct = nullptr,
                                        bool *rounded = nullptr,
                                        const std::function<arbgpu_status()> *prepare = nullptr,
                                        int plan_kind = 0) {
  const int64_t h = height_bound(prec, hs);
  std::vector<int32_t> hb;
  std::vector<BlockStats> hbs;
  Lines per = full;
  int hnb = 1;
  BlockStats init{};
  init.hA = init.hB = INT64_MIN;
  if (hs.hA <= h && hs.hB <= h) {
    hb = {0, (int32_t)K, 0};
    hbs = {hs};
    log_plan(ctx, plan_kind, h, K, hb);
  } else {
    const arbgpu_status est = entry_tops(ctx, Xv, Yv, M, K, N, ldx, ldy, (int64_t *)(ws + w.tA),
                                         (int64_t *)(ws + w.bA), (int64_t *)(ws + w.tB),
                                         (int64_t *)(ws + w.bB), s);
    if (est != ARBGPU_OK) return est;
    const arbgpu_status pst = plan_blocks(ctx, w, ws, M, K, N, h, s, hb);
    if (pst != ARBGPU_OK) return pst;
    hnb = (int)(hb.size() / 3);
    hbs.assign((size_t)hnb, init);
    BlockStats *bst = (BlockStats *)(ws + w.bstats);
    const int32_t *blocks = (const int32_t *)(ws + w.blocks);
    if (cudaMemcpyAsync(bst, hbs.data(), sizeof(BlockStats) * hnb, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return ARBGPU_ERR_CUDA;
    per = Lines{(int64_t *)(ws + w.brtop), (int64_t *)(ws + w.brbot), (int64_t *)(ws + w.brrad),
                (int64_t *)(ws + w.bctop), (int64_t *)(ws + w.bcbot), (int64_t *)(ws + w.bcrad),
                (int64_t *)(ws + w.bcplus)};
    {
      // chunks sized for the whole range (a block's chunks beyond its end return at once)
      const arbgpu_status sst = run_scans(
          ctx, s, Xv, M, K, ldx, Yv, N, ldy, blocks, hnb, K, (int64_t *)per.rtop,
          (int64_t *)per.rbot, (int64_t *)per.rrad, (int64_t *)per.ctop, (int64_t *)per.cbot,
          (int64_t *)per.crad, (int64_t *)per.cplus, bst, bst);
      if (sst != ARBGPU_OK) return sst;
    }
    if (cudaMemcpyAsync(hbs.data(), bst, sizeof(BlockStats) * hnb, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
    log_plan(ctx, 0, h, K, hb);
  }
  const bool planned = per.rtop != full.rtop;
  if (direct && planned && hnb == 1 && hb[2] == 0 && !negate) {
    // one full block after all (over the inner order): exact product, one rounding per entry
    const Lines lb{per.rtop, per.rbot, per.rrad, per.ctop, per.cbot, per.crad, per.cplus};
    RoundArgs ra{};
    const arbgpu_status st1 = run_block(ctx, w, ws, Xv, Yv, M, N, ldx, ldy, 0, K, hbs[0].hA,
                                        hbs[0].hB, hbs[0].radA != 0, hbs[0].radB != 0, lb, s,
                                        &ra.mid, &ra.rp1, &ra.rp2);
    if (st1 != ARBGPU_OK) return st1;
    ra.rtop = lb.rtop;
    ra.rbot = lb.rbot;
    ra.rrad = lb.rrad;
    ra.ctop = lb.ctop;
    ra.cbot = lb.cbot;
    ra.crad = lb.crad;
    ra.cplus = lb.cplus;
    ra.C = direct->C;
    ra.M = M;
    ra.N = N;
    ra.ldc = direct->ldc;
    ra.Mp = w.Mp;
    ra.Np = w.Np;
    ra.prec = prec;
    {
      const int64_t units =
          ra.mid.kind == 1 ? M * N * ra.mid.crt.NM * (int64_t)(2 * ra.mid.crt.NMW) : M * N;
      LaunchScope sc(ctx, s, "block_round", units);
      launch_block_round(ctx, ra, s);
    }
    *rounded = true;
    return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
  }
  if (prepare) {  // the accumulator's set-up, launched before its first use
    const arbgpu_status pst = (*prepare)();
    if (pst != ARBGPU_OK) return pst;
  }
  for (int b = 0; b < hnb; ++b) {
    const int64_t k0 = hb[3 * b], k1 = hb[3 * b + 1];
    if (hb[3 * b + 2]) {
      for (int64_t k = k0; k < k1; ++k)  // (inner indices of the caller's operands)
        basek.push_back((int32_t)(((kmap ? (int64_t)(*kmap)[k] : k) << 2) | combo));
      continue;
    }
    const int64_t oM = planned ? (int64_t)b * M : 0, oN = planned ? (int64_t)b * N : 0;
    // (the omission's per-line exponents belong to the whole-range lines: one block only)
    const Lines lb{per.rtop + oM,  per.rbot + oM,  per.rrad + oM,
                   per.ctop + oN,  per.cbot + oN,  per.crad + oN,
                   per.cplus + oN, planned ? nullptr : per.rtrunc,
                   planned ? nullptr : per.ctrunc};
    AccArgs aa{};
    arbgpu_status st1 = run_block(ctx, w, ws, Xv, Yv, M, N, ldx, ldy, k0, k1 - k0, hbs[b].hA,
                                  hbs[b].hB, hbs[b].radA != 0, hbs[b].radB != 0, lb, s, &aa.mid,
                                  &aa.rp1, &aa.rp2);
    if (st1 != ARBGPU_OK) return st1;
    aa.rtop = lb.rtop;
    aa.rbot = lb.rbot;
    aa.rrad = lb.rrad;
    aa.ctop = lb.ctop;
    aa.cbot = lb.cbot;
    aa.crad = lb.crad;
    aa.cplus = lb.cplus;
    aa.v = av;
    aa.M = M;
    aa.N = N;
    aa.Mp = w.Mp;
    aa.Np = w.Np;
    aa.negate = negate ? 1 : 0;
    LaunchScope sc(ctx, s, "accumulate", M * N);
    if (aa.mid.kind == 1) {
      // multimodular: the reconstruction on the tensor cores, adding into the window
      RoundArgs ra{};
      ra.mid = aa.mid;
      ra.rp1 = aa.rp1;
      ra.rp2 = aa.rp2;
      ra.rtop = aa.rtop;
      ra.rbot = aa.rbot;
      ra.rrad = aa.rrad;
      ra.ctop = aa.ctop;
      ra.cbot = aa.cbot;
      ra.crad = aa.crad;
      ra.cplus = aa.cplus;
      ra.M = M;
      ra.N = N;
      ra.Mp = w.Mp;
      ra.Np = w.Np;
      ra.prec = prec;
      ra.acc = av;
      ra.negate = aa.negate;
      arbgpu_status tst = ARBGPU_OK;
      if (launch_crt_round_tc(ctx, ra, s, &tst, true)) {
        if (tst != ARBGPU_OK) return tst;
        continue;
      }
    }
    accumulate_kernel<<<(unsigned)((M * N + 127) / 128), 128, 0, s>>>(aa);
  }
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

// ---- complex product by eq. 2 (Section IV-C: three real products of the midpoint matrices when
// the entries are uniformly scaled).  With one exponent per row of A and per column of B shared by
// both parts (merge_parts_kernel), X_re, X_im, Y_re, Y_im are integer matrices and
//   P_1 = X_re Y_re,  P_2 = X_im Y_im,  P_3 = (X_re + X_im)(Y_re + Y_im),
//   Re = P_1 - P_2,  Im = P_3 - P_1 - P_2
// hold exactly.  The three products run as one batch of residue products; Re and Im are formed
// modulus by modulus and reconstructed, so |Re|, |Im| < 2 K 2^(hA + hB) sets the modulus count.
// The radii are the four real radius products of the 4M path.
struct Plan3M {
  bool ok;
  bool several;  // the shared scaling needs several blocks (accumulate_eq2)
  int64_t hA, hB;
  int NM, nch;
  const CrtPlan *plan;
  RtLayout L;
  int64_t *rtop, *rbot, *ctop, *cbot;  // the shared lines
};

// Merge the parts' lines and decide: ok when the shared scaling fits one block of height
// <= h (the bound of Algorithm 2 for the operands' precisions) and the multimodular engine with
// the tensor-core residue kernel takes the sizes.  One statistics read-back.
static arbgpu_status plan_3m(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws, const Lines *rowsL,
                             const Lines *colsL, const BlockStats *hst, int64_t M, int64_t K,
                             int64_t N, int prec, cudaStream_t s, Plan3M *p) {
  p->ok = false;
  p->several = false;
  if (!w.r3A) return ARBGPU_OK;
  p->rtop = (int64_t *)(ws + w.brtop);
  p->rbot = (int64_t *)(ws + w.brbot);
  p->ctop = (int64_t *)(ws + w.bctop);
  p->cbot = (int64_t *)(ws + w.bcbot);
  BlockStats *dst = (BlockStats *)(ws + w.bstats);
  {
    LaunchScope sc(ctx, s, "merge_parts", M + N);
    merge_parts_kernel<<<1, 1024, 0, s>>>(rowsL[0].rtop, rowsL[0].rbot, rowsL[1].rtop,
                                          rowsL[1].rbot, M, p->rtop, p->rbot, colsL[0].ctop,
                                          colsL[0].cbot, colsL[1].ctop, colsL[1].cbot, N, p->ctop,
                                          p->cbot, dst);
    if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  }
  BlockStats hm{};
  const arbgpu_status st = read_stats(ctx, dst, &hm, 1, s);
  if (st != ARBGPU_OK) return st;
  if (hm.hA == INT64_MIN || hm.hB == INT64_MIN) return ARBGPU_OK;  // a zero operand
  BlockStats hs{};
  hs.pA = hst[0].pA > hst[1].pA ? hst[0].pA : hst[1].pA;
  hs.pB = hst[2].pB > hst[3].pB ? hst[2].pB : hst[3].pB;
  const int64_t h = height_bound(prec, hs);
  p->hA = hm.hA;  // (the shared heights, also when they need several blocks)
  p->hB = hm.hB;
  if (hm.hA > h || hm.hB > h) {
    p->several = true;
    return ARBGPU_OK;
  }
  p->NM = crt_moduli_for_bits((int)(p->hA + p->hB + bit_length(K) + 3));
  if (p->NM > w.NMmax) return ARBGPU_OK;
  p->plan = crt_plan(p->NM);
  if (!p->plan || p->plan->NMW + 1 > RD_MAXW) return ARBGPU_OK;
  p->nch = (int)(((p->hA > p->hB ? p->hA : p->hB) + 2 + 31) / 32) + 1;
  if (!residue_tc_layout(p->nch, p->NM, false, (M > N ? M : N) * w.Kp, &p->L)) return ARBGPU_OK;
  p->ok = true;
  log_plan(ctx, 2, h, K, {0, (int32_t)K, 0});
  return ARBGPU_OK;
}

// The three residue products of eq. 2 over the inner range [k0, k0 + Kb) under lines shared by
// both parts (rtop / rbot: rows of A, ctop / cbot: columns of B; radius windows of part q in
// pl[q]): the residues of each part, those of X_re + X_im and Y_re + Y_im, the 3 NM residue
// products, then Re = P1 - P2 and Im = P3 - P1 - P2 in place of P1 and P2 (z3m_kernel).  *z
// receives Re's NM planes of Mp x Np (Im's follow), *ct the tables to reconstruct them.
static arbgpu_status eq2_products(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws, int NM,
                                  const CrtPlan *plan, int nch, const RtLayout &L,
                                  const BallsView *Av, const BallsView *Bv, int64_t M, int64_t N,
                                  int64_t lda, int64_t ldb, int64_t k0, int64_t Kb,
                                  const int64_t *rtop, const int64_t *rbot, const int64_t *ctop,
                                  const int64_t *cbot, const Lines *pl, cudaStream_t s,
                                  uint16_t **z, CrtTables *ct) {
  const int64_t Kp = (Kb + TG_BK - 1) / TG_BK * TG_BK;
  if (ensure_crt_constants(ctx->device) != ARBGPU_OK) return ARBGPU_ERR_CUDA;
  CrtDevTables dt{};
  if (crt_device_tables(ctx, plan, &dt) != ARBGPU_OK) return ARBGPU_ERR_CUDA;
  // (the tensor-core reconstruction's weight table exists for NM <= 64)
  *ct = CrtTables{dt.Q32,        dt.M32,                    dt.y,      dt.rinv,
                  NM,            plan->NMW,                 plan->NW32P,
                  NM <= 64 ? dt.crt_wtab : nullptr, dt.mbytes, plan->NQ, plan->NQP,
                  dt.w8,         plan->K8,                  plan->NQ8,
                  dt.c32};
  // residue planes [re | im | re + im] of each side, 2 NM planes each
  __nv_bfloat16 *xr = (__nv_bfloat16 *)(ws + w.r3A), *yr = (__nv_bfloat16 *)(ws + w.r3B);
  const size_t setA = (size_t)2 * NM * M * Kp, setB = (size_t)2 * NM * N * Kp;
  for (int q = 0; q < 2; ++q) {
    LaunchScope sc(ctx, s, "residues",
                   (M * (8 * (int64_t)Av[q].nlimbs + 24) + N * (8 * (int64_t)Bv[q].nlimbs + 24)) *
                           Kb +
                       (int64_t)L.NPL * (M + N) * Kp * 2);
    RtArgs ra{};
    ra.side[0] = RtSide{Av[q], M, lda, rbot, rtop, pl[q].rrad, nullptr, SplitOut{}, dt.wtab};
    ra.side[1] = RtSide{Bv[q],      N,         ldb, cbot, ctop, pl[q].crad, pl[q].cplus,
                        SplitOut{}, dt.wtab + (size_t)plan->NPAD * 128};
    ra.k0 = k0, ra.K = Kb, ra.Kp = Kp, ra.NM = NM, ra.rinv = dt.rinv;
    const arbgpu_status st = launch_residues_tc(ctx, L, nch, s, ra, xr + q * setA, yr + q * setB);
    if (st != ARBGPU_OK) return st;
  }
  {
    const int64_t nv = (int64_t)NM * (M * Kp / 8 + N * Kp / 8);
    LaunchScope sc(ctx, s, "residue_sum", nv * 8);
    residue_sum_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(
        xr, xr + setA, xr + 2 * setA, M * Kp, yr, yr + setB, yr + 2 * setB, N * Kp, NM);
    if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  }
  *z = (uint16_t *)(ws + w.z3);
  DigitGemmArgs g{xr, yr, (int)M, (int)N, Kp, 2, 2, 1, ws + w.z3, (int32_t *)(ws + w.ccar),
                  "crt_gemm", 3 * NM};
  g.zout = *z;
  g.ztab = dt.ztab;
  g.zinv = dt.inv;
  arbgpu_status stg = launch_digit_gemm(ctx, g, s);
  if (stg != ARBGPU_OK) return stg;
  const int64_t plane = w.Mp * w.Np;
  const int64_t nv = (int64_t)NM * (plane / 8);
  LaunchScope sc(ctx, s, "z3m", nv * 8);
  z3m_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(*z, NM, plane);
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

// Run the planned eq. 2 product: the radius bounds of each part summed into av[q].rman / rexp
// (zeroed by the caller), then Re and Im reconstructed and rounded straight into C[0], C[1].
static arbgpu_status run_3m(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws, const Plan3M &p,
                            const arbgpu_balls *C, const BallsView *Av, const BallsView *Bv,
                            const Lines *rowsL, const Lines *colsL, const BlockStats *hst,
                            int64_t M, int64_t K, int64_t N, int64_t lda, int64_t ldb,
                            int64_t ldc, int prec, const AccView *av, cudaStream_t s) {
  const int NM = p.NM;
  const Lines pl[2] = {Lines{nullptr, nullptr, rowsL[0].rrad, nullptr, nullptr, colsL[0].crad,
                             colsL[0].cplus},
                       Lines{nullptr, nullptr, rowsL[1].rrad, nullptr, nullptr, colsL[1].crad,
                             colsL[1].cplus}};
  uint16_t *z = nullptr;
  CrtTables ct{};
  const arbgpu_status pst = eq2_products(ctx, w, ws, NM, p.plan, p.nch, p.L, Av, Bv, M, N, lda,
                                         ldb, 0, K, p.rtop, p.rbot, p.ctop, p.cbot, pl, s, &z,
                                         &ct);
  if (pst != ARBGPU_OK) return pst;
  const int64_t plane = w.Mp * w.Np;
  // radii: Re from A_re B_re and A_im B_im, Im from A_re B_im and A_im B_re, summed per entry
  const int pairs[4][3] = {{0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
  for (const auto &pr : pairs) {
    const int part = pr[0], xa = pr[1], yb = pr[2];
    const bool radA = hst[xa].radA != 0, radB = hst[2 + yb].radB != 0;
    if (!radA && !radB) continue;
    const Lines ln{rowsL[xa].rtop,  rowsL[xa].rbot, rowsL[xa].rrad,   colsL[yb].ctop,
                   colsL[yb].cbot,  colsL[yb].crad, colsL[yb].cplus,  rowsL[xa].rtrunc,
                   colsL[yb].ctrunc};
    AccArgs aa{};
    const arbgpu_status st = run_radius(ctx, w, ws, Av[xa], Bv[yb], M, N, lda, ldb, 0, K, radA,
                                        radB, ln, s, &aa.rp1, &aa.rp2);
    if (st != ARBGPU_OK) return st;
    aa.rtop = ln.rtop;
    aa.rbot = ln.rbot;
    aa.rrad = ln.rrad;
    aa.ctop = ln.ctop;
    aa.cbot = ln.cbot;
    aa.crad = ln.crad;
    aa.cplus = ln.cplus;
    aa.v = av[part];
    aa.M = M;
    aa.N = N;
    aa.Mp = w.Mp;
    aa.Np = w.Np;
    aa.skip_mid = 1;
    LaunchScope sc(ctx, s, "accumulate", M * N);
    accumulate_kernel<<<(unsigned)((M * N + 127) / 128), 128, 0, s>>>(aa);
  }
  if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  // Re and Im are exact integers under the shared lines: one rounding each, as for a real block
  for (int q = 0; q < 2; ++q) {
    RoundArgs ra{};
    ra.mid = IntProduct{(const uint8_t *)(z + (size_t)q * NM * plane), nullptr, 3, 1, {}, 1, ct};
    ra.mid.ends.e[0] = 3;
    ra.rtop = p.rtop;
    ra.rbot = p.rbot;
    ra.rrad = rowsL[q].rrad;
    ra.ctop = p.ctop;
    ra.cbot = p.cbot;
    ra.crad = colsL[q].crad;
    ra.cplus = colsL[q].cplus;
    ra.C = out_of(C[q]);
    ra.M = M;
    ra.N = N;
    ra.ldc = ldc;
    ra.Mp = w.Mp;
    ra.Np = w.Np;
    ra.prec = prec;
    ra.xrman = av[q].rman;
    ra.xrexp = av[q].rexp;
    LaunchScope sc(ctx, s, "block_round", M * N * (int64_t)NM * (2 * ct.NMW));
    launch_block_round(ctx, ra, s);
  }
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

// The omission for eq. 2 under p3's shared lines (E_0, E_1 already at w.etop): the thresholds,
// the truncated shared bottoms, each part's radius lines carrying the thresholds (rows_o[q],
// cols_o[q]) and hst_o (hst with the truncated parts' radius flags).  *po is planned as one block
// when the truncated shared heights fit h and the tensor-core residue kernel takes them (one
// statistics read-back); otherwise po->ok stays false.
static arbgpu_status omit_eq2(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws, const Plan3M &p3,
                              const Lines *rowsL, const Lines *colsL, const BlockStats *hst,
                              int64_t M, int64_t K, int64_t N, int prec, cudaStream_t s,
                              Plan3M *po, Lines *rows_o, Lines *cols_o, BlockStats *hst_o) {
  *po = Plan3M{};
  const int64_t off = (int64_t)prec + bit_length(K) + 9;
  const int64_t *E0 = (const int64_t *)(ws + w.etop[0]), *E1 = (const int64_t *)(ws + w.etop[1]);
  int64_t *rb = (int64_t *)(ws + w.om_rbot), *rt = (int64_t *)(ws + w.om_rtrunc);
  int64_t *rr[2] = {(int64_t *)(ws + w.om_rrad), (int64_t *)(ws + w.e2rrad)};
  int64_t *cb = (int64_t *)(ws + w.om_cbot), *ct = (int64_t *)(ws + w.om_ctrunc);
  int64_t *cr[2] = {(int64_t *)(ws + w.om_crad), (int64_t *)(ws + w.e2crad)};
  int64_t *cp[2] = {(int64_t *)(ws + w.om_cplus), (int64_t *)(ws + w.e2cplus)};
  BlockStats *st = (BlockStats *)(ws + w.e2mstats);  // [3]: shared heights, part 0, part 1
  if (cudaMemsetAsync(st, 0, 3 * sizeof(BlockStats), s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  {
    LaunchScope sc(ctx, s, "omission", M * N);
    omission_eq2_rows_kernel<<<(unsigned)((M + 7) / 8), 256, 0, s>>>(
        E0, E1, M, N, p3.rtop, p3.rbot, p3.ctop, rowsL[0].rtop, rowsL[1].rtop, rowsL[0].rrad,
        rowsL[1].rrad, off, rb, rt, rr[0], rr[1], st);
    omission_eq2_cols_kernel<<<(unsigned)((N + 31) / 32), 256, 0, s>>>(
        E0, E1, M, N, p3.rtop, p3.ctop, p3.cbot, colsL[0].ctop, colsL[1].ctop, colsL[0].crad,
        colsL[1].crad, off, cb, ct, cr[0], cr[1], cp[0], cp[1], st);
    if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  }
  BlockStats os[3];
  const arbgpu_status rs = read_stats(ctx, st, os, 3, s);
  if (rs != ARBGPU_OK) return rs;
  BlockStats hs{};
  hs.pA = hst[0].pA > hst[1].pA ? hst[0].pA : hst[1].pA;
  hs.pB = hst[2].pB > hst[3].pB ? hst[2].pB : hst[3].pB;
  const int64_t h = height_bound(prec, hs);
  if (os[0].hA > h || os[0].hB > h) return ARBGPU_OK;
  Plan3M &p = *po;
  p.hA = os[0].hA;
  p.hB = os[0].hB;
  p.NM = crt_moduli_for_bits((int)((p.hA > 0 ? p.hA : 0) + (p.hB > 0 ? p.hB : 0) +
                                   bit_length(K) + 3));
  if (p.NM > w.NMmax) return ARBGPU_OK;
  p.plan = crt_plan(p.NM);
  if (!p.plan || p.plan->NMW + 1 > RD_MAXW) return ARBGPU_OK;
  p.nch = (int)(((p.hA > p.hB ? p.hA : p.hB) + 2 + 31) / 32) + 1;
  if (!residue_tc_layout(p.nch, p.NM, false, (M > N ? M : N) * w.Kp, &p.L)) return ARBGPU_OK;
  p.rtop = p3.rtop;
  p.rbot = rb;
  p.ctop = p3.ctop;
  p.cbot = cb;
  for (int q = 0; q < 2; ++q) {
    rows_o[q] = Lines{rowsL[q].rtop, rowsL[q].rbot, rr[q], nullptr, nullptr, nullptr, nullptr,
                      rt, nullptr};
    cols_o[q] = Lines{nullptr, nullptr, nullptr, colsL[q].ctop, colsL[q].cbot, cr[q], cp[q],
                      nullptr, ct};
    hst_o[q] = hst[q];
    hst_o[q].radA = os[1 + q].radA;
    hst_o[2 + q] = hst[2 + q];
    hst_o[2 + q].radB = os[1 + q].radB;
  }
  p.ok = true;
  return ARBGPU_OK;
}

// accumulate_product over the inner order (see "inner ordering" above): the order and scaling
// from the per-index tops, reordered and scaled copies of X and Y, then the same greedy blocks,
// products and basecase dots; basecase indices are reported in X's and Y's own numbering.
static arbgpu_status accumulate_product_ordered(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws,
                                                const BallsView &Xv, const BallsView &Yv,
                                                int64_t M, int64_t K, int64_t N, int64_t ldx,
                                                int64_t ldy, int prec, const Lines &full,
                                                const BlockStats &hs, bool negate, int combo,
                                                const AccView &av, cudaStream_t s,
                                                std::vector<int32_t> &basek,
                                                const DirectRound *direct, bool *rounded,
                                                const std::function<arbgpu_status()> *prepare) {
  if (Xv.nlimbs > BL_MAX_NL || Yv.nlimbs > BL_MAX_NL) return ARBGPU_ERR_LIMIT;
  int64_t *tA = (int64_t *)(ws + w.tA), *bA = (int64_t *)(ws + w.bA);
  int64_t *tBT = (int64_t *)(ws + w.tB), *bBT = (int64_t *)(ws + w.bB);
  int64_t *da = (int64_t *)(ws + w.ia), *db = (int64_t *)(ws + w.ib);
  const arbgpu_status est = entry_tops(ctx, Xv, Yv, M, K, N, ldx, ldy, tA, bA, tBT, bBT, s);
  if (est != ARBGPU_OK) return est;
  {
    // a_k = largest top of column k of X, b_k = largest top of row k of Y
    LaunchScope sc(ctx, s, "inner_tops", M * K + K * N);
    colmax_kernel<<<(unsigned)((K + 31) / 32), 256, 0, s>>>(tA, M, K, da);
    colmax_kernel<<<(unsigned)((K + 31) / 32), 256, 0, s>>>(tBT, N, K, db);
  }
  std::vector<int64_t> a((size_t)K), b((size_t)K), g;
  std::vector<int32_t> ord;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(a.data(), da, 8 * (size_t)K, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(b.data(), db, 8 * (size_t)K, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  inner_order_host(a, b, ord, g);
  int32_t *dord = (int32_t *)(ws + w.iord);
  int64_t *dg = (int64_t *)(ws + w.ig);
  if (cudaMemcpyAsync(dord, ord.data(), 4 * (size_t)K, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(dg, g.data(), 8 * (size_t)K, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  const BallsOut oX = ball_array_at(ws + w.oA, M * K, Xv.nlimbs);
  const BallsOut oY = ball_array_at(ws + w.oB, K * N, Yv.nlimbs);
  int *drange = (int *)(ws + w.irange);
  int hrange = 0;
  if (cudaMemsetAsync(drange, 0, 4, s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  {
    LaunchScope sc(ctx, s, "gather_inner", M * K + K * N);
    gather_inner_kernel<<<(unsigned)((M * K + 255) / 256), 256, 0, s>>>(Xv, ldx, false, M, K, N,
                                                                        dord, dg, oX, drange);
    gather_inner_kernel<<<(unsigned)((K * N + 255) / 256), 256, 0, s>>>(Yv, ldy, true, M, K, N,
                                                                        dord, dg, oY, drange);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hrange, drange, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
  }
  if (hrange)  // a scaled exponent would leave the fast path's range: keep the original order
    return accumulate_product(ctx, w, ws, Xv, Yv, M, K, N, ldx, ldy, prec, full, hs, negate,
                              combo, av, s, basek, nullptr, nullptr, nullptr, prepare);
  const BallsView Xo{oX.limbs, oX.stride, oX.nlimbs, oX.exp, oX.flags, oX.rad_man, oX.rad_exp};
  const BallsView Yo{oY.limbs, oY.stride, oY.nlimbs, oY.exp, oY.flags, oY.rad_man, oY.rad_exp};
  // (`ord` and `g` stay alive until this returns: accumulate_product synchronises the stream)
  const size_t rec = ctx->plan_log.size();
  const arbgpu_status st = accumulate_product(ctx, w, ws, Xo, Yo, M, K, N, K, N, prec, full, hs,
                                              negate, combo, av, s, basek, &ord, direct, rounded,
                                              prepare);
  if (cudaStreamSynchronize(s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  if (st == ARBGPU_OK && rec < ctx->plan_log.size()) {
    // the record covers positions of the order: mark it and append the order and the scaling
    ctx->plan_log[rec] = 1;
    for (int64_t k = 0; k < K; ++k) ctx->plan_log.push_back(ord[(size_t)k]);
    for (int64_t k = 0; k < K; ++k) ctx->plan_log.push_back(g[(size_t)k]);
  }
  return st;
}

// ---- eq. 2 over several blocks (Section IV-C's second suggestion: one splitting of the inner
// range planned for the real and imaginary parts together).  The greedy extraction of Section
// IV-A runs on entries whose top is the larger and whose bottom the smaller of the two parts'
// (entry_tops with merge), so each full block admits one scaling per row of A and per column of
// B shared by both parts: the per-block scans of each part, merged line by line
// (merge_parts_kernel, one CTA per block).  Under it X_re + X_im and Y_re + Y_im are integers and
// the block's Re and Im come from three exact products (eq2_products).  Each part's exact block
// value goes into that part's window accumulator (one addition per block), and its radius bound
// comes from the part's two real radius products over the block; basecase blocks become
// complex dot products (both real products of each part, with the accumulated blocks as their
// initial term).  kmap: the caller's inner index of each position (inner order), or null.
// *done = false on return means nothing was accumulated (a block the tensor-core residue kernel
// cannot take): the caller then runs four real products.
static arbgpu_status accumulate_eq2(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws,
                                    const BallsView *Xv, const BallsView *Yv, int64_t M,
                                    int64_t K, int64_t N, int64_t ldx, int64_t ldy, int prec,
                                    const BlockStats *hst, const AccView *av, cudaStream_t s,
                                    std::vector<int32_t> *basek, const std::vector<int32_t> *kmap,
                                    const std::function<arbgpu_status()> &prepare, bool *done) {
  *done = false;
  BlockStats hs{};
  hs.pA = hst[0].pA > hst[1].pA ? hst[0].pA : hst[1].pA;
  hs.pB = hst[2].pB > hst[3].pB ? hst[2].pB : hst[3].pB;
  const int64_t h = height_bound(prec, hs);
  int64_t *tA = (int64_t *)(ws + w.tA), *bA = (int64_t *)(ws + w.bA);
  int64_t *tBT = (int64_t *)(ws + w.tB), *bBT = (int64_t *)(ws + w.bB);
  for (int q = 0; q < 2; ++q) {
    const arbgpu_status est =
        entry_tops(ctx, Xv[q], Yv[q], M, K, N, ldx, ldy, tA, bA, tBT, bBT, s, q == 1);
    if (est != ARBGPU_OK) return est;
  }
  std::vector<int32_t> hb;
  const arbgpu_status pst = plan_blocks(ctx, w, ws, M, K, N, h, s, hb);
  if (pst != ARBGPU_OK) return pst;
  const int nb = (int)(hb.size() / 3);
  const int32_t *blocks = (const int32_t *)(ws + w.blocks);
  // per-block lines: part 0 in the b* arrays, part 1 in the e2* arrays, shared in e2s*
  int64_t *L0[7] = {(int64_t *)(ws + w.brtop), (int64_t *)(ws + w.brbot),
                    (int64_t *)(ws + w.brrad), (int64_t *)(ws + w.bctop),
                    (int64_t *)(ws + w.bcbot), (int64_t *)(ws + w.bcrad),
                    (int64_t *)(ws + w.bcplus)};
  int64_t *L1[7] = {(int64_t *)(ws + w.e2rtop), (int64_t *)(ws + w.e2rbot),
                    (int64_t *)(ws + w.e2rrad), (int64_t *)(ws + w.e2ctop),
                    (int64_t *)(ws + w.e2cbot), (int64_t *)(ws + w.e2crad),
                    (int64_t *)(ws + w.e2cplus)};
  int64_t *srtop = (int64_t *)(ws + w.e2srtop), *srbot = (int64_t *)(ws + w.e2srbot);
  int64_t *sctop = (int64_t *)(ws + w.e2sctop), *scbot = (int64_t *)(ws + w.e2scbot);
  BlockStats *bst[2] = {(BlockStats *)(ws + w.bstats), (BlockStats *)(ws + w.e2stats)};
  BlockStats *mst = (BlockStats *)(ws + w.e2mstats);
  BlockStats init{};
  init.hA = init.hB = INT64_MIN;
  std::vector<BlockStats> hbs[2], hms((size_t)nb);
  for (int q = 0; q < 2; ++q) {
    hbs[q].assign((size_t)nb, init);
    if (cudaMemcpyAsync(bst[q], hbs[q].data(), sizeof(BlockStats) * nb, cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
    int64_t *const *L = q ? L1 : L0;
    const arbgpu_status sst = run_scans(ctx, s, Xv[q], M, K, ldx, Yv[q], N, ldy, blocks, nb, K,
                                        L[0], L[1], L[2], L[3], L[4], L[5], L[6], bst[q], bst[q]);
    if (sst != ARBGPU_OK) return sst;
  }
  {
    LaunchScope sc(ctx, s, "merge_parts", (M + N) * nb);
    merge_parts_kernel<<<(unsigned)nb, 1024, 0, s>>>(L0[0], L0[1], L1[0], L1[1], M, srtop, srbot,
                                                     L0[3], L0[4], L1[3], L1[4], N, sctop, scbot,
                                                     mst);
  }
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(hbs[0].data(), bst[0], sizeof(BlockStats) * nb, cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(hbs[1].data(), bst[1], sizeof(BlockStats) * nb, cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(hms.data(), mst, sizeof(BlockStats) * nb, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  // every full block with a nonzero midpoint product must fit the tensor-core residue kernel
  struct BlockPlan {
    int NM, nch;
    const CrtPlan *plan;
    RtLayout L;
  };
  std::vector<BlockPlan> bp((size_t)nb);
  for (int b = 0; b < nb; ++b) {
    bp[b] = BlockPlan{0, 0, nullptr, {}};
    const int64_t hA = hms[b].hA, hB = hms[b].hB;
    if (hb[3 * b + 2] || hA == INT64_MIN || hB == INT64_MIN) continue;
    const int64_t kc = hb[3 * b + 1] - hb[3 * b], Kpb = (kc + TG_BK - 1) / TG_BK * TG_BK;
    BlockPlan &q = bp[b];
    q.NM = crt_moduli_for_bits((int)(hA + hB + bit_length(kc) + 3));
    if (q.NM > w.NMmax) return ARBGPU_OK;
    q.plan = crt_plan(q.NM);
    if (!q.plan || q.plan->NMW + 1 > RD_MAXW) return ARBGPU_OK;
    q.nch = (int)(((hA > hB ? hA : hB) + 2 + 31) / 32) + 1;
    if (!residue_tc_layout(q.nch, q.NM, false, (M > N ? M : N) * Kpb, &q.L)) return ARBGPU_OK;
  }
  *done = true;
  log_plan(ctx, 2, h, K, hb);
  const arbgpu_status prs = prepare();  // the accumulators' window bounds
  if (prs != ARBGPU_OK) return prs;
  const int64_t plane = w.Mp * w.Np;
  for (int b = 0; b < nb; ++b) {
    const int64_t k0 = hb[3 * b], k1 = hb[3 * b + 1];
    if (hb[3 * b + 2]) {
      // both real products of each part over these indices (combos as in the four-product path)
      for (int64_t k = k0; k < k1; ++k) {
        const int32_t kk = (int32_t)((kmap ? (int64_t)(*kmap)[k] : k) << 2);
        basek[0].push_back(kk | 0);
        basek[0].push_back(kk | 1);
        basek[1].push_back(kk | 2);
        basek[1].push_back(kk | 3);
      }
      continue;
    }
    const int64_t oM = (int64_t)b * M, oN = (int64_t)b * N;
    const Lines pl[2] = {Lines{L0[0] + oM, L0[1] + oM, L0[2] + oM, L0[3] + oN, L0[4] + oN,
                               L0[5] + oN, L0[6] + oN},
                         Lines{L1[0] + oM, L1[1] + oM, L1[2] + oM, L1[3] + oN, L1[4] + oN,
                               L1[5] + oN, L1[6] + oN}};
    if (bp[b].plan) {
      uint16_t *z = nullptr;
      CrtTables ct{};
      const arbgpu_status st =
          eq2_products(ctx, w, ws, bp[b].NM, bp[b].plan, bp[b].nch, bp[b].L, Xv, Yv, M, N, ldx,
                       ldy, k0, k1 - k0, srtop + oM, srbot + oM, sctop + oN, scbot + oN, pl, s,
                       &z, &ct);
      if (st != ARBGPU_OK) return st;
      for (int q = 0; q < 2; ++q) {
        RoundArgs ra{};
        ra.mid = IntProduct{(const uint8_t *)(z + (size_t)q * bp[b].NM * plane), nullptr, 3, 1,
                            {}, 1, ct};
        ra.mid.ends.e[0] = 3;
        ra.rtop = srtop + oM;
        ra.rbot = srbot + oM;
        ra.rrad = pl[q].rrad;
        ra.ctop = sctop + oN;
        ra.cbot = scbot + oN;
        ra.crad = pl[q].crad;
        ra.cplus = pl[q].cplus;
        ra.M = M;
        ra.N = N;
        ra.Mp = w.Mp;
        ra.Np = w.Np;
        ra.prec = prec;
        ra.acc = av[q];
        LaunchScope sc(ctx, s, "accumulate", M * N);
        arbgpu_status tst = ARBGPU_OK;
        if (launch_crt_round_tc(ctx, ra, s, &tst, true)) {
          if (tst != ARBGPU_OK) return tst;
          continue;
        }
        AccArgs aa{};
        aa.mid = ra.mid;
        aa.rtop = ra.rtop;
        aa.rbot = ra.rbot;
        aa.rrad = ra.rrad;
        aa.ctop = ra.ctop;
        aa.cbot = ra.cbot;
        aa.crad = ra.crad;
        aa.cplus = ra.cplus;
        aa.v = av[q];
        aa.M = M;
        aa.N = N;
        aa.Mp = w.Mp;
        aa.Np = w.Np;
        aa.skip_rad = 1;
        accumulate_kernel<<<(unsigned)((M * N + 127) / 128), 128, 0, s>>>(aa);
      }
    }
    // radii: Re from X_re Y_re and X_im Y_im, Im from X_re Y_im and X_im Y_re, over this block
    const int pairs[4][3] = {{0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
    for (const auto &pr : pairs) {
      const int part = pr[0], xa = pr[1], yb = pr[2];
      const bool radA = hbs[xa][b].radA != 0, radB = hbs[yb][b].radB != 0;
      if (!radA && !radB) continue;
      const Lines ln{pl[xa].rtop, pl[xa].rbot, pl[xa].rrad, pl[yb].ctop,
                     pl[yb].cbot, pl[yb].crad, pl[yb].cplus};
      AccArgs aa{};
      const arbgpu_status st = run_radius(ctx, w, ws, Xv[xa], Yv[yb], M, N, ldx, ldy, k0,
                                          k1 - k0, radA, radB, ln, s, &aa.rp1, &aa.rp2);
      if (st != ARBGPU_OK) return st;
      aa.rtop = ln.rtop;
      aa.rbot = ln.rbot;
      aa.rrad = ln.rrad;
      aa.ctop = ln.ctop;
      aa.cbot = ln.cbot;
      aa.crad = ln.crad;
      aa.cplus = ln.cplus;
      aa.v = av[part];
      aa.M = M;
      aa.N = N;
      aa.Mp = w.Mp;
      aa.Np = w.Np;
      aa.skip_mid = 1;
      LaunchScope sc(ctx, s, "accumulate", M * N);
      accumulate_kernel<<<(unsigned)((M * N + 127) / 128), 128, 0, s>>>(aa);
    }
  }
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

// accumulate_eq2 over an inner order shared by the parts (the two suggestions of Sections IV-B and
// IV-C together): a_k = largest top over column k of both parts of A, b_k over row k of both parts
// of B, then the order and scaling of the real case (inner_order_host), reordered and scaled
// copies of all four operand parts, and accumulate_eq2 on the copies.  The plan record (kind 4)
// lists the order and the scaling after its blocks.
static arbgpu_status accumulate_eq2_ordered(arbgpu_ctx *ctx, const BlockWs &w, uint8_t *ws,
                                            const BallsView *Xv, const BallsView *Yv, int64_t M,
                                            int64_t K, int64_t N, int64_t ldx, int64_t ldy,
                                            int prec, const BlockStats *hst, const AccView *av,
                                            cudaStream_t s, std::vector<int32_t> *basek,
                                            const std::function<arbgpu_status()> &prepare,
                                            bool *done) {
  *done = false;
  for (int q = 0; q < 2; ++q)
    if (Xv[q].nlimbs > BL_MAX_NL || Yv[q].nlimbs > BL_MAX_NL) return ARBGPU_OK;
  int64_t *tA = (int64_t *)(ws + w.tA), *bA = (int64_t *)(ws + w.bA);
  int64_t *tBT = (int64_t *)(ws + w.tB), *bBT = (int64_t *)(ws + w.bB);
  int64_t *da = (int64_t *)(ws + w.ia), *db = (int64_t *)(ws + w.ib);
  for (int q = 0; q < 2; ++q) {
    const arbgpu_status est =
        entry_tops(ctx, Xv[q], Yv[q], M, K, N, ldx, ldy, tA, bA, tBT, bBT, s, q == 1);
    if (est != ARBGPU_OK) return est;
  }
  {
    LaunchScope sc(ctx, s, "inner_tops", M * K + K * N);
    colmax_kernel<<<(unsigned)((K + 31) / 32), 256, 0, s>>>(tA, M, K, da);
    colmax_kernel<<<(unsigned)((K + 31) / 32), 256, 0, s>>>(tBT, N, K, db);
  }
  std::vector<int64_t> a((size_t)K), b((size_t)K), g;
  std::vector<int32_t> ord;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(a.data(), da, 8 * (size_t)K, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(b.data(), db, 8 * (size_t)K, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  inner_order_host(a, b, ord, g);
  int32_t *dord = (int32_t *)(ws + w.iord);
  int64_t *dg = (int64_t *)(ws + w.ig);
  if (cudaMemcpyAsync(dord, ord.data(), 4 * (size_t)K, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(dg, g.data(), 8 * (size_t)K, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  BallsView Xo[2], Yo[2];
  int *drange = (int *)(ws + w.irange);
  int hrange = 0;
  if (cudaMemsetAsync(drange, 0, 4, s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  {
    LaunchScope sc(ctx, s, "gather_inner", 2 * (M * K + K * N));
    for (int q = 0; q < 2; ++q) {
      const BallsOut oX = ball_array_at(ws + (q ? w.oA2 : w.oA), M * K, Xv[q].nlimbs);
      const BallsOut oY = ball_array_at(ws + (q ? w.oB2 : w.oB), K * N, Yv[q].nlimbs);
      gather_inner_kernel<<<(unsigned)((M * K + 255) / 256), 256, 0, s>>>(Xv[q], ldx, false, M,
                                                                          K, N, dord, dg, oX,
                                                                          drange);
      gather_inner_kernel<<<(unsigned)((K * N + 255) / 256), 256, 0, s>>>(Yv[q], ldy, true, M,
                                                                          K, N, dord, dg, oY,
                                                                          drange);
      Xo[q] = BallsView{oX.limbs, oX.stride, oX.nlimbs, oX.exp, oX.flags, oX.rad_man, oX.rad_exp};
      Yo[q] = BallsView{oY.limbs, oY.stride, oY.nlimbs, oY.exp, oY.flags, oY.rad_man, oY.rad_exp};
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hrange, drange, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
  }
  if (hrange)  // a scaled exponent would leave the fast path's range: keep the original order
    return accumulate_eq2(ctx, w, ws, Xv, Yv, M, K, N, ldx, ldy, prec, hst, av, s, basek,
                          nullptr, prepare, done);
  const size_t rec = ctx->plan_log.size();
  const arbgpu_status st = accumulate_eq2(ctx, w, ws, Xo, Yo, M, K, N, K, N, prec, hst, av, s,
                                          basek, &ord, prepare, done);
  if (cudaStreamSynchronize(s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  if (st == ARBGPU_OK && *done && rec < ctx->plan_log.size()) {
    ctx->plan_log[rec] = 4;
    for (int64_t k = 0; k < K; ++k) ctx->plan_log.push_back(ord[(size_t)k]);
    for (int64_t k = 0; k < K; ++k) ctx->plan_log.push_back(g[(size_t)k]);
  }
  return st;
}

// Ball matrix product by Algorithm 2 (real, or complex by four real products, Section IV-C).
// Returns ARBGPU_ERR_LIMIT when the inputs hold special values or exceed the path's limits (the
// caller then uses the classical algorithm).
// The whole-range scans of a product: line arrays of each part and the four BlockStats (rows of
// A0, A1, columns of B0, B1), at pointers the caller lays out (`scan_region_at`).
struct ScanRegion {
  int64_t *rtop[2], *rbot[2], *rrad[2];
  int64_t *ctop[2], *cbot[2], *crad[2], *cplus[2];
  BlockStats *pst;  // [4]
};

static_assert(sizeof(BlockStats) * 4 + 2 * sizeof(unsigned) <= 256,
              "the stats and the finished-CTA counters share the scan region's first 256 bytes");

size_t block_scan_bytes(int64_t M, int64_t N, bool cplx) {
  const int parts = cplx ? 2 : 1;
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  return al(sizeof(BlockStats) * 4) + parts * (3 * al(8 * (size_t)M) + 4 * al(8 * (size_t)N));
}

static ScanRegion scan_region_at(uint8_t *base, int64_t M, int64_t N, bool cplx) {
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  ScanRegion r{};
  size_t off = 0;
  auto take = [&](size_t n) {
    uint8_t *p = base + off;
    off += al(n);
    return p;
  };
  r.pst = (BlockStats *)take(sizeof(BlockStats) * 4);
  for (int q = 0; q < (cplx ? 2 : 1); ++q) {
    r.rtop[q] = (int64_t *)take(8 * (size_t)M);
    r.rbot[q] = (int64_t *)take(8 * (size_t)M);
    r.rrad[q] = (int64_t *)take(8 * (size_t)M);
    r.ctop[q] = (int64_t *)take(8 * (size_t)N);
    r.cbot[q] = (int64_t *)take(8 * (size_t)N);
    r.crad[q] = (int64_t *)take(8 * (size_t)N);
    r.cplus[q] = (int64_t *)take(8 * (size_t)N);
  }
  return r;
}

// The larger limb count of an operand's parts.
static int operand_limbs(const arbgpu_balls *X, bool cplx) {
  int nl = X[0].nlimbs;
  if (cplx && X[1].nlimbs > nl) nl = X[1].nlimbs;
  return nl;
}

// Whether the block path takes the product at all (otherwise: ARBGPU_ERR_LIMIT, dot products).
static bool block_accepts(const arbgpu_balls *A, const arbgpu_balls *B, int64_t K, bool cplx) {
  for (int q = 0; q < (cplx ? 2 : 1); ++q)
    if (A[q].nlimbs > BL_MAX_NL || B[q].nlimbs > BL_MAX_NL) return false;
  return K >= BL_BASECASE;
}

// Phase 1: the whole-range scans (two launches per part); the stats start at zero (a height
// of 0 and no flags is the identity of every field).
arbgpu_status block_scan_launch(arbgpu_ctx *ctx, const arbgpu_balls *A, const arbgpu_balls *B,
                                int64_t M, int64_t K, int64_t N, int64_t lda, int64_t ldb,
                                bool cplx, void *region, BlockStats *stats, cudaStream_t s) {
  if (!block_accepts(A, B, K, cplx)) return ARBGPU_ERR_LIMIT;
  ScanRegion sr = scan_region_at((uint8_t *)region, M, N, cplx);
  // without a caller's stats array: the four BlockStats and the finished-CTA counters (in the
  // region's first 256 bytes) start at zero, and the last launch publishes the statistics to the
  // context's mapped words under a new sequence number (block_wait_stats)
  unsigned *done = (unsigned *)(sr.pst + 4);
  if (stats)
    sr.pst = stats;  // zeroed by the caller
  else if (cudaMemsetAsync(sr.pst, 0, 256, s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  const int parts = cplx ? 2 : 1;
  for (int q = 0; q < parts; ++q) {
    StatsPublish pub{};
    if (!stats && q == parts - 1) {
      pub = StatsPublish{sr.pst, 4, (uint32_t *)ctx->pub_dev, done + q, ++ctx->pub_seq};
      if (pub.seq == 0) pub.seq = ++ctx->pub_seq;  // (0 is the words' initial value)
    }
    LaunchScope sc(ctx, s, "scans", M * K + K * N);
    scan_full_kernel<<<(unsigned)((M + 7) / 8 + (N + 7) / 8), 1024, 0, s>>>(
        view_of(A[q]), view_of(B[q]), M, K, N, lda, ldb, sr.rtop[q], sr.rbot[q], sr.rrad[q],
        sr.pst + q, sr.ctop[q], sr.cbot[q], sr.crad[q], sr.cplus[q], sr.pst + 2 + q, pub);
    if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  }
  return ARBGPU_OK;
}

// Waits for the statistics that the last block_scan_launch without a stats array publishes
// (sequence number ctx->pub_seq) and copies the four BlockStats to `host`: a poll of the mapped
// sequence word, which answers as soon as the scan's last CTA has written it, where a stream
// synchronisation would also wait for the host to be woken.  Gives up after about 20 s, and
// reports a stream that has failed, or has finished without publishing.
arbgpu_status block_wait_stats(arbgpu_ctx *ctx, BlockStats *host, cudaStream_t s) {
  const volatile uint32_t *words = (const volatile uint32_t *)ctx->pub;
  const int nw = 4 * (int)(sizeof(BlockStats) / 4);
  const auto t0 = std::chrono::steady_clock::now();
  for (int64_t it = 0;; ++it) {
    if (words[nw] == ctx->pub_seq) break;
    if ((it & 1023) == 1023) {
      const cudaError_t q = cudaStreamQuery(s);
      if (q != cudaSuccess && q != cudaErrorNotReady) return ARBGPU_ERR_CUDA;
      if (q == cudaSuccess && words[nw] != ctx->pub_seq) return ARBGPU_ERR_CUDA;
      const double el =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > 20.0) return ARBGPU_ERR_TIMEOUT;
      if (el > 1e-3) std::this_thread::yield();
    }
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  memcpy(host, (const void *)ctx->pub, sizeof(BlockStats) * 4);
  return ARBGPU_OK;
}

// Phase 2: the products and the rounding, from the scan results (`region`, and their host copy
// `hst`, read after the scans finished) and the block workspace.
arbgpu_status block_finish(arbgpu_ctx *ctx, const arbgpu_balls *C, const arbgpu_balls *A,
                           const arbgpu_balls *B, int64_t M, int64_t K, int64_t N, int64_t lda,
                           int64_t ldb, int64_t ldc, int prec, bool cplx, bool m3, void *region,
                           const BlockStats *hst, void *workspace, size_t ws_bytes,
                           cudaStream_t s, bool *used_block) {
  *used_block = false;
  const int parts = cplx ? 2 : 1;
  BlockWs w = block_ws(ctx, M, K, N, prec, cplx, m3, operand_limbs(A, cplx),
                       operand_limbs(B, cplx));
  if (!workspace || ws_bytes < w.total) return ARBGPU_ERR_WORKSPACE;
  uint8_t *ws = (uint8_t *)workspace;
  const ScanRegion sr = scan_region_at((uint8_t *)region, M, N, cplx);
  BallsView Av[2], Bv[2];
  Lines rowsL[2], colsL[2];
  for (int q = 0; q < parts; ++q) {
    Av[q] = view_of(A[q]);
    Bv[q] = view_of(B[q]);
    rowsL[q] = Lines{sr.rtop[q], sr.rbot[q], sr.rrad[q], nullptr, nullptr, nullptr, nullptr};
    colsL[q] = Lines{nullptr, nullptr, nullptr, sr.ctop[q], sr.cbot[q], sr.crad[q], sr.cplus[q]};
  }
  for (int q = 0; q < parts; ++q)
    if (hst[q].special || hst[2 + q].special) return ARBGPU_ERR_LIMIT;
  auto lines_of = [&](int xa, int yb) {
    return Lines{rowsL[xa].rtop, rowsL[xa].rbot, rowsL[xa].rrad, colsL[yb].ctop,
                 colsL[yb].cbot, colsL[yb].crad, colsL[yb].cplus};
  };

  // the operands' tops relative to their lines (rel_tops_kernel), once per operand part per call:
  // the max-plus bound of the accumulator's window and the negligible-limb omission use them
  // (with a `wide` flag per operand part, zeroed before the first of them: the max-plus kernel
  // they feed runs on 16-bit halves unless a flag is set)
  bool rel_done[4] = {false, false, false, false};  // A0, A1, B0, B1
  int *wide = (int *)(ws + w.relwide);
  auto wide_of = [&](int q) -> const int * { return wide + q; };
  auto ensure_rel = [&](int xa, int yb) -> arbgpu_status {
    if (!rel_done[0] && !rel_done[1] && !rel_done[2] && !rel_done[3] &&
        cudaMemsetAsync(wide, 0, 4 * sizeof(int), s) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
    if (!rel_done[xa]) {
      LaunchScope sc(ctx, s, "rel_tops", M * K);
      rel_tops_kernel<<<(unsigned)((M * K + 255) / 256), 256, 0, s>>>(
          Av[xa], lda, M, K, rowsL[xa].rtop, true, (int32_t *)(ws + w.relA[xa]), wide + xa);
      rel_done[xa] = true;
    }
    if (!rel_done[2 + yb]) {
      LaunchScope sc(ctx, s, "rel_tops", K * N);
      rel_tops_kernel<<<(unsigned)((K * N + 255) / 256), 256, 0, s>>>(
          Bv[yb], ldb, K, N, colsL[yb].ctop, false, (int32_t *)(ws + w.relB[yb]), wide + 2 + yb);
      rel_done[2 + yb] = true;
    }
    return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
  };
  // The max-plus bound E_t of real product t (A_xa B_yb; t as in the product lists below),
  // computed once per call: the omission's thresholds and the window bound of the product's
  // output part both read it.
  bool e_done[4] = {false, false, false, false};
  auto E_of = [&](int t) { return (int64_t *)(ws + w.eprod) + (size_t)t * M * N; };
  auto ensure_E = [&](int t, int xa, int yb) -> arbgpu_status {
    if (e_done[t]) return ARBGPU_OK;
    const arbgpu_status rs = ensure_rel(xa, yb);
    if (rs != ARBGPU_OK) return rs;
    launch_maxplus(ctx, s, (const int32_t *)(ws + w.relA[xa]), (const int32_t *)(ws + w.relB[yb]),
                   wide_of(xa), wide_of(2 + yb), rowsL[xa].rtop, colsL[yb].ctop, M, K, N,
                   E_of(t), 1);
    e_done[t] = true;
    return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
  };

  if (!cplx) {
    const BlockStats hs = merge_stats(hst[0], hst[2]);
    const int64_t h = height_bound(prec, hs);
    const bool one = hs.hA <= h && hs.hB <= h;
    if (omission_wanted(prec, K, hs, one)) {
      // ---- negligible limbs omitted: one block of the truncated operands, rounded once
      arbgpu_status so = ensure_E(0, 0, 0);
      if (so != ARBGPU_OK) return so;
      Omitted om{};
      so = omit_product(ctx, w, ws, E_of(0), M, K, N, prec, lines_of(0, 0), hs, s, &om);
      if (so != ARBGPU_OK) return so;
      if (om.ok) {
        RoundArgs ra{};
        so = run_block(ctx, w, ws, Av[0], Bv[0], M, N, lda, ldb, 0, K, om.hs.hA, om.hs.hB,
                       om.hs.radA != 0, om.hs.radB != 0, om.lines, s, &ra.mid, &ra.rp1, &ra.rp2);
        if (so != ARBGPU_OK) return so;
        log_plan(ctx, 3, h, K, {0, (int32_t)K, 0});
        const Lines &ln = om.lines;
        ra.rtop = ln.rtop;
        ra.rbot = ln.rbot;
        ra.rrad = ln.rrad;
        ra.ctop = ln.ctop;
        ra.cbot = ln.cbot;
        ra.crad = ln.crad;
        ra.cplus = ln.cplus;
        ra.C = out_of(C[0]);
        ra.M = M;
        ra.N = N;
        ra.ldc = ldc;
        ra.Mp = w.Mp;
        ra.Np = w.Np;
        ra.prec = prec;
        {
          const int64_t units =
              ra.mid.kind == 1 ? M * N * ra.mid.crt.NM * (int64_t)(2 * ra.mid.crt.NMW) : M * N;
          LaunchScope sc(ctx, s, "block_round", units);
          launch_block_round(ctx, ra, s);
        }
        *used_block = true;
        return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
      }
    }
    if (one) {
      // ---- one block: exact product, one rounding per entry
      log_plan(ctx, 0, h, K, {0, (int32_t)K, 0});
      const Lines full = lines_of(0, 0);
      RoundArgs ra{};
      arbgpu_status st1 = run_block(ctx, w, ws, Av[0], Bv[0], M, N, lda, ldb, 0, K, hs.hA, hs.hB,
                                    hs.radA != 0, hs.radB != 0, full, s, &ra.mid, &ra.rp1,
                                    &ra.rp2);
      if (st1 != ARBGPU_OK) return st1;
      ra.rtop = full.rtop;
      ra.rbot = full.rbot;
      ra.rrad = full.rrad;
      ra.ctop = full.ctop;
      ra.cbot = full.cbot;
      ra.crad = full.crad;
      ra.cplus = full.cplus;
      ra.C = out_of(C[0]);
      ra.M = M;
      ra.N = N;
      ra.ldc = ldc;
      ra.Mp = w.Mp;
      ra.Np = w.Np;
      ra.prec = prec;
      {
        // work units: 32-bit multiply-adds of the CRT sums (multimodular), else entries
      const int64_t units =
          ra.mid.kind == 1 ? M * N * ra.mid.crt.NM * (int64_t)(2 * ra.mid.crt.NMW) : M * N;
      LaunchScope sc(ctx, s, "block_round", units);
        launch_block_round(ctx, ra, s);
      }
      *used_block = true;
      return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
    }
  }

  // complex by eq. 2 when the shared scaling of the parts fits one block
  Plan3M p3{};
  if (cplx && m3) {
    const arbgpu_status st = plan_3m(ctx, w, ws, rowsL, colsL, hst, M, K, N, prec, s, &p3);
    if (st != ARBGPU_OK) return st;
  }

  // ---- accumulate every real product into its output part, then finish each part
  // real: C = A B.  complex: Re C = Ar Br - Ai Bi, Im C = Ar Bi + Ai Br (four real products).
  struct Prod {
    int part, xa, yb, combo;
    bool neg;
  };
  const Prod real_prods[1] = {{0, 0, 0, 0, false}};
  const Prod cplx_prods[4] = {{0, 0, 0, 0, false}, {0, 1, 1, 1, true},
                              {1, 0, 1, 2, false}, {1, 1, 0, 3, false}};
  const Prod *prods = cplx ? cplx_prods : real_prods;
  const int nprods = cplx ? 4 : 1;
  const size_t MN = (size_t)M * N;
  AccView av[2];
  std::vector<int32_t> basek[2];
  for (int q = 0; q < parts; ++q) {
    av[q] = AccView{(uint64_t *)(ws + w.acc[q]), (uint32_t *)(ws + w.err[q]),
                    (uint32_t *)(ws + w.rman[q]), (int64_t *)(ws + w.rexp[q]), w.nacc,
                    bit_length(K) + (cplx ? 1 : 0), {nullptr, nullptr}, {nullptr, nullptr}};
    int np = 0;
    for (int t = 0; t < nprods; ++t)
      if (prods[t].part == q) {
        av[q].ftop_r[np] = rowsL[prods[t].xa].rtop;
        av[q].ftop_c[np] = colsL[prods[t].yb].ctop;
        ++np;
      }
    if (p3.ok) {  // both parts' products lie under the shared lines
      av[q].ftop_r[0] = p3.rtop;
      av[q].ftop_c[0] = p3.ctop;
      av[q].ftop_r[1] = av[q].ftop_c[1] = nullptr;
    }
    // (eq. 2 rounds the exact parts directly: only the radius sums are used)
    if ((!p3.ok && cudaMemsetAsync(av[q].acc, 0, 8 * (size_t)w.nacc * MN, s) != cudaSuccess) ||
        (!p3.ok && cudaMemsetAsync(av[q].err, 0, 4 * MN, s) != cudaSuccess) ||
        cudaMemsetAsync(av[q].rman, 0, 4 * MN, s) != cudaSuccess ||
        cudaMemsetAsync(av[q].rexp, 0, 8 * MN, s) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
  }
  // The window of each part's accumulator sits under the exact per-entry exponent bound, computed
  // once before the part's first accumulation (a real product rounded straight from one exact
  // block needs none).
  bool etop_done[2] = {false, false};
  auto etop_of = [&](int q) -> arbgpu_status {
    if (etop_done[q]) return ARBGPU_OK;
    etop_done[q] = true;
    int64_t *et = (int64_t *)(ws + w.etop[q]);
    const int64_t *src[2] = {nullptr, nullptr};
    int n = 0;
    for (int t = 0; t < nprods; ++t) {
      const Prod &pr = prods[t];
      if (pr.part != q) continue;
      const arbgpu_status rs = ensure_E(t, pr.xa, pr.yb);
      if (rs != ARBGPU_OK) return rs;
      src[n++] = E_of(t);
    }
    LaunchScope sc(ctx, s, "etop_max", M * N);
    etop_max_kernel<<<(unsigned)((M * N + 255) / 256), 256, 0, s>>>(src[0], src[1], et, M * N);
    return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
  };
  if (!p3.ok)
    for (int q = 0; q < parts; ++q) {
      av[q].etop = (int64_t *)(ws + w.etop[q]);
      av[q].ncols = N;
    }
  if (p3.ok) {
    const arbgpu_status st3 = run_3m(ctx, w, ws, p3, C, Av, Bv, rowsL, colsL, hst, M, K, N, lda,
                                     ldb, ldc, prec, av, s);
    if (st3 != ARBGPU_OK) return st3;
    *used_block = true;
    return ARBGPU_OK;
  }
  // eq. 2 after the negligible limbs of both parts were omitted under shared thresholds, when the
  // truncated parts fit one shared block: one rounding per part, as for the one-block case.  When
  // they do not, four real products, each with its own omission (per-product thresholds drop more
  // bits than thresholds shared by the parts), do less work than eq. 2 over several blocks; eq. 2
  // over several blocks runs when the omission is not wanted (or switched off).
  bool several_eq2 = p3.several;
  if (p3.several) {
    BlockStats hm{};
    hm.hA = p3.hA;
    hm.hB = p3.hB;
    if (omission_wanted(prec, K, hm, false)) {
      arbgpu_status so = etop_of(0);
      if (so == ARBGPU_OK) so = etop_of(1);
      if (so != ARBGPU_OK) return so;
      Plan3M po{};
      Lines ro[2], co[2];
      BlockStats ho[4];
      so = omit_eq2(ctx, w, ws, p3, rowsL, colsL, hst, M, K, N, prec, s, &po, ro, co, ho);
      if (so != ARBGPU_OK) return so;
      if (po.ok) {
        BlockStats hs{};
        hs.pA = hst[0].pA > hst[1].pA ? hst[0].pA : hst[1].pA;
        hs.pB = hst[2].pB > hst[3].pB ? hst[2].pB : hst[3].pB;
        log_plan(ctx, 5, height_bound(prec, hs), K, {0, (int32_t)K, 0});
        const arbgpu_status s3 = run_3m(ctx, w, ws, po, C, Av, Bv, ro, co, ho, M, K, N, lda,
                                        ldb, ldc, prec, av, s);
        if (s3 != ARBGPU_OK) return s3;
        *used_block = true;
        return ARBGPU_OK;
      }
      several_eq2 = false;
    }
  }
  // eq. 2 over several blocks shared by both parts (over their shared inner order when the
  // inner ordering is on)
  bool eq2 = false;
  if (several_eq2) {
    const std::function<arbgpu_status()> prep2 = [&etop_of]() {
      const arbgpu_status e0 = etop_of(0);
      return e0 != ARBGPU_OK ? e0 : etop_of(1);
    };
    const arbgpu_status se =
        w.oA2 ? accumulate_eq2_ordered(ctx, w, ws, Av, Bv, M, K, N, lda, ldb, prec, hst, av, s,
                                       basek, prep2, &eq2)
              : accumulate_eq2(ctx, w, ws, Av, Bv, M, K, N, lda, ldb, prec, hst, av, s, basek,
                               nullptr, prep2, &eq2);
    if (se != ARBGPU_OK) return se;
  }
  bool rounded[2] = {false, false};
  const DirectRound direct{out_of(C[0]), ldc};
  for (int t = 0; t < (eq2 ? 0 : nprods); ++t) {
    const Prod &pr = prods[t];
    const BlockStats hs = merge_stats(hst[pr.xa], hst[2 + pr.yb]);
    const int64_t hb = height_bound(prec, hs);
    const std::function<arbgpu_status()> prep = [&etop_of, q = pr.part]() { return etop_of(q); };
    if (cplx && omission_wanted(prec, K, hs, hs.hA <= hb && hs.hB <= hb)) {
      // negligible limbs omitted: when the truncated operands fit one block, that block is
      // accumulated (a real product tried this before reaching the loop)
      arbgpu_status so = ensure_E(t, pr.xa, pr.yb);
      if (so != ARBGPU_OK) return so;
      Omitted om{};
      so = omit_product(ctx, w, ws, E_of(t), M, K, N, prec, lines_of(pr.xa, pr.yb), hs, s, &om);
      if (so != ARBGPU_OK) return so;
      if (om.ok) {
        so = accumulate_product(ctx, w, ws, Av[pr.xa], Bv[pr.yb], M, K, N, lda, ldb, prec,
                                om.lines, om.hs, pr.neg, pr.combo, av[pr.part], s,
                                basek[pr.part], nullptr, nullptr, nullptr, &prep, 3);
        if (so != ARBGPU_OK) return so;
        continue;
      }
    }
    // several blocks: over the inner order when it is enabled (its workspace exists); a real
    // product whose inner order leaves one full block is rounded from it directly
    const bool ordered = w.oA && (hs.hA > hb || hs.hB > hb);
    arbgpu_status st1 =
        ordered ? accumulate_product_ordered(ctx, w, ws, Av[pr.xa], Bv[pr.yb], M, K, N, lda, ldb,
                                             prec, lines_of(pr.xa, pr.yb), hs, pr.neg, pr.combo,
                                             av[pr.part], s, basek[pr.part],
                                             cplx ? nullptr : &direct, &rounded[pr.part], &prep)
                : accumulate_product(ctx, w, ws, Av[pr.xa], Bv[pr.yb], M, K, N, lda, ldb, prec,
                                     lines_of(pr.xa, pr.yb), hs, pr.neg, pr.combo, av[pr.part], s,
                                     basek[pr.part], nullptr, nullptr, nullptr, &prep);
    if (st1 != ARBGPU_OK) return st1;
  }
  for (int q = 0; q < parts; ++q) {
    if (rounded[q]) continue;
    if (basek[q].empty()) {
      LaunchScope sc(ctx, s, "acc_round", M * N);
      acc_round_kernel<<<(unsigned)((M * N + 127) / 128), 128, 0, s>>>(av[q], out_of(C[q]), M, N,
                                                                       ldc, prec);
      continue;
    }
    // basecase blocks: dot products with the accumulated blocks as their initial term
    arbgpu_balls ib{};
    ib.limbs = (uint64_t *)(ws + w.ilimbs[q]);
    ib.limb_stride = (int64_t)MN;
    ib.nlimbs = w.nacc + 1;
    ib.exp = (int64_t *)(ws + w.iexp[q]);
    ib.flags = (uint32_t *)(ws + w.iflags[q]);
    ib.rad_man = (uint32_t *)(ws + w.irman[q]);
    ib.rad_exp = (int64_t *)(ws + w.irexp[q]);
    ib.count = (int64_t)MN;
    {
      LaunchScope sc(ctx, s, "acc_to_ball", M * N);
      acc_to_ball_kernel<<<(unsigned)((M * N + 127) / 128), 128, 0, s>>>(av[q], out_of(ib), M, N);
    }
    int32_t *bk = (int32_t *)(ws + w.bk[q]);
    if (cudaMemcpyAsync(bk, basek[q].data(), 4 * basek[q].size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return ARBGPU_ERR_CUDA;
    arbgpu_status st2 = launch_basecase_dot(ctx, C[q], A, B, cplx, ib, bk,
                                            (int64_t)basek[q].size(), M, N, lda, ldb, ldc, prec,
                                            s);
    if (st2 != ARBGPU_OK) return st2;
  }
  *used_block = true;
  // the host-side index lists must outlive their copies
  if (cudaStreamSynchronize(s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

// Ball matrix product by Algorithm 2 (real, or complex by four real products, Section IV-C):
// scans, one read-back of their statistics, then the products.  Returns ARBGPU_ERR_LIMIT when the
// inputs hold special values or exceed the path's limits (the caller then uses the classical
// algorithm).
__global__ void words_to_mapped_kernel(const uint32_t *src, uint32_t *dst, int words) {
  for (int q = threadIdx.x; q < words; q += blockDim.x) dst[q] = src[q];
}

arbgpu_status read_stats(arbgpu_ctx *ctx, const BlockStats *dev, BlockStats *host, size_t n,
                         cudaStream_t s) {
  const size_t bytes = n * sizeof(BlockStats);
  if (bytes > ctx->mapped_bytes) {
    if (ctx->mapped) cudaFreeHost(ctx->mapped);
    ctx->mapped = ctx->mapped_dev = nullptr;
    ctx->mapped_bytes = 0;
    const size_t want = bytes < 4096 ? 4096 : bytes;
    if (cudaHostAlloc(&ctx->mapped, want, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&ctx->mapped_dev, ctx->mapped, 0) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
    ctx->mapped_bytes = want;
  }
  {
    LaunchScope sc(ctx, s, "stats_read", (int64_t)n);
    words_to_mapped_kernel<<<1, 256, 0, s>>>((const uint32_t *)dev, (uint32_t *)ctx->mapped_dev,
                                             (int)(bytes / 4));
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  memcpy(host, ctx->mapped, bytes);
  return ARBGPU_OK;
}

arbgpu_status block_matmul(arbgpu_ctx *ctx, const arbgpu_balls *C, const arbgpu_balls *A,
                           const arbgpu_balls *B, int64_t M, int64_t K, int64_t N, int64_t lda,
                           int64_t ldb, int64_t ldc, int prec, bool cplx, bool m3,
                           void *workspace, size_t ws_bytes, cudaStream_t s, bool *used_block) {
  *used_block = false;
  if (!block_accepts(A, B, K, cplx)) return ARBGPU_ERR_LIMIT;
  BlockWs w = block_ws(ctx, M, K, N, prec, cplx, m3, operand_limbs(A, cplx),
                       operand_limbs(B, cplx));
  if (!workspace || ws_bytes < w.total) return ARBGPU_ERR_WORKSPACE;
  void *region = (uint8_t *)workspace + w.scan;
  arbgpu_status st = block_scan_launch(ctx, A, B, M, K, N, lda, ldb, cplx, region, nullptr, s);
  if (st != ARBGPU_OK) return st;
  BlockStats hst[4];
  st = block_wait_stats(ctx, hst, s);
  if (st != ARBGPU_OK) return st;
  return block_finish(ctx, C, A, B, M, K, N, lda, ldb, ldc, prec, cplx, m3, region, hst,
                      workspace, ws_bytes, s, used_block);
}

}  // namespace arbgpu
