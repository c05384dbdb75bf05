// arbgpu_int_mat_mul: exact product of signed multi-limb integer matrices on the tensor cores
// (the integer engine of the block algorithm, exposed on its own).
#include "internal.h"
#include "tc_gemm.cuh"

namespace arbgpu {

constexpr int IM_MAX_LIMBS = 32;

// Balanced base-256 digits of a two's-complement integer given as little-endian limbs.
// Writes S digits (S = 8 * nl + 1) as BF16 to dst[t * plane] for t < S.
__device__ __forceinline__ void balanced_digits_twos(const uint64_t *limb_at, int64_t limb_stride,
                                                     int nl, int S, __nv_bfloat16 *dst,
                                                     int64_t plane) {
  const bool neg = (limb_at[(int64_t)(nl - 1) * limb_stride] >> 63) != 0;
  int carry = 0;
  uint64_t w = 0;
  for (int t = 0; t < S; ++t) {
    if ((t & 7) == 0) {
      const int k = t >> 3;
      w = k < nl ? limb_at[(int64_t)k * limb_stride] : (neg ? ~(uint64_t)0 : 0);
    }
    int v = (int)((w >> (8 * (t & 7))) & 255u) + carry;
    if (v >= 128) {
      v -= 256;
      carry = 1;
    } else {
      carry = 0;
    }
    dst[(int64_t)t * plane] = __int2bfloat16_rn(v);
  }
}

// X (rows x K, row-major, nl limb planes of stride rows*K) -> digit planes [S][rows][Kp]; columns
// k >= K are zero.  transpose: X is K x rows (row-major) instead, read as its transpose.
__global__ void int_split_kernel(const uint64_t *X, int nl, int64_t rows, int64_t K, int64_t Kp,
                                 int S, bool transpose, __nv_bfloat16 *dst) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * Kp) return;
  const int64_t r = idx / Kp, k = idx - (idx / Kp) * Kp;
  const int64_t plane = rows * Kp;
  __nv_bfloat16 *out = dst + r * Kp + k;
  if (k >= K) {
    for (int t = 0; t < S; ++t) out[(int64_t)t * plane] = __int2bfloat16_rn(0);
    return;
  }
  const int64_t e = transpose ? (k * rows + r) : (r * K + k);
  balanced_digits_twos(X + e, rows * K, nl, S, out, plane);
}

// T = sum_d digits[d] 256^d + sum_g carries[g] 256^ends[g], written modulo 2^(64 tl).
struct GroupEnds {
  int e[TG_MAXG];
};

__global__ void int_recombine_kernel(const uint8_t *digits, const int32_t *carries, int ND,
                                     int groups, const GroupEnds ends, int64_t M, int64_t N,
                                     int64_t Mp, int64_t Np, uint64_t *T, int tl) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int64_t i = idx / N, j = idx - (idx / N) * N;
  constexpr int W = 2 * IM_MAX_LIMBS + 4;
  uint64_t acc[W];
  const int nw = (8 * ND + 32 + 63) / 64 + 1;
  for (int k = 0; k < nw; ++k) acc[k] = 0;
  for (int d = 0; d < ND; ++d)
    acc[d >> 3] |= (uint64_t)digits[((int64_t)d * Mp + i) * Np + j] << (8 * (d & 7));
  for (int g = 0; g < groups; ++g) {
    const int64_t c = carries[((int64_t)g * Mp + i) * Np + j];
    const int pos = 8 * ends.e[g];
    // add c * 2^pos (sign-extended) into acc[0..nw)
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
  const uint64_t sext = (acc[nw - 1] >> 63) ? ~(uint64_t)0 : 0;
  for (int k = 0; k < tl; ++k) T[(int64_t)k * (M * N) + idx] = k < nw ? acc[k] : sext;
}

}  // namespace arbgpu

using namespace arbgpu;

namespace {

struct IntWs {
  size_t digX, digY, digits, carries, total;
  int SX, SY, ND, G;
  int64_t Kp, Mp, Np;
};

IntWs int_ws_layout(arbgpu_ctx *ctx, int xl, int yl, int64_t M, int64_t K, int64_t N) {
  IntWs w{};
  w.SX = 8 * xl + 1;
  w.SY = 8 * yl + 1;
  w.ND = w.SX + w.SY - 1;
  w.Kp = (K + TG_BK - 1) / TG_BK * TG_BK;
  w.Mp = (M + TG_BM - 1) / TG_BM * TG_BM;
  w.Np = (N + TG_BN - 1) / TG_BN * TG_BN;
  w.G = digit_gemm_groups(ctx, (int)M, (int)N, w.ND);
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  size_t off = 0;
  w.digX = off;
  off += al((size_t)w.SX * M * w.Kp * 2);
  w.digY = off;
  off += al((size_t)w.SY * N * w.Kp * 2);
  w.digits = off;
  off += al((size_t)w.ND * w.Mp * w.Np);
  w.carries = off;
  off += al((size_t)w.G * w.Mp * w.Np * 4);
  w.total = off;
  return w;
}

}  // namespace

namespace arbgpu {

size_t int_mat_mul_workspace(arbgpu_ctx *ctx, int xl, int yl, int64_t M, int64_t K, int64_t N) {
  return int_ws_layout(ctx, xl, yl, M, K, N).total;
}

arbgpu_status int_mat_mul_run(arbgpu_ctx *ctx, uint64_t *T, int32_t t_limbs, const uint64_t *X,
                              int32_t x_limbs, const uint64_t *Y, int32_t y_limbs, int64_t M,
                              int64_t K, int64_t N, void *workspace, size_t ws_bytes,
                              cudaStream_t s) {
  if (!ctx || x_limbs < 1 || y_limbs < 1 || x_limbs > IM_MAX_LIMBS || y_limbs > IM_MAX_LIMBS ||
      t_limbs < 1 || t_limbs > 2 * IM_MAX_LIMBS + 4 || M < 0 || K < 0 || N < 0)
    return ARBGPU_ERR_INVALID;
  if (M == 0 || N == 0) return ARBGPU_OK;
  if (!T || (K > 0 && (!X || !Y))) return ARBGPU_ERR_INVALID;
  if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) return ARBGPU_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ARBGPU_ERR_CUDA;
  if (K == 0) {
    return cudaMemsetAsync(T, 0, sizeof(uint64_t) * t_limbs * M * N, s) == cudaSuccess
               ? ARBGPU_OK
               : ARBGPU_ERR_CUDA;
  }
  IntWs w = int_ws_layout(ctx, x_limbs, y_limbs, M, K, N);
  if (!workspace || ws_bytes < w.total) return ARBGPU_ERR_WORKSPACE;
  if (!digit_gemm_fits(w.SX, w.SY, w.Kp)) return ARBGPU_ERR_LIMIT;
  uint8_t *ws = (uint8_t *)workspace;
  __nv_bfloat16 *dx = (__nv_bfloat16 *)(ws + w.digX);
  __nv_bfloat16 *dy = (__nv_bfloat16 *)(ws + w.digY);
  uint8_t *digits = ws + w.digits;
  int32_t *carries = (int32_t *)(ws + w.carries);
  GroupEnds ends{};
  digit_gemm_group_ends(w.SX, w.SY, w.G, ends.e);
  {
    const int64_t n = M * w.Kp;
    LaunchScope sc(ctx, s, "int_split", n);
    int_split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, x_limbs, M, K, w.Kp, w.SX,
                                                                 false, dx);
  }
  {
    const int64_t n = N * w.Kp;
    LaunchScope sc(ctx, s, "int_split", n);
    int_split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Y, y_limbs, N, K, w.Kp, w.SY, true,
                                                                 dy);
  }
  if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  DigitGemmArgs a{dx, dy, (int)M, (int)N, w.Kp, w.SX, w.SY, w.G, digits, carries, "digit_gemm"};
  arbgpu_status st = launch_digit_gemm(ctx, a, s);
  if (st != ARBGPU_OK) return st;
  {
    LaunchScope sc(ctx, s, "int_recombine", M * N);
    int_recombine_kernel<<<(unsigned)((M * N + 255) / 256), 256, 0, s>>>(
        digits, carries, w.ND, w.G, ends, M, N, w.Mp, w.Np, T, t_limbs);
  }
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

}  // namespace arbgpu

extern "C" {

arbgpu_status arbgpu_int_mat_mul_workspace_size(arbgpu_ctx *ctx, int32_t x_limbs, int32_t y_limbs,
                                                int64_t M, int64_t K, int64_t N, size_t *bytes) {
  if (!ctx || !bytes || x_limbs < 1 || y_limbs < 1 || x_limbs > IM_MAX_LIMBS ||
      y_limbs > IM_MAX_LIMBS || M < 0 || K < 0 || N < 0)
    return ARBGPU_ERR_INVALID;
  *bytes = int_ws_layout(ctx, x_limbs, y_limbs, M, K, N).total;
  return ARBGPU_OK;
}

arbgpu_status arbgpu_int_mat_mul(arbgpu_ctx *ctx, uint64_t *T, int32_t t_limbs, const uint64_t *X,
                                 int32_t x_limbs, const uint64_t *Y, int32_t y_limbs, int64_t M,
                                 int64_t K, int64_t N, void *workspace, size_t ws_bytes,
                                 void *stream) {
  return arbgpu::int_mat_mul_run(ctx, T, t_limbs, X, x_limbs, Y, y_limbs, M, K, N, workspace,
                                 ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"
