// arbgpu_calibrate: throughput of the integer units the dot path and the alternative 8-bit tensor
// path would use, measured on the device the context runs on.  Three micro-kernels, each a
// grid of 4 CTAs of 256 threads per SM running independent chains long enough (a few
// milliseconds) that launch costs vanish:
//   imad       32-bit multiply-add (mad.lo.u32): 8 independent chains per thread;
//   imad_wide  32 x 32 + 64 -> 64-bit multiply-add (mad.wide.u32), the step of the CUDA-core
//              reconstruction's column sums: 8 independent chains per thread;
//   mma_s8     the legacy warp-level 8-bit tensor MMA (mma.sync m16n8k32 s8 x s8 + s32), four
//              independent accumulators per warp (the only 8-bit tensor form that assembles for
//              sm_103a: tcgen05 kind::i8 does not).
// Every chain's final value is written out, so no work can be dropped.
#include <cstring>

#include "internal.h"

namespace arbgpu {

constexpr int CAL_ITERS = 4096;

__global__ void __launch_bounds__(256) cal_imad_kernel(uint32_t seed, uint32_t *out) {
  uint32_t a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed + threadIdx.x + 977u * c;
  const uint32_t m = seed | 1u, k = seed ^ 0x9e3779b9u;
  for (int it = 0; it < CAL_ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(m), "r"(k));
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) r ^= a[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void __launch_bounds__(256) cal_imad_wide_kernel(uint32_t seed, uint64_t *out) {
  uint64_t a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed + threadIdx.x + 977u * c;
  const uint32_t m = seed | 1u;
  uint32_t x = seed ^ 0x85ebca6bu;
  for (int it = 0; it < CAL_ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a[c]) : "r"(x), "r"(m));
    x += 1u;
  }
  uint64_t r = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) r ^= a[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void __launch_bounds__(256) cal_mma_s8_kernel(uint32_t seed, int32_t *out) {
  // fragments of m16n8k32: A 4 x b32 (16 s8 each thread), B 2 x b32, C/D 4 x s32
  const uint32_t a0 = seed * 3u + threadIdx.x, a1 = a0 ^ 0x01010101u, a2 = a0 + 0x02020202u,
                 a3 = a0 ^ 0x7f7f7f7fu;
  const uint32_t b0 = seed * 7u + threadIdx.x, b1 = b0 ^ 0x03030303u;
  int32_t d[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r) d[q][r] = 0;
  for (int it = 0; it < CAL_ITERS / 16; ++it) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
          "{%8, %9}, {%0, %1, %2, %3};"
          : "+r"(d[q][0]), "+r"(d[q][1]), "+r"(d[q][2]), "+r"(d[q][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  int32_t r = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < 4; ++c) r ^= d[q][c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace arbgpu

using namespace arbgpu;

extern "C" {

arbgpu_status arbgpu_calibrate(arbgpu_ctx *ctx, arbgpu_calibration *out) {
  if (!ctx || !out) return ARBGPU_ERR_INVALID;
  memset(out, 0, sizeof(*out));
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ARBGPU_ERR_CUDA;
  const int blocks = 4 * ctx->sm_count, threads = 256;
  const size_t n = (size_t)blocks * threads;
  void *buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  arbgpu_status st = ARBGPU_ERR_CUDA;
  if (cudaMalloc(&buf, 8 * n) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    goto done;
  {
    auto timed = [&](auto launch, double ops, double *rate) -> bool {
      launch();  // warm-up
      if (cudaEventRecord(e0) != cudaSuccess) return false;
      for (int r = 0; r < 3; ++r) launch();
      if (cudaEventRecord(e1) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        return false;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) return false;
      *rate = 3.0 * ops / (ms * 1e-3) / 1e12;
      return cudaGetLastError() == cudaSuccess;
    };
    const double lanes = (double)n;
    if (!timed([&]() { cal_imad_kernel<<<blocks, threads>>>(12345u, (uint32_t *)buf); },
               lanes * CAL_ITERS * 8, &out->imad_tops) ||
        !timed([&]() { cal_imad_wide_kernel<<<blocks, threads>>>(777u, (uint64_t *)buf); },
               lanes * CAL_ITERS * 8, &out->imad_wide_tops) ||
        !timed([&]() { cal_mma_s8_kernel<<<blocks, threads>>>(99u, (int32_t *)buf); },
               (lanes / 32.0) * (CAL_ITERS / 16) * 4 * (2.0 * 16 * 8 * 32), &out->mma_s8_tops))
      goto done;
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, ctx->device);
    out->sm_count = ctx->sm_count;
    out->max_clock_mhz = clk / 1000.0;
    st = ARBGPU_OK;
  }
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  cudaSetDevice(prev);
  return st;
}

}  // extern "C"
