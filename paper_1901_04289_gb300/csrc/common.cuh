// Shared device-side definitions of the arbgpu library: the ball layout view, 128-bit limb
// arithmetic, the 30-bit upward-rounded radius ("mag", Section III-A) and the status word.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "arbgpu.h"

namespace arbgpu {

typedef unsigned __int128 u128;

constexpr int P_RAD = 30;                                  // radius precision (Section III-A)
constexpr int64_t EXP_LIMIT = (int64_t)1 << 60;            // |exponent| limit of the fast path
constexpr uint32_t SPECIAL_MASK = ARBGPU_FLAG_INF | ARBGPU_FLAG_NAN | ARBGPU_FLAG_RAD_INF;

// Read-only view of one ball array (see include/arbgpu.h for the layout).
struct BallsView {
  const uint64_t *limbs;
  int64_t stride;
  int32_t nlimbs;
  const int64_t *exp;
  const uint32_t *flags;
  const uint32_t *rad_man;
  const int64_t *rad_exp;
};

struct BallsOut {
  uint64_t *limbs;
  int64_t stride;
  int32_t nlimbs;
  int64_t *exp;
  uint32_t *flags;
  uint32_t *rad_man;
  int64_t *rad_exp;
};

inline BallsView view_of(const arbgpu_balls &b) {
  return BallsView{b.limbs, b.limb_stride, b.nlimbs, b.exp, b.flags, b.rad_man, b.rad_exp};
}
inline BallsOut out_of(const arbgpu_balls &b) {
  return BallsOut{b.limbs, b.limb_stride, b.nlimbs, b.exp, b.flags, b.rad_man, b.rad_exp};
}

__device__ __forceinline__ uint32_t nsig_of(uint32_t flags) { return (flags >> ARBGPU_NSIG_SHIFT) & 0xFFu; }

// Programmatic dependent launch: a kernel launched with launch_pdl may start while the previous
// kernel of its stream finishes; pdl_wait() returns once that kernel has completed and its writes
// are visible, so it comes before the first access to anything an earlier kernel writes.
// pdl_trigger() lets the next such kernel start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Device status word: the first error code wins (atomicCAS from 0).
__device__ __forceinline__ void set_status(int *status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// 64-bit funnel shift left: (hi:lo) << b, high word, 0 <= b < 64.
__device__ __forceinline__ uint64_t shl_funnel(uint64_t hi, uint64_t lo, int b) {
  return (hi << b) | ((lo >> 1) >> (63 - b));
}

__device__ __forceinline__ int bitlen64(uint64_t v) { return v ? 64 - __clzll((long long)v) : 0; }

// acc += a * b for 32-bit a, b and a 64-bit acc, as one widening multiply-add (mad.wide.u32).
__device__ __forceinline__ void mad_wide(uint64_t &acc, uint32_t a, uint32_t b) {
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// 30-bit radius value man * 2^(exp - 30), man = 0 (zero) or 2^29 <= man < 2^30.
struct Mag {
  uint32_t man;
  int64_t exp;
};

// Smallest 30-bit mag >= v * 2^base (v a 64-bit unsigned integer).
__device__ __forceinline__ Mag mag_from_u64(uint64_t v, int64_t base) {
  Mag m{0u, 0};
  if (v == 0) return m;
  int L = bitlen64(v);
  if (L <= P_RAD) {
    m.man = (uint32_t)(v << (P_RAD - L));
    m.exp = base + L;
    return m;
  }
  int sh = L - P_RAD;
  uint64_t b = v >> sh;
  if (v & ((((uint64_t)1) << sh) - 1)) b += 1;
  int64_t e = base + L;
  if (b == ((uint64_t)1 << P_RAD)) {
    b >>= 1;
    e += 1;
  }
  m.man = (uint32_t)b;
  m.exp = e;
  return m;
}

// Smallest 30-bit mag >= (multi-limb unsigned v[0..n)) * 2^base; dynamic n (finalisation only).
__device__ __forceinline__ Mag mag_from_limbs(const uint64_t *v, int n, int64_t base) {
  int top = -1;
  for (int k = n - 1; k >= 0; --k)
    if (v[k]) {
      top = k;
      break;
    }
  if (top < 0) return Mag{0u, 0};
  int lb = bitlen64(v[top]);
  int64_t L = (int64_t)top * 64 + lb;  // total bit length
  if (L <= 64) return mag_from_u64(v[0], base);
  // top 64 bits of v (bits [L-64, L)) plus a sticky flag for the rest
  uint64_t hi = v[top], lo = v[top - 1];
  uint64_t w = (lb == 64) ? hi : ((hi << (64 - lb)) | (lo >> lb));
  bool sticky = (lb == 64) ? (lo != 0) : ((lo << (64 - lb)) != 0);
  for (int k = top - 2; k >= 0 && !sticky; --k) sticky = v[k] != 0;
  // w holds bits [L-64, L); round up to 30 bits with the remaining bits as sticky
  uint64_t b = w >> 34;
  if ((w & ((((uint64_t)1) << 34) - 1)) || sticky) b += 1;
  int64_t e = base + L;
  if (b == ((uint64_t)1 << P_RAD)) {
    b >>= 1;
    e += 1;
  }
  return Mag{(uint32_t)b, e};
}

// Smallest 30-bit mag >= a + b (the exact sum rounded up once).
__device__ __forceinline__ Mag mag_add_up(Mag a, Mag b) {
  if (a.man == 0) return b;
  if (b.man == 0) return a;
  if (a.exp < b.exp) {
    Mag t = a;
    a = b;
    b = t;
  }
  int64_t d = a.exp - b.exp;
  if (d <= 33) {
    uint64_t s = ((uint64_t)a.man << d) + (uint64_t)b.man;
    return mag_from_u64(s, b.exp - P_RAD);
  }
  // b is below one unit of a's 30-bit mantissa and nonzero: round a up by one unit
  uint64_t m = (uint64_t)a.man + 1;
  int64_t e = a.exp;
  if (m == ((uint64_t)1 << P_RAD)) {
    m >>= 1;
    e += 1;
  }
  return Mag{(uint32_t)m, e};
}

}  // namespace arbgpu
