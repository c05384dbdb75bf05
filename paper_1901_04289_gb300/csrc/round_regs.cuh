// Rounding of a multi-limb magnitude to p bits in registers (fixed-size limb arrays indexed only
// by compile-time positions; the bit positions are runtime values), shared by the dot kernel
// (Algorithm 1's finalisation) and the block product's epilogue (Algorithm 2): round to nearest, ties to
// even, the exact rounding error (plus an error count) rounded up to a 30-bit mag, and the store of
// the rounded ball.
#pragma once

#include "common.cuh"

namespace arbgpu {

// Bit length of the N-limb magnitude a (0 for zero).
template <int N>
__device__ __forceinline__ int limbs_bitlen(const uint64_t (&a)[N]) {
  int L = 0;
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (a[k]) L = 64 * k + bitlen64(a[k]);
  return L;
}

// Smallest 30-bit mag >= v * 2^base for a fixed-size limb array (the same value as
// mag_from_limbs, without dynamically indexed arrays).
template <int N>
__device__ __forceinline__ Mag mag_up_regs(const uint64_t (&v)[N], int64_t base) {
  int top = -1;
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (v[k]) top = k;
  if (top < 0) return Mag{0u, 0};
  uint64_t hi = 0, lo = 0;
  bool rest = false;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (k == top) hi = v[k];
    if (k == top - 1) lo = v[k];
    if (k < top - 1) rest |= v[k] != 0;
  }
  const int lb = bitlen64(hi);
  const int64_t L = (int64_t)top * 64 + lb;
  if (L <= 64) return mag_from_u64(hi, base);
  const uint64_t w = (lb == 64) ? hi : ((hi << (64 - lb)) | (lo >> lb));
  const bool sticky = rest || ((lb == 64) ? (lo != 0) : ((lo << (64 - lb)) != 0));
  uint64_t b = w >> 34;
  if ((w & ((((uint64_t)1) << 34) - 1)) || sticky) b += 1;
  int64_t e = base + L;
  if (b == ((uint64_t)1 << P_RAD)) {
    b >>= 1;
    e += 1;
  }
  return Mag{(uint32_t)b, e};
}

// v <<= 64 q for 0 <= q < N (a barrel shifter over limbs: log2 N rounds of selects).
template <int N>
__device__ __forceinline__ void limbs_shift_up(uint64_t (&v)[N], int q) {
#pragma unroll
  for (int b = 1; b < N; b <<= 1) {
    const bool on = (q & b) != 0;
#pragma unroll
    for (int j = N - 1; j >= 0; --j) v[j] = on ? (j >= b ? v[j - b] : 0) : v[j];
  }
}

// Round the magnitude a (N limbs, bit length L with 1 <= L <= 64 N) to prec < 64 (N + 1) bits,
// nearest with ties to even.  On return ta[0..N] holds the rounded magnitude top-aligned (bit
// 64 (N + 1) - 1 set), L is its bit length (one more when rounding carried out of the top), and
// r1 is the smallest 30-bit mag >= (|rounded - a| + extra) 2^base.
template <int N>
__device__ __forceinline__ void round_abs_regs(const uint64_t (&a)[N], int &L, int prec,
                                               uint64_t extra, int64_t base,
                                               uint64_t (&ta)[N + 1], Mag &r1) {
  constexpr int NT = N + 1;
  // ta = a * 2^s0, top bit at 64 NT - 1 (s0 >= 64)
  const int s0 = 64 * NT - L;
  const int bs = s0 & 63;
  ta[0] = a[0] << bs;
#pragma unroll
  for (int j = 1; j < N; ++j) ta[j] = shl_funnel(a[j], a[j - 1], bs);
  ta[N] = shl_funnel(0, a[N - 1], bs);
  limbs_shift_up<NT>(ta, s0 >> 6);
  // keep the top p bits: cut at bit c of ta (bits below c are the rounding remainder)
  const int c = 64 * NT - prec;
  const int cl = c >> 6, cb = c & 63;
  const int rl = (c - 1) >> 6, rb = (c - 1) & 63;
  uint64_t rem[NT];
  uint64_t rword = 0, lword = 0;
  bool sticky = false;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const uint64_t low = j < cl ? ~(uint64_t)0 : (j == cl ? ((((uint64_t)1) << cb) - 1) : 0);
    rem[j] = ta[j] & low;
    ta[j] &= ~low;
    if (j == rl) rword = rem[j];
    if (j == cl) lword = ta[j];
    const uint64_t below_r = j < rl ? ~(uint64_t)0 : (j == rl ? ((((uint64_t)1) << rb) - 1) : 0);
    sticky |= (rem[j] & below_r) != 0;
  }
  const bool rbit = (rword >> rb) & 1;
  const bool lsb = (lword >> cb) & 1;
  const bool up = rbit && (sticky || lsb);
  // eps = |rounded - a| in units of ta: 2^c - rem when rounding up, else rem
  uint64_t E[NT + 1];
  if (up) {
    u128 cc = 0;
    uint64_t borrow = 0;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const uint64_t unit = j == cl ? (((uint64_t)1) << cb) : 0;
      cc += (u128)ta[j] + unit;
      ta[j] = (uint64_t)cc;
      cc >>= 64;
      const u128 dlt = (u128)unit - rem[j] - borrow;
      E[j] = (uint64_t)dlt;
      borrow = (uint64_t)(dlt >> 64) & 1;
    }
    if ((uint64_t)cc) {  // rounded up to 2^(64 NT): one bit longer
#pragma unroll
      for (int j = 0; j < NT; ++j) ta[j] = 0;
      ta[NT - 1] = ((uint64_t)1) << 63;
      L += 1;
    }
  } else {
#pragma unroll
    for (int j = 0; j < NT; ++j) E[j] = rem[j];
  }
  E[NT] = 0;
  // E += extra * 2^s0
  {
    const int q = s0 >> 6;
    const uint64_t lo = extra << bs;
    const uint64_t hi = bs ? (extra >> (64 - bs)) : 0;
    u128 cc = 0;
#pragma unroll
    for (int j = 0; j < NT + 1; ++j) {
      const uint64_t add = (j == q) ? lo : ((j == q + 1) ? hi : 0);
      cc += (u128)E[j] + add;
      E[j] = (uint64_t)cc;
      cc >>= 64;
    }
  }
  r1 = mag_up_regs<NT + 1>(E, base - s0);
}

// Store a rounded ball: mantissa ta[0..NT) top-aligned (ta[NT-1] holds the top bit), exponent
// oexp, radius r; `zero` stores [0 +- r].  Lanes gl = 0..G-1 write the limbs, lane 0 the rest.
template <int NT, int G>
__device__ __forceinline__ void store_rounded(const BallsOut &out, int64_t oi, int gl, bool zero,
                                              bool neg, const uint64_t (&ta)[NT], int64_t oexp,
                                              Mag r) {
  const int nl = out.nlimbs;
  // output limb nl-1-m is ta[NT-1-m] (m < NT), zero below
  for (int m = gl; m < nl; m += G) {
    uint64_t v = 0;
    if (!zero) {
#pragma unroll
      for (int j = 0; j < NT; ++j)
        if (m == NT - 1 - j) v = ta[j];
    }
    out.limbs[(int64_t)(nl - 1 - m) * out.stride + oi] = v;
  }
  if (gl == 0) {
    uint32_t fl;
    if (zero) {
      out.exp[oi] = 0;
      fl = ARBGPU_FLAG_ZERO;
    } else {
      // significant limbs: from the top limb down to the lowest nonzero one
      int jmin = NT - 1;
#pragma unroll
      for (int j = NT - 1; j >= 0; --j)
        if (ta[j] && NT - 1 - j < nl) jmin = j;
      out.exp[oi] = oexp;
      fl = (neg ? ARBGPU_FLAG_SIGN : 0u) | ((uint32_t)(NT - jmin) << ARBGPU_NSIG_SHIFT);
    }
    out.flags[oi] = fl;
    out.rad_man[oi] = r.man;
    out.rad_exp[oi] = r.man ? r.exp : 0;
  }
}

}  // namespace arbgpu
