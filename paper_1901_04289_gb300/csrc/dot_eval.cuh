// Kernel (a): ball dot products by Algorithm 1 of the paper (Section III), in two launches.
//
//   setup      (Section III-C)  one warp per dot: lanes scan the terms' flags and exponents; warp
//              max/sum reductions give e_max, e_rad, N_nonzero and the accumulator size n_s.  Dots
//              that are finished here (special values, [0 +- 0]) are written out; for the others
//              the setup is parked in the dot's own output entry (exp = e_s, rad_exp = e_rad,
//              flags = PENDING | size class | n_s | limbs to read), so no workspace is needed.
//   evaluate   one launch per size class (NX limbs read per factor, NS accumulator limbs), each
//              compiled for its own register budget, so a warp never mixes code paths and the
//              instruction cache holds one class at a time.  Warps scan chunks of dots for the
//              entries of their class and evaluate them:
//     products (Section III-D)  every lane multiplies its terms' leading limbs exactly
//                               (64x64->128-bit products), aligns each product to the accumulator
//                               and adds or subtracts it in two's complement; bits falling below
//                               the accumulator, cut factors and skipped terms add one ulp to err.
//     radius   (Section III-E)  30-bit upper bounds of |m| r', |m'| r, r r' summed in a 64-bit
//                               fixed-point integer srad.
//     reduction                 the lanes' n_s-limb accumulators, err and srad are added with a
//                               butterfly of warp shuffles; integer addition modulo 2^(64 NS) is
//                               associative, so the result equals the sequential sum bit for bit.
//     finalise (Algorithm 1's finalisation) negate if negative, round to p bits (nearest, ties to even),
//                               radius = eps_round + err ulps + srad, rounded up to 30 bits; all
//                               in registers (fixed-size limb arrays, runtime bit positions).
//
// The accumulator and the product live in registers: every operand is held top-aligned in a
// fixed-size array of NX limbs (unread low limbs are zero), so the 2NX-limb product sits at a fixed
// position and one runtime offset F = 64 n_s - shift places it in the accumulator frame.  A dot
// may run in any class at least as large as its own (NX >= limbs read, NS >= n_s): the class only
// sizes the register arrays, the arithmetic is fixed by n_s.
#pragma once

#include "common.cuh"
#include "round_regs.cuh"

namespace arbgpu {

// Size classes: NX limbs read per factor, NS accumulator limbs.  A dot runs in the smallest class
// that holds its n_s and the number of limbs it reads (min(n, n_s + 1)).
template <int C>
struct DotClass;
template <> struct DotClass<0> { static constexpr int NX = 1, NS = 2; };
template <> struct DotClass<1> { static constexpr int NX = 2, NS = 3; };
template <> struct DotClass<2> { static constexpr int NX = 3, NS = 4; };
template <> struct DotClass<3> { static constexpr int NX = 4, NS = 5; };
template <> struct DotClass<4> { static constexpr int NX = 6, NS = 7; };
template <> struct DotClass<5> { static constexpr int NX = 9, NS = 9; };
template <> struct DotClass<6> { static constexpr int NX = 13, NS = 13; };
template <> struct DotClass<7> { static constexpr int NX = 19, NS = 18; };
constexpr int DOT_NUM_CLASSES = 8;
constexpr int DOT_MAX_NS = 18;
constexpr int DOT_MAX_NX = 19;

__host__ __device__ inline int dot_class_nx(int c) {
  const int t[DOT_NUM_CLASSES] = {1, 2, 3, 4, 6, 9, 13, 19};
  return t[c];
}
__host__ __device__ inline int dot_class_ns(int c) {
  const int t[DOT_NUM_CLASSES] = {2, 3, 4, 5, 7, 9, 13, 18};
  return t[c];
}
// Smallest class with NX >= nx and NS >= ns, or -1.
__host__ __device__ inline int dot_class_for(int nx, int ns) {
  for (int c = 0; c < DOT_NUM_CLASSES; ++c)
    if (dot_class_nx(c) >= nx && dot_class_ns(c) >= ns) return c;
  return -1;
}

// Binary length bc(v) = ceil(log2(v + 1)).
__host__ __device__ inline int bc64(int64_t v) {
  int b = 0;
  while (v > 0) {
    ++b;
    v >>= 1;
  }
  return b;
}

// Accumulator size n_s for precision p, N terms in total and N_nonzero terms (Section III-C).
__host__ __device__ inline int dot_ns(int p, int64_t nterms, int64_t nnz) {
  int padding = 4 + bc64(nterms);
  int extend = bc64(nnz) + 1;
  int ns = (p + extend + padding + 63) / 64;
  return ns < 2 ? 2 : ns;
}

// The scalar fields of one operand.
struct Opnd {
  uint32_t flags;
  int64_t e;
  uint32_t rman;
  int64_t rexp;
};

__device__ __forceinline__ Opnd load_opnd(const BallsView &v, int64_t i) {
  Opnd o;
  o.flags = __ldg(v.flags + i);
  o.e = __ldg(v.exp + i);
  o.rman = __ldg(v.rad_man + i);
  o.rexp = __ldg(v.rad_exp + i);
  return o;
}
// Midpoint fields only (for dots without radius products the radius fields are never needed).
__device__ __forceinline__ Opnd load_opnd_mid(const BallsView &v, int64_t i) {
  Opnd o;
  o.flags = __ldg(v.flags + i);
  o.e = __ldg(v.exp + i);
  o.rman = 0;
  o.rexp = 0;
  return o;
}

// The exact ball [1 +- 0]: the second factor of the `initial` term.
__device__ __forceinline__ Opnd one_opnd() { return Opnd{1u << ARBGPU_NSIG_SHIFT, 1, 0u, 0}; }

__device__ __forceinline__ bool opnd_zero(const Opnd &o) { return (o.flags & ARBGPU_FLAG_ZERO) != 0; }

__device__ __forceinline__ bool opnd_special(const Opnd &o) {
  if (o.flags & SPECIAL_MASK) return true;
  if (!opnd_zero(o) && (o.e >= EXP_LIMIT || o.e <= -EXP_LIMIT)) return true;
  if (o.rman && (o.rexp >= EXP_LIMIT || o.rexp <= -EXP_LIMIT)) return true;
  return false;
}

// Per-dot quantities of the setup pass.
struct DotSetup {
  int64_t e_s;
  int64_t e_rad;
  int n_s;
  int nx;  // limbs to read per factor (at most)
  bool has_mid, has_rad;
  bool approx;  // midpoint only: no radius is formed or written
  int prec;     // working and output precision (the requested one, or Section III-C's reduction)
};

// The setup parked in the output entry's flags word (bit 31 never appears in a finished entry).
constexpr uint32_t DOT_PENDING = 1u << 31;
__device__ __forceinline__ uint32_t pack_setup(int cls, const DotSetup &su) {
  return DOT_PENDING | (uint32_t)cls | ((uint32_t)su.n_s << 4) | ((uint32_t)su.nx << 10) |
         (su.has_mid ? (1u << 16) : 0u) | (su.has_rad ? (1u << 17) : 0u) |
         (su.approx ? (1u << 18) : 0u) | ((uint32_t)su.prec << 19);
}
__device__ __forceinline__ int pending_class(uint32_t f) {
  return (f & DOT_PENDING) ? (int)(f & 15u) : -1;
}
__device__ __forceinline__ DotSetup unpack_setup(uint32_t f, int64_t e_s, int64_t e_rad) {
  DotSetup su;
  su.e_s = e_s;
  su.e_rad = e_rad;
  su.n_s = (int)((f >> 4) & 63u);
  su.nx = (int)((f >> 10) & 63u);
  su.has_mid = (f >> 16) & 1u;
  su.has_rad = (f >> 17) & 1u;
  su.approx = (f >> 18) & 1u;
  su.prec = (int)((f >> 19) & 2047u);
  return su;
}

__device__ __forceinline__ int64_t warp_max_i64(int64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    int64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

// Lane groups: a warp evaluates 32 / G dots at once, G consecutive lanes per dot.  Shuffles name
// only the group's lanes, so groups may take different paths; offsets stay below G.
template <int G>
__device__ __forceinline__ unsigned group_mask(int lane) {
  if constexpr (G == 32)
    return 0xffffffffu;
  else
    return ((1u << G) - 1u) << (lane & ~(G - 1));
}
template <int G>
__device__ __forceinline__ int64_t group_max_i64(int64_t v, unsigned gm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = imax64(v, __shfl_xor_sync(gm, v, o));
  return v;
}
template <int G>
__device__ __forceinline__ int64_t group_sum_i64(int64_t v, unsigned gm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gm, v, o);
  return v;
}
__device__ __forceinline__ bool group_any(bool p, unsigned gm) { return __ballot_sync(gm, p) != 0; }

// Radius exponents of the nonzero products |m| r', |m'| r, r r' of one term (Section III-C 5c).
__device__ __forceinline__ int64_t term_rad_exp_max(const Opnd &x, const Opnd &y, int64_t cur) {
  bool xz = opnd_zero(x), yz = opnd_zero(y);
  if (!xz && y.rman) cur = imax64(cur, x.e + y.rexp);
  if (!yz && x.rman) cur = imax64(cur, y.e + x.rexp);
  if (x.rman && y.rman) cur = imax64(cur, x.rexp + y.rexp);
  return cur;
}

// srad += upper bound of (a/2^30)(b/2^30) 2^e in units of 2^(e_rad - 30) (Section III-E); a, b
// are at most 2^31 and 2^30, so the product is one 32 x 32 -> 64-bit multiply.
__device__ __forceinline__ void srad_add(uint64_t &srad, uint32_t a, uint32_t b, int64_t e,
                                         int64_t e_rad) {
  int64_t d = e_rad - e;
  if (d < P_RAD)
    srad += (((uint64_t)a * b) >> (P_RAD + (int)d)) + 1;
  else
    srad += 1;
}

__device__ __forceinline__ void term_radius(uint64_t &srad, const Opnd &x, uint64_t xtop,
                                            const Opnd &y, uint64_t ytop, int64_t e_rad) {
  bool xz = opnd_zero(x), yz = opnd_zero(y);
  if (!xz && y.rman)
    srad_add(srad, (uint32_t)(xtop >> (64 - P_RAD)) + 1, y.rman, x.e + y.rexp, e_rad);
  if (!yz && x.rman)
    srad_add(srad, (uint32_t)(ytop >> (64 - P_RAD)) + 1, x.rman, y.e + x.rexp, e_rad);
  if (x.rman && y.rman) srad_add(srad, x.rman, y.rman, x.rexp + y.rexp, e_rad);
}

// Load the r leading limbs of entry i top-aligned into a[NX] (a[NX-1] = top limb, zeros below).
template <int NX>
__device__ __forceinline__ void load_leading(const BallsView &v, int64_t i, int r, uint64_t (&a)[NX]) {
  const uint64_t *base = v.limbs + (int64_t)(v.nlimbs - 1) * v.stride + i;
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    uint64_t w = 0;
    if (j < r) w = __ldg(base - (int64_t)j * v.stride);
    a[NX - 1 - j] = w;
  }
}

// (c0, c1, c2) += a * b for 32-bit a, b: the 64-bit product into a three-word column accumulator
// (carries stay inside the one asm statement).
__device__ __forceinline__ void mac3(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t a,
                                     uint32_t b) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(c0), "+r"(c1), "+r"(c2)
      : "r"(a), "r"(b));
}

// p = a * b exactly (NX 64-bit limbs each): product scanning over 32-bit words, one column of the
// 2NX x 2NX partial products at a time (row products of 64-bit limbs for long operands).
template <int NX>
__device__ __forceinline__ void mul_limbs(const uint64_t (&a)[NX], const uint64_t (&b)[NX],
                                          uint64_t (&p)[2 * NX]) {
  if constexpr (NX > 6) {  // long operands: 64-bit row products keep fewer words live
#pragma unroll
    for (int k = 0; k < 2 * NX; ++k) p[k] = 0;
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      uint64_t carry = 0;
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        const u128 t = (u128)a[i] * b[j] + p[i + j] + carry;
        p[i + j] = (uint64_t)t;
        carry = (uint64_t)(t >> 64);
      }
      p[i + NX] = carry;
    }
    return;
  }
  constexpr int n = 2 * NX;
  uint32_t A[n], B[n], R[2 * n];
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    A[2 * i] = (uint32_t)a[i];
    A[2 * i + 1] = (uint32_t)(a[i] >> 32);
    B[2 * i] = (uint32_t)b[i];
    B[2 * i + 1] = (uint32_t)(b[i] >> 32);
  }
  uint32_t c0 = 0, c1 = 0, c2 = 0;
#pragma unroll
  for (int k = 0; k < 2 * n - 1; ++k) {
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const int j = k - i;
      if (j >= 0 && j < n) mac3(c0, c1, c2, A[i], B[j]);
    }
    R[k] = c0;
    c0 = c1;
    c1 = c2;
    c2 = 0;
  }
  R[2 * n - 1] = c0;
#pragma unroll
  for (int k = 0; k < 2 * NX; ++k) p[k] = (uint64_t)R[2 * k] | ((uint64_t)R[2 * k + 1] << 32);
}

// Per-lane accumulation state.
template <int NS>
struct LaneAcc {
  uint64_t s[NS];
  uint64_t err;
  uint64_t srad;
};

// Add the product p (NT limbs, the product of two top-aligned NT/2-limb factors) of a term to the
// lane accumulator: bit j of p lands at bit j + F of a frame whose limbs [NT, NT + n_s) are the
// accumulator; bits below it add one ulp to err.
template <int NT, int NS>
__device__ __forceinline__ void acc_add_product(LaneAcc<NS> &acc, const uint64_t (&p)[NT], int F,
                                                bool negative) {
  const int L0 = F >> 6, b0 = F & 63;
  uint64_t u[NT + 1];
  u[0] = p[0] << b0;
#pragma unroll
  for (int i = 1; i < NT; ++i) u[i] = shl_funnel(p[i], p[i - 1], b0);
  u[NT] = shl_funnel(0, p[NT - 1], b0);
  uint64_t disc = 0;
#pragma unroll
  for (int i = 0; i < NT; ++i)
    if (i < NT - L0) disc |= u[i];
  if (disc) acc.err += 1;
  uint64_t w[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    uint64_t v = 0;
#pragma unroll
    for (int l = 0; l < NS; ++l) {
      const int i = NT + k - l;
      if (i >= 0 && i <= NT) v = (L0 == l) ? u[i] : v;
    }
    w[k] = v;
  }
  const uint64_t flip = negative ? ~(uint64_t)0 : 0;
  u128 c = negative ? 1 : 0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    c += (u128)acc.s[k] + (w[k] ^ flip);
    acc.s[k] = (uint64_t)c;
    c >>= 64;
  }
}

// Add one midpoint term (both factors nonzero, shift < 64 n_s) to the lane accumulator.
template <int NX, int NS>
__device__ __forceinline__ void acc_term(LaneAcc<NS> &acc, const uint64_t (&xa)[NX],
                                         const uint64_t (&ya)[NX], int F, bool negative) {
  uint64_t p[2 * NX];
  mul_limbs<NX>(xa, ya, p);
  acc_add_product<2 * NX, NS>(acc, p, F, negative);
}

// The `initial` term x [1 +- 0]: with the one top-aligned in NXI limbs (2^63 in its top limb), the
// product is x times 2^(63 + 64 (NXI - 1)), a shift, so it needs no limb products.
template <int NXI, int NS>
__device__ __forceinline__ void acc_term_one(LaneAcc<NS> &acc, const uint64_t (&xa)[NXI], int F,
                                             bool negative) {
  uint64_t p[2 * NXI];
#pragma unroll
  for (int k = 0; k < 2 * NXI; ++k) {
    const int jl = k - NXI + 1, jh = k - NXI;  // limbs of x shifted into limb k
    const uint64_t lo = (jl >= 0 && jl < NXI) ? (xa[jl] << 63) : 0;
    const uint64_t hi = (jh >= 0 && jh < NXI) ? (xa[jh] >> 1) : 0;
    p[k] = lo | hi;
  }
  acc_add_product<2 * NXI, NS>(acc, p, F, negative);
}

// ---------------------------------------------------------------- finalise (registers only)

// Round the reduced accumulator to p bits and write output entry `oi` (Algorithm 1's finalisation).
// Every lane of the group holds the reduced sums and computes the same values; the output limbs are
// written by the group's lanes in parallel, the scalar fields by its first lane.
template <int NS, int G>
__device__ void dot_finalise(const LaneAcc<NS> &acc, const DotSetup &su, int prec,
                             const BallsOut &out, int64_t oi, int gl) {
  uint64_t a[NS];
  const bool neg = (acc.s[NS - 1] >> 63) != 0;
  {
    const uint64_t flip = neg ? ~(uint64_t)0 : 0;
    u128 c = neg ? 1 : 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      c += (u128)(acc.s[k] ^ flip);
      a[k] = (uint64_t)c;
      c >>= 64;
    }
  }
  int L = limbs_bitlen<NS>(a);
  const int64_t ulp_e = su.e_s - 64LL * su.n_s;
  const bool zero = (L == 0) || !su.has_mid;
  uint64_t ta[NS + 1];
  Mag r1{0u, 0};
  if (!zero)
    round_abs_regs<NS>(a, L, prec, acc.err, ulp_e, ta, r1);
  else if (su.has_mid)
    r1 = mag_from_u64(acc.err, ulp_e);
  const Mag r2 = su.has_rad ? mag_from_u64(acc.srad, su.e_rad - P_RAD) : Mag{0u, 0};
  store_rounded<NS + 1, G>(out, oi, gl, zero, neg, ta, ulp_e + L,
                           su.approx ? Mag{0u, 0} : mag_add_up(r1, r2));
}

template <int G>
__device__ __forceinline__ void write_special(const BallsOut &out, int64_t oi, int gl) {
  for (int j = gl; j < out.nlimbs; j += G) out.limbs[(int64_t)j * out.stride + oi] = 0;
  if (gl == 0) {
    out.exp[oi] = 0;
    out.flags[oi] = ARBGPU_FLAG_NAN | ARBGPU_FLAG_RAD_INF;
    out.rad_man[oi] = 0;
    out.rad_exp[oi] = 0;
  }
}

template <int G>
__device__ __forceinline__ void write_zero(const BallsOut &out, int64_t oi, int gl) {
  for (int j = gl; j < out.nlimbs; j += G) out.limbs[(int64_t)j * out.stride + oi] = 0;
  if (gl == 0) {
    out.exp[oi] = 0;
    out.flags[oi] = ARBGPU_FLAG_ZERO;
    out.rad_man[oi] = 0;
    out.rad_exp[oi] = 0;
  }
}

// One term of a dot as the source describes it: which array (0/1 = real/imaginary part) and
// which entry for each factor, and whether the product is subtracted.
struct TermLoc {
  int xa;
  int64_t xi;
  int ya;
  int64_t yi;
  bool neg;
};

// A term source provides, per dot d, a cursor (the dot's row/column/offsets, computed once) and
// through it: nterms, term(t), the optional `initial` entry, the output entry and the precision.

// Terms a lane takes per step of the evaluation loop.  The scalar fields and the leading limbs of
// all of them are requested together (the limbs speculatively, min(NX, n) of them, masked once the
// flags and exponents are in), so a step waits for one memory round trip.
template <int NX>
struct TermsPerStep {
  static constexpr int U = NX <= 2 ? 2 : 1;
};

// Load the leading min(NX, n) limbs of entry i top-aligned into a[NX] (zeros below).
template <int NX>
__device__ __forceinline__ void load_top(const BallsView &v, int64_t i, uint64_t (&a)[NX]) {
  const uint64_t *base = v.limbs + (int64_t)(v.nlimbs - 1) * v.stride + i;
#pragma unroll
  for (int j = 0; j < NX; ++j) a[NX - 1 - j] = j < v.nlimbs ? __ldg(base - (int64_t)j * v.stride) : 0;
}

// Keep the r leading limbs of a top-aligned operand.
template <int NX>
__device__ __forceinline__ void keep_leading(uint64_t (&a)[NX], int r) {
#pragma unroll
  for (int j = 0; j < NX; ++j)
    if (j >= r) a[NX - 1 - j] = 0;
}

// Evaluate the dot under cursor `cur` with a group of G lanes in size class C.
template <int C, int G, class Src>
__device__ void dot_eval_class(const Src &src, const typename Src::Cursor &cur,
                               const DotSetup &su, int prec, int gl, unsigned gm) {
  constexpr int NX = DotClass<C>::NX;
  constexpr int NS = DotClass<C>::NS;
  constexpr int U = TermsPerStep<NX>::U;
  LaneAcc<NS> acc;
#pragma unroll
  for (int k = 0; k < NS; ++k) acc.s[k] = 0;
  acc.err = 0;
  acc.srad = 0;
  const int64_t nt = src.nterms(cur);
  const int64_t width = 64LL * su.n_s;
  const bool rad = su.has_rad;
  // the regular terms (NX limbs per factor); the `initial` term follows below
  for (int64_t t0 = gl; t0 < nt; t0 += G * U) {
    Opnd x[U], y[U];
    const BallsView *xv[U];
    const BallsView *yv[U];
    int64_t xi[U], yi[U];
    bool negate[U], valid[U];
    // scalar fields and leading limbs of U terms
    uint64_t xa[U][NX], ya[U][NX];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t t = t0 + G * u;
      valid[u] = t < nt;
      xv[u] = nullptr;
      yv[u] = nullptr;
      xi[u] = yi[u] = 0;
      negate[u] = false;
      x[u] = y[u] = Opnd{ARBGPU_FLAG_ZERO, 0, 0u, 0};
#pragma unroll
      for (int j = 0; j < NX; ++j) xa[u][j] = ya[u][j] = 0;
      if (valid[u]) {
        const TermLoc tl = src.term(cur, t);
        xv[u] = &src.xview(cur, tl.xa);
        yv[u] = &src.yview(cur, tl.ya);
        xi[u] = tl.xi;
        yi[u] = tl.yi;
        negate[u] = tl.neg;
        x[u] = rad ? load_opnd(*xv[u], xi[u]) : load_opnd_mid(*xv[u], xi[u]);
        y[u] = rad ? load_opnd(*yv[u], yi[u]) : load_opnd_mid(*yv[u], yi[u]);
        load_top<NX>(*xv[u], xi[u], xa[u]);
        load_top<NX>(*yv[u], yi[u], ya[u]);
      }
    }
    // which terms reach the accumulator, and how many limbs of each factor they use
    int F[U];
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      live[u] = false;
      F[u] = 0;
      if (valid[u] && !opnd_zero(x[u]) && !opnd_zero(y[u])) {
        const int64_t shift = su.e_s - (x[u].e + y[u].e);
        if (shift >= width) {
          acc.err += 1;
        } else {
          live[u] = true;
          F[u] = (int)(width - shift);
          const int n2 = (F[u] + 63) / 64 + 1;
          const int nx = min((int)nsig_of(x[u].flags), xv[u]->nlimbs);
          const int ny = min((int)nsig_of(y[u].flags), yv[u]->nlimbs);
          if (nx > n2 || ny > n2) acc.err += 1;
          keep_leading<NX>(xa[u], min(nx, n2));
          keep_leading<NX>(ya[u], min(ny, n2));
        }
      }
    }
    // products and radii
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (live[u]) {
        const bool negative =
            (((x[u].flags ^ y[u].flags) & ARBGPU_FLAG_SIGN) != 0) != negate[u];
        acc_term<NX, NS>(acc, xa[u], ya[u], F[u], negative);
      }
      if (rad && valid[u] && (x[u].rman || y[u].rman))
        term_radius(acc.srad, x[u], xa[u][NX - 1], y[u], ya[u][NX - 1], su.e_rad);
    }
  }
  // the `initial` term x [1 +- 0], in the group's first lane, its limbs in NS + 1 >= n_s + 1
  // registers (at most n_s + 1 limbs of a term reach the accumulator)
  if (src.has_initial() && gl == 0) {
    constexpr int NXI = NS + 1;
    const BallsView &iv = src.initial_view(cur);
    const int64_t ii = src.initial_index(cur);
    const Opnd x = rad ? load_opnd(iv, ii) : load_opnd_mid(iv, ii);
    const Opnd y = one_opnd();
    uint64_t xa[NXI];
#pragma unroll
    for (int j = 0; j < NXI; ++j) xa[j] = 0;
    if (!opnd_zero(x)) {
      const int64_t shift = su.e_s - (x.e + y.e);
      if (shift >= width) {
        acc.err += 1;
      } else {
        const int F = (int)(width - shift);
        const int n2 = (F + 63) / 64 + 1;
        const int nx = min((int)nsig_of(x.flags), iv.nlimbs);
        if (nx > n2) acc.err += 1;
        load_top<NXI>(iv, ii, xa);
        keep_leading<NXI>(xa, min(nx, n2));
        acc_term_one<NXI, NS>(acc, xa, F, (x.flags & ARBGPU_FLAG_SIGN) != 0);
      }
    }
    if (rad && x.rman) {
      uint64_t xtop = xa[NXI - 1];
      if (!opnd_zero(x) && xtop == 0)
        xtop = __ldg(iv.limbs + (int64_t)(iv.nlimbs - 1) * iv.stride + ii);
      term_radius(acc.srad, x, xtop, y, (uint64_t)1 << 63, su.e_rad);
    }
  }
  // butterfly reduction over the group: every lane ends with the full sums
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    u128 c = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      uint64_t v = __shfl_xor_sync(gm, acc.s[k], o);
      c += (u128)acc.s[k] + v;
      acc.s[k] = (uint64_t)c;
      c >>= 64;
    }
    acc.err += __shfl_xor_sync(gm, acc.err, o);
    acc.srad += __shfl_xor_sync(gm, acc.srad, o);
  }
  dot_finalise<NS, G>(acc, su, prec, src.out_view(cur), src.out_index(cur), gl);
}

// Setup pass of dot d (Section III-C): finishes the dot (special values, limits, [0 +- 0]) or
// parks its setup in the output entry.  CMAX bounds the classes the launch will evaluate.
// Returns true with the setup in `su` and the dot's class in `cls` when the dot still needs its
// evaluation; otherwise the dot has been written out.
template <int G, class Src>
__device__ bool dot_setup_core(const Src &src, const typename Src::Cursor &cur, int cmax, int gl,
                               unsigned gm, int *status, DotSetup &su, int &cls) {
  const int prec = src.prec(cur);
  const int64_t nt = src.nterms(cur);
  const bool has_init = src.has_initial();
  const BallsOut &out = src.out_view(cur);
  const int64_t oi = src.out_index(cur);
  if (prec < 2 || prec > src.prec_max || nt < 0 || nt > src.len_max ||
      (int64_t)out.nlimbs * 64 < prec) {
    if (gl == 0) set_status(status, ARBGPU_ERR_LIMIT);
    write_special<G>(out, oi, gl);
    return false;
  }
  bool special = false;
  int64_t nnz = 0;
  int64_t e_max = INT64_MIN, e_rad = INT64_MIN;
  int64_t e_min = INT64_MAX;  // lowest possible bit of a product ("optimize p", when p > 2 beta)
  const bool track_min = src.reduce && prec > 128;
  int nsig_max = 0;
  constexpr int U = 2;  // terms per lane per step, loads issued together
  const int64_t ntot = nt + (has_init ? 1 : 0);
  for (int64_t t0 = gl; t0 < ntot; t0 += G * U) {
    Opnd x[U], y[U];
    bool valid[U], regular[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t t = t0 + G * u;
      valid[u] = t < ntot;
      regular[u] = t < nt;
      x[u] = y[u] = Opnd{ARBGPU_FLAG_ZERO, 0, 0u, 0};
      if (t < nt) {
        const TermLoc tl = src.term(cur, t);
        x[u] = load_opnd(src.xview(cur, tl.xa), tl.xi);
        y[u] = load_opnd(src.yview(cur, tl.ya), tl.yi);
      } else if (valid[u]) {
        x[u] = load_opnd(src.initial_view(cur), src.initial_index(cur));
        y[u] = one_opnd();
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!valid[u]) continue;
      if (opnd_special(x[u]) || opnd_special(y[u])) {
        special = true;
        continue;
      }
      if (!opnd_zero(x[u]) && !opnd_zero(y[u])) {
        ++nnz;
        e_max = imax64(e_max, x[u].e + y[u].e);
        if (track_min) {
          const int64_t lo = x[u].e + y[u].e -
                             64LL * ((int64_t)nsig_of(x[u].flags) + (int64_t)nsig_of(y[u].flags));
          e_min = lo < e_min ? lo : e_min;
        }
        // the `initial` term has its own limb array, so only the regular terms size the class
        if (regular[u])
          nsig_max = max(nsig_max, (int)max(nsig_of(x[u].flags), nsig_of(y[u].flags)));
      }
      e_rad = term_rad_exp_max(x[u], y[u], e_rad);
    }
  }
  if (group_any(special, gm)) {
    if (gl == 0) set_status(status, ARBGPU_ERR_UNSUPPORTED_VALUE);
    write_special<G>(out, oi, gl);
    return false;
  }
  nnz = group_sum_i64<G>(nnz, gm);
  e_max = group_max_i64<G>(e_max, gm);
  e_rad = group_max_i64<G>(e_rad, gm);
  nsig_max = (int)group_max_i64<G>(nsig_max, gm);
  if (track_min) e_min = -group_max_i64<G>(-e_min, gm);
  su.has_mid = e_max != INT64_MIN;
  su.approx = src.approx;
  su.has_rad = !su.approx && e_rad != INT64_MIN;  // approx: the radii are ignored
  if (!su.has_mid && !su.has_rad) {  // [0 +- 0]
    write_zero<G>(out, oi, gl);
    return false;
  }
  // "optimize p" of Section III-C, when asked for: a radius above the arithmetic error, or terms that
  // fit in a narrow window, lower the precision
  int p = prec;
  if (src.reduce) {
    if (!su.has_mid) {
      p = 2;
    } else {
      if (e_rad != INT64_MIN && e_max - e_rad + P_RAD < p) p = (int)(e_max - e_rad + P_RAD);
      if (track_min && e_min != INT64_MAX && e_max - e_min + P_RAD < p)
        p = (int)(e_max - e_min + P_RAD);
      if (p < 2) p = 2;
    }
  }
  su.prec = p;
  const int extend = bc64(nnz) + 1;
  su.n_s = dot_ns(p, ntot, nnz);
  su.e_s = su.has_mid ? e_max + extend : 0;
  su.e_rad = e_rad;
  su.nx = min(nsig_max, su.n_s + 1);
  if (su.nx < 1) su.nx = 1;
  const int c = dot_class_for(su.nx, su.n_s);
  if (c < 0 || c > cmax) {
    if (gl == 0) set_status(status, ARBGPU_ERR_LIMIT);
    write_special<G>(out, oi, gl);
    return false;
  }
  cls = c;
  return true;
}

// Setup of dot d, parked in its output entry for the evaluation launch of its class.
template <int G, class Src>
__device__ void dot_setup(const Src &src, int64_t d, int cmax, int gl, unsigned gm, int *status) {
  const typename Src::Cursor cur = src.cursor(d);
  DotSetup su;
  int c = 0;
  if (!dot_setup_core<G>(src, cur, cmax, gl, gm, status, su, c)) return;
  if (gl == 0) {
    const BallsOut &out = src.out_view(cur);
    const int64_t oi = src.out_index(cur);
    out.exp[oi] = su.e_s;
    out.rad_exp[oi] = su.e_rad;
    out.flags[oi] = pack_setup(c, su);
  }
}

template <int G, class Src>
__global__ void __launch_bounds__(256, 4) dot_setup_kernel(const __grid_constant__ Src src, int cmax,
                                                        int *status) {
  constexpr int DPW = 32 / G;  // dots per warp step
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const unsigned gm = group_mask<G>(lane);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nd = src.ndots();
  for (int64_t d0 = warp * DPW; d0 < nd; d0 += nwarps * DPW) {
    const int64_t d = d0 + lane / G;
    if (d < nd) dot_setup<G>(src, d, cmax, gl, gm, status);
  }
}

// Largest number of dots a warp scans per step of an evaluation launch.
constexpr int DOT_CHUNK = 32;

// Resident 256-thread blocks per SM the register budget of each class is sized for.
template <int C>
struct DotClassBlocks {
  static constexpr int B = C <= 2 ? 3 : (C <= 4 ? 2 : 1);
};

// Evaluation of every pending dot of class C: a warp reads the parked flags of `chunk` dots and
// evaluates those of its class, 32 / G at a time (one per lane group).
template <int C, int G, class Src>
__global__ void __launch_bounds__(256, DotClassBlocks<C>::B)
    dot_eval_kernel(const __grid_constant__ Src src, int chunk) {
  constexpr int DPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int g = lane / G, gl = lane & (G - 1);
  const unsigned gm = group_mask<G>(lane);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nd = src.ndots();
  const int64_t nchunks = (nd + chunk - 1) / chunk;
  for (int64_t ch = warp; ch < nchunks; ch += nwarps) {
    const int64_t d0 = ch * chunk;
    uint32_t f = 0;
    if (lane < chunk && d0 + lane < nd) {
      const typename Src::Cursor c = src.cursor(d0 + lane);
      f = __ldg(src.out_view(c).flags + src.out_index(c));
    }
    unsigned mask = __ballot_sync(0xffffffffu, pending_class(f) == C);
    while (mask) {
      // group g takes the g-th remaining dot of the chunk
      unsigned m = mask;
      for (int k = 0; k < g; ++k) m &= m - 1;
      const int pos = m ? __ffs(m) - 1 : 0;
      const bool has = m != 0;
#pragma unroll
      for (int k = 0; k < DPW; ++k) mask &= mask - 1;
      const uint32_t fd = __shfl_sync(0xffffffffu, f, pos);
      if (has) {
        const typename Src::Cursor cd = src.cursor(d0 + pos);
        const BallsOut &out = src.out_view(cd);
        const int64_t oi = src.out_index(cd);
        const DotSetup su = unpack_setup(fd, __ldg(out.exp + oi), __ldg(out.rad_exp + oi));
        dot_eval_class<C, G>(src, cd, su, su.prec, gl, gm);
      }
      __syncwarp();
    }
  }
}

// Setup and evaluation in one launch, every dot in class C (the largest class of the problem):
// for sources whose dots share one precision, so that all of them need (nearly) the same class.
template <int C, int G, class Src>
__global__ void __launch_bounds__(256, DotClassBlocks<C>::B)
    dot_fused_kernel(const __grid_constant__ Src src, int *status) {
  constexpr int DPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const unsigned gm = group_mask<G>(lane);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nd = src.ndots();
  for (int64_t d0 = warp * DPW; d0 < nd; d0 += nwarps * DPW) {
    const int64_t d = d0 + lane / G;
    if (d < nd) {
      const typename Src::Cursor cur = src.cursor(d);
      DotSetup su;
      int c = 0;
      if (dot_setup_core<G>(src, cur, C, gl, gm, status, su, c))
        dot_eval_class<C, G>(src, cur, su, su.prec, gl, gm);
    }
    __syncwarp();
  }
}

}  // namespace arbgpu
