// Kernel (a): one warp evaluates one ball dot product by Algorithm 1 of the paper (Section III).
//
//   setup      (Section III-C)  lanes scan the terms' flags and exponents; warp max/sum reductions
//                               give e_max, e_rad, N_nonzero and the accumulator size n_s.
//   evaluation (Section III-D)  every lane multiplies its terms' leading limbs exactly
//                               (64x64->128-bit products), aligns each product to the accumulator
//                               and adds or subtracts it in two's complement; bits falling below
//                               the accumulator, cut factors and skipped terms add one ulp to err.
//   radius     (Section III-E)  30-bit upper bounds of |m| r', |m'| r, r r' summed in a 64-bit
//                               fixed-point integer srad.
//   reduction                   the lanes' n_s-limb accumulators, err and srad are added with a
//                               butterfly of warp shuffles; integer addition modulo 2^(64 NS) is
//                               associative, so the result equals the sequential sum bit for bit.
//   finalise   (Algorithm 1, step 4) negate if negative, round to p bits (nearest, ties to even),
//                               radius = eps_round + err ulps + srad, rounded up to 30 bits.
//
// The accumulator and the product live in registers: every operand is held top-aligned in a
// fixed-size array of NX limbs (unread low limbs are zero), so the 2NX-limb product sits at a fixed
// position and one runtime offset F = 64 n_s - shift places it in the accumulator frame.
#pragma once

#include "common.cuh"

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
};

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

// Radius exponents of the nonzero products |m| r', |m'| r, r r' of one term (Section III-C 5c).
__device__ __forceinline__ int64_t term_rad_exp_max(const Opnd &x, const Opnd &y, int64_t cur) {
  bool xz = opnd_zero(x), yz = opnd_zero(y);
  if (!xz && y.rman) cur = imax64(cur, x.e + y.rexp);
  if (!yz && x.rman) cur = imax64(cur, y.e + x.rexp);
  if (x.rman && y.rman) cur = imax64(cur, x.rexp + y.rexp);
  return cur;
}

// srad += upper bound of (a/2^30)(b/2^30) 2^e in units of 2^(e_rad - 30) (Section III-E).
__device__ __forceinline__ void srad_add(uint64_t &srad, uint64_t a, uint64_t b, int64_t e,
                                         int64_t e_rad) {
  int64_t d = e_rad - e;
  if (d < P_RAD)
    srad += ((a * b) >> (P_RAD + (int)d)) + 1;
  else
    srad += 1;
}

__device__ __forceinline__ void term_radius(uint64_t &srad, const Opnd &x, uint64_t xtop,
                                            const Opnd &y, uint64_t ytop, int64_t e_rad) {
  bool xz = opnd_zero(x), yz = opnd_zero(y);
  if (!xz && y.rman) srad_add(srad, (xtop >> (64 - P_RAD)) + 1, y.rman, x.e + y.rexp, e_rad);
  if (!yz && x.rman) srad_add(srad, (ytop >> (64 - P_RAD)) + 1, x.rman, y.e + x.rexp, e_rad);
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

// p = a * b (schoolbook, exact).
template <int NX>
__device__ __forceinline__ void mul_limbs(const uint64_t (&a)[NX], const uint64_t (&b)[NX],
                                          uint64_t (&p)[2 * NX]) {
#pragma unroll
  for (int k = 0; k < 2 * NX; ++k) p[k] = 0;
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    uint64_t carry = 0;
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      u128 t = (u128)a[i] * b[j] + p[i + j] + carry;
      p[i + j] = (uint64_t)t;
      carry = (uint64_t)(t >> 64);
    }
    p[i + NX] = carry;
  }
}

// Per-lane accumulation state.
template <int NS>
struct LaneAcc {
  uint64_t s[NS];
  uint64_t err;
  uint64_t srad;
};

// Add one midpoint term (both factors nonzero, shift < 64 n_s) to the lane accumulator.
template <int NX, int NS>
__device__ __forceinline__ void acc_term(LaneAcc<NS> &acc, const uint64_t (&xa)[NX],
                                         const uint64_t (&ya)[NX], int F, bool negative) {
  constexpr int NT = 2 * NX;
  uint64_t p[NT];
  mul_limbs<NX>(xa, ya, p);
  // bit j of p lands at bit j + F of a frame whose limbs [NT, NT + n_s) are the accumulator
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

// ---------------------------------------------------------------- multi-limb helpers (finalise)

__device__ __forceinline__ bool limbs_bit(const uint64_t *a, int n, int64_t pos) {
  if (pos < 0 || pos >= 64LL * n) return false;
  return (a[pos >> 6] >> (pos & 63)) & 1;
}
__device__ __forceinline__ bool limbs_any_below(const uint64_t *a, int n, int64_t pos) {
  if (pos <= 0) return false;
  int64_t lim = pos >> 6;
  for (int k = 0; k < n && k < lim; ++k)
    if (a[k]) return true;
  int rb = pos & 63;
  if (rb && lim < n) return (a[lim] & ((((uint64_t)1) << rb) - 1)) != 0;
  return false;
}
// out[0..nout) = floor(a * 2^-sh) mod 2^(64 nout) for sh >= 0, or a * 2^(-sh) for sh < 0.
__device__ __forceinline__ void limbs_shift(const uint64_t *a, int n, int64_t sh, uint64_t *out,
                                            int nout) {
  for (int k = 0; k < nout; ++k) {
    // bits [64k + sh, 64k + sh + 64) of a
    int64_t lo = 64LL * k + sh;
    int64_t li = lo >= 0 ? (lo >> 6) : -((-lo + 63) >> 6);
    int bi = (int)(lo - li * 64);
    uint64_t w0 = (li >= 0 && li < n) ? a[li] : 0;
    uint64_t w1 = (li + 1 >= 0 && li + 1 < n) ? a[li + 1] : 0;
    out[k] = bi ? ((w0 >> bi) | (w1 << (64 - bi))) : w0;
  }
}

// Finalise a reduced accumulator (Algorithm 1, step 4) and write output entry `oi`.
template <int NS>
__device__ void dot_finalise(const LaneAcc<NS> &acc, const DotSetup &su, int prec,
                             const BallsOut &out, int64_t oi, int lane) {
  if (lane != 0) return;  // every lane holds the reduced sums; one finishes the dot
  uint64_t a[NS + 1];
  for (int k = 0; k < NS; ++k) a[k] = acc.s[k];
  a[NS] = 0;
  bool neg = (a[NS - 1] >> 63) != 0;
  if (neg) {
    u128 c = 1;
    for (int k = 0; k < NS; ++k) {
      c += (u128)(~a[k]);
      a[k] = (uint64_t)c;
      c >>= 64;
    }
  }
  int top = -1;
  for (int k = NS - 1; k >= 0; --k)
    if (a[k]) {
      top = k;
      break;
    }
  const int64_t ulp_e = su.e_s - 64LL * su.n_s;
  uint64_t E[NS + 2];  // eps_round + err, in accumulator ulps
  for (int k = 0; k < NS + 2; ++k) E[k] = 0;
  const int nl = out.nlimbs;
  uint64_t field[64];
  int64_t oexp = 0;
  bool zero = (top < 0) || !su.has_mid;
  if (!zero) {
    int64_t L = 64LL * top + bitlen64(a[top]);
    int64_t k = L > prec ? L - prec : 0;
    if (k > 0) {
      bool rbit = limbs_bit(a, NS, k - 1);
      bool sticky = limbs_any_below(a, NS, k - 1);
      bool up = rbit && (sticky || limbs_bit(a, NS, k));
      // rem = a mod 2^k
      uint64_t rem[NS + 1];
      for (int j = 0; j < NS + 1; ++j) {
        int64_t lo = 64LL * j;
        rem[j] = (lo + 64 <= k) ? a[j] : (lo < k ? (a[j] & ((((uint64_t)1) << (k - lo)) - 1)) : 0);
      }
      // clear the low k bits of a
      for (int j = 0; j < NS + 1; ++j) a[j] ^= rem[j];
      if (up) {
        // eps = 2^k - rem (0 < rem < 2^k here), then a += 2^k
        for (int j = 0; j < NS + 1; ++j) E[j] = 0;
        E[k >> 6] = ((uint64_t)1) << (k & 63);
        uint64_t borrow = 0;
        for (int j = 0; j < NS + 1; ++j) {
          u128 dlt = (u128)E[j] - rem[j] - borrow;
          E[j] = (uint64_t)dlt;
          borrow = (uint64_t)(dlt >> 64) & 1;
        }
        int64_t pos = k;
        u128 cc = ((u128)1) << (pos & 63);
        for (int j = (int)(pos >> 6); j < NS + 1; ++j) {
          cc += a[j];
          a[j] = (uint64_t)cc;
          cc >>= 64;
        }
        if (limbs_bit(a, NS + 1, L)) L += 1;
      } else {
        for (int j = 0; j < NS + 1; ++j) E[j] = rem[j];
      }
    }
    // field = top-aligned mantissa in nl limbs: a * 2^(64 nl - L)
    limbs_shift(a, NS + 1, L - 64LL * nl, field, nl);
    oexp = ulp_e + L;
  }
  // E += err
  {
    u128 c = acc.err;
    for (int j = 0; j < NS + 2; ++j) {
      c += E[j];
      E[j] = (uint64_t)c;
      c >>= 64;
    }
  }
  Mag r1 = su.has_mid ? mag_from_limbs(E, NS + 2, ulp_e) : Mag{0u, 0};
  Mag r2 = su.has_rad ? mag_from_u64(acc.srad, su.e_rad - P_RAD) : Mag{0u, 0};
  Mag r = mag_add_up(r1, r2);
  if (lane == 0) {
    uint32_t fl;
    if (zero) {
      for (int j = 0; j < nl; ++j) out.limbs[(int64_t)j * out.stride + oi] = 0;
      out.exp[oi] = 0;
      fl = ARBGPU_FLAG_ZERO;
    } else {
      int nsig = 0;
      for (int j = 0; j < nl; ++j) {
        out.limbs[(int64_t)j * out.stride + oi] = field[j];
        if (nsig == 0 && field[j]) nsig = nl - j;
      }
      out.exp[oi] = oexp;
      fl = (neg ? ARBGPU_FLAG_SIGN : 0u) | ((uint32_t)nsig << ARBGPU_NSIG_SHIFT);
    }
    out.flags[oi] = fl;
    out.rad_man[oi] = r.man;
    out.rad_exp[oi] = r.man ? r.exp : 0;
  }
}

__device__ __forceinline__ void write_special(const BallsOut &out, int64_t oi, int lane) {
  if (lane == 0) {
    for (int j = 0; j < out.nlimbs; ++j) out.limbs[(int64_t)j * out.stride + oi] = 0;
    out.exp[oi] = 0;
    out.flags[oi] = ARBGPU_FLAG_NAN | ARBGPU_FLAG_RAD_INF;
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

// Evaluate dot d of `src` with one warp in size class C.
template <int C, class Src>
__device__ void dot_eval_class(const Src &src, int64_t d, const DotSetup &su, int prec, int lane) {
  constexpr int NX = DotClass<C>::NX;
  constexpr int NS = DotClass<C>::NS;
  LaneAcc<NS> acc;
#pragma unroll
  for (int k = 0; k < NS; ++k) acc.s[k] = 0;
  acc.err = 0;
  acc.srad = 0;
  const int64_t nt = src.nterms(d);
  const bool has_init = src.has_initial(d);
  const int64_t width = 64LL * su.n_s;
  for (int64_t t = lane; t < nt + (has_init ? 1 : 0); t += 32) {
    Opnd x, y;
    const BallsView *xv = nullptr;
    const BallsView *yv = nullptr;
    int64_t xi = 0, yi = 0;
    bool negate = false;
    if (t < nt) {
      TermLoc tl = src.term(d, t);
      xv = &src.xview(tl.xa);
      yv = &src.yview(tl.ya);
      xi = tl.xi;
      yi = tl.yi;
      negate = tl.neg;
      x = load_opnd(*xv, xi);
      y = load_opnd(*yv, yi);
    } else {
      xv = &src.initial_view(d);
      xi = src.initial_index(d);
      x = load_opnd(*xv, xi);
      y = one_opnd();
    }
    const bool xz = opnd_zero(x), yz = opnd_zero(y);
    uint64_t xtop = 0, ytop = 0;
    if (!xz && !yz) {
      const int64_t shift = su.e_s - (x.e + y.e);
      if (shift >= width) {
        acc.err += 1;
      } else {
        const int F = (int)(width - shift);
        const int n2 = (F + 63) / 64 + 1;
        const int nx = min((int)nsig_of(x.flags), xv->nlimbs);
        const int ny = yv ? min((int)nsig_of(y.flags), yv->nlimbs) : 1;
        if (nx > n2 || ny > n2) acc.err += 1;
        const int rx = min(nx, n2), ry = min(ny, n2);
        uint64_t xa[NX], ya[NX];
        load_leading<NX>(*xv, xi, rx, xa);
        if (yv) {
          load_leading<NX>(*yv, yi, ry, ya);
        } else {
#pragma unroll
          for (int j = 0; j < NX; ++j) ya[j] = 0;
          ya[NX - 1] = (uint64_t)1 << 63;
        }
        xtop = xa[NX - 1];
        ytop = ya[NX - 1];
        const bool negative = (((x.flags ^ y.flags) & ARBGPU_FLAG_SIGN) != 0) != negate;
        acc_term<NX, NS>(acc, xa, ya, F, negative);
      }
    }
    if (su.has_rad && (x.rman || y.rman)) {
      if (!xz && xtop == 0) xtop = __ldg(xv->limbs + (int64_t)(xv->nlimbs - 1) * xv->stride + xi);
      if (!yz && ytop == 0)
        ytop = yv ? __ldg(yv->limbs + (int64_t)(yv->nlimbs - 1) * yv->stride + yi)
                  : ((uint64_t)1 << 63);
      term_radius(acc.srad, x, xtop, y, ytop, su.e_rad);
    }
  }
  // butterfly reduction: every lane ends with the full sums
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u128 c = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      uint64_t v = __shfl_xor_sync(0xffffffffu, acc.s[k], o);
      c += (u128)acc.s[k] + v;
      acc.s[k] = (uint64_t)c;
      c >>= 64;
    }
    acc.err += __shfl_xor_sync(0xffffffffu, acc.err, o);
    acc.srad += __shfl_xor_sync(0xffffffffu, acc.srad, o);
  }
  dot_finalise<NS>(acc, su, prec, src.out_view(d), src.out_index(d), lane);
}

// Whole dot: setup pass, class dispatch, evaluation.  CMAX bounds the classes compiled in.
template <int CMAX, class Src>
__device__ void dot_run(const Src &src, int64_t d, int lane, int *status) {
  const int prec = src.prec(d);
  const int64_t nt = src.nterms(d);
  const bool has_init = src.has_initial(d);
  const BallsOut &out = src.out_view(d);
  const int64_t oi = src.out_index(d);
  if (prec < 2 || prec > src.prec_max || nt < 0 || nt > src.len_max ||
      (int64_t)out.nlimbs * 64 < prec) {
    set_status(status, ARBGPU_ERR_LIMIT);
    write_special(out, oi, lane);
    return;
  }
  // ---- setup pass (Section III-C)
  bool special = false;
  int64_t nnz = 0;
  int64_t e_max = INT64_MIN, e_rad = INT64_MIN;
  int nsig_max = 0;
  for (int64_t t = lane; t < nt + (has_init ? 1 : 0); t += 32) {
    Opnd x, y;
    if (t < nt) {
      TermLoc tl = src.term(d, t);
      x = load_opnd(src.xview(tl.xa), tl.xi);
      y = load_opnd(src.yview(tl.ya), tl.yi);
    } else {
      x = load_opnd(src.initial_view(d), src.initial_index(d));
      y = one_opnd();
    }
    if (opnd_special(x) || opnd_special(y)) {
      special = true;
      continue;
    }
    if (!opnd_zero(x) && !opnd_zero(y)) {
      ++nnz;
      e_max = imax64(e_max, x.e + y.e);
      nsig_max = max(nsig_max, (int)max(nsig_of(x.flags), nsig_of(y.flags)));
    }
    e_rad = term_rad_exp_max(x, y, e_rad);
  }
  special = __any_sync(0xffffffffu, special);
  if (special) {
    set_status(status, ARBGPU_ERR_UNSUPPORTED_VALUE);
    write_special(out, oi, lane);
    return;
  }
  nnz = warp_sum_i64(nnz);
  e_max = warp_max_i64(e_max);
  e_rad = warp_max_i64(e_rad);
  nsig_max = (int)warp_max_i64(nsig_max);
  DotSetup su;
  su.has_mid = e_max != INT64_MIN;
  su.has_rad = e_rad != INT64_MIN;
  if (!su.has_mid && !su.has_rad) {  // [0 +- 0]
    if (lane == 0) {
      for (int j = 0; j < out.nlimbs; ++j) out.limbs[(int64_t)j * out.stride + oi] = 0;
      out.exp[oi] = 0;
      out.flags[oi] = ARBGPU_FLAG_ZERO;
      out.rad_man[oi] = 0;
      out.rad_exp[oi] = 0;
    }
    return;
  }
  const int64_t ntot = nt + (has_init ? 1 : 0);
  const int extend = bc64(nnz) + 1;
  su.n_s = dot_ns(prec, ntot, nnz);
  su.e_s = su.has_mid ? e_max + extend : 0;
  su.e_rad = e_rad;
  su.nx = min(nsig_max, su.n_s + 1);
  if (su.nx < 1) su.nx = 1;
  const int c = dot_class_for(su.nx, su.n_s);
  if (c < 0 || c > CMAX) {
    set_status(status, ARBGPU_ERR_LIMIT);
    write_special(out, oi, lane);
    return;
  }
  switch (c) {
    case 0: if constexpr (CMAX >= 0) dot_eval_class<0>(src, d, su, prec, lane); break;
    case 1: if constexpr (CMAX >= 1) dot_eval_class<1>(src, d, su, prec, lane); break;
    case 2: if constexpr (CMAX >= 2) dot_eval_class<2>(src, d, su, prec, lane); break;
    case 3: if constexpr (CMAX >= 3) dot_eval_class<3>(src, d, su, prec, lane); break;
    case 4: if constexpr (CMAX >= 4) dot_eval_class<4>(src, d, su, prec, lane); break;
    case 5: if constexpr (CMAX >= 5) dot_eval_class<5>(src, d, su, prec, lane); break;
    case 6: if constexpr (CMAX >= 6) dot_eval_class<6>(src, d, su, prec, lane); break;
    case 7: if constexpr (CMAX >= 7) dot_eval_class<7>(src, d, su, prec, lane); break;
    default: break;
  }
}

template <int CMAX, class Src>
__global__ void __launch_bounds__(256) dot_kernel(const __grid_constant__ Src src, int *status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nd = src.ndots();
  for (int64_t d = warp; d < nd; d += nwarps) dot_run<CMAX>(src, d, lane, status);
}

}  // namespace arbgpu
