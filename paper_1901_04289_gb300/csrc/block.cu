// The block algorithm for ball matrix products (Algorithm 2, Section IV-A) around the tensor-core
// integer engine:
//
//   scan   per row of A / column of B: largest exponent (top), exponent of the lowest set bit
//          (bottom), largest radius exponent; global p_A, p_B and the largest heights.
//   plan   h = 1.25 min(p, max(p_A, p_B)) + 192 (Algorithm 2, step 2); the product is one block when
//          every row of A and column of B scales to integers of height <= h (the common case the
//          paper describes: uniformly scaled inputs need a single block).
//   split  E A and B F with the minimal-height scalings e_i = -bottom_i, f_j = -bottom_j (Fig. 2),
//          written as balanced base-256 digits; the radius operands |A|, R_A, R_B, |B| + R_B become
//          nonnegative integers rounded UP in 13-bit windows under each row's / column's top.
//   gemm   T = (E A)(B F) exactly on the tensor cores; P1 = U(|A|) V(R_B), P2 = U(R_A) V(|B|+R_B).
//   round  C_ij = RNE_p(T_ij 2^(-e_i - f_j)) (one rounding of the exact entry) and
//          R_ij >= eps_round + P1 2^(...) + P2 2^(...), rounded up to a 30-bit radius.
#include <cstring>

#include "internal.h"
#include "tc_gemm.cuh"

namespace arbgpu {

constexpr int BL_W = 13;          // radius window bits: operands rounded up to <= 2^13
constexpr int BL_SR = 2;          // digits per radius operand (2^13 fits two balanced digits)
constexpr int BL_MAX_NL = 32;     // input limbs the block path accepts
constexpr int BL_BASECASE = 30;   // Algorithm 2: blocks shorter than this go to dot products

struct BlockStats {
  int64_t pA, pB;         // largest significant-bit count of an entry
  int64_t hA, hB;         // largest row / column height (top - bottom)
  int32_t special;        // NaN / infinity / out-of-range exponent seen
  int32_t radA, radB;     // a nonzero radius seen
  int32_t pad;
};

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
    const uint64_t low = __ldg(v.limbs + (int64_t)(v.nlimbs - ns) * v.stride + idx);
    s.bot = e - 64LL * ns + (low ? __ffsll((long long)low) - 1 : 0);
  }
  if (s.rad && (re >= EXP_LIMIT || re <= -EXP_LIMIT)) s.special = true;
  return s;
}

// One warp per row of A (lanes over k): row top / bottom / radius top.
__global__ void scan_rows_kernel(const BallsView A, int64_t M, int64_t K, int64_t lda,
                                 int64_t *rtop, int64_t *rbot, int64_t *rrad, BlockStats *st) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= M) return;
  int64_t top = INT64_MIN, bot = INT64_MAX, rad = INT64_MIN, pm = 0;
  bool special = false, anyrad = false;
  for (int64_t k = lane; k < K; k += 32) {
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
    rtop[i] = top;
    rbot[i] = bot;
    rrad[i] = rad;
    if (top != INT64_MIN) atomic_max_i64(&st->hA, top - bot);
    atomic_max_i64(&st->pA, pm);
    if (special) atomicOr(&st->special, 1);
    if (anyrad) atomicOr(&st->radA, 1);
  }
}

// Columns of B: block (32 columns) x (32 k-slices); reads coalesced along the row.
__global__ void scan_cols_kernel(const BallsView B, int64_t K, int64_t N, int64_t ldb,
                                 int64_t *ctop, int64_t *cbot, int64_t *crad, int64_t *cplus,
                                 BlockStats *st) {
  __shared__ int64_t s_top[32][33], s_bot[32][33], s_rad[32][33], s_pm[32][33];
  __shared__ int s_flags[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t j = (int64_t)blockIdx.x * 32 + tx;
  int64_t top = INT64_MIN, bot = INT64_MAX, rad = INT64_MIN, pm = 0;
  int flags = 0;
  if (j < N) {
    for (int64_t k = ty; k < K; k += 32) {
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
    for (int y = 1; y < 32; ++y) {
      top = max((long long)top, (long long)s_top[y][tx]);
      bot = min((long long)bot, (long long)s_bot[y][tx]);
      rad = max((long long)rad, (long long)s_rad[y][tx]);
      pm = max((long long)pm, (long long)s_pm[y][tx]);
      flags |= s_flags[y][tx];
    }
    ctop[j] = top;
    cbot[j] = bot;
    crad[j] = rad;
    // |b| + r_b < 2^(max(top, rexp) + 1)
    const int64_t mx = top > rad ? top : rad;
    cplus[j] = mx == INT64_MIN ? INT64_MIN : mx + 1;
    if (top != INT64_MIN) atomic_max_i64(&st->hB, top - bot);
    atomic_max_i64(&st->pB, pm);
    if (flags & 1) atomicOr(&st->special, 1);
    if (flags & 2) atomicOr(&st->radB, 1);
  }
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
__global__ void split_kernel(const BallsView X, bool is_b, int64_t rows, int64_t K, int64_t Kp,
                             int64_t ld, int S, const int64_t *bot, const int64_t *top,
                             const int64_t *radtop, const int64_t *plustop, SplitOut o) {
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
  const int64_t e = is_b ? (k * ld + r) : (r * ld + k);
  const uint32_t fl = __ldg(X.flags + e);
  const bool nz = !(fl & (ARBGPU_FLAG_ZERO | SPECIAL_MASK));
  const int64_t ex = __ldg(X.exp + e);
  if (nz) {
    const int64_t sh = ex - 64LL * X.nlimbs - bot[r];
    split_mid_digits(X, e, sh, (fl & ARBGPU_FLAG_SIGN) != 0, S, o.mid + off, plane);
  } else {
    for (int t = 0; t < S; ++t) o.mid[(int64_t)t * plane + off] = z;
  }
  const Mag rad{__ldg(X.rad_man + e), __ldg(X.rad_exp + e)};
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

struct IntProduct {  // one exact integer product in digit + carry form
  const uint8_t *digits;
  const int32_t *carries;
  int ND, groups;
  Ends ends;
};

constexpr int RD_MAXW = 48;  // limbs of the assembled product (ND <= 8 * 46)

// Assemble T_ij (two's complement, nw limbs) from its digits and carries.
__device__ __forceinline__ int assemble(const IntProduct &p, int64_t i, int64_t j, int64_t Mp,
                                        int64_t Np, uint64_t *acc) {
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

struct RoundArgs {
  IntProduct mid;
  IntProduct rp1, rp2;  // radius products (ND = 0 when absent)
  const int64_t *rtop, *rbot, *rrad;            // rows of A
  const int64_t *ctop, *cbot, *crad, *cplus;    // columns of B
  BallsOut C;
  int64_t M, N, ldc, Mp, Np;
  int prec;
};

__device__ __forceinline__ Mag product_mag(const IntProduct &p, int64_t i, int64_t j, int64_t Mp,
                                           int64_t Np, int64_t base) {
  if (p.ND == 0) return Mag{0u, 0};
  uint64_t acc[4];
  assemble(p, i, j, Mp, Np, acc);  // nonnegative and < 2^64 (13+13+log2 K + 2 bits)
  return mag_from_u64(acc[0], base);
}

__global__ void block_round_kernel(const RoundArgs a) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.M * a.N) return;
  const int64_t i = idx / a.N, j = idx - (idx / a.N) * a.N;
  uint64_t T[RD_MAXW];
  const int nw = assemble(a.mid, i, j, a.Mp, a.Np, T);
  const bool rowz = a.rtop[i] == INT64_MIN, colz = a.ctop[j] == INT64_MIN;
  const int64_t sigma = (rowz ? 0 : a.rbot[i]) + (colz ? 0 : a.cbot[j]);  // T * 2^sigma
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
  const BallsOut &C = a.C;
  const int64_t oi = i * a.ldc + j;
  const int nl = C.nlimbs;
  uint64_t E[RD_MAXW];
  for (int k = 0; k < nw; ++k) E[k] = 0;
  bool zero = top < 0;
  uint32_t fl = ARBGPU_FLAG_ZERO;
  int64_t oexp = 0;
  if (!zero) {
    int64_t L = 64LL * top + bitlen64(T[top]);
    const int64_t k = L > a.prec ? L - a.prec : 0;
    if (k > 0) {
      // round to nearest, ties to even, at bit k; E = |rounded - T|
      auto bit = [&](int64_t pos) -> bool {
        return pos >= 0 && pos < 64LL * nw && ((T[pos >> 6] >> (pos & 63)) & 1);
      };
      bool sticky = false;
      for (int64_t w = 0; w < ((k - 1) >> 6) && !sticky; ++w) sticky = T[w] != 0;
      if (!sticky && ((k - 1) & 63)) sticky = (T[(k - 1) >> 6] & ((((uint64_t)1) << ((k - 1) & 63)) - 1)) != 0;
      const bool up = bit(k - 1) && (sticky || bit(k));
      uint64_t rem[RD_MAXW];
      for (int w = 0; w < nw; ++w) {
        const int64_t lo = 64LL * w;
        rem[w] = (lo + 64 <= k) ? T[w] : (lo < k ? (T[w] & ((((uint64_t)1) << (k - lo)) - 1)) : 0);
        T[w] ^= rem[w];
      }
      if (up) {
        for (int w = 0; w < nw; ++w) E[w] = 0;
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
  // radius: eps_round * 2^sigma + P1 2^(top_i + crad_j - 2W) + P2 2^(rrad_i + cplus_j - 2W)
  Mag r = mag_from_limbs(E, nw, sigma);
  if (a.rp1.ND && a.rtop[i] != INT64_MIN && a.crad[j] != INT64_MIN)
    r = mag_add_up(r, product_mag(a.rp1, i, j, a.Mp, a.Np, a.rtop[i] + a.crad[j] - 2 * BL_W));
  if (a.rp2.ND && a.rrad[i] != INT64_MIN && a.cplus[j] != INT64_MIN)
    r = mag_add_up(r, product_mag(a.rp2, i, j, a.Mp, a.Np, a.rrad[i] + a.cplus[j] - 2 * BL_W));
  C.rad_man[oi] = r.man;
  C.rad_exp[oi] = r.man ? r.exp : 0;
}

// ------------------------------------------------------------------------- workspace and driver

struct BlockWs {
  size_t stats, rtop, rbot, rrad, ctop, cbot, crad, cplus;
  size_t dA, dB, rA1, rA2, rB1, rB2;
  size_t mdig, mcar, r1dig, r1car, r2dig, r2car;
  size_t total;
  int Smax, NDmax, Gmax, Gr;
  int64_t Kp, Mp, Np;
};

static BlockWs block_ws(arbgpu_ctx *ctx, int64_t M, int64_t K, int64_t N, int prec) {
  BlockWs w{};
  const int64_t hmax = (5LL * prec) / 4 + 192;
  w.Smax = (int)((hmax + 2 + 7) / 8);
  w.NDmax = 2 * w.Smax - 1;
  w.Kp = (K + TG_BK - 1) / TG_BK * TG_BK;
  w.Mp = (M + TG_BM - 1) / TG_BM * TG_BM;
  w.Np = (N + TG_BN - 1) / TG_BN * TG_BN;
  w.Gmax = digit_gemm_groups(ctx, (int)M, (int)N, w.NDmax);
  w.Gr = digit_gemm_groups(ctx, (int)M, (int)N, 2 * BL_SR - 1);
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += al(bytes);
    return o;
  };
  w.stats = take(sizeof(BlockStats));
  w.rtop = take(8 * M);
  w.rbot = take(8 * M);
  w.rrad = take(8 * M);
  w.ctop = take(8 * N);
  w.cbot = take(8 * N);
  w.crad = take(8 * N);
  w.cplus = take(8 * N);
  w.dA = take((size_t)w.Smax * M * w.Kp * 2);
  w.dB = take((size_t)w.Smax * N * w.Kp * 2);
  w.rA1 = take((size_t)BL_SR * M * w.Kp * 2);
  w.rA2 = take((size_t)BL_SR * M * w.Kp * 2);
  w.rB1 = take((size_t)BL_SR * N * w.Kp * 2);
  w.rB2 = take((size_t)BL_SR * N * w.Kp * 2);
  w.mdig = take((size_t)w.NDmax * w.Mp * w.Np);
  w.mcar = take((size_t)w.Gmax * w.Mp * w.Np * 4);
  w.r1dig = take((size_t)(2 * BL_SR - 1) * w.Mp * w.Np);
  w.r1car = take((size_t)w.Gr * w.Mp * w.Np * 4);
  w.r2dig = take((size_t)(2 * BL_SR - 1) * w.Mp * w.Np);
  w.r2car = take((size_t)w.Gr * w.Mp * w.Np * 4);
  w.total = off;
  return w;
}

size_t block_workspace_size(arbgpu_ctx *ctx, int64_t M, int64_t K, int64_t N, int prec) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  return block_ws(ctx, M, K, N, prec).total;
}

// Real block product.  Returns ARBGPU_ERR_LIMIT when the inputs need more than one block or hold
// special values (the caller then uses the classical algorithm).
arbgpu_status block_matmul_real(arbgpu_ctx *ctx, const arbgpu_balls &C, const arbgpu_balls &A,
                                const arbgpu_balls &B, int64_t M, int64_t K, int64_t N,
                                int64_t lda, int64_t ldb, int64_t ldc, int prec, void *workspace,
                                size_t ws_bytes, cudaStream_t s, bool *used_block) {
  *used_block = false;
  if (A.nlimbs > BL_MAX_NL || B.nlimbs > BL_MAX_NL) return ARBGPU_ERR_LIMIT;
  if (K < BL_BASECASE) return ARBGPU_ERR_LIMIT;
  BlockWs w = block_ws(ctx, M, K, N, prec);
  if (!workspace || ws_bytes < w.total) return ARBGPU_ERR_WORKSPACE;
  uint8_t *ws = (uint8_t *)workspace;
  BlockStats *st = (BlockStats *)(ws + w.stats);
  int64_t *rtop = (int64_t *)(ws + w.rtop), *rbot = (int64_t *)(ws + w.rbot);
  int64_t *rrad = (int64_t *)(ws + w.rrad);
  int64_t *ctop = (int64_t *)(ws + w.ctop), *cbot = (int64_t *)(ws + w.cbot);
  int64_t *crad = (int64_t *)(ws + w.crad), *cplus = (int64_t *)(ws + w.cplus);
  BlockStats init{};
  init.hA = init.hB = INT64_MIN;
  if (cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  const BallsView Av = view_of(A), Bv = view_of(B);
  {
    LaunchScope sc(ctx, s, "scan_rows", M * K);
    scan_rows_kernel<<<(unsigned)((M * 32 + 255) / 256), 256, 0, s>>>(Av, M, K, lda, rtop, rbot,
                                                                        rrad, st);
  }
  {
    LaunchScope sc(ctx, s, "scan_cols", K * N);
    scan_cols_kernel<<<(unsigned)((N + 31) / 32), dim3(32, 32), 0, s>>>(Bv, K, N, ldb, ctop, cbot,
                                                                         crad, cplus, st);
  }
  BlockStats hs{};
  if (cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  if (hs.special) return ARBGPU_ERR_LIMIT;
  const int64_t pmax = hs.pA > hs.pB ? hs.pA : hs.pB;
  const int64_t h = (5 * (prec < pmax ? (int64_t)prec : pmax)) / 4 + 192;
  if (hs.hA > h || hs.hB > h) return ARBGPU_ERR_LIMIT;  // needs several blocks
  const int SA = hs.hA < 0 ? 1 : (int)((hs.hA + 2 + 7) / 8);
  const int SB = hs.hB < 0 ? 1 : (int)((hs.hB + 2 + 7) / 8);
  if (SA > w.Smax || SB > w.Smax || !digit_gemm_fits(SA, SB, w.Kp)) return ARBGPU_ERR_LIMIT;
  const bool radB = hs.radB != 0, radA = hs.radA != 0;
  __nv_bfloat16 *dA = (__nv_bfloat16 *)(ws + w.dA), *dB = (__nv_bfloat16 *)(ws + w.dB);
  __nv_bfloat16 *rA1 = (__nv_bfloat16 *)(ws + w.rA1), *rA2 = (__nv_bfloat16 *)(ws + w.rA2);
  __nv_bfloat16 *rB1 = (__nv_bfloat16 *)(ws + w.rB1), *rB2 = (__nv_bfloat16 *)(ws + w.rB2);
  {
    const int64_t n = M * w.Kp;
    SplitOut o{dA, radB ? rA1 : nullptr, radA ? rA2 : nullptr};
    LaunchScope sc(ctx, s, "split_a", n);
    split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Av, false, M, K, w.Kp, lda, SA, rbot,
                                                             rtop, rrad, nullptr, o);
  }
  {
    const int64_t n = N * w.Kp;
    SplitOut o{dB, radB ? rB1 : nullptr, radA ? rB2 : nullptr};
    LaunchScope sc(ctx, s, "split_b", n);
    split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Bv, true, N, K, w.Kp, ldb, SB, cbot,
                                                             ctop, crad, cplus, o);
  }
  if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  RoundArgs ra{};
  const int ND = SA + SB - 1;
  const int G = digit_gemm_groups(ctx, (int)M, (int)N, ND);
  if (G > w.Gmax) return ARBGPU_ERR_LIMIT;
  {
    DigitGemmArgs g{dA, dB, (int)M, (int)N, w.Kp, SA, SB, G, ws + w.mdig,
                    (int32_t *)(ws + w.mcar), "digit_gemm_mid"};
    arbgpu_status stg = launch_digit_gemm(ctx, g, s);
    if (stg != ARBGPU_OK) return stg;
    ra.mid = IntProduct{ws + w.mdig, (int32_t *)(ws + w.mcar), ND, G, {}};
    digit_gemm_group_ends(SA, SB, G, ra.mid.ends.e);
  }
  const int NDr = 2 * BL_SR - 1;
  if (radB) {
    DigitGemmArgs g{rA1, rB1, (int)M, (int)N, w.Kp, BL_SR, BL_SR, w.Gr, ws + w.r1dig,
                    (int32_t *)(ws + w.r1car), "digit_gemm_rad"};
    arbgpu_status stg = launch_digit_gemm(ctx, g, s);
    if (stg != ARBGPU_OK) return stg;
    ra.rp1 = IntProduct{ws + w.r1dig, (int32_t *)(ws + w.r1car), NDr, w.Gr, {}};
    digit_gemm_group_ends(BL_SR, BL_SR, w.Gr, ra.rp1.ends.e);
  }
  if (radA) {
    DigitGemmArgs g{rA2, rB2, (int)M, (int)N, w.Kp, BL_SR, BL_SR, w.Gr, ws + w.r2dig,
                    (int32_t *)(ws + w.r2car), "digit_gemm_rad"};
    arbgpu_status stg = launch_digit_gemm(ctx, g, s);
    if (stg != ARBGPU_OK) return stg;
    ra.rp2 = IntProduct{ws + w.r2dig, (int32_t *)(ws + w.r2car), NDr, w.Gr, {}};
    digit_gemm_group_ends(BL_SR, BL_SR, w.Gr, ra.rp2.ends.e);
  }
  ra.rtop = rtop;
  ra.rbot = rbot;
  ra.rrad = rrad;
  ra.ctop = ctop;
  ra.cbot = cbot;
  ra.crad = crad;
  ra.cplus = cplus;
  ra.C = out_of(C);
  ra.M = M;
  ra.N = N;
  ra.ldc = ldc;
  ra.Mp = w.Mp;
  ra.Np = w.Np;
  ra.prec = prec;
  {
    LaunchScope sc(ctx, s, "block_round", M * N);
    block_round_kernel<<<(unsigned)((M * N + 127) / 128), 128, 0, s>>>(ra);
  }
  *used_block = true;
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

}  // namespace arbgpu
