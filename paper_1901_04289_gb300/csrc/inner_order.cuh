// One entry of the reordered, scaled operand copies of the inner ordering (Section IV-B's
// suggested inner scaling combined with a permutation of the inner index), for the GPU kernel in
// block.cu and for host-side tests alike.
#pragma once

#include "common.cuh"

namespace arbgpu {

// Entry idx of the copy: A'[i, t] = A[i, ord[t]] 2^g[ord[t]] (rows x K, row-major with leading
// dimension K) or, for B, B'[t, j] = B[ord[t], j] 2^-g[ord[t]] (K x cols).  Midpoint and radius
// exponents move by the same amount, so the ball is scaled exactly.  Returns true when a moved
// exponent leaves the fast path's range (the caller then keeps the original order).
__host__ __device__ inline bool gather_inner_entry(const BallsView &X, int64_t ld, bool is_b,
                                                   int64_t K, int64_t cols, const int32_t *ord,
                                                   const int64_t *g, const BallsOut &Y,
                                                   int64_t idx) {
  int64_t src, k;
  if (is_b) {
    const int64_t t = idx / cols, j = idx - t * cols;
    k = ord[t];
    src = k * ld + j;
  } else {
    const int64_t i = idx / K, t = idx - i * K;
    k = ord[t];
    src = i * ld + k;
  }
  const int64_t d = is_b ? -g[k] : g[k];
  for (int q = 0; q < X.nlimbs; ++q)
    Y.limbs[(int64_t)q * Y.stride + idx] = X.limbs[(int64_t)q * X.stride + src];
  const uint32_t fl = X.flags[src];
  const uint32_t rm = X.rad_man[src];
  const int64_t e = X.exp[src], re = X.rad_exp[src];
  const bool mid = !(fl & (ARBGPU_FLAG_ZERO | SPECIAL_MASK));
  const int64_t e2 = mid ? e + d : e, re2 = rm ? re + d : re;
  Y.flags[idx] = fl;
  Y.exp[idx] = e2;
  Y.rad_man[idx] = rm;
  Y.rad_exp[idx] = re2;
  return (mid && (e2 >= EXP_LIMIT || e2 <= -EXP_LIMIT)) ||
         (rm && (re2 >= EXP_LIMIT || re2 <= -EXP_LIMIT));
}

}  // namespace arbgpu
