// Term sources of kernel (a) and the launch sequence shared by its callers: batched dots (arb_dot /
// acb_dot counterparts, Section III), the classical matrix product as M*N dots (Section IV), the
// basecase blocks of Algorithm 2 and grouped classical products.  Each source is compiled in its
// own translation unit (dot_*.cu).
#pragma once

#include "dot_eval.cuh"
#include "internal.h"

namespace arbgpu {

// Batched dots: dot b reads x[xoff[b] + i*xstep[b]] and y[yoff[b] + i*ystep[b]], i < len[b].
// A complex dot b is two virtual real dots (2b: real part, 2b+1: imaginary part) of length 2N:
// re = sum a c - b d, im = sum a d + b c (Section III-F).
struct BatchDotSrc {
  bool approx;  // midpoints only (radii ignored, zero output radii)
  bool reduce;  // the precision reduction ("optimize p") of Section III-C
  BallsView x[2], y[2], init[2];
  BallsOut out[2];
  const int64_t *xoff, *xstep, *yoff, *ystep, *len;
  const int32_t *precs;
  const uint8_t *subs;
  int64_t batch;
  int cplx;
  bool has_init;
  int prec_max;
  int64_t len_max;
  int64_t ndots_host;

  struct Cursor {
    int64_t b, xo, xs, yo, ys, n;
    int part;
    bool sub;
  };
  __device__ int64_t ndots() const { return cplx ? 2 * batch : batch; }
  __device__ Cursor cursor(int64_t d) const {
    Cursor c;
    c.b = cplx ? (d >> 1) : d;
    c.part = cplx ? (int)(d & 1) : 0;
    c.xo = __ldg(xoff + c.b);
    c.xs = __ldg(xstep + c.b);
    c.yo = __ldg(yoff + c.b);
    c.ys = __ldg(ystep + c.b);
    c.n = __ldg(len + c.b);
    c.sub = subs ? (__ldg(subs + c.b) != 0) : false;
    return c;
  }
  __device__ int64_t nterms(const Cursor &c) const { return cplx ? 2 * c.n : c.n; }
  __device__ TermLoc term(const Cursor &c, int64_t t) const {
    if (!cplx) return TermLoc{0, c.xo + t * c.xs, 0, c.yo + t * c.ys, c.sub};
    const int64_t i = t >> 1;
    const int w = (int)(t & 1);
    const int64_t xi = c.xo + i * c.xs, yi = c.yo + i * c.ys;
    if (c.part == 0) return w == 0 ? TermLoc{0, xi, 0, yi, c.sub} : TermLoc{1, xi, 1, yi, !c.sub};
    return w == 0 ? TermLoc{0, xi, 1, yi, c.sub} : TermLoc{1, xi, 0, yi, c.sub};
  }
  __device__ const BallsView &xview(const Cursor &, int a) const { return x[a]; }
  __device__ const BallsView &yview(const Cursor &, int a) const { return y[a]; }
  __device__ bool has_initial() const { return has_init; }
  __device__ const BallsView &initial_view(const Cursor &c) const { return init[c.part]; }
  __device__ int64_t initial_index(const Cursor &c) const { return c.b; }
  __device__ const BallsOut &out_view(const Cursor &c) const { return out[c.part]; }
  __device__ int64_t out_index(const Cursor &c) const { return c.b; }
  __device__ int prec(const Cursor &c) const { return __ldg(precs + c.b); }
  int64_t units() const { return ndots_host; }
};

// Classical product: entry (i, j) is the dot of row i of A and column j of B.  Consecutive warps
// take consecutive j, so the lanes' reads of B rows are shared through L1.
struct MatDotSrc {
  static constexpr bool approx = false;
  static constexpr bool reduce = false;
  BallsView A[2], B[2];
  BallsOut C[2];
  int64_t M, K, N, lda, ldb, ldc;
  int prec_v;
  int cplx;
  int prec_max;
  int64_t len_max;

  struct Cursor {
    int64_t xrow, j, oi;
    int part;
  };
  __device__ int64_t ndots() const { return (cplx ? 2 : 1) * M * N; }
  __device__ Cursor cursor(int64_t d) const {
    Cursor c;
    const int64_t e = cplx ? (d >> 1) : d;
    c.part = cplx ? (int)(d & 1) : 0;
    const int64_t i = e / N;
    c.j = e - i * N;
    c.xrow = i * lda;
    c.oi = i * ldc + c.j;
    return c;
  }
  __device__ int64_t nterms(const Cursor &) const { return cplx ? 2 * K : K; }
  __device__ TermLoc term(const Cursor &c, int64_t t) const {
    if (!cplx) return TermLoc{0, c.xrow + t, 0, t * ldb + c.j, false};
    const int64_t k = t >> 1;
    const int w = (int)(t & 1);
    const int64_t xi = c.xrow + k, yi = k * ldb + c.j;
    if (c.part == 0) return w == 0 ? TermLoc{0, xi, 0, yi, false} : TermLoc{1, xi, 1, yi, true};
    return w == 0 ? TermLoc{0, xi, 1, yi, false} : TermLoc{1, xi, 0, yi, false};
  }
  __device__ const BallsView &xview(const Cursor &, int a) const { return A[a]; }
  __device__ const BallsView &yview(const Cursor &, int a) const { return B[a]; }
  __device__ bool has_initial() const { return false; }
  __device__ const BallsView &initial_view(const Cursor &) const { return A[0]; }
  __device__ int64_t initial_index(const Cursor &) const { return 0; }
  __device__ const BallsOut &out_view(const Cursor &c) const { return C[c.part]; }
  __device__ int64_t out_index(const Cursor &c) const { return c.oi; }
  __device__ int prec(const Cursor &) const { return prec_v; }
  int64_t units() const { return M * N * K; }
};

// The basecase of Algorithm 2: entry (i, j) sums +- X[i, k] Y[k, j] over the tagged inner indices
// in bk (the basecase blocks of each real product), starting from the accumulated block products
// as `initial`.
struct BasecaseSrc {
  static constexpr bool approx = false;
  static constexpr bool reduce = false;
  BallsView A[2], B[2], init;
  BallsOut C;
  const int32_t *bk;
  int64_t nbk, M, N, lda, ldb, ldc;
  int prec_v;
  int prec_max;
  int64_t len_max;

  struct Cursor {
    int64_t d, xrow, j, oi;
  };
  __device__ int64_t ndots() const { return M * N; }
  __device__ Cursor cursor(int64_t d) const {
    Cursor c;
    const int64_t i = d / N;
    c.d = d;
    c.j = d - i * N;
    c.xrow = i * lda;
    c.oi = i * ldc + c.j;
    return c;
  }
  __device__ int64_t nterms(const Cursor &) const { return nbk; }
  __device__ TermLoc term(const Cursor &c, int64_t t) const {
    const int32_t e = __ldg(bk + t);
    const int64_t k = e >> 2;
    const int combo = e & 3;
    const int xa = (combo == 1 || combo == 3) ? 1 : 0;
    const int yb = (combo == 1 || combo == 2) ? 1 : 0;
    return TermLoc{xa, c.xrow + k, yb, k * ldb + c.j, combo == 1};
  }
  __device__ const BallsView &xview(const Cursor &, int a) const { return A[a]; }
  __device__ const BallsView &yview(const Cursor &, int b) const { return B[b]; }
  __device__ bool has_initial() const { return true; }
  __device__ const BallsView &initial_view(const Cursor &) const { return init; }
  __device__ int64_t initial_index(const Cursor &c) const { return c.d; }
  __device__ const BallsOut &out_view(const Cursor &) const { return C; }
  __device__ int64_t out_index(const Cursor &c) const { return c.oi; }
  __device__ int prec(const Cursor &) const { return prec_v; }
  int64_t units() const { return M * N * nbk; }
};

// Grouped classical products: virtual dot d belongs to the item q with ends[q-1] <= d < ends[q]
// (binary search over a device work list); inside the item it is entry (i, j) (and, for complex
// items, its part).
struct GroupedDotSrc {
  static constexpr bool approx = false;
  static constexpr bool reduce = false;
  const GroupItem *items;
  const int64_t *ends;
  int32_t count;
  int64_t total;
  int prec_max;
  int64_t len_max;

  struct Cursor {
    const GroupItem *it;
    int64_t xrow, j, oi;
    int part;
  };
  __device__ int item(int64_t d) const {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(ends + mid) > d) hi = mid;
      else lo = mid + 1;
    }
    return lo;
  }
  __device__ int64_t ndots() const { return total; }
  __device__ Cursor cursor(int64_t d) const {
    Cursor c;
    const int q = item(d);
    c.it = items + q;
    const int64_t e0 = d - (q ? __ldg(ends + q - 1) : 0);
    const bool cx = c.it->cplx != 0;
    c.part = cx ? (int)(e0 & 1) : 0;
    const int64_t e = cx ? (e0 >> 1) : e0;
    const int64_t N = c.it->N;
    const int64_t i = e / N;
    c.j = e - i * N;
    c.xrow = i * c.it->lda;
    c.oi = i * c.it->ldc + c.j;
    return c;
  }
  __device__ int64_t nterms(const Cursor &c) const { return c.it->cplx ? 2 * c.it->K : c.it->K; }
  __device__ TermLoc term(const Cursor &c, int64_t t) const {
    const int64_t ldb = c.it->ldb;
    if (!c.it->cplx) return TermLoc{0, c.xrow + t, 0, t * ldb + c.j, false};
    const int64_t k = t >> 1;
    const int w = (int)(t & 1);
    const int64_t xi = c.xrow + k, yi = k * ldb + c.j;
    if (c.part == 0) return w == 0 ? TermLoc{0, xi, 0, yi, false} : TermLoc{1, xi, 1, yi, true};
    return w == 0 ? TermLoc{0, xi, 1, yi, false} : TermLoc{1, xi, 0, yi, false};
  }
  __device__ const BallsView &xview(const Cursor &c, int a) const { return c.it->A[a]; }
  __device__ const BallsView &yview(const Cursor &c, int b) const { return c.it->B[b]; }
  __device__ bool has_initial() const { return false; }
  __device__ const BallsView &initial_view(const Cursor &c) const { return c.it->A[0]; }
  __device__ int64_t initial_index(const Cursor &) const { return 0; }
  __device__ const BallsOut &out_view(const Cursor &c) const { return c.it->C[c.part]; }
  __device__ int64_t out_index(const Cursor &c) const { return c.oi; }
  __device__ int prec(const Cursor &c) const { return c.it->prec; }
  int64_t units() const { return total; }
};

// Lanes per dot.  Matrix-shaped sources take 4 lanes per entry: a warp then evaluates eight
// neighbouring entries of a row of C at once, and at every step their groups read neighbouring
// entries of a row of B (coalesced) and the same entries of A.  Batched dots with unit strides are
// coalesced within a group, so they take whole warps unless they are short.
inline int dot_group_matrix() { return 4; }
inline int dot_group_batched(int64_t terms) {
  return terms >= 128 ? 32 : (terms >= 64 ? 16 : (terms >= 32 ? 8 : 4));
}

template <int C, int G, class Src>
static void launch_eval(const Src &src, unsigned blocks, int chunk, cudaStream_t stream) {
  dot_eval_kernel<C, G, Src><<<blocks, 256, 0, stream>>>(src, chunk);
}

// Evaluation launches of classes 0..cmax; the classes of long products (5 and up) always take
// whole warps.
template <int G, class Src>
static arbgpu_status launch_dot_group(arbgpu_ctx *ctx, const Src &src, int64_t ndots, int cmax,
                                      cudaStream_t stream) {
  constexpr int DPW = 32 / G;
  const int threads = 256;
  const int64_t cap = (int64_t)ctx->sm_count * 16;
  {
    int64_t blocks = (ndots + 8 * DPW - 1) / (8 * DPW);
    if (blocks > cap) blocks = cap;
    LaunchScope scope(ctx, stream, "dot_setup", src.units());
    dot_setup_kernel<G, Src><<<(unsigned)blocks, threads, 0, stream>>>(src, cmax, ctx->status);
    if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  }
  // chunks of DPW to 8 DPW dots per warp step (at most DOT_CHUNK): as many as keeps every SM busy
  const int64_t most = 8 * DPW < DOT_CHUNK ? 8 * DPW : DOT_CHUNK;
  int64_t chunk = ndots / ((int64_t)ctx->sm_count * 32);
  chunk = chunk < DPW ? DPW : (chunk > most ? most : chunk);
  const int64_t chunks = (ndots + chunk - 1) / chunk;
  int64_t blocks = (chunks + 7) / 8;
  if (blocks > cap) blocks = cap;
  const unsigned b = (unsigned)blocks;
  const int ck = (int)chunk;
  for (int c = 0; c <= cmax; ++c) {
    LaunchScope scope(ctx, stream, "dot_eval", c == cmax ? src.units() : 0);
    switch (c) {
      case 0: launch_eval<0, G>(src, b, ck, stream); break;
      case 1: launch_eval<1, G>(src, b, ck, stream); break;
      case 2: launch_eval<2, G>(src, b, ck, stream); break;
      case 3: launch_eval<3, G>(src, b, ck, stream); break;
      case 4: launch_eval<4, G>(src, b, ck, stream); break;
      case 5: launch_eval<5, 32>(src, b, ck, stream); break;
      case 6: launch_eval<6, 32>(src, b, ck, stream); break;
      case 7: launch_eval<7, 32>(src, b, ck, stream); break;
      default: return ARBGPU_ERR_INVALID;
    }
    if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  }
  return ARBGPU_OK;
}

// Setup launch, then one evaluation launch per size class up to cmax, with `group` lanes per dot.
template <class Src>
static arbgpu_status launch_dot_src(arbgpu_ctx *ctx, const Src &src, int64_t ndots, int cmax,
                                    int group, cudaStream_t stream) {
  if (ndots <= 0) return ARBGPU_OK;
  switch (group) {
    case 4: return launch_dot_group<4>(ctx, src, ndots, cmax, stream);
    case 8: return launch_dot_group<8>(ctx, src, ndots, cmax, stream);
    case 16: return launch_dot_group<16>(ctx, src, ndots, cmax, stream);
    default: return launch_dot_group<32>(ctx, src, ndots, cmax, stream);
  }
}

template <int C, int G, class Src>
static void launch_fused(const Src &src, unsigned blocks, int *status, cudaStream_t stream) {
  dot_fused_kernel<C, G, Src><<<blocks, 256, 0, stream>>>(src, status);
}

// One launch: setup and evaluation of every dot in class cmax, `group` lanes per dot.  For sources
// whose dots share one precision (a matrix product), where the class hardly varies.
template <class Src>
static arbgpu_status launch_dot_fused(arbgpu_ctx *ctx, const Src &src, int64_t ndots, int cmax,
                                      int group, cudaStream_t stream) {
  if (ndots <= 0) return ARBGPU_OK;
  const int G = cmax >= 5 ? 32 : group;
  const int64_t per_block = 8 * (32 / G);
  int64_t blocks = (ndots + per_block - 1) / per_block;
  const int64_t cap = (int64_t)ctx->sm_count * 16;
  if (blocks > cap) blocks = cap;
  const unsigned b = (unsigned)blocks;
  int *st = ctx->status;
  LaunchScope scope(ctx, stream, "dot_fused", src.units());
#define ARB_FUSED(C)                                             \
  switch (G) {                                                   \
    case 4: launch_fused<C, 4>(src, b, st, stream); break;       \
    case 8: launch_fused<C, 8>(src, b, st, stream); break;       \
    case 16: launch_fused<C, 16>(src, b, st, stream); break;     \
    default: launch_fused<C, 32>(src, b, st, stream); break;     \
  }
  switch (cmax) {
    case 0: ARB_FUSED(0); break;
    case 1: ARB_FUSED(1); break;
    case 2: ARB_FUSED(2); break;
    case 3: ARB_FUSED(3); break;
    case 4: ARB_FUSED(4); break;
    case 5: launch_fused<5, 32>(src, b, st, stream); break;
    case 6: launch_fused<6, 32>(src, b, st, stream); break;
    case 7: launch_fused<7, 32>(src, b, st, stream); break;
    default: return ARBGPU_ERR_INVALID;
  }
#undef ARB_FUSED
  return cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
}

}  // namespace arbgpu
