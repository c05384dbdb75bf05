// arbgpu_series_exp: the power series exponential by the dot-product recurrence of Section V
// ("The power series exponential ... uses the dot product-friendly recurrence"):
//
//   exp(a_1 x + a_2 x^2 + ...) = b_0 + b_1 x + b_2 x^2 + ...,   b_0 = 1,
//   b_k = (sum_{j=1}^k (j a_j) b_{k-j}) / k,
//
// for many series at once.  Coefficient k of series s sits at index k * batch + s, so that the
// coefficients of one step form one contiguous batch of the ball dot kernel (Algorithm 1):
//   1. a'_j = j a_j for every j and s: one batched dot of length 1 against the exact balls j;
//   2. per k = 1 .. len - 1: c_k = sum_j a'_j b_{k-j} (a batched dot of length k, b read
//      backwards with a negative stride), then b_k = c_k * [1/k] (a dot of length 1 against a
//      ball that contains 1/k).
// Every step is a rigorous ball operation, so every output ball contains the exact coefficient
// for every choice of input points.
#include <cstring>

#include "internal.h"

namespace arbgpu {

// The exact ball of the integer v >= 0 at index i, v = i / per.
__global__ void index_int_balls_kernel(BallsOut o, int64_t n, int64_t per) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t v = (uint64_t)(i / per);
  for (int q = 0; q < o.nlimbs; ++q) o.limbs[(int64_t)q * o.stride + i] = 0;
  o.rad_man[i] = 0;
  o.rad_exp[i] = 0;
  if (v == 0) {
    o.exp[i] = 0;
    o.flags[i] = ARBGPU_FLAG_ZERO;
    return;
  }
  const int bl = 64 - __clzll((long long)v);
  o.limbs[(int64_t)(o.nlimbs - 1) * o.stride + i] = v << (64 - bl);
  o.exp[i] = bl;
  o.flags[i] = 1u << ARBGPU_NSIG_SHIFT;
}

// A ball containing 1/k at index k (k >= 1; index 0 gets zero): the first 64 (nlimbs + 1) bits of
// the binary expansion of 1/k by long division, normalised, the top nlimbs limbs kept (rounded
// toward zero), radius one unit of the last kept limb when anything nonzero was dropped.
__global__ void reciprocal_balls_kernel(BallsOut o, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int nl = o.nlimbs;
  for (int q = 0; q < nl; ++q) o.limbs[(int64_t)q * o.stride + k] = 0;
  o.rad_man[k] = 0;
  o.rad_exp[k] = 0;
  if (k == 0) {
    o.exp[k] = 0;
    o.flags[k] = ARBGPU_FLAG_ZERO;
    return;
  }
  const uint64_t d = (uint64_t)k;
  if ((d & (d - 1)) == 0) {  // a power of two: exact
    o.limbs[(int64_t)(nl - 1) * o.stride + k] = (uint64_t)1 << 63;
    o.exp[k] = 1 - (63 - __clzll((long long)d));
    o.flags[k] = 1u << ARBGPU_NSIG_SHIFT;
    return;
  }
  // F = floor(2^(64 (nl + 1)) / d), limbs F[nl] (top) .. F[0]; rem = the division's remainder
  uint64_t F[65];
  uint64_t rem = 1;  // the leading "1" of 2^(64 (nl + 1)), one limb above F[nl]
  for (int q = nl; q >= 0; --q) {
    const unsigned __int128 num = ((unsigned __int128)rem << 64);
    F[q] = (uint64_t)(num / d);
    rem = (uint64_t)(num % d);
  }
  // normalise: F[nl] >= 1 since d < 2^63 here
  const int s = __clzll((long long)F[nl]);
  bool lost = rem != 0;
  uint64_t M[64];
  for (int q = 0; q < nl; ++q) {  // limbs 1 .. nl of F << s
    const uint64_t hi = F[q + 1], lo = F[q];
    M[q] = s ? ((hi << s) | (lo >> (64 - s))) : hi;
  }
  const uint64_t low = s ? (F[0] << s) : F[0];  // the part of limb 0 that is dropped
  lost = lost || low != 0;
  int nsig = 0;
  for (int q = 0; q < nl; ++q) {
    o.limbs[(int64_t)q * o.stride + k] = M[q];
    if (M[q] && nsig == 0) nsig = nl - q;
  }
  // 1/k ~ M 2^(-64 nl - s): exponent -s
  o.exp[k] = -s;
  o.flags[k] = (uint32_t)nsig << ARBGPU_NSIG_SHIFT;
  if (lost) {  // the dropped part is below 2^(exp - 64 nl)
    o.rad_man[k] = 1u << 29;
    o.rad_exp[k] = -s - 64LL * nl + 1;
  }
}

// b_0 = 1 for every series (indices [0, batch)).
__global__ void one_balls_kernel(BallsOut o, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = 0; q < o.nlimbs; ++q)
    o.limbs[(int64_t)q * o.stride + i] = q == o.nlimbs - 1 ? ((uint64_t)1 << 63) : 0;
  o.exp[i] = 1;
  o.flags[i] = 1u << ARBGPU_NSIG_SHIFT;
  o.rad_man[i] = 0;
  o.rad_exp[i] = 0;
}

// Dot descriptors of every step, [len][batch] each: step k, series s.
//   sum:   x = a' from index batch + s with stride batch, y = b from (k - 1) batch + s with stride
//          -batch, length k;
//   scale: x = c from s, y = [1/k] at index k, length 1 (strides from `zero`).
// Step 0 (unused) gets length 0.  The precomputation a'_j = j a_j reads x = a at i (an iota) and
// y = the integer ball j at cyoff[i] = i / batch = j.
struct SeriesDesc {
  int64_t *xoff, *xstep, *yoff, *ystep, *len;  // sum
  int64_t *cxoff, *cyoff, *one, *zero;         // scale: offsets, the constants 1 and 0
  int32_t *prec;
};

__global__ void series_desc_kernel(SeriesDesc d, int64_t len, int64_t batch, int prec) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len * batch) return;
  const int64_t k = i / batch, s = i - k * batch;
  d.xoff[i] = batch + s;
  d.xstep[i] = batch;
  d.yoff[i] = k >= 1 ? (k - 1) * batch + s : 0;
  d.ystep[i] = -batch;
  d.len[i] = k;
  d.cxoff[i] = s;
  d.cyoff[i] = k;
  d.one[i] = 1;
  d.zero[i] = 0;
  d.prec[i] = prec;
}

struct SeriesWs {
  size_t ap, jb, inv, c, xoff, xstep, yoff, ystep, len, cxoff, cyoff, one, zero, prec, idx, total;
};

static size_t ball_bytes(int64_t count, int nl) {
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t c = (size_t)(count > 0 ? count : 1);
  return al(8 * c * nl) + al(8 * c) + al(4 * c) + al(4 * c) + al(8 * c);
}

static arbgpu_balls ball_at(uint8_t *base, int64_t count, int nl) {
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t c = (size_t)(count > 0 ? count : 1);
  arbgpu_balls b{};
  b.limbs = (uint64_t *)base;
  b.limb_stride = (int64_t)c;
  b.nlimbs = nl;
  size_t o = al(8 * c * nl);
  b.exp = (int64_t *)(base + o);
  o += al(8 * c);
  b.flags = (uint32_t *)(base + o);
  o += al(4 * c);
  b.rad_man = (uint32_t *)(base + o);
  o += al(4 * c);
  b.rad_exp = (int64_t *)(base + o);
  b.count = count;
  return b;
}

static SeriesWs series_ws(int64_t len, int64_t batch, int nl) {
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  SeriesWs w{};
  size_t off = 0;
  auto take = [&](size_t n) {
    const size_t o = off;
    off += al(n);
    return o;
  };
  const size_t n = (size_t)(len * batch);
  w.ap = take(ball_bytes(len * batch, nl));
  w.jb = take(ball_bytes(len, 1));
  w.inv = take(ball_bytes(len, nl));
  w.c = take(ball_bytes(batch, nl));
  w.xoff = take(8 * n);
  w.xstep = take(8 * n);
  w.yoff = take(8 * n);
  w.ystep = take(8 * n);
  w.len = take(8 * n);
  w.cxoff = take(8 * n);
  w.cyoff = take(8 * n);
  w.one = take(8 * n);
  w.zero = take(8 * n);
  w.prec = take(4 * n);
  w.idx = take(8 * n);
  w.total = off;
  return w;
}

// x offsets of the precomputation: x[i] = i.
__global__ void iota_kernel(int64_t *xo, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  xo[i] = i;
}

}  // namespace arbgpu

using namespace arbgpu;

extern "C" {

arbgpu_status arbgpu_series_exp_workspace_size(arbgpu_ctx *ctx, int64_t len, int64_t batch,
                                               int32_t prec, size_t *bytes) {
  if (!ctx || !bytes || len < 0 || batch < 0 || prec < 2 || prec > 1024) return ARBGPU_ERR_INVALID;
  *bytes = (len == 0 || batch == 0) ? 0 : series_ws(len, batch, (prec + 63) / 64 + 1).total;
  return ARBGPU_OK;
}

}  // extern "C"

namespace {

// The launches of one exponential call (checked arguments) on stream s.
arbgpu_status series_exp_launches(arbgpu_ctx *ctx, const arbgpu_balls *res, const arbgpu_balls *a,
                                  int64_t len, int64_t batch, int32_t prec, uint8_t *ws,
                                  const SeriesWs &w, int nl, cudaStream_t s) {
  const int64_t n = len * batch;
  const unsigned gn = (unsigned)((n + 255) / 256), gl = (unsigned)((len + 255) / 256);
  arbgpu_balls ap = ball_at(ws + w.ap, n, nl), jb = ball_at(ws + w.jb, len, 1);
  arbgpu_balls inv = ball_at(ws + w.inv, len, nl), c = ball_at(ws + w.c, batch, nl);
  SeriesDesc d{(int64_t *)(ws + w.xoff),  (int64_t *)(ws + w.xstep), (int64_t *)(ws + w.yoff),
               (int64_t *)(ws + w.ystep), (int64_t *)(ws + w.len),   (int64_t *)(ws + w.cxoff),
               (int64_t *)(ws + w.cyoff), (int64_t *)(ws + w.one),   (int64_t *)(ws + w.zero),
               (int32_t *)(ws + w.prec)};
  int64_t *idx = (int64_t *)(ws + w.idx);
  {
    LaunchScope sc(ctx, s, "series_desc", n);
    series_desc_kernel<<<gn, 256, 0, s>>>(d, len, batch, prec);
  }
  {
    LaunchScope sc(ctx, s, "series_consts", len);
    index_int_balls_kernel<<<gl, 256, 0, s>>>(out_of(jb), len, 1);
  }
  {
    LaunchScope sc(ctx, s, "series_consts", len);
    reciprocal_balls_kernel<<<gl, 256, 0, s>>>(out_of(inv), len);
  }
  {
    LaunchScope sc(ctx, s, "series_desc", n);
    iota_kernel<<<gn, 256, 0, s>>>(idx, n);
  }
  if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  // 1. a'_j = j a_j (every j, every series; j = 0 gives zero): x = a at i, y = the ball j at
  //    d.cyoff[i] = i / batch, length 1
  arbgpu_status st = launch_batched_dot(ctx, &ap, nullptr, nullptr, a, idx, d.zero, &jb, d.cyoff,
                                        d.zero, d.one, d.prec, n, prec, 1, 0, s);
  if (st != ARBGPU_OK) return st;
  {
    LaunchScope sc(ctx, s, "series_consts", batch);
    one_balls_kernel<<<(unsigned)((batch + 255) / 256), 256, 0, s>>>(out_of(*res), batch);
    if (cudaGetLastError() != cudaSuccess) return ARBGPU_ERR_CUDA;
  }
  // 2. the recurrence, one coefficient of every series per step
  for (int64_t k = 1; k < len; ++k) {
    const int64_t o = k * batch;
    st = launch_batched_dot(ctx, &c, nullptr, nullptr, &ap, d.xoff + o, d.xstep + o, res,
                            d.yoff + o, d.ystep + o, d.len + o, d.prec + o, batch, prec, k, 0, s,
                            false, false, true);
    if (st != ARBGPU_OK) return st;
    arbgpu_balls rk = *res;  // coefficient k of every series: indices [k batch, (k + 1) batch)
    rk.limbs += o;
    rk.exp += o;
    rk.flags += o;
    rk.rad_man += o;
    rk.rad_exp += o;
    rk.count = batch;
    st = launch_batched_dot(ctx, &rk, nullptr, nullptr, &c, d.cxoff + o, d.zero + o, &inv,
                            d.cyoff + o, d.zero + o, d.one + o, d.prec + o, batch, prec, 1, 0, s,
                            false, false, true);
    if (st != ARBGPU_OK) return st;
  }
  return ARBGPU_OK;
}

constexpr size_t SERIES_GRAPHS_KEPT = 4;

}  // namespace

extern "C" {

arbgpu_status arbgpu_series_exp(arbgpu_ctx *ctx, const arbgpu_balls *res, const arbgpu_balls *a,
                                int64_t len, int64_t batch, int32_t prec, void *workspace,
                                size_t ws_bytes, void *stream) {
  if (!ctx || !res || !a || len < 0 || batch < 0 || prec < 2 || prec > 1024)
    return ARBGPU_ERR_INVALID;
  if (len == 0 || batch == 0) return ARBGPU_OK;
  if ((int64_t)res->nlimbs * 64 < prec || res->count < len * batch || a->count < len * batch ||
      res->limb_stride < res->count || a->limb_stride < a->count || !res->limbs || !a->limbs ||
      !balls_ok(*res) || !balls_ok(*a) || balls_alias(*res, *a))
    return ARBGPU_ERR_INVALID;
  if (len > ((int64_t)1 << 24) || len * batch > ((int64_t)1 << 34)) return ARBGPU_ERR_LIMIT;
  const int nl = (prec + 63) / 64 + 1;  // working balls: one guard limb over the output
  const SeriesWs w = series_ws(len, batch, nl);
  if (!workspace || ws_bytes < w.total) return ARBGPU_ERR_WORKSPACE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ARBGPU_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t *ws = (uint8_t *)workspace;
  // Replay of the recorded launches when this call's arguments were seen before; direct launches
  // while tracing, while `s` is itself being captured, or with ARBGPU_SERIES_GRAPH=0.
  const char *e = getenv("ARBGPU_SERIES_GRAPH");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (ctx->trace || (e && !strcmp(e, "0")) || cudaStreamIsCapturing(s, &cap) != cudaSuccess ||
      cap != cudaStreamCaptureStatusNone)
    return series_exp_launches(ctx, res, a, len, batch, prec, ws, w, nl, s);
  const std::vector<uintptr_t> key{
      (uintptr_t)res->limbs, (uintptr_t)res->exp,     (uintptr_t)res->flags,
      (uintptr_t)res->rad_man, (uintptr_t)res->rad_exp, (uintptr_t)res->limb_stride,
      (uintptr_t)res->nlimbs, (uintptr_t)a->limbs,     (uintptr_t)a->exp,
      (uintptr_t)a->flags,   (uintptr_t)a->rad_man,   (uintptr_t)a->rad_exp,
      (uintptr_t)a->limb_stride, (uintptr_t)a->nlimbs, (uintptr_t)len,
      (uintptr_t)batch,      (uintptr_t)prec,         (uintptr_t)workspace};
  auto &gs = ctx->series_graphs;
  for (size_t q = 0; q < gs.size(); ++q)
    if (gs[q].key == key) {
      if (cudaGraphLaunch(gs[q].exec, s) != cudaSuccess) return ARBGPU_ERR_CUDA;
      ctx->launches += gs[q].kernels;
      return ARBGPU_OK;
    }
  // record: the launches on a private stream under capture, then one replay on `s`
  if (!ctx->capture_stream &&
      cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  cudaStream_t cs = ctx->capture_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  const int64_t l0 = ctx->launches;
  const arbgpu_status st = series_exp_launches(ctx, res, a, len, batch, prec, ws, w, nl, cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  const int64_t kernels = ctx->launches - l0;
  ctx->launches = l0;  // counted when the graph runs
  if (st != ARBGPU_OK || ce != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return st != ARBGPU_OK ? st : ARBGPU_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return ARBGPU_ERR_CUDA;
  if (gs.size() >= SERIES_GRAPHS_KEPT) {
    cudaGraphExecDestroy(gs.front().exec);
    gs.erase(gs.begin());
  }
  gs.push_back({key, exec, kernels});
  if (cudaGraphLaunch(exec, s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  ctx->launches += kernels;
  return ARBGPU_OK;
}

}  // extern "C"
