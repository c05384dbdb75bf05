// The C ABI of the arbgpu library: context, status word, argument checks and dispatch.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

using namespace arbgpu;

namespace arbgpu {

bool balls_ok(const arbgpu_balls &b) {
  if (b.count < 0 || b.nlimbs < 1 || b.nlimbs > 64) return false;
  if (b.count == 0) return true;
  if (!b.limbs || !b.exp || !b.flags || !b.rad_man || !b.rad_exp) return false;
  if (b.limb_stride < b.count) return false;
  return true;
}

bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
  const char *pa = (const char *)a, *pb = (const char *)b;
  return pa < pb + nb && pb < pa + na;
}

// True if any array of `out` shares memory with any array of `in`.
bool balls_alias(const arbgpu_balls &out, const arbgpu_balls &in) {
  if (out.count == 0 || in.count == 0) return false;
  const void *op[5] = {out.limbs, out.exp, out.flags, out.rad_man, out.rad_exp};
  const size_t on[5] = {(size_t)out.limb_stride * out.nlimbs * 8, (size_t)out.count * 8,
                        (size_t)out.count * 4, (size_t)out.count * 4, (size_t)out.count * 8};
  const void *ip[5] = {in.limbs, in.exp, in.flags, in.rad_man, in.rad_exp};
  const size_t in_[5] = {(size_t)in.limb_stride * in.nlimbs * 8, (size_t)in.count * 8,
                         (size_t)in.count * 4, (size_t)in.count * 4, (size_t)in.count * 8};
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j)
      if (overlaps(op[i], on[i], ip[j], in_[j])) return true;
  return false;
}

}  // namespace arbgpu

namespace arbgpu {

static cudaEvent_t pool_event(arbgpu_ctx *c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

LaunchScope::LaunchScope(arbgpu_ctx *c, cudaStream_t s, const char *name, int64_t units)
    : ctx(c), stream(s), idx(-1) {
  ctx->launches += 1;
  if (ctx->trace) {
    arbgpu_trace_rec r{name, pool_event(ctx), pool_event(ctx), units};
    cudaEventRecord(r.start, stream);
    ctx->recs.push_back(r);
    idx = (int)ctx->recs.size() - 1;
  }
}

LaunchScope::~LaunchScope() {
  if (idx >= 0) cudaEventRecord(ctx->recs[idx].stop, stream);
}

}  // namespace arbgpu

extern "C" {

arbgpu_status arbgpu_launch_count(arbgpu_ctx *ctx, int64_t *count) {
  if (!ctx || !count) return ARBGPU_ERR_INVALID;
  *count = ctx->launches;
  return ARBGPU_OK;
}

arbgpu_status arbgpu_trace_enable(arbgpu_ctx *ctx, int enable) {
  if (!ctx) return ARBGPU_ERR_INVALID;
  ctx->trace = enable != 0;
  return ARBGPU_OK;
}

arbgpu_status arbgpu_trace_read(arbgpu_ctx *ctx, arbgpu_trace_entry *out, int32_t max_entries,
                                int32_t *n_entries) {
  if (!ctx || !n_entries || (max_entries > 0 && !out)) return ARBGPU_ERR_INVALID;
  int32_t n = 0;
  const cudaEvent_t t0 = ctx->recs.empty() ? nullptr : ctx->recs.front().start;
  for (auto &r : ctx->recs) {
    if (cudaEventSynchronize(r.stop) != cudaSuccess) return ARBGPU_ERR_CUDA;
    if (n < max_entries) {
      float ms = 0.f, at = 0.f;
      cudaEventElapsedTime(&ms, r.start, r.stop);
      cudaEventElapsedTime(&at, t0, r.start);
      out[n].name = r.name;
      out[n].ms = ms;
      out[n].units = r.units;
      out[n].start_ms = at;
      ++n;
    }
    ctx->event_pool.push_back(r.start);
    ctx->event_pool.push_back(r.stop);
  }
  ctx->recs.clear();
  *n_entries = n;
  return ARBGPU_OK;
}

arbgpu_status arbgpu_set_autotune(arbgpu_ctx *ctx, int enable) {
  if (!ctx) return ARBGPU_ERR_INVALID;
  ctx->autotune = enable != 0;
  return ARBGPU_OK;
}

arbgpu_status arbgpu_autotune_stats(arbgpu_ctx *ctx, int64_t *buckets, int64_t *timing_runs,
                                    int64_t *crt_buckets) {
  if (!ctx) return ARBGPU_ERR_INVALID;
  int64_t crt = 0;
  for (const auto &kv : ctx->engine_tuned) crt += kv.second ? 1 : 0;
  if (buckets) *buckets = (int64_t)ctx->engine_tuned.size();
  if (timing_runs) *timing_runs = ctx->tune_runs;
  if (crt_buckets) *crt_buckets = crt;
  return ARBGPU_OK;
}

arbgpu_status arbgpu_autotune_alg_stats(arbgpu_ctx *ctx, int64_t *buckets, int64_t *timing_runs,
                                        int64_t *block_buckets) {
  if (!ctx) return ARBGPU_ERR_INVALID;
  int64_t blk = 0;
  for (const auto &kv : ctx->alg_tuned) blk += kv.second ? 1 : 0;
  if (buckets) *buckets = (int64_t)ctx->alg_tuned.size();
  if (timing_runs) *timing_runs = ctx->alg_tune_runs;
  if (block_buckets) *block_buckets = blk;
  return ARBGPU_OK;
}

int arbgpu_version(void) { return 100; }

const char *arbgpu_status_string(arbgpu_status s) {
  switch (s) {
    case ARBGPU_OK: return "ok";
    case ARBGPU_ERR_INVALID: return "invalid argument";
    case ARBGPU_ERR_UNSUPPORTED_VALUE: return "unsupported value (NaN, infinity or huge exponent)";
    case ARBGPU_ERR_WORKSPACE: return "workspace too small";
    case ARBGPU_ERR_CUDA: return "CUDA error";
    case ARBGPU_ERR_TIMEOUT: return "device wait timed out";
    case ARBGPU_ERR_LIMIT: return "size limit exceeded";
  }
  return "unknown status";
}

arbgpu_status arbgpu_create(arbgpu_ctx **ctx, int device) {
  if (!ctx) return ARBGPU_ERR_INVALID;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return ARBGPU_ERR_CUDA;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return ARBGPU_ERR_CUDA;
  arbgpu_ctx *c = new (std::nothrow) arbgpu_ctx();
  if (!c) return ARBGPU_ERR_INVALID;
  c->device = device;
  c->launches = 0;
  c->trace = false;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  // the status word and the mapped pinned buffer of the block path's statistics read-back (room
  // for the statistics of 256 block products; a larger batch grows it once)
  if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess ||
      cudaHostAlloc(&c->mapped, 4 * 256 * sizeof(BlockStats), cudaHostAllocMapped) !=
          cudaSuccess ||
      cudaHostGetDevicePointer(&c->mapped_dev, c->mapped, 0) != cudaSuccess ||
      cudaHostAlloc(&c->pub, 256, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&c->pub_dev, c->pub, 0) != cudaSuccess) {
    if (c->status) cudaFree(c->status);
    if (c->mapped) cudaFreeHost(c->mapped);
    if (c->pub) cudaFreeHost(c->pub);
    delete c;
    cudaSetDevice(prev);
    return ARBGPU_ERR_CUDA;
  }
  c->mapped_bytes = 4 * 256 * sizeof(BlockStats);
  memset(c->pub, 0, 256);
  cudaDeviceSynchronize();
  cudaSetDevice(prev);
  *ctx = c;
  return ARBGPU_OK;
}

arbgpu_status arbgpu_reserve(arbgpu_ctx *ctx, int32_t max_prec, int64_t max_inner) {
  if (!ctx || max_prec < 2 || max_prec > 1024 || max_inner < 1) return ARBGPU_ERR_INVALID;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ARBGPU_ERR_CUDA;
  const arbgpu_status st = block_reserve(ctx, max_prec, max_inner);
  cudaSetDevice(prev);
  return st;
}

arbgpu_status arbgpu_destroy(arbgpu_ctx *ctx) {
  if (!ctx) return ARBGPU_ERR_INVALID;
  for (auto &r : ctx->recs) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  for (auto &t : ctx->crt_tables) cudaFree(t.second);
  if (ctx->mapped) cudaFreeHost(ctx->mapped);
  if (ctx->pub) cudaFreeHost(ctx->pub);
  for (int l = 0; l < arbgpu_ctx::kLanes; ++l) {
    if (ctx->lanes[l]) cudaStreamDestroy(ctx->lanes[l]);
    if (ctx->lane_done[l]) cudaEventDestroy(ctx->lane_done[l]);
  }
  if (ctx->lane_fork) cudaEventDestroy(ctx->lane_fork);
  for (auto &g : ctx->series_graphs) cudaGraphExecDestroy(g.exec);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  cudaFree(ctx->status);
  delete ctx;
  return ARBGPU_OK;
}

arbgpu_status arbgpu_get_status(arbgpu_ctx *ctx, void *stream) {
  if (!ctx) return ARBGPU_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, ctx->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  if (v != 0) cudaMemset(ctx->status, 0, sizeof(int));
  return (arbgpu_status)v;
}

static arbgpu_status dot_entry(arbgpu_ctx *ctx, const arbgpu_balls *res,
                               const arbgpu_balls *initial, const uint8_t *sub,
                               const arbgpu_balls *x, const int64_t *xoff, const int64_t *xstep,
                               const arbgpu_balls *y, const int64_t *yoff, const int64_t *ystep,
                               const int64_t *len, const int32_t *prec, int64_t batch,
                               int32_t prec_max, int64_t len_max, int complex_mode,
                               void *workspace, size_t ws_bytes, void *stream, uint32_t options) {
  (void)workspace;
  (void)ws_bytes;
  if (!ctx || !res || !x || !y || batch < 0) return ARBGPU_ERR_INVALID;
  if (options & ~(ARBGPU_DOT_APPROX | ARBGPU_DOT_REDUCE_PREC)) return ARBGPU_ERR_INVALID;
  if (batch == 0) return ARBGPU_OK;
  if (!xoff || !xstep || !yoff || !ystep || !len || !prec) return ARBGPU_ERR_INVALID;
  if (prec_max < 2 || prec_max > 1024 || len_max < 0 || len_max > ((int64_t)1 << 40))
    return ARBGPU_ERR_INVALID;
  const int parts = complex_mode ? 2 : 1;
  for (int q = 0; q < parts; ++q) {
    if (!balls_ok(res[q]) || !balls_ok(x[q]) || !balls_ok(y[q])) return ARBGPU_ERR_INVALID;
    if (initial && !balls_ok(initial[q])) return ARBGPU_ERR_INVALID;
    if (res[q].count < batch) return ARBGPU_ERR_INVALID;
    if (initial && initial[q].count < batch) return ARBGPU_ERR_INVALID;
    if ((int64_t)res[q].nlimbs * 64 < prec_max) return ARBGPU_ERR_INVALID;
    for (int r = 0; r < parts; ++r) {
      if (balls_alias(res[q], x[r]) || balls_alias(res[q], y[r])) return ARBGPU_ERR_INVALID;
      if (initial && balls_alias(res[q], initial[r])) return ARBGPU_ERR_INVALID;
      if (r != q && balls_alias(res[q], res[r])) return ARBGPU_ERR_INVALID;
    }
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ARBGPU_ERR_CUDA;
  return launch_batched_dot(ctx, res, initial, sub, x, xoff, xstep, y, yoff, ystep, len, prec,
                            batch, prec_max, len_max, complex_mode, (cudaStream_t)stream,
                            (options & ARBGPU_DOT_APPROX) != 0,
                            (options & ARBGPU_DOT_REDUCE_PREC) != 0);
}

arbgpu_status arbgpu_dot(arbgpu_ctx *ctx, const arbgpu_balls *res, const arbgpu_balls *initial,
                         const uint8_t *sub, const arbgpu_balls *x, const int64_t *xoff,
                         const int64_t *xstep, const arbgpu_balls *y, const int64_t *yoff,
                         const int64_t *ystep, const int64_t *len, const int32_t *prec,
                         int64_t batch, int32_t prec_max, int64_t len_max, int complex_mode,
                         void *workspace, size_t ws_bytes, void *stream) {
  return dot_entry(ctx, res, initial, sub, x, xoff, xstep, y, yoff, ystep, len, prec, batch,
                   prec_max, len_max, complex_mode, workspace, ws_bytes, stream, 0u);
}

arbgpu_status arbgpu_dot_ex(arbgpu_ctx *ctx, const arbgpu_balls *res, const arbgpu_balls *initial,
                            const uint8_t *sub, const arbgpu_balls *x, const int64_t *xoff,
                            const int64_t *xstep, const arbgpu_balls *y, const int64_t *yoff,
                            const int64_t *ystep, const int64_t *len, const int32_t *prec,
                            int64_t batch, int32_t prec_max, int64_t len_max, int complex_mode,
                            uint32_t options, void *workspace, size_t ws_bytes, void *stream) {
  return dot_entry(ctx, res, initial, sub, x, xoff, xstep, y, yoff, ystep, len, prec, batch,
                   prec_max, len_max, complex_mode, workspace, ws_bytes, stream, options);
}

arbgpu_status arbgpu_approx_dot(arbgpu_ctx *ctx, const arbgpu_balls *res,
                                const arbgpu_balls *initial, const uint8_t *sub,
                                const arbgpu_balls *x, const int64_t *xoff, const int64_t *xstep,
                                const arbgpu_balls *y, const int64_t *yoff, const int64_t *ystep,
                                const int64_t *len, const int32_t *prec, int64_t batch,
                                int32_t prec_max, int64_t len_max, int complex_mode,
                                void *workspace, size_t ws_bytes, void *stream) {
  return dot_entry(ctx, res, initial, sub, x, xoff, xstep, y, yoff, ystep, len, prec, batch,
                   prec_max, len_max, complex_mode, workspace, ws_bytes, stream,
                   ARBGPU_DOT_APPROX);
}

// AUTO: the block algorithm from this size on (the paper's default cutoff lies at N = 40..60).
static bool auto_uses_block(int64_t M, int64_t K, int64_t N) {
  return M >= 48 && N >= 48 && K >= 48;
}

// AUTO with the autotuner on: around the crossover (both algorithms apply and neither dominates
// by construction) the choice is timed once per size bucket: M, K and N rounded up to powers of
// two, the precision in limbs, complex and eq. 2.
static bool auto_tunable(int64_t M, int64_t K, int64_t N) {
  return K >= 30 && M >= 8 && N >= 8 && M <= 512 && N <= 512 && K <= 512;
}

static int clog2(int64_t v) {
  int b = 0;
  while (((int64_t)1 << b) < v) ++b;
  return b;
}

static uint64_t alg_bucket(int64_t M, int64_t K, int64_t N, int prec, bool cplx, bool m3) {
  return (uint64_t)clog2(M) | (uint64_t)clog2(K) << 8 | (uint64_t)clog2(N) << 16 |
         (uint64_t)((prec + 63) / 64) << 24 | (uint64_t)(cplx ? 1 : 0) << 40 |
         (uint64_t)(m3 ? 1 : 0) << 41;
}

// The AUTO choice: 1 block, 0 classical dots, -1 a bucket the autotuner has yet to time.
static int auto_choice(const arbgpu_ctx *ctx, int64_t M, int64_t K, int64_t N, int prec,
                       bool cplx, bool m3) {
  if (ctx->autotune && auto_tunable(M, K, N)) {
    const auto it = ctx->alg_tuned.find(alg_bucket(M, K, N, prec, cplx, m3));
    return it == ctx->alg_tuned.end() ? -1 : (it->second ? 1 : 0);
  }
  return auto_uses_block(M, K, N) ? 1 : 0;
}

// Whether an AUTO product may run the block algorithm (so its workspace must hold it).
static bool auto_may_use_block(const arbgpu_ctx *ctx, int64_t M, int64_t K, int64_t N) {
  return auto_uses_block(M, K, N) || (ctx->autotune && auto_tunable(M, K, N));
}

// One product by the block algorithm (*used: it ran; false with ARBGPU_ERR_LIMIT when the
// inputs need the classical one) or by the classical dots.
static arbgpu_status run_matmul_alg(arbgpu_ctx *ctx, bool block, const arbgpu_balls *C,
                                    const arbgpu_balls *A, const arbgpu_balls *B, int64_t M,
                                    int64_t K, int64_t N, int64_t lda, int64_t ldb, int64_t ldc,
                                    int32_t prec, int complex_mode, uint32_t flags,
                                    void *workspace, size_t ws_bytes, cudaStream_t s,
                                    bool *used) {
  *used = false;
  if (block) {
    const arbgpu_status st =
        block_matmul(ctx, C, A, B, M, K, N, lda, ldb, ldc, prec, complex_mode != 0,
                     (flags & ARBGPU_MM_COMPLEX_3M) != 0, workspace, ws_bytes, s, used);
    if (*used || st != ARBGPU_ERR_LIMIT) return st;
  }
  return launch_matmul_dot(ctx, C, A, B, M, K, N, lda, ldb, ldc, prec, complex_mode, s);
}

// The first AUTO product of an undecided bucket: both algorithms once untimed, then once each
// timed with CUDA events on `s` (which this synchronises); the faster is kept for the bucket and
// its result is the one left in C.  No timing while `s` is being captured, nor when the block
// algorithm does not take these inputs (the fixed rule, or the dots, decide then).
static arbgpu_status tune_auto(arbgpu_ctx *ctx, const arbgpu_balls *C, const arbgpu_balls *A,
                               const arbgpu_balls *B, int64_t M, int64_t K, int64_t N,
                               int64_t lda, int64_t ldb, int64_t ldc, int32_t prec,
                               int complex_mode, uint32_t flags, void *workspace,
                               size_t ws_bytes, cudaStream_t s) {
  auto run = [&](bool block, bool *used) {
    return run_matmul_alg(ctx, block, C, A, B, M, K, N, lda, ldb, ldc, prec, complex_mode, flags,
                          workspace, ws_bytes, s, used);
  };
  bool used = false;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return run(auto_uses_block(M, K, N), &used);
  arbgpu_status st = run(true, &used);
  if (st == ARBGPU_ERR_WORKSPACE) return run(false, &used);  // (a workspace sized without it)
  if (st != ARBGPU_OK) return st;
  const uint64_t key =
      alg_bucket(M, K, N, prec, complex_mode != 0, (flags & ARBGPU_MM_COMPLEX_3M) != 0);
  // the inputs (special values, limits), not the sizes, sent this product to the classical
  // algorithm inside the block call: nothing to time, the bucket stays undecided
  if (!used) return ARBGPU_OK;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (auto &f : ev)
        if (f) cudaEventDestroy(f);
      return ARBGPU_ERR_CUDA;
    }
  bool u2 = false;
  float t_blk = 0.f, t_dot = 0.f;
  st = run(false, &u2);
  if (st == ARBGPU_OK && cudaEventRecord(ev[0], s) != cudaSuccess) st = ARBGPU_ERR_CUDA;
  if (st == ARBGPU_OK) st = run(true, &u2);
  if (st == ARBGPU_OK && cudaEventRecord(ev[1], s) != cudaSuccess) st = ARBGPU_ERR_CUDA;
  if (st == ARBGPU_OK) st = run(false, &u2);
  if (st == ARBGPU_OK && (cudaEventRecord(ev[2], s) != cudaSuccess ||
                          cudaEventSynchronize(ev[2]) != cudaSuccess ||
                          cudaEventElapsedTime(&t_blk, ev[0], ev[1]) != cudaSuccess ||
                          cudaEventElapsedTime(&t_dot, ev[1], ev[2]) != cudaSuccess))
    st = ARBGPU_ERR_CUDA;
  for (auto &e : ev) cudaEventDestroy(e);
  if (st != ARBGPU_OK) return st;
  const bool block_faster = t_blk < t_dot;
  ctx->alg_tuned[key] = block_faster;
  ctx->alg_tune_runs += 4;
  // the dots ran last; a block choice runs once more so that its result (and plan) is the one
  // the call leaves
  ctx->plan_log.clear();
  return block_faster ? run(true, &u2) : ARBGPU_OK;
}

arbgpu_status arbgpu_mat_mul_workspace_size(arbgpu_ctx *ctx, int64_t M, int64_t K, int64_t N,
                                            int32_t prec, int32_t a_nlimbs, int32_t b_nlimbs,
                                            int complex_mode, int alg, uint32_t flags,
                                            size_t *bytes) {
  if (!ctx || !bytes || M < 0 || K < 0 || N < 0 || prec < 2 || prec > 1024 || a_nlimbs < 1 ||
      b_nlimbs < 1 || a_nlimbs > 64 || b_nlimbs > 64)
    return ARBGPU_ERR_INVALID;
  if (flags & ~ARBGPU_MM_COMPLEX_3M) return ARBGPU_ERR_INVALID;
  *bytes = 0;
  if (alg == ARBGPU_ALG_DOT) return ARBGPU_OK;
  if (alg != ARBGPU_ALG_BLOCK && alg != ARBGPU_ALG_AUTO) return ARBGPU_ERR_INVALID;
  if (alg == ARBGPU_ALG_AUTO && !auto_may_use_block(ctx, M, K, N)) return ARBGPU_OK;
  *bytes = block_workspace_size(ctx, M, K, N, prec, complex_mode != 0,
                                (flags & ARBGPU_MM_COMPLEX_3M) != 0, a_nlimbs, b_nlimbs);
  return ARBGPU_OK;
}

arbgpu_status arbgpu_mat_mul(arbgpu_ctx *ctx, const arbgpu_balls *C, const arbgpu_balls *A,
                             const arbgpu_balls *B, int64_t M, int64_t K, int64_t N, int64_t lda,
                             int64_t ldb, int64_t ldc, int32_t prec, int complex_mode, int alg,
                             uint32_t flags, void *workspace, size_t ws_bytes, void *stream) {
  if (!ctx || !C || !A || !B || M < 0 || K < 0 || N < 0) return ARBGPU_ERR_INVALID;
  if (flags & ~ARBGPU_MM_COMPLEX_3M) return ARBGPU_ERR_INVALID;
  if (prec < 2 || prec > 1024) return ARBGPU_ERR_INVALID;
  if (M == 0 || N == 0) return ARBGPU_OK;
  if (lda < K || ldb < N || ldc < N) return ARBGPU_ERR_INVALID;
  const int parts = complex_mode ? 2 : 1;
  for (int q = 0; q < parts; ++q) {
    if (!balls_ok(C[q]) || !balls_ok(A[q]) || !balls_ok(B[q])) return ARBGPU_ERR_INVALID;
    if (K > 0 && (A[q].count < (M - 1) * lda + K || B[q].count < (K - 1) * ldb + N))
      return ARBGPU_ERR_INVALID;
    if (C[q].count < (M - 1) * ldc + N) return ARBGPU_ERR_INVALID;
    if ((int64_t)C[q].nlimbs * 64 < prec) return ARBGPU_ERR_INVALID;
    for (int r = 0; r < parts; ++r) {
      if (balls_alias(C[q], A[r]) || balls_alias(C[q], B[r])) return ARBGPU_ERR_INVALID;
      if (r != q && balls_alias(C[q], C[r])) return ARBGPU_ERR_INVALID;
    }
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ARBGPU_ERR_CUDA;
  if (alg != ARBGPU_ALG_DOT && alg != ARBGPU_ALG_BLOCK && alg != ARBGPU_ALG_AUTO)
    return ARBGPU_ERR_INVALID;
  ctx->plan_log.clear();
  const int choice =
      alg == ARBGPU_ALG_BLOCK
          ? 1
          : alg == ARBGPU_ALG_DOT
                ? 0
                : auto_choice(ctx, M, K, N, prec, complex_mode != 0,
                              (flags & ARBGPU_MM_COMPLEX_3M) != 0);
  if (choice < 0 && K > 0)
    return tune_auto(ctx, C, A, B, M, K, N, lda, ldb, ldc, prec, complex_mode, flags, workspace,
                     ws_bytes, (cudaStream_t)stream);
  // (the block call hands inputs it cannot take -- special values, limits -- to the dots)
  bool used = false;
  return run_matmul_alg(ctx, choice == 1 && K > 0, C, A, B, M, K, N, lda, ldb, ldc, prec,
                        complex_mode, flags, workspace, ws_bytes, (cudaStream_t)stream, &used);
}

arbgpu_status arbgpu_last_plans(arbgpu_ctx *ctx, int64_t *words, int64_t max_words,
                                int64_t *n_words) {
  if (!ctx || !n_words || max_words < 0 || (max_words > 0 && !words)) return ARBGPU_ERR_INVALID;
  const int64_t n = (int64_t)ctx->plan_log.size();
  *n_words = n;
  for (int64_t q = 0; q < n && q < max_words; ++q) words[q] = ctx->plan_log[(size_t)q];
  return ARBGPU_OK;
}

}  // extern "C"

namespace {

bool matmul_args_ok(const arbgpu_balls *C, const arbgpu_balls *A, const arbgpu_balls *B, int64_t M,
                    int64_t K, int64_t N, int64_t lda, int64_t ldb, int64_t ldc, int32_t prec,
                    int complex_mode) {
  if (!C || !A || !B || M < 0 || K < 0 || N < 0 || prec < 2 || prec > 1024) return false;
  if (M == 0 || N == 0) return true;
  if (lda < K || ldb < N || ldc < N) return false;
  const int parts = complex_mode ? 2 : 1;
  for (int q = 0; q < parts; ++q) {
    if (!balls_ok(C[q]) || !balls_ok(A[q]) || !balls_ok(B[q])) return false;
    if (K > 0 && (A[q].count < (M - 1) * lda + K || B[q].count < (K - 1) * ldb + N)) return false;
    if (C[q].count < (M - 1) * ldc + N) return false;
    if ((int64_t)C[q].nlimbs * 64 < prec) return false;
    for (int r = 0; r < parts; ++r) {
      if (balls_alias(C[q], A[r]) || balls_alias(C[q], B[r])) return false;
      if (r != q && balls_alias(C[q], C[r])) return false;
    }
  }
  return true;
}

// The item's AUTO choice (1 block, 0 dots, -1 to be timed), as for arbgpu_mat_mul.
int item_choice(const arbgpu_ctx *ctx, const arbgpu_matmul_desc &d) {
  if (d.M == 0 || d.N == 0 || d.K == 0) return 0;
  if (d.alg != ARBGPU_ALG_AUTO) return d.alg == ARBGPU_ALG_BLOCK ? 1 : 0;
  return auto_choice(ctx, d.M, d.K, d.N, d.prec, d.complex_mode != 0,
                     (d.flags & ARBGPU_MM_COMPLEX_3M) != 0);
}

bool item_uses_block(const arbgpu_ctx *ctx, const arbgpu_matmul_desc &d) {
  return item_choice(ctx, d) == 1;
}

// Whether the item may run the block algorithm (its share of the workspace must hold it).
bool item_may_use_block(const arbgpu_ctx *ctx, const arbgpu_matmul_desc &d) {
  if (d.M == 0 || d.N == 0 || d.K == 0) return false;
  if (d.alg != ARBGPU_ALG_AUTO) return d.alg == ARBGPU_ALG_BLOCK;
  return auto_may_use_block(ctx, d.M, d.K, d.N);
}

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" {

arbgpu_status arbgpu_mat_mul_batched_workspace_size(arbgpu_ctx *ctx,
                                                    const arbgpu_matmul_desc *descs,
                                                    int32_t count, size_t *bytes) {
  if (!ctx || !bytes || count < 0 || (count > 0 && !descs)) return ARBGPU_ERR_INVALID;
  size_t grouped = al256(sizeof(GroupItem) * (size_t)count) + al256(8 * (size_t)count);
  size_t blk = 0, scans = al256(sizeof(BlockStats) * 4 * (size_t)count);
  for (int32_t q = 0; q < count; ++q) {
    const arbgpu_matmul_desc &d = descs[q];
    if (!item_may_use_block(ctx, d)) continue;
    int nlA = d.A[0].nlimbs, nlB = d.B[0].nlimbs;
    if (d.complex_mode) {
      nlA = d.A[1].nlimbs > nlA ? d.A[1].nlimbs : nlA;
      nlB = d.B[1].nlimbs > nlB ? d.B[1].nlimbs : nlB;
    }
    const size_t b = block_workspace_size(ctx, d.M, d.K, d.N, d.prec, d.complex_mode != 0,
                                          (d.flags & ARBGPU_MM_COMPLEX_3M) != 0, nlA, nlB);
    blk = b > blk ? b : blk;
    scans += al256(block_scan_bytes(d.M, d.N, d.complex_mode != 0));
  }
  int nblock = 0;
  for (int32_t q = 0; q < count; ++q) nblock += item_may_use_block(ctx, descs[q]) ? 1 : 0;
  const size_t lanes = nblock < arbgpu_ctx::kLanes ? (size_t)nblock : (size_t)arbgpu_ctx::kLanes;
  *bytes = grouped + scans + (lanes > 1 ? lanes * al256(blk) : blk);
  return ARBGPU_OK;
}

arbgpu_status arbgpu_mat_mul_batched(arbgpu_ctx *ctx, const arbgpu_matmul_desc *descs,
                                     int32_t count, void *workspace, size_t ws_bytes,
                                     void *stream) {
  if (!ctx || count < 0 || (count > 0 && !descs)) return ARBGPU_ERR_INVALID;
  if (count == 0) return ARBGPU_OK;
  for (int32_t q = 0; q < count; ++q) {
    const arbgpu_matmul_desc &d = descs[q];
    if (d.alg != ARBGPU_ALG_AUTO && d.alg != ARBGPU_ALG_DOT && d.alg != ARBGPU_ALG_BLOCK)
      return ARBGPU_ERR_INVALID;
    if (d.flags & ~ARBGPU_MM_COMPLEX_3M) return ARBGPU_ERR_INVALID;
    if (!matmul_args_ok(d.C, d.A, d.B, d.M, d.K, d.N, d.lda, d.ldb, d.ldc, d.prec,
                        d.complex_mode))
      return ARBGPU_ERR_INVALID;
  }
  size_t need = 0;
  arbgpu_status st = arbgpu_mat_mul_batched_workspace_size(ctx, descs, count, &need);
  if (st != ARBGPU_OK) return st;
  if (ws_bytes < need || (need && !workspace)) return ARBGPU_ERR_WORKSPACE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ARBGPU_ERR_CUDA;
  ctx->plan_log.clear();
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t *ws = (uint8_t *)workspace;
  const size_t items_off = 0, ends_off = al256(sizeof(GroupItem) * (size_t)count);
  const size_t blk_off = ends_off + al256(8 * (size_t)count);
  // 0. AUTO items of buckets the autotuner has yet to time: each alone, as arbgpu_mat_mul would
  //    (its product is then computed again below, by the chosen algorithm), in the workspace past
  //    the grouped arrays (at least one item's block workspace)
  for (int32_t q = 0; q < count; ++q) {
    const arbgpu_matmul_desc &d = descs[q];
    if (item_choice(ctx, d) >= 0) continue;
    st = tune_auto(ctx, d.C, d.A, d.B, d.M, d.K, d.N, d.lda, d.ldb, d.ldc, d.prec,
                   d.complex_mode, d.flags, ws + blk_off, ws_bytes - blk_off, s);
    if (st != ARBGPU_OK) return st;
  }
  ctx->plan_log.clear();
  // 1. every classical item in one launch of the dot kernel
  std::vector<GroupItem> items;
  std::vector<int64_t> ends;
  std::vector<int32_t> block_items;
  int64_t total = 0, kmax = 0;
  int pmax = 2, nlmax = 1;
  for (int32_t q = 0; q < count; ++q) {
    const arbgpu_matmul_desc &d = descs[q];
    if (d.M == 0 || d.N == 0) continue;
    if (item_uses_block(ctx, d)) {
      block_items.push_back(q);
      continue;
    }
    GroupItem it{};
    const int parts = d.complex_mode ? 2 : 1;
    for (int r = 0; r < 2; ++r) {
      const int src = r < parts ? r : 0;
      it.A[r] = view_of(d.A[src]);
      it.B[r] = view_of(d.B[src]);
      it.C[r] = out_of(d.C[src]);
      nlmax = d.A[src].nlimbs > nlmax ? d.A[src].nlimbs : nlmax;
      nlmax = d.B[src].nlimbs > nlmax ? d.B[src].nlimbs : nlmax;
    }
    it.M = d.M;
    it.N = d.N;
    it.K = d.K;
    it.lda = d.lda;
    it.ldb = d.ldb;
    it.ldc = d.ldc;
    it.prec = d.prec;
    it.cplx = d.complex_mode ? 1 : 0;
    total += (int64_t)parts * d.M * d.N;
    items.push_back(it);
    ends.push_back(total);
    pmax = d.prec > pmax ? d.prec : pmax;
    kmax = d.K > kmax ? d.K : kmax;
  }
  if (!items.empty()) {
    GroupItem *ditems = (GroupItem *)(ws + items_off);
    int64_t *dends = (int64_t *)(ws + ends_off);
    if (cudaMemcpyAsync(ditems, items.data(), sizeof(GroupItem) * items.size(),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dends, ends.data(), 8 * ends.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
      return ARBGPU_ERR_CUDA;
    st = launch_grouped_dot(ctx, ditems, dends, (int32_t)items.size(), total, pmax, kmax, nlmax, s);
    if (st != ARBGPU_OK) return st;
  }
  // 2. the block items: every item's scans, one read-back of all their statistics, then the
  //    products one after the other, sharing the rest of the workspace
  if (!block_items.empty()) {
    const size_t nb = block_items.size();
    BlockStats *dstats = (BlockStats *)(ws + blk_off);
    size_t off = blk_off + al256(sizeof(BlockStats) * 4 * (size_t)count);
    std::vector<size_t> region(nb);
    for (size_t i = 0; i < nb; ++i) {
      const arbgpu_matmul_desc &d = descs[block_items[i]];
      region[i] = off;
      off += al256(block_scan_bytes(d.M, d.N, d.complex_mode != 0));
    }
    const size_t prod_off = off;
    if (cudaMemsetAsync(dstats, 0, sizeof(BlockStats) * 4 * nb, s) != cudaSuccess)
      return ARBGPU_ERR_CUDA;
    std::vector<char> scanned(nb, 0);
    for (size_t i = 0; i < nb; ++i) {
      const arbgpu_matmul_desc &d = descs[block_items[i]];
      st = block_scan_launch(ctx, d.A, d.B, d.M, d.K, d.N, d.lda, d.ldb, d.complex_mode != 0,
                             ws + region[i], dstats + 4 * i, s);
      if (st == ARBGPU_OK)
        scanned[i] = 1;
      else if (st != ARBGPU_ERR_LIMIT)
        return st;
    }
    std::vector<BlockStats> hstats(4 * nb);
    st = read_stats(ctx, dstats, hstats.data(), 4 * nb, s);
    if (st != ARBGPU_OK) return st;
    // the products themselves on up to kLanes streams side by side, each with its own share of
    // the workspace, forked from and joined back into `s`: in item order, each item goes to the
    // lane with the least work so far (estimated as M N K (p / 64)^2)
    const int lanes = nb < (size_t)arbgpu_ctx::kLanes ? (int)nb : arbgpu_ctx::kLanes;
    size_t lane_bytes = ws_bytes - prod_off;
    if (lanes > 1) {
      lane_bytes = (ws_bytes - prod_off) / (size_t)lanes / 256 * 256;
      if (!ctx->lane_fork && cudaEventCreateWithFlags(&ctx->lane_fork, cudaEventDisableTiming) !=
                                 cudaSuccess)
        return ARBGPU_ERR_CUDA;
      for (int l = 0; l < lanes; ++l) {
        if (!ctx->lanes[l] &&
            (cudaStreamCreateWithFlags(&ctx->lanes[l], cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&ctx->lane_done[l], cudaEventDisableTiming) != cudaSuccess))
          return ARBGPU_ERR_CUDA;
      }
      if (cudaEventRecord(ctx->lane_fork, s) != cudaSuccess) return ARBGPU_ERR_CUDA;
      for (int l = 0; l < lanes; ++l)
        if (cudaStreamWaitEvent(ctx->lanes[l], ctx->lane_fork, 0) != cudaSuccess)
          return ARBGPU_ERR_CUDA;
    }
    arbgpu_status first = ARBGPU_OK;
    double load[arbgpu_ctx::kLanes] = {};
    for (size_t i = 0; i < nb; ++i) {
      const arbgpu_matmul_desc &d = descs[block_items[i]];
      int l = 0;
      for (int c = 1; c < lanes; ++c)
        if (load[c] < load[l]) l = c;
      const double w64 = (d.prec + 63) / 64;
      load[l] += (double)d.M * (double)d.N * (double)d.K * w64 * w64;
      cudaStream_t ls = lanes > 1 ? ctx->lanes[l] : s;
      bool used = false;
      st = ARBGPU_ERR_LIMIT;
      if (scanned[i])
        st = block_finish(ctx, d.C, d.A, d.B, d.M, d.K, d.N, d.lda, d.ldb, d.ldc, d.prec,
                          d.complex_mode != 0, (d.flags & ARBGPU_MM_COMPLEX_3M) != 0,
                          ws + region[i], hstats.data() + 4 * i,
                          ws + prod_off + (size_t)l * lane_bytes, lane_bytes, ls, &used);
      if (!used && st == ARBGPU_ERR_LIMIT)
        st = launch_matmul_dot(ctx, d.C, d.A, d.B, d.M, d.K, d.N, d.lda, d.ldb, d.ldc, d.prec,
                               d.complex_mode, ls);
      if (st != ARBGPU_OK) {
        first = st;
        break;
      }
    }
    if (lanes > 1) {  // join (also after an error, so that `s` orders everything launched)
      for (int l = 0; l < lanes; ++l)
        if (cudaEventRecord(ctx->lane_done[l], ctx->lanes[l]) != cudaSuccess ||
            cudaStreamWaitEvent(s, ctx->lane_done[l], 0) != cudaSuccess)
          return ARBGPU_ERR_CUDA;
    }
    if (first != ARBGPU_OK) return first;
  }
  return ARBGPU_OK;
}

}  // extern "C"
