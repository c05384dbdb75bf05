// Kernel (a) for batched dots (arbgpu_dot).
#include <cstdlib>
#include <cstring>

#include "dot_src.cuh"

namespace arbgpu {

int dot_class_for_problem(int prec, int64_t max_terms, int max_nlimbs) {
  const int ns = dot_ns(prec, max_terms, max_terms);
  int nx = max_nlimbs < ns + 1 ? max_nlimbs : ns + 1;
  if (nx < 1) nx = 1;
  return dot_class_for(nx, ns);
}

arbgpu_status launch_batched_dot(arbgpu_ctx *ctx, const arbgpu_balls *res,
                                 const arbgpu_balls *initial, const uint8_t *sub,
                                 const arbgpu_balls *x, const int64_t *xoff, const int64_t *xstep,
                                 const arbgpu_balls *y, const int64_t *yoff, const int64_t *ystep,
                                 const int64_t *len, const int32_t *prec, int64_t batch,
                                 int32_t prec_max, int64_t len_max, int complex_mode,
                                 cudaStream_t stream, bool approx, bool reduce, bool fused) {
  const int parts = complex_mode ? 2 : 1;
  BatchDotSrc s{};
  int maxnl = 1;
  for (int q = 0; q < parts; ++q) {
    s.x[q] = view_of(x[q]);
    s.y[q] = view_of(y[q]);
    s.out[q] = out_of(res[q]);
    s.init[q] = initial ? view_of(initial[q]) : view_of(x[q]);
    maxnl = x[q].nlimbs > maxnl ? x[q].nlimbs : maxnl;
    maxnl = y[q].nlimbs > maxnl ? y[q].nlimbs : maxnl;
  }
  if (!complex_mode) {
    s.x[1] = s.x[0];
    s.y[1] = s.y[0];
    s.out[1] = s.out[0];
    s.init[1] = s.init[0];
  }
  s.xoff = xoff;
  s.xstep = xstep;
  s.yoff = yoff;
  s.ystep = ystep;
  s.len = len;
  s.precs = prec;
  s.subs = sub;
  s.batch = batch;
  s.cplx = complex_mode ? 1 : 0;
  s.has_init = initial != nullptr;
  s.approx = approx;
  s.reduce = reduce;
  s.prec_max = prec_max;
  const int64_t terms_max = (complex_mode ? 2 * len_max : len_max);
  s.len_max = terms_max;
  s.ndots_host = s.cplx ? 2 * batch : batch;
  const int cmax = dot_class_for_problem(prec_max, terms_max + 1, maxnl);
  if (cmax < 0) return ARBGPU_ERR_INVALID;
  // fused: setup and evaluation of every dot in one launch of class cmax.  Taken when asked (dots
  // of one precision, short chains of dependent calls) and whenever the largest class is small
  // (cmax <= 2, up to three limbs per factor): evaluating every dot at that class costs little,
  // each dot's fields are read twice within one pass instead of by two launches, and the batch
  // is one launch instead of cmax + 2 (65 536 dots at p <= 192: 0.52 ms against 0.61 ms).
  // ARBGPU_DOT_FUSED=0 keeps the setup and class launches for the small classes.
  const char *fe = getenv("ARBGPU_DOT_FUSED");
  if (cmax <= 2 && !(fe && !strcmp(fe, "0"))) fused = true;
  if (fused)
    return launch_dot_fused(ctx, s, s.cplx ? 2 * batch : batch, cmax, dot_group_batched(terms_max),
                            stream);
  return launch_dot_src(ctx, s, s.cplx ? 2 * batch : batch, cmax, dot_group_batched(terms_max), stream);
}

}  // namespace arbgpu
