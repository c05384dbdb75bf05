// Kernel (a) for the basecase blocks of Algorithm 2.
#include "dot_src.cuh"
#include "dot_tile.cuh"

namespace arbgpu {

arbgpu_status launch_basecase_dot(arbgpu_ctx *ctx, const arbgpu_balls &C, const arbgpu_balls *A,
                                  const arbgpu_balls *B, bool cplx, const arbgpu_balls &initial,
                                  const int32_t *bk, int64_t nbk, int64_t M, int64_t N,
                                  int64_t lda, int64_t ldb, int64_t ldc, int32_t prec,
                                  cudaStream_t stream) {
  BasecaseSrc s{};
  const int parts = cplx ? 2 : 1;
  int maxnl = 1;  // the `initial` term has its own limb array: only A and B size the class
  for (int q = 0; q < 2; ++q) {
    const int src = q < parts ? q : 0;
    s.A[q] = view_of(A[src]);
    s.B[q] = view_of(B[src]);
    maxnl = A[src].nlimbs > maxnl ? A[src].nlimbs : maxnl;
    maxnl = B[src].nlimbs > maxnl ? B[src].nlimbs : maxnl;
  }
  s.init = view_of(initial);
  s.C = out_of(C);
  s.bk = bk;
  s.nbk = nbk;
  s.M = M;
  s.N = N;
  s.lda = lda;
  s.ldb = ldb;
  s.ldc = ldc;
  s.prec_v = prec;
  s.prec_max = prec;
  s.len_max = nbk;
  const int cmax = dot_class_for_problem(prec, nbk + 1, maxnl);
  if (cmax < 0) return ARBGPU_ERR_INVALID;
  {
    TileSrc t{};
    t.A[0] = s.A[0];
    t.A[1] = s.A[1];
    t.B[0] = s.B[0];
    t.B[1] = s.B[1];
    t.C[0] = t.C[1] = s.C;
    t.init = s.init;
    t.M = M;
    t.N = N;
    t.lda = lda;
    t.ldb = ldb;
    t.ldc = ldc;
    t.nterms = nbk;
    t.mode = 2;
    t.bk = bk;
    t.prec = prec;
    t.has_init = 1;
    arbgpu_status st = ARBGPU_OK;
    if (launch_dot_tile(ctx, t, 1, cmax, stream, &st, M * N * nbk)) return st;
  }
  return launch_dot_fused(ctx, s, M * N, cmax, dot_group_matrix(), stream);
}

}  // namespace arbgpu
