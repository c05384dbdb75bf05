// Kernel (a) over rows x columns: the classical matrix product.
#include "dot_src.cuh"
#include "dot_tile.cuh"

namespace arbgpu {

arbgpu_status launch_matmul_dot(arbgpu_ctx *ctx, const arbgpu_balls *C, const arbgpu_balls *A,
                                const arbgpu_balls *B, int64_t M, int64_t K, int64_t N,
                                int64_t lda, int64_t ldb, int64_t ldc, int32_t prec,
                                int complex_mode, cudaStream_t stream) {
  const int parts = complex_mode ? 2 : 1;
  MatDotSrc s{};
  int maxnl = 1;
  for (int q = 0; q < parts; ++q) {
    s.A[q] = view_of(A[q]);
    s.B[q] = view_of(B[q]);
    s.C[q] = out_of(C[q]);
    maxnl = A[q].nlimbs > maxnl ? A[q].nlimbs : maxnl;
    maxnl = B[q].nlimbs > maxnl ? B[q].nlimbs : maxnl;
  }
  if (!complex_mode) {
    s.A[1] = s.A[0];
    s.B[1] = s.B[0];
    s.C[1] = s.C[0];
  }
  s.M = M;
  s.K = K;
  s.N = N;
  s.lda = lda;
  s.ldb = ldb;
  s.ldc = ldc;
  s.prec_v = prec;
  s.cplx = complex_mode ? 1 : 0;
  s.prec_max = prec;
  s.len_max = complex_mode ? 2 * K : K;
  const int cmax = dot_class_for_problem(prec, s.len_max, maxnl);
  if (cmax < 0) return ARBGPU_ERR_INVALID;
  {
    TileSrc t{};
    for (int q = 0; q < 2; ++q) {
      t.A[q] = s.A[q];
      t.B[q] = s.B[q];
      t.C[q] = s.C[q];
    }
    t.init = s.A[0];
    t.M = M;
    t.N = N;
    t.lda = lda;
    t.ldb = ldb;
    t.ldc = ldc;
    t.nterms = s.len_max;
    t.mode = complex_mode ? 1 : 0;
    t.prec = prec;
    t.has_init = 0;
    arbgpu_status st = ARBGPU_OK;
    const int parts = complex_mode ? 2 : 1;
    if (launch_dot_tile(ctx, t, parts, cmax, stream, &st, parts * M * N * s.len_max)) return st;
  }
  return launch_dot_fused(ctx, s, (complex_mode ? 2 : 1) * M * N, cmax, dot_group_matrix(), stream);
}

}  // namespace arbgpu
