// Kernel (a) for matrix-shaped sources -- the classical product's M N dots and the basecase blocks
// of Algorithm 2 -- tiled through shared memory.  Every dot of a tile of C has the same term
// list (the same inner index k and operand parts per term), so a CTA stages the tile's rows of A
// and columns of B for a chunk of terms once and every thread evaluates its entries from shared
// memory: each entry of A and B is read from global memory once per tile instead of once per
// dot, and a thread reuses its column's B operand for all its entries.
//
// The arithmetic is Algorithm 1's, the same as dot_eval_class: the setup pass (Section III-C)
// over the staged scalar fields, then the evaluation (Section III-D/E) with one thread per dot.
// Integer addition modulo 2^(64 NS) is associative and err / srad are integer sums, so one thread
// summing all terms gives the group-of-lanes result bit for bit.
#pragma once

#include <cstdlib>
#include <cstring>

#include "dot_eval.cuh"
#include "internal.h"

namespace arbgpu {

// One matrix-shaped dot source: entry (i, j) of output part `part` sums, over terms t < nterms,
// (-1)^neg X[xa][i lda + k] Y[ya][k ldb + j] with (k, xa, ya, neg) = term(part, t), plus the
// `initial` ball init[i N + j] when has_init.
struct TileSrc {
  BallsView A[2], B[2], init;
  BallsOut C[2];
  int64_t M, N, lda, ldb, ldc;
  int64_t nterms;
  int mode;  // 0: real product (k = t); 1: complex product (k = t / 2, four real products);
             // 2: tagged list bk[t] = k << 2 | combo (the basecase blocks)
  const int32_t *bk;
  int prec;
  int has_init;
  struct Term {
    int64_t k;
    int xa, ya;
    bool neg;
  };
  __device__ Term term(int part, int64_t t) const {
    if (mode == 0) return Term{t, 0, 0, false};
    if (mode == 1) {
      const int64_t k = t >> 1;
      const int w = (int)(t & 1);
      if (part == 0) return w == 0 ? Term{k, 0, 0, false} : Term{k, 1, 1, true};
      return w == 0 ? Term{k, 0, 1, false} : Term{k, 1, 0, false};
    }
    const int32_t e = __ldg(bk + t);
    const int combo = e & 3;
    return Term{(int64_t)(e >> 2), (combo == 1 || combo == 3) ? 1 : 0,
                (combo == 1 || combo == 2) ? 1 : 0, combo == 1};
  }
};

// Shape of the tiled kernel per size class: EPT entries per thread (rows 8 apart), TK terms per
// staged chunk.  Tiles are (8 EPT) x 32 entries of C, 256 threads.
template <int C>
struct TileShape {
  static constexpr int NX = DotClass<C>::NX;
  static constexpr int EPT = C <= 1 ? 4 : (C <= 3 ? 2 : 1);
  static constexpr int TM = 8 * EPT;
  static constexpr int TN = 32;
  static constexpr int TK = NX <= 4 ? 16 : 8;
};

// Shared-memory staging of one chunk: scalar fields and leading limbs (top-aligned, NX of them,
// zeros past the entry's limb count) of the tile's rows of A (TM x TK) and columns of B (TK x TN).
template <int C>
struct TileStage {
  using S = TileShape<C>;
  static constexpr int NX = S::NX;
  uint32_t af[S::TK][S::TM], arm[S::TK][S::TM];
  int64_t ae[S::TK][S::TM], are[S::TK][S::TM];
  uint64_t al[S::TK][NX][S::TM];
  uint32_t bf[S::TK][S::TN], brm[S::TK][S::TN];
  int64_t be[S::TK][S::TN], bre[S::TK][S::TN];
  uint64_t bl[S::TK][NX][S::TN];
  int32_t xa[S::TK], ya[S::TK];
  uint8_t neg[S::TK];
};

template <int C>
constexpr size_t tile_smem_bytes() {
  return sizeof(TileStage<C>);
}

// Stage the terms [t0, t0 + TK) of the tile (rows i0.., columns j0..); `limbs`: also the leading
// limbs (the evaluation pass) or only the scalar fields (the setup pass).
template <int C>
__device__ __forceinline__ void tile_load(const TileSrc &src, TileStage<C> &st, int part,
                                          int64_t i0, int64_t j0, int64_t t0, bool limbs) {
  using S = TileShape<C>;
  constexpr int NX = S::NX;
  if (threadIdx.x < S::TK) {
    const int64_t t = t0 + threadIdx.x;
    if (t < src.nterms) {
      const TileSrc::Term tm = src.term(part, t);
      st.xa[threadIdx.x] = tm.xa;
      st.ya[threadIdx.x] = tm.ya;
      st.neg[threadIdx.x] = tm.neg ? 1 : 0;
    } else {
      st.xa[threadIdx.x] = -1;  // past the last term
    }
  }
  __syncthreads();
  // A: TM rows x TK terms; consecutive threads take consecutive terms of a row (k contiguous for
  // the plain products)
  for (int q = threadIdx.x; q < S::TM * S::TK; q += blockDim.x) {
    const int r = q / S::TK, u = q - r * S::TK;
    const int64_t i = i0 + r, t = t0 + u;
    uint32_t fl = ARBGPU_FLAG_ZERO, rm = 0;
    int64_t e = 0, re = 0;
    uint64_t l[NX];
#pragma unroll
    for (int j = 0; j < NX; ++j) l[j] = 0;
    if (i < src.M && st.xa[u] >= 0) {
      const TileSrc::Term tm = src.term(part, t);
      const BallsView &X = src.A[tm.xa];
      const int64_t idx = i * src.lda + tm.k;
      fl = __ldg(X.flags + idx);
      e = __ldg(X.exp + idx);
      rm = __ldg(X.rad_man + idx);
      re = __ldg(X.rad_exp + idx);
      if (limbs) load_top<NX>(X, idx, l);
    }
    st.af[u][r] = fl;
    st.ae[u][r] = e;
    st.arm[u][r] = rm;
    st.are[u][r] = re;
    if (limbs) {
#pragma unroll
      for (int j = 0; j < NX; ++j) st.al[u][j][r] = l[j];
    }
  }
  // B: TK terms x TN columns; consecutive threads take consecutive columns (coalesced)
  for (int q = threadIdx.x; q < S::TK * S::TN; q += blockDim.x) {
    const int u = q / S::TN, c = q - u * S::TN;
    const int64_t j = j0 + c, t = t0 + u;
    uint32_t fl = ARBGPU_FLAG_ZERO, rm = 0;
    int64_t e = 0, re = 0;
    uint64_t l[NX];
#pragma unroll
    for (int jj = 0; jj < NX; ++jj) l[jj] = 0;
    if (j < src.N && st.xa[u] >= 0) {
      const TileSrc::Term tm = src.term(part, t);
      const BallsView &Y = src.B[tm.ya];
      const int64_t idx = tm.k * src.ldb + j;
      fl = __ldg(Y.flags + idx);
      e = __ldg(Y.exp + idx);
      rm = __ldg(Y.rad_man + idx);
      re = __ldg(Y.rad_exp + idx);
      if (limbs) load_top<NX>(Y, idx, l);
    }
    st.bf[u][c] = fl;
    st.be[u][c] = e;
    st.brm[u][c] = rm;
    st.bre[u][c] = re;
    if (limbs) {
#pragma unroll
      for (int jj = 0; jj < NX; ++jj) st.bl[u][jj][c] = l[jj];
    }
  }
  __syncthreads();
}

// The classical product / basecase dots of one tile: grid (column tiles, row tiles, parts).
template <int C>
__global__ void __launch_bounds__(256) dot_tile_kernel(const __grid_constant__ TileSrc src,
                                                       int *status) {
  using S = TileShape<C>;
  constexpr int NX = S::NX;
  constexpr int NS = DotClass<C>::NS;
  constexpr int EPT = S::EPT;
  extern __shared__ __align__(16) uint8_t tile_smem[];
  TileStage<C> &st = *(TileStage<C> *)tile_smem;
  const int part = blockIdx.z;
  const int64_t i0 = (int64_t)blockIdx.y * S::TM, j0 = (int64_t)blockIdx.x * S::TN;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t j = j0 + tx;
  const BallsOut &out = src.C[part];
  const int prec = src.prec;
  const int64_t nt = src.nterms;
  const int64_t ntot = nt + (src.has_init ? 1 : 0);

  // ---- setup pass (Section III-C) over the staged scalar fields
  bool special[EPT];
  int64_t nnz[EPT], e_max[EPT], e_rad[EPT];
  int nsig_max[EPT];
#pragma unroll
  for (int a = 0; a < EPT; ++a) {
    special[a] = false;
    nnz[a] = 0;
    e_max[a] = e_rad[a] = INT64_MIN;
    nsig_max[a] = 0;
  }
  for (int64_t t0 = 0; t0 < nt; t0 += S::TK) {
    tile_load<C>(src, st, part, i0, j0, t0, false);
    const int tk = (int)min((int64_t)S::TK, nt - t0);
    for (int u = 0; u < tk; ++u) {
      const Opnd y{st.bf[u][tx], st.be[u][tx], st.brm[u][tx], st.bre[u][tx]};
#pragma unroll
      for (int a = 0; a < EPT; ++a) {
        const int r = ty + 8 * a;
        const Opnd x{st.af[u][r], st.ae[u][r], st.arm[u][r], st.are[u][r]};
        if (opnd_special(x) || opnd_special(y)) {
          special[a] = true;
          continue;
        }
        if (!opnd_zero(x) && !opnd_zero(y)) {
          ++nnz[a];
          e_max[a] = imax64(e_max[a], x.e + y.e);
          nsig_max[a] = max(nsig_max[a], (int)max(nsig_of(x.flags), nsig_of(y.flags)));
        }
        e_rad[a] = term_rad_exp_max(x, y, e_rad[a]);
      }
    }
    __syncthreads();
  }
  DotSetup su[EPT];
  bool pending[EPT];
#pragma unroll
  for (int a = 0; a < EPT; ++a) {
    const int64_t i = i0 + ty + 8 * a;
    pending[a] = false;
    su[a] = DotSetup{};
    if (i >= src.M || j >= src.N) continue;
    const int64_t oi = i * src.ldc + j;
    if (src.has_init) {  // the `initial` term init [1 +- 0]
      const Opnd x = load_opnd(src.init, i * src.N + j);
      const Opnd y = one_opnd();
      if (opnd_special(x)) {
        special[a] = true;
      } else {
        if (!opnd_zero(x)) {
          ++nnz[a];
          e_max[a] = imax64(e_max[a], x.e + y.e);
        }
        e_rad[a] = term_rad_exp_max(x, y, e_rad[a]);
      }
    }
    if (special[a]) {
      set_status(status, ARBGPU_ERR_UNSUPPORTED_VALUE);
      write_special<1>(out, oi, 0);
      continue;
    }
    DotSetup &s = su[a];
    s.has_mid = e_max[a] != INT64_MIN;
    s.approx = false;
    s.has_rad = e_rad[a] != INT64_MIN;
    if (!s.has_mid && !s.has_rad) {
      write_zero<1>(out, oi, 0);
      continue;
    }
    s.prec = prec;
    const int extend = bc64(nnz[a]) + 1;
    s.n_s = dot_ns(prec, ntot, nnz[a]);
    s.e_s = s.has_mid ? e_max[a] + extend : 0;
    s.e_rad = e_rad[a];
    s.nx = min(nsig_max[a], s.n_s + 1);
    if (s.nx < 1) s.nx = 1;
    const int c = dot_class_for(s.nx, s.n_s);
    if (c < 0 || c > C) {
      set_status(status, ARBGPU_ERR_LIMIT);
      write_special<1>(out, oi, 0);
      continue;
    }
    pending[a] = true;
  }

  // ---- evaluation (Section III-D, III-E): one thread per dot, the terms from shared memory
  LaneAcc<NS> acc[EPT];
#pragma unroll
  for (int a = 0; a < EPT; ++a) {
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[a].s[k] = 0;
    acc[a].err = 0;
    acc[a].srad = 0;
  }
  for (int64_t t0 = 0; t0 < nt; t0 += S::TK) {
    tile_load<C>(src, st, part, i0, j0, t0, true);
    const int tk = (int)min((int64_t)S::TK, nt - t0);
    for (int u = 0; u < tk; ++u) {
      const Opnd y{st.bf[u][tx], st.be[u][tx], st.brm[u][tx], st.bre[u][tx]};
      uint64_t yfull[NX];
#pragma unroll
      for (int q = 0; q < NX; ++q) yfull[q] = st.bl[u][q][tx];
      const bool tneg = st.neg[u] != 0;
#pragma unroll
      for (int a = 0; a < EPT; ++a) {
        if (!pending[a]) continue;
        const int r = ty + 8 * a;
        const Opnd x{st.af[u][r], st.ae[u][r], st.arm[u][r], st.are[u][r]};
        const int64_t width = 64LL * su[a].n_s;
        uint64_t xa[NX], ya[NX];
#pragma unroll
        for (int q = 0; q < NX; ++q) {
          xa[q] = st.al[u][q][r];
          ya[q] = yfull[q];
        }
        if (!opnd_zero(x) && !opnd_zero(y)) {
          const int64_t shift = su[a].e_s - (x.e + y.e);
          if (shift >= width) {
            acc[a].err += 1;
          } else {
            const int F = (int)(width - shift);
            const int n2 = (F + 63) / 64 + 1;
            const int nx = min((int)nsig_of(x.flags), src.A[st.xa[u]].nlimbs);
            const int ny = min((int)nsig_of(y.flags), src.B[st.ya[u]].nlimbs);
            if (nx > n2 || ny > n2) acc[a].err += 1;
            keep_leading<NX>(xa, min(nx, n2));
            keep_leading<NX>(ya, min(ny, n2));
            const bool negative = (((x.flags ^ y.flags) & ARBGPU_FLAG_SIGN) != 0) != tneg;
            acc_term<NX, NS>(acc[a], xa, ya, F, negative);
          }
        }
        if (su[a].has_rad && (x.rman || y.rman))
          term_radius(acc[a].srad, x, st.al[u][NX - 1][r], y, yfull[NX - 1], su[a].e_rad);
      }
    }
    __syncthreads();
  }
  // the `initial` term, then the rounding
#pragma unroll
  for (int a = 0; a < EPT; ++a) {
    if (!pending[a]) continue;
    const int64_t i = i0 + ty + 8 * a;
    if (src.has_init) {
      constexpr int NXI = NS + 1;
      const BallsView &iv = src.init;
      const int64_t ii = i * src.N + j;
      const Opnd x = load_opnd(iv, ii);
      const Opnd y = one_opnd();
      const int64_t width = 64LL * su[a].n_s;
      uint64_t xa[NXI];
#pragma unroll
      for (int q = 0; q < NXI; ++q) xa[q] = 0;
      if (!opnd_zero(x)) {
        const int64_t shift = su[a].e_s - (x.e + y.e);
        if (shift >= width) {
          acc[a].err += 1;
        } else {
          const int F = (int)(width - shift);
          const int n2 = (F + 63) / 64 + 1;
          const int nx = min((int)nsig_of(x.flags), iv.nlimbs);
          if (nx > n2) acc[a].err += 1;
          load_top<NXI>(iv, ii, xa);
          keep_leading<NXI>(xa, min(nx, n2));
          acc_term_one<NXI, NS>(acc[a], xa, F, (x.flags & ARBGPU_FLAG_SIGN) != 0);
        }
      }
      if (su[a].has_rad && x.rman) {
        uint64_t xtop = xa[NXI - 1];
        if (!opnd_zero(x) && xtop == 0)
          xtop = __ldg(iv.limbs + (int64_t)(iv.nlimbs - 1) * iv.stride + ii);
        term_radius(acc[a].srad, x, xtop, y, (uint64_t)1 << 63, su[a].e_rad);
      }
    }
    dot_finalise<NS, 1>(acc[a], su[a], prec, out, i * src.ldc + j, 0);
  }
}

// Launch of the tiled kernel in class C: grid (column tiles, row tiles, parts).  False when the
// grid does not fit (the group-of-lanes kernel then runs).
template <int C>
static bool launch_dot_tile_c(arbgpu_ctx *ctx, const TileSrc &src, int parts, cudaStream_t s,
                              arbgpu_status *st, int64_t units) {
  using S = TileShape<C>;
  const int64_t gx = (src.N + S::TN - 1) / S::TN, gy = (src.M + S::TM - 1) / S::TM;
  if (gy > 65535 || gx > 0x7fffffff) return false;
  // a tile's dots run one per thread in sequence over the terms: too few tiles to fill the SMs
  // leave the short rows of lane groups faster (e.g. N = 32: 2 tiles against 32 warps)
  if (gx * gy * parts < ctx->sm_count) return false;
  const size_t smem = sizeof(TileStage<C>);
  static bool attr[256] = {};
  const int dev = ctx->device & 255;
  if (!attr[dev]) {
    if (cudaFuncSetAttribute(dot_tile_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
      *st = ARBGPU_ERR_CUDA;
      return true;
    }
    attr[dev] = true;
  }
  LaunchScope sc(ctx, s, "dot_tile", units);
  dot_tile_kernel<C><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)parts), 256, smem, s>>>(
      src, ctx->status);
  *st = cudaGetLastError() == cudaSuccess ? ARBGPU_OK : ARBGPU_ERR_CUDA;
  return true;
}

// The tiled kernel for a matrix-shaped source whose dots need at most class cmax; false when it
// does not take the problem.  ARBGPU_DOT_TILE=0 keeps the group-of-lanes kernel.
static bool launch_dot_tile(arbgpu_ctx *ctx, const TileSrc &src, int parts, int cmax,
                            cudaStream_t s, arbgpu_status *st, int64_t units) {
  const char *e = getenv("ARBGPU_DOT_TILE");
  if (e && !strcmp(e, "0")) return false;
  switch (cmax) {
    case 0: return launch_dot_tile_c<0>(ctx, src, parts, s, st, units);
    case 1: return launch_dot_tile_c<1>(ctx, src, parts, s, st, units);
    case 2: return launch_dot_tile_c<2>(ctx, src, parts, s, st, units);
    case 3: return launch_dot_tile_c<3>(ctx, src, parts, s, st, units);
    case 4: return launch_dot_tile_c<4>(ctx, src, parts, s, st, units);
    case 5: return launch_dot_tile_c<5>(ctx, src, parts, s, st, units);
    case 6: return launch_dot_tile_c<6>(ctx, src, parts, s, st, units);
    case 7: return launch_dot_tile_c<7>(ctx, src, parts, s, st, units);
    default: return false;
  }
}

}  // namespace arbgpu
