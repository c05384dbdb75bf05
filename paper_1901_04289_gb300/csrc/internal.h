// Host-side declarations shared by the translation units of the arbgpu library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <map>
#include <vector>

#include "arbgpu.h"
#include "common.cuh"

// One traced kernel launch: a pair of events recorded around it on its stream.
struct arbgpu_trace_rec {
  const char *name;
  cudaEvent_t start, stop;
  int64_t units;  // algorithmic work units the launch processes (caller-defined per kernel)
};

struct arbgpu_ctx {
  int device;
  std::map<int, void *> crt_tables;  // multimodular tables on the device, per modulus count
  int sm_count;
  int *status;       // device int: first recorded error code
  int64_t launches;  // kernels launched through this context
  bool trace;
  std::vector<arbgpu_trace_rec> recs;
  std::vector<cudaEvent_t> event_pool;
  // mapped pinned host memory (and its device address) for small device-to-host reads
  void *mapped = nullptr;
  void *mapped_dev = nullptr;
  size_t mapped_bytes = 0;
  // block plans of the last matrix-product call, one record per real product (arbgpu_last_plans)
  std::vector<int64_t> plan_log;
  // mapped pinned words that the scan kernel publishes a single product's statistics to (four
  // BlockStats and a sequence word), and the last sequence number used
  void *pub = nullptr;
  void *pub_dev = nullptr;
  uint32_t pub_seq = 0;
  // engine autotuner (arbgpu_set_autotune): per size bucket of a block product, whether the
  // multimodular engine measured faster than the digit engine; products run for the timings
  bool autotune = false;
  std::map<uint64_t, bool> engine_tuned;
  int64_t tune_runs = 0;
  // and, for ARBGPU_ALG_AUTO products near the crossover, per size bucket whether Algorithm 2
  // measured faster than the classical dots; products run for those timings
  std::map<uint64_t, bool> alg_tuned;
  int64_t alg_tune_runs = 0;
  // streams on which arbgpu_mat_mul_batched runs its block items side by side, forked from and
  // joined back into the caller's stream (created on the first batched call that needs them)
  static constexpr int kLanes = 4;
  cudaStream_t lanes[kLanes] = {};
  cudaEvent_t lane_done[kLanes] = {};
  cudaEvent_t lane_fork = nullptr;
  // arbgpu_series_exp's recurrence recorded as CUDA graphs, keyed by the call's arguments (the
  // graphs bake the pointers in), most recent last; the private stream they are captured on
  struct SeriesGraph {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec;
    int64_t kernels;
  };
  std::vector<SeriesGraph> series_graphs;
  cudaStream_t capture_stream = nullptr;
};

namespace arbgpu {

// Bracket a kernel launch: counts it and, when tracing is on, records events around it.
struct LaunchScope {
  arbgpu_ctx *ctx;
  cudaStream_t stream;
  int idx;
  LaunchScope(arbgpu_ctx *c, cudaStream_t s, const char *name, int64_t units = 0);
  ~LaunchScope();
};

}  // namespace arbgpu

namespace arbgpu {

// Argument checks of the C ABI (api.cu): a well-formed ball array; whether two arrays share memory.
bool balls_ok(const arbgpu_balls &b);
bool balls_alias(const arbgpu_balls &out, const arbgpu_balls &in);

// Kernel (a): batched dots (real or complex).
arbgpu_status launch_batched_dot(arbgpu_ctx *ctx, const arbgpu_balls *res,
                                 const arbgpu_balls *initial, const uint8_t *sub,
                                 const arbgpu_balls *x, const int64_t *xoff, const int64_t *xstep,
                                 const arbgpu_balls *y, const int64_t *yoff, const int64_t *ystep,
                                 const int64_t *len, const int32_t *prec, int64_t batch,
                                 int32_t prec_max, int64_t len_max, int complex_mode,
                                 cudaStream_t stream, bool approx = false, bool reduce = false,
                                 bool fused = false);

// Kernel (a) over rows x columns: the classical matrix product, one warp per output entry.
arbgpu_status launch_matmul_dot(arbgpu_ctx *ctx, const arbgpu_balls *C, const arbgpu_balls *A,
                                const arbgpu_balls *B, int64_t M, int64_t K, int64_t N,
                                int64_t lda, int64_t ldb, int64_t ldc, int32_t prec,
                                int complex_mode, cudaStream_t stream);

// Tensor-core digit GEMM (tc_gemm.cu): T = X * Y over Z from balanced base-256 digit planes.
//   A: BF16 [SA][M][Kp], B: BF16 [SB][N][Kp] (both K contiguous, Kp a multiple of 64, zero padded)
//   digits: uint8 [SA+SB-1][Mp][Np], carries: int32 [groups][Mp][Np] with Mp, Np = M, N rounded
//   up to 128.  T[i][j] = sum_d digits[d][i][j] 256^d + sum_g carries[g][i][j] 256^dend(g), where
//   dend(g) is the end of group g's diagonal range (digit_gemm_group_ends).
struct DigitGemmArgs {
  const void *A;
  const void *B;
  int M, N;
  int64_t Kp;
  int SA, SB;
  int groups;
  uint8_t *digits;
  int32_t *carries;
  const char *name;
  int batch = 1;  // independent products sharing the plane layout (item b: planes b*SA.., b*SB..)
  // multimodular mode (SA = SB = 2, one group): item b writes P_b mod m_b as uint16 [batch][Mp][Np]
  // instead of digits and carries; ztab [batch][4] = m, float(m), float(1 / m), 0 and zinv [batch] =
  // floor((2^64 - 1) / m)
  uint16_t *zout = nullptr;
  const uint32_t *ztab = nullptr;
  const uint64_t *zinv = nullptr;
  // in that mode, items from `nz` on (when zraw is set) write their exact P as int64 [Mp][Np]
  // to zraw instead (nonnegative products, for instance the radius bounds)
  int nz = 0;
  int64_t *zraw = nullptr;
};
// Whether multimodular-mode products of this inner dimension run in the one-chain kernel (the one
// that also takes raw items).
bool crt_gemm_one_chain(int64_t Kp);
arbgpu_status launch_digit_gemm(arbgpu_ctx *ctx, const DigitGemmArgs &a, cudaStream_t stream);
int digit_gemm_groups(arbgpu_ctx *ctx, int M, int N, int ND);
bool digit_gemm_fits(int SA, int SB, int64_t Kp);
// The diagonal ranges the launcher uses: ends[g] = first diagonal after group g (g < groups).
void digit_gemm_group_ends(int SA, int SB, int groups, int *ends);

// Statistics of the scans of one real product's operands (zero-initialised: every field's identity).
struct BlockStats {
  int64_t pA, pB;         // largest significant-bit count of an entry
  int64_t hA, hB;         // largest row / column height (top - bottom)
  int32_t special;        // NaN / infinity / out-of-range exponent seen
  int32_t radA, radB;     // a nonzero radius seen
  int32_t pad;
};

// Copy n BlockStats from device memory to `host` and wait for them: a kernel stores them into the
// context's mapped pinned buffer (no copy engine, so the read does not queue behind large copies
// that other streams have in flight), then the stream is synchronised.
arbgpu_status read_stats(arbgpu_ctx *ctx, const BlockStats *dev, BlockStats *host, size_t n,
                         cudaStream_t s);

// The block product in two phases, for callers that run many products: block_scan_launch (scans
// into a region of block_scan_bytes, no synchronisation; the four BlockStats -- rows of A0, A1,
// columns of B0, B1 -- go to `stats`, zeroed by the caller, or to the region when null), then,
// once those statistics are on the host, block_finish.  Either returns ARBGPU_ERR_LIMIT for a
// product the block path does not take (then: dot products).
size_t block_scan_bytes(int64_t M, int64_t N, bool cplx);
arbgpu_status block_scan_launch(arbgpu_ctx *ctx, const arbgpu_balls *A, const arbgpu_balls *B,
                                int64_t M, int64_t K, int64_t N, int64_t lda, int64_t ldb,
                                bool cplx, void *region, BlockStats *stats, cudaStream_t s);
arbgpu_status block_finish(arbgpu_ctx *ctx, const arbgpu_balls *C, const arbgpu_balls *A,
                           const arbgpu_balls *B, int64_t M, int64_t K, int64_t N, int64_t lda,
                           int64_t ldb, int64_t ldc, int prec, bool cplx, bool m3, void *region,
                           const BlockStats *hst, void *workspace, size_t ws_bytes,
                           cudaStream_t s, bool *used_block);

// Block algorithm (block.cu): real or complex (C, A, B point to one or two arbgpu_balls).  Returns
// ARBGPU_ERR_LIMIT (and *used_block = false) when the inputs hold special values or exceed the
// path's limits.
// m3: complex midpoints by eq. 2 (three real products) where the parts share one scaling in a
// single block; the workspace then holds the three products' planes.
size_t block_workspace_size(arbgpu_ctx *ctx, int64_t M, int64_t K, int64_t N, int prec,
                            bool cplx, bool m3, int nlA, int nlB);
// Uploads every multimodular table for products up to these sizes (arbgpu_reserve).
arbgpu_status block_reserve(arbgpu_ctx *ctx, int max_prec, int64_t max_inner);
arbgpu_status block_matmul(arbgpu_ctx *ctx, const arbgpu_balls *C, const arbgpu_balls *A,
                           const arbgpu_balls *B, int64_t M, int64_t K, int64_t N, int64_t lda,
                           int64_t ldb, int64_t ldc, int prec, bool cplx, bool m3,
                           void *workspace, size_t ws_bytes, cudaStream_t s, bool *used_block);

// Dot products that finish the basecase blocks of Algorithm 2 (dot_basecase.cu): entry (i, j) of C
// is initial[i*N + j] + sum over the tagged indices e = bk[t] (k = e >> 2, combo = e & 3) of
// +- X[i*lda + k] * Y[k*ldb + j] with (X, Y, sign) = (A0, B0, +), (A1, B1, -), (A0, B1, +),
// (A1, B0, +) for combo 0..3 (A1, B1: imaginary parts, used when cplx).
arbgpu_status launch_basecase_dot(arbgpu_ctx *ctx, const arbgpu_balls &C, const arbgpu_balls *A,
                                  const arbgpu_balls *B, bool cplx, const arbgpu_balls &initial,
                                  const int32_t *bk, int64_t nbk, int64_t M, int64_t N,
                                  int64_t lda, int64_t ldb, int64_t ldc, int32_t prec,
                                  cudaStream_t stream);

// Integer matrix product on a caller-provided workspace (intmm.cu); ctx->device must be current.
arbgpu_status int_mat_mul_run(arbgpu_ctx *ctx, uint64_t *T, int32_t t_limbs, const uint64_t *X,
                              int32_t x_limbs, const uint64_t *Y, int32_t y_limbs, int64_t M,
                              int64_t K, int64_t N, void *workspace, size_t ws_bytes,
                              cudaStream_t s);
size_t int_mat_mul_workspace(arbgpu_ctx *ctx, int xl, int yl, int64_t M, int64_t K, int64_t N);

// Grouped classical products (dot_grouped.cu): one launch sequence over the items of a device work
// list; `ends` holds the running totals of virtual dots (item q owns dots [ends[q-1], ends[q])).
struct GroupItem {
  BallsView A[2], B[2];
  BallsOut C[2];
  int64_t M, N, K, lda, ldb, ldc;
  int32_t prec, cplx;
};
arbgpu_status launch_grouped_dot(arbgpu_ctx *ctx, const GroupItem *dev_items,
                                 const int64_t *dev_ends, int32_t count, int64_t total_dots,
                                 int prec_max, int64_t k_max, int max_nlimbs, cudaStream_t stream);

// Multimodular engine (crt.cu): moduli = the NM largest primes below 2^16.
constexpr int CRT_MAX_CHUNKS32 = 50;  // 32-bit chunks of a scaled integer (1600 bits)
constexpr int CRT_MAX_MODULI = 256;
struct CrtPlan {
  int NM, NMW, NCHP, NW32P;       // moduli, limbs of M, columns of pow32, columns of Q32
  std::vector<uint32_t> mods;     // m_t
  std::vector<uint64_t> inv;      // [3 NM]: floor((2^64 - 1) / m_(t mod NM))
  std::vector<uint32_t> pow32;    // [NM][NCHP]: 2^(32c) mod m_t
  std::vector<uint32_t> Q32;      // [NM][NW32P]: M / m_t in 32-bit limbs, zero padded
  std::vector<uint32_t> M32;      // [NW32P]: M in 32-bit limbs
  std::vector<uint32_t> y;        // [NM]: (M / m_t)^-1 mod m_t
  std::vector<float> rinv;        // [NM]: 1 / m_t rounded to float
  std::vector<uint32_t> ztab;     // [3 NM][4]: m, float(m), float(1 / m), 0 (m = m_(t mod NM))
  std::vector<uint64_t> M;        // M
  int NPAD;                       // 2 NM rounded up to a multiple of 16
  // [2][NPAD][128] BF16 bits: row 2t + b of operand side o holds byte b (balanced, 256 h + l) of
  // the balanced w = 2^(8d) mod m_t (side 0) or 2^(8d) y_t mod m_t (side 1) in column d
  std::vector<uint16_t> wtab;
  // Reconstruction on the tensor cores (NM <= 64): the output has NQ byte columns (balanced
  // bytes of sum_t z_t Q_t, a q column follows); crt_wtab [NQP][128] BF16 bits, row n < NQ holding
  // byte n of Q_t in column 2t and byte n - 1 in column 2t + 1 (z_t = l + 256 h, bytes l, h), row
  // NQ holding 1 / m_t and 256 / m_t (rounded to BF16); mbytes [NQ]: the balanced bytes of M.
  int NQ, NQP;
  std::vector<uint16_t> crt_wtab;
  std::vector<float> mbytes;
  // The same bytes as 8-bit integers for the warp-level MMA reconstruction (every NM): w8
  // [NQ8][K8], row n holding byte n of Q_t in column 2t and byte n - 1 in column 2t + 1 (zero
  // padded: K8 = 2 NM and NQ8 = NQ rounded up to multiples of 32).
  int K8, NQ8;
  std::vector<int8_t> w8;
  // The z bytes enter that product offset by -128 (as signed bytes): c32 [2 NMW + 2] holds
  // 32896 sum_t Q_t in 32-bit words, the term that puts the offset back.
  std::vector<uint32_t> c32;
  // Residue weights as unsigned bytes for the warp-level MMA residue step (every NM): w8r
  // [2][N2][KR], side o, column n = 2t + b holding byte b of 2^(8d) mod m_t (times y_t for side
  // 1) in row d (N2 = 2 NM rounded up to 32, KR = 4 CRT_MAX_CHUNKS32 rounded up to 32).
  int N2, KR;
  std::vector<uint8_t> w8r;
};
int crt_moduli_for_bits(int bits);
const CrtPlan *crt_plan(int NM);
// Device copies of a plan's tables, uploaded once per context and modulus count.
struct CrtDevTables {
  const uint32_t *Q32, *M32, *y, *ztab, *pow32;
  const float *rinv;
  const uint16_t *wtab;
  const uint16_t *crt_wtab;
  const float *mbytes;
  const uint64_t *inv;
  const int8_t *w8;
  const uint32_t *c32;
  const uint8_t *w8r;
};
arbgpu_status crt_device_tables(arbgpu_ctx *ctx, const CrtPlan *plan, CrtDevTables *out);

// Inner ordering (inner_order.cu), from a_k / b_k = the largest tops of column k of A / row k of B
// (INT64_MIN when all zero): `ord` lists the indices with a nonzero midpoint product by a_k + b_k
// (ties by index), then the others; g_k = floor((b_k - a_k) / 2) for the former, 0 for the latter.
void inner_order_host(const std::vector<int64_t> &a, const std::vector<int64_t> &b,
                      std::vector<int32_t> &ord, std::vector<int64_t> &g);

// Dot-kernel size class for a precision, a maximal term count and operand limb counts (-1: none).
int dot_class_for_problem(int prec, int64_t max_terms, int max_nlimbs);

}  // namespace arbgpu
