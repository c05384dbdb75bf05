/*
 * arbgpu -- arbitrary-precision real and complex ball dot products and matrix multiplication on a
 * GB300 GPU (sm_103a), after F. Johansson, "Faster arbitrary-precision dot product and matrix
 * multiplication" (arXiv 1901.04289).
 *
 * Plain C ABI: device pointers, sizes and a CUDA stream passed as `void *`; no C++ or framework
 * types.  Every call is asynchronous on the given stream unless stated otherwise.  The caller owns
 * every buffer (inputs, outputs, workspace); the library never allocates device memory on these
 * paths and never falls back to the CPU.
 *
 * ---------------------------------------------------------------------------------------------
 * Ball layout (Section III-A).  An array of `count` balls is five device arrays:
 *
 *   limbs   uint64  limb k (0 = least significant) of entry i at limbs[k * limb_stride + i],
 *                   k < nlimbs ("limb planes").  A nonzero finite midpoint is
 *                   m = (-1)^sign * 2^exp * sum_k limbs[k] * 2^(64 (k - nlimbs))      (eq. 1)
 *                   with bit 63 of limb nlimbs-1 set; low limbs may be zero.
 *   exp     int64   2^(exp-1) <= |m| < 2^exp.
 *   flags   uint32  bit 0 sign, bit 1 zero (limbs must then be zero), bit 2 infinity, bit 3 NaN,
 *                   bit 4 infinite radius; bits 8..15: n, the number of limbs from the top down to
 *                   the lowest nonzero limb (1 <= n <= nlimbs) -- the "limb count" of eq. 1.
 *   rad_man uint32  radius r = rad_man * 2^(rad_exp - 30), rad_man = 0 or 2^29 <= rad_man < 2^30
 *   rad_exp int64   (a 30-bit "mag", p_rad = 30).
 *
 * Exponents must satisfy |exp| < 2^60 (and |rad_exp| < 2^60 for nonzero radii); NaN, infinities
 * and larger exponents are reported as ARBGPU_ERR_UNSUPPORTED_VALUE (where the paper leaves the
 * fixed-point path for a fallback, Section III-C) and the affected outputs are set to
 * [NaN +- inf] (flags = NaN | infinite radius).
 *
 * Outputs are written with the output array's own nlimbs (>= ceil(p/64)): the midpoint rounded to
 * nearest (ties to even) at p bits, top-aligned, and a radius rounded up.
 * ---------------------------------------------------------------------------------------------
 */
#ifndef ARBGPU_H
#define ARBGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ARBGPU_OK = 0,
  ARBGPU_ERR_INVALID = 1,           /* bad argument (returned synchronously) */
  ARBGPU_ERR_UNSUPPORTED_VALUE = 2, /* NaN / infinity / |exponent| >= 2^60 in an input */
  ARBGPU_ERR_WORKSPACE = 3,         /* workspace missing or too small */
  ARBGPU_ERR_CUDA = 4,              /* a CUDA runtime call failed */
  ARBGPU_ERR_TIMEOUT = 5,           /* a bounded device-side wait gave up */
  ARBGPU_ERR_LIMIT = 6              /* a per-call size hint (max precision / length) exceeded */
} arbgpu_status;

/* Flag bits of the layout above. */
#define ARBGPU_FLAG_SIGN 1u
#define ARBGPU_FLAG_ZERO 2u
#define ARBGPU_FLAG_INF 4u
#define ARBGPU_FLAG_NAN 8u
#define ARBGPU_FLAG_RAD_INF 16u
#define ARBGPU_NSIG_SHIFT 8

/* One ball array (all pointers device memory, caller-owned). */
typedef struct {
  uint64_t *limbs;
  int64_t limb_stride; /* elements between limb planes, >= count */
  int32_t nlimbs;      /* limbs per midpoint, 1..64 */
  int64_t *exp;
  uint32_t *flags;
  uint32_t *rad_man;
  int64_t *rad_exp;
  int64_t count;
} arbgpu_balls;

typedef struct arbgpu_ctx arbgpu_ctx;

/* Library context for one device: holds the device status word.  Create before use, on the host
 * thread that will use it; one context per host thread.  `device` is a CUDA device ordinal.
 * Allocates a few bytes of device memory and a small mapped pinned host buffer once (here, not on
 * the compute paths). */
arbgpu_status arbgpu_create(arbgpu_ctx **ctx, int device);
arbgpu_status arbgpu_destroy(arbgpu_ctx *ctx);

/* Set-up of the block algorithm's constant tables (host-only, synchronous): uploads, into device
 * memory owned by `ctx`, every table of the multimodular engine (the moduli, weights and cofactors
 * of Section IV-A's integer product) that a matrix product at precision <= max_prec with an inner
 * dimension <= max_inner can use.  Without it, the first product that needs a table uploads it
 * (one cudaMalloc per modulus count, kept until arbgpu_destroy); after it, such products allocate
 * nothing.  Call it before capturing matrix products in a CUDA graph.  max_prec in [2, 1024]. */
arbgpu_status arbgpu_reserve(arbgpu_ctx *ctx, int32_t max_prec, int64_t max_inner);

/* Calibration (host-side, synchronous, on the legacy default stream of ctx's device; a few tens
 * of milliseconds): measured throughput of the arithmetic units the two exact-product carriers of
 * Section III-D / IV-A would run on, by three micro-kernels of 4 x 256-thread CTAs per SM with
 * independent dependency chains:
 *   imad_tops       tera 32-bit multiply-adds per second (mad.lo.u32), the CUDA-core rate that
 *                   bounds Algorithm 1's limb products;
 *   imad_wide_tops  tera 32x32+64 -> 64-bit multiply-adds per second (mad.wide.u32);
 *   mma_s8_tops     tera integer operations per second (2 per multiply-add) of the warp-level
 *                   8-bit tensor MMA mma.sync m16n8k32 s8.s8.s32 (the tcgen05 8-bit kind is not
 *                   available on sm_103a), the alternative carrier to the BF16 digit products;
 *   sm_count, max_clock_mhz  the device's SM count and maximum SM clock.
 * Allocates and frees a small device buffer and two events.  ARBGPU_ERR_CUDA on any CUDA
 * failure (the fields are then zero). */
typedef struct {
  double imad_tops;
  double imad_wide_tops;
  double mma_s8_tops;
  int32_t sm_count;
  double max_clock_mhz;
} arbgpu_calibration;

arbgpu_status arbgpu_calibrate(arbgpu_ctx *ctx, arbgpu_calibration *out);

/* Engine autotuner for the block algorithm's exact integer products (Section IV-A).  The
 * library has two exact carriers for them: S_A x S_B products of balanced 8-bit digit slices, or
 * 4 NM products of residues modulo NM 16-bit primes followed by a Chinese-remainder
 * reconstruction.  Both give the same integers bit for bit, so the choice only changes the time.
 * By default a cost model with per-unit constants measured on GB300 chooses.  With the autotuner
 * on (enable != 0), the first block product of each size bucket (the digit counts, the modulus
 * count, and M, N and the padded inner length rounded up to powers of two) that both engines can
 * take runs on both, once untimed and once timed with CUDA events (four products in all).  That
 * call synchronises its stream. The faster engine
 * is kept for the bucket, for the context's lifetime, and later products of the bucket use it.
 * While the stream is being captured into a CUDA graph, no timing runs: undecided buckets use the
 * cost model.  Outputs never depend on the engine choice.
 * arbgpu_autotune_stats: buckets decided so far, products run for the timings, and how many of
 * the decided buckets chose the multimodular engine (any pointer may be null).
 *
 * The same switch times the algorithm of ARBGPU_ALG_AUTO matrix products near the crossover
 * between the classical dots and Algorithm 2 (the paper finds it at N = 40..60, Section V):
 * for 8 <= M, N <= 512 and 30 <= K <= 512, the first AUTO product of a size bucket (M, K, N
 * rounded up to powers of two, the precision in limbs, complex, eq. 2) runs both algorithms once
 * untimed and once timed (four products; the call synchronises its stream), keeps the faster for
 * the bucket and leaves its result in C; arbgpu_mat_mul_batched times such items alone before
 * the batch.  Outside that range, with the autotuner off, or while the stream is captured, the
 * fixed rule (Algorithm 2 for M, N, K >= 48) applies.  The two algorithms give different balls
 * (both contain the exact product within the accuracy bound), so with the autotuner on an AUTO
 * product's result depends on the measured choice.  The workspace size queries count the block
 * algorithm's workspace for the products the autotuner may give it: query them after
 * arbgpu_set_autotune.
 * arbgpu_autotune_alg_stats: AUTO buckets decided, products run for their timings, and how many
 * chose Algorithm 2 (any pointer may be null). */
arbgpu_status arbgpu_set_autotune(arbgpu_ctx *ctx, int enable);
arbgpu_status arbgpu_autotune_stats(arbgpu_ctx *ctx, int64_t *buckets, int64_t *timing_runs,
                                    int64_t *crt_buckets);
arbgpu_status arbgpu_autotune_alg_stats(arbgpu_ctx *ctx, int64_t *buckets, int64_t *timing_runs,
                                        int64_t *block_buckets);

/* Synchronises `stream`, returns the first device-side error recorded since the previous call
 * (ARBGPU_OK if none) and clears it. */
arbgpu_status arbgpu_get_status(arbgpu_ctx *ctx, void *stream);

/* Human-readable name of a status code (static string). */
const char *arbgpu_status_string(arbgpu_status s);

/* Library version as major*10000 + minor*100 + patch. */
int arbgpu_version(void);

/* Tracing (host-side, no effect on results).
 * arbgpu_launch_count: number of kernels launched through `ctx` so far.
 * arbgpu_trace_enable: when on, every kernel launch is bracketed by a pair of CUDA events recorded
 *   on its stream (a few microseconds of overhead per launch).
 * arbgpu_trace_read: waits for the recorded launches, writes up to `max_entries` records (kernel
 *   name -- a static string --, device time in ms, and the algorithmic work units the launch
 *   processed -- dot_fused / dot_setup / dot_eval (the last class launch of a call): dots
 *   (arbgpu_dot) or terms (matrix products); digit_gemm* / crt_gemm: digit multiply-adds on the
 *   tensor cores; residues_*: 32x16-bit multiply-adds; block_round: 32-bit multiply-adds of the
 *   CRT sums (multimodular) or entries; others: entries), the launch's start in ms after the
 *   first recorded launch's start, and clears the record list. */
typedef struct {
  const char *name;
  float ms;
  int64_t units;
  float start_ms;
} arbgpu_trace_entry;

arbgpu_status arbgpu_launch_count(arbgpu_ctx *ctx, int64_t *count);
arbgpu_status arbgpu_trace_enable(arbgpu_ctx *ctx, int enable);
arbgpu_status arbgpu_trace_read(arbgpu_ctx *ctx, arbgpu_trace_entry *out, int32_t max_entries,
                                int32_t *n_entries);

/*
 * Batched ball dot products: Algorithm 1 (Section III), the counterpart of arb_dot / acb_dot:
 *
 *   res[b]  contains  initial[b] + (-1)^sub[b] * sum_{i < len[b]} x[xoff[b] + i*xstep[b]]
 *                                                               * y[yoff[b] + i*ystep[b]]
 *
 * computed at precision prec[b] >= 2 (bits).  One warp evaluates one dot: a setup pass over the
 * terms (exponent bounds, accumulator size), exact limb products accumulated in a two's-complement
 * fixed-point window of n_s limbs, a ulp error counter and a fixed-point radius accumulator, then
 * one rounding to p bits (round to nearest, ties to even) and an upward-rounded radius.
 *
 *   res      output balls, entry b written (res->nlimbs >= ceil(prec[b]/64)); must not alias inputs
 *   initial  optional (NULL): entry b is added with a plus sign
 *   sub      optional (NULL = all 0) device uint8[batch]
 *   x, y     input ball arrays; xoff/xstep/yoff/ystep/len device int64[batch] (strides may be
 *            negative or zero; every index touched must lie in [0, count))
 *   prec     device int32[batch]
 *   prec_max, len_max  host-side upper bounds of prec[] and len[] over the batch, used to choose
 *            the kernel; a dot exceeding them is written as [NaN +- inf] with ARBGPU_ERR_LIMIT
 *            (prec_max <= 1024; larger precisions return ARBGPU_ERR_INVALID)
 *   complex_mode  0: real.  1: complex -- res, initial, x and y each point to TWO arbgpu_balls
 *            (real part, imaginary part); each part of the result is a real dot of length 2N
 *            (Section III-F).
 *   workspace, ws_bytes  unused (may be NULL / 0)
 *   stream   cudaStream_t
 * Errors: argument errors return synchronously; value errors through arbgpu_get_status.
 */
arbgpu_status arbgpu_dot(arbgpu_ctx *ctx, const arbgpu_balls *res, const arbgpu_balls *initial,
                         const uint8_t *sub, const arbgpu_balls *x, const int64_t *xoff,
                         const int64_t *xstep, const arbgpu_balls *y, const int64_t *yoff,
                         const int64_t *ystep, const int64_t *len, const int32_t *prec,
                         int64_t batch, int32_t prec_max, int64_t len_max, int complex_mode,
                         void *workspace, size_t ws_bytes, void *stream);

/* Options of arbgpu_dot_ex. */
#define ARBGPU_DOT_APPROX 1u      /* midpoints only: the input radii are ignored, zero radii out */
#define ARBGPU_DOT_REDUCE_PREC 2u /* the precision reduction ("optimize p") of Section III-C: per dot,
                                   * p <- min(p, e_max - e_rad + 30) when a radius is present and,
                                   * for p > 128, p <- min(p, e_max - e_min + 30) (e_min: the lowest
                                   * possible bit of a product); then p >= 2, and p = 2 when every
                                   * midpoint product is zero.  The midpoint is computed and rounded
                                   * at the reduced precision; the ball still contains the exact
                                   * result. */

/* arbgpu_dot with options (a bitwise OR of ARBGPU_DOT_*); the other arguments as for arbgpu_dot. */
arbgpu_status arbgpu_dot_ex(arbgpu_ctx *ctx, const arbgpu_balls *res, const arbgpu_balls *initial,
                            const uint8_t *sub, const arbgpu_balls *x, const int64_t *xoff,
                            const int64_t *xstep, const arbgpu_balls *y, const int64_t *yoff,
                            const int64_t *ystep, const int64_t *len, const int32_t *prec,
                            int64_t batch, int32_t prec_max, int64_t len_max, int complex_mode,
                            uint32_t options, void *workspace, size_t ws_bytes, void *stream);

/* Midpoint-only dots, the counterpart of arb_approx_dot / acb_approx_dot (Section III: the same
 * interface without error bounds).  Same arguments and errors as arbgpu_dot.  Each midpoint is the
 * one arbgpu_dot computes (the same accumulation, one rounding to prec bits); the input radii are
 * ignored and the output radii are zero: no error bound is claimed.  Special values give
 * [NaN +- inf] with ARBGPU_ERR_UNSUPPORTED_VALUE, as in arbgpu_dot. */
arbgpu_status arbgpu_approx_dot(arbgpu_ctx *ctx, const arbgpu_balls *res,
                                const arbgpu_balls *initial, const uint8_t *sub,
                                const arbgpu_balls *x, const int64_t *xoff, const int64_t *xstep,
                                const arbgpu_balls *y, const int64_t *yoff, const int64_t *ystep,
                                const int64_t *len, const int32_t *prec, int64_t batch,
                                int32_t prec_max, int64_t len_max, int complex_mode,
                                void *workspace, size_t ws_bytes, void *stream);

/* Algorithm selection for arbgpu_mat_mul. */
#define ARBGPU_ALG_AUTO 0
#define ARBGPU_ALG_DOT 1   /* classical: M*N dot products (Section IV, first paragraph) */
#define ARBGPU_ALG_BLOCK 2 /* scaled integer blocks (Algorithm 2, Section IV-A) */

/* Flags for arbgpu_mat_mul. */
/* Complex midpoints by eq. 2 (Section IV-C): when one exponent per row of A and per column of B,
 * shared by the real and imaginary parts, scales both parts to integers within one block of
 * Algorithm 2, Re = Ar Br - Ai Bi and Im = (Ar + Ai)(Br + Bi) - Ar Br - Ai Bi are formed exactly
 * from three integer products instead of four and rounded once; radii come from the four real
 * radius products as without the flag.  When the shared scaling needs several blocks and the
 * negligible-limb omission is on (ARBGPU_OMIT, see arbgpu_mat_mul), both parts drop their bits
 * below thresholds shared by the parts (each part's error stays within (1/32) 2^-p times the sum
 * of |a b| over its own terms); when the truncated parts fit one shared block, eq. 2 runs on them
 * and each part is rounded once, and otherwise four real products, each with its own omission,
 * run instead.  With the omission off, the inner range is cut once for both parts (Section IV-C's
 * second suggestion: the greedy extraction on the larger top and the smaller bottom of each
 * entry's two parts, over an inner order and scaling shared by the parts when the inner ordering
 * is on); each full block's Re and Im come from three exact products and are added into the
 * parts' window accumulators, the basecase blocks become complex dot products.  Blocks the
 * tensor-core residue kernel cannot take (more than 32 chunks or 128 moduli) leave the four real
 * products in place, and the dot path ignores the flag.  Any other flag bit is
 * ARBGPU_ERR_INVALID. */
#define ARBGPU_MM_COMPLEX_3M 1u

/*
 * Ball matrix product C = A * B (C contains the exact product of every choice of points in the
 * input balls).  A is M x K, B is K x N, C is M x N, all row-major with leading dimensions
 * lda, ldb, ldc (entry (i, k) of A is index i*lda + k of its ball array).  Precision prec >= 2.
 *
 *   ARBGPU_ALG_DOT    every entry is one Algorithm-1 dot (warp per entry).
 *   ARBGPU_ALG_BLOCK  Algorithm 2: the inner dimension is cut greedily into blocks in which every
 *                     row of A and column of B scales to integers of height <= h
 *                     (h = 1.25 min(p, max(p_A, p_B)) + 192); each block's scaled integer matrices
 *                     are multiplied exactly on the tensor cores by one of two engines, chosen by a
 *                     cost model (the environment variable ARBGPU_ENGINE=digits|crt forces one):
 *                     signed 8-bit digit products, or residues modulo 16-bit primes and the Chinese
 *                     remainder theorem (BF16 digits, FP32 accumulation kept below 2^24, so every
 *                     product is exact); blocks shorter than 30 indices are done by dot products.
 *                     A single block is rounded once from its exact integer; several blocks are
 *                     summed in a fixed-point window placed under each entry's largest term
 *                     exponent, max_k top(a_ik) + top(b_kj), and the bits below it go to the
 *                     radius.  When the inner index in its own order needs several blocks, it is
 *                     first permuted and scaled (Section IV-B: column k of A times 2^g_k, row k of
 *                     B times 2^-g_k, indices sorted by their product bound), which often leaves
 *                     one block; a real product with one such block is rounded once from it.
 *                     The environment variable ARBGPU_INNER_ORDER=0 keeps the own order.
 *                     Before that, a product that needs several blocks and holds lines much
 *                     taller than p needs has its negligible limbs omitted (Section IV-B, last
 *                     paragraph): with E_ij = max_k top(a_ik) + top(b_kj), the bits of row i of A
 *                     below min_j (E_ij - top_j(B)) - p - bc(K) - 8 (and likewise for the
 *                     columns of B) are dropped and added to those entries' radii; the midpoint
 *                     error stays below (3/64) 2^-p sum_k |a_ik b_kj| and the ball stays
 *                     rigorous.  When the truncated operands fit one block, that block is used.
 *                     ARBGPU_OMIT=0 keeps every bit.  Radii:
 *                     |A| R_B + R_A (|B| + R_B) from exact integer products of magnitudes rounded
 *                     up to 8*S_r-bit windows.
 *   ARBGPU_ALG_AUTO   picks by size and precision.
 *
 *   complex_mode  0 real; 1 complex: C, A, B each point to TWO arbgpu_balls (real, imaginary)
 *   flags         0 or ARBGPU_MM_COMPLEX_3M (complex only; the same flags must be given to
 *                 arbgpu_mat_mul_workspace_size)
 *   workspace     device memory of at least arbgpu_mat_mul_workspace_size() bytes (BLOCK/AUTO)
 * The block path reads back a few bytes of statistics, and its plan when there are several blocks,
 * each with one stream synchronisation.
 */
arbgpu_status arbgpu_mat_mul(arbgpu_ctx *ctx, const arbgpu_balls *C, const arbgpu_balls *A,
                             const arbgpu_balls *B, int64_t M, int64_t K, int64_t N, int64_t lda,
                             int64_t ldb, int64_t ldc, int32_t prec, int complex_mode, int alg,
                             uint32_t flags, void *workspace, size_t ws_bytes, void *stream);

/*
 * Grouped batch of independent ball matrix products (the same operation as arbgpu_mat_mul, item by
 * item).  `descs` is a HOST array of `count` descriptors (device pointers inside).  Items that use
 * the classical algorithm (ARBGPU_ALG_DOT, or ARBGPU_ALG_AUTO below the block size) run together
 * in ONE launch of the dot kernel over a device work list (one warp per output entry, each item at
 * its own precision).  The other items run the block algorithm: their scans on `stream`, one
 * read-back of all their statistics, then the products on up to four internal streams of the
 * context side by side (created on the first batched call that needs them; forked from `stream`
 * and joined back into it, so work queued on `stream` afterwards sees every output).  Each
 * internal stream has its own share of the workspace; items keep their order within a stream.
 * Workspace: arbgpu_mat_mul_batched_workspace_size() (it covers the internal streams' shares).
 */
typedef struct {
  arbgpu_balls C[2], A[2], B[2]; /* [1] is the imaginary part when complex_mode */
  int64_t M, K, N, lda, ldb, ldc;
  int32_t prec;
  int32_t complex_mode;
  int32_t alg;    /* as for arbgpu_mat_mul */
  uint32_t flags; /* as for arbgpu_mat_mul: 0 or ARBGPU_MM_COMPLEX_3M */
} arbgpu_matmul_desc;

arbgpu_status arbgpu_mat_mul_batched(arbgpu_ctx *ctx, const arbgpu_matmul_desc *descs,
                                     int32_t count, void *workspace, size_t ws_bytes,
                                     void *stream);
arbgpu_status arbgpu_mat_mul_batched_workspace_size(arbgpu_ctx *ctx,
                                                    const arbgpu_matmul_desc *descs,
                                                    int32_t count, size_t *bytes);

/*
 * The block plans (Algorithm 2's greedy extraction, Section IV-A) that the last arbgpu_mat_mul or
 * arbgpu_mat_mul_batched call on `ctx` used, for inspection and testing (host-only, synchronous;
 * the plans are known on the host once that call has returned).  One record per real product
 * that ran the block algorithm, in the order they ran (a complex product by four real products
 * gives Ar Br, Ai Bi, Ar Bi, Ai Br; batched items in item order):
 *   kind   0: blocks over the inner index in its own order; 1: over the inner ordering (the
 *          block positions index the order listed after the triples); 2: the blocks of a
 *          complex product by eq. 2 (ARBGPU_MM_COMPLEX_3M) shared by both parts, planned on
 *          the larger top and smaller bottom of each entry's two parts (Section IV-C; one record
 *          for the whole complex product); 3: one block of the operands with their negligible
 *          limbs omitted (see arbgpu_mat_mul); 4: the shared blocks of kind 2 over an inner
 *          order and scaling shared by both parts (listed as for kind 1); 5: one block shared by
 *          both parts of a complex product by eq. 2 after both parts' negligible limbs were
 *          omitted under thresholds shared by the parts
 *   h      the height bound, floor(1.25 min(p, max(p_A, p_B))) + 192
 *   K      the inner dimension
 *   nb     the number of blocks, then nb triples (start, stop, basecase): [start, stop) covers
 *          positions of the inner index; basecase = 1 for a block done by dot products
 *   kinds 1 and 4 only: K positions' inner indices (the order), then K inner scaling
 *          exponents g_k
 * `words` receives the first min(n, max_words) words; *n_words is set to n.  A call that took
 * the classical algorithm leaves no record.
 */
arbgpu_status arbgpu_last_plans(arbgpu_ctx *ctx, int64_t *words, int64_t max_words,
                                int64_t *n_words);

/* Workspace bytes arbgpu_mat_mul needs for these sizes (host-only, synchronous).  `a_nlimbs` and
 * `b_nlimbs` are the input arrays' limb counts (the larger of the two parts when complex, 1..64):
 * the inner ordering keeps reordered copies of the operands at these widths. */
arbgpu_status arbgpu_mat_mul_workspace_size(arbgpu_ctx *ctx, int64_t M, int64_t K, int64_t N,
                                            int32_t prec, int32_t a_nlimbs, int32_t b_nlimbs,
                                            int complex_mode, int alg, uint32_t flags,
                                            size_t *bytes);

/*
 * Power series exponential, the consumer of the dot product that Section V describes: for each of
 * `batch` series a_1 x + a_2 x^2 + ... (a_0 is ignored), the coefficients b_0 .. b_{len-1} of its
 * exponential by the recurrence b_0 = 1, b_k = (sum_{j=1}^k (j a_j) b_{k-j}) / k, each step one
 * batched call of the Algorithm 1 dot kernel over all series (j a_j and the division by k are dots
 * of length one against exact integer balls and balls containing 1/k).
 *   a, res   ball arrays of len * batch entries: coefficient k of series s at index k batch + s
 *            (res->nlimbs >= ceil(prec / 64)); res must not alias a
 *   prec     working and output precision in bits, 2..1024
 *   workspace  device memory of at least arbgpu_series_exp_workspace_size() bytes
 * Every output ball contains the exact coefficient of the exponential of every series whose
 * coefficients lie in the input balls.  2 (len - 1) + 1 batched dot calls, each one launch of the
 * dot kernel (setup and evaluation fused: the dots of a call share one precision).
 * The first call with a given set of arguments (pointers, sizes, precision, workspace) records its
 * launches as a CUDA graph, on a private stream of the context (host time of a few milliseconds
 * for long series), and replays it on `stream`; later calls with the same arguments only replay
 * it.  The context keeps the four most recent graphs.  While tracing is on, while `stream` is
 * itself being captured, or with ARBGPU_SERIES_GRAPH=0, the launches go to `stream` directly.
 * The outputs are the same either way.
 */
arbgpu_status arbgpu_series_exp(arbgpu_ctx *ctx, const arbgpu_balls *res, const arbgpu_balls *a,
                                int64_t len, int64_t batch, int32_t prec, void *workspace,
                                size_t ws_bytes, void *stream);
arbgpu_status arbgpu_series_exp_workspace_size(arbgpu_ctx *ctx, int64_t len, int64_t batch,
                                               int32_t prec, size_t *bytes);

/*
 * Exact integer matrix product T = X * Y over Z, reduced modulo 2^(64 t_limbs): the engine behind
 * the block path (it replaces the paper's FLINT fmpz_mat_mul, Section IV).  Signed integers in
 * two's complement limb planes: X[k * (M*K) + i*K + kk] is limb k (little-endian) of X[i][kk],
 * x_limbs limbs per entry; likewise Y (K x N, y_limbs) and T (M x N, t_limbs).  The operands are
 * split into balanced signed base-256 digits and every digit product is formed exactly on the
 * tensor cores.  `workspace` must hold arbgpu_int_mat_mul_workspace_size() bytes.
 */
arbgpu_status arbgpu_int_mat_mul(arbgpu_ctx *ctx, uint64_t *T, int32_t t_limbs, const uint64_t *X,
                                 int32_t x_limbs, const uint64_t *Y, int32_t y_limbs, int64_t M,
                                 int64_t K, int64_t N, void *workspace, size_t ws_bytes,
                                 void *stream);

arbgpu_status arbgpu_int_mat_mul_workspace_size(arbgpu_ctx *ctx, int32_t x_limbs, int32_t y_limbs,
                                                int64_t M, int64_t K, int64_t N, size_t *bytes);

/*
 * Allocation-free integer product.  The paper has no counterpart: this is a convenience of this
 * library for callers that cannot call cudaMalloc -- for example a host program whose device
 * memory is entirely held by another allocator's pool, or a thread that must not enter the CUDA
 * allocator at all.  It computes exactly what arbgpu_int_mat_mul computes (same argument meaning
 * and layout) but allocates nothing and needs no context: its scratch space is one device array of
 * ARBGPU_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the library keeps
 * until the process exits.
 *   - Runs on the current device and on `stream`.  The first call on each device looks up the
 *     array's device address (cudaGetSymbolAddress with that device current) and keeps it for
 *     the life of the process; make that first call before any stream capture, and do not use
 *     this call after cudaDeviceReset (the kept address would then be stale).
 *   - Empty products (M or N zero) return ARBGPU_OK and write nothing; K = 0 writes zeros; none
 *     of these touch the scratch array.
 *   - Sizes whose scratch would exceed ARBGPU_NOALLOC_SCRATCH_BYTES are rejected synchronously
 *     with ARBGPU_ERR_LIMIT (arbgpu_int_mat_mul_workspace_size gives the scratch a size needs).
 *   - Every call shares the one array, which keeps the last call's contents: calls whose GPU work
 *     overlaps (other streams, other host threads) race; order them on one stream.
 *   - status: optional device int (NULL allowed); the call sets it to 0 and the kernels record
 *     the first device-side error (ARBGPU_ERR_TIMEOUT) there.
 */
#define ARBGPU_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
arbgpu_status arbgpu_int_mat_mul_noalloc(uint64_t *T, int32_t t_limbs, const uint64_t *X,
                                         int32_t x_limbs, const uint64_t *Y, int32_t y_limbs,
                                         int64_t M, int64_t K, int64_t N, int *status,
                                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ARBGPU_H */
