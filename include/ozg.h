/*
 * ozg.h -- C ABI of the GB300 (sm_103a) library for FP64 / complex128 GEMM emulated with
 * INT8-range integer slices on the tensor cores, with a tunable slice count.
 *
 * Method: the Ozaki scheme on an integer matrix-multiply unit (Sec. 2.2 of "A Pilot Study on
 * Tunable Precision Emulation via Automatic BLAS Offloading", PEARC'25); the slice count is
 * the paper's split number, its compute modes "dgemm" (native FP64) and fp64_int8_3 ..
 * fp64_int8_18 (Sec. 3.1) map to slices = -1 and slices = 3..18.
 *
 *   - Row i of op(A) is scaled by 2^-e_i and column j of op(B) by 2^-f_j (e_i, f_j: frexp
 *     exponents of the row / column maximum), then split by truncation into s signed 7-bit
 *     digits (|d| <= 127, an INT8 value) per entry.
 *   - The s(s+1)/2 slice pairs (p, q), p + q <= s + 1, are multiplied exactly as integers and
 *     summed per group g = p + q.
 *   - The epilogue forms T_ij = 2^{e_i + f_j - 7(s+1)} sum_g G_g,ij 2^{7(s+1-g)} in FP64 and
 *     writes C = alpha * T + beta * C.
 *   - ZGEMM: real and imaginary parts share one exponent per row / column; the four real
 *     sub-products come from one product of the stacked operands and are combined exactly
 *     (Re = P_rr - P_ii, Im = P_ri + P_ir) before the FP64 epilogue.
 *
 * Conventions (BLAS ?gemm): column-major storage; op(A) is m x k, op(B) is k x n;
 * trans in {'N','n','T','t'} for DGEMM, plus {'C','c'} for ZGEMM.  Complex matrices are
 * interleaved complex128 (re, im pairs); leading dimensions count complex elements.
 *
 * Memory and ownership: every matrix pointer is a DEVICE pointer (or managed memory) owned by
 * the caller and never freed by the library.  The context owns its device workspace, which it
 * grows on demand with cudaMalloc (only between calls, after synchronising its stream).
 * Calls are asynchronous on the context's stream unless stated otherwise.
 *
 * Return codes: 0 on success; -i when argument i is invalid, numbered as in BLAS
 * (transa = 1, transb = 2, m = 3, n = 4, k = 5, lda = 8, ldb = 10, ldc = 13, slices = 14);
 * positive values are runtime errors (OZG_ERR_*).  A call that returns an error leaves C
 * unspecified only for runtime errors; argument errors return before any work is queued.
 */
#ifndef OZG_H
#define OZG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OZG_OK 0
#define OZG_ERR_CUDA 1         /* a CUDA runtime call failed (see ozg_last_cuda_error) */
#define OZG_ERR_ALLOC 2        /* device workspace allocation failed */
#define OZG_ERR_TIMEOUT 3      /* a bounded device-side wait gave up; the kernel returned */
#define OZG_ERR_UNSUPPORTED 4  /* the request is valid BLAS but outside what this library implements */
#define OZG_ERR_INVALID 5      /* null context or other non-BLAS argument error */

#define OZG_MAX_SLICES 18      /* fp64_int8_18 is the largest mode of Sec. 3.1 */
#define OZG_NATIVE (-1)        /* slices = -1: native FP64 ("dgemm" mode of Sec. 3.1) */

typedef struct ozg_ctx ozg_ctx;

/* Per-call report.  When a report is requested the call synchronises its stream before
 * returning, so every field is final on return. */
typedef struct ozg_report {
  int slices_used;        /* s actually used; -1 when the call ran in native FP64 */
  int nonfinite;          /* 1 if an input held Inf/NaN and the call was routed to native FP64 */
  int status;             /* OZG_OK or a positive error code for this call */
  int samples;            /* entries checked in double-double (0: check disabled) */
  double est_err;         /* max over the samples of |C - C_dd| / (|alpha||A||B| + |beta||C_old|);
                             NaN when not checked or routed to native FP64 */
  int selected;           /* slice count the learned selector chose (0: the count was fixed) */
  int repaired;           /* re-runs the check forced on a learned call: 0 none; in a grouped call
                             1 = re-run at min(selected + 2, fallback), 2 = re-run again at the
                             fallback count; in a single call 1 = re-run at the fallback count
                             (slices_used holds the count of the last run) */
  double max_real;        /* complex calls: max over the samples of |Re C - Re C_dd| / |Re C_dd| and */
  double max_imag;        /* the same for Im: the per-part relative error of the paper's MuST study
                             (Sec. 3.2); NaN for real calls or when not checked */
} ozg_report;

/* Create a context on the current CUDA device.  workspace_bytes pre-reserves device
 * workspace (0: grow on first use).  *out receives the context.  Returns 0 or OZG_ERR_*. */
int ozg_create(ozg_ctx** out, size_t workspace_bytes);

/* Destroy a context: synchronises its stream, frees its workspace.  NULL is accepted. */
int ozg_destroy(ozg_ctx* ctx);

/* Set the CUDA stream (a cudaStream_t passed as void*) on which the context queues work;
 * NULL selects the legacy default stream.  The caller keeps ownership of the stream. */
int ozg_set_stream(ozg_ctx* ctx, void* stream);

/* Block until all work queued by this context has finished; returns the first device-side
 * status raised since the previous ozg_sync (OZG_ERR_TIMEOUT if a bounded wait expired). */
int ozg_sync(ozg_ctx* ctx);

/* Sampled error check (the per-result error report): samples > 0 makes every later emulated
 * call recompute `samples` output entries (the four corners plus hashed positions) in
 * double-double on the GPU after the GEMM and report the largest componentwise error relative
 * to |alpha||A||B| + |beta||C_old| in ozg_report.est_err.  0 disables (the default). */
int ozg_set_check_samples(ozg_ctx* ctx, int samples);

/* ---- learned slice selector (slices = 0: automatic) ----
 * The paper proposes adjusting the split number to the accuracy each computation needs
 * (Sec. 4).  With a model loaded, a call with slices = 0 computes per-GEMM features on the GPU
 * (log2 m, n, k; 10-bin histograms of the within-row / within-column exponent gaps of op(A) and
 * op(B); log10 of the target error), evaluates a 24-64-64-11 MLP (BF16 weights, FP32
 * accumulation) on the GPU and uses the smallest s in 2..12 whose cumulative predicted
 * probability reaches the model's threshold -- all on the device, no host round trip.  The
 * sampled double-double check is always on for such calls (>= 64 samples); if its estimate
 * exceeds the target the call is recomputed, again on the device: a call of a grouped launch at
 * min(s + 2, fallback) and, if the check rejects that too, at the fallback count
 * (ozg_set_fallback_slices; a count at or above the fallback is not recomputed); a single call
 * at the fallback count.  Without a model, slices = 0 means the fallback count. */

/* Load a selector model file (format in the library's selector source); also sets the
 * context's fallback count to the model's conservative count.  Returns 0 or OZG_ERR_INVALID
 * (unreadable or malformed file). */
int ozg_load_selector(ozg_ctx* ctx, const char* path);

/* Target componentwise error for automatic slice counts (default 1e-12). */
int ozg_set_target_error(ozg_ctx* ctx, double target);

/* Selector features of one GEMM, computed by the same kernels as the automatic path:
 * feat_out (device float[24]); prob_out (device float[11] or NULL) and s_out (device int or
 * NULL) receive the loaded model's class probabilities and decision (left untouched without a
 * model).  Synchronous. */
int ozg_selector_features(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k,
                          const double* A, int64_t lda, const double* B, int64_t ldb, float* feat_out,
                          float* prob_out, int* s_out);

/* On-GPU training of the selector's MLP (FP32 master parameters; BF16-rounded weights in the
 * forward pass, straight-through gradients; mean cross-entropy).  Parameters are the HOST array
 * theta[OZG_SELECTOR_PARAMS] = W1[64x24], b1[64], W2[64x64], b2[64], W3[11x64], b3[11]
 * (row-major [out][in]).  X: DEVICE float[B][24] normalised features, y: DEVICE int[B] class
 * indices 0..10.  Each call is synchronous. */
#define OZG_SELECTOR_PARAMS 6475
int ozg_selector_set_params(ozg_ctx* ctx, const float* theta);     /* also resets Adam state */
int ozg_selector_get_params(ozg_ctx* ctx, float* theta);
int ozg_selector_grads(ozg_ctx* ctx, const float* X, const int* y, int B, float* grad, float* loss);
int ozg_selector_train_step(ozg_ctx* ctx, const float* X, const int* y, int B, float lr, float* loss);

/* enable != 0: correctly rounded mode for single calls with s <= 13.  The group products are
 * summed exactly as 128-bit integers and each result is rounded to FP64 once: RN of the exact
 * value, subnormal and overflowing results included.  The default epilogue is exact in the same
 * way while its sum fits two int64 windows (s <= 10 at any k, s <= 12 for k <= 512) and continues
 * in FP64 beyond that (one rounding per further window); this mode stays exact up to s = 13 at
 * any k, moves 16 bytes of scratch per output and is slower.  Grouped calls always use the
 * default epilogue. */
int ozg_set_exact_epilogue(ozg_ctx* ctx, int enable);

/* Human-readable text for a return code (static storage). */
const char* ozg_strerror(int code);

/* Emulated DGEMM, C = alpha op(A) op(B) + beta C (Sec. 2.2 / 3.1; ?gemm semantics).
 *   transa, transb: 'N' or 'T' (case-insensitive).  m, n, k >= 0.
 *   A: device, column-major, lda >= max(1, rows of A); B likewise with ldb; C: m x n, ldc >= max(1, m).
 *   slices: 1..OZG_MAX_SLICES fixed split number; OZG_NATIVE (-1) runs native FP64; 0 lets the
 *   learned selector choose (see below; the fallback count when no model is loaded).
 *   beta == 0: C is not read (NaNs in C are ignored).  Quick returns: m == 0 or n == 0, or
 *   ((alpha == 0 or k == 0) and beta == 1).  alpha == 0 or k == 0 gives C = beta C.
 *   Inputs holding Inf/NaN are detected on the device and the call is completed by the native
 *   FP64 kernel (still on the GPU); rep->nonfinite reports it.
 *   rep may be NULL (asynchronous call); with a report the call returns after its work finished. */
int ozg_dgemm(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
              const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
              int64_t ldc, int slices, ozg_report* rep);

/* Emulated ZGEMM (complex128, interleaved), C = alpha op(A) op(B) + beta C; trans in N/T/C.
 * alpha and beta point to HOST arrays {re, im}.  Other arguments as for ozg_dgemm. */
int ozg_zgemm(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k,
              const double* alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
              const double* beta, double* C, int64_t ldc, int slices, ozg_report* rep);

/* Native FP64 GEMM on the CUDA cores (the "dgemm" mode of Sec. 3.1, and the comparison
 * kernel of Sec. 4's performance discussion).  Same arguments as ozg_dgemm minus slices. */
int ozg_native_dgemm(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k,
                     double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                     double beta, double* C, int64_t ldc);

/* Native complex128 GEMM (same conventions as ozg_zgemm). */
int ozg_native_zgemm(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k,
                     const double* alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                     const double* beta, double* C, int64_t ldc);

/* ---- grouped (batched) emulated DGEMM ----
 * Many independent, uneven GEMMs with per-call slice counts in one short launch sequence: a
 * batched split of every operand, ONE persistent tensor-core launch over the tiles of all calls
 * (longest-first load balancing across the SMs), a batched native FP64 fallback for calls whose
 * inputs held Inf/NaN, and a batched sampled error check.  On a non-default context stream the
 * sequence is captured into a CUDA graph and replayed for as long as the same batch (same
 * descriptors and slice counts) is submitted again; the matrices' contents may change between
 * submissions.  Grouping many small GEMMs is an addition of this library; the
 * paper has no grouped interface (its offload intercepts one BLAS call at a time, Sec. 3.1). */
typedef struct ozg_gemm_desc {
  char transa, transb; /* 'N' or 'T' (case-insensitive; 'C' means 'T') */
  char reserved[6];    /* set to zero */
  int64_t m, n, k;
  double alpha, beta;
  const double* A; /* device, column-major */
  int64_t lda;
  const double* B;
  int64_t ldb;
  double* C;
  int64_t ldc;
} ozg_gemm_desc;

/* descs: HOST array of count descriptors; slices: HOST array (NULL: all 0), per call 1..18, or
 * 0: the learned selector's choice when a selector is loaded (ozg_load_selector), else the
 * context's fallback count (ozg_set_fallback_slices, default 7).  reps: NULL or a HOST
 * array of count reports (status holds -i for an invalid argument i of that call); with reports
 * the call returns after the batch finished.  Returns OZG_ERR_INVALID if any descriptor is
 * invalid (nothing is queued), else 0 or a runtime error. */
int ozg_dgemm_grouped(ozg_ctx* ctx, int64_t count, const ozg_gemm_desc* descs, const int* slices,
                      ozg_report* reps);

/* The grouped emulated DGEMM on matrices in HOST memory: the descriptors' A, B and C are host
 * (CPU) pointers, everything else is as for ozg_dgemm_grouped (slices, reports, the selector, the
 * check and its escalation).  Synchronous: on return C holds the results and the reports are
 * final.  The library stages the matrices in device memory it owns (grown with cudaMalloc) and
 * cuts the batch into parts (ozg_set_host_parts, default 16) whose shares of the work rise and
 * fall (1, 2, 3, .., 3, 2, 1: small first and last parts, whose copies cannot overlap): a part's inputs
 * are copied in while earlier parts compute and their results are copied out, each part on its
 * own internal stream and CUDA graph.  Matrices whose host regions touch or overlap move as one
 * copy; C is written back only where the calls write it (rows 0..m-1 of each column; C is read
 * only when beta != 0).  Page-locked (pinned) host memory lets the copies run at full rate and
 * overlap the computation; pageable memory works too.  Returns OZG_ERR_INVALID if any
 * descriptor is invalid (nothing is copied), else 0 or a runtime error. */
int ozg_dgemm_grouped_host(ozg_ctx* ctx, int64_t count, const ozg_gemm_desc* descs, const int* slices,
                           ozg_report* reps);

/* Parts of the pipeline of ozg_dgemm_grouped_host (1..64; -2 for other values). */
int ozg_set_host_parts(ozg_ctx* ctx, int parts);

/* 3M (Karatsuba) ZGEMM: the same contract as ozg_zgemm, computed from three real emulated
 * products instead of four real sub-products.  With Ar, Ai the real and imaginary parts of op(A)
 * (conjugated for 'C'), Sa = RN(Ar + Ai) and the same for op(B):
 *   P1 = emu(Ar, Br), P2 = emu(Ai, Bi), P3 = emu(Sa, Sb)   (one grouped launch, s slices each)
 *   Re = RN(P1 - P2), Im = RN(RN(P3 - P1) - P2), then alpha and beta as ozg_zgemm.
 * It does 3/4 of the slice-product work, with the 3M form's weaker error bound: the error of Im
 * scales with (|Ar| + |Ai|)(|Br| + |Bi|) instead of |Ar||Bi| + |Ai||Br|, and Sa, Sb add one
 * rounding each.  slices: 1..18 or -1 (native FP64, as ozg_zgemm); the learned selector is not
 * used here (0 is invalid, argument 14).  The report's est_err / max_real / max_imag come from
 * the context's sampled check of the complex result.  Workspace: 3 (mk + kn + mn) doubles.
 * Non-finite inputs reach the native kernel per real product. */
int ozg_zgemm3m(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k, const double* alpha,
                const double* A, int64_t lda, const double* B, int64_t ldb, const double* beta, double* C,
                int64_t ldc, int slices, ozg_report* rep);

/* Region-adaptive slice counts (the paper's proposed adjustment of the split number to the
 * accuracy a region needs, Sec. 4): C = alpha op(A) op(B) + beta C computed as row_blocks x
 * col_blocks regions of C.  The rows of C are cut into row_blocks bands and its columns into
 * col_blocks bands, as equal as possible.  Each region is one call of a grouped launch over the
 * full k with slice count 0, so with a selector loaded every region gets the count that its own
 * rows of op(A) and columns of op(B) need.  Each region is then exactly the emulated product
 * at that count (the digits of a row depend only on that row, so they are the same as in the
 * whole-matrix call).  Arguments as ozg_dgemm (device pointers, BLAS numbering; row_blocks = 14,
 * col_blocks = 15, each >= 1).  reps: NULL or a HOST array of row_blocks x col_blocks reports,
 * band-row-major (region (i, j) at i * col_blocks + j).  Each of the operands' rows is split
 * once per region that uses it. */
int ozg_dgemm_regions(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                      const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                      int64_t ldc, int row_blocks, int col_blocks, ozg_report* reps);

/* enable != 0 (default): capture grouped calls into CUDA graphs when the context stream is not
 * the legacy default stream.  Changing it drops the cached graph. */
int ozg_set_graphs(ozg_ctx* ctx, int enable);

/* Slice count used for calls that request 0 (default 7). */
int ozg_set_fallback_slices(ozg_ctx* ctx, int slices);

/* Tile variants of the slice-product kernel.  Variants 0..3: bit 0 picks the output tile (0:
 * 128 x 256, 1: 128 x 128).  Bit 1: for 128 x 256 tiles, spread each intermediate epilogue
 * accumulation over the next chains' drains instead of running it at once (pays for long k,
 * costs for short k); for 128 x 128 tiles, stage one 64-wide k slice per pipeline stage in 6
 * stages instead of two in 3 (deeper prefetch, more issue overhead).  Variant 4: grouped calls
 * run on CTA pairs (2-CTA clusters sharing one tcgen05 MMA of 256 x 128 tiles; each CTA stages
 * its own 128 rows of A and half of B); single calls run it as variant 1.  Variant 5: 128 x 128
 * tiles over which the slice groups are taken two at a time (groups g and g + 1 share their
 * digit planes: one pass loads A_1..A_g and B_1..B_g once and issues one N = 256 MMA per plane
 * pair), up to 16 slices; a call with more slices, the exact epilogue or the group-product
 * export runs as variant 1.  All variants give bit-identical C while the exact sum needs at most
 * two int64 windows (s <= 10 at any k); beyond that the FP64 continuation may round differently
 * in the last bits between the 256- and 128-wide families. */
#define OZG_NUM_TILE_VARIANTS 6

/* Tile-variant autotuner: enable != 0 times the variants the first time a shape bucket
 * (rounded log2 of m, n, k and the slice count; variants 0..3 and 5) or a grouped batch (every
 * variant) is seen, keeps the fastest,
 * and appends single-call choices to cache_path (may be NULL) as "bucket variant" lines that
 * later contexts read back.  Tuning runs only for calls with beta == 0 (C is then write-only);
 * other calls use the heuristic: the stacked group pairs (variant 5) for single calls with at
 * most 16 slices outside the exact epilogue; otherwise the width that pads least, then for
 * 128 x 256 tiles deferral when k >= 2048 (for a grouped batch, the mean k weighted by m n s^2)
 * and for 128 x 128 tiles variant 5 in grouped calls whose slice counts allow it, else two k
 * slices per stage (variant 1). */
int ozg_set_autotune(ozg_ctx* ctx, int enable, const char* cache_path);

/* Force tile variant 0..5 for every later call (single and grouped), or -1 (default) for the
 * autotuned / heuristic choice.  Returns OZG_ERR_INVALID for other values, OZG_ERR_UNSUPPORTED
 * for variant 4 when no 2-CTA cluster of the kernel fits on the device. */
int ozg_set_tile_variant(ozg_ctx* ctx, int variant);

/* Tile variant of the context's most recent grouped call (the autotuned, heuristic or forced
 * choice), or -1 when it has made none; written to *variant. */
int ozg_get_tile_variant(ozg_ctx* ctx, int* variant);

/* Kernel launches this library has issued in this process, written to *out (a replay of a
 * captured grouped call counts every kernel it replays).  For launch accounting in benchmarks. */
int ozg_kernel_launches(long long* out);

/* ---- inspection entry points (used by the parity tests; same kernels as the GEMM path) ---- */

/* Split the rows of op(X) (rows x k, real FP64, device) into exponents and digit planes, the
 * first step of Sec. 2.2's scheme.  trans: 'N' (row i of X) or 'T' (column i of X).
 *   e_out: device int32[rows]; digits_out: device int8[s][rows][k] (k contiguous).
 * Synchronous (returns after the copy-out kernel finished). */
int ozg_debug_split(ozg_ctx* ctx, char trans, int64_t rows, int64_t k, const double* X, int64_t ld,
                    int slices, int32_t* e_out, int8_t* digits_out);

/* Complex variant: op(X) rows x k complex128; trans 'N', 'T' or 'C'.  digits_out is
 * int8[s][2*rows][k] with Re of row i at 2i and Im at 2i+1; e_out int32[rows]. */
int ozg_debug_zsplit(ozg_ctx* ctx, char trans, int64_t rows, int64_t k, const double* X, int64_t ld,
                     int slices, int32_t* e_out, int8_t* digits_out);

/* Exact group products G_g = sum_{p+q=g} D^A_p (D^B_q)^T of the emulated DGEMM (the integer
 * slice products of Sec. 2.2), computed by the tensor-core kernel and exported as
 * int64[s][m][n] (row-major, group g = 2..s+1 at index g-2) in device memory G_out.  The kernel
 * folds a group's int32 sum out every 64 accumulation chains of 1024 products (65,536 products);
 * the export adds those partial sums in int64, so it holds the exact G_g at any k.
 * Synchronous. */
int ozg_debug_group_products(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k,
                             const double* A, int64_t lda, const double* B, int64_t ldb, int slices,
                             int64_t* G_out);

/* ---- fault-path hooks (tests; no GPU fault is involved) ----
 * ozg_debug_wait: queues one CTA that waits on an mbarrier nothing arrives at, bounded at
 * `cycles` clock cycles (1000 .. 4e9); when the wait runs out, the kernel raises the
 * context's timeout status and returns.  ozg_sync then reports OZG_ERR_TIMEOUT once, and the
 * context stays usable.
 * ozg_debug_fail_allocs: the next n workspace allocations of this context fail on the host side,
 * as if cudaMalloc had failed.  The call that needs one returns OZG_ERR_ALLOC with C untouched,
 * and later calls allocate again.  Both return 0 or OZG_ERR_INVALID. */
int ozg_debug_wait(ozg_ctx* ctx, long long cycles);
int ozg_debug_fail_allocs(ozg_ctx* ctx, int n);

/* ---- emulated DGEMM without any device allocation ----
 * No counterpart in the paper.  For callers that must not call cudaMalloc: an interposed dgemm_
 * inside a host application that owns all device memory through its own pool or a fixed budget
 * (an allocation behind its back can fail or break its accounting), and latency-critical paths
 * where cudaMalloc / cudaFree would synchronise the device.  Same arithmetic, kernels and results
 * as ozg_dgemm (transa, transb in N/T; slices 1..18 or -1 for native FP64), but no context: the
 * work is queued on `stream` (a cudaStream_t, NULL = legacy default stream) and all scratch lives
 * in one fixed device array of OZG_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that
 * loads the library's device code holds until the process exits.
 *   - The problem must fit the array: 2 s (m + n) round8(k) bytes of digit planes plus
 *     12 (m + n) bytes of row data (each part rounded up to 256 bytes) plus at least one
 *     OZG_NOALLOC_TILE_BYTES tile of partial sums (128 x 256 outputs x 16 bytes); with less room
 *     than one tile per SM the kernel runs on fewer CTAs, each looping over several tiles (e.g.
 *     m = n = k = 1024, s = 8 fits; 2048 does not).  Larger problems return OZG_ERR_UNSUPPORTED
 *     before any work is queued.
 *   - The first call on each device does the set-up: it resolves the array's device address
 *     (cudaGetSymbolAddress, with that device current).  Make that first call before any stream
 *     capture begins.  If the device's context is destroyed and created again (cudaDeviceReset),
 *     the next call does the set-up again.
 *   - Every call reuses the same array; each call clears what must start at zero.  Calls whose
 *     work overlaps on the GPU (other streams, unordered host threads) race on the array.
 *   - Asynchronous; device-side wait time-outs are not reported by this entry point (C is then
 *     unspecified).  Inf/NaN inputs are handled as in ozg_dgemm (native FP64 on the GPU).
 * Returns 0, a BLAS argument error -i, OZG_ERR_UNSUPPORTED (too large) or OZG_ERR_CUDA. */
#define OZG_NOALLOC_SCRATCH_BYTES (64u << 20)
#define OZG_NOALLOC_TILE_BYTES (128u * 256u * 16u)
int ozg_dgemm_noalloc(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                      const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                      int64_t ldc, int slices, void* stream);

/* ---- per-phase device timing (CUDA events on the context's stream) ---- */
#define OZG_PHASE_SPLIT 0    /* exponent + digit extraction of both operands */
#define OZG_PHASE_GEMM 1     /* fused slice-product GEMM + epilogue (also each grouped GEMM launch
                                of a grouped call issued without a graph) */
#define OZG_PHASE_NATIVE 2   /* native FP64 kernel (native mode, or the gated non-finite path) */
#define OZG_PHASE_CHECK 3    /* sampled double-double error check */
#define OZG_PHASE_SELECT 4   /* learned slice selector */
#define OZG_PHASE_GROUPED 5  /* a whole grouped call (graph launch or direct launches) */
#define OZG_NUM_PHASES 8

/* enable != 0: every later call records a CUDA event pair around each of its phases. */
int ozg_set_profiling(ozg_ctx* ctx, int enable);

/* Synchronise the context's stream, then return the device milliseconds accumulated per
 * phase since the previous call (ms[OZG_NUM_PHASES]) and the number of timed launches per
 * phase (counts[OZG_NUM_PHASES]); either pointer may be NULL.  Resets the accumulators. */
int ozg_phase_times(ozg_ctx* ctx, double* ms, int64_t* counts);

/* Message of the last failing CUDA runtime call seen by the library in this process. */
const char* ozg_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OZG_H */
