// Internal launch interfaces shared by the library's translation units (not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace ozg {

// ---------------------------------------------------------------------------------- split
// Rows of op(X): element (i, l) at X[i + l*ld] when `strided`, at X[l + i*ld] otherwise
// (complex: interleaved pairs, same indexing in complex elements; `conj` negates Im).
// Kernel launches issued by this library in this process (graph replays add the kernels they
// replay); every launch site calls note_launch() right after its launch.
long long& launch_counter();
inline void note_launch() { __atomic_fetch_add(&launch_counter(), 1LL, __ATOMIC_RELAXED); }

struct SplitArgs {
  const double* X = nullptr;
  int64_t ld = 0;
  int64_t rows = 0;   // rows of op(X) (complex rows for cplx)
  int64_t k = 0;
  int strided = 0;
  int conj = 0;
  int cplx = 0;
  int s = 0;
  int64_t Kp = 0;                 // row pitch of the digit planes (elements), multiple of 8, >= k
  int64_t plane_rows = 0;         // rows per digit plane (rows, or 2*rows for complex)
  __half* D = nullptr;            // digit planes [s][plane_rows][Kp], fp16 holding integers |d| <= 127
  unsigned long long* maxbits = nullptr;  // [rows] scratch, zeroed by the launcher
  int32_t* exps = nullptr;        // [rows] output exponents
  int* nonfinite = nullptr;       // set to 1 if any entry is Inf/NaN
  unsigned long long* hist = nullptr;  // selector features: 10 gap-histogram counters (nullable)
  // digit planes t_lo .. t_hi are written, t_lo = (plane_from ? *plane_from + 1 : 1),
  // t_hi = (plane_to ? *plane_to : s); a job whose *gate is non-zero writes nothing
  const int* plane_from = nullptr;
  const int* plane_to = nullptr;
  const int* gate = nullptr;
};
cudaError_t launch_split(const SplitArgs& a, cudaStream_t st);
// the two passes of launch_split (row maxima; digits over the plane range of a)
cudaError_t launch_rowmax(const SplitArgs& a, cudaStream_t st);
cudaError_t launch_digits(const SplitArgs& a, cudaStream_t st);

// int8 copy of fp16 digit planes (inspection path): out[p][r][l] = D[p][r][l], l < k
cudaError_t launch_digits_to_i8(const __half* D, int64_t planes, int64_t plane_rows, int64_t k, int64_t Kp,
                                int8_t* out, cudaStream_t st);

// ---------------------------------------------------------------------------------- slice GEMM
struct GemmArgs {
  int64_t rows = 0, cols = 0;   // stacked output rows / cols of the real product (complex: 2m, 2n)
  int64_t m = 0, n = 0;         // output matrix dims (complex: m, n)
  int64_t k = 0;
  int s = 0;
  int cplx = 0;
  const int32_t* e = nullptr;   // [m] row exponents
  const int32_t* f = nullptr;   // [n] column exponents
  double* C = nullptr;
  int64_t ldc = 0;
  double alpha[2] = {1, 0}, beta[2] = {0, 0};
  int beta_zero = 1;
  double* Rws = nullptr;        // Horner partial sums, 16 bytes per output, [grid][BN][BM] per CTA
  int64_t* Gdbg = nullptr;      // inspection: int64 [s][rows][cols] group products (no epilogue)
  int* status = nullptr;        // device status word (0 ok, 3 timeout)
  const int* nonfinite = nullptr;  // if non-null and set, the kernel exits (native path takes over)
  int grid = 0;                 // CTAs to launch (<= tiles); Rws must hold grid tiles
  int variant = 0;              // bit 0: 128-wide tiles; bit 1: deferred pushes (256-wide) or
                                // one 64-wide k sub-tile per stage, 6 stages (128-wide)
  int defer = 0;                // 1: spread intermediate epilogue pushes over the next drains
  const int* s_dev = nullptr;   // if set, the slice count is read here (device-chosen); s = plane count
  int exact = 0;                // 1: exact 128-bit Horner sum and one rounding (s <= 13)
};

// Grouped (batched) GEMM: one persistent launch over the tiles of many independent problems.
struct GroupCall {
  CUtensorMap tmA, tmB;         // digit planes of this call (64-byte aligned inside the struct)
  CUtensorMap tmBh;             // B planes with half-height boxes (the CTA-pair variant)
  int64_t rows = 0, cols = 0, m = 0, n = 0, k = 0;
  int s = 0, cplx = 0, beta_zero = 1, pad = 0;
  const int32_t* e = nullptr;
  const int32_t* f = nullptr;
  double* C = nullptr;
  int64_t ldc = 0;
  double alpha[2] = {1, 0}, beta[2] = {0, 0};
  const int* nonfinite = nullptr;  // this call's Inf/NaN flag (its tiles are skipped when set)
};
struct GroupTile {
  int call;  // < 0: empty slot
  int tm, tn, pad;
};
struct GroupArgs {
  const GroupTile* tiles = nullptr;  // in decreasing cost; CTA b starts with tile b, then claims
  int ntiles = 0;                    // grid + atomicAdd(tile_counter, 1) until the list ends
  int* tile_counter = nullptr;       // zero before the launch
  const int* run = nullptr;          // if non-null and *run == 0 the launch returns at once
  const GroupCall* calls = nullptr;
  int* status = nullptr;
  double* Rws = nullptr;
  int defer = 0;  // as GemmArgs::defer
};
// Tile variant 4: grouped launches on CTA pairs (2-CTA clusters, tcgen05.mma.cta_group::2 over
// 256 x 128 pair tiles; GroupTile::tm counts 256-row tiles).  Single calls take variant 1 instead.
constexpr int kPairVariant = 4;
// Tile variant 5: 128 x 128 tiles over which the groups are taken two at a time (one N = 256 MMA
// for both), up to stacked_max_slices() slices; other calls of that variant run as variant 1.
constexpr int kStackedVariant = 5;
int stacked_max_slices();
cudaError_t launch_slice_gemm_grouped(const GroupArgs& g, int variant, int grid, cudaStream_t st);
int slice_gemm_tile_m_of(int variant);
int pair_max_ctas();  // resident CTAs of the pair variant (0 if the query fails)
// deferred epilogue pushes apply to 256-wide tiles only (128-wide tiles keep R in TMEM)
inline int variant_defers(int variant) { return (variant & 3) == 2 ? 1 : 0; }
// set the kernels' dynamic shared-memory limits (once per process, before any stream capture)
cudaError_t prepare_kernels();
int slice_gemm_tile_n_of(int variant);
// Tensor maps over the digit planes: dims {k, rows, s}, box {64, 128 | 256, 1}, fp16, SW128.
cudaError_t make_digit_tmap(CUtensorMap* map, const __half* D, int64_t k, int64_t rows, int64_t Kp, int s,
                            int box_rows);
cudaError_t launch_slice_gemm(const CUtensorMap& tmA, const CUtensorMap& tmB, const GemmArgs& a, cudaStream_t st);
int slice_gemm_tile_m();
int slice_gemm_tile_n();
size_t slice_gemm_smem_bytes();

// ---------------------------------------------------------------------------------- native FP64
struct NativeArgs {
  char ta = 'N', tb = 'N';
  int64_t m = 0, n = 0, k = 0;
  const double* A = nullptr;
  int64_t lda = 0;
  const double* B = nullptr;
  int64_t ldb = 0;
  double* C = nullptr;
  int64_t ldc = 0;
  double alpha[2] = {1, 0}, beta[2] = {0, 0};
  int beta_zero = 1;
  int cplx = 0;
  const int* gate = nullptr;  // if non-null, the kernel only runs when *gate != 0
};
cudaError_t launch_native_gemm(const NativeArgs& a, cudaStream_t st);

// ---------------------------------------------------------------------------------- sampled check
struct CheckArgs {
  char ta = 'N', tb = 'N';
  int64_t m = 0, n = 0, k = 0;
  const double* A = nullptr;
  int64_t lda = 0;
  const double* B = nullptr;
  int64_t ldb = 0;
  const double* C = nullptr;
  int64_t ldc = 0;
  double alpha[2] = {1, 0}, beta[2] = {0, 0};
  int beta_zero = 1;
  int cplx = 0;
  int nsamp = 0;
  uint64_t seed = 0;
  double* cold = nullptr;     // [nsamp][2] C_old at the samples (beta != 0)
  double* err_out = nullptr;  // max error (device double), reset by launch_check_post
  const int* gate = nullptr;  // skip when *gate != 0 (call routed to native FP64)
  double* part_err = nullptr;  // complex: [2] max relative error of the real / imaginary parts
  // real calls: the split's exponents of the rows of op(A) and the columns of op(B)
  // (|a_il| < 2^ea[i], |b_lj| < 2^fb[j]); when both are set the reference is summed exactly
  // in integers instead of by Dot2
  const int32_t* ea = nullptr;
  const int32_t* fb = nullptr;
};
cudaError_t launch_check_pre(const CheckArgs& a, cudaStream_t st);
cudaError_t launch_check_post(const CheckArgs& a, cudaStream_t st);
// batched: ncalls x nsamp samples; CheckArgs::err_out of call c must point at errs_dev[c]
cudaError_t launch_check_batched_pre(const CheckArgs* calls_dev, int ncalls, int nsamp, cudaStream_t st);
cudaError_t launch_check_batched_post(const CheckArgs* calls_dev, int ncalls, int nsamp, double* errs_dev,
                                      cudaStream_t st);

// ---------------------------------------------------------------------------------- batched
// prefix arrays: njobs + 1 entries, prefix[0] = 0, prefix[njobs] = units
// Batched split: one launch per pass over every job of a batch.  Work units come from device
// tables of (job, unit within the job): row-max units are 32 rows x kRmStridedK k of a strided
// job or 8 rows x kRmContigK k of a contiguous one; digit (and feature) units are 32 rows x
// kDgK k, processed as 64-wide sub-tiles.
constexpr int kRmStridedK = 128, kRmContigK = 1024, kDgK = 64;
// Fused statistics units hold whole rows of real jobs with k <= kStatsK: 16 rows of a strided job,
// 8 rows of a contiguous one.  Longer (or complex) jobs take the two-pass row-maximum units.
constexpr int64_t kStatsK = 2048;
// Short rows: one unit takes several consecutive row blocks (about kStatsBlockElems elements per
// row of the unit), so a CTA's fixed costs (job lookup, reductions, histogram flush) are shared.
constexpr int64_t kStatsBlockElems = 1024;
__host__ __device__ inline int64_t stats_blocks_per_unit(int64_t k) {
  return k >= kStatsBlockElems ? 1 : kStatsBlockElems / (k > 0 ? k : 1);
}
inline bool stats_fused(const SplitArgs& x) { return !x.cplx && x.k >= 1 && x.k <= kStatsK; }
inline int64_t stats_units_of(const SplitArgs& x) {
  const int64_t blocks = x.strided ? (x.rows + 15) / 16 : (x.rows + 7) / 8;
  const int64_t g = stats_blocks_per_unit(x.k);
  return (blocks + g - 1) / g;
}
inline int64_t rowmax_units_of(const SplitArgs& x) {
  return x.strided ? ((x.rows + 31) / 32) * ((x.k + kRmStridedK - 1) / kRmStridedK)
                   : ((x.rows + 7) / 8) * ((x.k + kRmContigK - 1) / kRmContigK);
}
inline int64_t digit_units_of(const SplitArgs& x) { return ((x.rows + 31) / 32) * ((x.k + kDgK - 1) / kDgK); }
// the two passes separately (row maxima; digits) for batches whose slice counts are chosen
// between them
cudaError_t launch_rowmax_batched(const SplitArgs* jobs_dev, const int2* units_dev, int64_t units, cudaStream_t st);
// fused statistics over stats units (job, row block): row maxima written directly (no merge) and,
// with hist != 0, the gap histograms of the jobs that have one, in the same read
cudaError_t launch_stats_batched(const SplitArgs* jobs_dev, const int2* units_dev, int64_t units, int hist,
                                 cudaStream_t st);
// the same for the two operands of one call (both must satisfy stats_fused); hist when either
// operand's hist is set
cudaError_t launch_stats_pair(const SplitArgs& a, const SplitArgs& b, cudaStream_t st);
// run: if non-null and *run == 0 the launch does nothing; grid_cap > 0 bounds the grid (grid-stride)
cudaError_t launch_digits_batched(const SplitArgs* jobs_dev, const int2* units_dev, int64_t units, const int* run,
                                  int grid_cap, cudaStream_t st);
// Gated digit pass of an escalation stage: the jobs whose gate is open (unit_start: njobs + 1
// entries, job j's units at [unit_start[j], unit_start[j+1]) of the job-major unit table) are
// listed on the device (list, prefix, total: njobs, njobs + 1 and 2 entries of scratch), then only
// their units are processed; nothing when *run == 0.
cudaError_t launch_digits_gated(const SplitArgs* jobs_dev, int njobs, const int64_t* unit_start_dev, const int* run,
                                int* list_dev, int64_t* prefix_dev, int64_t* total_dev, int grid, cudaStream_t st);
// Grouped automatic calls, check-driven escalation: after the check of a stage, a call is re-run
// in the next stage (*skip_next = 0, else 1) when it is automatic, finite, ran in this stage
// (ran == nullptr or *ran == 0), its sampled error is above the target and its count *s_cur is
// below the fallback s_fb; the next count, min(*s_cur + s_add, s_fb) (s_fb when s_add == 0), is
// written to *s_next and *s_copy.  Save / restore C of automatic calls with beta != 0 (restore
// only for the calls being re-run).
struct RepairJob {
  int auto_mode = 0, beta_nz = 0;
  const double* err = nullptr;
  const int* ran = nullptr;
  const int* s_cur = nullptr;
  int* s_next = nullptr;
  int* s_copy = nullptr;
  int s_add = 0, s_fb = 0;
  int* skip_next = nullptr;
  const int* nonfinite = nullptr;
  double* C = nullptr;
  double* saved = nullptr;
  int64_t m = 0, n = 0, ldc = 0;
};
// sets *any_rerun (zeroed by the caller) when some call is re-run
cudaError_t launch_repair_prep_batched(const RepairJob* jobs_dev, int njobs, double target, int* any_rerun,
                                       cudaStream_t st);
cudaError_t launch_save_restore_batched(const RepairJob* jobs_dev, const int64_t* prefix_dev, int64_t units,
                                        int njobs, int restore, cudaStream_t st);
// native FP64 for the real calls whose *flags_dev[c] != 0 (list, prefix, total: device scratch
// of ncalls, ncalls + 1 and 2 entries)
cudaError_t launch_native_batched(const NativeArgs* calls_dev, int ncalls, const int* const* flags_dev, int* list_dev,
                                  int64_t* prefix_dev, int64_t* total_dev, int grid, cudaStream_t st);

// C = beta * C (beta == 0: zero fill), m x n, complex if cplx
cudaError_t launch_scale_c(double* C, int64_t m, int64_t n, int64_t ldc, const double* beta, int cplx,
                           cudaStream_t st);

// ---------------------------------------------------------------------------------- selector
constexpr int kSelIn = 24, kSelH = 64, kSelOut = 11;
constexpr int kSelParams = kSelH * kSelIn + kSelH + kSelH * kSelH + kSelH + kSelOut * kSelH + kSelOut;
struct SelectorDev {
  float mean[kSelIn], inv_std[kSelIn];
  uint16_t W1[kSelH * kSelIn];  // BF16 bit patterns, row-major [out][in]
  float b1[kSelH];
  uint16_t W2[kSelH * kSelH];
  float b2[kSelH];
  uint16_t W3[kSelOut * kSelH];
  float b3[kSelOut];
  float threshold;
  int s_lo, fallback, pad;
};
struct SelectJob {
  const unsigned long long* histA = nullptr;
  const unsigned long long* histB = nullptr;
  int64_t m = 0, n = 0, k = 0;
  int* s_out1 = nullptr;  // e.g. the grouped call's slice count
  int* s_out2 = nullptr;  // e.g. the report slot
  int s_cap = 0, active = 0;
};
cudaError_t launch_gap_hist_pair(const SplitArgs& a, const SplitArgs& b, cudaStream_t st);
// the features of every job with a histogram, over the row-maximum unit table
cudaError_t launch_gap_hist_batched(const SplitArgs* jobs_dev, const int2* rowmax_units_dev, int64_t units,
                                    cudaStream_t st);
// M may be null: then only feat_out is written
cudaError_t launch_select_single(const SelectorDev* M, const unsigned long long* hA, const unsigned long long* hB,
                                 int64_t m, int64_t n, int64_t k, float log10_target, int s_cap, int* s_out,
                                 float* feat_out, float* prob_out, cudaStream_t st);
cudaError_t launch_select_batched(const SelectorDev* M, const SelectJob* jobs_dev, int njobs, float log10_target,
                                  cudaStream_t st);
int read_selector_file(const char* path, SelectorDev* out);
// after the check of an automatic call: not_repaired = (err <= target); when not, restore C from
// `saved` (m x n, ld m, w doubles per element) if restore != 0
cudaError_t launch_repair_prep(const double* err, double target, int* not_repaired, const double* saved, double* C,
                               int64_t m, int64_t n, int64_t ldc, int w, int restore, cudaStream_t st);
// training: theta = [W1, b1, W2, b2, W3, b3] FP32 master weights (kSelParams floats)
cudaError_t launch_mlp_grads(const float* theta, const float* X, const int* y, int B, float* grad, float* loss,
                             cudaStream_t st);
cudaError_t launch_adam(float* theta, const float* grad, float* m1, float* m2, int step, float lr, float b1, float b2,
                        float eps, float scale, cudaStream_t st);

}  // namespace ozg
