// Batched companions of the split, native and check kernels for the grouped GEMM: one launch
// covers every call of a batch (a device-side job table plus a prefix sum of work units per job;
// each CTA finds its job by binary search), so a batch of thousands of uneven GEMMs costs a
// handful of launches and captures into a short CUDA graph.
//   * split: the same exponents and digits as the single-call kernels (Sec. 2.2's split), one
//     job per operand;
//   * native: FP64 GEMM (real) for the calls whose inputs held Inf/NaN, on a device-compacted list;
//   * check: the sampled double-double error of every call (one warp per sample).
#include "ozg_internal.h"
#include "ozg_split_dev.cuh"

namespace ozg {
namespace {

// largest j with prefix[j] <= unit (prefix[0] = 0, prefix[njobs] = total)
__device__ __forceinline__ int find_job(const int64_t* prefix, int njobs, int64_t unit) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= unit)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// element (i, l) of the job's op(X) as raw bits; complex gives (re, im) with conjugation applied
__device__ __forceinline__ void load_elem(const SplitArgs& J, int64_t i, int64_t l, uint64_t& re, uint64_t& im) {
  if (!J.cplx) {
    const uint64_t* p = reinterpret_cast<const uint64_t*>(J.X);
    re = __ldg(J.strided ? p + i + l * J.ld : p + l + i * J.ld);
    im = 0;
  } else {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(J.X);
    ulonglong2 v = __ldg(J.strided ? p + i + l * J.ld : p + l + i * J.ld);
    re = v.x;
    im = J.conj ? (v.y ^ 0x8000000000000000ull) : v.y;
  }
}

// Row maxima.  A unit is 32 rows x 128 k of a strided job (lanes = consecutive rows, the eight
// warps interleave along k, 16 loads in flight per thread) or 8 rows x 1024 k of a contiguous
// job (a warp per row, lanes along k).  Partial maxima merge by atomicMax into the zeroed maxbits.
__global__ void __launch_bounds__(256) rowmax_batched(const SplitArgs* jobs, const int2* units) {
  const int2 ur = units[blockIdx.x];
  const SplitArgs J = jobs[ur.x];
  const int64_t u = ur.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long mx = 0;
  if (J.strided) {
    __shared__ unsigned long long red[8][32];
    const int64_t kt = (J.k + kRmStridedK - 1) / kRmStridedK;
    const int64_t row = (u / kt) * 32 + lane, l0 = (u % kt) * kRmStridedK + w;
    if (row < J.rows) {
#pragma unroll
      for (int i = 0; i < kRmStridedK / 8; ++i) {
        const int64_t l = l0 + 8 * i;
        if (l < J.k) {
          uint64_t re, im;
          load_elem(J, row, l, re, im);
          re &= kAbsMask;
          im &= kAbsMask;
          re = re > im ? re : im;
          mx = re > mx ? re : mx;
        }
      }
    }
    red[w][lane] = mx;
    __syncthreads();
    if (w == 0 && row < J.rows) {
#pragma unroll
      for (int i = 1; i < 8; ++i) mx = red[i][lane] > mx ? red[i][lane] : mx;
      if (mx) {
        atomicMax(&J.maxbits[row], mx);
        if (mx >= kInfBits) atomicExch(J.nonfinite, 1);
      }
    }
  } else {
    const int64_t kt = (J.k + kRmContigK - 1) / kRmContigK;
    const int64_t row = (u / kt) * 8 + w, l0 = (u % kt) * kRmContigK + lane;
    if (row >= J.rows) return;
#pragma unroll 8
    for (int i = 0; i < kRmContigK / 32; ++i) {
      const int64_t l = l0 + 32 * i;
      if (l < J.k) {
        uint64_t re, im;
        load_elem(J, row, l, re, im);
        re &= kAbsMask;
        im &= kAbsMask;
        re = re > im ? re : im;
        mx = re > mx ? re : mx;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    if (lane == 0 && mx) {
      atomicMax(&J.maxbits[row], mx);
      if (mx >= kInfBits) atomicExch(J.nonfinite, 1);
    }
  }
}

// Digits (real jobs: the grouped GEMM is real).  A unit is 32 rows x kDgK k, walked as 64-wide
// sub-tiles.  Thread t computes row t/8 and the 8 consecutive k at (t%8)*8 of a sub-tile;
// strided jobs are staged (transposed) through shared memory so that global loads stay
// coalesced.  The loads of the next sub-tile are issued before the current one is processed.
__device__ __forceinline__ void digits_unit(const SplitArgs* jobs, int2 ur) {
  __shared__ uint64_t tile[64][33];
  {
    const int* gate = jobs[ur.x].gate;
    if (gate != nullptr && *gate) return;
  }
  const SplitArgs J = jobs[ur.x];
  const int t_lo = J.plane_from != nullptr ? *J.plane_from + 1 : 1;
  const int t_hi = J.plane_to != nullptr ? *J.plane_to : J.s;
  if (t_lo > t_hi) return;
  const int64_t u = ur.y;
  const int64_t ktiles = (J.k + kDgK - 1) / kDgK;
  const int64_t r0 = (u / ktiles) * 32, lbase = (u % ktiles) * kDgK;
  const int tid = threadIdx.x;
  const int r = tid / 8, lg = (tid % 8) * 8;
  const int64_t row = r0 + r;
  const bool row_ok = row < J.rows;
  const uint64_t* X = reinterpret_cast<const uint64_t*>(J.X);
  const int e = row_ok ? exponent_from_maxbits(J.maxbits[row]) : 0;
  if (row_ok && lbase == 0 && lg == 0 && t_lo == 1) J.exps[row] = e;
  const int64_t plane = J.plane_rows * J.Kp;
  const int rr = tid % 32;
  const bool rrok = r0 + rr < J.rows;
  uint64_t nx[8];
  auto load = [&](int64_t l0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (J.strided) {
        const int64_t l = l0 + tid / 32 + 8 * q;
        nx[q] = (rrok && l < J.k) ? __ldg(X + (r0 + rr) + l * J.ld) : 0ull;
      } else {
        const int64_t l = l0 + lg + q;
        nx[q] = (row_ok && l < J.k) ? __ldg(X + row * J.ld + l) : 0ull;
      }
    }
  };
  load(lbase);
  for (int sub = 0; sub < kDgK / 64; ++sub) {
    const int64_t l0 = lbase + 64 * sub;
    if (l0 >= J.k) break;
    uint64_t b[8];
    if (J.strided) {
      __syncthreads();  // the previous sub-tile's reads of the tile are done
#pragma unroll
      for (int q = 0; q < 8; ++q) tile[tid / 32 + 8 * q][rr] = nx[q];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 8; ++q) b[q] = tile[lg + q][r];
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) b[q] = nx[q];
    }
    if (sub + 1 < kDgK / 64 && l0 + 64 < J.k) load(l0 + 64);
    if (!row_ok || l0 + lg >= J.k) continue;
    DigitSrc ds[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ds[q] = digit_src(b[q], e);
    __half* out = J.D + row * J.Kp + l0 + lg;
    store_digit_planes<kMaxPlanes>(ds, t_lo, t_hi, out, plane);
  }
}

// Grid-stride over the units; a gated pass (re-run completion) first reads one step-wide flag.
__global__ void __launch_bounds__(256) digits_batched(const SplitArgs* jobs, const int2* units, int64_t nunits,
                                                      const int* run) {
  if (run != nullptr && *run == 0) return;  // nothing to do in this pass
  for (int64_t unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
    digits_unit(jobs, units[unit]);
    __syncthreads();  // the next unit reuses the staging tile
  }
}

// ---------------------------------------------------------------------------- native fallback
// Device-side compaction of the calls whose non-finite flag is set, then a persistent FP64
// kernel over their 64 x 64 output tiles.
// One CTA: the flags are scanned in parallel (list order does not matter), then one thread
// forms the tile prefix over the flagged calls only (usually none).
__global__ void __launch_bounds__(1024) native_compact(const NativeArgs* calls, int ncalls, const int* const* flags,
                                                       int* list, int64_t* tile_prefix, int64_t* total) {
  __shared__ int n_sh;
  if (threadIdx.x == 0) n_sh = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < ncalls; c += blockDim.x)
    if (*flags[c] != 0) list[atomicAdd(&n_sh, 1)] = c;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int n = n_sh;
  int64_t acc = 0;
  for (int i = 0; i < n; ++i) {
    const int c = list[i];
    tile_prefix[i] = acc;
    acc += ((calls[c].m + 63) / 64) * ((calls[c].n + 63) / 64);
  }
  tile_prefix[n] = acc;
  total[0] = acc;
  total[1] = n;
}

__global__ void __launch_bounds__(256) native_batched(const NativeArgs* calls, const int* list,
                                                      const int64_t* tile_prefix, const int64_t* total) {
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  const int64_t ntiles = total[0];
  const int ncl = (int)total[1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int64_t w = blockIdx.x; w < ntiles; w += gridDim.x) {
    const int li = find_job(tile_prefix, ncl, w);
    const NativeArgs P = calls[list[li]];
    const int64_t t = w - tile_prefix[li];
    const int64_t tn_count = (P.n + 63) / 64;
    const int64_t m0 = (t / tn_count) * 64, n0 = (t % tn_count) * 64;
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < P.k; k0 += 16) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = threadIdx.x + 256 * q;
        const int rr = idx % 64, kk = idx / 64;
        const int64_t gr = m0 + rr, gk = k0 + kk, gc = n0 + rr;
        double va = 0, vb = 0;
        if (gr < P.m && gk < P.k) va = (P.ta == 'N') ? P.A[gr + gk * P.lda] : P.A[gk + gr * P.lda];
        if (gc < P.n && gk < P.k) vb = (P.tb == 'N') ? P.B[gk + gc * P.ldb] : P.B[gc + gk * P.ldb];
        As[kk][rr] = va;
        Bs[kk][rr] = vb;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jn = 0; jn < 4; ++jn) acc[i][jn] = fma(As[kk][ty + 16 * i], Bs[kk][tx + 16 * jn], acc[i][jn]);
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jn = 0; jn < 4; ++jn) {
        const int64_t r = m0 + ty + 16 * i, c = n0 + tx + 16 * jn;
        if (r >= P.m || c >= P.n) continue;
        double* cp = P.C + r + c * P.ldc;
        *cp = P.beta_zero ? P.alpha[0] * acc[i][jn] : fma(P.alpha[0], acc[i][jn], P.beta[0] * *cp);
      }
  }
}

__global__ void repair_prep_batched(const RepairJob* jobs, int njobs, double target, int* any_rerun) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= njobs) return;
  const RepairJob J = jobs[i];
  const double e = J.err ? *J.err : 0.0;
  const bool bad = J.auto_mode && !(J.nonfinite && *J.nonfinite) && !(e <= target);
  *J.skip2 = bad ? 0 : 1;
  if (bad && any_rerun != nullptr) atomicOr(any_rerun, 1);
}

// unit = 256 elements of one automatic, beta != 0 call
__global__ void save_restore_batched(const RepairJob* jobs, const int64_t* prefix, int njobs, int restore) {
  const int64_t unit = blockIdx.x;
  const int jb = find_job(prefix, njobs, unit);
  const RepairJob J = jobs[jb];
  if (restore && *J.skip2) return;
  const int64_t e = (unit - prefix[jb]) * 256 + threadIdx.x;
  if (e >= J.m * J.n) return;
  const int64_t i = e % J.m, j = e / J.m;
  if (restore)
    J.C[i + j * J.ldc] = J.saved[e];
  else
    J.saved[e] = J.C[i + j * J.ldc];
}

}  // namespace

cudaError_t launch_repair_prep_batched(const RepairJob* jobs_dev, int njobs, double target, int* any_rerun,
                                       cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  { repair_prep_batched<<<(njobs + 127) / 128, 128, 0, st>>>(jobs_dev, njobs, target, any_rerun); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_save_restore_batched(const RepairJob* jobs_dev, const int64_t* prefix_dev, int64_t units,
                                        int njobs, int restore, cudaStream_t st) {
  if (units <= 0 || njobs <= 0) return cudaSuccess;
  { save_restore_batched<<<(unsigned)units, 256, 0, st>>>(jobs_dev, prefix_dev, njobs, restore); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_rowmax_batched(const SplitArgs* jobs_dev, const int2* units_dev, int64_t units, cudaStream_t st) {
  if (units > 0) { rowmax_batched<<<(unsigned)units, 256, 0, st>>>(jobs_dev, units_dev); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_digits_batched(const SplitArgs* jobs_dev, const int2* units_dev, int64_t units, const int* run,
                                  int grid_cap, cudaStream_t st) {
  if (units <= 0) return cudaSuccess;
  const int64_t grid = grid_cap > 0 && units > grid_cap ? grid_cap : units;
  { digits_batched<<<(unsigned)grid, 256, 0, st>>>(jobs_dev, units_dev, units, run); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_split_batched(const SplitArgs* jobs_dev, const int2* rowmax_units_dev, int64_t rowmax_units,
                                 const int2* digit_units_dev, int64_t digit_units, cudaStream_t st) {
  if (rowmax_units > 0) { rowmax_batched<<<(unsigned)rowmax_units, 256, 0, st>>>(jobs_dev, rowmax_units_dev); note_launch(); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (digit_units > 0) { digits_batched<<<(unsigned)digit_units, 256, 0, st>>>(jobs_dev, digit_units_dev, digit_units, nullptr); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_native_batched(const NativeArgs* calls_dev, int ncalls, const int* const* flags_dev, int* list_dev,
                                  int64_t* prefix_dev, int64_t* total_dev, int grid, cudaStream_t st) {
  if (ncalls <= 0) return cudaSuccess;
  { native_compact<<<1, 1024, 0, st>>>(calls_dev, ncalls, flags_dev, list_dev, prefix_dev, total_dev); note_launch(); }
  { native_batched<<<grid, 256, 0, st>>>(calls_dev, list_dev, prefix_dev, total_dev); note_launch(); }
  return cudaGetLastError();
}

}  // namespace ozg
