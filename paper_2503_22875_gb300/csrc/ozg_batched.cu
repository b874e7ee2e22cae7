// Batched companions of the split, native and check kernels for the grouped GEMM: one launch
// covers every call of a batch (a device-side job table plus a prefix sum of work units per job;
// each CTA finds its job by binary search), so a batch of thousands of uneven GEMMs costs a
// handful of launches and captures into a short CUDA graph.
//   * split: the same exponents and digits as the single-call kernels (Sec. 2.2's split), one
//     job per operand;
//   * native: FP64 GEMM (real) for the calls whose inputs held Inf/NaN, on a device-compacted list;
//   * check: the sampled double-double error of every call (one warp per sample).
#include "ozg_internal.h"

namespace ozg {
namespace {

constexpr uint64_t kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr uint64_t kInfBits = 0x7FF0000000000000ull;

__device__ __forceinline__ int find_job(const int64_t* prefix, int njobs, int64_t unit) {
  // largest j with prefix[j] <= unit (prefix[0] = 0, prefix[njobs] = total)
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

__device__ __forceinline__ int exponent_from_maxbits(unsigned long long mb) {
  if (mb == 0) return 0;
  int eb = (int)(mb >> 52);
  if (eb) return eb - 1022;
  return (64 - __clzll((long long)mb)) - 1074;
}

__device__ __forceinline__ unsigned __int128 fixed_point(uint64_t b, int e, int s7) {
  int eb = (int)((b >> 52) & 0x7FF);
  uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  int ex;
  if (eb == 0) {
    ex = -1074;
  } else {
    mant |= 1ull << 52;
    ex = eb - 1075;
  }
  int sh = ex - e + s7;
  if (sh >= 0) return sh < 128 ? ((unsigned __int128)mant << sh) : (unsigned __int128)0;
  if (sh > -64) return (unsigned __int128)(mant >> (-sh));
  return 0;
}

__device__ __forceinline__ uint16_t digit_half_bits(unsigned __int128 F, int shift, bool neg) {
  int d = (int)((uint32_t)(F >> shift) & 127u);
  return __half_as_ushort(__int2half_rn(neg ? -d : d));
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

// Units: strided jobs -> 256 rows per unit (thread per row); contiguous -> 8 rows (warp per row).
__global__ void __launch_bounds__(256) rowmax_batched(const SplitArgs* jobs, const int64_t* prefix, int njobs) {
  const int64_t unit = blockIdx.x;
  const int jb = find_job(prefix, njobs, unit);
  const SplitArgs J = jobs[jb];
  const int64_t u = unit - prefix[jb];
  unsigned long long mx = 0;
  if (J.strided) {
    const int64_t row = u * 256 + threadIdx.x;
    if (row >= J.rows) return;
    for (int64_t l = 0; l < J.k; ++l) {
      uint64_t re, im;
      load_elem(J, row, l, re, im);
      re &= kAbsMask;
      im &= kAbsMask;
      re = re > im ? re : im;
      mx = re > mx ? re : mx;
    }
    J.maxbits[row] = mx;
    if (mx >= kInfBits) atomicExch(J.nonfinite, 1);
  } else {
    const int64_t row = u * 8 + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= J.rows) return;
    for (int64_t l = lane; l < J.k; l += 32) {
      uint64_t re, im;
      load_elem(J, row, l, re, im);
      re &= kAbsMask;
      im &= kAbsMask;
      re = re > im ? re : im;
      mx = re > mx ? re : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    if (lane == 0) {
      J.maxbits[row] = mx;
      if (mx >= kInfBits) atomicExch(J.nonfinite, 1);
    }
  }
}

// Units: 32 rows x 64 k tiles.  Thread t computes row t/8 and the 8 consecutive k at (t%8)*8.
__global__ void __launch_bounds__(256) digits_batched(const SplitArgs* jobs, const int64_t* prefix, int njobs) {
  __shared__ uint64_t tile[2][64][33];
  const int64_t unit = blockIdx.x;
  const int jb = find_job(prefix, njobs, unit);
  const SplitArgs J = jobs[jb];
  const int64_t u = unit - prefix[jb];
  const int64_t ltiles = (J.k + 63) / 64;
  const int64_t r0 = (u / ltiles) * 32, l0 = (u % ltiles) * 64;
  const int tid = threadIdx.x;
  const int r = tid / 8, lg = (tid % 8) * 8;
  const int64_t row = r0 + r;
  uint64_t bre[8], bim[8];
  if (J.strided) {
    // stage through shared memory: consecutive threads read consecutive rows of one column
    const int rr = tid % 32;
    for (int q = 0; q < 8; ++q) {
      const int li = tid / 32 + 8 * q;
      uint64_t re = 0, im = 0;
      if (r0 + rr < J.rows && l0 + li < J.k) load_elem(J, r0 + rr, l0 + li, re, im);
      tile[0][li][rr] = re;
      tile[1][li][rr] = im;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      bre[q] = tile[0][lg + q][r];
      bim[q] = tile[1][lg + q][r];
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      bre[q] = 0;
      bim[q] = 0;
      if (row < J.rows && l0 + lg + q < J.k) load_elem(J, row, l0 + lg + q, bre[q], bim[q]);
    }
  }
  if (row >= J.rows || l0 + lg >= J.k) return;
  const int e = exponent_from_maxbits(J.maxbits[row]);
  if (l0 + lg == 0) J.exps[row] = e;
  const int s7 = 7 * J.s;
  const int parts = J.cplx ? 2 : 1;
  for (int part = 0; part < parts; ++part) {
    unsigned __int128 F[8];
    bool neg[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint64_t b = part ? bim[q] : bre[q];
      F[q] = fixed_point(b, e, s7);
      neg[q] = (b >> 63) != 0;
    }
    const int64_t orow = J.cplx ? 2 * row + part : row;
    for (int t = 1; t <= J.s; ++t) {
      const int sh = 7 * (J.s - t);
      uint16_t h[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) h[q] = digit_half_bits(F[q], sh, neg[q]);
      uint4 out;
      out.x = h[0] | ((uint32_t)h[1] << 16);
      out.y = h[2] | ((uint32_t)h[3] << 16);
      out.z = h[4] | ((uint32_t)h[5] << 16);
      out.w = h[6] | ((uint32_t)h[7] << 16);
      *reinterpret_cast<uint4*>(J.D + ((int64_t)(t - 1) * J.plane_rows + orow) * J.Kp + l0 + lg) = out;
    }
  }
}

// ---------------------------------------------------------------------------- native fallback
// Device-side compaction of the calls whose non-finite flag is set, then a persistent FP64
// kernel over their 64 x 64 output tiles.
__global__ void native_compact(const NativeArgs* calls, int ncalls, const int* const* flags, int* list,
                               int64_t* tile_prefix, int64_t* total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t acc = 0;
  int n = 0;
  for (int c = 0; c < ncalls; ++c) {
    if (*flags[c] == 0) continue;
    list[n] = c;
    tile_prefix[n] = acc;
    acc += ((calls[c].m + 63) / 64) * ((calls[c].n + 63) / 64);
    ++n;
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

__global__ void repair_prep_batched(const RepairJob* jobs, int njobs, double target) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= njobs) return;
  const RepairJob J = jobs[i];
  const double e = J.err ? *J.err : 0.0;
  const bool bad = J.auto_mode && !(J.nonfinite && *J.nonfinite) && !(e <= target);
  *J.skip2 = bad ? 0 : 1;
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

cudaError_t launch_repair_prep_batched(const RepairJob* jobs_dev, int njobs, double target, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  repair_prep_batched<<<(njobs + 127) / 128, 128, 0, st>>>(jobs_dev, njobs, target);
  return cudaGetLastError();
}

cudaError_t launch_save_restore_batched(const RepairJob* jobs_dev, const int64_t* prefix_dev, int64_t units,
                                        int njobs, int restore, cudaStream_t st) {
  if (units <= 0 || njobs <= 0) return cudaSuccess;
  save_restore_batched<<<(unsigned)units, 256, 0, st>>>(jobs_dev, prefix_dev, njobs, restore);
  return cudaGetLastError();
}

cudaError_t launch_split_batched(const SplitArgs* jobs_dev, const int64_t* rowmax_prefix_dev, int64_t rowmax_units,
                                 const int64_t* digit_prefix_dev, int64_t digit_units, int njobs, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (rowmax_units > 0) rowmax_batched<<<(unsigned)rowmax_units, 256, 0, st>>>(jobs_dev, rowmax_prefix_dev, njobs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (digit_units > 0) digits_batched<<<(unsigned)digit_units, 256, 0, st>>>(jobs_dev, digit_prefix_dev, njobs);
  return cudaGetLastError();
}

cudaError_t launch_native_batched(const NativeArgs* calls_dev, int ncalls, const int* const* flags_dev, int* list_dev,
                                  int64_t* prefix_dev, int64_t* total_dev, int grid, cudaStream_t st) {
  if (ncalls <= 0) return cudaSuccess;
  native_compact<<<1, 32, 0, st>>>(calls_dev, ncalls, flags_dev, list_dev, prefix_dev, total_dev);
  native_batched<<<grid, 256, 0, st>>>(calls_dev, list_dev, prefix_dev, total_dev);
  return cudaGetLastError();
}

}  // namespace ozg
