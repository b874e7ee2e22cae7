// K1: per-row power-of-two scale and INT8-range digit planes (the split step of the Ozaki
// scheme, Sec. 2.2).  Row i of op(X) gets e_i = frexp exponent of max_l |x_il|; digit t of
// x is the t-th base-2^7 digit of |x| 2^-e_i taken by truncation, with the sign of x:
//   d_t = sign(x) * (floor(|x| 2^{7s - e_i}) >> 7(s - t)) & 127.
// Only integer bit operations are used (FP64 arithmetic is slow on this part and not
// needed: the fixed-point value is the 53-bit significand shifted).  HBM-bound: one read of
// op(X) for the maxima, one read plus s fp16 writes for the digits.
#include "../../include/ozg.h"
#include "ozg_internal.h"
#include "ozg_split_dev.cuh"

static_assert(ozg::kMaxPlanes == OZG_MAX_SLICES, "digit planes of the widest split");

namespace ozg {
namespace {

// Digit planes t_lo .. t_hi a launch writes: t_lo = *from + 1 (else 1), t_hi = *to (else s);
// nothing when *gate is non-zero.
struct PlaneRange {
  const int* from;
  const int* to;
  const int* gate;
  __device__ __forceinline__ bool resolve(int s, int& lo, int& hi) const {
    if (gate != nullptr && *gate) return false;
    lo = from != nullptr ? *from + 1 : 1;
    hi = to != nullptr ? *to : s;
    return lo <= hi;
  }
};

__device__ __forceinline__ void flag_nonfinite(uint64_t absbits, int* nonfinite) {
  if (absbits >= kInfBits) atomicExch(nonfinite, 1);
}

// ---------------------------------------------------------------- row maxima, contiguous rows
// one warp per row; lanes stride along l
__global__ void rowmax_contig(const double* __restrict__ X, int64_t ld, int64_t rows, int64_t k, int cplx,
                              unsigned long long* __restrict__ maxbits, int* nonfinite) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x % 32;
  if (row >= rows) return;
  unsigned long long mx = 0;
  if (!cplx) {
    const uint64_t* p = reinterpret_cast<const uint64_t*>(X) + row * ld;
    for (int64_t l = lane; l < k; l += 32) {
      uint64_t v = __ldg(p + l) & kAbsMask;
      mx = v > mx ? v : mx;
    }
  } else {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(X) + row * ld;
    for (int64_t l = lane; l < k; l += 32) {
      ulonglong2 v = __ldg(p + l);
      uint64_t a = v.x & kAbsMask, b = v.y & kAbsMask;
      a = a > b ? a : b;
      mx = a > mx ? a : mx;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  if (lane == 0) {
    maxbits[row] = mx;
    flag_nonfinite(mx, nonfinite);
  }
}

// ---------------------------------------------------------------- row maxima, strided rows
// thread per row (consecutive rows are contiguous in memory), grid.y splits k; atomicMax merges
__global__ void rowmax_strided(const double* __restrict__ X, int64_t ld, int64_t rows, int64_t k, int64_t kchunk,
                               int cplx, unsigned long long* __restrict__ maxbits, int* nonfinite) {
  int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows) return;
  int64_t l0 = (int64_t)blockIdx.y * kchunk, l1 = min(k, l0 + kchunk);
  unsigned long long mx = 0;
  if (!cplx) {
    const uint64_t* p = reinterpret_cast<const uint64_t*>(X);
    for (int64_t l = l0; l < l1; ++l) {
      uint64_t v = __ldg(p + row + l * ld) & kAbsMask;
      mx = v > mx ? v : mx;
    }
  } else {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(X);
    for (int64_t l = l0; l < l1; ++l) {
      ulonglong2 v = __ldg(p + row + l * ld);
      uint64_t a = v.x & kAbsMask, b = v.y & kAbsMask;
      a = a > b ? a : b;
      mx = a > mx ? a : mx;
    }
  }
  if (mx) {
    atomicMax(&maxbits[row], mx);
    flag_nonfinite(mx, nonfinite);
  }
}

// ---------------------------------------------------------------- digits, contiguous rows
// thread per (row, group of 8 consecutive l); 16-byte stores per digit plane
template <int CPLX>
__global__ void digits_contig(const double* __restrict__ X, int64_t ld, int64_t rows, int64_t k, int conj, int s,
                              int64_t Kp, int64_t plane_rows, const unsigned long long* __restrict__ maxbits,
                              int32_t* __restrict__ exps, __half* __restrict__ D, PlaneRange pr) {
  int t_lo, t_hi;
  if (!pr.resolve(s, t_lo, t_hi)) return;
  int64_t groups = (k + 7) / 8;
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= rows * groups) return;
  int64_t row = gid / groups, l0 = (gid % groups) * 8;
  int e = exponent_from_maxbits(maxbits[row]);
  if (l0 == 0 && t_lo == 1) exps[row] = e;
  const int nparts = CPLX ? 2 : 1;
  uint64_t bits[2][8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int64_t l = l0 + j;
    if (CPLX) {
      ulonglong2 v = (l < k) ? __ldg(reinterpret_cast<const ulonglong2*>(X) + row * ld + l) : make_ulonglong2(0, 0);
      bits[0][j] = v.x;
      bits[1][j] = conj ? (v.y ^ 0x8000000000000000ull) : v.y;
    } else {
      bits[0][j] = (l < k) ? __ldg(reinterpret_cast<const uint64_t*>(X) + row * ld + l) : 0ull;
    }
  }
#pragma unroll
  for (int part = 0; part < nparts; ++part) {
    DigitSrc ds[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) ds[j] = digit_src(bits[part][j], e);
    int64_t orow = CPLX ? 2 * row + part : row;
    store_digit_planes<kMaxPlanes>(ds, t_lo, t_hi, D + orow * Kp + l0, plane_rows * Kp);
  }
}

// ---------------------------------------------------------------- digits, strided rows
// block: 32 rows x 64 l tile staged (transposed) through shared memory
template <int CPLX>
__global__ void __launch_bounds__(256) digits_strided(const double* __restrict__ X, int64_t ld, int64_t rows,
                                                      int64_t k, int conj, int s, int64_t Kp, int64_t plane_rows,
                                                      const unsigned long long* __restrict__ maxbits,
                                                      int32_t* __restrict__ exps, __half* __restrict__ D,
                                                      PlaneRange pr) {
  int t_lo, t_hi;
  if (!pr.resolve(s, t_lo, t_hi)) return;
  constexpr int TR = 32, TL = 64;
  constexpr int W = CPLX ? 2 : 1;
  __shared__ uint64_t tile[TL][TR * W + 1];
  int64_t r0 = (int64_t)blockIdx.x * TR, l0 = (int64_t)blockIdx.y * TL;
  int tid = threadIdx.x;
  // load: thread -> (row = tid % 32, l = tid / 32 + 8 j)
  {
    int r = tid % TR;
    int64_t row = r0 + r;
    for (int j = 0; j < TL / 8; ++j) {
      int li = tid / TR + 8 * j;
      int64_t l = l0 + li;
      bool ok = row < rows && l < k;
      if (CPLX) {
        ulonglong2 v = ok ? __ldg(reinterpret_cast<const ulonglong2*>(X) + row + l * ld) : make_ulonglong2(0, 0);
        tile[li][2 * r] = v.x;
        tile[li][2 * r + 1] = conj ? (v.y ^ 0x8000000000000000ull) : v.y;
      } else {
        tile[li][r] = ok ? __ldg(reinterpret_cast<const uint64_t*>(X) + row + l * ld) : 0ull;
      }
    }
  }
  __syncthreads();
  // compute: thread -> (row = tid / 8, 8 consecutive l at (tid % 8) * 8)
  int r = tid / 8;
  int64_t row = r0 + r;
  int lg = (tid % 8) * 8;
  if (row >= rows || l0 + lg >= k) return;
  int e = exponent_from_maxbits(maxbits[row]);
  if (l0 + lg == 0 && t_lo == 1) exps[row] = e;
#pragma unroll
  for (int part = 0; part < W; ++part) {
    DigitSrc ds[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) ds[j] = digit_src(tile[lg + j][W * r + part], e);
    int64_t orow = CPLX ? 2 * row + part : row;
    store_digit_planes<kMaxPlanes>(ds, t_lo, t_hi, D + orow * Kp + l0 + lg, plane_rows * Kp);
  }
}

__global__ void digits_to_i8(const __half* __restrict__ D, int64_t planes_rows, int64_t k, int64_t Kp,
                             int8_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= planes_rows * k) return;
  int64_t r = i / k, l = i % k;
  out[i] = (int8_t)__half2int_rn(D[r * Kp + l]);
}

}  // namespace

cudaError_t launch_rowmax(const SplitArgs& a, cudaStream_t st) {
  if (a.rows <= 0) return cudaSuccess;
  cudaError_t err = cudaMemsetAsync(a.maxbits, 0, sizeof(unsigned long long) * a.rows, st);
  if (err != cudaSuccess) return err;
  if (a.k > 0) {
    if (!a.strided) {
      int wpb = 8;
      unsigned grid = (unsigned)((a.rows + wpb - 1) / wpb);
      { rowmax_contig<<<grid, 32 * wpb, 0, st>>>(a.X, a.ld, a.rows, a.k, a.cplx, a.maxbits, a.nonfinite); note_launch(); }
    } else {
      int64_t rb = (a.rows + 255) / 256;
      int64_t ksplit = (608 + rb - 1) / rb;  // ~4 CTAs per SM in total
      if (ksplit > a.k) ksplit = a.k;
      if (ksplit > 65535) ksplit = 65535;
      if (ksplit < 1) ksplit = 1;
      int64_t kchunk = (a.k + ksplit - 1) / ksplit;
      ksplit = (a.k + kchunk - 1) / kchunk;
      { rowmax_strided<<<dim3((unsigned)rb, (unsigned)ksplit), 256, 0, st>>>(a.X, a.ld, a.rows, a.k, kchunk, a.cplx,
                                                                           a.maxbits, a.nonfinite); note_launch(); }
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_digits(const SplitArgs& a, cudaStream_t st) {
  if (a.rows <= 0) return cudaSuccess;
  const PlaneRange pr{a.plane_from, a.plane_to, a.gate};
  int64_t kk = a.k > 0 ? a.k : 1;
  if (!a.strided || a.k == 0) {
    int64_t groups = (kk + 7) / 8;
    int64_t total = a.rows * groups;
    unsigned grid = (unsigned)((total + 255) / 256);
    if (a.cplx)
      { digits_contig<1><<<grid, 256, 0, st>>>(a.X, a.ld, a.rows, a.k, a.conj, a.s, a.Kp, a.plane_rows, a.maxbits,
                                             a.exps, a.D, pr); note_launch(); }
    else
      { digits_contig<0><<<grid, 256, 0, st>>>(a.X, a.ld, a.rows, a.k, a.conj, a.s, a.Kp, a.plane_rows, a.maxbits,
                                             a.exps, a.D, pr); note_launch(); }
  } else {
    dim3 grid((unsigned)((a.rows + 31) / 32), (unsigned)((a.k + 63) / 64));
    if (a.cplx)
      { digits_strided<1><<<grid, 256, 0, st>>>(a.X, a.ld, a.rows, a.k, a.conj, a.s, a.Kp, a.plane_rows, a.maxbits,
                                              a.exps, a.D, pr); note_launch(); }
    else
      { digits_strided<0><<<grid, 256, 0, st>>>(a.X, a.ld, a.rows, a.k, a.conj, a.s, a.Kp, a.plane_rows, a.maxbits,
                                              a.exps, a.D, pr); note_launch(); }
  }
  return cudaGetLastError();
}

cudaError_t launch_split(const SplitArgs& a, cudaStream_t st) {
  cudaError_t e = launch_rowmax(a, st);
  if (e != cudaSuccess) return e;
  return launch_digits(a, st);
}

cudaError_t launch_digits_to_i8(const __half* D, int64_t planes, int64_t plane_rows, int64_t k, int64_t Kp,
                                int8_t* out, cudaStream_t st) {
  int64_t total = planes * plane_rows * k;
  if (total <= 0) return cudaSuccess;
  { digits_to_i8<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(D, planes * plane_rows, k, Kp, out); note_launch(); }
  return cudaGetLastError();
}

}  // namespace ozg
