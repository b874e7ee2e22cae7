// K8: per-call error report.  For S sampled output entries (i, j) the kernel recomputes
// alpha * sum_l op(A)_il op(B)_lj + beta * C_old in double-double (the "quad using double"
// arithmetic of Sec. 2.2: TwoProd by fma, TwoSum) and returns
//   max |C_ij - ref_ij| / (|alpha| (|A||B|)_ij + |beta| |C_old,ij|)
// -- the componentwise error relative to |A||B|.  One warp per sample; lanes split k.
// For complex data the four real sub-sums are tracked and both parts are checked; optionally the
// per-part errors relative to the parts themselves are reported as well, the max_real / max_imag
// accuracy measure of the paper's MuST study (Sec. 3.2, relative error of the real and of the
// imaginary part, maximised over the sampled entries).
#include "ozg_exactdot.cuh"
#include "ozg_internal.h"

namespace ozg {
namespace {

__device__ __forceinline__ dd dd_add_prod(dd a, double x, double y) {  // a + x*y
  double p = x * y;
  double e = fma(x, y, -p);
  return dd_add(a, {p, e});
}
__device__ __forceinline__ dd dd_shfl_xor(dd a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ void sample_ij(const CheckArgs& P, int idx, int64_t& i, int64_t& j) {
  // the four corners first, then hashed positions
  if (idx < 4) {
    i = (idx & 1) ? P.m - 1 : 0;
    j = (idx & 2) ? P.n - 1 : 0;
    return;
  }
  uint64_t h = splitmix64(P.seed + (uint64_t)idx);
  i = (int64_t)((h & 0xFFFFFFFFull) % (uint64_t)P.m);
  j = (int64_t)((h >> 32) % (uint64_t)P.n);
}

__device__ __forceinline__ double ld_op(const double* X, int64_t ld, char t, int64_t r, int64_t c, int cplx,
                                        double* im) {
  if (!cplx) return (t == 'N') ? X[r + c * ld] : X[c + r * ld];
  const double* p = (t == 'N') ? X + 2 * (r + c * ld) : X + 2 * (c + r * ld);
  *im = (t == 'C') ? -p[1] : p[1];
  return p[0];
}

// One warp per (call, sample); the call's error goes to its own slot of err_out.
__device__ void check_one(const CheckArgs& P, int sample, int lane, double* err_slot);

__global__ void check_pre(CheckArgs P) {
  if (P.gate != nullptr && *P.gate) return;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.nsamp) return;
  int64_t i, j;
  sample_ij(P, idx, i, j);
  if (!P.cplx) {
    P.cold[2 * idx] = P.C[i + j * P.ldc];
    P.cold[2 * idx + 1] = 0.0;
  } else {
    P.cold[2 * idx] = P.C[2 * (i + j * P.ldc)];
    P.cold[2 * idx + 1] = P.C[2 * (i + j * P.ldc) + 1];
  }
}

// Compensated dot product (Dot2 of Ogita, Rump and Oishi, "Accurate sum and dot product",
// SIAM J. Sci. Comput. 26, 2005): the running sum s is updated by TwoSum with the exact product
// error from TwoProd, and both rounding errors go into one plain-double correction c.  The result
// s + c is as accurate as the dot product computed in twice the working precision and then
// rounded, at about half the FP64 operations of a full double-double accumulation.
struct dot2 {
  double s, c;
};
__device__ __forceinline__ void dot2_add(dot2& a, double x, double y) {
  const double p = x * y;
  const double pe = fma(x, y, -p);
  const double t = a.s + p;
  const double z = t - a.s;
  const double se = (a.s - (t - z)) + (p - z);
  a.s = t;
  a.c += se + pe;
}
__device__ __forceinline__ dd dot2_reduce_warp(dot2 a) {
  // pairwise: TwoSum of the partial sums, the corrections added plainly
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double os = __shfl_xor_sync(0xffffffffu, a.s, o), oc = __shfl_xor_sync(0xffffffffu, a.c, o);
    const dd t = two_sum(a.s, os);
    a.s = t.hi;
    a.c = a.c + oc + t.lo;
  }
  return fast_two_sum(a.s, a.c);
}

__device__ __forceinline__ dd exact_dot_reduce_warp(i128 a, int unit) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const i128 other = {__shfl_xor_sync(0xffffffffu, a.lo, o), __shfl_xor_sync(0xffffffffu, a.hi, o)};
    i128_add(a, other);
  }
  return i128_to_dd(a, unit);
}

__device__ void check_one(const CheckArgs& P, int sample, int lane, double* err_slot) {
  int64_t i, j;
  sample_ij(P, sample, i, j);
  dd re = {0, 0}, im = {0, 0};
  double sabs = 0.0;
  if (!P.cplx && P.ea != nullptr && P.fb != nullptr && P.k < (1ll << 26)) {
    const int unit = P.ea[i] + P.fb[j] - 100;
    i128 acc = {0ull, 0ll};
    for (int64_t l = lane; l < P.k; l += 32) {
      const double ar = (P.ta == 'N') ? P.A[i + l * P.lda] : P.A[l + i * P.lda];
      const double br = (P.tb == 'N') ? P.B[l + j * P.ldb] : P.B[j + l * P.ldb];
      add_exact_term(acc, __double_as_longlong(ar), __double_as_longlong(br), unit);
      sabs = fma(fabs(ar), fabs(br), sabs);
    }
    re = exact_dot_reduce_warp(acc, unit);
  } else if (!P.cplx) {
    dot2 acc = {0.0, 0.0};
    for (int64_t l = lane; l < P.k; l += 32) {
      const double ar = (P.ta == 'N') ? P.A[i + l * P.lda] : P.A[l + i * P.lda];
      const double br = (P.tb == 'N') ? P.B[l + j * P.ldb] : P.B[j + l * P.ldb];
      dot2_add(acc, ar, br);
      sabs = fma(fabs(ar), fabs(br), sabs);
    }
    re = dot2_reduce_warp(acc);
  }
  for (int64_t l = lane; P.cplx && l < P.k; l += 32) {
    double ai = 0, bi = 0;
    const double ar = ld_op(P.A, P.lda, P.ta, i, l, P.cplx, &ai);
    const double br = ld_op(P.B, P.ldb, P.tb, l, j, P.cplx, &bi);
    re = dd_add_prod(re, ar, br);
    re = dd_add_prod(re, -ai, bi);
    im = dd_add_prod(im, ar, bi);
    im = dd_add_prod(im, ai, br);
    sabs += (fabs(ar) + fabs(ai)) * (fabs(br) + fabs(bi));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (P.cplx) {
      re = dd_add(re, dd_shfl_xor(re, o));
      im = dd_add(im, dd_shfl_xor(im, o));
    }
    sabs += __shfl_xor_sync(0xffffffffu, sabs, o);
  }
  if (lane != 0) return;
  const double cr_old = P.beta_zero ? 0.0 : P.cold[2 * sample], ci_old = P.beta_zero ? 0.0 : P.cold[2 * sample + 1];
  double err;
  if (!P.cplx) {
    // ref = alpha * re + beta * c_old, kept to double-double accuracy before the comparison
    dd ref = {P.alpha[0] * re.hi, fma(P.alpha[0], re.hi, -P.alpha[0] * re.hi) + P.alpha[0] * re.lo};
    if (!P.beta_zero) ref = dd_add_prod(ref, P.beta[0], cr_old);
    const double c = P.C[i + j * P.ldc];
    const double diff = fabs((c - ref.hi) - ref.lo);
    const double scale = fabs(P.alpha[0]) * sabs + fabs(P.beta[0]) * fabs(cr_old);
    err = scale > 0 ? diff / scale : (diff > 0 ? INFINITY : 0.0);
  } else {
    dd rr = {0, 0}, ri = {0, 0};
    rr = dd_add_prod(rr, P.alpha[0], re.hi);
    rr = dd_add_prod(rr, P.alpha[0], re.lo);
    rr = dd_add_prod(rr, -P.alpha[1], im.hi);
    rr = dd_add_prod(rr, -P.alpha[1], im.lo);
    ri = dd_add_prod(ri, P.alpha[0], im.hi);
    ri = dd_add_prod(ri, P.alpha[0], im.lo);
    ri = dd_add_prod(ri, P.alpha[1], re.hi);
    ri = dd_add_prod(ri, P.alpha[1], re.lo);
    if (!P.beta_zero) {
      rr = dd_add_prod(rr, P.beta[0], cr_old);
      rr = dd_add_prod(rr, -P.beta[1], ci_old);
      ri = dd_add_prod(ri, P.beta[0], ci_old);
      ri = dd_add_prod(ri, P.beta[1], cr_old);
    }
    const double* cp = P.C + 2 * (i + j * P.ldc);
    const double dre = fabs((cp[0] - rr.hi) - rr.lo), dim = fabs((cp[1] - ri.hi) - ri.lo);
    const double d = fmax(dre, dim);
    if (P.part_err != nullptr) {  // per-part error relative to the part itself (max_real / max_imag)
      const double pr = rr.hi != 0.0 ? dre / fabs(rr.hi) : (dre > 0 ? INFINITY : 0.0);
      const double pi = ri.hi != 0.0 ? dim / fabs(ri.hi) : (dim > 0 ? INFINITY : 0.0);
      atomicMax(reinterpret_cast<unsigned long long*>(P.part_err), (unsigned long long)__double_as_longlong(pr));
      atomicMax(reinterpret_cast<unsigned long long*>(P.part_err + 1), (unsigned long long)__double_as_longlong(pi));
    }
    const double scale = (fabs(P.alpha[0]) + fabs(P.alpha[1])) * sabs +
                         (fabs(P.beta[0]) + fabs(P.beta[1])) * (fabs(cr_old) + fabs(ci_old));
    err = scale > 0 ? d / scale : (d > 0 ? INFINITY : 0.0);
  }
  // non-negative doubles order like their bit patterns; NaN (bits above +Inf) wins the max
  atomicMax(reinterpret_cast<unsigned long long*>(err_slot), (unsigned long long)__double_as_longlong(err));
}

__global__ void check_post(CheckArgs P) {
  if (P.gate != nullptr && *P.gate) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= P.nsamp) return;
  check_one(P, warp, lane, P.err_out);
}

// batched: calls[c] with nsamp samples each; warp w -> call w / nsamp, sample w % nsamp
__global__ void check_pre_batched(const CheckArgs* calls, int ncalls, int nsamp) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ncalls * nsamp) return;
  const CheckArgs* Pp = calls + idx / nsamp;
  if (Pp->beta_zero) return;
  const int* gate = Pp->gate;
  if (gate != nullptr && *gate) return;
  const CheckArgs P = *Pp;
  const int smp = (int)(idx % nsamp);
  int64_t i, j;
  sample_ij(P, smp, i, j);
  P.cold[2 * smp] = P.C[i + j * P.ldc];
  P.cold[2 * smp + 1] = 0.0;
}

__global__ void check_post_batched(const CheckArgs* calls, int ncalls, int nsamp) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (int64_t)ncalls * nsamp) return;
  const CheckArgs* Pp = calls + warp / nsamp;
  const int* gate = Pp->gate;  // read the gate before anything else (most re-run checks skip)
  if (gate != nullptr && *gate) return;
  const CheckArgs P = *Pp;
  check_one(P, (int)(warp % nsamp), lane, P.err_out);
}

}  // namespace

cudaError_t launch_check_pre(const CheckArgs& a, cudaStream_t st) {
  if (a.nsamp <= 0 || a.beta_zero) return cudaSuccess;
  { check_pre<<<(a.nsamp + 127) / 128, 128, 0, st>>>(a); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_check_batched_pre(const CheckArgs* calls_dev, int ncalls, int nsamp, cudaStream_t st) {
  const int64_t total = (int64_t)ncalls * nsamp;
  if (total <= 0) return cudaSuccess;
  { check_pre_batched<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(calls_dev, ncalls, nsamp); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_check_batched_post(const CheckArgs* calls_dev, int ncalls, int nsamp, double* errs_dev,
                                      cudaStream_t st) {
  const int64_t total = (int64_t)ncalls * nsamp;
  if (total <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(errs_dev, 0, sizeof(double) * ncalls, st);
  if (e != cudaSuccess) return e;
  { check_post_batched<<<(unsigned)((total + 3) / 4), 128, 0, st>>>(calls_dev, ncalls, nsamp); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_check_post(const CheckArgs& a, cudaStream_t st) {
  if (a.nsamp <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.err_out, 0, sizeof(double), st);
  if (e == cudaSuccess && a.part_err != nullptr) e = cudaMemsetAsync(a.part_err, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int warps_per_block = 4;
  { check_post<<<(a.nsamp + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(a); note_launch(); }
  return cudaGetLastError();
}

}  // namespace ozg
