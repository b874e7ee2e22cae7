// Exact real dot product on the integer pipes, for the sampled error check of a real GEMM, and
// the double-double primitives it ends with.  The functions use only integer, conversion and
// plain FP64 operations (no warp shuffles), so the unit tests also compile them for the host.
#pragma once
#include <cstdint>

namespace ozg {

struct dd {
  double hi, lo;
};
__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}

// Exact real dot product on the integer pipes.  With E = e_i + f_j from the split's row and
// column exponents, every |a_il b_lj| < 2^E, so each term -- the 106-bit product of the two 53-bit
// significands times a power of two -- is below 2^100 in units of 2^(E - 100).  The terms are
// summed in a signed 128-bit fixed-point accumulator with that unit; bits below it are truncated
// (each term toward zero), so the sum is exact to within k units, k 2^(E - 100), a relative 2^-100
// of the largest term per term.  For k < 2^26 the sum stays below 2^126.  The double-double
// result is formed from three exact 52-bit pieces.  FP64 is this part's slowest pipe; this path
// issues no FP64 instruction per term beyond the |a||b| scale.
struct i128 {
  unsigned long long lo;
  long long hi;
};
__device__ __forceinline__ void significand(uint64_t bits, uint64_t& m, int& x) {  // |v| = m 2^x
  const int eb = (int)((bits >> 52) & 0x7FF);
  m = bits & 0xFFFFFFFFFFFFFull;
  if (eb != 0) {
    m |= 1ull << 52;
    x = eb - 1075;
  } else {
    x = -1074;
  }
}
__device__ __forceinline__ void add_exact_term(i128& acc, uint64_t abits, uint64_t bbits, int unit) {
  if ((abits << 1) == 0 || (bbits << 1) == 0) return;  // a zero factor (either sign)
  uint64_t ma, mb;
  int xa, xb;
  significand(abits, ma, xa);
  significand(bbits, mb, xb);
  const unsigned long long plo = ma * mb, phi = __umul64hi(ma, mb);
  const int sh = xa + xb - unit;  // the term is (phi, plo) 2^sh units, below 2^100 units
  unsigned long long qlo, qhi;
  if (sh >= 0) {
    if (sh >= 64) {  // then the product is below 2^36 and phi == 0
      qhi = plo << (sh - 64);
      qlo = 0;
    } else if (sh == 0) {
      qhi = phi;
      qlo = plo;
    } else {
      qhi = (phi << sh) | (plo >> (64 - sh));
      qlo = plo << sh;
    }
  } else {
    const int r = -sh;
    if (r >= 128) {
      qhi = qlo = 0;
    } else if (r >= 64) {
      qhi = 0;
      qlo = phi >> (r - 64);
    } else {
      qhi = phi >> r;
      qlo = (plo >> r) | (phi << (64 - r));
    }
  }
  if (((abits ^ bbits) >> 63) == 0) {
    const unsigned long long nl = acc.lo + qlo;
    acc.hi += (long long)qhi + (nl < acc.lo ? 1 : 0);
    acc.lo = nl;
  } else {
    const unsigned long long nl = acc.lo - qlo;
    acc.hi -= (long long)qhi + (acc.lo < qlo ? 1 : 0);
    acc.lo = nl;
  }
}
// a += b (two's complement, 128 bits)
__device__ __forceinline__ void i128_add(i128& a, const i128& b) {
  const unsigned long long nl = a.lo + b.lo;
  a.hi += b.hi + (nl < a.lo ? 1 : 0);
  a.lo = nl;
}
// S 2^unit as a double-double for |S| < 2^126: S = s2 2^104 + s1 2^52 + s0 with s0, s1 in
// [0, 2^52) and |s2| < 2^22, three exact doubles summed with TwoSum and one dd addition.
__device__ __forceinline__ dd i128_to_dd(const i128& a, int unit) {
  const unsigned long long m52 = (1ull << 52) - 1;
  const double s0 = (double)(long long)(a.lo & m52);
  const double s1 = ldexp((double)(long long)(((a.lo >> 52) | ((unsigned long long)a.hi << 12)) & m52), 52);
  const double s2 = ldexp((double)(a.hi >> 40), 104);
  dd r = two_sum(s2, s1);
  r = dd_add(r, {s0, 0.0});
  return {ldexp(r.hi, unit), ldexp(r.lo, unit)};
}

}  // namespace ozg
