// Device helpers of the split step (Sec. 2.2): the power-of-two row scale from the row maximum's
// bits, and the base-2^7 digits of |x| 2^-e by truncation, with the sign of x.  Integer bit
// operations only (FP64 arithmetic is the slowest pipe of this GPU and not needed: a digit is
// seven bits of the 53-bit significand at a position fixed by the exponents).
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

namespace ozg {

constexpr uint64_t kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr uint64_t kInfBits = 0x7FF0000000000000ull;

// e = frexp exponent of the row maximum (max = 0.1f... 2^e), 0 for an all-zero row
__device__ __forceinline__ int exponent_from_maxbits(unsigned long long mb) {
  if (mb == 0) return 0;
  const int eb = (int)(mb >> 52);
  if (eb) return eb - 1022;                     // normal: 1.f 2^(eb-1023) = 0.1f 2^(eb-1022)
  return (64 - __clzll((long long)mb)) - 1074;  // subnormal: max in [2^(L-1), 2^L) 2^-1074
}

// |x| = mant 2^ex exactly (mant < 2^53); q0 = ex - e positions the significand against the
// row scale: digit t of |x| 2^-e is floor(mant 2^(q0 + 7t)) mod 128.
struct DigitSrc {
  uint64_t mant;
  int q0;
  bool neg;
};
__device__ __forceinline__ DigitSrc digit_src(uint64_t b, int e) {
  DigitSrc d;
  const int eb = (int)((b >> 52) & 0x7FF);
  d.mant = b & 0xFFFFFFFFFFFFFull;
  int ex = -1074;
  if (eb != 0) {
    d.mant |= 1ull << 52;
    ex = eb - 1075;
  }
  d.q0 = ex - e;
  d.neg = (b >> 63) != 0;
  return d;
}
// |digit t| in [0, 127]: bits [-q, -q + 7) of the significand, q = q0 + 7t
__device__ __forceinline__ uint32_t digit_mag(const DigitSrc& d, int t) {
  const int q = d.q0 + 7 * t;
  if (q >= 7) return 0u;
  if (q >= 0) return (uint32_t)(d.mant << q) & 127u;
  if (q > -64) return (uint32_t)(d.mant >> (-q)) & 127u;
  return 0u;
}
// Two signed digits as packed FP16 (low half = first): 1024 + |d| has the FP16 bits 0x6400 | |d|
// (ulp 1 on [1024, 2048)), so one exact half2 subtraction gives |d|; the sign bit is set for
// negative non-zero digits (zero stays +0).
__device__ __forceinline__ uint32_t digits_to_half2(uint32_t m0, bool n0, uint32_t m1, bool n1) {
  const uint32_t biased = 0x64006400u | m0 | (m1 << 16);
  const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&biased), __halves2half2(__ushort_as_half(0x6400),
                                                                                       __ushort_as_half(0x6400)));
  uint32_t r = *reinterpret_cast<const uint32_t*>(&v);
  r |= (n0 && m0 ? 0x8000u : 0u) | (n1 && m1 ? 0x80000000u : 0u);
  return r;
}
// Eight consecutive elements' digit t as one 16-byte store word.
__device__ __forceinline__ uint4 digits8(const DigitSrc (&d)[8], int t) {
  uint4 o;
  o.x = digits_to_half2(digit_mag(d[0], t), d[0].neg, digit_mag(d[1], t), d[1].neg);
  o.y = digits_to_half2(digit_mag(d[2], t), d[2].neg, digit_mag(d[3], t), d[3].neg);
  o.z = digits_to_half2(digit_mag(d[4], t), d[4].neg, digit_mag(d[5], t), d[5].neg);
  o.w = digits_to_half2(digit_mag(d[6], t), d[6].neg, digit_mag(d[7], t), d[7].neg);
  return o;
}

}  // namespace ozg
