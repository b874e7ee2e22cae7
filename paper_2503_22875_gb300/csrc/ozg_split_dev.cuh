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
constexpr int kMaxPlanes = 18;  // digit planes of the widest split (the largest slice count)

// e = frexp exponent of the row maximum (max = 0.1f... 2^e), 0 for an all-zero row
__device__ __forceinline__ int exponent_from_maxbits(unsigned long long mb) {
  if (mb == 0) return 0;
  const int eb = (int)(mb >> 52);
  if (eb) return eb - 1022;                     // normal: 1.f 2^(eb-1023) = 0.1f 2^(eb-1022)
  return (64 - __clzll((long long)mb)) - 1074;  // subnormal: max in [2^(L-1), 2^L) 2^-1074
}

// Fixed-point words of |x| 2^-e in [0, 1): fa = floor(|x| 2^(63 - e)) holds digits 1..9 and
// fb = floor(|x| 2^(126 - e)) mod 2^63 holds digits 10..18, so digit t (the t-th base-2^7 digit,
// by truncation) is one shift and mask:
//   t <= 9:  (fa >> (63 - 7t)) & 127        t >= 10:  (fb >> (126 - 7t)) & 127.
// |x| = mant 2^ex exactly (mant < 2^53, and mant 2^ex < 2^e, so ex - e <= -53).
struct DigitSrc {
  uint64_t fa, fb;
  uint32_t neg;  // 0x8000 for negative x (the FP16 sign bit), else 0
};
__device__ __forceinline__ uint64_t shift_signed(uint64_t m, int sh) {  // floor(m 2^sh), 0 past 63 bits
  if (sh >= 0) return sh < 64 ? (m << sh) : 0ull;
  return sh > -64 ? (m >> (-sh)) : 0ull;
}
__device__ __forceinline__ DigitSrc digit_src(uint64_t b, int e) {
  DigitSrc d;
  const int eb = (int)((b >> 52) & 0x7FF);
  uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  int ex = -1074;
  if (eb != 0) {
    mant |= 1ull << 52;
    ex = eb - 1075;
  }
  const int sa = ex - e + 63;  // <= 10: fa < 2^63
  d.fa = shift_signed(mant, sa);
  d.fb = shift_signed(mant, sa + 63) & 0x7FFFFFFFFFFFFFFFull;
  d.neg = (b >> 63) != 0 ? 0x8000u : 0u;
  return d;
}
// The same with only fa (digits 1 .. 9); fb is left 0.
__device__ __forceinline__ DigitSrc digit_src_first(uint64_t b, int e) {
  DigitSrc d;
  const int eb = (int)((b >> 52) & 0x7FF);
  uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  int ex = -1074;
  if (eb != 0) {
    mant |= 1ull << 52;
    ex = eb - 1075;
  }
  d.fa = shift_signed(mant, ex - e + 63);
  d.fb = 0;
  d.neg = (b >> 63) != 0 ? 0x8000u : 0u;
  return d;
}
// |digit t| in [0, 127]
__device__ __forceinline__ uint32_t digit_mag(const DigitSrc& d, int t) {
  return t <= 9 ? (uint32_t)(d.fa >> (63 - 7 * t)) & 127u : (uint32_t)(d.fb >> (126 - 7 * t)) & 127u;
}
// Two signed digits as packed FP16 (low half = first): 1024 + |d| has the FP16 bits 0x6400 | |d|
// (ulp 1 on [1024, 2048)), so one exact half2 subtraction gives |d|, and the sign bit is ORed in
// (a negative zero digit multiplies and sums exactly like +0).
__device__ __forceinline__ uint32_t digits_to_half2(uint32_t m0, uint32_t m1, uint32_t negmask) {
  const uint32_t biased = 0x64006400u | m0 | (m1 << 16);
  const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&biased), __halves2half2(__ushort_as_half(0x6400),
                                                                                       __ushort_as_half(0x6400)));
  return *reinterpret_cast<const uint32_t*>(&v) | negmask;
}
// Eight consecutive elements' digit t as one 16-byte store word.
__device__ __forceinline__ uint4 digits8(const DigitSrc (&d)[8], int t) {
  uint4 o;
  o.x = digits_to_half2(digit_mag(d[0], t), digit_mag(d[1], t), d[0].neg | (d[1].neg << 16));
  o.y = digits_to_half2(digit_mag(d[2], t), digit_mag(d[3], t), d[2].neg | (d[3].neg << 16));
  o.z = digits_to_half2(digit_mag(d[4], t), digit_mag(d[5], t), d[4].neg | (d[5].neg << 16));
  o.w = digits_to_half2(digit_mag(d[6], t), digit_mag(d[7], t), d[6].neg | (d[7].neg << 16));
  return o;
}

// Digit planes t_lo .. t_hi of eight consecutive elements, one 16-byte store per plane at
// out + (t - 1) plane.  The loop runs over every possible t, unrolled, so that each digit is a
// shift by a constant; planes outside [t_lo, t_hi] are skipped.
template <int TMAX>
__device__ __forceinline__ void store_digit_planes(const DigitSrc (&d)[8], int t_lo, int t_hi, __half* out,
                                                   int64_t plane) {
#pragma unroll
  for (int t = 1; t <= TMAX; ++t)
    if (t >= t_lo && t <= t_hi) *reinterpret_cast<uint4*>(out + (int64_t)(t - 1) * plane) = digits8(d, t);
}

}  // namespace ozg
