// The single rounding of the exact epilogue: RN(N 2^E) for a 128-bit integer N (|N| < 2^127)
// and a power of two 2^E, rounded once to FP64 with ties to even (the result T of the emulated
// product, Sec. 2.2, taken as one rounding of the exact sum).  Integer instructions and one
// correctly rounded u64 -> f64 conversion; results outside the normal range (subnormal, zero
// or overflow) take round_edge, which rounds onto the grid of the smallest subnormal directly,
// so that no second rounding follows the 53-bit one.
#pragma once
#include <cstdint>

namespace ozg {

// RN(|N| 2^E) with the sign applied, for |N| = (mh, ml) != 0, |N| < 2^127.  The ulp of the
// result is 2^q, q = max(top - 52, -1074), top = the exponent of N's leading bit in N 2^E;
// |N| is cut r = q - E bits below its top, with the round bit and a sticky bit.
static __device__ __noinline__ double round_edge(bool neg, uint64_t mh, uint64_t ml, int E) {
  const double sgn = neg ? -1.0 : 1.0;
  const int p = mh != 0 ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);  // bit length
  const int top = p - 1 + E;
  if (top > 1023) return sgn * __longlong_as_double(0x7FF0000000000000ll);
  const int q = max(top - 52, -1074);
  const int r = q - E;
  if (r <= 0) return sgn * ldexp((double)ml, E);  // |N| < 2^53 and a multiple of 2^E: exact
  if (r >= 128) return sgn * 0.0;                 // |N| 2^E < 2^-1075: below half the smallest step
  uint64_t Q, rb, st;
  if (r < 64) {
    Q = (ml >> r) | (mh << (64 - r));
    rb = (ml >> (r - 1)) & 1ull;
    st = (ml & ((1ull << (r - 1)) - 1ull)) != 0 ? 1ull : 0ull;
  } else if (r == 64) {
    Q = mh;
    rb = ml >> 63;
    st = (ml << 1) != 0 ? 1ull : 0ull;
  } else {
    Q = mh >> (r - 64);
    rb = (mh >> (r - 65)) & 1ull;
    st = (ml != 0 || (mh & ((1ull << (r - 65)) - 1ull)) != 0) ? 1ull : 0ull;
  }
  Q += rb & (st | (Q & 1ull));                   // Q <= 2^53 after the carry
  return sgn * ldexp((double)Q, q);              // exact, or +-inf when the carry passes 2^1024
}

// RN(N 2^E) for the 128-bit two's complement integer N = (hi, lo), |N| < 2^127: the top 64 bits
// of |N| with a sticky bit for the rest are converted with one correct rounding (the sticky bit
// sits below the guard bit, so the rounding is that of N itself), and the power of two goes into
// the exponent field when the result is a normal double.
__device__ __forceinline__ double round_i128(int64_t hi, uint64_t lo, int E) {
  const bool neg = hi < 0;
  uint64_t mh = (uint64_t)hi, ml = lo;
  if (neg) {
    ml = ~ml + 1;
    mh = ~mh + (ml == 0 ? 1 : 0);
  }
  if ((mh | ml) == 0) return 0.0;
  int sh = 0;
  uint64_t t = ml;
  if (mh != 0) {
    sh = 64 - __clzll((long long)mh);
    t = sh == 64 ? (mh | (ml != 0 ? 1ull : 0ull))
                 : ((mh << (64 - sh)) | (ml >> sh) | ((ml << (64 - sh)) != 0 ? 1ull : 0ull));
  }
  const long long bits = __double_as_longlong(__ull2double_rn(t));
  const int ex = (int)(bits >> 52) + E + sh;  // biased exponent of the result
  if (ex < 1 || ex > 2046) return round_edge(neg, mh, ml, E);
  const long long rb = bits + ((long long)(E + sh) << 52);
  return __longlong_as_double(neg ? (rb | (long long)0x8000000000000000ull) : rb);
}

}  // namespace ozg
