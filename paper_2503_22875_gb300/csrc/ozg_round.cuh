// The single rounding of the epilogues: RN(N 2^E) for an exact integer N and a power of two
// 2^E, rounded once to FP64 with ties to even (the result T of the emulated product, Sec. 2.2,
// taken as one rounding of the exact sum).  N is a 128-bit integer (the exact epilogue's Horner
// sum) or two int64 windows N = W0 2^S + W1 (the default epilogue).  Integer instructions and
// one correctly rounded 64-bit integer -> f64 conversion; results outside the normal range (subnormal,
// zero or overflow) take round_edge, which rounds onto the grid of the smallest subnormal
// directly, so that no second rounding follows the 53-bit one.  The functions use only integer
// operations, conversion intrinsics and exact ldexp scalings, so the unit tests also compile
// them for the host.
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

// ---- integer windows (default epilogue) ----------------------------------------------------
// The group sums enter R by Horner's rule in exact int64 arithmetic, c consecutive groups per
// window, where c is the largest count whose worst case stays below 2^63:
//   |G_g| <= (g - 1) * kpad * 127^2 (x2 for the complex combine) <= gmax < 2^L,
//   |window| <= gmax (128^c - 1) / 127 < 2^(L + 7 c) / 127 <= 2^69 / 127   with
//   c = (62 - L) / 7 + 1, i.e. L + 7 c <= 69: below 2^62 (128/127) < 2^63 - 2^57.
// Two windows form the exact 128-bit N = W0 128^len1 + W1, rounded to FP64 once with integer
// instructions only; a third and later window continue in FP64 (one rounding per window).
__device__ __forceinline__ int window_len(int s, int64_t kpad, int cplx) {
  const unsigned long long gmax = (unsigned long long)s * (unsigned long long)kpad * 16129ull * (cplx ? 2ull : 1ull);
  const int L = 64 - __clzll((long long)gmax);
  const int c = (62 - L) / 7 + 1;
  return c < 1 ? 1 : c;
}

// (a 2^sh + b) as a 128-bit two's complement integer (hi, lo), 1 <= sh <= 63.
__device__ __forceinline__ void i128_shl_add(long long a, int sh, long long b, long long& hi, unsigned long long& lo) {
  lo = (unsigned long long)a << sh;
  hi = a >> (64 - sh);
  const unsigned long long nl = lo + (unsigned long long)b;
  hi += (b < 0 ? -1 : 0) + (nl < lo ? 1 : 0);
  lo = nl;
}

static __device__ __noinline__ double round_i128_slow(long long hi, unsigned long long lo, int E) {
  return round_i128(hi, lo, E);
}

// RN(N 2^E) for the 128-bit integer N = (hi, lo), |N| < 2^126: the magnitude's top 64 bits with
// a sticky bit for everything below are converted with one correctly rounded conversion (the
// sticky bit sits below the guard bit, so the rounding is that of N itself), and the power of
// two is applied by adding to the exponent field.  Results outside the normal range take the
// general path.
__device__ __forceinline__ double rn_i128_pow2(long long hi, unsigned long long lo, int E) {
  const bool neg = hi < 0;
  unsigned long long mh = (unsigned long long)hi, ml = lo;
  if (neg) {
    ml = ~ml + 1;
    mh = ~mh + (ml == 0 ? 1 : 0);
  }
  double mag;
  int sh = 0;
  if (mh == 0) {
    if (ml == 0) return 0.0;
    mag = __ull2double_rn(ml);
  } else {
    sh = 64 - __clzll((long long)mh);  // 1 .. 62 for |N| < 2^126
    if (sh >= 64) return round_i128_slow(hi, lo, E);
    const unsigned long long top = (mh << (64 - sh)) | (ml >> sh);
    const unsigned long long sticky = (ml << (64 - sh)) != 0 ? 1ull : 0ull;
    mag = __ull2double_rn(top | sticky);
  }
  const long long bits = __double_as_longlong(mag);
  const int ex = (int)(bits >> 52) + E + sh;  // biased exponent of the result
  if (ex < 1 || ex > 2046) return round_i128_slow(hi, lo, E);
  const long long r = bits + ((long long)(E + sh) << 52);
  return __longlong_as_double(neg ? (r | (long long)0x8000000000000000ull) : r);
}

// RN(N 2^E) for N = W0 2^S + W1 (S = 7 wlen in [7, 56], |W0|, |W1| < 2^63 - 2^57, which the
// windows of window_len satisfy; W0 = 0 for a single window) without data-dependent branches,
// so the outputs of a chunk interleave.  With q = W0 + floor(W1 / 2^S) and r = W1 mod 2^S,
// N = q 2^S + r (0 <= r < 2^S).  Cut z low bits so that floor(N / 2^z) fits 63 bits past its
// sign, and fold whether any cut bit was set into its lowest bit: that is N rounded to odd at
// 2^z, with 63 significant bits whenever z > 0, so the correctly rounded signed int64 -> f64
// conversion rounds it to nearest exactly as it would round N itself (an odd-rounded value with
// at least two bits more than the target precision never creates or hides a tie).  The power of
// two goes into the exponent field.  `ok` is false when the result is not a normal double (the
// caller then takes final_val, which rounds the 128-bit N).
__device__ __forceinline__ double rn_windows(long long W0, long long W1, int S, int E, bool& ok) {
  const long long q = W0 + (W1 >> S);
  const unsigned long long r = (unsigned long long)W1 & ((1ull << S) - 1ull);
  const int bl = 64 - __clzll(q ^ (q >> 63));  // bits of q past its sign: -2^bl <= q < 2^bl
  const int z = max(0, bl + S - 63);           // <= S
  const long long t = (long long)(((unsigned long long)q << (S - z)) | (r >> z) |
                                  ((r & ((1ull << z) - 1ull)) != 0 ? 1ull : 0ull));
  const long long bits = __double_as_longlong(__ll2double_rn(t));
  const int ex = (int)((bits >> 52) & 0x7ff) + z + E;  // biased exponent of the result
  ok = t == 0 || (ex >= 1 && ex <= 2046);
  return t == 0 ? 0.0 : __longlong_as_double(bits + ((long long)(z + E) << 52));
}

}  // namespace ozg
