"""The epilogue's final rounding, compiled for the host (no GPU).  ozg_round.cuh uses only integer
and conversion intrinsics, so with host stand-ins for those (__clzll, a round-to-nearest u64 ->
f64 conversion, bit casts) g++ builds the same source.  Every result is compared with exact
rational rounding done by Python integers: RN(N 2^E), one rounding, ties to even, subnormals
and overflow included (CPython's int / int true division rounds correctly).  The cases cover
random magnitudes, ties and near-ties at the cut, the subnormal range and the overflow edge,
for the 128-bit form (exact epilogue) and the two-window form (default epilogue, with the
kernel's fallback for results that are not normal doubles)."""
import os
import random
import struct
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2503_22875_gb300", "csrc", "ozg_round.cuh")

HARNESS = r"""
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#define __device__
#define __noinline__ __attribute__((noinline))
#define __forceinline__ inline
static inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
static inline double __ull2double_rn(unsigned long long x) { return (double)x; }
static inline double __ll2double_rn(long long x) { return (double)x; }
static inline long long __double_as_longlong(double d) { long long r; std::memcpy(&r, &d, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; std::memcpy(&r, &x, 8); return r; }
using std::max;
#include "HEADER"
static void put(double v) { unsigned long long b; std::memcpy(&b, &v, 8); std::printf("%016llx\n", b); }
int main() {
  char mode;
  while (std::scanf(" %c", &mode) == 1) {
    if (mode == 'i') {  // 128-bit form
      long long hi; unsigned long long lo; int E;
      if (std::scanf("%lld %llu %d", &hi, &lo, &E) != 3) return 1;
      put(ozg::round_i128(hi, lo, E));
    } else if (mode == 'l') {  // window length
      int sw, cplx; long long kpad;
      if (std::scanf("%d %lld %d", &sw, &kpad, &cplx) != 3) return 1;
      std::printf("%d\n", ozg::window_len(sw, kpad, cplx));
    } else {            // two windows, as the default epilogue takes them
      long long W0, W1; int S, E;
      if (std::scanf("%lld %lld %d %d", &W0, &W1, &S, &E) != 4) return 1;
      bool ok = true;
      double v = ozg::rn_windows(W0, W1, S, E, ok);
      if (!ok) {
        long long hi; unsigned long long lo;
        ozg::i128_shl_add(W0, S, W1, hi, lo);
        v = ozg::rn_i128_pow2(hi, lo, E);
      }
      put(v);
    }
  }
  return 0;
}
"""


def exact_rn(N, E):
    if N == 0:
        return 0.0
    try:
        return N / 2 ** (-E) if E < 0 else float(N * 2 ** E)
    except OverflowError:
        return float("inf") if N > 0 else float("-inf")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("round")
    src = d / "h.cpp"
    src.write_text(HARNESS.replace("HEADER", HEADER))
    exe = str(d / "h")
    subprocess.check_call(["g++", "-O2", "-std=c++17", str(src), "-o", exe])
    return exe


def run(exe, lines):
    out = subprocess.run([exe], input="".join(lines), capture_output=True, text=True, check=True).stdout.split()
    return [struct.unpack(">d", bytes.fromhex(h))[0] for h in out]


def pick_exponent(g, p):
    """E for a p-bit magnitude: near the subnormal range, near overflow, or anywhere normal."""
    u = g.random()
    top = g.randint(-1140, -1015) if u < 0.4 else (g.randint(1010, 1030) if u < 0.6 else g.randint(-1000, 1000))
    return top - (p - 1)


def shaped(g, p):
    """A p-bit magnitude, sometimes cut to a tie or to zeros below a random position."""
    N = g.getrandbits(p) | (1 << (p - 1))
    u, k = g.random(), g.randint(1, p)
    if u < 0.2 and k < p:
        N = (N >> k << k) | (1 << (k - 1))
    elif u < 0.3:
        N = N >> k << k
    return N


def check(exe, cases, fmt):
    got = run(exe, [fmt(c) for c in cases])
    bad = [(c, x, exact_rn(c[0], c[1])) for c, x in zip(cases, got) if x != exact_rn(c[0], c[1])]
    assert not bad, f"{len(bad)} of {len(cases)} differ, e.g. {bad[:3]}"


def test_round_i128_equals_exact_rounding(harness):
    g = random.Random(11)
    cases = [(2 ** 55 + 1, -1130), (-(2 ** 55 + 1), -1130), (2 ** 55, -1130), (3, -1076), (3, -1075),
             (2 ** 53 - 1, -1074), (2 ** 54 - 1, 970), (2 ** 53 + 1, 970), (1, -1200), (2 ** 126 - 1, 900)]
    for _ in range(60000):
        p = g.randint(1, 126)
        N = shaped(g, p) * (-1 if g.random() < 0.5 else 1)
        cases.append((N, pick_exponent(g, p)))

    def fmt(c):
        u = c[0] % 2 ** 128
        hi = u >> 64
        return f"i {hi - 2 ** 64 if hi >= 2 ** 63 else hi} {u & (2 ** 64 - 1)} {c[1]}\n"
    check(harness, cases, fmt)


def test_two_window_rounding_equals_exact_rounding(harness):
    g = random.Random(12)
    raw = [(0, 2 ** 55 + 1, 7, -1130), (1, -1, 56, -1074 - 56), (-1, 1, 7, -1080), (2 ** 61, 2 ** 61, 56, 900)]
    wmax = 2 ** 69 // 127        # the largest window window_len admits (see the window test)
    raw += [(wmax, wmax, 56, 900), (-wmax, -wmax, 7, -1100), (wmax, -wmax, 49, 0)]
    for _ in range(60000):
        S = 7 * g.randint(1, 8)
        W0 = 0 if g.random() < 0.2 else g.randint(-wmax, wmax) >> g.randint(0, 61)
        W1 = g.randint(-wmax, wmax) >> g.randint(0, 61)
        if g.random() < 0.2:   # a tie or zeros in W1's low bits
            k = g.randint(1, 40)
            W1 = (W1 >> k << k) | ((1 << (k - 1)) if g.random() < 0.5 else 0)
        N = W0 * 2 ** S + W1
        p = max(abs(N).bit_length(), 1)
        raw.append((W0, W1, S, pick_exponent(g, p)))
    cases = [(W0 * 2 ** S + W1, E, W0, W1, S) for W0, W1, S, E in raw]
    check(harness, cases, lambda c: f"w {c[2]} {c[3]} {c[4]} {c[1]}\n")


def test_two_window_rounding_ties_and_near_ties_of_both_signs(harness):
    """Exact ties and one-unit neighbours of ties at the 53-bit cut, for sums of 60 to 118 bits of
    either sign (the sum then has bits both above and below the 63-bit window the two-window
    form keeps, so the folded sticky bit decides), split into the two windows in every way the
    epilogue can produce (the second window signed, its magnitude below 2^S or reaching past it)."""
    g = random.Random(13)
    wmax = 2 ** 69 // 127
    raw = []
    while len(raw) < 30000:
        S = 7 * g.randint(1, 8)
        L = g.randint(60, 118)
        m = g.getrandbits(53) | (1 << 52)
        N = m * 2 ** (L - 53) + 2 ** (L - 54) + g.choice([-1, 0, 0, 1])
        N = -N if g.random() < 0.5 else N
        W1 = N % 2 ** S - (2 ** S if g.random() < 0.5 else 0) + g.choice([0, 0, 1, -1]) * 2 ** S
        W0 = (N - W1) // 2 ** S
        if abs(W0) > wmax or abs(W1) > wmax:
            continue
        raw.append((W0, W1, S, pick_exponent(g, abs(N).bit_length())))
    cases = [(W0 * 2 ** S + W1, E, W0, W1, S) for W0, W1, S, E in raw]
    check(harness, cases, lambda c: f"w {c[2]} {c[3]} {c[4]} {c[1]}\n")


def test_window_length_keeps_every_window_in_int64(harness):
    """window_len(s, kpad, cplx) is the closed form c = (62 - L) / 7 + 1 (L the bit length of
    gmax = s kpad 127^2, doubled for complex), and the worst-case window, gmax (128^c - 1) / 127,
    stays below 2^69 / 127 < 2^63 - 2^57 -- the range rn_windows assumes -- over s = 1..18 and
    k padded to 64 (small k, then every 4099th multiple of 64 up to 2^26)."""
    params = [(s, 64 * kb, c) for c in (0, 1) for s in range(1, 19)
              for kb in sorted(set([1, 2, 3, 7, 8, 9, 16, 17] + list(range(1, 2 ** 20 + 1, 4099)) + [2 ** 20]))]
    got = subprocess.run([harness], input="".join(f"l {s} {k} {c}\n" for s, k, c in params), capture_output=True,
                         text=True, check=True).stdout.split()
    assert len(got) == len(params)
    for (s, kpad, cplx), w in zip(params, got):
        gmax = s * kpad * 127 * 127 * (2 if cplx else 1)
        c = max(1, (62 - gmax.bit_length()) // 7 + 1)
        assert int(w) == c
        assert gmax * (128 ** c - 1) // 127 <= 2 ** 69 // 127 < 2 ** 63 - 2 ** 57
