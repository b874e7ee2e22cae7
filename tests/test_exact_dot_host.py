"""The sampled check's exact dot product (ozg_exactdot.cuh), compiled for the host (no GPU).  The
header uses integer, conversion and plain FP64 operations only, so with a host __umul64hi g++
builds the same source.  The harness accumulates the terms in 32 lane accumulators (as the
warp's lanes split k) and combines them with i128_add, as the warp reduction does.  Against
Python integers: the 128-bit sum equals sum_l sign(a_l b_l) floor(|a_l b_l| / 2^unit) with
unit = e + f - 100 (e, f the frexp exponents of max |a| and max |b|, as the split gives them),
the double-double result equals that sum times 2^unit to within 2^-104 relative, and the sum is
within k units of the exact dot product.  Cases: wide exponent spreads, signed zeros, exact
cancellation, subnormal factors."""
import math
import os
import random
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2503_22875_gb300", "csrc", "ozg_exactdot.cuh")

HARNESS = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#define __device__
#define __forceinline__ inline
static inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
#include "HEADER"
static unsigned long long b64(double v) { unsigned long long b; std::memcpy(&b, &v, 8); return b; }
int main() {
  int k, unit;
  while (std::scanf("%d %d", &k, &unit) == 2) {
    ozg::i128 lane[32];
    for (int i = 0; i < 32; ++i) lane[i] = {0ull, 0ll};
    for (int l = 0; l < k; ++l) {
      unsigned long long a, b;
      if (std::scanf("%llx %llx", &a, &b) != 2) return 1;
      ozg::add_exact_term(lane[l % 32], a, b, unit);
    }
    for (int o = 16; o > 0; o >>= 1)
      for (int i = 0; i < 32; ++i)
        if ((i & o) == 0) { ozg::i128 t = lane[i ^ o]; ozg::i128_add(lane[i], t); lane[i ^ o] = lane[i]; }
    const ozg::dd r = ozg::i128_to_dd(lane[0], unit);
    std::printf("%llx %llx %016llx %016llx\n", (unsigned long long)lane[0].hi, lane[0].lo, b64(r.hi), b64(r.lo));
  }
  return 0;
}
"""


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def unbits(h):
    return struct.unpack("<d", struct.pack("<Q", int(h, 16)))[0]


def split_parts(x):
    """|x| = M 2^X with M an integer (the significand, subnormals included)."""
    if x == 0:
        return 0, 0
    m, e = math.frexp(abs(x))
    return int(m * 2 ** 53), e - 53


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("exactdot")
    src = d / "h.cpp"
    src.write_text(HARNESS.replace("HEADER", HEADER))
    exe = str(d / "h")
    subprocess.check_call(["g++", "-O2", "-std=c++17", str(src), "-o", exe])
    return exe


def vector(g, k, phi, base):
    out = []
    for _ in range(k):
        u = g.random()
        if u < 0.05:
            out.append(0.0 if g.random() < 0.5 else -0.0)
        else:
            out.append(g.choice([-1, 1]) * (0.5 + g.random() / 2) * math.exp(phi * g.gauss(0, 1)) * 2.0 ** base)
    return out


def test_exact_dot_equals_the_truncated_integer_sum(harness):
    g = random.Random(31)
    cases = []
    for c in range(300):
        k = g.choice([1, 2, 31, 32, 33, 100, 1000, 3000])
        phi = g.choice([0.0, 1.0, 4.0, 8.0])
        a, b = vector(g, k, phi, g.randint(-300, 300)), vector(g, k, phi, g.randint(-300, 300))
        if c % 10 == 0:           # exact cancellation: the second half negates the first
            a = a[: k // 2] + [-x for x in a[: k // 2]] + a[2 * (k // 2):]
            b = b[: k // 2] + b[: k // 2] + b[2 * (k // 2):]
        elif c % 10 == 1:         # subnormal a (and b near 2^600, so that the products are normal)
            a = [g.choice([-1, 1]) * g.randint(0, 2 ** 52 - 1) * 2.0 ** -1074 for _ in range(k)]
            b = vector(g, k, phi, 600)
        ma, mb = max(abs(x) for x in a), max(abs(x) for x in b)
        e = math.frexp(ma)[1] if ma else 0
        f = math.frexp(mb)[1] if mb else 0
        cases.append((a, b, e + f - 100))
    inp = "".join(f"{len(a)} {unit}\n" + "".join(f"{bits(x):x} {bits(y):x}\n" for x, y in zip(a, b))
                  for a, b, unit in cases)
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout.splitlines()
    assert len(out) == len(cases)
    for (a, b, unit), line in zip(cases, out):
        hi, lo, rh, rl = line.split()
        acc = (int(hi, 16) << 64 | int(lo, 16))
        acc = acc - 2 ** 128 if acc >= 2 ** 127 else acc
        S, exact = 0, Fraction(0)
        for x, y in zip(a, b):
            (mx, ex), (my, ey) = split_parts(x), split_parts(y)
            sh = ex + ey - unit
            t = mx * my << sh if sh >= 0 else (mx * my) >> -sh
            S += t if (x < 0) == (y < 0) else -t
            exact += Fraction(x) * Fraction(y)
        assert acc == S
        val = Fraction(S) * Fraction(2) ** unit
        got = Fraction(unbits(rh)) + Fraction(unbits(rl))
        assert abs(got - val) <= abs(val) * Fraction(1, 2 ** 104)
        assert abs(val - exact) <= len(a) * Fraction(2) ** unit
