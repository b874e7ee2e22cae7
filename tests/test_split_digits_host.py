"""The split's digit extraction, compiled for the host (no GPU).  exponent_from_maxbits, digit_src,
digit_mag and digits_to_half2 (ozg_split_dev.cuh) use integer operations and one exact half2
subtraction, which cuda_fp16.h also provides for the host, so g++ builds the same source.  For
every value x and row maximum m >= |x| the result is compared with the definition of the split
(Sec. 2.2), computed with Python integers: e = frexp exponent of m (0 for m = 0), and the digit
t is sign(x) times the t-th base-2^7 digit of |x| 2^-e (truncation digits), stored as FP16 with
the sign of x also on a zero digit.  Cases: normal, subnormal and zero values, maxima from the
value itself up to 2^130 times larger, subnormal maxima."""
import math
import os
import random
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2503_22875_gb300", "csrc", "ozg_split_dev.cuh")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
T = 18

HARNESS = r"""
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#define __device__
#define __forceinline__ inline
static inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
#include "HEADER"
static_assert(ozg::kMaxPlanes == TPLANES, "planes");
int main() {
  unsigned long long xb, mb;
  while (std::scanf("%llx %llx", &xb, &mb) == 2) {
    const int e = ozg::exponent_from_maxbits(mb);
    const ozg::DigitSrc d = ozg::digit_src(xb, e);
    std::printf("%d", e);
    for (int t = 1; t <= ozg::kMaxPlanes; ++t)
      std::printf(" %04x", ozg::digits_to_half2(ozg::digit_mag(d, t), 0, d.neg) & 0xFFFFu);
    std::printf("\n");
  }
  return 0;
}
"""


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def expected(x, m):
    e = 0 if m == 0 else math.frexp(m)[1]
    M, ex = (0, 0) if x == 0 else (abs(int(math.ldexp(math.frexp(x)[0], 53))), math.frexp(x)[1] - 53)
    out = []
    for t in range(1, T + 1):
        sh = ex - e + 7 * t                    # floor(|x| 2^-e 128^t) = floor(M 2^sh)
        F = M << sh if sh >= 0 else M >> -sh
        dig = F & 127                          # the t-th base-128 digit of |x| 2^-e
        val = -float(dig) if (x < 0 or (x == 0 and math.copysign(1, x) < 0)) else float(dig)
        out.append(int(np.array(val, dtype=np.float16).view(np.uint16)))
    return e, out


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if not os.path.exists(os.path.join(CUDA_INC, "cuda_fp16.h")):
        pytest.skip("cuda_fp16.h not found")
    d = tmp_path_factory.mktemp("digits")
    src = d / "h.cpp"
    src.write_text(HARNESS.replace("HEADER", HEADER).replace("TPLANES", str(T)))
    exe = str(d / "h")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CUDA_INC, str(src), "-o", exe])
    return exe


def test_digits_equal_the_split_definition(harness):
    g = random.Random(21)
    cases = [(0.0, 0.0), (-0.0, 1.0), (1.0, 1.0), (-0.75, 1.5), (5e-324, 5e-324), (-3e-320, 1e-310),
             (2.0 ** -1022, 2.0 ** -1022), (1.0 - 2.0 ** -53, 1.0), (float.fromhex("0x1.fffffffffffffp+1023"),) * 2]
    for _ in range(40000):
        u = g.random()
        if u < 0.1:
            x = g.choice([-1, 1]) * g.randint(1, 2 ** 52 - 1) * 2.0 ** -1074       # subnormal
        else:
            x = g.choice([-1, 1]) * math.ldexp(0.5 + g.random() / 2, g.randint(-1020, 1023))
        if g.random() < 0.05:
            x = 0.0
        gap = 0 if g.random() < 0.2 else g.randint(0, 130)
        m = abs(x) * 2.0 ** gap if abs(x) * 2.0 ** gap < float("inf") else abs(x)
        if m == 0 and g.random() < 0.5:
            m = math.ldexp(1.0, g.randint(-1074, 1000))
        cases.append((x, m))
    inp = "".join(f"{bits(x):x} {bits(m):x}\n" for x, m in cases)
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout.splitlines()
    bad = []
    for (x, m), line in zip(cases, out):
        f = line.split()
        got = (int(f[0]), [int(h, 16) for h in f[1:]])
        if got != expected(x, m):
            bad.append((x, m, got, expected(x, m)))
    assert len(out) == len(cases) and not bad, f"{len(bad)} differ, e.g. {bad[:2]}"
