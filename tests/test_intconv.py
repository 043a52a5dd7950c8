"""The paint's integer conversions (csrc/intconv.cuh), compiled for the host with g++ from the
same header the kernels include, against the C library's round-to-nearest-even conversions:
double -> int64 and float -> int64 below 2^62, int64 -> float over the whole range, and the
exponent test that decides a grid coordinate's validity (|t| < 2^62), over edge values (ties,
subnormals, the bounds, NaN and infinities) and seeded random bit patterns."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1704_02357_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "intconv.cuh"
using namespace pspec;
static float bitsf(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static double bitsd(unsigned long long u) { double d; std::memcpy(&d, &u, 8); return d; }
int main() {
  std::mt19937_64 g(7);
  long long bad = 0, n = 0;
  const double lim = 4611686018427387904.0;  // 2^62
  const float fedge[] = {0.f, -0.f, 0.5f, -0.5f, 1.5f, 2.5f, -2.5f, 0.49999997f, 1e-40f, -1e-40f,
                         8388607.5f, 8388608.5f, 16777215.f, 4.6e18f, -4.6e18f};
  for (float f : fedge) { n++; bad += f2ll_rn_int(f) != llrintf(f); }
  for (int i = 0; i < 2000000; i++) {
    const unsigned b = ((unsigned)(g() & 1) << 31) | ((unsigned)(g() % 190) << 23) | (unsigned)(g() & 0x7fffff);
    const float f = bitsf(b);
    if (!(std::fabs(f) < 4.6e18f)) continue;
    n++; bad += f2ll_rn_int(f) != llrintf(f);
  }
  const long long ledge[] = {1, -1, 16777215, 16777216, 16777217, 16777218, 16777219, 33554431,
                             (1ll << 62) - 1, -(1ll << 62), (1ll << 53) + 1, 9223372036854775807ll,
                             -9223372036854775807ll - 1};
  for (long long x : ledge) { n++; bad += ll2f_rn_int(x) != (float)x; }
  for (int i = 0; i < 2000000; i++) {
    long long x = (long long)(g() >> (g() % 64));
    if (g() & 1) x = -x;
    if (i % 7 == 0) x = ((x | (1ll << 40)) & ~((1ll << 16) - 1)) | (1ll << 15);  // exact ties
    n++; bad += ll2f_rn_int(x) != (float)x;
  }
  const double dedge[] = {0.5, 1.5, 2.5, -2.5, -0.5, 0.49999999999999994, 4503599627370495.5,
                          4503599627370496.5, lim, -lim, NAN, INFINITY, -INFINITY};
  for (double t : dedge) {
    const bool ok = std::fabs(t) < lim;
    n++; bad += exp_below(t, 62) != ok || (ok && d2ll_rn_int(t) != llrint(t));
  }
  for (int i = 0; i < 2000000; i++) {
    const unsigned long long b = ((unsigned long long)(g() & 1) << 63) |
                                 ((unsigned long long)(960 + g() % 130) << 52) | (g() & 0xfffffffffffffull);
    const double t = bitsd(b);
    const bool ok = std::fabs(t) < lim;
    n++; bad += exp_below(t, 62) != ok || (ok && d2ll_rn_int(t) != llrint(t));
  }
  std::printf("%lld %lld\n", n, bad);
  return bad != 0;
}
"""


def test_integer_conversions_round_like_the_c_library(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    src = tmp_path / "intconv_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "intconv_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    n, bad = (int(v) for v in out.stdout.split())
    assert n > 5_000_000 and bad == 0 and out.returncode == 0
