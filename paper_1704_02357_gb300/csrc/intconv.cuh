// Round to nearest, ties to even, between FP64 / FP32 and 64-bit integers with integer
// instructions only, and the exponent test of a paint grid coordinate. On GB300 the conversion
// instructions between floating point and 64-bit integers, and FP64 compares, run on the narrow
// FP64 pipe; the paint's tile prep and per-tile sums were bound by it. The functions compile for
// the device (the paint kernels) and for the host (a CPU test checks them against the C
// library), so they include nothing from CUDA.
#pragma once
#include <cstring>

#ifndef __CUDACC__
#define PSPEC_HD inline
#else
#define PSPEC_HD __host__ __device__ __forceinline__
#endif

namespace pspec {

PSPEC_HD unsigned long long ic_bits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}
PSPEC_HD unsigned ic_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}
PSPEC_HD float ic_float(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
#endif
}
// leading zeros of a nonzero 64-bit value
PSPEC_HD int ic_clz64(unsigned long long a) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return __builtin_clzll(a);
#endif
}

// True when |t| < 2^(max_log2) (NaN and infinities fail): the biased exponent is below
// 1023 + max_log2.
PSPEC_HD bool exp_below(double t, int max_log2) { return (int)((ic_bits(t) >> 52) & 0x7ff) < 1023 + max_log2; }

// round to nearest, ties to even, of a finite double with |t| < 2^62
PSPEC_HD long long d2ll_rn_int(double t) {
  const unsigned long long b = ic_bits(t);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;  // 53 bits
  long long q;
  if (e >= 1075) {
    q = (long long)(m << (e - 1075));  // integral; shift <= 9
  } else if (e < 1022) {
    q = 0;  // |t| < 1/2
  } else {
    const int sh = 1075 - e;  // 1..53
    const unsigned long long r = m >> sh, rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    q = (long long)(r + (unsigned long long)((rem > half) | ((rem == half) & (r & 1ull))));
  }
  return (b >> 63) ? -q : q;
}

// round to nearest, ties to even, of a finite float with |f| < 2^62
PSPEC_HD long long f2ll_rn_int(float f) {
  const unsigned b = ic_bits(f);
  const int e = (int)((b >> 23) & 0xffu);
  const unsigned m = (b & 0x7fffffu) | 0x800000u;  // 24 bits
  long long q;
  if (e >= 150) {
    q = (long long)((unsigned long long)m << (e - 150));  // integral; shift <= 38
  } else if (e < 126) {
    q = 0;  // |f| < 1/2, zero and subnormals included
  } else {
    const int sh = 150 - e;  // 1..24
    const unsigned r = m >> sh, rem = m & ((1u << sh) - 1u), half = 1u << (sh - 1);
    q = (long long)(r + (unsigned)((rem > half) | ((rem == half) & (r & 1u))));
  }
  return (b >> 31) ? -q : q;
}

// round to nearest, ties to even, of any 64-bit integer to float
PSPEC_HD float ll2f_rn_int(long long x) {
  if (x == 0) return 0.f;
  const unsigned sgn = x < 0 ? 0x80000000u : 0u;
  const unsigned long long a = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
  const int nb = 64 - ic_clz64(a);  // a in [2^(nb-1), 2^nb)
  unsigned long long r;
  int e = nb - 1;
  if (nb <= 24) {
    r = a << (24 - nb);
  } else {
    const int sh = nb - 24;
    const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    r = a >> sh;
    r += (unsigned long long)((rem > half) | ((rem == half) & (r & 1ull)));
    if (r == (1ull << 24)) {  // rounded up to the next power of two
      r >>= 1;
      e++;
    }
  }
  return ic_float(sgn | ((unsigned)(e + 127) << 23) | ((unsigned)r & 0x7fffffu));
}

}  // namespace pspec
