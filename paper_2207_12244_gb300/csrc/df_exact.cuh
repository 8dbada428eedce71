// Exact fixed-point sums of floats, the arithmetic behind the persistent
// solvers' reductions (df_sync.cuh): the digits a float contributes, and the
// double-float value of a sum of digits. Host and device code, so that the
// CPU tests can check it against exact rational arithmetic.
//
// A finite float is m 2^(b - 149) with an integer m < 2^24 and 0 <= b <= 253
// (subnormals: b = 0). As an integer in units of 2^-149 it has at most 277
// bits; written in eight 36-bit digits, a float touches at most two
// neighbouring digits. A CTA's double-float partial (two floats) adds less
// than 2^37 to each digit, so the digit sums of up to 1023 CTAs stay below
// 2^47 in magnitude: integer additions of the digits are exact and the order
// in which they happen does not change the total. The value of such a sum is
// below 2^139; totals beyond the float range come out as infinities.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace df {

struct ff2 {
  float hi, lo;
};

DF_HD unsigned int df_float_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned int u;
  memcpy(&u, &f, 4);
  return u;
#endif
}

DF_HD float df_bits_float(unsigned int u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

DF_HD int df_clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

constexpr int kSumDigits = 8;
constexpr int kSumQ = 4;  // quantities per reduction
constexpr long long kDigitMask = (1LL << 36) - 1;
constexpr unsigned long long kDigitBias = 1ull << 37;
constexpr unsigned long long kArrival = 1ull << 48;

// Digit k of a finite float's fixed-point value (signed, |d| < 2^36).
DF_HD long long float_digit(float f, int k) {
  const unsigned int u = df_float_bits(f);
  const int e = (int)((u >> 23) & 0xffu);
  const unsigned int m = e == 0 ? (u & 0x7fffffu) : ((u & 0x7fffffu) | 0x800000u);
  const int b = e == 0 ? 0 : e - 1;  // f = m 2^(b - 149)
  const int kf = b / 36, s = b - kf * 36;
  const unsigned long long v = (unsigned long long)m << s;  // < 2^59
  long long d = 0;
  if (k == kf) d = (long long)(v & (unsigned long long)kDigitMask);
  if (k == kf + 1) d = (long long)(v >> 36);
  return (u >> 31) ? -d : d;
}

// Digit k of what one CTA adds for its double-float partial t: the digits of
// both floats. A finite partial adds less than 2^26 to digit 7 (its floats
// are below 2^129); a non-finite one adds 2^37 - 2^26 there instead, so the
// digit-7 sum of up to 1023 CTAs is below 2^36 exactly when every partial
// was finite.
constexpr long long kNonFiniteMark = (1LL << 37) - (1LL << 26);
DF_HD long long ff_digit(ff2 t, int k) {
  const bool finite = ((df_float_bits(t.hi) >> 23) & 0xffu) != 0xffu &&
                      ((df_float_bits(t.lo) >> 23) & 0xffu) != 0xffu;
  if (!finite) return k == 7 ? kNonFiniteMark : 0;
  return float_digit(t.hi, k) + float_digit(t.lo, k);
}

// x 2^p for an integer-valued float x < 2^24, p in [-200, 127]: exact unless
// the result leaves the normal range.
DF_HD float scale_pow2(float x, int p) {
  if (p < -126) {
    x *= df_bits_float((unsigned int)(p + 126 + 127) << 23);
    p = -126;
  }
  return x * df_bits_float((unsigned int)(p + 127) << 23);
}

// The double-float of a fixed-point magnitude in normalised digits (each in
// [0, 2^36)) whose leading non-zero digit is d2 = digit K, with d1, d0 the
// two digits below it (0 where K < 1, 2), negated if neg; truncated after 48
// significant bits.
DF_HD ff2 leading_to_ff(int K, unsigned long long d2, unsigned long long d1,
                        unsigned long long d0, bool neg) {
  // the 64 bits below and at the leading one of d2 2^72 + d1 2^36 + d0
  const int lz = df_clz64(d2) - 28;  // leading zeros in the 36-bit digit
  unsigned long long w = d2 << (28 + lz);
  const int s1 = lz - 8;
  w |= s1 >= 0 ? (d1 << s1) : (d1 >> -s1);
  w |= d0 >> (44 - lz);
  const int e63 = 36 * K + 35 - lz - 149;  // the leading one is 2^e63
  float hi = scale_pow2((float)(unsigned int)(w >> 40), e63 - 23);
  float lo = scale_pow2((float)(unsigned int)((w >> 16) & 0xffffffull), e63 - 47);
  if (neg) {
    hi = -hi;
    lo = -lo;
  }
  return ff2{hi, lo};
}

// The fixed-point total (raw digit sums dg[0..7], each |dg| < 2^47) as a
// double-float, truncated after 48 significant bits. A digit-7 sum of 2^36
// or more marks a non-finite partial: the total is then NaN.
DF_HD ff2 digits_to_ff(const long long (&raw)[kSumDigits]) {
  if (raw[7] >= (1LL << 36)) return ff2{df_bits_float(0x7fc00000), df_bits_float(0x7fc00000)};
  long long dg[kSumDigits];
  long long c = 0;
#pragma unroll
  for (int k = 0; k < kSumDigits; ++k) {
    const long long t = raw[k] + c;
    dg[k] = t & kDigitMask;
    c = t >> 36;  // arithmetic: floor
  }
  // value = c 2^288 + sum dg[k] 2^(36 k); c = 0 or -1 unless the value is
  // beyond 2^139 (float overflow either way)
  if (c > 0) return ff2{df_bits_float(0x7f800000), 0.0f};
  if (c < -1) return ff2{df_bits_float(0xff800000), 0.0f};
  const bool neg = c < 0;
  if (neg) {  // two's complement: -N = sum (mask - dg[k]) 2^(36 k) + 1
    long long cc = 1;
#pragma unroll
    for (int k = 0; k < kSumDigits; ++k) {
      const long long t = (kDigitMask - dg[k]) + cc;
      dg[k] = t & kDigitMask;
      cc = t >> 36;
    }
  }
  int K = -1;
  unsigned long long d2 = 0, d1 = 0, d0 = 0;
#pragma unroll
  for (int k = 0; k < kSumDigits; ++k) {
    if (dg[k] != 0) {
      K = k;
      d2 = (unsigned long long)dg[k];
      d1 = k >= 1 ? (unsigned long long)dg[k - 1] : 0ull;
      d0 = k >= 2 ? (unsigned long long)dg[k - 2] : 0ull;
    }
  }
  if (K < 0) return ff2{0.0f, 0.0f};
  return leading_to_ff(K, d2, d1, d0, neg);
}

}  // namespace df
