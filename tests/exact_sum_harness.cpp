// Host harness for the exact-sum arithmetic of the persistent solvers
// (paper_2207_12244_gb300/csrc/df_exact.cuh), built by tests/test_exact_sum.py
// with the host compiler: n double-float partials (hi, lo pairs) are turned
// into digits and summed exactly as the CTAs' additions do, then converted.
#include "df_exact.cuh"

extern "C" void exact_total(const float *pairs, int n, float *out) {
  long long raw[df::kSumDigits] = {0};
  for (int i = 0; i < n; ++i) {
    const df::ff2 t{pairs[2 * i], pairs[2 * i + 1]};
    for (int k = 0; k < df::kSumDigits; ++k) raw[k] += df::ff_digit(t, k);
  }
  const df::ff2 r = df::digits_to_ff(raw);
  out[0] = r.hi;
  out[1] = r.lo;
}

// digit k of one float (for the digit layout checks)
extern "C" long long float_digit_of(float f, int k) { return df::float_digit(f, k); }

// The solvers' sum_total resolves the carries across the 8 lanes of a group
// in rounds (df_sync.cuh carry_rounds); this is the same procedure with the
// lanes as an array, to check it against digits_to_ff on the host.
static long long rounds(long long d[8]) {
  long long c8 = 0;
  for (;;) {
    long long c[8];
    for (int k = 0; k < 8; ++k) {
      c[k] = d[k] >> 36;
      d[k] &= df::kDigitMask;
    }
    for (int k = 1; k < 8; ++k) d[k] += c[k - 1];
    c8 += c[7];
    bool more = false;
    for (int k = 0; k < 8; ++k) more = more || (d[k] >> 36) != 0;
    if (!more) return c8;
  }
}

extern "C" void total_by_rounds(const long long *raw, float *out) {
  long long d[8];
  for (int k = 0; k < 8; ++k) d[k] = raw[k];
  const bool nonfinite = raw[7] >= (1LL << 36);
  const long long top = rounds(d);
  const bool neg = top == -1;
  if (neg)
    for (int k = 0; k < 8; ++k) d[k] = (df::kDigitMask - d[k]) + (k == 0 ? 1 : 0);
  rounds(d);
  int K = -1;
  for (int k = 0; k < 8; ++k)
    if (d[k] != 0) K = k;
  df::ff2 r;
  if (nonfinite) {
    r = df::ff2{__builtin_nanf(""), __builtin_nanf("")};
  } else if (top > 0) {
    r = df::ff2{__builtin_inff(), 0.0f};
  } else if (top < -1) {
    r = df::ff2{-__builtin_inff(), 0.0f};
  } else if (K < 0) {
    r = df::ff2{0.0f, 0.0f};
  } else {
    r = df::leading_to_ff(K, (unsigned long long)d[K], K >= 1 ? (unsigned long long)d[K - 1] : 0ull,
                          K >= 2 ? (unsigned long long)d[K - 2] : 0ull, neg);
  }
  out[0] = r.hi;
  out[1] = r.lo;
}

extern "C" void total_sequential(const long long *raw, float *out) {
  long long d[8];
  for (int k = 0; k < 8; ++k) d[k] = raw[k];
  const df::ff2 r = df::digits_to_ff(d);
  out[0] = r.hi;
  out[1] = r.lo;
}
