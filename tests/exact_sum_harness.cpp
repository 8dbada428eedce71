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
