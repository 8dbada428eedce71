// Synchronisation shared by the persistent solvers: launch-plan header,
// double-float arithmetic, the exact per-keyframe sums whose words also
// order the passes (their waits give up after a time limit), and the exit
// protocol that leaves the words clean for the next launch.
#pragma once

#include "df_exact.cuh"
#include "df_internal.cuh"

namespace df {

// Kinds of launch plans (PlanHeader::kind).
enum : int { kPlanStreaming = 0, kPlanResident = 1 };

struct PlanHeader {
  int kind;        // kPlanStreaming / kPlanResident
  int nkf, G, ntiles, nslots;
  int vec;
  int th;  // streaming: longest piece a warp walks at once (0: no limit);
           // resident: shared-memory stride of a band array
  int debug_skip_cta;  // test hook: this CTA leaves without arriving (-1: none)
  unsigned int bar_count, bar_gen, exit_count, abort;  // bar_*: unused (zero)
  // off_slots: the plan's exact-sum groups, one SumGroup per keyframe
  // off_cta_work: per-CTA work table (streaming: the G * 8 + 1 warp row
  // starts; resident: one band descriptor per CTA)
  long long off_cta_work, off_cta_kf, off_cta_slot, off_kf, off_slots;
  long long bytes;
  int smem_bytes;  // dynamic shared memory per CTA (resident plans)
  int in_smem;     // resident plans: 1 = each band's input planes are staged
                   // in shared memory for the whole launch
  long long off_flags;  // resident plans: the CTAs' edge flags (four words
                        // per CTA, the first used) right after the sum
                        // groups; 0 in streaming plans
  int asm_pieces;  // streaming plans: pieces of the separate assembly kernel
  int asm_pad;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---- double-float reductions ------------------------------------------------
//
// GB300 executes FP64 adds at about 2 per clock per SM, 64x below FP32, so an
// FP64 shuffle tree over a CTA costs microseconds. The solver's inner
// products are therefore carried as an unevaluated sum of two floats
// (hi + lo, about 44 significant bits) from the warp level up, combined by
// the error-free TwoSum transformation (Knuth / Dekker) in a fixed order; the
// totals stay double-float for the CG scalars and become doubles only where
// an FP64 value is stored or reported. All operations are FP32 adds, so the
// reduction is deterministic and as cheap as an FP32 one.
__device__ __forceinline__ ff2 ff_add(ff2 a, ff2 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return ff2{hi, e - (hi - s)};
}

__device__ __forceinline__ ff2 ff_shfl_down(ff2 a, int o) {
  return ff2{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

// fixed-order warp tree; result in lane 0
__device__ __forceinline__ ff2 warp_sum_ff(ff2 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = ff_add(a, ff_shfl_down(a, o));
  return a;
}

// NQ fixed-order warp trees side by side, level by level, so that their
// shuffle and add latencies overlap (each tree's arithmetic is warp_sum_ff's);
// results in lane 0
template <int NQ>
__device__ __forceinline__ void warp_sum_ff_n(ff2 (&a)[NQ]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ff2 t[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = ff_shfl_down(a[q], o);
#pragma unroll
    for (int q = 0; q < NQ; ++q) a[q] = ff_add(a[q], t[q]);
  }
}

__device__ __forceinline__ double ff_to_double(ff2 a) { return (double)a.hi + (double)a.lo; }

// ---- double-float scalar arithmetic -----------------------------------------
//
// The CG scalars (gamma = r.z, alpha, beta, and p.Ap = delta - beta gamma /
// alpha_prev) are formed from the double-float sums above by one thread
// between two CTA barriers, so their latency is on every pass's critical
// path. On GB300 a dependent FP64 operation takes ~64 cycles and an FP64
// division ~550, so three divisions cost ~0.8 us per pass. The same
// quantities in double-float arithmetic (Dekker, "A floating-point technique
// for extending the available precision", Numer. Math. 18, 1971: the exact
// product of two floats by one fused multiply-add, and the double-length
// quotient q1 + q2 with q2 the correction from the exact remainder) take a
// few FP32 operations each and keep ~44 significant bits, the precision of
// the sums they come from.

// a + b for |a| >= |b| (or a == 0), exactly as hi + lo
__device__ __forceinline__ ff2 ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  return ff2{s, b - (s - a)};
}

__device__ __forceinline__ ff2 ff_neg(ff2 a) { return ff2{-a.hi, -a.lo}; }

__device__ __forceinline__ ff2 ff_sub(ff2 a, ff2 b) { return ff_add(a, ff_neg(b)); }

// a * b: the float product and its exact rounding error (fma), plus the
// cross terms of the low parts
__device__ __forceinline__ ff2 ff_mul(ff2 a, ff2 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}

// a / b: q1 from the hardware reciprocal of b.hi, the remainder a - q1 b with
// q1 b.hi split exactly, q2 = remainder / b.hi. b.hi must be finite and
// non-zero (callers test the denominator's sign first).
__device__ __forceinline__ ff2 ff_div(ff2 a, ff2 b) {
  const float rb = __fdividef(1.0f, b.hi);
  const float q1 = a.hi * rb;
  const float p = q1 * b.hi;
  const float pe = fmaf(q1, b.hi, -p);
  const float r = (((a.hi - p) - pe) + a.lo) - q1 * b.lo;
  return ff_fast_two_sum(q1, r * rb);
}

// a double as hi + lo (for the FP64 values of the joint solve's border)
__device__ __forceinline__ ff2 ff_from_double(double d) {
  const float hi = (float)d;
  return ff2{hi, (float)(d - (double)hi)};
}

// A CTA's sums of one keyframe segment: up to four double-float values.
struct alignas(32) Slot {
  ff2 v[4];
};

// A CTA's FP32 per-thread partials -> double-float CTA totals in a fixed
// order: a warp tree per quantity, then warp q adds quantity q over the warps
// (the kQ second-level trees run side by side).
// The totals land in shared memory out[0..kQ-1] (valid after the caller's
// next __syncthreads).
template <int kQ>
__device__ __forceinline__ void cta_partial_sum_split(const float (&acc)[kQ], ff2 *red,
                                                      ff2 *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const ff2 s = warp_sum_ff(ff2{acc[q], 0.0f});
    if (lane == 0) red[warp * kQ + q] = s;
  }
  __syncthreads();
  if (warp < kQ) {
    const ff2 x = lane < nwarps ? red[lane * kQ + warp] : ff2{0.0f, 0.0f};
    const ff2 t = warp_sum_ff(x);
    if (lane == 0) out[warp] = t;
  }
}

// ---- exact sums over the CTAs of a keyframe, without a grid barrier ---------
//
// Each CTA's double-float partial of a quantity is added, exactly, into a
// fixed-point integer whose unit is 2^-149 (the smallest float step), kept as
// eight 36-bit digits. Every finite float is m 2^(b - 149) with m < 2^24 and
// 0 <= b <= 253, so it lands in at most two neighbouring digits; integer
// addition is associative, so the total does not depend on the order in
// which the CTAs arrive and every reader gets the same bits (df_exact.cuh:
// up to 1023 CTAs per keyframe).
//
// Each digit lives in a 64-bit word that also counts its own arrivals: a
// CTA adds (digit + 2^37) + 2^48 with one red.add per word, so bits 0..47
// hold the biased digit sum and bits 48..63 the number of CTAs added so far.
// A reader polls the words of a quantity until every word shows all n
// arrivals; it needs no barrier word, and no word waits for another. The
// words are never cleared during a launch: each CTA remembers the value at
// which a word last completed and works with the difference (modulo 2^64).
// Two sets alternate between consecutive reductions; a CTA can reach the
// reduction after next on a set only after every CTA has contributed to the
// next one, that is, after every CTA has read this one. Before its adds a
// CTA fences, so everything it wrote in the pass (the band or tile edges its
// neighbours read next) is visible to whoever sees its arrival.
// Two quantities of one set share a 128-byte line, eight digit words each
// (a warp's adds and loads of two quantities are one request each; fewer
// lines polled and added to by all the keyframe's CTAs measured faster,
// spreading the words over eight lines per quantity slower).
struct alignas(128) SumLine {
  unsigned long long w[16];
};
// The reduction words of one keyframe: [set][quantity pair].
struct SumGroup {
  SumLine line[2][(kSumQ + 1) / 2];
};
__device__ __forceinline__ unsigned long long *sum_word(SumGroup *g, int set, int q, int k) {
  return &g->line[set][q >> 1].w[((q & 1) << 3) + k];
}
// What a CTA remembers of a group's words (shared memory).
struct SumPrev {
  unsigned long long v[2][kSumQ][kSumDigits];
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Release / acquire fence at GPU scope (lighter than the sequentially
// consistent __threadfence): before relaxed adds it makes them a release,
// after relaxed loads an acquire.
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Warp-collective (one whole warp): fence, then add the nq (1..4) totals
// tot[] of this CTA into set 'set' of group g (lane q * 8 + k adds digit k
// of quantity q).
__device__ __forceinline__ void sum_push(SumGroup *g, int set, const ff2 *tot, int nq,
                                         bool fence = true) {
  const int lane = threadIdx.x & 31;
  if (fence) fence_acq_rel_gpu();  // (a caller that fenced already passes false)
  if (lane < 8 * nq) {
    const int q = lane >> 3, k = lane & 7;
    const long long d = ff_digit(tot[q], k);
    red_add_u64(sum_word(g, set, q, k), (unsigned long long)(d + (long long)kDigitBias) + kArrival);
  }
}

// Warp-collective (one whole warp): add digits d[q][k] (k < 8, q < nq) that
// the CTA formed already (ff_digit of its totals); the caller has fenced.
__device__ __forceinline__ void sum_push_digits(SumGroup *g, int set, const long long (*d)[kSumDigits],
                                                int nq) {
  const int lane = threadIdx.x & 31;
  if (lane < 8 * nq) {
    const int q = lane >> 3, k = lane & 7;
    red_add_u64(sum_word(g, set, q, k), (unsigned long long)(d[q][k] + (long long)kDigitBias) + kArrival);
  }
}

// Warp-collective: wait until all n CTAs have added their nq quantities to
// set 'set' of g (every lane q * 8 + k < 8 nq polls its own word with an
// acquire load: one request per line of two quantities and spin). Returns false if
// the wait ran past limit_ns or another CTA raised the abort word (and then
// raises it too). On success each lane q * 8 + k < 8 nq holds digit k of
// quantity q in *digit, prev is updated, and the warp has acquired what the
// other CTAs wrote before their adds.
__device__ __forceinline__ bool sum_wait(SumGroup *g, int set, int n, int nq, SumPrev *prev,
                                         PlanHeader *h, unsigned long long limit_ns,
                                         long long *digit) {
  const int lane = threadIdx.x & 31;
  const bool act = lane < 8 * nq;
  const int q = lane >> 3, k = lane & 7;
  const unsigned long long *wp = act ? sum_word(g, set, q, k) : nullptr;
  const unsigned long long pv = act ? prev->v[set][q][k] : 0ull;
  unsigned long long v = 0ull;
  const unsigned long long t0 = global_ns();
  unsigned int spins = 0;
  bool ok = true;
  for (;;) {
    bool done = true;
    if (act) {
      v = ld_acquire_u64(wp);
      done = ((v - pv) >> 48) == (unsigned long long)n;
    }
    if (__all_sync(0xffffffffu, done)) break;
    if (((++spins) & 63u) == 0u) {
      int bad = 0;
      if (lane == 0) bad = (ld_acquire(&h->abort) != 0u || global_ns() - t0 > limit_ns) ? 1 : 0;
      if (__shfl_sync(0xffffffffu, bad, 0)) {
        ok = false;
        break;
      }
    }
  }
  if (!ok) {
    if (lane == 0) atomicExch(&h->abort, 1u);
    return false;
  }
  if (act) {
    prev->v[set][q][k] = v;
    *digit = (long long)((v - pv) & (kArrival - 1ull)) - (long long)n * (long long)kDigitBias;
  }
  return true;
}

// Edge hand-off between neighbouring bands without a reduction: after its
// edge stores (and a barrier of its CTA), one thread raises the CTA's flag
// to epoch e; fence first, so that whoever sees e sees the edges.
__device__ __forceinline__ void edge_flag_raise(unsigned long long *f, unsigned long long e) {
  fence_acq_rel_gpu();
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(f), "l"(e) : "memory");
}

// Warp-collective (one whole warp): lanes with a non-null p wait until *p
// reaches e (acquire loads). Bounded like sum_wait: false (abort raised)
// once limit_ns has passed or another CTA raised the abort word.
__device__ __forceinline__ bool edge_flags_wait(const unsigned long long *p, unsigned long long e,
                                                PlanHeader *h, unsigned long long limit_ns) {
  const int lane = threadIdx.x & 31;
  const unsigned long long t0 = global_ns();
  unsigned int spins = 0;
  for (;;) {
    const bool done = p == nullptr || ld_acquire_u64(p) >= e;
    if (__all_sync(0xffffffffu, done)) return true;
    if (((++spins) & 63u) == 0u) {
      int bad = 0;
      if (lane == 0) bad = (ld_acquire(&h->abort) != 0u || global_ns() - t0 > limit_ns) ? 1 : 0;
      if (__shfl_sync(0xffffffffu, bad, 0)) {
        if (lane == 0) atomicExch(&h->abort, 1u);
        return false;
      }
    }
  }
}

// Carry rounds over the 8-lane digit groups of a warp: each round keeps the
// low 36 bits of every digit and adds the carry of the digit below it (lane
// k - 1 of the group); the carry out of digit 7 goes to *c8 (lane 7). Rounds
// repeat until every digit of every group is in [0, 2^36).
__device__ __forceinline__ long long carry_rounds(long long d, long long *c8) {
  const int k = threadIdx.x & 7;
  for (;;) {
    const long long c = d >> 36;  // floor(d / 2^36)
    d &= kDigitMask;
    const long long cin = __shfl_up_sync(0xffffffffu, c, 1);
    if (k > 0) d += cin;
    if (k == 7) *c8 += c;
    if (!__any_sync(0xffffffffu, (d >> 36) != 0)) return d;
  }
}

// Warp-collective after sum_wait: every lane of the group of quantity q
// (lanes 8 q .. 8 q + 7) returns its total. The same value as digits_to_ff
// of the group's raw digit sums (the normalised digits of an integer are
// unique), with the carries resolved across the group's lanes in a few
// rounds instead of one digit after another.
__device__ __forceinline__ ff2 sum_total(long long digit) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, k = lane & 7, base = lane & ~7;
  const bool nonfinite = __shfl_sync(full, digit, base + 7) >= (1LL << 36);
  long long c8 = 0;
  long long d = carry_rounds(digit, &c8);
  const long long top = __shfl_sync(full, c8, base + 7);  // 0 or -1 unless beyond 2^139
  const bool neg = top == -1;
  // two's complement of negative totals: -N = sum (mask - d_k) 2^(36 k) + 1
  if (neg) d = (kDigitMask - d) + (k == 0 ? 1 : 0);
  long long c8n = 0;
  d = carry_rounds(d, &c8n);
  const unsigned gm = (__ballot_sync(full, d != 0) >> base) & 0xffu;
  const int K = gm ? 31 - __clz(gm) : 0;
  const unsigned long long d2 = (unsigned long long)__shfl_sync(full, d, base + K);
  const unsigned long long d1 = (unsigned long long)__shfl_sync(full, d, base + (K >= 1 ? K - 1 : 0));
  const unsigned long long d0 = (unsigned long long)__shfl_sync(full, d, base + (K >= 2 ? K - 2 : 0));
  if (nonfinite) return ff2{__int_as_float(0x7fc00000), __int_as_float(0x7fc00000)};
  if (top > 0) return ff2{__int_as_float(0x7f800000), 0.0f};
  if (top < -1) return ff2{__int_as_float((int)0xff800000u), 0.0f};
  if (gm == 0) return ff2{0.0f, 0.0f};
  return leading_to_ff(K, d2, K >= 1 ? d1 : 0ull, K >= 2 ? d0 : 0ull, neg);
}

// Called once by every CTA as its last action: the last CTA out resets the
// abort and exit words (also after an abort, since every CTA does exit), and clears
// n_sum words of exact-sum groups at 'sums' (nullptr: none).
__device__ __forceinline__ void grid_exit(PlanHeader *h, int G, unsigned long long *sums = nullptr,
                                          long long n_sum = 0) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int done = atomicAdd(&h->exit_count, 1u) + 1u;
    s_last = done == (unsigned int)G ? 1 : 0;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (long long i = threadIdx.x; i < n_sum; i += blockDim.x) sums[i] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
      h->bar_count = 0u;
      h->abort = 0u;
      h->exit_count = 0u;
      __threadfence();
    }
  }
}

}  // namespace df
