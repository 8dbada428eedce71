// Grid-wide synchronisation shared by the persistent solvers: launch-plan
// header, a generation-counting grid barrier whose waits give up after a
// time limit, and the exit protocol that leaves the barrier words clean.
#pragma once

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
  unsigned int bar_count, bar_gen, exit_count, abort;
  // off_cta_work: per-CTA work table (streaming: the G * 8 + 1 warp row
  // starts; resident: one band descriptor per CTA)
  long long off_cta_work, off_cta_kf, off_cta_slot, off_kf, off_slots;
  long long bytes;
  int smem_bytes;  // dynamic shared memory per CTA (resident plans)
  int pad1;
  long long slot_stride;  // doubles per parity of the reduction slots / inboxes
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

// Grid barrier over the G CTAs of one cooperative launch. The arrival
// counter only grows during a launch: the n-th barrier of a CTA waits until
// the counter reaches n * G, so the last arriver has nothing to release and
// the waiters see it one L2 round trip after it lands. Every wait gives up
// after limit_ns; a CTA that gives up (or sees that another one did) raises
// the abort word and returns false, and the caller then skips all remaining
// work. 'epoch' is the CTA's count of barriers passed (shared memory).
__device__ __forceinline__ bool grid_sync(PlanHeader *h, int G, unsigned long long limit_ns,
                                          unsigned int *epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && (int)blockIdx.x == h->debug_skip_cta) {
    s_ok = 0;  // test hook: leave silently, the other CTAs' waits run out
  } else if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int target = (*epoch + 1u) * (unsigned int)G;
    *epoch += 1u;
    __threadfence();  // the CTA's writes (ordered before by __syncthreads) first
    const unsigned int arrived = atomicAdd(&h->bar_count, 1u) + 1u;
    if (arrived < target) {
      const unsigned long long t0 = global_ns();
      unsigned int spins = 0;
      while (ld_acquire(&h->bar_count) < target) {
        if (((++spins) & 63u) == 0u) {
          if (ld_acquire(&h->abort) != 0u || global_ns() - t0 > limit_ns) {
            ok = 0;
            break;
          }
        }
      }
    }
    if (ok && ld_acquire(&h->abort) != 0u) ok = 0;
    if (!ok) atomicExch(&h->abort, 1u);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---- double-float reductions ------------------------------------------------
//
// GB300 executes FP64 adds at about 2 per clock per SM, 64x below FP32, so an
// FP64 shuffle tree over a CTA costs microseconds. The solver's inner
// products are therefore carried as an unevaluated sum of two floats
// (hi + lo, about 44 significant bits) from the warp level up, combined by
// the error-free TwoSum transformation (Knuth / Dekker) in a fixed order, and
// turned into one double per scalar at the very end. All operations are
// FP32 adds, so the reduction is deterministic and as cheap as an FP32 one.
struct ff2 {
  float hi, lo;
};

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

__device__ __forceinline__ double ff_to_double(ff2 a) { return (double)a.hi + (double)a.lo; }

// Reduction slot: kQ double-float values padded to 32 bytes (kQ <= 4).
struct alignas(32) Slot {
  ff2 v[4];
};

// Slots a reader's inbox holds for n writers: padded to whole warps so that
// every lane loads whole slots without bounds checks (padding stays zero).
__host__ __device__ __forceinline__ int inbox_slots(int n) { return (n + 31) & ~31; }

// Sum of one inbox of n writers (slot order, then a fixed warp tree) by one
// warp: every lane issues all its loads before adding. Result in lane 0.
template <int kQ>
__device__ __forceinline__ void warp_inbox_sum(const Slot *box, int n, double (&out)[kQ]) {
  const int lane = threadIdx.x & 31;
  const int np = inbox_slots(n);
  constexpr int kU = 8;
  ff2 acc[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) acc[q] = ff2{0.0f, 0.0f};
  for (int base = 0; base < np; base += 32 * kU) {
    float4 v[kU][2];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const int sl = base + lane + 32 * j;
      const float4 *p = reinterpret_cast<const float4 *>(box + sl);
      if (base + 32 * j < np) {
        v[j][0] = __ldcg(p);
        // slots of one or two sums are written without their second half
        v[j][1] = kQ > 2 ? __ldcg(p + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        v[j][0] = v[j][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const ff2 s[4] = {ff2{v[j][0].x, v[j][0].y}, ff2{v[j][0].z, v[j][0].w},
                        ff2{v[j][1].x, v[j][1].y}, ff2{v[j][1].z, v[j][1].w}};
#pragma unroll
      for (int q = 0; q < kQ; ++q) acc[q] = ff_add(acc[q], s[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) out[q] = ff_to_double(warp_sum_ff(acc[q]));
}

// A CTA's FP32 per-thread partials -> double-float CTA total (fixed order),
// valid in warp 0 lane 0. red must hold 32 * kQ ff2.
template <int kQ>
__device__ __forceinline__ void cta_partial_sum(const float (&acc)[kQ], ff2 *red,
                                                ff2 (&out)[kQ]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const ff2 s = warp_sum_ff(ff2{acc[q], 0.0f});
    if (lane == 0) red[warp * kQ + q] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const ff2 x = lane < nwarps ? red[lane * kQ + q] : ff2{0.0f, 0.0f};
      out[q] = warp_sum_ff(x);
    }
  }
}

// As cta_partial_sum, with the second level split over warps: warp q adds
// quantity q (same order, same result), so the kQ trees run side by side.
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

// One quantity q of an inbox of n writers, summed by one warp in the order of
// warp_inbox_sum (slot order per lane, then a fixed warp tree).
__device__ __forceinline__ double warp_inbox_sum_q(const Slot *box, int n, int q) {
  const int lane = threadIdx.x & 31;
  const int np = inbox_slots(n);
  constexpr int kU = 8;
  ff2 acc = ff2{0.0f, 0.0f};
  for (int base = 0; base < np; base += 32 * kU) {
    float2 v[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const int sl = base + lane + 32 * j;
      v[j] = (base + 32 * j < np) ? __ldcg(reinterpret_cast<const float2 *>(&box[sl].v[q]))
                                  : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) acc = ff_add(acc, ff2{v[j].x, v[j].y});
  }
  return ff_to_double(warp_sum_ff(acc));
}

// Called once by every CTA as its last action: the last CTA out resets the
// barrier words (also after an abort, since every CTA does exit).
__device__ __forceinline__ void grid_exit(PlanHeader *h, int G) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int done = atomicAdd(&h->exit_count, 1u) + 1u;
    if (done == (unsigned int)G) {
      h->bar_count = 0u;
      h->abort = 0u;
      h->exit_count = 0u;
      __threadfence();
    }
  }
}

}  // namespace df
