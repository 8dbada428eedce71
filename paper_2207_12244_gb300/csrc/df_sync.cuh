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
  int vec, th;
  int debug_skip_cta;  // test hook: this CTA leaves without arriving (-1: none)
  unsigned int bar_count, bar_gen, exit_count, abort;
  long long off_cta_tile, off_cta_kf, off_cta_slot, off_kf, off_slots;
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

// Deterministic FP64 sum of this keyframe's slots [sb, se) (kQ values each)
// by one warp: every lane issues all its loads before adding, so the whole
// reduction costs one L2 round trip; lanes add in slot order, then a fixed
// shuffle tree. Result in lane 0.
template <int kQ>
__device__ __forceinline__ void warp_slot_sum(const double *pslots, int sb, int se,
                                              double (&out)[kQ]) {
  const int lane = threadIdx.x & 31;
  constexpr int kU = 8;  // slots per lane loaded at once
  double acc[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) acc[q] = 0.0;
  for (int base = sb; base < se; base += 32 * kU) {
    double v[kU][kQ];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const int sl = base + lane + 32 * j;
#pragma unroll
      for (int q = 0; q < kQ; ++q) v[j][q] = sl < se ? __ldcg(pslots + (size_t)sl * kQ + q) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) {
#pragma unroll
      for (int q = 0; q < kQ; ++q) acc[q] += v[j][q];
    }
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) out[q] = warp_sum(acc[q]);
}

// A CTA's FP32 per-thread partials -> FP64 CTA total (fixed order) in
// thread 0's 'out'. red must hold 32 * kQ floats.
template <int kQ>
__device__ __forceinline__ void cta_partial_sum(const float (&acc)[kQ], float *red,
                                                double (&out)[kQ]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const float s = warp_sum_f(acc[q]);
    if (lane == 0) red[warp * kQ + q] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      double x = lane < nwarps ? (double)red[lane * kQ + q] : 0.0;
      out[q] = warp_sum(x);
    }
  }
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
