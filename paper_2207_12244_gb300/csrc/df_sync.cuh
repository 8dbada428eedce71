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

// Grid barrier over the G CTAs of one cooperative launch. Every wait gives up
// after limit_ns; a CTA that gives up (or sees that another one did) raises
// the abort word and returns false, and the caller then skips all remaining
// work. The last arriver resets the count before it bumps the generation.
__device__ __forceinline__ bool grid_sync(PlanHeader *h, int G, unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && (int)blockIdx.x == h->debug_skip_cta) {
    s_ok = 0;  // test hook: leave silently, the other CTAs' waits run out
  } else if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int gen = ld_acquire(&h->bar_gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(&h->bar_count, 1u) + 1u;
    if (arrived == (unsigned int)G) {
      h->bar_count = 0u;
      __threadfence();
      atomicAdd(&h->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned int spins = 0;
      while (ld_acquire(&h->bar_gen) == gen) {
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
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
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
