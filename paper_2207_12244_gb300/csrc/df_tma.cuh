// Asynchronous bulk copies (TMA engine) of tile rows into shared memory for
// the streaming solver: PTX wrappers for mbarriers and cp.async.bulk, and a
// per-warp ring of row stages.
//
// A stage holds, for each plane a pass needs, one row segment of a warp's
// tile: the tile's 128 columns plus 16 bytes on each side (the west / east
// neighbours of the tile's edge columns come with the row). Copies start and
// end on 16-byte boundaries: rows are padded to a multiple of 128 elements,
// tiles start at multiples of 128 elements, and the side halos are 16 bytes.
#pragma once

#include <stdint.h>

#include "df_sync.cuh"

namespace df {

constexpr int kStages = 4;           // rows in flight per warp (ring depth)
constexpr int kSlotBytes = 576;      // one plane's staged row (<= 144 f32 / 288 half)
constexpr int kMaxStagePlanes = 9;
constexpr int kStageBytes = kSlotBytes * kMaxStagePlanes;
constexpr int kWarpStageBytes = kStages * kStageBytes;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// global -> shared bulk copy whose completion is counted on 'bar'
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// generic-proxy accesses before async-proxy accesses of the same memory
// The same with the shared addresses of the destination and the mbarrier
// already converted.
__device__ __forceinline__ void bulk_copy_g2s_a(uint32_t dst, const void *src, uint32_t bytes,
                                                uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// One plane of a staged row: its global base and element size (4 or 2).
struct StagePlane {
  const void *base;
  int esize;
};

// A warp's ring of row stages. Lane 0 issues the copies (the tile's row
// walker does), every lane waits and reads.
struct RowRing {
  char *smem;         // kWarpStageBytes of this warp
  uint64_t *bars;     // kStages mbarriers
  uint32_t parity;    // bit s: parity the next wait on stage s expects
  uint32_t pending;   // bit s: copies issued, not yet waited for
  unsigned long long limit_ns;

  __device__ __forceinline__ char *slot(int s, int p) const {
    return smem + s * kStageBytes + p * kSlotBytes;
  }

  // Wait until stage s has landed; false if the wait ran out of time.
  __device__ __forceinline__ bool wait(int s) {
    const uint32_t ph = (parity >> s) & 1u;
    if (!mbar_try_wait(&bars[s], ph)) {
      const unsigned long long t0 = global_ns();
      while (!mbar_try_wait(&bars[s], ph)) {
        if (global_ns() - t0 > limit_ns) return false;
      }
    }
    parity ^= 1u << s;
    pending &= ~(1u << s);
    return true;
  }

  // Before leaving: wait (with the same limit) for copies still in flight.
  __device__ __forceinline__ void drain() {
    for (int s = 0; s < kStages; ++s)
      if (pending & (1u << s)) wait(s);
  }

  // f32 plane p: this lane's 4 columns, and single columns by slot index
  // (west neighbour of the tile: index 3, east neighbour: index 132).
  __device__ __forceinline__ float4 f4(int s, int p) const {
    return *reinterpret_cast<const float4 *>(slot(s, p) + (4 * (threadIdx.x & 31) + 4) * 4);
  }
  __device__ __forceinline__ float f1(int s, int p, int idx) const {
    return *reinterpret_cast<const float *>(slot(s, p) + idx * 4);
  }
  // 16-bit plane p (bf16 / f16 codes): this lane's 4 columns; single columns
  // (west: index 7, east: index 136).
  __device__ __forceinline__ uint2 h4(int s, int p) const {
    return *reinterpret_cast<const uint2 *>(slot(s, p) + (4 * (threadIdx.x & 31) + 8) * 2);
  }
  __device__ __forceinline__ unsigned short h1(int s, int p, int idx) const {
    return *reinterpret_cast<const unsigned short *>(slot(s, p) + idx * 2);
  }
};

}  // namespace df
