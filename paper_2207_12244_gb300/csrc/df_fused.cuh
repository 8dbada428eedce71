// Fused persistent solver: the whole per-frame solve of one or more
// keyframes in a single cooperative launch (host interface).
#pragma once

#include <vector>

#include "df_internal.cuh"

namespace df {

constexpr int kMaxBatch = 256;  // keyframes per fused launch

enum : int { kModeAuto = 0, kModeStreaming = 1, kModeResident = 2 };

// Launch shape knobs. 0 = chosen from the problem size.
struct FusedTuning {
  int mode = kModeAuto;  // resident if the state fits in shared memory, else streaming
  int vec = 0;           // streaming: pixels per lane along a row (1 or 4)
  int tile_rows = 0;     // streaming: rows per warp tile
  int max_ctas = 0;      // cap on the cooperative grid
  int gn_per_launch = 0; // GN iterations per launch (0: all)
  int debug_skip_cta = -1;  // test hook, see df_tuning
  int assembly = 0;      // streaming: 0 auto (separate kernel), 1 inside the
                         // persistent kernel, 2 separate kernel
};

// What one fused launch looks like (filled by fused_build_plan).
struct LaunchShape {
  int kind = -1;  // kPlanStreaming / kPlanResident (df_sync.cuh)
  int G = 0;      // CTAs
  int vec = 0;    // streaming tile width selector
  int smem = 0;   // dynamic shared memory per CTA (resident)
  int asm_pieces = 0;  // streaming: pieces of the separate assembly (0: none)
};

// True when the current device can run the fused solver.
bool fused_supported();

// Largest cooperative grid the fused kernel can use on the current device.
int fused_max_ctas();

// Bytes of a launch plan for nkf keyframes and a grid of G CTAs.
size_t fused_plan_bytes(int nkf, int G);

// Bytes a single keyframe reserves for its own launch plan (either kernel).
size_t fused_plan_cap_single();

// Host-side plan of one launch (tiles, CTA ranges, exact-sum words, exit
// words). Returns false if the keyframes cannot share one launch (then
// split the batch).
bool fused_build_plan(const Planes *const *kfs, int n, const FusedTuning &tune,
                      std::vector<char> &out, LaunchShape &shape);

// Launch on stream s with a plan already copied to device memory 'dplan'.
// limit_ns bounds every device-side wait (sum words, staged rows).
// 'first' = 1 for the first launch of a solve (the reported PCG iteration
// count starts at 0), 0 for later launches of the same solve.
cudaError_t fused_launch(void *dplan, const LaunchShape &shape, const SolveCfg &c, int n_gn,
                         int n_pcg, unsigned long long limit_ns, cudaStream_t s, int first = 1);

// The two kernels behind fused_*: streaming (df_fused.cu) and resident
// (df_resident.cu).
bool streaming_supported();
int streaming_max_ctas();
size_t streaming_plan_bytes(int nkf, int G);
bool streaming_build_plan(const Planes *const *kfs, int n, const FusedTuning &tune,
                          std::vector<char> &out, LaunchShape &shape);
cudaError_t streaming_launch(void *dplan, const LaunchShape &shape, const SolveCfg &c, int n_gn,
                             int n_pcg, unsigned long long limit_ns, cudaStream_t s, int first);
int resident_max_ctas();
size_t resident_plan_bytes(int nkf, int G);
bool resident_build_plan(const Planes *const *kfs, int n, const FusedTuning &tune,
                         std::vector<char> &out, LaunchShape &shape);
cudaError_t resident_launch(void *dplan, const LaunchShape &shape, const SolveCfg &c, int n_gn,
                            int n_pcg, unsigned long long limit_ns, cudaStream_t s, int first);

}  // namespace df
