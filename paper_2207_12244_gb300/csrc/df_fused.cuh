// Fused persistent solver: the whole per-frame solve of one or more
// keyframes in a single cooperative launch (host interface).
#pragma once

#include <vector>

#include "df_internal.cuh"

namespace df {

constexpr int kMaxBatch = 256;  // keyframes per fused launch

// Launch shape. 0 = chosen from the problem size.
struct FusedTuning {
  int vec = 0;        // pixels per lane along a row: 1 or 4
  int tile_rows = 0;  // rows per warp tile
  int max_ctas = 0;   // cap on the cooperative grid
};

// True when the current device can run the fused solver.
bool fused_supported();

// Largest cooperative grid the fused kernel can use on the current device.
int fused_max_ctas();

// Bytes of a launch plan for nkf keyframes and a grid of G CTAs.
size_t fused_plan_bytes(int nkf, int G);

// Host-side plan of one launch (tiles, CTA ranges, reduction slots, barrier
// words). Returns false if the keyframes cannot share one launch (then
// split the batch).
bool fused_build_plan(const Planes *const *kfs, int n, const FusedTuning &tune,
                      std::vector<char> &out, int &G, int &vec);

// Launch on stream s with a plan already copied to device memory 'dplan'.
// limit_ns bounds every grid-barrier wait.
cudaError_t fused_launch(void *dplan, int G, int vec, const SolveCfg &c, int n_gn, int n_pcg,
                         unsigned long long limit_ns, cudaStream_t s);

}  // namespace df
