// Fused persistent solver: the whole per-frame solve of one or more
// keyframes in a single cooperative launch (declarations).
#pragma once

#include "df_internal.cuh"

namespace df {

constexpr int kMaxBatch = 256;  // keyframes per fused launch

// True when the current device can run the fused solver.
bool fused_supported();

// Solve n keyframes (n <= kMaxBatch) with one launch on stream s.
cudaError_t launch_solve_fused(const Planes *const *kfs, int n, const SolveCfg &c, int n_gn,
                               int n_pcg, cudaStream_t s);

}  // namespace df
