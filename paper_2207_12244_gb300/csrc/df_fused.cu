#include "df_fused.cuh"

namespace df {

bool fused_supported() { return false; }

cudaError_t launch_solve_fused(const Planes *const *, int, const SolveCfg &, int, int,
                               cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace df
