// Batched per-frame bookkeeping of many keyframes (df_batch_io.cu): the
// launch parameters and the host-side launch wrapper.
#pragma once

#include "df_internal.cuh"

namespace df {

// Keyframes per launch: the item table travels as a kernel parameter and
// stays under the classic 4 KB parameter limit.
constexpr int kIoBatch = 24;

struct IoItem {
  const void *src[6];  // caller's dense planes (reset: the six network planes;
                       // update: mu_s, var_s)
  void *dst[6];        // the keyframe's pitched planes (reset: cnn[0..5];
                       // update: mu_s, var_s); fetch: dst[0] = dense output
  float *x;            // the keyframe's log-depth (reset: written; fetch: read)
  float *var_s;        // the keyframe's semi-dense variance (reset: zeroed)
  Scalars *sc;         // the keyframe's scalars (reset: zeroed, then flagged)
  int W, H, P, dtype;  // size, pitch (elements), df_dtype of the network planes
  int vec;             // every row of the caller's planes is 16-byte aligned
  int row0;            // first row of this keyframe in the flattened row list
};

struct IoBatch {
  int n;          // items used
  int total;      // rows of all items
  int check;      // reset: run the device-side input check
  int log_space;  // fetch: x instead of exp(x)
  IoItem item[kIoBatch];
};

static_assert(sizeof(IoBatch) < 4000, "the item table must fit the kernel parameter space");

enum class IoKind { kReset, kUpdate, kFetch };

cudaError_t launch_io(IoKind kind, const IoBatch &b, cudaStream_t s);

// Load the batched-bookkeeping kernels on the current device now rather than
// at their first launch.
void preload_io_kernels();

}  // namespace df
