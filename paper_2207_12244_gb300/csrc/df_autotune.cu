// Autotuner of the fused solver's launch shape (df_autotune): times
// candidate shapes on the caller's own keyframes, each trial starting from
// the same state, and keeps the fastest.
#include <algorithm>
#include <vector>

#include "df_internal.cuh"

namespace {

struct Snapshot {
  std::vector<float *> x;
  std::vector<double> t;
};

}  // namespace

extern "C" df_status df_autotune(df_keyframe *const *kfs, int32_t n, const df_solve_params *params,
                                 void *stream, df_tuning *best, float *best_ms) {
  if (!kfs || n < 1 || !best) return df::report(DF_EINVAL, "bad arguments");
  df_solve_params p;
  if (params) {
    p = *params;
  } else {
    df_default_params(&p);
  }
  p.solver = DF_SOLVER_FUSED;
  df_status st = df::check_solve_params(&p);
  if (st != DF_OK) return st;
  // the list is checked before anything is allocated or any state changes
  for (int32_t j = 0; j < n; ++j) {
    if (!kfs[j]) return df::report(DF_EINVAL, "keyframe %d is NULL", (int)j);
    for (int32_t m = 0; m < j; ++m)
      if (kfs[m] == kfs[j]) return df::report(DF_EINVAL, "keyframe %d appears twice", (int)j);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  df_tuning saved;
  df_get_tuning(&saved);
  // snapshot every keyframe's (x, t); on a failure part-way, only the
  // snapshots taken so far are freed (no keyframe has been touched yet)
  Snapshot snap;
  auto free_snap = [&]() {
    cudaStreamSynchronize(s);
    for (float *q : snap.x) cudaFree(q);
    snap.x.clear();
    snap.t.clear();
  };
  for (int32_t j = 0; j < n; ++j) {
    df_keyframe_desc d;
    size_t bytes = 0;
    st = df_keyframe_info(kfs[j], &d, &bytes);
    if (st != DF_OK) {
      free_snap();
      return st;
    }
    float *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, (size_t)d.width * d.height * sizeof(float));
    if (e != cudaSuccess) {
      free_snap();
      return df::report(DF_ENOMEM, "autotune snapshot: %s", cudaGetErrorString(e));
    }
    double t = 0.0;
    st = df_keyframe_get_state(kfs[j], buf, &t, 0, stream);
    if (st != DF_OK) {
      cudaFree(buf);
      free_snap();
      return st;
    }
    snap.x.push_back(buf);
    snap.t.push_back(t);
  }
  auto restore = [&]() -> df_status {
    for (size_t j = 0; j < snap.x.size(); ++j) {
      df_status r = df_keyframe_set_state(kfs[j], snap.x[j], snap.t[j], 1, stream);
      if (r != DF_OK) return r;
    }
    return DF_OK;
  };
  auto solve = [&]() -> df_status {
    return n == 1 ? df_optimise(kfs[0], &p, stream, nullptr)
                  : df_optimise_batch(kfs, n, &p, stream, nullptr);
  };
  std::vector<df_tuning> cand;
  // resident kernel: all GN iterations in one launch, or one per launch;
  // streaming kernel: each warp walks its whole row share (tile_rows 0) or
  // pieces of at most tile_rows rows, at both vector widths, and the whole
  // share with 1 or 2 GN iterations per launch
  for (int g : {0, 1}) cand.push_back(df_tuning{2, 0, 0, 0, g, -1, 0});
  for (int vec : {1, 4})
    for (int th : {0, 4, 8, 16, 32, 64}) cand.push_back(df_tuning{1, vec, th, 0, 0, -1, 0});
  for (int g : {1, 2}) cand.push_back(df_tuning{1, 4, 0, 0, g, -1, 0});
  cand.push_back(df_tuning{1, 4, 0, 0, 0, -1, 1});  // the assembly inside the persistent kernel
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    free_snap();
    return df::report(DF_ECUDA, "autotune: cannot create timing events");
  }
  // each candidate: one untimed solve, then the median of kReps timed ones
  constexpr int kReps = 5;
  float best_t = 0.0f;
  bool have = false;
  for (const df_tuning &c : cand) {
    df_set_tuning(&c);
    if (restore() != DF_OK) continue;
    if (solve() != DF_OK) {  // e.g. the resident kernel cannot hold these keyframes
      cudaStreamSynchronize(s);
      continue;
    }
    float ms[kReps];
    int got = 0;
    for (int rep = 0; rep < kReps; ++rep) {
      if (restore() != DF_OK) break;
      cudaEventRecord(e0, s);
      if (solve() != DF_OK) break;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float v = 0.0f;
      cudaEventElapsedTime(&v, e0, e1);
      ms[got++] = v;
    }
    if (got < kReps) {
      cudaStreamSynchronize(s);
      continue;
    }
    std::sort(ms, ms + kReps);
    const float med = ms[kReps / 2];
    if (!have || med < best_t) {
      best_t = med;
      *best = c;
      have = true;
    }
  }
  df_status rs = restore();
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  free_snap();
  if (!have) {
    df_set_tuning(&saved);
    return df::report(DF_ENOTSUP, "no launch shape could solve these keyframes");
  }
  df_set_tuning(best);
  if (best_ms) *best_ms = best_t;
  return rs;
}
