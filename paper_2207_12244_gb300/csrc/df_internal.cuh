// Internal declarations of the GB300 keyframe optimiser (not part of the ABI).
//
// Device layout of one keyframe (one allocation, every plane 256-B aligned,
// rows padded to a pitch P that is a multiple of 128 elements so that every
// row starts on a 256-B boundary and 16-B vector loads never straddle it;
// the padding columns stay zero):
//
//   network planes (Section II-A outputs, f32 / bf16 / f16):
//     mu_n, var_n, gx, var_gx, gy, var_gy
//   semi-dense planes (Section II-B, f32): mu_s, var_s
//   state (f32): x = ln d
//   solver workspace (f32): diag, wx, wy and kWorkPlanes vectors
//   Scalars (FP64 scale t and CG scalars) + per-block FP64 partial sums
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "deepfusion.h"

namespace df {

constexpr int kPitchElems = 128;    // row pitch granularity (elements): a warp's
                                    // 32 x 4-element segment never crosses a row
constexpr int kWorkPlanes = 8;      // solver vectors beyond diag / wx / wy
constexpr int kMaxPartialBlocks = 4096;
constexpr int kNumQ = 6;            // FP64 quantities per partial slot

enum : int { kFlagBadInput = 1, kFlagTimeout = 2, kFlagBreakdown = 4 };

// Per-keyframe FP64 scalars, device resident for the whole life of the
// keyframe, so a solve needs no host round trip.
struct alignas(64) Scalars {
  double t;       // log scale correction, t = ln s (Eq. 6b)
  double rho;     // r.z of the current PCG iteration
  double alpha;   // CG step
  double beta;    // CG direction update
  double rr;      // r.r (convergence norm / report)
  double bb;      // b.b (relative tolerance)
  double gamma;   // p.Ap
  double cost;    // last cost evaluation
  // joint (x, t) solve: the t components of the bordered PCG
  double j_s;     // S = sum of the semi-dense weights (the border's diagonal)
  double j_rt;    // residual
  double j_pt;    // direction
  double j_qt;    // operator applied to the direction
  double acc_in, acc_valid;  // last accuracy count (df_depth_accuracy)
  int stop;       // the current depth step has ended early
  int iters;      // PCG iterations executed in the current solve
  int flags;      // kFlag* bits, sticky
  int valid;      // 1 once inputs passed the device-side check
  unsigned int count;  // last-block-done counter for the launch path
  unsigned int pad[3];
};

// Everything a kernel needs to address one keyframe.
struct Planes {
  int W, H, P;          // width, height, pitch (elements)
  int dtype;            // df_dtype of cnn[]
  const void *cnn[6];   // mu_n, var_n, gx, var_gx, gy, var_gy
  const float *mu_s, *var_s;
  float *x;
  float *diag, *wx, *wy;
  float *v[kWorkPlanes];  // solver vectors (meaning depends on the schedule)
  Scalars *sc;
  double *partial;      // [kMaxPartialBlocks * kNumQ]
};

struct SolveCfg {
  float delta;      // robust threshold on whitened residuals (<= 0 or inf: L2)
  int loss;         // DF_LOSS_*
  int terms;        // DF_TERM_* bits
  int scale_step;   // DF_SCALE_*
  double tol;       // relative residual tolerance (0: fixed count)
};

// ---- element loads --------------------------------------------------------

template <int DT>
__device__ __forceinline__ float ld_cnn(const void *base, size_t i) {
  if constexpr (DT == DF_BF16) {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(base)[i]);
  } else if constexpr (DT == DF_F16) {
    return __half2float(reinterpret_cast<const __half *>(base)[i]);
  } else {
    return reinterpret_cast<const float *>(base)[i];
  }
}

// ---- robust weights (Section II-C, last paragraphs) -----------------------
//
// The IRLS weight of a term with residual r and variance V is omega(u) / V,
// u = r / sqrt(V): omega = 1 (least squares), min(1, delta/|u|) (Huber),
// (1 - (u/delta)^2)^2 for |u| < delta else 0 (Tukey).
__device__ __forceinline__ bool robust_active(float delta) {
  return delta > 0.0f && delta < INFINITY;
}

// The special-function unit's reciprocal and reciprocal square root with
// subnormal operands and results flushed to zero (PTX rcp.approx.ftz.f32,
// rsqrt.approx.ftz.f32; a few ulp, far inside the solve's tolerance).
// Without .ftz the same approximations come wrapped in range handling for
// subnormal operands, extra instructions in every IRLS weight and diagonal
// reciprocal: the assembly and scale-step passes of a 1920 x 1440 solve
// (the passes with the most arithmetic per byte) ran 15 % longer. Callers keep the operands normal where it matters:
// variances are clamped up to FLT_MIN, a diagonal below FLT_MIN counts as an
// empty equation, and a subnormal u^2 flushes to 0, where rsqrt gives +inf
// exactly as at u = 0.
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kFltMin = 1.17549435e-38f;  // smallest normal float

// 1 / d for a diagonal entry d >= 0; 0 for an empty equation (d below the
// smallest normal float).
__device__ __forceinline__ float inv_diag(float d) { return d >= kFltMin ? rcp_ftz(d) : 0.0f; }

// IRLS weight omega(u) / V of a residual r with variance V, u^2 = r^2 / V.
// Huber: omega = min(1, delta / |u|), written min(1, delta rsqrt(u^2)) (1
// at u = 0, where rsqrt gives +inf). Tukey: omega = (1 - u^2 / delta^2)^2
// for u^2 < delta^2, else 0. Both are continuous at the threshold, so no
// result hinges on a comparison. A variance below the smallest normal float
// weighs as that float does (1 / V saturates at ~8.5e37).
//
// The fused kernels fix the loss at compile time (one instance per loss
// kind), so their inner loops carry no branch on it; robust_weight picks the
// same arithmetic at run time for the other kernels.
enum : int { LK_LSQ = 0, LK_HUBER = 1, LK_TUKEY = 2 };

__host__ __device__ inline int loss_kind(int loss, float delta) {
  if (!(delta > 0.0f && delta < INFINITY)) return LK_LSQ;
  return loss == DF_LOSS_TUKEY ? LK_TUKEY : LK_HUBER;
}

template <int LK>
__device__ __forceinline__ float robust_weight_k(float r, float V, float delta) {
  const float iv = rcp_ftz(fmaxf(V, kFltMin));
  if constexpr (LK == LK_LSQ) {
    return iv;
  } else if constexpr (LK == LK_TUKEY) {
    const float u2 = r * r * iv;
    const float q = 1.0f - u2 * rcp_ftz(fmaxf(delta * delta, kFltMin));
    return u2 < delta * delta ? q * q * iv : 0.0f;
  } else {
    const float u2 = r * r * iv;
    return iv * fminf(1.0f, delta * rsqrt_ftz(u2));
  }
}

__device__ __forceinline__ float robust_weight(float r, float V, float delta, int loss) {
  switch (loss_kind(loss, delta)) {
    case LK_LSQ: return robust_weight_k<LK_LSQ>(r, V, delta);
    case LK_TUKEY: return robust_weight_k<LK_TUKEY>(r, V, delta);
    default: return robust_weight_k<LK_HUBER>(r, V, delta);
  }
}

// Robust loss rho(u) (the cost of Eq. 5 with each squared whitened residual
// replaced), in FP64 for the cost reduction.
__device__ __forceinline__ double robust_rho(double r, double V, double delta, int loss) {
  const double u = r / sqrt(V);
  if (!(delta > 0.0 && delta < INFINITY)) return u * u;
  const double a = fabs(u);
  if (loss == DF_LOSS_TUKEY) {
    if (a >= delta) return delta * delta / 3.0;
    const double q = 1.0 - (u / delta) * (u / delta);
    return delta * delta / 3.0 * (1.0 - q * q * q);
  }
  return a <= delta ? u * u : 2.0 * delta * a - delta * delta;
}

__device__ __forceinline__ bool semi_valid(float mu, float var) {
  return isfinite(mu) && isfinite(var) && var > 0.0f;
}

// ---- reductions -----------------------------------------------------------

// FP32 butterfly-free warp sum (lane 0 holds the result). Used for the
// per-warp stage of the solver's inner products: GB300's FP64 rate is a tiny
// fraction of FP32, so FP64 starts above the warp (cross-warp and cross-CTA
// sums of a few hundred values).
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NQ doubles in a fixed order; the result is valid in
// thread 0. 'sm' must hold 32 * NQ doubles.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double *sm) {
  const int lane = threadIdx.x & 31;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if ((tid & 31) == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[warp * NQ + q] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = (lane < nwarps) ? sm[lane * NQ + q] : 0.0;
      v[q] = warp_sum(s);
    }
  }
  (void)lane;
}

// Grid-wide FP64 sum by "last block done": every block stores its partial,
// the last block to arrive adds all partials in block order (so the result
// does not depend on which block came last) and returns true in thread 0
// with the totals in 'out'. The counter is left at zero for the next use.
template <int NQ>
__device__ bool grid_sum_last_block(double (&v)[NQ], double *partial, unsigned int *count,
                                    double (&out)[NQ]) {
  __shared__ double sm[32 * NQ];
  __shared__ bool last;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  const int nblk = gridDim.x;
  block_sum<NQ>(v, sm);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) partial[blockIdx.x * NQ + q] = v[q];
    __threadfence();
    const unsigned int prev = atomicAdd(count, 1u);
    last = (prev == (unsigned int)nblk - 1u);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) s[q] = 0.0;
  for (int b = tid; b < nblk; b += nthr) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] += __ldcg(partial + b * NQ + q);
  }
  block_sum<NQ>(s, sm);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) out[q] = s[q];
    *count = 0u;
  }
  return tid == 0;
}

// ---- host-side launch wrappers (launch path, df_launch.cu) ----------------

// Counts kernel launches (df_kernel_launches); call once per launch.
void count_launches(unsigned n);

// Shared with the entry points outside df_api.cu: record an error message
// for df_last_error() and return the status; check / convert solve params.
df_status report(df_status s, const char *fmt, ...);
df_status check_solve_params(const df_solve_params *p);
// The schedule split at the end of its Huber warm start: writes 1 or 2
// phases of whole GN iterations (each with warm_gn = 0) and returns their
// number.
int split_schedule(const df_solve_params &p, df_solve_params ph[2]);
SolveCfg solve_cfg(const df_solve_params *p);
// df_optimise_batch through caller-owned plan buffers (device 'dplan' of
// dcap bytes, pinned host 'hplan' of hcap bytes): no allocation; falls back
// to df_optimise_batch for lists that cannot use them (df_api.cu).
// one_launch: keep each phase one cooperative launch (no separate assembly
// kernel under the automatic placement).
df_status optimise_batch_buffered(df_keyframe *const *kfs, int32_t n, const df_solve_params *params,
                                  cudaStream_t s, void *dplan, size_t dcap, void *hplan,
                                  size_t hcap, bool one_launch);

int launch_grid(int tiles);  // blocks for a grid-stride launch over 32x8 tiles

cudaError_t launch_init_state(const Planes &k, cudaStream_t s);
cudaError_t launch_check_inputs(const Planes &k, cudaStream_t s);
cudaError_t launch_solve_launches(const Planes &k, const SolveCfg &c, int n_gn, int n_pcg,
                                  cudaStream_t s);
cudaError_t launch_fetch(const Planes &k, float *out, int log_space, cudaStream_t s);
cudaError_t launch_cost(const Planes &k, const SolveCfg &c, cudaStream_t s);
cudaError_t launch_accuracy(const Planes &k, const float *d_true, double rel_tol, cudaStream_t s);
cudaError_t launch_set_x(const Planes &k, const float *x_dense, cudaStream_t s);
cudaError_t launch_set_scale(const Planes &k, double t, cudaStream_t s);
cudaError_t launch_ls_scale_fit(const Planes &k, cudaStream_t s);
cudaError_t launch_semi_to_log(const float *d, const float *vd, float *mu, float *var,
                               int64_t n, cudaStream_t s);

}  // namespace df
