// Batched per-frame bookkeeping of many keyframes in a few launches
// (df_keyframe_reset_batch, df_frame_update_batch, df_fetch_depth_batch):
// the network planes' reload with the keyframe initialisation x = mu_n,
// t = 0 (Section II: a new keyframe starts from the network's prediction)
// and the device-side input check; the frame's semi-dense planes; the depth
// output d = exp(x) (Eq. 5's d, from the log-depth x).
//
// One launch covers up to kIoBatch keyframes, whose pointers and sizes
// travel as a kernel parameter (no upload, so the calls can be captured in
// a CUDA graph). The work is the flattened list of every keyframe's rows;
// each warp takes one row at a time, and its lanes walk the row in 16-byte
// vectors when the caller's rows are 16-byte aligned, else element by
// element (a row of 320 f32 values is 80 vectors: a whole warp stays busy,
// where a whole block per row would leave most of its threads idle). The
// keyframe's own planes are pitched (every row starts on a 256-byte
// boundary), the caller's are dense.
#include "df_batch_io.cuh"

namespace df {
namespace {

constexpr int kIoThreads = 256;
constexpr int kIoWarps = kIoThreads / 32;

__device__ __forceinline__ int item_of(const IoBatch &b, int row) {
  int j = 0;
  while (j + 1 < b.n && b.item[j + 1].row0 <= row) ++j;
  return j;
}

__device__ __forceinline__ bool ok_value(float m) { return isfinite(m); }
__device__ __forceinline__ bool ok_variance(float v) { return isfinite(v) && v > 0.0f; }

// Element e of a 16-byte vector of DT values, as float.
template <int DT>
__device__ __forceinline__ float unpack(const uint4 &q, int e) {
  const uint32_t w = (&q.x)[DT == DF_F32 ? e : e >> 1];
  if constexpr (DT == DF_F32) {
    return __uint_as_float(w);
  } else {
    const unsigned short h = (unsigned short)((e & 1) ? (w >> 16) : (w & 0xffffu));
    if constexpr (DT == DF_BF16) return __bfloat162float(__ushort_as_bfloat16(h));
    return __half2float(__ushort_as_half(h));
  }
}

template <int DT>
__device__ __forceinline__ float load_elem(const void *base, size_t i) {
  return ld_cnn<DT>(base, i);
}

template <int DT>
__device__ __forceinline__ void copy_elem(void *dst, size_t di, const void *src, size_t si) {
  if constexpr (DT == DF_F32) {
    static_cast<float *>(dst)[di] = static_cast<const float *>(src)[si];
  } else {
    static_cast<unsigned short *>(dst)[di] = static_cast<const unsigned short *>(src)[si];
  }
}

// One row v of a keyframe's reset: the six network planes copied into the
// keyframe's layout, x = mu_n, the semi-dense variance zeroed (no
// semi-dense term until the next frame update); returns whether any input
// of the row is invalid (checked only when asked).
template <int DT>
__device__ bool reset_row(const IoItem &it, int v, bool check) {
  constexpr int ES = DT == DF_F32 ? 4 : 2;
  constexpr int PER = 16 / ES;  // elements per 16-byte vector
  const int W = it.W;
  const size_t srow = (size_t)v * W, drow = (size_t)v * it.P;
  const bool last_row = v == it.H - 1;
  bool bad = false;
  if (it.vec) {
    const int nv = W / PER;
    for (int c = threadIdx.x & 31; c < nv; c += 32) {
      uint4 q[6];
#pragma unroll
      for (int j = 0; j < 6; ++j)
        q[j] = __ldcs(reinterpret_cast<const uint4 *>(static_cast<const char *>(it.src[j]) +
                                                      (srow + (size_t)c * PER) * ES));
#pragma unroll
      for (int j = 0; j < 6; ++j)
        *reinterpret_cast<uint4 *>(static_cast<char *>(it.dst[j]) + (drow + (size_t)c * PER) * ES) =
            q[j];
      float xs[PER];
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const float m = unpack<DT>(q[0], e);
        xs[e] = m;
        if (check) {
          const int u = c * PER + e;
          bad |= !(ok_value(m) && ok_variance(unpack<DT>(q[1], e)));
          if (u < W - 1) bad |= !(ok_value(unpack<DT>(q[2], e)) && ok_variance(unpack<DT>(q[3], e)));
          if (!last_row) bad |= !(ok_value(unpack<DT>(q[4], e)) && ok_variance(unpack<DT>(q[5], e)));
        }
      }
      float4 *xr = reinterpret_cast<float4 *>(it.x + drow + (size_t)c * PER);
      float4 *zr = reinterpret_cast<float4 *>(it.var_s + drow + (size_t)c * PER);
#pragma unroll
      for (int g = 0; g < PER / 4; ++g) {
        xr[g] = make_float4(xs[4 * g], xs[4 * g + 1], xs[4 * g + 2], xs[4 * g + 3]);
        zr[g] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
    }
  } else {
    for (int u = threadIdx.x & 31; u < W; u += 32) {
#pragma unroll
      for (int j = 0; j < 6; ++j) copy_elem<DT>(it.dst[j], drow + u, it.src[j], srow + u);
      const float m = load_elem<DT>(it.src[0], srow + u);
      it.x[drow + u] = m;
      it.var_s[drow + u] = 0.0f;
      if (check) {
        bad |= !(ok_value(m) && ok_variance(load_elem<DT>(it.src[1], srow + u)));
        if (u < W - 1)
          bad |= !(ok_value(load_elem<DT>(it.src[2], srow + u)) &&
                   ok_variance(load_elem<DT>(it.src[3], srow + u)));
        if (!last_row)
          bad |= !(ok_value(load_elem<DT>(it.src[4], srow + u)) &&
                   ok_variance(load_elem<DT>(it.src[5], srow + u)));
      }
    }
  }
  return bad;
}

// Every item's Scalars to zero (t = 0, no flags, no CG state); runs before
// k_io_reset, whose input check may then raise the flag.
__global__ void k_io_zero_scalars(IoBatch b) {
  const int j = blockIdx.x;
  if (j >= b.n) return;
  uint4 *p = reinterpret_cast<uint4 *>(b.item[j].sc);
  for (int q = threadIdx.x; q < (int)(sizeof(Scalars) / sizeof(uint4)); q += blockDim.x)
    p[q] = make_uint4(0u, 0u, 0u, 0u);
}

// The flattened row list, one row per warp at a time.
#define IO_FOR_EACH_ROW(b, r)                                                    \
  for (int r = blockIdx.x * kIoWarps + (threadIdx.x >> 5); r < (b).total;       \
       r += gridDim.x * kIoWarps)

__global__ void __launch_bounds__(kIoThreads) k_io_reset(IoBatch b) {
  IO_FOR_EACH_ROW(b, r) {
    const IoItem &it = b.item[item_of(b, r)];
    const int v = r - it.row0;
    bool bad;
    if (it.dtype == DF_BF16)
      bad = reset_row<DF_BF16>(it, v, b.check);
    else if (it.dtype == DF_F16)
      bad = reset_row<DF_F16>(it, v, b.check);
    else
      bad = reset_row<DF_F32>(it, v, b.check);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
      atomicOr(&it.sc->flags, kFlagBadInput);
  }
}

// One row of a frame update: mu_s and var_s (f32) into the keyframe's layout.
__global__ void __launch_bounds__(kIoThreads) k_io_update(IoBatch b) {
  const int lane = threadIdx.x & 31;
  IO_FOR_EACH_ROW(b, r) {
    const IoItem &it = b.item[item_of(b, r)];
    const int v = r - it.row0;
    const size_t srow = (size_t)v * it.W, drow = (size_t)v * it.P;
    if (it.vec) {
      for (int c = lane; c < it.W / 4; c += 32) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const float4 q = __ldcs(reinterpret_cast<const float4 *>(
              static_cast<const float *>(it.src[j]) + srow + (size_t)4 * c));
          *reinterpret_cast<float4 *>(static_cast<float *>(it.dst[j]) + drow + (size_t)4 * c) = q;
        }
      }
    } else {
      for (int u = lane; u < it.W; u += 32) {
#pragma unroll
        for (int j = 0; j < 2; ++j)
          static_cast<float *>(it.dst[j])[drow + u] = static_cast<const float *>(it.src[j])[srow + u];
      }
    }
  }
}

// One row of the depth output: out = exp(x) (or x), dense.
__global__ void __launch_bounds__(kIoThreads) k_io_fetch(IoBatch b) {
  const int lane = threadIdx.x & 31;
  IO_FOR_EACH_ROW(b, r) {
    const IoItem &it = b.item[item_of(b, r)];
    const int v = r - it.row0;
    const size_t srow = (size_t)v * it.P, drow = (size_t)v * it.W;
    float *out = static_cast<float *>(it.dst[0]);
    if (it.vec) {
      for (int c = lane; c < it.W / 4; c += 32) {
        float4 q = *reinterpret_cast<const float4 *>(it.x + srow + (size_t)4 * c);
        if (!b.log_space) q = make_float4(expf(q.x), expf(q.y), expf(q.z), expf(q.w));
        __stcs(reinterpret_cast<float4 *>(out + drow + (size_t)4 * c), q);
      }
    } else {
      for (int u = lane; u < it.W; u += 32) {
        const float xi = it.x[srow + u];
        out[drow + u] = b.log_space ? xi : expf(xi);
      }
    }
  }
}

int io_grid(int total_rows) {
  const int blocks = (total_rows + kIoWarps - 1) / kIoWarps;
  const int cap = 152 * 8;  // a few waves of 256-thread blocks on every SM
  return blocks < 1 ? 1 : (blocks < cap ? blocks : cap);
}

}  // namespace

void preload_io_kernels() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, k_io_zero_scalars);
  cudaFuncGetAttributes(&fa, k_io_reset);
  cudaFuncGetAttributes(&fa, k_io_update);
  cudaFuncGetAttributes(&fa, k_io_fetch);
  cudaGetLastError();
}

cudaError_t launch_io(IoKind kind, const IoBatch &b, cudaStream_t s) {
  if (b.n <= 0 || b.total <= 0) return cudaSuccess;
  const int grid = io_grid(b.total);
  switch (kind) {
    case IoKind::kReset:
      count_launches(2);
      k_io_zero_scalars<<<b.n, 32, 0, s>>>(b);
      k_io_reset<<<grid, kIoThreads, 0, s>>>(b);
      break;
    case IoKind::kUpdate:
      count_launches(1);
      k_io_update<<<grid, kIoThreads, 0, s>>>(b);
      break;
    case IoKind::kFetch:
      count_launches(1);
      k_io_fetch<<<grid, kIoThreads, 0, s>>>(b);
      break;
  }
  return cudaGetLastError();
}

}  // namespace df
