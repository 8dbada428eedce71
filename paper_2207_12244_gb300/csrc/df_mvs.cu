// Semi-dense two-view depth (Section II-B): the epipolar search that feeds
// the optimisation's semi-dense term, on the GPU.
//
// Two launches per update:
//  1. k_mvs_select (one thread per pixel): texture and interval tests; the
//     candidates are appended to a compact list (one atomic per warp), the
//     others get their status.
//  2. k_mvs_search (a group of kGroup lanes per listed pixel): the lanes
//     split the 1-pixel steps of the epipolar segment, each computing the
//     5-sample error (Eq. 2) of its steps; a group argmin (first minimum on
//     ties) picks the best step; three lanes recompute the best step and its
//     two neighbours, and the group's first lane fits the sub-pixel depth
//     between the best step and its
//     better neighbour, sets sigma^2 = photo_var (J^T J)^-1 (Eqs. 3, 4) and
//     fuses the measurement with the current estimate.
//
// The reference image is read through the read-only path (it is small and
// reused by every step of neighbouring pixels); everything runs in FP32.
#include <math.h>

#include <algorithm>

#include "df_internal.cuh"

struct df_mvs {
  int W, H;
  int device;
  int *list;   // W * H candidate pixel indices
  int *count;  // number of listed pixels
  unsigned long long *steps;  // epipolar steps evaluated by the last update
};

namespace df {
namespace {

constexpr int kSelThreads = 256;
constexpr int kSearchThreads = 256;  // 8 warps, one pixel each at a time

struct MvsGeo {
  float fx, fy, cx, cy;
  float ifx, ify;  // 1 / fx, 1 / fy
  float R[9], t[3];
  float C[3];  // reference camera centre in keyframe coordinates, -R^T t
};

struct MvsCfg {
  float grad_min, d_min, d_max, sigma_range, ssd_max, photo_var;
  int max_steps;
};

__device__ __forceinline__ bool mvs_interval(float dp, float vp, const MvsCfg &p, float *lo,
                                             float *hi) {
  float a = p.d_min, b = p.d_max;
  if (dp > 0.0f && isfinite(dp) && vp > 0.0f && isfinite(vp)) {
    const float sp = sqrtf(vp);
    a = fmaxf(dp - p.sigma_range * sp, p.d_min);
    b = fminf(dp + p.sigma_range * sp, p.d_max);
  }
  *lo = a;
  *hi = b;
  return a < b;
}

__global__ void k_mvs_select(int W, int H, const float *__restrict__ img_key,
                             const float *__restrict__ depth, const float *__restrict__ var,
                             MvsCfg p, int *__restrict__ list, int *__restrict__ count,
                             int *__restrict__ status, int *__restrict__ best_step) {
  const int n = W * H;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    int st = DF_MVS_FLAT;
    if (i < n) {
      const int v = i / W, u = i - v * W;
      if (u >= 1 && u <= W - 2 && v >= 1 && v <= H - 2) {
        const float gx = 0.5f * (img_key[i + 1] - img_key[i - 1]);
        const float gy = 0.5f * (img_key[i + W] - img_key[i - W]);
        if (sqrtf(gx * gx + gy * gy) >= p.grad_min) {
          float lo, hi;
          st = mvs_interval(depth[i], var[i], p, &lo, &hi) ? -1 : DF_MVS_INTERVAL;
        }
      }
    }
    const bool take = i < n && st < 0;
    const unsigned mask = __ballot_sync(0xffffffffu, take);
    int slot0 = 0;
    if ((threadIdx.x & 31) == 0 && mask) slot0 = atomicAdd(count, __popc(mask));
    slot0 = __shfl_sync(0xffffffffu, slot0, 0);
    if (take) {
      list[slot0 + __popc(mask & ((1u << (threadIdx.x & 31)) - 1u))] = i;
    } else if (i < n) {
      if (status) status[i] = st;
      if (best_step) best_step[i] = -1;
    }
  }
}

__device__ __forceinline__ bool bilin(const float *__restrict__ I, int W, int H, float x, float y,
                                      float *out) {
  if (!(x >= 0.0f && y >= 0.0f && x <= (float)(W - 1) && y <= (float)(H - 1))) return false;
  int x0 = (int)floorf(x), y0 = (int)floorf(y);
  x0 = min(x0, W - 2);
  y0 = min(y0, H - 2);
  const float ax = x - (float)x0, ay = y - (float)y0;
  const float *r0 = I + (size_t)y0 * W + x0;
  const float *r1 = r0 + W;
  const float top = (1.0f - ax) * __ldg(r0) + ax * __ldg(r0 + 1);
  const float bot = (1.0f - ax) * __ldg(r1) + ax * __ldg(r1 + 1);
  *out = (1.0f - ay) * top + ay * bot;
  return true;
}

// Per-pixel constants of the walk.
struct Walk {
  float P0x, P0y, dx, dy;  // near end of the segment, unit direction
  int n;                   // steps
  bool use_x;              // depth from the x (else y) image coordinate
  float a0[3];             // R K^-1 [u v 1]^T
  float a1[3];             // R K^-1 [e0x e0y 0]^T (one sample spacing)
  float key[5];            // keyframe samples
};

// Photometric error 5-vector, SSD and depth of step j (Eq. 2).
__device__ __forceinline__ bool step_error(const Walk &w, const MvsGeo &g,
                                           const float *__restrict__ I1, int W, int H, int j,
                                           float e[5], float *ssd, float *dj) {
  const float qx = w.P0x + (float)j * w.dx, qy = w.P0y + (float)j * w.dy;
  // the depth whose projection is q: Y = d a0 + t, q~ = Y_x / Y_z, so
  // d (q~ a0_z - a0_x) = t_x - q~ t_z (or the y row)
  float d;
  if (w.use_x) {
    const float qt = (qx - g.cx) * g.ifx;
    d = (g.t[0] - qt * g.t[2]) / (qt * w.a0[2] - w.a0[0]);
  } else {
    const float qt = (qy - g.cy) * g.ify;
    d = (g.t[1] - qt * g.t[2]) / (qt * w.a0[2] - w.a0[1]);
  }
  if (!(d > 0.0f) || !isfinite(d)) return false;
  float s2 = 0.0f;
#pragma unroll
  for (int s = -2; s <= 2; ++s) {
    const float sf = (float)s;
    const float Y0 = d * (w.a0[0] + sf * w.a1[0]) + g.t[0];
    const float Y1 = d * (w.a0[1] + sf * w.a1[1]) + g.t[1];
    const float Y2 = d * (w.a0[2] + sf * w.a1[2]) + g.t[2];
    if (!(Y2 > 0.0f)) return false;
    const float iz = 1.0f / Y2;  // one exact reciprocal for both coordinates
    const float pu = g.fx * Y0 * iz + g.cx, pv = g.fy * Y1 * iz + g.cy;
    float val;
    if (!bilin(I1, W, H, pu, pv, &val)) return false;
    e[s + 2] = val - w.key[s + 2];
    s2 += e[s + 2] * e[s + 2];
  }
  *ssd = s2;
  *dj = d;
  return true;
}

// Lanes per listed pixel: a warp serves 32 / kGroup pixels at once. With an
// estimate the search interval spans only a few steps, so a whole warp per
// pixel would leave most lanes idle; long walks take more rounds per pixel
// but as many steps per warp and round.
constexpr int kGroup = 8;

__global__ void __launch_bounds__(kSearchThreads)
    k_mvs_search(int W, int H, const float *__restrict__ img_key,
                 const float *__restrict__ img_ref, MvsGeo g, MvsCfg p,
                 const int *__restrict__ list, const int *__restrict__ count,
                 float *__restrict__ depth, float *__restrict__ var, int *__restrict__ status,
                 int *__restrict__ best_step, unsigned long long *__restrict__ steps) {
  constexpr int kPerWarp = 32 / kGroup;
  const int wl = threadIdx.x & 31;
  const int grp = wl / kGroup, lane = wl % kGroup, g0 = grp * kGroup;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int total = *count;
  // every lane runs every round (the shuffles span the warp); groups past
  // the end of the list compute nothing and write nothing
  for (int base = warp * kPerWarp; base < total; base += nwarps * kPerWarp) {
    const int e = base + grp;
    const bool live = e < total;
    const int i = live ? list[e] : list[base];
    const int v = i / W, u = i - v * W;
    const float uf = (float)u, vf = (float)v;
    const float dp = depth[i], vp = var[i];
    const bool has = dp > 0.0f && isfinite(dp) && vp > 0.0f && isfinite(vp);
    float lo, hi;
    mvs_interval(dp, vp, p, &lo, &hi);
    int st = DF_MVS_LINE, bk = -1;
    float d_new = dp, v_new = vp;
    Walk w;
    // keyframe ray and epipolar direction (x - epipole, scaled by C_z)
    const float r0 = (uf - g.cx) * g.ifx, r1 = (vf - g.cy) * g.ify;
#pragma unroll
    for (int k = 0; k < 3; ++k) w.a0[k] = g.R[3 * k] * r0 + g.R[3 * k + 1] * r1 + g.R[3 * k + 2];
    float e0x = g.C[2] * (uf - g.cx) - g.fx * g.C[0];
    float e0y = g.C[2] * (vf - g.cy) - g.fy * g.C[1];
    const float ne = sqrtf(e0x * e0x + e0y * e0y);
    bool ok = ne > 0.0f;
    // ends of the segment
    float P0x = 0.0f, P0y = 0.0f, P1x = 0.0f, P1y = 0.0f;
    if (ok) {
      const float Ya[3] = {lo * w.a0[0] + g.t[0], lo * w.a0[1] + g.t[1], lo * w.a0[2] + g.t[2]};
      const float Yb[3] = {hi * w.a0[0] + g.t[0], hi * w.a0[1] + g.t[1], hi * w.a0[2] + g.t[2]};
      ok = Ya[2] > 0.0f && Yb[2] > 0.0f;
      if (ok) {
        P0x = g.fx * Ya[0] / Ya[2] + g.cx;
        P0y = g.fy * Ya[1] / Ya[2] + g.cy;
        P1x = g.fx * Yb[0] / Yb[2] + g.cx;
        P1y = g.fy * Yb[1] / Yb[2] + g.cy;
      }
    }
    float L = 0.0f;
    if (ok) {
      const float dx = P1x - P0x, dy = P1y - P0y;
      L = sqrtf(dx * dx + dy * dy);
      ok = L > 0.0f;
      if (ok) {
        w.n = (int)floorf(L) + 1;
        ok = w.n <= p.max_steps;
        w.P0x = P0x;
        w.P0y = P0y;
        w.dx = dx / L;
        w.dy = dy / L;
        w.use_x = fabsf(w.dx) >= fabsf(w.dy);
      }
    }
    if (ok) {
      e0x /= ne;
      e0y /= ne;
      const float s0 = e0x * g.ifx, s1 = e0y * g.ify;
#pragma unroll
      for (int k = 0; k < 3; ++k) w.a1[k] = g.R[3 * k] * s0 + g.R[3 * k + 1] * s1;
#pragma unroll
      for (int s = -2; s <= 2 && ok; ++s)
        ok = bilin(img_key, W, H, uf + (float)s * e0x, vf + (float)s * e0y, &w.key[s + 2]);
    }
    ok = ok && live;
    if (live && ok && lane == 0) atomicAdd(steps, (unsigned long long)(w.n + 3));  // + 3 recomputed
    {
      // the walk: group-strided steps, then a group argmin (first minimum)
      float best = INFINITY;
      int bj = 0x7fffffff;
      const int n = ok ? w.n : 0;
      for (int j = lane; j < n; j += kGroup) {
        float ev[5], ssd, dj;
        if (step_error(w, g, img_ref, W, H, j, ev, &ssd, &dj) && ssd < best) {
          best = ssd;
          bj = j;
        }
      }
#pragma unroll
      for (int o = kGroup / 2; o > 0; o >>= 1) {  // xor below kGroup stays in the group
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob < best || (ob == best && oj < bj)) {
          best = ob;
          bj = oj;
        }
      }
      // the sub-pixel fit: lanes 0, 1, 2 of the group evaluate steps
      // bj - 1, bj, bj + 1; every lane runs the shuffles that gather them
      const bool have = ok && bj != 0x7fffffff;
      const bool fit = have && best <= p.ssd_max;
      float ev[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, ssd = 0.0f, dj = 0.0f;
      bool okj = false;
      if (fit && lane < 3) okj = step_error(w, g, img_ref, W, H, bj - 1 + lane, ev, &ssd, &dj);
      float em[5], ea[5], ep[5];
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        em[s] = __shfl_sync(0xffffffffu, ev[s], g0);
        ea[s] = __shfl_sync(0xffffffffu, ev[s], g0 + 1);
        ep[s] = __shfl_sync(0xffffffffu, ev[s], g0 + 2);
      }
      const float sm = __shfl_sync(0xffffffffu, ssd, g0), sq = __shfl_sync(0xffffffffu, ssd, g0 + 2);
      const float dm = __shfl_sync(0xffffffffu, dj, g0), da = __shfl_sync(0xffffffffu, dj, g0 + 1),
                  dq = __shfl_sync(0xffffffffu, dj, g0 + 2);
      const bool okm = __shfl_sync(0xffffffffu, okj, g0), okp = __shfl_sync(0xffffffffu, okj, g0 + 2);
      if (!ok) {
        st = DF_MVS_LINE;
      } else if (!have) {
        st = DF_MVS_NOSTEP;
      } else if (!fit) {
        bk = bj;
        st = DF_MVS_SSD;
      } else {
        bk = bj;
        st = DF_MVS_NEIGHBOUR;
        if (okm || okp) {
          const bool take_m = okm && (!okp || sm <= sq);
          float D2 = 0.0f, ade = 0.0f;
#pragma unroll
          for (int s = 0; s < 5; ++s) {
            const float de = (take_m ? em[s] : ep[s]) - ea[s];
            D2 += de * de;
            ade += ea[s] * de;
          }
          if (D2 > 0.0f) {
            const float sstar = fminf(fmaxf(-ade / D2, 0.0f), 1.0f);
            const float dd = (take_m ? dm : dq) - da;
            const float d_obs = da + sstar * dd;
            const float v_obs = p.photo_var * dd * dd / D2;
            if (v_obs > 0.0f && isfinite(v_obs)) {
              if (has) {
                d_new = (dp * v_obs + d_obs * vp) / (vp + v_obs);
                v_new = vp * v_obs / (vp + v_obs);
              } else {
                d_new = d_obs;
                v_new = v_obs;
              }
              st = DF_MVS_OK;
            }
          }
        }
      }
    }
    if (live && lane == 0) {
      if (st == DF_MVS_OK) {
        depth[i] = d_new;
        var[i] = v_new;
      }
      if (status) status[i] = st;
      if (best_step) best_step[i] = bk;
    }
  }
}

}  // namespace
}  // namespace df

extern "C" {

void df_mvs_default_params(df_mvs_params *p) {
  if (!p) return;
  p->grad_min = 20.0f;
  p->d_min = 0.3f;
  p->d_max = 10.0f;
  p->sigma_range = 2.0f;
  p->ssd_max = 5.0f * 20.0f * 20.0f;
  p->photo_var = 1.0f;
  p->max_steps = 512;
}

df_status df_mvs_create(int32_t width, int32_t height, df_mvs **out) {
  if (!out) return df::report(DF_EINVAL, "out is NULL");
  *out = nullptr;
  if (width < 1 || height < 1 || (int64_t)width * height > (int64_t)1 << 30)
    return df::report(DF_EINVAL, "bad image size %d x %d", width, height);
  df_mvs *m = new df_mvs();
  m->W = width;
  m->H = height;
  cudaGetDevice(&m->device);
  cudaError_t e = cudaMalloc(&m->list, sizeof(int) * ((size_t)width * height + 1));
  if (e == cudaSuccess) e = cudaMalloc(&m->count, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&m->steps, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaGetLastError();
    df_mvs_destroy(m);
    return df::report(DF_ENOMEM, "df_mvs_create: %s", cudaGetErrorString(e));
  }
  *out = m;
  return DF_OK;
}

void df_mvs_destroy(df_mvs *m) {
  if (!m) return;
  if (m->list) cudaFree(m->list);
  if (m->count) cudaFree(m->count);
  if (m->steps) cudaFree(m->steps);
  delete m;
}

df_status df_mvs_update(df_mvs *m, const float *img_key, const float *img_ref,
                        const df_camera *cam, const df_pose *key_to_ref,
                        const df_mvs_params *params, float *depth, float *var,
                        int32_t *status, int32_t *best_step, void *stream) {
  using namespace df;
  if (!m || !img_key || !img_ref || !cam || !key_to_ref || !depth || !var)
    return report(DF_EINVAL, "df_mvs_update: NULL argument");
  df_mvs_params pp;
  if (params) {
    pp = *params;
  } else {
    df_mvs_default_params(&pp);
  }
  if (!(pp.d_min > 0.0f) || !(pp.d_max > pp.d_min) || !isfinite(pp.d_max) || pp.max_steps < 1 ||
      !(pp.grad_min >= 0.0f) || !(pp.sigma_range >= 0.0f) || !(pp.ssd_max >= 0.0f) ||
      !(pp.photo_var > 0.0f))
    return report(DF_EINVAL, "df_mvs_update: invalid parameters");
  if (!(cam->fx != 0.0f) || !(cam->fy != 0.0f) || !isfinite(cam->fx) || !isfinite(cam->fy))
    return report(DF_EINVAL, "df_mvs_update: invalid focal lengths");
  MvsGeo g;
  g.fx = cam->fx;
  g.fy = cam->fy;
  g.cx = cam->cx;
  g.cy = cam->cy;
  g.ifx = 1.0f / cam->fx;
  g.ify = 1.0f / cam->fy;
  for (int k = 0; k < 9; ++k) g.R[k] = key_to_ref->R[k];
  for (int k = 0; k < 3; ++k) g.t[k] = key_to_ref->t[k];
  for (int r = 0; r < 3; ++r)
    g.C[r] = -(g.R[r] * g.t[0] + g.R[3 + r] * g.t[1] + g.R[6 + r] * g.t[2]);
  MvsCfg c{pp.grad_min, pp.d_min, pp.d_max, pp.sigma_range, pp.ssd_max, pp.photo_var, pp.max_steps};
  int cur = 0;
  if (cudaGetDevice(&cur) == cudaSuccess && cur != m->device) cudaSetDevice(m->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = m->W * m->H;
  cudaError_t e = cudaMemsetAsync(m->count, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->steps, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
    if (sms < 1) sms = 1;
    const int sel_blocks = std::min((n + kSelThreads - 1) / kSelThreads, sms * 8);
    count_launches(2);
    k_mvs_select<<<sel_blocks, kSelThreads, 0, s>>>(m->W, m->H, img_key, depth, var, c, m->list,
                                                     m->count, status, best_step);
    k_mvs_search<<<sms * 8, kSearchThreads, 0, s>>>(m->W, m->H, img_key, img_ref, g, c, m->list,
                                                     m->count, depth, var, status, best_step,
                                                     m->steps);
    e = cudaGetLastError();
  }
  if (cur != m->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return report(DF_ECUDA, "df_mvs_update: %s", cudaGetErrorString(e));
  return DF_OK;
}

df_status df_mvs_last_steps(df_mvs *m, void *stream, uint64_t *steps) {
  if (!m || !steps) return df::report(DF_EINVAL, "NULL argument");
  unsigned long long h = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&h, m->steps, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return df::report(DF_ECUDA, "df_mvs_last_steps: %s", cudaGetErrorString(e));
  *steps = (uint64_t)h;
  return DF_OK;
}

}  // extern "C"
