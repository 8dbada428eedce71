// Resident persistent solver: the same per-frame solve as df_fused.cu
// (Section II-C: n_gn Gauss-Newton iterations alternating scale and depth;
// Jacobi-PCG in the Chronopoulos-Gear arrangement, one exchange of the
// keyframe's exact sums per pass), for keyframes small enough that the whole
// solver state fits in the GPU's shared memory.
//
// Each CTA owns a band of whole rows [rb, re) of one keyframe and keeps
// x, r, p, s, w, diag, wx, wy and u of its band in shared memory for the
// whole launch. Only the band's first and last rows cross CTAs: after each
// pass a CTA writes them to the keyframe's global planes (L2), and the
// neighbouring band recomputes the new u of those rows from them in the next
// pass, exactly as the streaming kernel recomputes its tile halos. The global
// planes are thus touched only at band edges, plus one read of the inputs per
// Gauss-Newton iteration and one write of x at the end.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include <type_traits>

#include "df_fused.cuh"
#include "df_sync.cuh"

namespace df {

namespace {

constexpr int kRThreads = 512;
constexpr int kRQ = 4;
constexpr int kHalo = 9;  // halo arrays of W floats kept in shared memory
constexpr int kFlagWords = 4;  // u64 words per CTA edge flag (one 32-byte sector)

struct ResKf {
  Planes pl;
  int cta_begin, cta_end;  // CTAs of this keyframe
};

struct ResCta {
  int kf, rb, re, pad;
};

struct ResSeg {
  double t, bb, rr;
  ff2 gam, alpha, beta;  // CG scalars (double-float)
  // joint (x, t) solve: the border components of the CG vectors and the
  // change of t during the current depth step (folded into t at its end)
  ff2 jS, jrt, jut, jwt, jpt, jst, jdt;
  int stop, iters, active, pad;
};

// What the halo stage arrays are loaded with right after an exchange, for
// the pass that follows it.
enum HaloKind : int { HK_NONE = 0, HK_X, HK_INIT, HK_ITER };

// Shared-memory arrays of one band (stride BS floats each): x, r, p, s, w,
// 1/diag, wx, wy, u; when the plan stages the inputs, IN[0..7] = mu_n,
// var_n, gx, var_gx, gy, var_gy, mu_s, var_s of the band (as f32). Then the
// halo arrays (W floats each): HA[0..3] the row above the band, HA[4..7] the
// row below, WYT the y-coupling of the row above, and with staged inputs
// GYT / VYT, gy and var_gy of the row above.
constexpr int kIn = 8;  // staged input planes
enum : int { I_MN = 0, I_VN, I_GX, I_VX, I_GY, I_VY, I_MS, I_VS };

struct Smem {
  float *X, *R, *P, *S, *Wv, *ID, *WX, *WY, *U;
  float *IN[kIn];
  float *HA[8];
  float *WYT, *GYT, *VYT;
};

__device__ __forceinline__ Smem smem_of(float *base, int stride, int W, bool in_smem) {
  Smem m;
  float *p = base;
  m.X = p; p += stride;
  m.R = p; p += stride;
  m.P = p; p += stride;
  m.S = p; p += stride;
  m.Wv = p; p += stride;
  m.ID = p; p += stride;
  m.WX = p; p += stride;
  m.WY = p; p += stride;
  m.U = p; p += stride;
  for (int j = 0; j < kIn; ++j) {
    m.IN[j] = in_smem ? p : nullptr;
    if (in_smem) p += stride;
  }
  for (int j = 0; j < 8; ++j) { m.HA[j] = p; p += W; }
  m.WYT = p; p += W;
  m.GYT = in_smem ? p : nullptr;
  if (in_smem) p += W;
  m.VYT = in_smem ? p : nullptr;
  return m;
}

// Per-thread walk over the band's pixels q = tid, tid + T, ... with the row
// and column kept incrementally (no integer division per pixel).
struct Walk {
  int q, v, u, dv, du, W, step;
  __device__ __forceinline__ Walk(int W_, int t = threadIdx.x, int step_ = kRThreads)
      : W(W_), step(step_) {
    q = t;
    v = q / W;
    u = q - v * W;
    dv = step / W;
    du = step - dv * W;
  }
  __device__ __forceinline__ void next() {
    q += step;
    v += dv;
    u += du;
    if (u >= W) {
      u -= W;
      ++v;
    }
  }
};

// Walks the band two pixels per step: eval(q, u, v, out) only loads from
// shared memory, commit(q, u, v, out) stores, so the two pixels' load and
// arithmetic chains overlap (a store between them would order every later
// shared-memory load after it). Per thread the pixels are committed in walk
// order, so every per-thread partial sum is added in the same order as a
// one-pixel walk.
template <class T, class Eval, class Commit>
__device__ __forceinline__ void walk_pairs(int W, int bp, Eval &&eval, Commit &&commit) {
  Walk it(W);
  for (; it.q + kRThreads < bp;) {
    const int qa = it.q, ua = it.u, va = it.v;
    it.next();
    const int qb = it.q, ub = it.u, vb = it.v;
    it.next();
    T a, b;
    eval(qa, ua, va, a);
    eval(qb, ub, vb, b);
    commit(qa, ua, va, a);
    commit(qb, ub, vb, b);
  }
  if (it.q < bp) {
    T a;
    eval(it.q, it.u, it.v, a);
    commit(it.q, it.u, it.v, a);
  }
}

// w = A u = r - N u for the band (A = diag - N; u = r / diag exactly, so
// diag * u is r). Halo u: HA[0] above, HA[4] below; y-coupling of the row
// above the band in WYT. Accumulates (r, u), (w, u), (r, r). The band's edge
// rows of w also go to wpub (global plane, rows rb and rb + nr - 1) as they
// are formed, for the neighbouring bands.
__device__ __forceinline__ void apply_band(const Smem &m, int W, int nr, int bp, bool has_below,
                                           float acc[kRQ], float *wpub, int rb, size_t P) {
  struct Px {
    float r, uq, w;
  };
  walk_pairs<Px>(
      W, bp,
      [&](int q, int u, int v, Px &o) {
        o.uq = m.U[q];
        float nu = 0.0f;
        if (u < W - 1) nu += m.WX[q] * m.U[q + 1];
        if (u > 0) nu += m.WX[q - 1] * m.U[q - 1];
        if (v < nr - 1) {
          nu += m.WY[q] * m.U[q + W];
        } else if (has_below) {
          nu += m.WY[q] * m.HA[4][u];
        }
        nu += (v > 0) ? m.WY[q - W] * m.U[q - W] : m.WYT[u] * m.HA[0][u];
        o.r = m.R[q];
        o.w = o.r - nu;
      },
      [&](int q, int u, int v, const Px &o) {
        m.Wv[q] = o.w;
        if (v == 0 || v == nr - 1) __stcg(wpub + (size_t)(rb + v) * P + u, o.w);
        acc[0] += o.r * o.uq;
        acc[1] += o.w * o.uq;
        acc[2] += o.r * o.r;
      });
}

// Joint (x, t) variant of apply_band: w = A u - ws u_t with u = r / diag
// formed on the fly (the U array holds ws, the semi-dense weights). Halo u as
// in apply_band. Accumulates (r, u), (w, u), (r, r) and (ws, u).
__device__ __forceinline__ void apply_band_joint(const Smem &m, int W, int nr, int bp,
                                                 bool has_below, float ut, float acc[kRQ]) {
  for (Walk it(W); it.q < bp; it.next()) {
    const int q = it.q, u = it.u, v = it.v;
    const float r = m.R[q];
    const float uq = r * m.ID[q];
    float nu = 0.0f;
    if (u < W - 1) nu += m.WX[q] * (m.R[q + 1] * m.ID[q + 1]);
    if (u > 0) nu += m.WX[q - 1] * (m.R[q - 1] * m.ID[q - 1]);
    if (v < nr - 1) {
      nu += m.WY[q] * (m.R[q + W] * m.ID[q + W]);
    } else if (has_below) {
      nu += m.WY[q] * m.HA[4][u];
    }
    nu += (v > 0) ? m.WY[q - W] * (m.R[q - W] * m.ID[q - W]) : m.WYT[u] * m.HA[0][u];
    const float ws = m.U[q];
    const float w = r - nu - ws * ut;
    m.Wv[q] = w;
    acc[0] += r * uq;
    acc[1] += w * uq;
    acc[2] += r * r;
    acc[3] += ws * uq;
  }
}

// Write the band's first and last rows of a shared array to a global plane.
__device__ __forceinline__ void publish_edges(const float *src, float *dst, int W, int nr, int rb,
                                              size_t P) {
  for (int u = threadIdx.x; u < W; u += kRThreads) {
    __stcg(dst + (size_t)rb * P + u, src[u]);
    if (nr > 1) __stcg(dst + (size_t)(rb + nr - 1) * P + u, src[(nr - 1) * W + u]);
  }
}

// Input plane j (I_MN .. I_VS) at band pixel q / global index gi: from the
// band's staged copy (SM) or from the keyframe's planes.
template <bool SM, int DT>
__device__ __forceinline__ float band_in(const Smem &m, const Planes &k, int j, int q, size_t gi) {
  if constexpr (SM) {
    return m.IN[j][q];
  } else {
    if (j == I_MS) return __ldg(k.mu_s + gi);
    if (j == I_VS) return __ldg(k.var_s + gi);
    return ld_cnn<DT>(k.cnn[j], gi);
  }
}

// Copy the band's input planes (and gy, var_gy of the row above) into shared
// memory, as f32; they are constant for the whole launch.
template <int DT>
__device__ void stage_inputs(const Smem &m, const Planes &k, int rb, int bp, bool has_above) {
  const int W = k.W;
  const size_t P = k.P;
  for (Walk it(W); it.q < bp; it.next()) {
    const size_t gi = (size_t)(rb + it.v) * P + it.u;
    float v[kIn];
#pragma unroll
    for (int j = 0; j < 6; ++j) v[j] = ld_cnn<DT>(k.cnn[j], gi);
    v[I_MS] = __ldg(k.mu_s + gi);
    v[I_VS] = __ldg(k.var_s + gi);
#pragma unroll
    for (int j = 0; j < kIn; ++j) m.IN[j][it.q] = v[j];
  }
  for (int u = threadIdx.x; u < W; u += kRThreads) {
    const size_t gi = (size_t)(rb - 1) * P + u;
    m.GYT[u] = has_above ? ld_cnn<DT>(k.cnn[I_GY], gi) : 0.0f;
    m.VYT[u] = has_above ? ld_cnn<DT>(k.cnn[I_VY], gi) : 1.0f;
  }
}

// The assembly in two parts. assemble_pre needs only the band's x and its
// inputs: the x-terms, the y-terms inside the band and the prior term, so
// it can run while the previous pass's sums are still being exchanged
// (threads t, t + nt, ...). wx, wy, ex, ey go to WX, WY, P, S (p and s are
// free during assembly), the prior's weight wn and residual part
// wn (mu_n - x) to ID and R.
template <int DT, int LK, bool SM>
__device__ void assemble_pre(const Smem &m, const Planes &k, int rb, int nr, const SolveCfg &c,
                             int t, int nt) {
  const int W = k.W, H = k.H, bp = nr * W;
  const size_t P = k.P;
  const bool net = c.terms & DF_TERM_NET, grad = c.terms & DF_TERM_GRAD;
  auto in = [&](int j, int q, size_t gi) { return band_in<SM, DT>(m, k, j, q, gi); };
  for (Walk it(W, t, nt); it.q < bp; it.next()) {
    const int q = it.q, u = it.u, v = it.v;
    const size_t gi = (size_t)(rb + v) * P + u;
    const float xq = m.X[q];
    float wx = 0.0f, ex = 0.0f, wy = 0.0f, ey = 0.0f;
    if (grad && u < W - 1) {
      ex = m.X[q + 1] - xq - in(I_GX, q, gi);
      wx = robust_weight_k<LK>(ex, in(I_VX, q, gi), c.delta);
    }
    if (grad && v < nr - 1 && rb + v < H - 1) {  // the last row's y-term needs the halo
      ey = m.X[q + W] - xq - in(I_GY, q, gi);
      wy = robust_weight_k<LK>(ey, in(I_VY, q, gi), c.delta);
    }
    float wn = 0.0f, rn = 0.0f;
    if (net) {
      const float mn = in(I_MN, q, gi);
      wn = robust_weight_k<LK>(xq - mn, in(I_VN, q, gi), c.delta);
      rn = wn * (mn - xq);
    }
    m.WX[q] = wx;
    m.WY[q] = wy;
    m.P[q] = ex;
    m.S[q] = ey;
    m.ID[q] = wn;
    m.R[q] = rn;
  }
}

// The rest of the assembly, once t and the x halo (HA[0] above, HA[4]
// below) are known: the last row's y-term, the y-term above the band, the
// semi-dense term, then 1/diag and r0 = b - A x in residual form.
// JOINT: also keep ws in the U array and sum the border's S = sum ws and
// r_t = sum ws (x - t - mu_s) into acc[2], acc[3] (b.b is not formed: the
// joint solve runs with a fixed iteration count here). SM: the inputs are
// staged in shared memory (DT is then unused).
template <int DT, bool JOINT, int LK, bool SM>
__device__ void assemble_post(const Smem &m, const Planes &k, int rb, int nr, float t,
                              const SolveCfg &c, float acc[kRQ], float *rpub, float *idpub) {
  const int W = k.W, H = k.H, bp = nr * W;
  const size_t P = k.P;
  const bool semi = c.terms & DF_TERM_SEMI, net = c.terms & DF_TERM_NET,
             grad = c.terms & DF_TERM_GRAD;
  const bool has_above = rb > 0;
  auto in = [&](int j, int q, size_t gi) { return band_in<SM, DT>(m, k, j, q, gi); };
  for (int u = threadIdx.x; u < W; u += kRThreads) {
    {  // the band's last row: its y-term reaches the row below
      const int v = nr - 1, q = v * W + u;
      const size_t gi = (size_t)(rb + v) * P + u;
      float wy = 0.0f, ey = 0.0f;
      if (grad && rb + v < H - 1) {
        ey = m.HA[4][u] - m.X[q] - in(I_GY, q, gi);
        wy = robust_weight_k<LK>(ey, in(I_VY, q, gi), c.delta);
      }
      m.WY[q] = wy;
      m.S[q] = ey;
    }
    float wy = 0.0f, ey = 0.0f, gy = 0.0f;
    if (grad && has_above) {
      const size_t gi = (size_t)(rb - 1) * P + u;
      float vy;
      if constexpr (SM) {
        gy = m.GYT[u];
        vy = m.VYT[u];
      } else {
        gy = ld_cnn<DT>(k.cnn[I_GY], gi);
        vy = ld_cnn<DT>(k.cnn[I_VY], gi);
      }
      ey = m.X[u] - m.HA[0][u] - gy;
      wy = robust_weight_k<LK>(ey, vy, c.delta);
    }
    m.WYT[u] = wy;
    m.HA[1][u] = ey;
    m.HA[2][u] = gy;
  }
  __syncthreads();
  for (Walk it(W); it.q < bp; it.next()) {
    const int q = it.q, u = it.u, v = it.v;
    const size_t gi = (size_t)(rb + v) * P + u;
    const float xq = m.X[q];
    float ws = 0.0f, rs = 0.0f, bs = 0.0f;
    if (semi) {
      const float ms = in(I_MS, q, gi), vs = in(I_VS, q, gi);
      if (semi_valid(ms, vs)) {
        ws = robust_weight_k<LK>(xq - t - ms, vs, c.delta);
        rs = ws * (t + ms - xq);
        bs = ws * (t + ms);
      }
    }
    const float wn = m.ID[q], rn = m.R[q];
    const float wx = m.WX[q], ex = m.P[q], wy = m.WY[q], ey = m.S[q];
    const float wxl = u > 0 ? m.WX[q - 1] : 0.0f, exl = u > 0 ? m.P[q - 1] : 0.0f;
    const float wyu = v > 0 ? m.WY[q - W] : m.WYT[u], eyu = v > 0 ? m.S[q - W] : m.HA[1][u];
    const float d = ws + wn + wx + wxl + wy + wyu;
    const float r = rs + rn + wx * ex - wxl * exl + wy * ey - wyu * eyu;
    const float id = inv_diag(d);
    acc[0] += r * (r * id);
    acc[1] += r * r;
    if (JOINT) {
      acc[2] += ws;
      acc[3] -= rs;  // ws (x - t - mu_s)
    } else if (c.tol > 0.0) {
      const float mn = net ? in(I_MN, q, gi) : 0.0f;
      const float gx = (grad && u < W - 1) ? in(I_GX, q, gi) : 0.0f;
      const float gxl = (grad && u > 0) ? in(I_GX, q - 1, gi - 1) : 0.0f;
      const float gy = (grad && rb + v < H - 1) ? in(I_GY, q, gi) : 0.0f;
      const float gyu = v > 0 ? ((grad) ? in(I_GY, q - W, gi - P) : 0.0f) : m.HA[2][u];
      const float b = bs + wn * mn - wx * gx + wxl * gxl - wy * gy + wyu * gyu;
      acc[2] += b * b;
    }
    m.ID[q] = id;
    m.R[q] = r;
    if (JOINT) m.U[q] = ws;
    if (v == 0 || v == nr - 1) {  // the edge rows, for the neighbouring bands
      __stcg(rpub + gi, r);
      __stcg(idpub + gi, id);
    }
  }
}

template <int N>
using IC = std::integral_constant<int, N>;

// JOINT: the joint (x, t) variant (c.scale_step == DF_SCALE_JOINT with the
// semi-dense term); the alternating solve is the other instance. LK: the
// loss kind (least squares, Huber, Tukey), fixed per instance.
template <bool JOINT, int LK>
__global__ void __launch_bounds__(kRThreads, 1)
    k_resident(PlanHeader *h, SolveCfg c, int n_gn, int n_pcg, unsigned long long limit_ns,
               int first) {
  extern __shared__ float4 dyn_smem[];
  __shared__ ff2 s_red[32 * kRQ];
  __shared__ long long s_dig[kRQ][kSumDigits];
  __shared__ ff2 s_tot[kRQ];  // this pass's totals
  __shared__ int s_ok;
  __shared__ SumPrev s_prev;
  __shared__ ResKf s_kf;
  __shared__ ResSeg s_seg;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = h->G;
  const char *hb = reinterpret_cast<const char *>(h);
  const ResCta *ctas = reinterpret_cast<const ResCta *>(hb + h->off_cta_work);
  const ResKf *kfs = reinterpret_cast<const ResKf *>(hb + h->off_kf);
  const ResCta me = ctas[blockIdx.x];
  if (tid == 0) {
    s_kf = kfs[me.kf];
    const Scalars *sc = s_kf.pl.sc;
    s_seg.t = sc->t;
    s_seg.gam = s_seg.alpha = s_seg.beta = ff2{0.0f, 0.0f};
    s_seg.jS = s_seg.jrt = s_seg.jut = s_seg.jwt = s_seg.jpt = s_seg.jst = s_seg.jdt =
        ff2{0.0f, 0.0f};
    s_seg.bb = 0.0;
    s_seg.rr = sc->rr;
    s_seg.stop = 0;
    s_seg.iters = first ? 0 : sc->iters;
    s_seg.active = (sc->flags & kFlagBadInput) ? 0 : 1;
  }
  for (int i = tid; i < 2 * kSumQ * kSumDigits; i += kRThreads) (&s_prev.v[0][0][0])[i] = 0ull;
  __syncthreads();
  const Planes &k = s_kf.pl;
  const int W = k.W, H = k.H;
  const size_t P = k.P;
  const int rb = me.rb, nr = me.re - me.rb, bp = nr * W;
  const bool has_above = rb > 0, has_below = me.re < H;
  const bool in_sm = h->in_smem != 0;
  const Smem m = smem_of(reinterpret_cast<float *>(dyn_smem), h->th, W, in_sm);
  float *Rg[2] = {k.v[1], k.v[2]}, *Sg[2] = {k.v[3], k.v[4]}, *Wg[2] = {k.v[5], k.v[6]};
  float *IDg = k.diag;  // the fused kernels keep 1/diag in the diag plane
  const bool active = s_seg.active != 0;
  const bool do_scale = (c.terms & DF_TERM_SEMI) && c.scale_step == DF_SCALE_ALTERNATE;
  constexpr bool joint = JOINT;
  int parity = 0;
  bool alive = true;

  for (Walk it(W); it.q < bp; it.next()) m.X[it.q] = __ldcg(k.x + (size_t)(rb + it.v) * P + it.u);
  if (in_sm && active) {
    if (k.dtype == DF_BF16)
      stage_inputs<DF_BF16>(m, k, rb, bp, has_above);
    else if (k.dtype == DF_F16)
      stage_inputs<DF_F16>(m, k, rb, bp, has_above);
    else
      stage_inputs<DF_F32>(m, k, rb, bp, has_above);
  }

  // Load the halo rows the next pass needs (raw values; the new u of the
  // rows above / below needs this pass's alpha, beta and is formed there).
  // called by threads [t0, kRThreads)
  auto prefetch_halo = [&](int kind, int cb, int t0 = 32) {
    if (!active || kind == HK_NONE) return;
    const size_t ia = (size_t)(rb - 1) * P, ib = (size_t)(rb + nr) * P;
    const int nt = kRThreads - t0;
    const float *Rc = kind == HK_INIT ? Rg[0] : Rg[cb];
    // two columns per thread and round: both columns' loads are issued
    // before either is stored, so a round costs one L2 round trip
    for (int u0 = tid - t0; u0 < W; u0 += 2 * nt) {
      float a[2][4] = {}, b[2][4] = {};
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int u = u0 + h2 * nt;
        if (u >= W) continue;
        if (kind == HK_X) {
          if (has_above) a[h2][0] = __ldcg(k.x + ia + u);
          if (has_below) b[h2][0] = __ldcg(k.x + ib + u);
        } else {
          if (has_above) {
            a[h2][0] = __ldcg(Rc + ia + u);
            a[h2][3] = __ldcg(IDg + ia + u);
            if (kind == HK_ITER) {
              a[h2][1] = __ldcg(Sg[cb] + ia + u);
              a[h2][2] = __ldcg(Wg[cb] + ia + u);
            }
          }
          if (has_below) {
            b[h2][0] = __ldcg(Rc + ib + u);
            b[h2][3] = __ldcg(IDg + ib + u);
            if (kind == HK_ITER) {
              b[h2][1] = __ldcg(Sg[cb] + ib + u);
              b[h2][2] = __ldcg(Wg[cb] + ib + u);
            }
          }
        }
      }
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int u = u0 + h2 * nt;
        if (u >= W) continue;
        m.HA[0][u] = a[h2][0];
        m.HA[4][u] = b[h2][0];
        if (kind != HK_X) {
          m.HA[1][u] = a[h2][1]; m.HA[2][u] = a[h2][2]; m.HA[3][u] = a[h2][3];
          m.HA[5][u] = b[h2][1]; m.HA[6][u] = b[h2][2]; m.HA[7][u] = b[h2][3];
        }
      }
    }
  };

  // Deferred halo (the first CG pass and the CG iterations, keyframes up to
  // 2 x 480 pixels wide): right after the exchange, threads 32.. issue the
  // loads of the raw halo values of up to two columns each into registers
  // hv; they store the halo's new u into HA[0] / HA[4] only after the pass's
  // vector update, which needs no halo, so the loads' round trip overlaps
  // the CG scalars and that update instead of preceding them.
  float hv[2][8];
  bool halo_deferred = false;
  const bool can_defer = W <= 2 * (kRThreads - 32);
  auto halo_issue = [&](int kind, int cb) {
    if (!active) return;
    const size_t ia = (size_t)(rb - 1) * P, ib = (size_t)(rb + nr) * P;
    const float *Rc = kind == HK_INIT ? Rg[0] : Rg[cb];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
#pragma unroll
      for (int j = 0; j < 8; ++j) hv[h2][j] = 0.0f;
      const int u = tid - 32 + h2 * (kRThreads - 32);
      if (u >= W) continue;
      if (has_above) {
        hv[h2][0] = __ldcg(Rc + ia + u);
        hv[h2][3] = __ldcg(IDg + ia + u);
        if (kind == HK_ITER) {
          hv[h2][1] = __ldcg(Sg[cb] + ia + u);
          hv[h2][2] = __ldcg(Wg[cb] + ia + u);
        }
      }
      if (has_below) {
        hv[h2][4] = __ldcg(Rc + ib + u);
        hv[h2][7] = __ldcg(IDg + ib + u);
        if (kind == HK_ITER) {
          hv[h2][5] = __ldcg(Sg[cb] + ib + u);
          hv[h2][6] = __ldcg(Wg[cb] + ib + u);
        }
      }
    }
  };
  // the halo's new u: r' = r - alpha (w + beta s), u' = r' / diag (CG
  // iterations; the arithmetic of the in-place update below), or u0 = r0 /
  // diag (the first CG pass)
  auto halo_store = [&](bool iter, bool first_it, float fa_, float fb_) {
    if (tid < 32) return;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int u = tid - 32 + h2 * (kRThreads - 32);
      if (u >= W) continue;
      if (iter) {
        const float sa = first_it ? hv[h2][2] : hv[h2][2] + fb_ * hv[h2][1];
        m.HA[0][u] = (hv[h2][0] - fa_ * sa) * hv[h2][3];
        const float sb = first_it ? hv[h2][6] : hv[h2][6] + fb_ * hv[h2][5];
        m.HA[4][u] = (hv[h2][4] - fa_ * sb) * hv[h2][7];
      } else {
        m.HA[0][u] = hv[h2][0] * hv[h2][3];
        m.HA[4][u] = hv[h2][4] * hv[h2][7];
      }
    }
  };

  // partial sums -> exact sum words -> prefetch next halo + this keyframe's totals.
  // Reductions: every CTA of a keyframe adds its double-float partials into
  // the keyframe's fixed-point sum words (a fence first, so its band edges
  // are visible to whoever sees the arrival) and polls them until all of the
  // keyframe's CTAs have arrived; the total is exact and identical
  // everywhere. No grid barrier: a keyframe's CTAs wait only for each other.
  const int nk = s_kf.cta_end - s_kf.cta_begin;
  SumGroup *groups = reinterpret_cast<SumGroup *>(reinterpret_cast<char *>(h) + h->off_slots);
  SumGroup *grp = groups + me.kf;
  unsigned long long *flags =
      reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(h) + h->off_flags);
  // test hook: never arrive (nor raise the CTA's edge flag)
  const bool skip_me = (int)blockIdx.x == h->debug_skip_cta;
  // nq: std::integral_constant with the number of sums this pass needs
  // (acc[0 .. NQ-1]). post() runs on thread 0 once the totals are in s_tot,
  // while the other warps load the next pass's halo; its writes to s_seg are
  // visible to every thread when end_pass returns.
  // The part of the next assembly that needs neither t nor the x halo, on
  // threads t, t + nt, ... (see assemble_pre).
  auto pre_assemble = [&](int t, int nt) {
    if (!active) return;
    if (in_sm)
      assemble_pre<DF_F32, LK, true>(m, k, rb, nr, c, t, nt);
    else if (k.dtype == DF_BF16)
      assemble_pre<DF_BF16, LK, false>(m, k, rb, nr, c, t, nt);
    else if (k.dtype == DF_F16)
      assemble_pre<DF_F16, LK, false>(m, k, rb, nr, c, t, nt);
    else
      assemble_pre<DF_F32, LK, false>(m, k, rb, nr, c, t, nt);
  };
  // overlap_pre: the pass that ends here is followed by an assembly, whose
  // first part the warps other than warp 0 run while warp 0 exchanges the
  // sums (the pass's own reads of the band arrays are done by then).
  bool overlap_pre = false, pre_done = false;
  auto end_pass = [&](auto nq, const float *acc, int next_halo, int next_cb,
                      auto &&post) -> bool {
    constexpr int NQ = decltype(nq)::value;
    // the CTA tree: a warp tree per quantity, then warp 1 + q adds quantity
    // q over the warps and writes its digits while warp 0 runs the release
    // fence of the pass's edge stores (the barrier before orders every
    // warp's stores first)
    {
      ff2 sw[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) sw[q] = ff2{acc[q], 0.0f};
      warp_sum_ff_n<NQ>(sw);
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) s_red[warp * NQ + q] = sw[q];
      }
    }
    __syncthreads();
    if (warp == 0) {
      fence_acq_rel_gpu();
    } else if (warp <= NQ) {
      const int q = warp - 1;
      const ff2 x = lane < kRThreads / 32 ? s_red[lane * NQ + q] : ff2{0.0f, 0.0f};
      const ff2 tq = warp_sum_ff(x);
      const ff2 tb = ff2{__shfl_sync(0xffffffffu, tq.hi, 0), __shfl_sync(0xffffffffu, tq.lo, 0)};
      if (lane < kSumDigits) s_dig[q][lane] = ff_digit(tb, lane);
    }
    __syncthreads();
    long long digit = 0;
    if (warp == 0) {
      bool ok = false;
      if (!skip_me) {
        sum_push_digits(grp, parity, s_dig, NQ);
        ok = sum_wait(grp, parity, nk, NQ, &s_prev, h, limit_ns, &digit);
      }
      if (lane == 0) s_ok = ok ? 1 : 0;
    } else if (overlap_pre) {
      pre_assemble(tid - 32, kRThreads - 32);
    }
    pre_done = overlap_pre;
    overlap_pre = false;
    halo_deferred = can_defer && (next_halo == HK_INIT || next_halo == HK_ITER);
    __syncthreads();
    if (!s_ok) return false;
    // warp 0 forms the totals and the pass's scalars; the other warps load
    // the halo
    if (warp == 0) {
      const ff2 tot = sum_total(digit);
      if ((lane & 7) == 0 && (lane >> 3) < NQ) s_tot[lane >> 3] = tot;
      __syncwarp();
      if (lane == 0) post();
    } else {
      if (halo_deferred)
        halo_issue(next_halo, next_cb);
      else
        prefetch_halo(next_halo, next_cb, 32);
    }
    __syncthreads();
    parity ^= 1;
    return true;
  };

  auto scale_partials = [&](float acc[kRQ], int q0, float t) {
    for (Walk it(W); it.q < bp; it.next()) {
      const size_t gi = (size_t)(rb + it.v) * P + it.u;
      const float ms = in_sm ? m.IN[I_MS][it.q] : __ldg(k.mu_s + gi);
      const float vs = in_sm ? m.IN[I_VS][it.q] : __ldg(k.var_s + gi);
      if (semi_valid(ms, vs)) {
        const float xq = m.X[it.q];
        const float w = robust_weight_k<LK>(xq - t - ms, vs, c.delta);
        acc[q0] += w;
        acc[q0 + 1] += w * (xq - ms);
      }
    }
  };
  // thread 0: the scale step's t from the sums s_tot[qw], s_tot[qwr]
  auto scale_update = [&](int qw, int qwr) {
    if (s_seg.active && s_tot[qw].hi > 0.0f) s_seg.t = ff_to_double(ff_div(s_tot[qwr], s_tot[qw]));
  };

  // The border of the joint solve moves with the iteration's alpha, beta
  // (thread 0, right after they are formed): p_t = u_t + beta p_t,
  // s_t = w_t + beta s_t, t += alpha p_t, r_t -= alpha s_t, u_t = r_t / S.
  auto joint_border_step = [&](bool first_it) {
    const ff2 a = s_seg.alpha;
    s_seg.jpt = first_it ? s_seg.jut : ff_add(s_seg.jut, ff_mul(s_seg.beta, s_seg.jpt));
    s_seg.jst = first_it ? s_seg.jwt : ff_add(s_seg.jwt, ff_mul(s_seg.beta, s_seg.jst));
    s_seg.jdt = ff_add(s_seg.jdt, ff_mul(a, s_seg.jpt));
    s_seg.jrt = ff_sub(s_seg.jrt, ff_mul(a, s_seg.jst));
    s_seg.jut = s_seg.jS.hi > 0.0f ? ff_div(s_seg.jrt, s_seg.jS) : ff2{0.0f, 0.0f};
  };

  // the first pass is either the scale step or the assembly; both need the
  // x halo, which is current in global memory at launch
  prefetch_halo(HK_X, 0, 0);
  __syncthreads();

  bool scale_pending = false;
  for (int gn = 0; gn < n_gn && alive; ++gn) {
    if (do_scale) {
      if (!scale_pending) {
        float acc[kRQ] = {};
        if (active) scale_partials(acc, 0, (float)s_seg.t);
        overlap_pre = true;
        if (!(alive = end_pass(IC<2>{}, acc, HK_X, 0, [&] { scale_update(0, 1); }))) break;
      }
      scale_pending = false;
    }
    // Without the joint solve, the first CG pass needs of the assembly only
    // the neighbouring bands' edge rows of r0 and 1/diag; its sums are not
    // used before that pass's scalars. So the assembly ends in an edge
    // hand-off with the two neighbours instead of an exchange, and its sums
    // travel with the first CG pass's.
    const bool merged = !JOINT && n_pcg > 0;
    float asm_acc[kRQ] = {};
    {  // ASSEMBLE
      float acc[kRQ] = {};
      if (active) {
        const float t = (float)s_seg.t;
        if (!pre_done) {  // no exchange before it to hide the first part in
          pre_assemble(tid, kRThreads);
          __syncthreads();
        }
        if (in_sm)
          assemble_post<DF_F32, JOINT, LK, true>(m, k, rb, nr, t, c, acc, Rg[0], IDg);
        else if (k.dtype == DF_BF16)
          assemble_post<DF_BF16, JOINT, LK, false>(m, k, rb, nr, t, c, acc, Rg[0], IDg);
        else if (k.dtype == DF_F16)
          assemble_post<DF_F16, JOINT, LK, false>(m, k, rb, nr, t, c, acc, Rg[0], IDg);
        else
          assemble_post<DF_F32, JOINT, LK, false>(m, k, rb, nr, t, c, acc, Rg[0], IDg);
      }
      // sums needed: r.z; r.r and b.b only for a tolerance or a report
      // without CG iterations; the joint solve also S and r_t
      const int next_a = n_pcg > 0 ? HK_INIT : HK_X;
      const bool wide = c.tol > 0.0 || n_pcg == 0;
      auto post = [&] {
        if constexpr (JOINT) {
          // border of the bordered system: S = sum ws, r_t, u_t = r_t / S
          const ff2 S = s_tot[2], rt = s_tot[3];
          const ff2 ut = S.hi > 0.0f ? ff_div(rt, S) : ff2{0.0f, 0.0f};
          s_seg.jS = S;
          s_seg.jrt = rt;
          s_seg.jut = ut;
          s_seg.jdt = ff2{0.0f, 0.0f};
          s_seg.gam = ff_add(s_tot[0], ff_mul(rt, ut));
          s_seg.rr = ff_to_double(ff_add(s_tot[1], ff_mul(rt, rt)));
          s_seg.stop = 0;
        } else {
          s_seg.gam = s_tot[0];
          s_seg.stop = 0;
          if (wide) {
            s_seg.rr = ff_to_double(s_tot[1]);
            s_seg.bb = ff_to_double(s_tot[2]);
            s_seg.stop = (c.tol > 0.0 && sqrt(s_seg.rr) < c.tol * sqrt(s_seg.bb)) ? 1 : 0;
          }
        }
      };
      if (merged) {
#pragma unroll
        for (int q = 0; q < kRQ; ++q) asm_acc[q] = acc[q];
        if (tid == 0) s_seg.stop = 0;
        __syncthreads();  // the band's r0, 1/diag and its edge stores are done
        if (warp == 0) {
          bool ok = true;
          if (active) {
            const unsigned long long e = (unsigned long long)gn + 1ull;
            if (lane == 0 && !skip_me) edge_flag_raise(flags + kFlagWords * blockIdx.x, e);
            const unsigned long long *nbr = nullptr;
            if (lane == 0 && has_above) nbr = flags + kFlagWords * (blockIdx.x - 1);
            if (lane == 1 && has_below) nbr = flags + kFlagWords * (blockIdx.x + 1);
            ok = edge_flags_wait(nbr, e, h, limit_ns);
          }
          if (lane == 0) s_ok = ok ? 1 : 0;
        } else if (active) {  // u0 = r0 / diag of the band, meanwhile
          for (int q = tid - 32; q < bp; q += kRThreads - 32) m.U[q] = m.R[q] * m.ID[q];
        }
        halo_deferred = can_defer;
        __syncthreads();
        if (!s_ok) {
          alive = false;
          break;
        }
        if (halo_deferred) {
          halo_issue(HK_INIT, 0);
        } else {
          prefetch_halo(HK_INIT, 0, 0);
          __syncthreads();
        }
      } else {
        if constexpr (JOINT) {
          alive = end_pass(IC<4>{}, acc, next_a, 0, post);
        } else {
          alive = wide ? end_pass(IC<3>{}, acc, next_a, 0, post)
                       : end_pass(IC<1>{}, acc, next_a, 0, post);
        }
        if (!alive) break;
      }
    }
    if (n_pcg == 0) continue;  // no depth update in this GN iteration
    {  // INIT: w0 = A u0
      float acc[kRQ] = {};
      if (active && !s_seg.stop) {
        if (!halo_deferred) {
          for (int u = tid; u < W; u += kRThreads) {
            m.HA[0][u] = m.HA[0][u] * m.HA[3][u];
            m.HA[4][u] = m.HA[4][u] * m.HA[7][u];
          }
        }
        if constexpr (JOINT) {
          if (halo_deferred) halo_store(false, false, 0.0f, 0.0f);
          __syncthreads();
          apply_band_joint(m, W, nr, bp, has_below, s_seg.jut.hi, acc);
        } else {
          if (!merged)
            walk_pairs<float>(
                W, bp, [&](int q, int, int, float &o) { o = m.R[q] * m.ID[q]; },
                [&](int q, int, int, float o) { m.U[q] = o; });
          if (halo_deferred) halo_store(false, false, 0.0f, 0.0f);
          __syncthreads();
          apply_band(m, W, nr, bp, has_below, acc, Wg[0], rb, P);
        }
        if constexpr (JOINT) {
          __syncthreads();
          publish_edges(m.Wv, Wg[0], W, nr, rb, P);
        }
      }
      // sums needed: (w0, u0); the joint solve also (ws, u0)
      const int next_i = n_pcg > 1 ? HK_ITER : HK_NONE;
      auto post = [&] {
        if (merged) {  // the assembly's sums (its exchange's scalars)
          s_seg.gam = s_tot[0];
          if (c.tol > 0.0) {
            s_seg.rr = ff_to_double(s_tot[2]);
            s_seg.bb = ff_to_double(s_tot[3]);
            s_seg.stop = (c.tol > 0.0 && sqrt(s_seg.rr) < c.tol * sqrt(s_seg.bb)) ? 1 : 0;
          }
        }
        if (s_seg.stop) return;
        ff2 dl = merged ? s_tot[1] : s_tot[0];
        if constexpr (JOINT) {  // w_t = S u_t - (ws, u); (w, u) gains w_t u_t
          s_seg.jwt = ff_sub(ff_mul(s_seg.jS, s_seg.jut), s_tot[1]);
          dl = ff_add(dl, ff_mul(s_seg.jwt, s_seg.jut));
        }
        if (s_seg.gam.hi == 0.0f || !(dl.hi > 0.0f)) {
          s_seg.stop = 1;
        } else {
          s_seg.alpha = ff_div(s_seg.gam, dl);
          s_seg.beta = ff2{0.0f, 0.0f};
          if constexpr (JOINT) joint_border_step(true);
        }
      };
      if constexpr (JOINT) {
        const float a2[2] = {acc[1], acc[3]};
        alive = end_pass(IC<2>{}, a2, next_i, 0, post);
      } else if (merged) {  // (r0, u0) [, r0.r0, b.b] of the assembly, (w0, u0)
        if (c.tol > 0.0) {
          const float a4[4] = {asm_acc[0], acc[1], asm_acc[1], asm_acc[2]};
          alive = end_pass(IC<4>{}, a4, next_i, 0, post);
        } else {
          const float a2[2] = {asm_acc[0], acc[1]};
          alive = end_pass(IC<2>{}, a2, next_i, 0, post);
        }
      } else {
        alive = end_pass(IC<1>{}, acc + 1, next_i, 0, post);
      }
      if (!alive) break;
    }
    for (int it = 0; it < n_pcg && alive; ++it) {
      const int cb = it & 1, nb = cb ^ 1;
      // hi is the float nearest to a double-float value
      const float fa = s_seg.alpha.hi, fb = s_seg.beta.hi;
      const bool first = it == 0;
      const bool run = active && !s_seg.stop;
      float acc[kRQ] = {};
      if (it == n_pcg - 1) {  // FINAL
        const bool fs = do_scale && gn + 1 < n_gn;
        if (run) {
          struct Fin {
            float x, rn;
          };
          walk_pairs<Fin>(
              W, bp,
              [&](int q, int, int, Fin &o) {
                const float id = m.ID[q], r = m.R[q];
                const float p = first ? r * id : r * id + fb * m.P[q];
                o.x = m.X[q] + fa * p;
                const float si = first ? m.Wv[q] : m.Wv[q] + fb * m.S[q];
                o.rn = r - fa * si;
              },
              [&](int q, int u, int v, const Fin &o) {
                m.X[q] = o.x;
                if (v == 0 || v == nr - 1) __stcg(k.x + (size_t)(rb + v) * P + u, o.x);
                acc[0] += o.rn * o.rn;
              });
        } else if (active) {
          // x may also have moved in earlier passes of a depth step that
          // stopped early: the neighbours' next assembly needs the edges
          publish_edges(m.X, k.x, W, nr, rb, P);
        }
        if (fs && active) scale_partials(acc, 1, (float)s_seg.t);
        // sums needed: the next scale step's two; r.r for a tolerance and
        // for the report after the last Gauss-Newton iteration
        const bool need_rr = c.tol > 0.0 || gn + 1 == n_gn;
        overlap_pre = gn + 1 < n_gn;  // the next Gauss-Newton iteration's assembly
        auto post = [&] {
          if constexpr (JOINT) {  // the depth step's change of t
            s_seg.t += ff_to_double(s_seg.jdt);
            s_seg.jdt = ff2{0.0f, 0.0f};
          }
          if (run) {
            s_seg.iters += 1;
            if (need_rr || !fs)
              s_seg.rr = ff_to_double(joint ? ff_add(s_tot[0], ff_mul(s_seg.jrt, s_seg.jrt))
                                            : s_tot[0]);
          }
          if (fs) {
            if (need_rr)
              scale_update(1, 2);
            else
              scale_update(0, 1);
          }
        };
        if (fs && need_rr)
          alive = end_pass(IC<3>{}, acc, HK_X, 0, post);
        else if (fs)
          alive = end_pass(IC<2>{}, acc + 1, HK_X, 0, post);
        else
          alive = end_pass(IC<1>{}, acc, HK_X, 0, post);
        if (!alive) break;
        if (fs) scale_pending = true;
      } else {  // ITER
        if (run) {
          if (!halo_deferred) {
            for (int u = tid; u < W; u += kRThreads) {
              // r' = r - alpha (w + beta s), u' = r' / diag at the halo rows
              const float sa = first ? m.HA[2][u] : m.HA[2][u] + fb * m.HA[1][u];
              m.HA[0][u] = (m.HA[0][u] - fa * sa) * m.HA[3][u];
              const float sb = first ? m.HA[6][u] : m.HA[6][u] + fb * m.HA[5][u];
              m.HA[4][u] = (m.HA[4][u] - fa * sb) * m.HA[7][u];
            }
          }
          struct Upd {
            float x, p, s, r, id;
          };
          walk_pairs<Upd>(
              W, bp,
              [&](int q, int, int, Upd &o) {
                o.id = m.ID[q];
                const float r = m.R[q];
                o.p = first ? r * o.id : r * o.id + fb * m.P[q];
                o.x = m.X[q] + fa * o.p;
                o.s = first ? m.Wv[q] : m.Wv[q] + fb * m.S[q];
                o.r = r - fa * o.s;
              },
              [&](int q, int u, int v, const Upd &o) {
                m.X[q] = o.x;
                m.P[q] = o.p;
                m.S[q] = o.s;
                m.R[q] = o.r;
                if (!joint) m.U[q] = o.r * o.id;
                // r and s of the band's edge rows are final: they go to the
                // other parity's planes now and drain while the stencil runs
                // (the neighbours read them after the exchange)
                if (v == 0 || v == nr - 1) {
                  const size_t gi = (size_t)(rb + v) * P + u;
                  __stcg(Rg[nb] + gi, o.r);
                  __stcg(Sg[nb] + gi, o.s);
                }
              });
          if (halo_deferred) halo_store(true, first, fa, fb);
          __syncthreads();
          if constexpr (JOINT) {
            apply_band_joint(m, W, nr, bp, has_below, s_seg.jut.hi, acc);
            __syncthreads();
            publish_edges(m.Wv, Wg[nb], W, nr, rb, P);
          } else {
            apply_band(m, W, nr, bp, has_below, acc, Wg[nb], rb, P);
          }
        }
        const int next_kind = (it + 1 < n_pcg - 1) ? HK_ITER : HK_NONE;
        // sums needed: (r, u), (w, u); (r, r) for a tolerance; the joint
        // solve also (ws, u)
        auto post = [&] {
          if (!run) return;
          s_seg.iters += 1;
          ff2 gn_ = s_tot[0], dl = s_tot[1];
          if constexpr (JOINT) {  // border terms of (r, u) and (w, u)
            s_seg.jwt = ff_sub(ff_mul(s_seg.jS, s_seg.jut), s_tot[2]);
            gn_ = ff_add(gn_, ff_mul(s_seg.jrt, s_seg.jut));
            dl = ff_add(dl, ff_mul(s_seg.jwt, s_seg.jut));
          } else if (c.tol > 0.0) {
            s_seg.rr = ff_to_double(s_tot[2]);
          }
          if (c.tol > 0.0 && sqrt(s_seg.rr) < c.tol * sqrt(s_seg.bb)) {
            s_seg.stop = 1;
          } else {
            // beta = gamma / gamma_prev; p.Ap = delta - beta gamma / alpha_prev,
            // so alpha = gamma / p.Ap = gamma ag / (delta ag - gamma^2) with
            // ag = alpha_prev gamma_prev > 0: one division after the sums
            // arrive (beta's runs beside it) instead of three in a row
            const ff2 beta = ff_div(gn_, s_seg.gam);
            const ff2 ag = ff_mul(s_seg.alpha, s_seg.gam);
            const ff2 den = ff_sub(ff_mul(dl, ag), ff_mul(gn_, gn_));
            if (gn_.hi == 0.0f || !(den.hi > 0.0f)) {
              s_seg.stop = 1;
            } else {
              s_seg.beta = beta;
              s_seg.alpha = ff_div(ff_mul(gn_, ag), den);
              s_seg.gam = gn_;
              if constexpr (JOINT) joint_border_step(false);
            }
          }
        };
        if constexpr (JOINT) {
          const float a3[3] = {acc[0], acc[1], acc[3]};
          alive = end_pass(IC<3>{}, a3, next_kind, nb, post);
        } else {
          alive = c.tol > 0.0 ? end_pass(IC<3>{}, acc, next_kind, nb, post)
                              : end_pass(IC<2>{}, acc, next_kind, nb, post);
        }
        if (!alive) break;
      }
    }
  }

  if (alive && active) {
    for (Walk it(W); it.q < bp; it.next())
      __stcg(k.x + (size_t)(rb + it.v) * P + it.u, m.X[it.q]);
  }
  if (tid == 0) {
    Scalars *sc = k.sc;
    if (!alive) {
      atomicOr(&sc->flags, kFlagTimeout);
    } else if (active && s_kf.cta_begin == (int)blockIdx.x) {
      sc->t = s_seg.t;
      sc->rr = s_seg.rr;
      sc->rho = ff_to_double(s_seg.gam);
      sc->iters = s_seg.iters;
      sc->stop = s_seg.stop;
    }
  }
  grid_exit(h, G, reinterpret_cast<unsigned long long *>(groups),
            (long long)h->nkf * (long long)(sizeof(SumGroup) / 8) + (long long)kFlagWords * G);
}

// The kernel instance of a variant and a loss kind.
static const void *resident_fn(bool joint, int lk) {
  if (joint) {
    if (lk == LK_LSQ) return reinterpret_cast<const void *>(k_resident<true, LK_LSQ>);
    if (lk == LK_TUKEY) return reinterpret_cast<const void *>(k_resident<true, LK_TUKEY>);
    return reinterpret_cast<const void *>(k_resident<true, LK_HUBER>);
  }
  if (lk == LK_LSQ) return reinterpret_cast<const void *>(k_resident<false, LK_LSQ>);
  if (lk == LK_TUKEY) return reinterpret_cast<const void *>(k_resident<false, LK_TUKEY>);
  return reinterpret_cast<const void *>(k_resident<false, LK_HUBER>);
}

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

struct ResDev {
  int sms = 0, smem_optin = 0, occ = 0, static_smem = 0;
};
ResDev g_rdev[64];
bool g_rdev_init[64] = {false};
std::mutex g_rdev_mu;

const ResDev &rdev() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lk(g_rdev_mu);
  if (!g_rdev_init[dev]) {
    ResDev d;
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    for (int v = 0; v < 2; ++v)  // the largest static share of the instances
      for (int lk = LK_LSQ; lk <= LK_TUKEY; ++lk)
        if (cudaFuncGetAttributes(&fa, resident_fn(v == 1, lk)) == cudaSuccess)
          d.static_smem = std::max(d.static_smem, (int)fa.sharedSizeBytes);
    cudaGetLastError();
    g_rdev[dev] = d;
    g_rdev_init[dev] = true;
  }
  return g_rdev[dev];
}

}  // namespace

// Plan bytes: header, CTA table, keyframe table, then one exact-sum group
// per keyframe and the CTAs' edge flags (32 bytes each; the launch's last
// CTA clears groups and flags together on its way out).
static size_t resident_bytes(int nkf, int G) {
  size_t off = align16(sizeof(PlanHeader));
  off += align16(sizeof(ResCta) * (size_t)G);
  off += align16(sizeof(ResKf) * (size_t)nkf);
  off = (off + 255) & ~(size_t)255;
  off += sizeof(SumGroup) * (size_t)nkf;
  off += kFlagWords * 8 * (size_t)G;
  return off;
}

size_t resident_plan_bytes(int nkf, int G) { return resident_bytes(nkf, G); }

int resident_max_ctas() { return rdev().sms; }

// The plan with or without the input planes staged in shared memory; false
// if the keyframes' bands do not fit the CTAs / shared memory that way.
static bool resident_build_plan_with(const Planes *const *kfs, int n, const FusedTuning &tune,
                                     bool in_smem, std::vector<char> &out, LaunchShape &shape);

bool resident_build_plan(const Planes *const *kfs, int n, const FusedTuning &tune,
                         std::vector<char> &out, LaunchShape &shape) {
  // the input planes stay in shared memory for the launch where the bands
  // still fit with them; otherwise the assembly reads them from L2 / HBM
  return resident_build_plan_with(kfs, n, tune, true, out, shape) ||
         resident_build_plan_with(kfs, n, tune, false, out, shape);
}

static bool resident_build_plan_with(const Planes *const *kfs, int n, const FusedTuning &tune,
                                     bool in_smem, std::vector<char> &out, LaunchShape &shape) {
  const ResDev &d = rdev();
  if (n < 1 || d.sms <= 0 || d.smem_optin <= 0) return false;
  const long long arrays = in_smem ? 9 + kIn : 9, halo = in_smem ? kHalo + 2 : kHalo;
  // the exact-sum words hold up to 1023 CTAs per keyframe
  int G_cap = std::min(d.sms, 1023);
  if (tune.max_ctas > 0) G_cap = std::min(G_cap, tune.max_ctas);
  const long long avail = (long long)d.smem_optin - d.static_smem - 1024;
  long long total_px = 0;
  int Wmax = 0;
  for (int k = 0; k < n; ++k) {
    total_px += (long long)kfs[k]->W * kfs[k]->H;
    Wmax = std::max(Wmax, kfs[k]->W);
  }
  // rows a band may hold within the shared-memory budget, per keyframe
  std::vector<int> nb(n), maxrows(n);
  long long need = 0;
  for (int k = 0; k < n; ++k) {
    const long long Wk = kfs[k]->W;
    const long long rows = (avail / 4 - halo * Wmax) / (arrays * Wk);
    if (rows < 1) return false;
    maxrows[k] = (int)std::min<long long>(rows, kfs[k]->H);
    nb[k] = (kfs[k]->H + maxrows[k] - 1) / maxrows[k];
    need += nb[k];
  }
  if (need > G_cap) return false;
  // hand the remaining CTAs out in proportion to pixels (more bands = less
  // work per CTA), never more bands than rows
  int spare = G_cap - (int)need;
  while (spare > 0) {
    int best = -1;
    double best_load = 0.0;
    for (int k = 0; k < n; ++k) {
      if (nb[k] >= kfs[k]->H) continue;
      const double load = (double)kfs[k]->W * kfs[k]->H / nb[k];
      if (load > best_load) {
        best_load = load;
        best = k;
      }
    }
    if (best < 0) break;
    ++nb[best];
    --spare;
  }
  int G = 0;
  for (int k = 0; k < n; ++k) G += nb[k];
  std::vector<ResCta> ctas(G);
  std::vector<ResKf> rk(n);
  int band_px_max = 0, cI = 0;
  for (int k = 0; k < n; ++k) {
    const int H = kfs[k]->H;
    rk[k].pl = *kfs[k];
    rk[k].cta_begin = cI;
    for (int b = 0; b < nb[k]; ++b) {
      const int r0 = (int)((long long)H * b / nb[k]), r1 = (int)((long long)H * (b + 1) / nb[k]);
      ctas[cI].kf = k;
      ctas[cI].rb = r0;
      ctas[cI].re = r1;
      band_px_max = std::max(band_px_max, (r1 - r0) * kfs[k]->W);
      ++cI;
    }
    rk[k].cta_end = cI;
  }
  const int stride = (band_px_max + 3) & ~3;
  const long long smem = (arrays * stride + halo * Wmax) * 4;
  if (smem > avail) return false;
  out.assign(resident_bytes(n, G), 0);
  char *base = out.data();
  PlanHeader *hd = reinterpret_cast<PlanHeader *>(base);
  size_t off = align16(sizeof(PlanHeader));
  hd->off_cta_work = (long long)off;
  off += align16(sizeof(ResCta) * (size_t)G);
  hd->off_kf = (long long)off;
  off += align16(sizeof(ResKf) * (size_t)n);
  off = (off + 255) & ~(size_t)255;
  hd->off_slots = (long long)off;
  hd->off_flags = (long long)(off + sizeof(SumGroup) * (size_t)n);
  hd->kind = kPlanResident;
  hd->debug_skip_cta = tune.debug_skip_cta;
  hd->nkf = n;
  hd->G = G;
  hd->nslots = G;
  hd->th = stride;  // shared-memory stride of one band array
  hd->smem_bytes = (int)smem;
  hd->in_smem = in_smem ? 1 : 0;
  hd->bytes = (long long)out.size();
  memcpy(base + hd->off_cta_work, ctas.data(), sizeof(ResCta) * G);
  memcpy(base + hd->off_kf, rk.data(), sizeof(ResKf) * n);
  shape.kind = kPlanResident;
  shape.G = G;
  shape.vec = 0;
  shape.smem = (int)smem;
  (void)total_px;
  return true;
}

cudaError_t resident_launch(void *dplan, const LaunchShape &shape, const SolveCfg &c, int n_gn,
                            int n_pcg, unsigned long long limit_ns, cudaStream_t s, int first) {
  PlanHeader *h = static_cast<PlanHeader *>(dplan);
  const bool joint = (c.terms & DF_TERM_SEMI) && c.scale_step == DF_SCALE_JOINT;
  const void *fn = resident_fn(joint, loss_kind(c.loss, c.delta));
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, shape.smem);
  if (e != cudaSuccess) return e;
  void *args[] = {&h, const_cast<SolveCfg *>(&c), &n_gn, &n_pcg, &limit_ns, &first};
  count_launches(1);
  return cudaLaunchCooperativeKernel(fn, dim3(shape.G), dim3(kRThreads), args, (size_t)shape.smem,
                                     s);
}

}  // namespace df
