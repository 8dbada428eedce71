// Fused persistent solver: one cooperative launch runs a whole per-frame
// solve (Section II-C: n_gn Gauss-Newton iterations alternating scale and
// depth) for one keyframe or a batch of keyframes of different sizes.
//
// Depth step: Jacobi-preconditioned CG in the Chronopoulos-Gear arrangement,
// which has the iterates of textbook PCG in exact arithmetic but needs one
// global reduction per iteration instead of two:
//   u = r / diag,  w = A u,  gamma = (r, u),  delta = (w, u)
//   beta  = gamma_i / gamma_{i-1},  alpha = gamma_i / (delta_i - beta gamma_i / alpha_{i-1})
//   p = u + beta p,  s = w + beta s  (= A p),  x += alpha p,  r -= alpha s
// The breakdown / stop rules are those of the textbook form: stop when
// gamma = r.z = 0 or when p.Ap = delta - beta gamma / alpha <= 0, or (tol > 0)
// when ||r|| < tol ||b||.
//
// Passes, each ended by one exchange of the keyframes' sums:
//   SCALE     scale-step partial sums (first GN iteration only)
//   ASSEMBLE  IRLS weights of Eqs. 6-8 at (x, t), 5-point system, r0
//   INIT      w0 = A u0
//   ITER      one CG iteration (all but the last of a depth step)
//   FINAL     last CG iteration's x update, plus the next GN iteration's
//             scale-step sums taken at the new x
//
// Work: the planes are cut into tiles of (32 * VEC) columns x th rows; a warp
// owns a tile and walks down its rows keeping the row above / below in
// registers (5-point stencil), lanes exchange the left / right neighbours by
// shuffles. Tiles are cut into contiguous ranges, one per CTA; a CTA's range
// may span a few keyframes ("segments").
//
// Reductions: per tile a warp sums its FP32 per-lane partials as a
// double-float (df_sync.cuh), per CTA the warps' sums of a keyframe segment
// are added in warp order, and warp sg adds segment sg's sums exactly into
// that keyframe's fixed-point sum words (df_exact.cuh), whose arrival counts
// also end the pass: a CTA waits only for the CTAs that share its
// keyframes, never for the whole grid. Integer addition is associative, so
// every CTA reads bitwise identical totals and the result does not depend on
// timing. The CG scalars formed from the sums are double-float too.
//
// Waits: every poll of the sum words and every wait on a staged row gives
// up after a time limit (%globaltimer); a CTA that gives up raises an abort
// word, every CTA then skips the remaining passes, the keyframes are
// flagged kFlagTimeout and the host reports DF_ETIMEOUT. The last CTA to
// exit clears the sum and abort words, so the next launch starts clean
// either way.
#include <math.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "df_batch_io.cuh"
#include "df_fused.cuh"
#include "df_sync.cuh"
#include "df_tma.cuh"

namespace df {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSeg = 8;  // keyframes a CTA's tile range may span
constexpr int kQ = 3;       // double-float partial sums per slot
static_assert(kQ == 3, "a pass's reduction selects among three accumulators");

enum PassKind : int { P_SCALE = 0, P_ASSEMBLE, P_INIT, P_ITER, P_FINAL };

struct FusedKf {
  Planes pl;
  int row_begin;   // first row of its strips in the plan's concatenated row list
  int rows;        // strips * H: a strip is one column tile (32 * VEC columns) over all rows
  int blk;         // rows per row block of its work list (H: one block, strip by strip)
  int asm_rows;    // separate assembly kernel: rows of one piece (one strip's rows)
  int slot_begin;  // this keyframe's slots: [slot_begin, slot_end)
  int slot_end;
  int writer_cta;  // the CTA that writes the final scalars back
  int asm_p0;      // separate assembly kernel: the keyframe's first piece
  int group;       // its exact-sum words: the plan's group 'group'
  int pad;
};



// ---- small vector helpers ---------------------------------------------------

template <int VEC>
struct F {
  float v[VEC];
};

template <int VEC>
__device__ __forceinline__ F<VEC> fzero() {
  F<VEC> a;
#pragma unroll
  for (int e = 0; e < VEC; ++e) a.v[e] = 0.0f;
  return a;
}

// coherent (L2) loads / stores for planes the kernel itself rewrites
template <int VEC>
__device__ __forceinline__ F<VEC> ldm(const float *p) {
  F<VEC> a;
  if constexpr (VEC == 4) {
    const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
    a.v[0] = q.x; a.v[1] = q.y; a.v[2] = q.z; a.v[3] = q.w;
  } else {
    a.v[0] = __ldcg(p);
  }
  return a;
}

template <int VEC>
__device__ __forceinline__ void stm(float *p, const F<VEC> &a) {
  if constexpr (VEC == 4) {
    __stcg(reinterpret_cast<float4 *>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
  } else {
    __stcg(p, a.v[0]);
  }
}

// read-only planes (network and semi-dense inputs) through the read-only path
template <int VEC>
__device__ __forceinline__ F<VEC> ldr(const float *p) {
  F<VEC> a;
  if constexpr (VEC == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    a.v[0] = q.x; a.v[1] = q.y; a.v[2] = q.z; a.v[3] = q.w;
  } else {
    a.v[0] = __ldg(p);
  }
  return a;
}

template <int VEC, int DT>
__device__ __forceinline__ F<VEC> ldc(const void *base, size_t i) {
  if constexpr (DT == DF_F32) {
    return ldr<VEC>(reinterpret_cast<const float *>(base) + i);
  } else {
    F<VEC> a;
    if constexpr (VEC == 4) {
      const uint2 q = __ldg(reinterpret_cast<const uint2 *>(
          reinterpret_cast<const unsigned short *>(base) + i));
      const unsigned short h[4] = {(unsigned short)(q.x & 0xffff), (unsigned short)(q.x >> 16),
                                   (unsigned short)(q.y & 0xffff), (unsigned short)(q.y >> 16)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if constexpr (DT == DF_BF16)
          a.v[e] = __bfloat162float(__ushort_as_bfloat16(h[e]));
        else
          a.v[e] = __half2float(__ushort_as_half(h[e]));
      }
    } else {
      a.v[0] = ld_cnn<DT>(base, i);
    }
    return a;
  }
}

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }


struct Geo {
  int c0, r0, nrows, col;
};

template <int VEC>
__device__ __forceinline__ Geo geo_of(int c0, int r0, int nrows) {
  Geo g;
  g.c0 = c0;
  g.r0 = r0;
  g.nrows = nrows;
  g.col = c0 + (threadIdx.x & 31) * VEC;
  return g;
}

// ---- SCALE: partial sums of the scale step (Eq. 6 with x fixed) ------------
template <int VEC, int LK>
__device__ void scale_tile(const FusedKf &K, const Geo &g, float t, const SolveCfg &c, float acc[kQ]) {
  const Planes &k = K.pl;
  for (int j = 0; j < g.nrows; ++j) {
    const size_t i = (size_t)(g.r0 + j) * k.P + g.col;
    const F<VEC> x = ldm<VEC>(k.x + i);
    const F<VEC> ms = ldr<VEC>(k.mu_s + i), vs = ldr<VEC>(k.var_s + i);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      if (g.col + e < k.W && semi_valid(ms.v[e], vs.v[e])) {
        const float w = robust_weight_k<LK>(x.v[e] - t - ms.v[e], vs.v[e], c.delta);
        acc[0] += w;
        acc[1] += w * (x.v[e] - ms.v[e]);
      }
    }
  }
}

// ---- ASSEMBLE: weights, 5-point system and r0 (see df_launch.cu) -----------
template <int VEC, int DT, int LK, bool WIDE = true>  // WIDE: also r.r and b.b
__device__ void assemble_tile(const FusedKf &K, const Geo &g, float t, const SolveCfg &c,
                              float acc[kQ]) {
  const Planes &k = K.pl;
  const int lane = threadIdx.x & 31;
  const int W = k.W, H = k.H;
  const size_t P = k.P;
  const bool semi = c.terms & DF_TERM_SEMI, net = c.terms & DF_TERM_NET,
             grad = c.terms & DF_TERM_GRAD;
  float *r_out = k.v[1];
  F<VEC> x_cur = ldm<VEC>(k.x + (size_t)g.r0 * P + g.col);
  F<VEC> wy_up = fzero<VEC>(), ey_up = fzero<VEC>(), gy_up = fzero<VEC>();
  if (grad && g.r0 > 0) {
    const size_t iu = (size_t)(g.r0 - 1) * P + g.col;
    const F<VEC> xu = ldm<VEC>(k.x + iu);
    const F<VEC> gyu = ldc<VEC, DT>(k.cnn[4], iu), vyu = ldc<VEC, DT>(k.cnn[5], iu);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      if (g.col + e < W) {
        gy_up.v[e] = gyu.v[e];
        ey_up.v[e] = x_cur.v[e] - xu.v[e] - gyu.v[e];
        wy_up.v[e] = robust_weight_k<LK>(ey_up.v[e], vyu.v[e], c.delta);
      }
    }
  }
  for (int j = 0; j < g.nrows; ++j) {
    const int v = g.r0 + j;
    const size_t i = (size_t)v * P + g.col;
    const F<VEC> x_dn = (v + 1 < H) ? ldm<VEC>(k.x + i + P) : fzero<VEC>();
    // east neighbour of every element
    F<VEC> x_e;
#pragma unroll
    for (int e = 0; e < VEC - 1; ++e) x_e.v[e] = x_cur.v[e + 1];
    {
      float xe = shfl_dn1(x_cur.v[0]);
      if (lane == 31) xe = (g.col + VEC < W) ? __ldcg(k.x + i + VEC) : 0.0f;
      x_e.v[VEC - 1] = xe;
    }
    // x-term at this pixel (pairs i, i+1) and y-term (pairs i, i+W)
    F<VEC> wxv = fzero<VEC>(), exv = fzero<VEC>(), gxv = fzero<VEC>();
    F<VEC> wyv = fzero<VEC>(), eyv = fzero<VEC>(), gyv = fzero<VEC>();
    if (grad) {
      const F<VEC> gxr = ldc<VEC, DT>(k.cnn[2], i), vxr = ldc<VEC, DT>(k.cnn[3], i);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        if (g.col + e < W - 1) {
          gxv.v[e] = gxr.v[e];
          exv.v[e] = x_e.v[e] - x_cur.v[e] - gxr.v[e];
          wxv.v[e] = robust_weight_k<LK>(exv.v[e], vxr.v[e], c.delta);
        }
      }
      if (v < H - 1) {
        const F<VEC> gyr = ldc<VEC, DT>(k.cnn[4], i), vyr = ldc<VEC, DT>(k.cnn[5], i);
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          if (g.col + e < W) {
            gyv.v[e] = gyr.v[e];
            eyv.v[e] = x_dn.v[e] - x_cur.v[e] - gyr.v[e];
            wyv.v[e] = robust_weight_k<LK>(eyv.v[e], vyr.v[e], c.delta);
          }
        }
      }
    }
    // x-term of the west pair (i-1, i)
    F<VEC> wxw, exw, gxw;
#pragma unroll
    for (int e = 1; e < VEC; ++e) {
      wxw.v[e] = wxv.v[e - 1];
      exw.v[e] = exv.v[e - 1];
      gxw.v[e] = gxv.v[e - 1];
    }
    {
      float a = shfl_up1(wxv.v[VEC - 1]), b = shfl_up1(exv.v[VEC - 1]),
            gg = shfl_up1(gxv.v[VEC - 1]);
      if (lane == 0) {
        a = b = gg = 0.0f;
        if (grad && g.col > 0 && g.col < W) {
          const float xw = __ldcg(k.x + i - 1);
          gg = ld_cnn<DT>(k.cnn[2], i - 1);
          b = x_cur.v[0] - xw - gg;
          a = robust_weight_k<LK>(b, ld_cnn<DT>(k.cnn[3], i - 1), c.delta);
        }
      }
      wxw.v[0] = a;
      exw.v[0] = b;
      gxw.v[0] = gg;
    }
    const F<VEC> ms = ldr<VEC>(k.mu_s + i), vs = ldr<VEC>(k.var_s + i);
    const F<VEC> mn = ldc<VEC, DT>(k.cnn[0], i), vn = ldc<VEC, DT>(k.cnn[1], i);
    F<VEC> dd, rr_, wxo, wyo;  // dd holds 1 / diag
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      float d = 0.0f, r = 0.0f, b = 0.0f;
      if (g.col + e < W) {
        const float xi = x_cur.v[e];
        float ws = 0.0f, rs = 0.0f, bs = 0.0f;
        if (semi && semi_valid(ms.v[e], vs.v[e])) {
          ws = robust_weight_k<LK>(xi - t - ms.v[e], vs.v[e], c.delta);
          rs = ws * (t + ms.v[e] - xi);
          bs = ws * (t + ms.v[e]);
        }
        float wn = 0.0f, m = 0.0f;
        if (net) {
          m = mn.v[e];
          wn = robust_weight_k<LK>(xi - m, vn.v[e], c.delta);
        }
        d = ws + wn + wxv.v[e] + wxw.v[e] + wyv.v[e] + wy_up.v[e];
        r = rs + wn * (m - xi) + wxv.v[e] * exv.v[e] - wxw.v[e] * exw.v[e] +
            wyv.v[e] * eyv.v[e] - wy_up.v[e] * ey_up.v[e];
        if (WIDE)
          b = bs + wn * m - wxv.v[e] * gxv.v[e] + wxw.v[e] * gxw.v[e] - wyv.v[e] * gyv.v[e] +
              wy_up.v[e] * gy_up.v[e];
      }
      const float id = inv_diag(d);
      dd.v[e] = id;
      rr_.v[e] = r;
      wxo.v[e] = wxv.v[e];
      wyo.v[e] = wyv.v[e];
      acc[0] += r * (r * id);
      if (WIDE) {
        acc[1] += r * r;
        acc[2] += b * b;
      }
    }
    stm<VEC>(k.diag + i, dd);
    stm<VEC>(k.wx + i, wxo);
    stm<VEC>(k.wy + i, wyo);
    stm<VEC>(r_out + i, rr_);
    wy_up = wyv;
    ey_up = eyv;
    gy_up = gyv;
    x_cur = x_dn;
  }
}

// ---- INIT / ITER: one CG pass over a tile ---------------------------------
//
// Values of the pass at one row (for this lane's VEC columns): the new
// residual r' = r - alpha s_i, with s_i = w + beta s_prev (s_i = w in the first
// iteration, s_i = 0 and r' = r for INIT), and u' = r' / diag.
template <int VEC>
struct RowNew {
  F<VEC> d, r, s, u, r_in;  // 1/diag, r', s_i, u', and the residual entering the pass
};

template <int VEC, int KIND>  // KIND: 0 INIT, 1 first iteration, 2 later iteration
__device__ __forceinline__ RowNew<VEC> row_new(const float *r_cur, const float *s_prev,
                                               const float *w_cur, const float *diag, size_t i,
                                               float alpha, float beta) {
  RowNew<VEC> o;
  o.d = ldm<VEC>(diag + i);
  const F<VEC> r = ldm<VEC>(r_cur + i);
  o.r_in = r;
  if constexpr (KIND == 0) {
    o.r = r;
    o.s = fzero<VEC>();
  } else {
    const F<VEC> w = ldm<VEC>(w_cur + i);
    F<VEC> s;
    if constexpr (KIND == 2) s = ldm<VEC>(s_prev + i);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      o.s.v[e] = (KIND == 2) ? w.v[e] + beta * s.v[e] : w.v[e];
      o.r.v[e] = r.v[e] - alpha * o.s.v[e];
    }
  }
#pragma unroll
  for (int e = 0; e < VEC; ++e) o.u.v[e] = o.r.v[e] * o.d.v[e];
  return o;
}

template <int KIND>
__device__ __forceinline__ float col_new_u(const float *r_cur, const float *s_prev,
                                           const float *w_cur, const float *diag, size_t i,
                                           float alpha, float beta) {
  const float id = __ldcg(diag + i);
  float r = __ldcg(r_cur + i);
  if constexpr (KIND != 0) {
    float s = __ldcg(w_cur + i);
    if constexpr (KIND == 2) s += beta * __ldcg(s_prev + i);
    r -= alpha * s;
  }
  return r * id;
}

template <int VEC, int KIND>
__device__ void cg_tile(const FusedKf &K, const Geo &g, float alpha, float beta, const float *r_cur,
                        const float *s_prev, const float *w_cur, float *r_nxt, float *s_cur,
                        float *w_nxt, float acc[kQ]) {
  const Planes &k = K.pl;
  const int lane = threadIdx.x & 31;
  const int W = k.W, H = k.H;
  const size_t P = k.P;
  F<VEC> u_up = fzero<VEC>(), wy_up = fzero<VEC>();
  if (g.r0 > 0) {
    const size_t iu = (size_t)(g.r0 - 1) * P + g.col;
    u_up = row_new<VEC, KIND>(r_cur, s_prev, w_cur, k.diag, iu, alpha, beta).u;
    wy_up = ldm<VEC>(k.wy + iu);
  }
  size_t i = (size_t)g.r0 * P + g.col;
  RowNew<VEC> cur = row_new<VEC, KIND>(r_cur, s_prev, w_cur, k.diag, i, alpha, beta);
  for (int j = 0; j < g.nrows; ++j) {
    const int v = g.r0 + j;
    // the row below: owned (keep everything) or halo (u only)
    RowNew<VEC> nxt;
    F<VEC> u_dn = fzero<VEC>();
    if (v + 1 < H) {
      nxt = row_new<VEC, KIND>(r_cur, s_prev, w_cur, k.diag, i + P, alpha, beta);
      u_dn = nxt.u;
    }
    const F<VEC> wxr = ldm<VEC>(k.wx + i), wyr = ldm<VEC>(k.wy + i);
    // west / east neighbours of u and the west coupling
    F<VEC> u_w, u_e, wx_w;
#pragma unroll
    for (int e = 1; e < VEC; ++e) {
      u_w.v[e] = cur.u.v[e - 1];
      wx_w.v[e] = wxr.v[e - 1];
    }
#pragma unroll
    for (int e = 0; e < VEC - 1; ++e) u_e.v[e] = cur.u.v[e + 1];
    {
      float uw = shfl_up1(cur.u.v[VEC - 1]);
      float wxl = shfl_up1(wxr.v[VEC - 1]);
      float ue = shfl_dn1(cur.u.v[0]);
      if (lane == 0) {
        uw = 0.0f;
        wxl = 0.0f;
        if (g.col > 0 && g.col < W) {
          uw = col_new_u<KIND>(r_cur, s_prev, w_cur, k.diag, i - 1, alpha, beta);
          wxl = __ldcg(k.wx + i - 1);
        }
      }
      if (lane == 31) {
        ue = (g.col + VEC < W)
                 ? col_new_u<KIND>(r_cur, s_prev, w_cur, k.diag, i + VEC, alpha, beta)
                 : 0.0f;
      }
      u_w.v[0] = uw;
      wx_w.v[0] = wxl;
      u_e.v[VEC - 1] = ue;
    }
    F<VEC> w_new;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      // A u = r - N u (u = r / diag, A = diag - N)
      w_new.v[e] = cur.r.v[e] - (wxr.v[e] * u_e.v[e] + wx_w.v[e] * u_w.v[e] +
                                 wyr.v[e] * u_dn.v[e] + wy_up.v[e] * u_up.v[e]);
      acc[0] += cur.r.v[e] * cur.u.v[e];
      acc[1] += w_new.v[e] * cur.u.v[e];
      acc[2] += cur.r.v[e] * cur.r.v[e];
    }
    stm<VEC>(w_nxt + i, w_new);
    if constexpr (KIND != 0) {
      // p_i = u_i + beta p_{i-1} with u_i = r_i / diag (the residual entering
      // this iteration), x += alpha p_i; r' and s_i go to the other buffers
      const F<VEC> &r_old = cur.r_in;
      F<VEC> p = (KIND == 2) ? ldm<VEC>(k.v[0] + i) : fzero<VEC>();
      F<VEC> x = ldm<VEC>(k.x + i);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const float ui = r_old.v[e] * cur.d.v[e];
        p.v[e] = (KIND == 2) ? ui + beta * p.v[e] : ui;
        x.v[e] += alpha * p.v[e];
      }
      stm<VEC>(k.v[0] + i, p);
      stm<VEC>(k.x + i, x);
      stm<VEC>(r_nxt + i, cur.r);
      stm<VEC>(s_cur + i, cur.s);
    }
    u_up = cur.u;
    wy_up = wyr;
    cur = nxt;
    i += P;
  }
}

// ---- FINAL: last CG iteration (no stencil) + next scale-step sums ----------
template <int VEC, int LK>
__device__ void final_tile(const FusedKf &K, const Geo &g, bool first, bool update, float alpha,
                           float beta, bool scale, float t, const SolveCfg &c,
                           const float *r_cur, const float *s_prev, const float *w_cur,
                           float acc[kQ]) {
  const Planes &k = K.pl;
  for (int j = 0; j < g.nrows; ++j) {
    const size_t i = (size_t)(g.r0 + j) * k.P + g.col;
    F<VEC> x = ldm<VEC>(k.x + i);
    if (update) {
      const F<VEC> d = ldm<VEC>(k.diag + i), r = ldm<VEC>(r_cur + i), w = ldm<VEC>(w_cur + i);
      const F<VEC> p = first ? fzero<VEC>() : ldm<VEC>(k.v[0] + i);
      const F<VEC> s = first ? fzero<VEC>() : ldm<VEC>(s_prev + i);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const float ui = r.v[e] * d.v[e];
        const float pi = first ? ui : ui + beta * p.v[e];
        x.v[e] += alpha * pi;
        const float si = first ? w.v[e] : w.v[e] + beta * s.v[e];
        const float rn = r.v[e] - alpha * si;
        acc[0] += rn * rn;
      }
      stm<VEC>(k.x + i, x);
    }
    if (scale) {
      const F<VEC> ms = ldr<VEC>(k.mu_s + i), vs = ldr<VEC>(k.var_s + i);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        if (g.col + e < k.W && semi_valid(ms.v[e], vs.v[e])) {
          const float w = robust_weight_k<LK>(x.v[e] - t - ms.v[e], vs.v[e], c.delta);
          acc[1] += w;
          acc[2] += w * (x.v[e] - ms.v[e]);
        }
      }
    }
  }
}

// ---- VEC = 4 tiles fed by bulk copies (df_tma.cuh) --------------------------
//
// Same arithmetic as the tiles above; the rows of a tile (one halo row above
// and below where they exist) are staged in the warp's ring, kStages rows in
// flight, and every value, including the tile's west / east neighbour
// columns, is read from shared memory. Each function returns false if a wait
// for staged rows ran out of time.

__device__ __forceinline__ F<4> f4v(float4 q) {
  F<4> a;
  a.v[0] = q.x; a.v[1] = q.y; a.v[2] = q.z; a.v[3] = q.w;
  return a;
}

template <int DT>
__device__ __forceinline__ F<4> cnn4(const RowRing &ring, int s, int p) {
  if constexpr (DT == DF_F32) {
    return f4v(ring.f4(s, p));
  } else {
    const uint2 q = ring.h4(s, p);
    const unsigned short h[4] = {(unsigned short)(q.x & 0xffff), (unsigned short)(q.x >> 16),
                                 (unsigned short)(q.y & 0xffff), (unsigned short)(q.y >> 16)};
    F<4> a;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if constexpr (DT == DF_BF16)
        a.v[e] = __bfloat162float(__ushort_as_bfloat16(h[e]));
      else
        a.v[e] = __half2float(__ushort_as_half(h[e]));
    }
    return a;
  }
}

template <int DT>
__device__ __forceinline__ float cnn1(const RowRing &ring, int s, int p, int idx32) {
  // idx32: slot index of an f32 plane (3 = west, 132 = east); 16-bit planes
  // carry 8 halo elements, hence the shift by 4
  if constexpr (DT == DF_F32) {
    return ring.f1(s, p, idx32);
  } else {
    const unsigned short h = ring.h1(s, p, idx32 + 4);
    if constexpr (DT == DF_BF16)
      return __bfloat162float(__ushort_as_bfloat16(h));
    else
      return __half2float(__ushort_as_half(h));
  }
}

template <int DT>
__device__ __forceinline__ void store4(float *p, const F<4> &a) {
  __stcg(reinterpret_cast<float4 *>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
}

// Rows jb..je of a tile go through the ring in order; 'ensure(k)' waits for
// the k-th of them, 'release()' frees the oldest waited row's stage and
// stages the next row of the tile. Each plane is
// one bulk copy per row: the tile's 128 columns plus 16 bytes on each side,
// clipped to the padded row; element size 4, or 2 for the planes in HALF
// (16-bit network planes). Rows at index 0 (when has_above) and R - 1 (when
// has_below) are halo rows and stage only planes 0..NH-1; the others stage
// the planes of 'mask' (all NP unless a pass leaves some out). Lane p owns
// plane p: it keeps that plane's source pointer, size and slot, so a row's
// NP copies leave as one warp instruction (lane 0 posts the row's byte count
// on the stage's mbarrier first).
template <int NP, int NH, uint32_t HALF>
struct TileRows {
  static_assert(NP <= 32 && NH <= NP, "one lane per staged plane");
  RowRing &ring;
  const char *src = nullptr;  // this lane's plane: the next row's copy start
  uint32_t bytes = 0;         // this lane's copy size
  uint32_t dst = 0;           // shared address of this lane's slot in stage 0
  uint32_t step = 0;          // row pitch of this lane's plane, bytes
  uint32_t tx_full = 0, tx_halo = 0;  // bytes a full / halo row brings
  int R, issued = 0, waited = 0;
  bool has_above, has_below, ok = true;
  bool mine_full = false, mine_halo = false;  // this lane copies in a full / halo row
  static constexpr uint32_t kAll = (NP >= 32) ? 0xffffffffu : ((1u << NP) - 1u);
  __device__ TileRows(RowRing &r, const StagePlane (&pl)[NP], int c0, int P, int jb, int R_,
                      bool above, bool below, uint32_t mask = kAll)
      : ring(r), R(R_), has_above(above), has_below(below) {
    const int lane = threadIdx.x & 31;
    // column range [cs, ce) of a staged row: the tile's 128 columns and
    // 16 bytes on each side, clipped to the padded row
    const int cs4 = c0 - 4 > 0 ? c0 - 4 : 0, ce4 = c0 + 132 < P ? c0 + 132 : P;
    const int cs2 = c0 - 8 > 0 ? c0 - 8 : 0, ce2 = c0 + 136 < P ? c0 + 136 : P;
    const uint32_t b4 = (uint32_t)(ce4 - cs4) * 4u, d4 = (uint32_t)(cs4 - (c0 - 4)) * 4u;
    const uint32_t b2 = (uint32_t)(ce2 - cs2) * 2u, d2 = (uint32_t)(cs2 - (c0 - 8)) * 2u;
    const uint32_t rb4 = (uint32_t)P * 4u, rb2 = (uint32_t)P * 2u;
    const uint32_t s0 = smem_addr(ring.smem);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      constexpr uint32_t H = HALF;
      const bool h = (H >> p) & 1u;
      const uint32_t bp = h ? b2 : b4;
      if (p < NH) tx_halo += bp;
      if ((mask >> p) & 1u) tx_full += bp;
      if (p == lane) {
        src = static_cast<const char *>(pl[p].base) + (size_t)jb * (h ? rb2 : rb4) +
              (size_t)(h ? cs2 * 2 : cs4 * 4);
        bytes = bp;
        dst = s0 + (uint32_t)(p * kSlotBytes) + (h ? d2 : d4);
        step = h ? rb2 : rb4;
        mine_halo = p < NH;
        mine_full = (mask >> p) & 1u;
      }
    }
    if (mine_full || mine_halo) fence_proxy_async_global();  // see the previous pass's stores
    while (issued < R && issued < kStages) issue_one();
  }
  __device__ __forceinline__ void issue_one() {
    __syncwarp();
    const bool halo = (has_above && issued == 0) || (has_below && issued == R - 1);
    const int s = issued % kStages;
    uint64_t *bar = &ring.bars[s];
    if ((threadIdx.x & 31) == 0) mbar_arrive_expect_tx(bar, halo ? tx_halo : tx_full);
    __syncwarp();
    if (halo ? mine_halo : mine_full) {
      fence_proxy_async_shared();  // earlier generic reads of this stage come first
      bulk_copy_g2s_a(dst + (uint32_t)(s * kStageBytes), src, bytes, smem_addr(bar));
    }
    ring.pending |= 1u << s;
    src += step;
    ++issued;
  }
  __device__ __forceinline__ int stage(int k) const { return k % kStages; }
  __device__ __forceinline__ bool ensure(int k) {
    while (ok && waited <= k) {
      ok = ring.wait(stage(waited));
      ++waited;
    }
    return ok;
  }
  __device__ __forceinline__ void release() {
    if (issued < R) issue_one();
  }
};

// Plane order of a CG pass's staged rows: the planes a halo row needs
// (r, s, w, 1/diag, wy) first, then wx, p, x of the own rows.
template <int KIND, bool JOINT = false>
struct CgIdx {
  static constexpr int R = 0;
  static constexpr int S = KIND == 2 ? 1 : 0;
  static constexpr int W = KIND == 0 ? 0 : (KIND == 1 ? 1 : 2);
  static constexpr int ID = KIND == 0 ? 1 : (KIND == 1 ? 2 : 3);
  static constexpr int WY = KIND == 0 ? 2 : (KIND == 1 ? 3 : 4);
  static constexpr int NH = WY + 1;
  static constexpr int WX = NH;
  static constexpr int P = KIND == 2 ? WX + 1 : 0;
  static constexpr int X = KIND == 0 ? 0 : (KIND == 1 ? WX + 1 : WX + 2);
  static constexpr int NP0 = KIND == 0 ? 4 : (KIND == 1 ? 6 : 8);
  static constexpr int WS = NP0;  // joint: the semi-dense weights (own rows only)
  static constexpr int NP = NP0 + (JOINT ? 1 : 0);
};
static_assert(CgIdx<2, true>::NP <= kMaxStagePlanes, "the joint CG pass stages one more plane");

template <int KIND>
__device__ __forceinline__ RowNew<4> ring_row_new(const RowRing &ring, int s, float alpha,
                                                  float beta) {
  using I = CgIdx<KIND>;
  RowNew<4> o;
  o.d = f4v(ring.f4(s, I::ID));
  const F<4> r = f4v(ring.f4(s, I::R));
  o.r_in = r;
  if constexpr (KIND == 0) {
    o.r = r;
    o.s = fzero<4>();
  } else {
    const F<4> w = f4v(ring.f4(s, I::W));
    F<4> sp;
    if constexpr (KIND == 2) sp = f4v(ring.f4(s, I::S));
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      o.s.v[e] = (KIND == 2) ? w.v[e] + beta * sp.v[e] : w.v[e];
      o.r.v[e] = r.v[e] - alpha * o.s.v[e];
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) o.u.v[e] = o.r.v[e] * o.d.v[e];
  return o;
}

template <int KIND>
__device__ __forceinline__ float ring_col_u(const RowRing &ring, int s, int idx, float alpha,
                                            float beta) {
  using I = CgIdx<KIND>;
  const float id = ring.f1(s, I::ID, idx);
  float r = ring.f1(s, I::R, idx);
  if constexpr (KIND != 0) {
    float w = ring.f1(s, I::W, idx);
    if constexpr (KIND == 2) w += beta * ring.f1(s, I::S, idx);
    r -= alpha * w;
  }
  return r * id;
}

// JOINT: w = A u - ws u_t (ut: the border's u_t, the same in every CTA), and
// acc[2] gathers (ws, u) instead of (r, r).
template <int KIND, bool JOINT = false>
__device__ __forceinline__ bool tma_cg_tile(RowRing &ring, const FusedKf &K, const Geo &g, float alpha, float beta,
                            const float *r_cur, const float *s_prev, const float *w_cur,
                            float *r_nxt, float *s_cur, float *w_nxt, float acc[kQ],
                            float ut = 0.0f) {
  using I = CgIdx<KIND, JOINT>;
  const Planes &k = K.pl;
  const int lane = threadIdx.x & 31;
  const int W = k.W, H = k.H;
  const size_t P = k.P;
  StagePlane pl[I::NP];
  pl[I::R] = {r_cur, 4};
  if constexpr (KIND == 2) pl[I::S] = {s_prev, 4};
  if constexpr (KIND != 0) pl[I::W] = {w_cur, 4};
  pl[I::ID] = {k.diag, 4};
  if constexpr (KIND == 2) pl[I::P] = {k.v[0], 4};
  if constexpr (KIND != 0) pl[I::X] = {k.x, 4};
  pl[I::WX] = {k.wx, 4};
  pl[I::WY] = {k.wy, 4};
  if constexpr (JOINT) pl[I::WS] = {k.v[7], 4};
  const int jb = g.r0 > 0 ? g.r0 - 1 : g.r0;
  const int je = min(g.r0 + g.nrows, H - 1);
  TileRows<I::NP, I::NH, 0u> rows(ring, pl, g.c0, (int)P, jb, je - jb + 1, g.r0 > 0,
                                  g.r0 + g.nrows < H);
  F<4> u_up = fzero<4>(), wy_up = fzero<4>();
  int kc = 0;
  if (g.r0 > 0) {
    if (!rows.ensure(0)) return false;
    u_up = ring_row_new<KIND>(ring, rows.stage(0), alpha, beta).u;
    wy_up = f4v(ring.f4(rows.stage(0), I::WY));
    rows.release();
    kc = 1;
  }
  if (!rows.ensure(kc)) return false;
  RowNew<4> cur = ring_row_new<KIND>(ring, rows.stage(kc), alpha, beta);
  size_t i = (size_t)g.r0 * P + g.col;
  for (int j = 0; j < g.nrows; ++j) {
    const int v = g.r0 + j;
    const int sc = rows.stage(kc);
    RowNew<4> nxt;
    F<4> u_dn = fzero<4>();
    if (v + 1 < H) {
      if (!rows.ensure(kc + 1)) return false;
      nxt = ring_row_new<KIND>(ring, rows.stage(kc + 1), alpha, beta);
      u_dn = nxt.u;
    }
    const F<4> wxr = f4v(ring.f4(sc, I::WX)), wyr = f4v(ring.f4(sc, I::WY));
    F<4> u_w, u_e, wx_w;
#pragma unroll
    for (int e = 1; e < 4; ++e) {
      u_w.v[e] = cur.u.v[e - 1];
      wx_w.v[e] = wxr.v[e - 1];
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) u_e.v[e] = cur.u.v[e + 1];
    {
      float uw = shfl_up1(cur.u.v[3]);
      float wxl = shfl_up1(wxr.v[3]);
      float ue = shfl_dn1(cur.u.v[0]);
      if (lane == 0) {
        const bool west = g.col > 0;
        uw = west ? ring_col_u<KIND>(ring, sc, 3, alpha, beta) : 0.0f;
        wxl = west ? ring.f1(sc, I::WX, 3) : 0.0f;
      }
      if (lane == 31) ue = (g.col + 4 < W) ? ring_col_u<KIND>(ring, sc, 132, alpha, beta) : 0.0f;
      u_w.v[0] = uw;
      wx_w.v[0] = wxl;
      u_e.v[3] = ue;
    }
    F<4> w_new;
    if constexpr (JOINT) {
      const F<4> wsr = f4v(ring.f4(sc, I::WS));
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        w_new.v[e] = cur.r.v[e] - (wxr.v[e] * u_e.v[e] + wx_w.v[e] * u_w.v[e] +
                                   wyr.v[e] * u_dn.v[e] + wy_up.v[e] * u_up.v[e]) -
                     wsr.v[e] * ut;
        acc[0] += cur.r.v[e] * cur.u.v[e];
        acc[1] += w_new.v[e] * cur.u.v[e];
        acc[2] += wsr.v[e] * cur.u.v[e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        w_new.v[e] = cur.r.v[e] - (wxr.v[e] * u_e.v[e] + wx_w.v[e] * u_w.v[e] +
                                   wyr.v[e] * u_dn.v[e] + wy_up.v[e] * u_up.v[e]);
        acc[0] += cur.r.v[e] * cur.u.v[e];
        acc[1] += w_new.v[e] * cur.u.v[e];
        acc[2] += cur.r.v[e] * cur.r.v[e];
      }
    }
    stm<4>(w_nxt + i, w_new);
    if constexpr (KIND != 0) {
      F<4> p = (KIND == 2) ? f4v(ring.f4(sc, I::P)) : fzero<4>();
      F<4> x = f4v(ring.f4(sc, I::X));
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float ui = cur.r_in.v[e] * cur.d.v[e];
        p.v[e] = (KIND == 2) ? ui + beta * p.v[e] : ui;
        x.v[e] += alpha * p.v[e];
      }
      stm<4>(k.v[0] + i, p);
      stm<4>(k.x + i, x);
      stm<4>(r_nxt + i, cur.r);
      stm<4>(s_cur + i, cur.s);
    }
    rows.release();
    u_up = cur.u;
    wy_up = wyr;
    cur = nxt;
    ++kc;
    i += P;
  }
  // the halo row below was waited for but is not needed any more
  return rows.ensure(rows.R - 1);
}

template <int LK>
__device__ __forceinline__ bool tma_final_tile(RowRing &ring, const FusedKf &K, const Geo &g, bool first, bool update,
                               float alpha, float beta, bool scale, bool rr, float t, const SolveCfg &c,
                               const float *r_cur, const float *s_prev, const float *w_cur,
                               float acc[kQ]) {
  const Planes &k = K.pl;
  // fixed plane slots; a launch stages only the ones its pass reads
  enum : int { iX = 0, iR, iW, iD, iS, iP, iMS, iVS };
  const StagePlane pl[8] = {{k.x, 4},    {r_cur, 4},  {w_cur, 4},   {k.diag, 4},
                            {s_prev, 4}, {k.v[0], 4}, {k.mu_s, 4}, {k.var_s, 4}};
  uint32_t mask = 1u << iX;
  if (update) mask |= (1u << iR) | (1u << iW) | (1u << iD);
  if (update && !first) mask |= 1u << iP;
  if (update && !first && rr) mask |= 1u << iS;
  if (scale) mask |= (1u << iMS) | (1u << iVS);
  TileRows<8, 8, 0u> rows(ring, pl, g.c0, k.P, g.r0, g.nrows, false, false, mask);
  size_t i = (size_t)g.r0 * k.P + g.col;
  for (int j = 0; j < g.nrows; ++j) {
    if (!rows.ensure(j)) return false;
    const int s = rows.stage(j);
    F<4> x = f4v(ring.f4(s, iX));
    if (update) {
      const F<4> d = f4v(ring.f4(s, iD)), r = f4v(ring.f4(s, iR)), w = f4v(ring.f4(s, iW));
      const F<4> p = first ? fzero<4>() : f4v(ring.f4(s, iP));
      const F<4> sp = first || !rr ? fzero<4>() : f4v(ring.f4(s, iS));
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float ui = r.v[e] * d.v[e];
        const float pi = first ? ui : ui + beta * p.v[e];
        x.v[e] += alpha * pi;
        if (rr) {
          const float si = first ? w.v[e] : w.v[e] + beta * sp.v[e];
          const float rn = r.v[e] - alpha * si;
          acc[0] += rn * rn;
        }
      }
      stm<4>(k.x + i, x);
    }
    if (scale) {
      const F<4> ms = f4v(ring.f4(s, iMS)), vs = f4v(ring.f4(s, iVS));
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (g.col + e < k.W && semi_valid(ms.v[e], vs.v[e])) {
          const float w = robust_weight_k<LK>(x.v[e] - t - ms.v[e], vs.v[e], c.delta);
          acc[1] += w;
          acc[2] += w * (x.v[e] - ms.v[e]);
        }
      }
    }
    rows.release();
    i += k.P;
  }
  return true;
}

template <int LK>
__device__ __forceinline__ bool tma_scale_tile(RowRing &ring, const FusedKf &K, const Geo &g, float t,
                               const SolveCfg &c, float acc[kQ]) {
  const Planes &k = K.pl;
  const StagePlane pl[3] = {{k.x, 4}, {k.mu_s, 4}, {k.var_s, 4}};
  TileRows<3, 3, 0u> rows(ring, pl, g.c0, k.P, g.r0, g.nrows, false, false);
  for (int j = 0; j < g.nrows; ++j) {
    if (!rows.ensure(j)) return false;
    const int s = rows.stage(j);
    const F<4> x = f4v(ring.f4(s, 0)), ms = f4v(ring.f4(s, 1)), vs = f4v(ring.f4(s, 2));
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (g.col + e < k.W && semi_valid(ms.v[e], vs.v[e])) {
        const float w = robust_weight_k<LK>(x.v[e] - t - ms.v[e], vs.v[e], c.delta);
        acc[0] += w;
        acc[1] += w * (x.v[e] - ms.v[e]);
      }
    }
    rows.release();
  }
  return true;
}

// planes of the assembly: the halo rows need x, gy, var_gy (staged first);
// the own rows also mu_s, var_s (f32) and the other network planes
enum : int { A_X = 0, A_GY, A_VY, A_MS, A_VS, A_MN, A_VN, A_GX, A_VX, A_NP };

// JOINT: also keep ws (the semi-dense weights, the x-t coupling of the
// bordered system) in the free work plane v[7], and sum the border's
// S = sum ws and r_t = sum ws (x - t - mu_s) into acc[1], acc[2] (the joint
// solve runs with a fixed iteration count: no r.r, b.b here).
template <int DT, int LK, bool JOINT = false>
__device__ __forceinline__ bool tma_assemble_tile(RowRing &ring, const FusedKf &K, const Geo &g, float t,
                                  const SolveCfg &c, bool wide, float acc[kQ]) {
  const Planes &k = K.pl;
  const int lane = threadIdx.x & 31;
  const int W = k.W, H = k.H;
  const size_t P = k.P;
  const bool semi = c.terms & DF_TERM_SEMI, net = c.terms & DF_TERM_NET,
             grad = c.terms & DF_TERM_GRAD;
  const int es = DT == DF_F32 ? 4 : 2;
  const StagePlane pl[A_NP] = {{k.x, 4},       {k.cnn[4], es}, {k.cnn[5], es},
                               {k.mu_s, 4},    {k.var_s, 4},   {k.cnn[0], es},
                               {k.cnn[1], es}, {k.cnn[2], es}, {k.cnn[3], es}};
  float *r_out = k.v[1];
  const int jb = g.r0 > 0 ? g.r0 - 1 : g.r0;
  const int je = min(g.r0 + g.nrows, H - 1);
  // 16-bit planes: the network planes when DT is BF16 / FP16
  constexpr uint32_t kHalf =
      DT == DF_F32 ? 0u
                   : ((1u << A_GY) | (1u << A_VY) | (1u << A_MN) | (1u << A_VN) | (1u << A_GX) |
                      (1u << A_VX));
  TileRows<A_NP, 3, kHalf> rows(ring, pl, g.c0, (int)P, jb, je - jb + 1, g.r0 > 0,
                                g.r0 + g.nrows < H);
  int kc = 0;
  F<4> wy_up = fzero<4>(), ey_up = fzero<4>(), gy_up = fzero<4>();
  if (g.r0 > 0) {
    if (!rows.ensure(1)) return false;
    const int s0 = rows.stage(0), s1 = rows.stage(1);
    if (grad) {
      const F<4> xu = f4v(ring.f4(s0, A_X)), xc = f4v(ring.f4(s1, A_X));
      const F<4> gyu = cnn4<DT>(ring, s0, A_GY), vyu = cnn4<DT>(ring, s0, A_VY);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (g.col + e < W) {
          gy_up.v[e] = gyu.v[e];
          ey_up.v[e] = xc.v[e] - xu.v[e] - gyu.v[e];
          wy_up.v[e] = robust_weight_k<LK>(ey_up.v[e], vyu.v[e], c.delta);
        }
      }
    }
    rows.release();
    kc = 1;
  }
  size_t i = (size_t)g.r0 * P + g.col;
  for (int j = 0; j < g.nrows; ++j) {
    const int v = g.r0 + j;
    if (!rows.ensure(kc)) return false;
    const int sc = rows.stage(kc);
    const F<4> x_cur = f4v(ring.f4(sc, A_X));
    F<4> x_dn = fzero<4>();
    if (v + 1 < H) {
      if (!rows.ensure(kc + 1)) return false;
      x_dn = f4v(ring.f4(rows.stage(kc + 1), A_X));
    }
    F<4> x_e;
#pragma unroll
    for (int e = 0; e < 3; ++e) x_e.v[e] = x_cur.v[e + 1];
    {
      float xe = shfl_dn1(x_cur.v[0]);
      if (lane == 31) xe = (g.col + 4 < W) ? ring.f1(sc, A_X, 132) : 0.0f;
      x_e.v[3] = xe;
    }
    F<4> wxv = fzero<4>(), exv = fzero<4>(), gxv = fzero<4>();
    F<4> wyv = fzero<4>(), eyv = fzero<4>(), gyv = fzero<4>();
    if (grad) {
      const F<4> gxr = cnn4<DT>(ring, sc, A_GX), vxr = cnn4<DT>(ring, sc, A_VX);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (g.col + e < W - 1) {
          gxv.v[e] = gxr.v[e];
          exv.v[e] = x_e.v[e] - x_cur.v[e] - gxr.v[e];
          wxv.v[e] = robust_weight_k<LK>(exv.v[e], vxr.v[e], c.delta);
        }
      }
      if (v < H - 1) {
        const F<4> gyr = cnn4<DT>(ring, sc, A_GY), vyr = cnn4<DT>(ring, sc, A_VY);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (g.col + e < W) {
            gyv.v[e] = gyr.v[e];
            eyv.v[e] = x_dn.v[e] - x_cur.v[e] - gyr.v[e];
            wyv.v[e] = robust_weight_k<LK>(eyv.v[e], vyr.v[e], c.delta);
          }
        }
      }
    }
    F<4> wxw, exw, gxw;
#pragma unroll
    for (int e = 1; e < 4; ++e) {
      wxw.v[e] = wxv.v[e - 1];
      exw.v[e] = exv.v[e - 1];
      gxw.v[e] = gxv.v[e - 1];
    }
    {
      float a = shfl_up1(wxv.v[3]), b = shfl_up1(exv.v[3]), gg = shfl_up1(gxv.v[3]);
      if (lane == 0) {
        a = b = gg = 0.0f;
        if (grad && g.col > 0 && g.col < W) {
          const float xw = ring.f1(sc, A_X, 3);
          gg = cnn1<DT>(ring, sc, A_GX, 3);
          b = x_cur.v[0] - xw - gg;
          a = robust_weight_k<LK>(b, cnn1<DT>(ring, sc, A_VX, 3), c.delta);
        }
      }
      wxw.v[0] = a;
      exw.v[0] = b;
      gxw.v[0] = gg;
    }
    const F<4> ms = f4v(ring.f4(sc, A_MS)), vs = f4v(ring.f4(sc, A_VS));
    const F<4> mn = cnn4<DT>(ring, sc, A_MN), vn = cnn4<DT>(ring, sc, A_VN);
    F<4> dd, rr_, wsv;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.0f, r = 0.0f, b = 0.0f;
      wsv.v[e] = 0.0f;
      if (g.col + e < W) {
        const float xi = x_cur.v[e];
        float ws = 0.0f, rs = 0.0f, bs = 0.0f;
        if (semi && semi_valid(ms.v[e], vs.v[e])) {
          ws = robust_weight_k<LK>(xi - t - ms.v[e], vs.v[e], c.delta);
          rs = ws * (t + ms.v[e] - xi);
          bs = ws * (t + ms.v[e]);
        }
        if (JOINT) {
          wsv.v[e] = ws;
          acc[1] += ws;
          acc[2] -= rs;  // ws (x - t - mu_s)
        }
        float wn = 0.0f, m = 0.0f;
        if (net) {
          m = mn.v[e];
          wn = robust_weight_k<LK>(xi - m, vn.v[e], c.delta);
        }
        d = ws + wn + wxv.v[e] + wxw.v[e] + wyv.v[e] + wy_up.v[e];
        r = rs + wn * (m - xi) + wxv.v[e] * exv.v[e] - wxw.v[e] * exw.v[e] +
            wyv.v[e] * eyv.v[e] - wy_up.v[e] * ey_up.v[e];
        if (wide)  // b only for the norms a tolerance or a report reads
          b = bs + wn * m - wxv.v[e] * gxv.v[e] + wxw.v[e] * gxw.v[e] - wyv.v[e] * gyv.v[e] +
              wy_up.v[e] * gy_up.v[e];
      }
      const float id = inv_diag(d);
      dd.v[e] = id;
      rr_.v[e] = r;
      acc[0] += r * (r * id);
      if (!JOINT && wide) {
        acc[1] += r * r;
        acc[2] += b * b;
      }
    }
    stm<4>(k.diag + i, dd);
    stm<4>(k.wx + i, wxv);
    stm<4>(k.wy + i, wyv);
    stm<4>(r_out + i, rr_);
    if (JOINT) stm<4>(k.v[7] + i, wsv);
    rows.release();
    wy_up = wyv;
    ey_up = eyv;
    gy_up = gyv;
    ++kc;
    i += P;
  }
  return rows.ensure(rows.R - 1);
}

// ---- the assembly as a kernel of its own ------------------------------------
//
// For streaming plans the IRLS weights, the 5-point system and r0 of each
// Gauss-Newton iteration can run as this ordinary kernel between two
// cooperative launches (the scale step or the previous depth step, and the
// depth step). The persistent kernel runs every pass with one CTA of 8 warps
// per SM, which leaves the assembly (the pass with the most arithmetic per
// byte) bound by instruction latency; here one warp takes one piece (one
// 128-column strip over asm_rows rows), each warp holds the next row's loads
// in registers while it works on the current row (up to 170 registers:
// three blocks of 4 warps per SM), so the loads and the arithmetic overlap.
// Each piece's sums (r.z; r.r and b.b when WIDE) go to its keyframe's
// partial-sum array as double-float pairs, one entry per piece; the depth
// step adds them in a fixed order, so every CTA forms the same scalars.
constexpr int kAsmThreads = 128;
constexpr int kAsmWarps = kAsmThreads / 32;
constexpr int kAsmMaxPieces = kMaxPartialBlocks * kNumQ / kQ;  // float2 entries per keyframe / kQ

__host__ __device__ __forceinline__ int asm_pieces_of(int W, int H, int rows) {
  return ((W + 127) / 128) * ((H + rows - 1) / rows);
}

// One piece of the separate assembly: the arithmetic of assemble_tile (same
// operations in the same order, so the same bits), with every load of the
// next row issued before any of this row's arithmetic (the plane loads do
// not wait for the term flags or for each other), and the inputs read
// through the read-only path (nothing here writes them).
template <int DT, int LK, bool WIDE>
__device__ __forceinline__ void assemble_piece(const Planes &k, const Geo &g, float t,
                                               const SolveCfg &c, float acc[kQ]) {
  const int lane = threadIdx.x & 31;
  const int W = k.W, H = k.H;
  const size_t P = k.P;
  const bool semi = c.terms & DF_TERM_SEMI, net = c.terms & DF_TERM_NET,
             grad = c.terms & DF_TERM_GRAD;
  float *r_out = k.v[1];
  size_t i = (size_t)g.r0 * P + g.col;
  F<4> x_cur = ldr<4>(k.x + i);
  F<4> wy_up = fzero<4>(), ey_up = fzero<4>(), gy_up = fzero<4>();
  if (grad && g.r0 > 0) {
    const F<4> xu = ldr<4>(k.x + i - P);
    const F<4> gyu = ldc<4, DT>(k.cnn[4], i - P), vyu = ldc<4, DT>(k.cnn[5], i - P);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (g.col + e < W) {
        gy_up.v[e] = gyu.v[e];
        ey_up.v[e] = x_cur.v[e] - xu.v[e] - gyu.v[e];
        wy_up.v[e] = robust_weight_k<LK>(ey_up.v[e], vyu.v[e], c.delta);
      }
    }
  }
  const bool has_w = g.col > 0 && g.col < W, has_e = g.col + 4 < W;
  // A row's inputs: x of the row below, the network planes, the semi-dense
  // pair, and the single values past the strip's edges. The next row's are
  // loaded before this row's arithmetic, so each warp keeps two rows of
  // loads in flight.
  struct RowIn {
    F<4> x_dn, gx, vx, gy, vy, ms, vs, mn, vn;
    float xe_l, xw_l, gw_l, vw_l;
  };
  auto load_row = [&](size_t ir, int vr, RowIn &R) {
    R.x_dn = ldr<4>(k.x + (vr + 1 < H ? ir + P : ir));
    R.gx = ldc<4, DT>(k.cnn[2], ir);
    R.vx = ldc<4, DT>(k.cnn[3], ir);
    R.gy = ldc<4, DT>(k.cnn[4], ir);
    R.vy = ldc<4, DT>(k.cnn[5], ir);
    R.ms = ldr<4>(k.mu_s + ir);
    R.vs = ldr<4>(k.var_s + ir);
    R.mn = ldc<4, DT>(k.cnn[0], ir);
    R.vn = ldc<4, DT>(k.cnn[1], ir);
    R.xe_l = R.xw_l = R.gw_l = 0.0f;
    R.vw_l = 1.0f;
    if (lane == 31 && has_e) R.xe_l = __ldg(k.x + ir + 4);
    if (lane == 0 && has_w) {
      R.xw_l = __ldg(k.x + ir - 1);
      R.gw_l = ld_cnn<DT>(k.cnn[2], ir - 1);
      R.vw_l = ld_cnn<DT>(k.cnn[3], ir - 1);
    }
  };
  RowIn cur;
  load_row(i, g.r0, cur);
  for (int j = 0; j < g.nrows; ++j, i += P) {
    const int v = g.r0 + j;
    const bool has_dn = v + 1 < H;
    RowIn nxt;
    if (j + 1 < g.nrows) load_row(i + P, v + 1, nxt);
    const F<4> &x_dn = cur.x_dn, &gxr = cur.gx, &vxr = cur.vx, &gyr = cur.gy, &vyr = cur.vy;
    const F<4> &ms = cur.ms, &vs = cur.vs, &mn = cur.mn, &vn = cur.vn;
    const float xe_l = cur.xe_l, xw_l = cur.xw_l, gw_l = cur.gw_l, vw_l = cur.vw_l;
    F<4> x_e;
#pragma unroll
    for (int e = 0; e < 3; ++e) x_e.v[e] = x_cur.v[e + 1];
    {
      const float xe = shfl_dn1(x_cur.v[0]);
      x_e.v[3] = lane == 31 ? xe_l : xe;
    }
    F<4> wxv = fzero<4>(), exv = fzero<4>(), gxv = fzero<4>();
    F<4> wyv = fzero<4>(), eyv = fzero<4>(), gyv = fzero<4>();
    if (grad) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (g.col + e < W - 1) {
          gxv.v[e] = gxr.v[e];
          exv.v[e] = x_e.v[e] - x_cur.v[e] - gxr.v[e];
          wxv.v[e] = robust_weight_k<LK>(exv.v[e], vxr.v[e], c.delta);
        }
      }
      if (has_dn) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (g.col + e < W) {
            gyv.v[e] = gyr.v[e];
            eyv.v[e] = x_dn.v[e] - x_cur.v[e] - gyr.v[e];
            wyv.v[e] = robust_weight_k<LK>(eyv.v[e], vyr.v[e], c.delta);
          }
        }
      }
    }
    F<4> wxw, exw, gxw;
#pragma unroll
    for (int e = 1; e < 4; ++e) {
      wxw.v[e] = wxv.v[e - 1];
      exw.v[e] = exv.v[e - 1];
      gxw.v[e] = gxv.v[e - 1];
    }
    {
      float a = shfl_up1(wxv.v[3]), b = shfl_up1(exv.v[3]), gg = shfl_up1(gxv.v[3]);
      if (lane == 0) {
        a = b = gg = 0.0f;
        if (grad && has_w) {
          gg = gw_l;
          b = x_cur.v[0] - xw_l - gg;
          a = robust_weight_k<LK>(b, vw_l, c.delta);
        }
      }
      wxw.v[0] = a;
      exw.v[0] = b;
      gxw.v[0] = gg;
    }
    F<4> dd, rr_;  // dd holds 1 / diag
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.0f, r = 0.0f, b = 0.0f;
      if (g.col + e < W) {
        const float xi = x_cur.v[e];
        float ws = 0.0f, rs = 0.0f, bs = 0.0f;
        if (semi && semi_valid(ms.v[e], vs.v[e])) {
          ws = robust_weight_k<LK>(xi - t - ms.v[e], vs.v[e], c.delta);
          rs = ws * (t + ms.v[e] - xi);
          bs = ws * (t + ms.v[e]);
        }
        float wn = 0.0f, m = 0.0f;
        if (net) {
          m = mn.v[e];
          wn = robust_weight_k<LK>(xi - m, vn.v[e], c.delta);
        }
        d = ws + wn + wxv.v[e] + wxw.v[e] + wyv.v[e] + wy_up.v[e];
        r = rs + wn * (m - xi) + wxv.v[e] * exv.v[e] - wxw.v[e] * exw.v[e] +
            wyv.v[e] * eyv.v[e] - wy_up.v[e] * ey_up.v[e];
        if (WIDE)
          b = bs + wn * m - wxv.v[e] * gxv.v[e] + wxw.v[e] * gxw.v[e] - wyv.v[e] * gyv.v[e] +
              wy_up.v[e] * gy_up.v[e];
      }
      const float id = inv_diag(d);
      dd.v[e] = id;
      rr_.v[e] = r;
      acc[0] += r * (r * id);
      if (WIDE) {
        acc[1] += r * r;
        acc[2] += b * b;
      }
    }
    stm<4>(k.diag + i, dd);
    stm<4>(k.wx + i, wxv);
    stm<4>(k.wy + i, wyv);
    stm<4>(r_out + i, rr_);
    wy_up = wyv;
    ey_up = eyv;
    gy_up = gyv;
    x_cur = x_dn;
    cur = nxt;
  }
}

template <int LK, bool WIDE>
__global__ void __launch_bounds__(kAsmThreads, 3) k_assemble_pieces(const PlanHeader *h, SolveCfg c) {
  const int piece = blockIdx.x * kAsmWarps + (threadIdx.x >> 5);
  if (piece >= h->asm_pieces) return;  // whole warps leave
  const FusedKf *kfs =
      reinterpret_cast<const FusedKf *>(reinterpret_cast<const char *>(h) + h->off_kf);
  // the keyframe of this piece: the last one whose first piece is <= piece
  int lo = 0, hi = h->nkf - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (kfs[mid].asm_p0 <= piece) lo = mid; else hi = mid - 1;
  }
  const FusedKf &K = kfs[lo];
  if (K.pl.sc->flags & kFlagBadInput) return;
  const int strips = (K.pl.W + 127) / 128;
  const int q = piece - K.asm_p0, b = q / strips, sx = q - b * strips;
  const int r0 = b * K.asm_rows;
  const Geo g = geo_of<4>(sx * 128, r0, min(K.asm_rows, K.pl.H - r0));
  const float t = (float)K.pl.sc->t;
  float acc[kQ] = {0.0f, 0.0f, 0.0f};
  if (K.pl.dtype == DF_BF16)
    assemble_piece<DF_BF16, LK, WIDE>(K.pl, g, t, c, acc);
  else if (K.pl.dtype == DF_F16)
    assemble_piece<DF_F16, LK, WIDE>(K.pl, g, t, c, acc);
  else
    assemble_piece<DF_F32, LK, WIDE>(K.pl, g, t, c, acc);
  float2 *out = reinterpret_cast<float2 *>(K.pl.partial) + (size_t)q * kQ;
#pragma unroll
  for (int j = 0; j < (WIDE ? kQ : 1); ++j) {
    const ff2 sj = warp_sum_ff(ff2{acc[j], 0.0f});
    if ((threadIdx.x & 31) == 0) __stcg(out + j, make_float2(sj.hi, sj.lo));
  }
}

// Quantity q of a keyframe's n piece sums, this warp's share of a CTA-wide
// sum: thread tid adds entries tid, tid + kThreads, ... in order, eight loads
// in flight at a time, then a fixed warp tree (valid in lane 0); the caller
// adds the warps' results in warp order. Every CTA forms the same value. (One
// warp alone walked the 5400 pieces of a 1920 x 1440 keyframe in ~40
// dependent L2 round trips, ~28 us at the start of every depth-step launch.)
__device__ __forceinline__ ff2 cta_piece_part(const double *partial, int n, int q) {
  const float2 *p = reinterpret_cast<const float2 *>(partial);
  constexpr int kU = 8;
  ff2 acc = ff2{0.0f, 0.0f};
  for (int base = threadIdx.x; base < n; base += kThreads * kU) {
    float2 v[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const int e = base + j * kThreads;
      v[j] = e < n ? __ldcg(p + (size_t)e * kQ + q) : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) acc = ff_add(acc, ff2{v[j].x, v[j].y});
  }
  return warp_sum_ff(acc);
}

// Launch modes of the persistent kernel: the whole schedule, the scale step
// alone, or one Gauss-Newton iteration's depth step after the separate
// assembly (with M_FS: take the next scale step's sums in its last pass;
// with M_RR: reduce r.r in its last pass).
enum : int { M_FULL = 0, M_SCALE = 1, M_DEPTH = 2, M_FS = 4, M_RR = 8 };

struct Seg {
  double t, bb, rr;
  ff2 gam, alpha, beta;  // CG scalars (double-float)
  // joint (x, t) solve: the border's S = sum ws and the t components of the
  // CG vectors (r_t, u_t, w_t, p_t, s_t) and of the step (the change of t)
  ff2 jS, jrt, jut, jwt, jpt, jst, jdt;
  int stop, iters, active, pad;
};

// dynamic shared memory of the VEC = 4 kernel: the warps' row rings + mbarriers
constexpr int kRingSmem = kWarps * kWarpStageBytes + kWarps * kStages * 8;

// JOINT (VEC = 4 only): the joint (x, t) variant, Chronopoulos-Gear PCG on
// the bordered normal equations; each CTA carries the border in its Seg
// scalars, updated identically everywhere from the reduced sums.
template <int VEC, int LK, bool JOINT = false>
__global__ void __launch_bounds__(kThreads, VEC == 4 ? 1 : 2)
    k_fused(PlanHeader *h, SolveCfg c, int n_gn, int n_pcg, unsigned long long limit_ns,
            int first, int mode) {
  extern __shared__ __align__(128) char dyn_ring[];
  __shared__ FusedKf s_kf[kMaxSeg];
  __shared__ Seg s_seg[kMaxSeg];
  __shared__ ff2 s_acc[kWarps][kMaxSeg][kQ];
  __shared__ Slot s_push[kMaxSeg];
  __shared__ SumPrev s_sumprev[kMaxSeg];
  __shared__ int s_okseg[kMaxSeg];
  __shared__ ff2 s_tot[kMaxSeg][kQ];  // this pass's totals
  __shared__ int s_nseg;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = h->G, nkf = h->nkf;
  const char *hb = reinterpret_cast<const char *>(h);
  const int *warp_row = reinterpret_cast<const int *>(hb + h->off_cta_work);
  const int *cta_kf = reinterpret_cast<const int *>(hb + h->off_cta_kf);
  const FusedKf *kfs = reinterpret_cast<const FusedKf *>(hb + h->off_kf);
  SumGroup *groups = reinterpret_cast<SumGroup *>(reinterpret_cast<char *>(h) + h->off_slots);
  const int cta = blockIdx.x;
  const int re = warp_row[(cta + 1) * kWarps];  // end of the CTA's rows
  const int wb = warp_row[cta * kWarps + warp], we = warp_row[cta * kWarps + warp + 1];
  const int th_max = h->th;

  if (tid == 0) {
    int n = 0;
    for (int kk = cta_kf[cta]; kk < nkf && kfs[kk].row_begin < re && n < kMaxSeg; ++kk) {
      s_kf[n] = kfs[kk];
      Seg &s = s_seg[n];
      const Scalars *sc = kfs[kk].pl.sc;
      s.t = sc->t;
      s.gam = s.alpha = s.beta = ff2{0.0f, 0.0f};
      s.jS = s.jrt = s.jut = s.jwt = s.jpt = s.jst = s.jdt = ff2{0.0f, 0.0f};
      s.bb = 0.0;
      s.rr = sc->rr;
      s.stop = 0;
      s.iters = first ? 0 : sc->iters;
      s.active = (sc->flags & kFlagBadInput) ? 0 : 1;
      ++n;
    }
    s_nseg = n;
  }
  // every launch starts from cleared exact-sum words (the plan upload, or
  // the last CTA out of the previous launch, leaves them zero)
  for (int i = tid; i < kMaxSeg * 2 * kSumQ * kSumDigits; i += kThreads)
    (&s_sumprev[0].v[0][0][0])[i] = 0ull;
  RowRing ring;
  if constexpr (VEC == 4) {
    ring.smem = dyn_ring + warp * kWarpStageBytes;
    ring.bars = reinterpret_cast<uint64_t *>(dyn_ring + kWarps * kWarpStageBytes) + warp * kStages;
    ring.parity = 0u;
    ring.pending = 0u;
    ring.limit_ns = limit_ns;
    if (lane == 0) {
      for (int st = 0; st < kStages; ++st) mbar_init(&ring.bars[st], 1u);
      mbar_fence_init();
    }
  }
  __syncthreads();
  const int nseg = s_nseg;
  const bool do_scale = (c.terms & DF_TERM_SEMI) && c.scale_step == DF_SCALE_ALTERNATE;
  int parity = 0;
  bool alive = true;
  const bool wide = c.tol > 0.0 || n_pcg == 0;  // the assembly's r.r and b.b are read

  // One pass over the CTA's tiles, then the exchange of the per-keyframe sums.
  // fin (the last x update only): bit 0 the next scale step's sums, bit 1 r.r
  auto run_pass = [&](int kind, int it, int fin) __attribute__((always_inline)) -> bool {
    // the sums this pass's consumers use: a[q0 .. q0 + nq) of the tiles'
    // accumulators, reduced into s_tot[.][0 .. nq)
    int q0 = 0, nq = kQ;
    switch (kind) {
      case P_SCALE: nq = 2; break;                                      // sum w, sum w (x - mu_s)
      case P_ASSEMBLE: nq = (JOINT || wide) ? 3 : 1; break;              // r.z (r.r, b.b | S, r_t)
      case P_INIT: q0 = 1; nq = JOINT ? 2 : 1; break;                    // (w, u) ((ws, u))
      case P_ITER: nq = (JOINT || c.tol > 0.0) ? 3 : 2; break;           // (r, u), (w, u) (r.r | (ws, u))
      default:                                                           // (r.r) (scale sums)
        q0 = (fin & 2) ? 0 : 1;
        nq = ((fin & 2) ? 1 : 0) + ((fin & 1) ? 2 : 0);
        break;
    }
    for (int q = tid; q < kWarps * kMaxSeg * kQ; q += kThreads) (&s_acc[0][0][0])[q] = ff2{0.0f, 0.0f};
    __syncthreads();
    int seg = 0;
    RowRing rg = ring;  // the ring's phase bits stay in registers for the pass
    // the warp walks its share [wb, we) of the work list in pieces that end
    // at the end of a strip's rows within a row block (or after th_max rows)
    for (int pos = wb; pos < we;) {
      while (pos >= s_kf[seg].row_begin + s_kf[seg].rows) ++seg;
      const FusedKf &K = s_kf[seg];
      const int H = K.pl.H, rel = pos - K.row_begin;
      int sx, r0, end;
      if (K.blk >= H) {  // one block: the strips one after another
        sx = rel / H;
        r0 = rel - sx * H;
        end = H;
      } else {  // row blocks of blk rows (the last one shorter), strips inside
        const int L = K.blk, nstrip = K.rows / H, nb = (H + L - 1) / L;
        const int b = min(rel / (L * nstrip), nb - 1), len = min(L, H - b * L);
        const int off = rel - b * L * nstrip;
        sx = off / len;
        r0 = b * L + (off - sx * len);
        end = b * L + len;
      }
      int nrows = min(end - r0, we - pos);
      if (th_max > 0) nrows = min(nrows, th_max);
      pos += nrows;
      const Seg &S = s_seg[seg];
      if (!S.active) continue;
      const Geo g = geo_of<VEC>(sx * 32 * VEC, r0, nrows);
      float a[kQ] = {0.0f, 0.0f, 0.0f};
      // hi is the float nearest to a double-float value
      const float ft = (float)S.t, fa = S.alpha.hi, fb = S.beta.hi, fu = S.jut.hi;
      float *R0 = K.pl.v[1], *R1 = K.pl.v[2], *S0 = K.pl.v[3], *S1 = K.pl.v[4];
      float *W0 = K.pl.v[5], *W1 = K.pl.v[6];
      float *Rc = (it & 1) ? R1 : R0, *Rn = (it & 1) ? R0 : R1;
      float *Sp = (it & 1) ? S1 : S0, *Sc = (it & 1) ? S0 : S1;
      float *Wc = (it & 1) ? W1 : W0, *Wn = (it & 1) ? W0 : W1;
      if constexpr (VEC == 4) {
        bool ok = true;
        switch (kind) {
          case P_SCALE:
            ok = tma_scale_tile<LK>(rg, K, g, ft, c, a);
            break;
          case P_ASSEMBLE:
            if (K.pl.dtype == DF_BF16)
              ok = tma_assemble_tile<DF_BF16, LK, JOINT>(rg, K, g, ft, c, wide, a);
            else if (K.pl.dtype == DF_F16)
              ok = tma_assemble_tile<DF_F16, LK, JOINT>(rg, K, g, ft, c, wide, a);
            else
              ok = tma_assemble_tile<DF_F32, LK, JOINT>(rg, K, g, ft, c, wide, a);
            break;
          case P_INIT:
            if (!S.stop)
              ok = tma_cg_tile<0, JOINT>(rg, K, g, 0.0f, 0.0f, R0, S0, W1, R1, S1, W0, a, fu);
            break;
          case P_ITER:
            if (!S.stop) {
              if (it == 0)
                ok = tma_cg_tile<1, JOINT>(rg, K, g, fa, fb, Rc, Sp, Wc, Rn, Sc, Wn, a, fu);
              else
                ok = tma_cg_tile<2, JOINT>(rg, K, g, fa, fb, Rc, Sp, Wc, Rn, Sc, Wn, a, fu);
            }
            break;
          default:  // P_FINAL
            ok = tma_final_tile<LK>(rg, K, g, it == 0, !S.stop, fa, fb, fin & 1, fin & 2, ft, c, Rc, Sp,
                                Wc, a);
            break;
        }
        if (!ok) {  // a staged row never arrived: give up the launch
          if (lane == 0) atomicExch(&h->abort, 1u);
          break;
        }
      } else {
      switch (kind) {
        case P_SCALE:
          scale_tile<VEC, LK>(K, g, ft, c, a);
          break;
        case P_ASSEMBLE:
          if (K.pl.dtype == DF_BF16)
            assemble_tile<VEC, DF_BF16, LK>(K, g, ft, c, a);
          else if (K.pl.dtype == DF_F16)
            assemble_tile<VEC, DF_F16, LK>(K, g, ft, c, a);
          else
            assemble_tile<VEC, DF_F32, LK>(K, g, ft, c, a);
          break;
        case P_INIT:
          if (!S.stop) cg_tile<VEC, 0>(K, g, 0.0f, 0.0f, R0, S0, W1, R1, S1, W0, a);
          break;
        case P_ITER:
          if (!S.stop) {
            if (it == 0)
              cg_tile<VEC, 1>(K, g, fa, fb, Rc, Sp, Wc, Rn, Sc, Wn, a);
            else
              cg_tile<VEC, 2>(K, g, fa, fb, Rc, Sp, Wc, Rn, Sc, Wn, a);
          }
          break;
        default:  // P_FINAL
          final_tile<VEC, LK>(K, g, it == 0, !S.stop, fa, fb, fin & 1, ft, c, Rc, Sp, Wc, a);
          break;
      }
      }
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        if (q < nq) {
          const int qa = q0 + q;  // selects, not a dynamic index into a[]
          const float aq = qa == 0 ? a[0] : (qa == 1 ? a[1] : a[2]);
          const ff2 dq = warp_sum_ff(ff2{aq, 0.0f});
          if (lane == 0) s_acc[warp][seg][q] = ff_add(s_acc[warp][seg][q], dq);
        }
      }
    }
    ring = rg;
    __syncthreads();
    // Each keyframe segment's CTA sum, in warp order, then warp sg adds it to
    // keyframe sg's exact-sum words and waits until every CTA of that
    // keyframe has (no grid barrier: a CTA waits only for the CTAs that share
    // its keyframes). A pass without sums still exchanges one zero, which
    // orders its writes before the next pass's reads by the keyframe's CTAs.
    if (tid < nseg * 4) {
      const int sg = tid >> 2, q = tid & 3;
      ff2 s = ff2{0.0f, 0.0f};
      if (q < kQ && q < nq)
        for (int w = 0; w < kWarps; ++w) s = ff_add(s, s_acc[w][sg][q]);
      s_push[sg].v[q] = s;
    }
    __syncthreads();
    long long digit = 0;
    if (warp < nseg) {
      const FusedKf &K = s_kf[warp];
      SumGroup *grp = groups + K.group;
      const int nk = K.slot_end - K.slot_begin;
      bool ok = false;
      if (cta != h->debug_skip_cta) {  // test hook: never arrive
        const int nx = nq > 0 ? nq : 1;
        sum_push(grp, parity, s_push[warp].v, nx);
        ok = sum_wait(grp, parity, nk, nx, &s_sumprev[warp], h, limit_ns, &digit);
      }
      if (lane == 0) s_okseg[warp] = ok ? 1 : 0;
    }
    __syncthreads();
    for (int sg = 0; sg < nseg; ++sg)
      if (!s_okseg[sg]) return false;
    if (warp < nseg) {
      const ff2 tot = sum_total(digit);
      if ((lane & 7) == 0 && (lane >> 3) < nq) s_tot[warp][lane >> 3] = tot;
    }
    __syncthreads();
    parity ^= 1;
    return true;
  };

  auto scale_update = [&](int qw, int qwr) {
    if (tid < nseg) {
      Seg &S = s_seg[tid];
      if (S.active && s_tot[tid][qw].hi > 0.0f)
        S.t = ff_to_double(ff_div(s_tot[tid][qwr], s_tot[tid][qw]));
    }
    __syncthreads();
  };

  // The border of the joint solve moves with the iteration's alpha, beta
  // (right after they are formed): p_t = u_t + beta p_t, s_t = w_t + beta
  // s_t, the change of t += alpha p_t, r_t -= alpha s_t, u_t = r_t / S.
  auto joint_border_step = [](Seg &S, bool first_it) {
    const ff2 a = S.alpha;
    S.jpt = first_it ? S.jut : ff_add(S.jut, ff_mul(S.beta, S.jpt));
    S.jst = first_it ? S.jwt : ff_add(S.jwt, ff_mul(S.beta, S.jst));
    S.jdt = ff_add(S.jdt, ff_mul(a, S.jpt));
    S.jrt = ff_sub(S.jrt, ff_mul(a, S.jst));
    S.jut = S.jS.hi > 0.0f ? ff_div(S.jrt, S.jS) : ff2{0.0f, 0.0f};
  };
  static_assert(!JOINT || VEC == 4, "the joint variant runs on the 4-wide kernel");

  const int lmode = mode & 3;
  if (lmode == M_SCALE) {  // the scale step alone, before a separate assembly
    if (do_scale) {
      alive = run_pass(P_SCALE, 0, 0);
      if (alive) scale_update(0, 1);
    }
    n_gn = 0;
  }
  bool scale_pending = false;
  for (int gn = 0; gn < n_gn && alive; ++gn) {
    if (lmode == M_DEPTH) {
      // the assembly ran as its own kernel: this iteration's r.z (and r.r,
      // b.b) from its pieces' sums, in piece order
      const int nqa = wide ? 3 : 1;
      for (int pq = 0; pq < nseg * nqa; ++pq) {
        const int sg = pq / nqa, q = pq - sg * nqa;
        const FusedKf &K = s_kf[sg];
        const ff2 part =
            cta_piece_part(K.pl.partial, asm_pieces_of(K.pl.W, K.pl.H, K.asm_rows), q);
        if (lane == 0) s_acc[warp][sg][q] = part;
      }
      __syncthreads();
      if (tid < nseg * nqa) {
        const int sg = tid / nqa, q = tid - sg * nqa;
        ff2 tot = s_acc[0][sg][q];
        for (int w = 1; w < kWarps; ++w) tot = ff_add(tot, s_acc[w][sg][q]);
        s_tot[sg][q] = tot;
      }
      __syncthreads();
    } else {
      if (do_scale) {
        if (!scale_pending) {
          alive = run_pass(P_SCALE, 0, 0);
          if (!alive) break;
          scale_update(0, 1);
        }
        scale_pending = false;
      }
      alive = run_pass(P_ASSEMBLE, 0, 0);
      if (!alive) break;
    }
    if (tid < nseg) {
      Seg &S = s_seg[tid];
      S.gam = s_tot[tid][0];
      S.stop = 0;
      if constexpr (JOINT) {
        // border of the bordered system: S = sum ws, r_t, u_t = r_t / S
        S.jS = s_tot[tid][1];
        S.jrt = s_tot[tid][2];
        S.jut = S.jS.hi > 0.0f ? ff_div(S.jrt, S.jS) : ff2{0.0f, 0.0f};
        S.jdt = ff2{0.0f, 0.0f};
        S.gam = ff_add(S.gam, ff_mul(S.jrt, S.jut));
      } else if (c.tol > 0.0 || n_pcg == 0) {
        S.rr = ff_to_double(s_tot[tid][1]);
        S.bb = ff_to_double(s_tot[tid][2]);
        S.stop = (c.tol > 0.0 && sqrt(S.rr) < c.tol * sqrt(S.bb)) ? 1 : 0;
      }
    }
    __syncthreads();
    if (n_pcg == 0) continue;
    alive = run_pass(P_INIT, 0, 0);
    if (!alive) break;
    if (tid < nseg) {
      Seg &S = s_seg[tid];
      if (!S.stop) {
        ff2 dl = s_tot[tid][0];  // (w0, u0)
        if constexpr (JOINT) {  // w_t = S u_t - (ws, u); (w, u) gains w_t u_t
          S.jwt = ff_sub(ff_mul(S.jS, S.jut), s_tot[tid][1]);
          dl = ff_add(dl, ff_mul(S.jwt, S.jut));
        }
        if (S.gam.hi == 0.0f || !(dl.hi > 0.0f)) {
          S.stop = 1;
        } else {
          S.alpha = ff_div(S.gam, dl);
          S.beta = ff2{0.0f, 0.0f};
          if constexpr (JOINT) joint_border_step(S, true);
        }
      }
    }
    __syncthreads();
    for (int it = 0; it < n_pcg; ++it) {
      if (it == n_pcg - 1) {
        // sums needed: the next scale step's two; r.r for a tolerance and
        // for the report after the launch's last GN iteration
        const bool fs = lmode == M_DEPTH ? (mode & M_FS) != 0 : do_scale && gn + 1 < n_gn;
        const bool rr = lmode == M_DEPTH ? (mode & M_RR) != 0 : c.tol > 0.0 || gn + 1 == n_gn;
        alive = run_pass(P_FINAL, it, (fs ? 1 : 0) | (rr ? 2 : 0));
        if (!alive) break;
        if (tid < nseg) {
          Seg &S = s_seg[tid];
          if constexpr (JOINT) {  // the depth step's change of t
            S.t += ff_to_double(S.jdt);
            S.jdt = ff2{0.0f, 0.0f};
          }
          if (!S.stop) {
            S.iters += 1;
            if (rr)
              S.rr = ff_to_double(JOINT ? ff_add(s_tot[tid][0], ff_mul(S.jrt, S.jrt))
                                        : s_tot[tid][0]);
          }
        }
        __syncthreads();
        if (fs) {
          if (rr) scale_update(1, 2);
          else scale_update(0, 1);
          scale_pending = true;
        }
      } else {
        alive = run_pass(P_ITER, it, 0);
        if (!alive) break;
        if (tid < nseg) {
          Seg &S = s_seg[tid];
          if (!S.stop) {
            S.iters += 1;
            ff2 gn_ = s_tot[tid][0], dl = s_tot[tid][1];
            if constexpr (JOINT) {  // border terms of (r, u) and (w, u)
              S.jwt = ff_sub(ff_mul(S.jS, S.jut), s_tot[tid][2]);
              gn_ = ff_add(gn_, ff_mul(S.jrt, S.jut));
              dl = ff_add(dl, ff_mul(S.jwt, S.jut));
            } else if (c.tol > 0.0) {
              S.rr = ff_to_double(s_tot[tid][2]);
            }
            if (c.tol > 0.0 && sqrt(S.rr) < c.tol * sqrt(S.bb)) {
              S.stop = 1;
            } else {
              // beta = gamma / gamma_prev; p.Ap = delta - beta gamma / alpha_prev
              const ff2 beta = ff_div(gn_, S.gam);
              const ff2 denom = ff_sub(dl, ff_div(ff_mul(beta, gn_), S.alpha));
              if (gn_.hi == 0.0f || !(denom.hi > 0.0f)) {
                S.stop = 1;
              } else {
                S.beta = beta;
                S.alpha = ff_div(gn_, denom);
                S.gam = gn_;
                if constexpr (JOINT) joint_border_step(S, false);
              }
            }
          }
        }
        __syncthreads();
      }
    }
  }

  if (tid < nseg) {
    const Seg &S = s_seg[tid];
    const FusedKf &K = s_kf[tid];
    Scalars *sc = K.pl.sc;
    if (!alive) {
      atomicOr(&sc->flags, kFlagTimeout);
    } else if (S.active && K.writer_cta == cta) {
      sc->t = S.t;
      sc->rr = S.rr;
      sc->rho = ff_to_double(S.gam);
      sc->iters = S.iters;
      sc->stop = S.stop;
    }
  }
  if constexpr (VEC == 4) ring.drain();
  grid_exit(h, G, reinterpret_cast<unsigned long long *>(groups),
            (long long)nkf * (long long)(sizeof(SumGroup) / 8));
}

struct DevInfo {
  int sms = 0;
  int occ[2] = {0, 0};  // resident CTAs per SM for VEC = 1, 4
  bool coop = false;
};

DevInfo g_dev[64];
bool g_dev_init[64] = {false};
std::mutex g_dev_mu;

// The kernel instance of a vector width, a loss kind and the joint variant
// (4-wide only).
const void *fused_fn(int vec, int lk, bool joint = false) {
  if (vec == 4 && joint) {
    if (lk == LK_LSQ) return reinterpret_cast<const void *>(k_fused<4, LK_LSQ, true>);
    if (lk == LK_TUKEY) return reinterpret_cast<const void *>(k_fused<4, LK_TUKEY, true>);
    return reinterpret_cast<const void *>(k_fused<4, LK_HUBER, true>);
  }
  if (vec == 4) {
    if (lk == LK_LSQ) return reinterpret_cast<const void *>(k_fused<4, LK_LSQ>);
    if (lk == LK_TUKEY) return reinterpret_cast<const void *>(k_fused<4, LK_TUKEY>);
    return reinterpret_cast<const void *>(k_fused<4, LK_HUBER>);
  }
  if (lk == LK_LSQ) return reinterpret_cast<const void *>(k_fused<1, LK_LSQ>);
  if (lk == LK_TUKEY) return reinterpret_cast<const void *>(k_fused<1, LK_TUKEY>);
  return reinterpret_cast<const void *>(k_fused<1, LK_HUBER>);
}

// The separate assembly's instance of a loss kind (WIDE: with r.r, b.b).
const void *assemble_fn(int lk, bool wide) {
  if (lk == LK_LSQ)
    return wide ? reinterpret_cast<const void *>(k_assemble_pieces<LK_LSQ, true>)
                : reinterpret_cast<const void *>(k_assemble_pieces<LK_LSQ, false>);
  if (lk == LK_TUKEY)
    return wide ? reinterpret_cast<const void *>(k_assemble_pieces<LK_TUKEY, true>)
                : reinterpret_cast<const void *>(k_assemble_pieces<LK_TUKEY, false>);
  return wide ? reinterpret_cast<const void *>(k_assemble_pieces<LK_HUBER, true>)
              : reinterpret_cast<const void *>(k_assemble_pieces<LK_HUBER, false>);
}

const DevInfo &dev_info() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (!g_dev_init[dev]) {
    DevInfo d;
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    d.coop = coop != 0;
    // the instances of one vector width differ only in the loss: the grid
    // follows the least resident of them
    d.occ[0] = d.occ[1] = 1 << 20;
    for (int lk = LK_LSQ; lk <= LK_TUKEY; ++lk) {
      int o1 = 0, o4 = 0, o4j = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, fused_fn(1, lk), kThreads, 0);
      cudaFuncSetAttribute(fused_fn(4, lk), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kRingSmem);
      cudaFuncSetAttribute(fused_fn(4, lk, true), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kRingSmem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o4, fused_fn(4, lk), kThreads, kRingSmem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o4j, fused_fn(4, lk, true), kThreads,
                                                    kRingSmem);
      d.occ[0] = std::min(d.occ[0], o1);
      d.occ[1] = std::min(d.occ[1], std::min(o4, o4j));
      // load the kernels a solve may switch to now, not at their first
      // launch in the middle of a run (lazy module loading can stall a
      // launch for milliseconds)
      cudaFuncAttributes fa;
      cudaFuncGetAttributes(&fa, assemble_fn(lk, false));
      cudaFuncGetAttributes(&fa, assemble_fn(lk, true));
    }
    preload_io_kernels();
    cudaGetLastError();
    g_dev[dev] = d;
    g_dev_init[dev] = true;
  }
  return g_dev[dev];
}

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

}  // namespace

bool streaming_supported() {
  const DevInfo &d = dev_info();
  return d.coop && d.sms > 0 && d.occ[0] > 0 && d.occ[1] > 0;
}

int streaming_max_ctas() {
  const DevInfo &d = dev_info();
  return d.sms * std::max(1, std::max(d.occ[0], d.occ[1]));
}

static size_t streaming_bytes(int nkf, int G) {
  size_t off = align16(sizeof(PlanHeader));
  off += align16(sizeof(int) * ((size_t)G * kWarps + 1));
  off += align16(sizeof(int) * (size_t)G);
  off += align16(sizeof(int) * (size_t)G);
  off += align16(sizeof(FusedKf) * (size_t)nkf);
  off = (off + 255) & ~(size_t)255;
  off += sizeof(SumGroup) * (size_t)nkf;  // one exact-sum group per keyframe
  return off;
}

size_t streaming_plan_bytes(int nkf, int G) { return streaming_bytes(nkf, G); }

bool streaming_build_plan(const Planes *const *kfs, int n, const FusedTuning &tune,
                          std::vector<char> &out, LaunchShape &shape) {
  const DevInfo &d = dev_info();
  if (n < 1 || d.sms <= 0) return false;
  long long rows4 = 0, rows1 = 0;
  for (int k = 0; k < n; ++k) {
    rows4 += (long long)((kfs[k]->W + 127) / 128) * kfs[k]->H;
    rows1 += (long long)((kfs[k]->W + 31) / 32) * kfs[k]->H;
  }
  const int cap_of[2] = {d.sms * std::max(1, d.occ[0]), d.sms * std::max(1, d.occ[1])};
  // 4 pixels per lane once every warp gets at least 2 rows: measured on
  // single keyframes the 4-wide kernel is 1.4x (1024 x 768, ~5 rows per
  // warp) to 1.7x (1280 x 960) faster than the 1-wide one; the 1-wide kernel
  // stays for narrow or small work (many tiny keyframes)
  int vec = tune.vec;
  if (vec != 1 && vec != 4) vec = (rows4 >= 2LL * cap_of[1] * kWarps) ? 4 : 1;
  const int G_cap = std::max(1, std::min(tune.max_ctas > 0 ? tune.max_ctas : cap_of[vec == 4],
                                         cap_of[vec == 4]));
  // Work list: the rows of every keyframe's strips (one column tile of
  // 32 * VEC columns over all H rows), keyframe after keyframe. Each CTA
  // takes a contiguous share of these rows and splits it evenly over its
  // warps, so every warp walks about the same number of rows whatever the
  // keyframes' shapes; a piece of a warp ends at a strip's last row within a
  // row block (or after tile_rows rows, when set). Within a keyframe the list
  // runs over row blocks and within a block over the strips in column order.
  // With blocks of one warp's share, warps next to each other in the list
  // walk neighbouring strips over the same rows at the same time, so the
  // 16-byte side halo a tile row stages from the next strip is still in L2
  // when that strip's own warp reads it.
  std::vector<long long> rb(n + 1, 0);
  for (int k = 0; k < n; ++k)
    rb[k + 1] = rb[k] + (long long)((kfs[k]->W + 32 * vec - 1) / (32 * vec)) * kfs[k]->H;
  const long long R = rb[n];
  if (R > (long long)INT32_MAX / 2) return false;
  const int th_max = tune.tile_rows > 0 ? tune.tile_rows : 0;
  // at least min_rows rows per warp: fewer CTAs for small work (a cheaper
  // exchange); VEC = 4 warps need a few rows to fill their copy ring
  const long long min_rows = std::max<long long>(vec == 4 ? 4 : 1, th_max);
  int G = (int)std::min<long long>(G_cap, std::max<long long>(1, (R + min_rows * kWarps - 1) /
                                                                      (min_rows * kWarps)));
  if (tune.max_ctas > 0) G = std::min(G, tune.max_ctas);
  std::vector<int> wr((size_t)G * kWarps + 1, (int)R), ck(G, n);
  {
    long long pos = 0;
    int kf = 0;
    for (int cI = 0; cI < G; ++cI) {
      while (kf < n && rb[kf + 1] <= pos) ++kf;
      ck[cI] = kf;
      const long long left = R - pos, ctas_left = G - cI;
      long long end = std::min(R, pos + (left + ctas_left - 1) / ctas_left);
      // cap the number of keyframes a CTA touches
      int segs = 0;
      for (int kk = kf; kk < n && rb[kk] < end; ++kk) {
        if (++segs > kMaxSeg) {
          end = rb[kk];
          break;
        }
      }
      for (int w = 0; w < kWarps; ++w) wr[(size_t)cI * kWarps + w] = (int)(pos + (end - pos) * w / kWarps);
      pos = end;
    }
    if (pos != R) return false;  // does not fit: the caller splits the batch
  }
  // drop empty trailing CTAs
  while (G > 1 && wr[(size_t)(G - 1) * kWarps] == R) --G;
  // Row block height. With short warp shares (a few dozen rows) the strips
  // one after another keep neighbouring strips' warps within a few rows of
  // each other, and blocks of a share's height would split most shares into
  // two pieces (two ring fills, two halo rows); measured, blocks cost 6 % at
  // 1920 x 1440 (18-row shares). With long shares (batches: ~200 rows) the
  // warps of neighbouring strips drift a whole share apart and the side halos
  // come from DRAM twice; blocks of one share saved 22 % of the DRAM reads
  // and 7 % of the time on the 64-keyframe batch.
  const long long share = (R + (long long)G * kWarps - 1) / ((long long)G * kWarps);
  const long long blk = share > 32 ? share : (long long)INT32_MAX;
  wr.resize((size_t)G * kWarps + 1);
  wr[(size_t)G * kWarps] = (int)R;
  ck.resize(G);
  // slots: one per (CTA, keyframe segment), in CTA order
  std::vector<int> cs(G);
  std::vector<int> sb(n, -1), se(n, -1), wc(n, -1);
  int ns = 0;
  for (int cI = 0; cI < G; ++cI) {
    cs[cI] = ns;
    const long long c_beg = wr[(size_t)cI * kWarps], c_end = wr[(size_t)(cI + 1) * kWarps];
    for (int kk = ck[cI]; kk < n && rb[kk] < c_end; ++kk) {
      if (rb[kk + 1] <= c_beg) continue;
      if (sb[kk] < 0) {
        sb[kk] = ns;
        wc[kk] = cI;
      }
      se[kk] = ns + 1;
      ++ns;
    }
  }
  for (int k = 0; k < n; ++k)
    if (sb[k] < 0) return false;
  const int nslots = ns;
  for (int k = 0; k < n; ++k)
    if (se[k] - sb[k] > 1023) return false;  // CTAs an exact-sum group counts
  out.assign(streaming_bytes(n, G), 0);
  char *base = out.data();
  PlanHeader *hd = reinterpret_cast<PlanHeader *>(base);
  size_t off = align16(sizeof(PlanHeader));
  hd->off_cta_work = (long long)off;
  off += align16(sizeof(int) * ((size_t)G * kWarps + 1));
  hd->off_cta_kf = (long long)off;
  off += align16(sizeof(int) * (size_t)G);
  hd->off_cta_slot = (long long)off;
  off += align16(sizeof(int) * (size_t)G);
  hd->off_kf = (long long)off;
  off += align16(sizeof(FusedKf) * (size_t)n);
  off = (off + 255) & ~(size_t)255;
  hd->off_slots = (long long)off;
  hd->kind = kPlanStreaming;
  hd->debug_skip_cta = tune.debug_skip_cta;
  hd->nkf = n;
  hd->G = G;
  hd->ntiles = (int)R;  // rows of the work list
  hd->th = th_max;
  hd->nslots = nslots;
  hd->off_flags = 0;
  hd->vec = vec;
  hd->bytes = (long long)out.size();
  memcpy(base + hd->off_cta_work, wr.data(), sizeof(int) * wr.size());
  memcpy(base + hd->off_cta_kf, ck.data(), sizeof(int) * G);
  memcpy(base + hd->off_cta_slot, cs.data(), sizeof(int) * G);
  FusedKf *fk = reinterpret_cast<FusedKf *>(base + hd->off_kf);
  // Pieces of the separate assembly kernel (VEC = 4 plans): strips of
  // asm_rows rows, row block by row block, the strips of a block side by
  // side. Rows per piece: about kAsmTarget pieces over the whole plan (enough
  // warps to cover every SM a few times), at least 4 and at most 32 rows
  // (each piece also weighs the row above it), and few enough pieces per
  // keyframe for its partial-sum array.
  // Auto placement: a kernel of its own when the warps' shares are long
  // (the 64-keyframe batch: ~200 rows, 8 % faster), the persistent kernel's
  // pass when they are shorter (one large keyframe: ~18 rows per warp,
  // where two more launches per GN iteration cost more than the pass
  // gains). Measured on batches of equal keyframes (10 GN x 3 or 5 PCG) the
  // two break even at ~48 rows per warp (six 1280 x 960 keyframes) and the
  // separate kernel is ahead from ~56 (eight 1280 x 960, or 32 of 640 x 480).
  constexpr long long kAsmTarget = 8192;
  const int asm_rows = (int)std::min<long long>(32, std::max<long long>(4, rb[n] / kAsmTarget));
  long long pieces = 0;
  bool split = vec == 4 && (tune.assembly == 2 || (tune.assembly == 0 && share >= 56));
  for (int k = 0; k < n; ++k) {
    fk[k].group = k;
    fk[k].pad = 0;
    fk[k].pl = *kfs[k];
    fk[k].row_begin = (int)rb[k];
    fk[k].rows = (int)(rb[k + 1] - rb[k]);
    fk[k].blk = (int)std::min<long long>(kfs[k]->H, blk);
    fk[k].slot_begin = sb[k];
    fk[k].slot_end = se[k];
    fk[k].writer_cta = wc[k];
    const int strips = (kfs[k]->W + 127) / 128, H = kfs[k]->H;
    int ar = asm_rows;
    if (strips > kAsmMaxPieces) {
      split = false;
    } else if ((long long)strips * ((H + ar - 1) / ar) > kAsmMaxPieces) {
      const int nb = kAsmMaxPieces / strips;
      ar = (H + nb - 1) / nb;
    }
    fk[k].asm_rows = ar;
    fk[k].asm_p0 = (int)pieces;
    pieces += asm_pieces_of(kfs[k]->W, H, ar);
  }
  if (pieces > INT32_MAX / 2) split = false;
  hd->asm_pieces = split ? (int)pieces : 0;
  shape.kind = kPlanStreaming;
  shape.G = G;
  shape.vec = vec;
  shape.smem = 0;
  shape.asm_pieces = hd->asm_pieces;
  return true;
}


// With a separate assembly (shape.asm_pieces > 0 and a depth step to run),
// a launch of n_gn Gauss-Newton iterations becomes: the scale step (when it
// is on), then per iteration the assembly kernel and one depth-step launch
// of the persistent kernel; otherwise one launch of the persistent kernel
// runs them all.
cudaError_t streaming_launch(void *dplan, const LaunchShape &shape, const SolveCfg &c, int n_gn,
                             int n_pcg, unsigned long long limit_ns, cudaStream_t s, int first) {
  PlanHeader *h = static_cast<PlanHeader *>(dplan);
  const int G = shape.G, vec = shape.vec;
  const int lk = loss_kind(c.loss, c.delta);
  const bool joint = (c.terms & DF_TERM_SEMI) && c.scale_step == DF_SCALE_JOINT;
  const void *fn = fused_fn(vec, lk, joint);
  SolveCfg cc = c;
  auto coop = [&](int mode, int ngn, int fst) {
    void *args[] = {&h, &cc, &ngn, &n_pcg, &limit_ns, &fst, &mode};
    count_launches(1);
    return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kThreads), args,
                                       vec == 4 ? (size_t)kRingSmem : 0, s);
  };
  if (shape.asm_pieces <= 0 || n_pcg == 0 || n_gn == 0 || joint)  // joint: the in-kernel pass
    return coop(M_FULL, n_gn, first);
  const bool do_scale = (c.terms & DF_TERM_SEMI) && c.scale_step == DF_SCALE_ALTERNATE;
  const bool wide = c.tol > 0.0;
  const void *afn = assemble_fn(lk, wide);
  const int ablocks = (shape.asm_pieces + kAsmWarps - 1) / kAsmWarps;
  int fst = first;
  cudaError_t e = cudaSuccess;
  if (do_scale) {
    e = coop(M_SCALE, 0, fst);
    fst = 0;
  }
  for (int g = 0; g < n_gn && e == cudaSuccess; ++g) {
    const PlanHeader *hc = h;
    void *aargs[] = {&hc, &cc};
    count_launches(1);
    e = cudaLaunchKernel(afn, dim3(ablocks), dim3(kAsmThreads), aargs, 0, s);
    if (e != cudaSuccess) break;
    const int mode = M_DEPTH | ((do_scale && g + 1 < n_gn) ? M_FS : 0) |
                     ((c.tol > 0.0 || g + 1 == n_gn) ? M_RR : 0);
    e = coop(mode, 1, fst);
    fst = 0;
  }
  return e;
}

// ---- dispatch between the resident and the streaming kernels -------------

bool fused_supported() { return streaming_supported(); }

int fused_max_ctas() { return std::max(streaming_max_ctas(), resident_max_ctas()); }

size_t fused_plan_bytes(int nkf, int G) {
  return std::max(streaming_plan_bytes(nkf, G), resident_plan_bytes(nkf, G));
}

size_t fused_plan_cap_single() {
  return std::max(streaming_plan_bytes(1, streaming_max_ctas()),
                  resident_plan_bytes(1, resident_max_ctas()));
}

bool fused_build_plan(const Planes *const *kfs, int n, const FusedTuning &tune,
                      std::vector<char> &out, LaunchShape &shape) {
  if (tune.mode != kModeStreaming && resident_build_plan(kfs, n, tune, out, shape)) return true;
  if (tune.mode == kModeResident) return false;
  return streaming_build_plan(kfs, n, tune, out, shape);
}

cudaError_t fused_launch(void *dplan, const LaunchShape &shape, const SolveCfg &c, int n_gn,
                         int n_pcg, unsigned long long limit_ns, cudaStream_t s, int first) {
  if (shape.kind == kPlanResident)
    return resident_launch(dplan, shape, c, n_gn, n_pcg, limit_ns, s, first);
  return streaming_launch(dplan, shape, c, n_gn, n_pcg, limit_ns, s, first);
}

}  // namespace df
