// Per-phase kernels of the keyframe optimisation (the "launch" schedule):
// one grid-stride launch per phase, scalars kept on the device in FP64.
//
// Per Gauss-Newton iteration (Section II-C, last paragraph: 10 iterations
// alternating scale and depth):
//   k_scale      scale half: t <- sum w (x - mu_s) / sum w over Eq. 6
//   k_assemble   re-weighting of Eqs. 6-8 at (x, t), the 5-point normal
//                equations (diag, wx, wy) and the PCG start r = b - A x
//   n_pcg x { k_pcg_dir   p = z + beta p (z = r / diag), q = A p, p.q
//             k_pcg_step  x += alpha p, r -= alpha q, r.z }
// Vectors: v[0] = r, v[1], v[2] = p (ping-pong), v[3] = q.
#include <math.h>

#include "df_internal.cuh"

namespace df {

namespace {

constexpr int TX = 32, TY = 8;

struct TileIter {
  int tiles_x, ntiles;
  __device__ TileIter(int W, int H) {
    tiles_x = (W + TX - 1) / TX;
    ntiles = tiles_x * ((H + TY - 1) / TY);
  }
};

__device__ __forceinline__ bool pixel_of(int tile, int tiles_x, int W, int H, int &u, int &v) {
  u = (tile % tiles_x) * TX + threadIdx.x;
  v = (tile / tiles_x) * TY + threadIdx.y;
  return u < W && v < H;
}

// ---- keyframe init: x <- mu_n, t <- 0 (Section II: the CNN prediction
// initialises the keyframe) --------------------------------------------------
template <int DT>
__global__ void k_init_state(Planes k) {
  TileIter it(k.W, k.H);
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const size_t i = (size_t)v * k.P + u;
    k.x[i] = ld_cnn<DT>(k.cnn[0], i);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    k.sc->t = 0.0;
    k.sc->stop = 0;
    k.sc->iters = 0;
    k.sc->count = 0;
    k.sc->rr = 0.0;
  }
}

// ---- device-side input validation (device-pointer inputs) ----------------
template <int DT>
__global__ void k_check_inputs(Planes k) {
  TileIter it(k.W, k.H);
  bool bad = false;
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const size_t i = (size_t)v * k.P + u;
    const float mn = ld_cnn<DT>(k.cnn[0], i), vn = ld_cnn<DT>(k.cnn[1], i);
    bad |= !(isfinite(mn) && isfinite(vn) && vn > 0.0f);
    if (u < k.W - 1) {
      const float g = ld_cnn<DT>(k.cnn[2], i), vg = ld_cnn<DT>(k.cnn[3], i);
      bad |= !(isfinite(g) && isfinite(vg) && vg > 0.0f);
    }
    if (v < k.H - 1) {
      const float g = ld_cnn<DT>(k.cnn[4], i), vg = ld_cnn<DT>(k.cnn[5], i);
      bad |= !(isfinite(g) && isfinite(vg) && vg > 0.0f);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0)
    atomicOr(&k.sc->flags, kFlagBadInput);
}

// ---- scale half of a GN iteration (Eq. 6, t with x fixed) ----------------
__global__ void k_scale(Planes k, SolveCfg c) {
  if (k.sc->flags & kFlagBadInput) return;
  TileIter it(k.W, k.H);
  const float t = (float)k.sc->t;
  float sw = 0.0f, swr = 0.0f;
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const size_t i = (size_t)v * k.P + u;
    const float ms = k.mu_s[i], vs = k.var_s[i];
    if (!semi_valid(ms, vs)) continue;
    const float xi = k.x[i];
    const float w = robust_weight(xi - t - ms, vs, c.delta, c.loss);
    sw += w;
    swr += w * (xi - ms);
  }
  double a[2] = {(double)sw, (double)swr}, out[2];
  if (grid_sum_last_block<2>(a, k.partial, &k.sc->count, out)) {
    if (out[0] > 0.0) k.sc->t = out[1] / out[0];
  }
}

// ---- re-weighting + normal equations + PCG start -------------------------
//
// With weights ws, wn, wx, wy (omega(u)/V of Eqs. 6-8 at the current x, t)
// the depth step minimises
//   sum ws (x_i - t - mu_s)^2 + wn (x_i - mu_n)^2
//     + wx (x_{i+1} - x_i - gx)^2 + wy (x_{i+W} - x_i - gy)^2,
// whose normal equations are the 5-point system
//   diag_i = ws + wn + wx_i + wx_{i-1} + wy_i + wy_{i-W},
//   A_{i,i+1} = -wx_i,  A_{i,i+W} = -wy_i.
// The PCG start residual r = b - A x is formed directly from the term
// residuals (ex = x_{i+1} - x_i - gx_i, ey likewise), which avoids the FP32
// cancellation of forming b and A x separately:
//   r_i = ws (t + mu_s - x_i) + wn (mu_n - x_i) + wx_i ex_i - wx_{i-1} ex_{i-1}
//         + wy_i ey_i - wy_{i-W} ey_{i-W}.
//
// Joint variant (JOINT, scale_step = DF_SCALE_JOINT): the same weights give
// the bordered system in y = (x, t)
//   [ A     -ws ] [x]   [ b - ws t  ]
//   [ -ws^T  S  ] [t] = [ -ws.mu_s  ],   S = sum ws,
// whose residual at (x, t) is r (above) for the x rows and
// r_t = sum ws (x - t - mu_s) for the border; ws is kept in v[4] for the
// operator, and the preconditioner is diag(A) and S.
template <int DT, bool JOINT>
__global__ void k_assemble(Planes k, SolveCfg c) {
  if (k.sc->flags & kFlagBadInput) return;
  TileIter it(k.W, k.H);
  const float t = (float)k.sc->t;
  const bool semi = c.terms & DF_TERM_SEMI, net = c.terms & DF_TERM_NET,
             grad = c.terms & DF_TERM_GRAD;
  const size_t P = k.P;
  float rz = 0.0f, rr = 0.0f, bb = 0.0f;
  float js = 0.0f, jrt = 0.0f, jbt = 0.0f;  // joint: sum ws, r_t, sum ws mu_s
  float *r_out = k.v[0];
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const size_t i = (size_t)v * P + u;
    const float xi = k.x[i];
    float ws = 0.0f, rs = 0.0f, bs = 0.0f;
    if (semi) {
      const float ms = k.mu_s[i], vs = k.var_s[i];
      if (semi_valid(ms, vs)) {
        ws = robust_weight(xi - t - ms, vs, c.delta, c.loss);
        rs = ws * (t + ms - xi);
        bs = JOINT ? ws * ms : ws * (t + ms);
        if (JOINT) {
          js += ws;
          jrt -= rs;
          jbt += ws * ms;
        }
      }
    }
    float wn = 0.0f, mn = 0.0f;
    if (net) {
      mn = ld_cnn<DT>(k.cnn[0], i);
      wn = robust_weight(xi - mn, ld_cnn<DT>(k.cnn[1], i), c.delta, c.loss);
    }
    float wxi = 0.0f, ex = 0.0f, gxi = 0.0f, wxl = 0.0f, exl = 0.0f, gxl = 0.0f;
    float wyi = 0.0f, ey = 0.0f, gyi = 0.0f, wyu = 0.0f, eyu = 0.0f, gyu = 0.0f;
    if (grad) {
      if (u < k.W - 1) {
        gxi = ld_cnn<DT>(k.cnn[2], i);
        ex = k.x[i + 1] - xi - gxi;
        wxi = robust_weight(ex, ld_cnn<DT>(k.cnn[3], i), c.delta, c.loss);
      }
      if (u > 0) {
        gxl = ld_cnn<DT>(k.cnn[2], i - 1);
        exl = xi - k.x[i - 1] - gxl;
        wxl = robust_weight(exl, ld_cnn<DT>(k.cnn[3], i - 1), c.delta, c.loss);
      }
      if (v < k.H - 1) {
        gyi = ld_cnn<DT>(k.cnn[4], i);
        ey = k.x[i + P] - xi - gyi;
        wyi = robust_weight(ey, ld_cnn<DT>(k.cnn[5], i), c.delta, c.loss);
      }
      if (v > 0) {
        gyu = ld_cnn<DT>(k.cnn[4], i - P);
        eyu = xi - k.x[i - P] - gyu;
        wyu = robust_weight(eyu, ld_cnn<DT>(k.cnn[5], i - P), c.delta, c.loss);
      }
    }
    const float d = ws + wn + wxi + wxl + wyi + wyu;
    const float r = rs + wn * (mn - xi) + wxi * ex - wxl * exl + wyi * ey - wyu * eyu;
    k.diag[i] = d;
    k.wx[i] = wxi;
    k.wy[i] = wyi;
    r_out[i] = r;
    if (JOINT) k.v[4][i] = ws;
    const float z = r * inv_diag(d);
    rz += r * z;
    rr += r * r;
    if (c.tol > 0.0) {
      const float b = bs + wn * mn - wxi * gxi + wxl * gxl - wyi * gyi + wyu * gyu;
      bb += b * b;
    }
  }
  if constexpr (!JOINT) {
    double a[3] = {(double)rz, (double)rr, (double)bb}, out[3];
    if (grid_sum_last_block<3>(a, k.partial, &k.sc->count, out)) {
      k.sc->rho = out[0];
      k.sc->rr = out[1];
      k.sc->bb = out[2];
      k.sc->stop = (c.tol > 0.0 && sqrt(out[1]) < c.tol * sqrt(out[2])) ? 1 : 0;
    }
  } else {
    double a[6] = {(double)rz, (double)rr, (double)bb, (double)js, (double)jrt, (double)jbt},
           out[6];
    if (grid_sum_last_block<6>(a, k.partial, &k.sc->count, out)) {
      const double S = out[3], rt = out[4], zt = S > 0.0 ? rt / S : 0.0;
      k.sc->j_s = S;
      k.sc->j_rt = rt;
      k.sc->rho = out[0] + rt * zt;
      k.sc->rr = out[1] + rt * rt;
      k.sc->bb = out[2] + out[5] * out[5];
      k.sc->stop =
          (c.tol > 0.0 && sqrt(k.sc->rr) < c.tol * sqrt(k.sc->bb)) ? 1 : 0;
    }
  }
}

// ---- PCG direction: p_new = z + beta p_old (z = r / diag), q = A p_new -----
// p_new at the four neighbours is recomputed from their r, diag, p_old, so
// one launch both updates p and applies the stencil (p is double-buffered).
// Joint: the direction's border component p_t = z_t + beta p_t (z_t = r_t / S)
// enters q_x = A p_x - ws p_t, and q_t = S p_t - ws.p_x follows from one more
// sum.
template <bool JOINT>
__global__ void k_pcg_dir(Planes k, int first, const float *__restrict__ p_old,
                          float *__restrict__ p_new) {
  if (k.sc->stop || (k.sc->flags & kFlagBadInput)) return;
  TileIter it(k.W, k.H);
  const float beta = first ? 0.0f : (float)k.sc->beta;
  double pt = 0.0;
  if (JOINT) {
    const double S = k.sc->j_s, zt = S > 0.0 ? k.sc->j_rt / S : 0.0;
    pt = first ? zt : zt + k.sc->beta * k.sc->j_pt;
  }
  const float ptf = (float)pt;
  const float *r = k.v[0];
  float *q = k.v[3];
  const size_t P = k.P;
  auto pn = [&](size_t j) {
    const float d = k.diag[j];
    const float z = r[j] * inv_diag(d);
    return first ? z : z + beta * p_old[j];
  };
  float pq = 0.0f, wp = 0.0f;
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const size_t i = (size_t)v * P + u;
    const float pc = pn(i);
    float a = k.diag[i] * pc;
    if (u < k.W - 1) a -= k.wx[i] * pn(i + 1);
    if (u > 0) a -= k.wx[i - 1] * pn(i - 1);
    if (v < k.H - 1) a -= k.wy[i] * pn(i + P);
    if (v > 0) a -= k.wy[i - P] * pn(i - P);
    if (JOINT) {
      const float ws = k.v[4][i];
      a -= ws * ptf;
      wp += ws * pc;
    }
    p_new[i] = pc;
    q[i] = a;
    pq += pc * a;
  }
  double s[2] = {(double)pq, (double)wp}, out[2];
  if (grid_sum_last_block<2>(s, k.partial, &k.sc->count, out)) {
    double gamma = out[0];
    if (JOINT) {
      const double qt = k.sc->j_s * pt - out[1];
      k.sc->j_pt = pt;
      k.sc->j_qt = qt;
      gamma += pt * qt;
    }
    k.sc->gamma = gamma;
    if (gamma <= 0.0 || k.sc->rho == 0.0) {
      k.sc->stop = 1;  // breakdown or exact solution: this depth step ends
    } else {
      k.sc->alpha = k.sc->rho / gamma;
    }
  }
}

// ---- PCG step: x += alpha p, r -= alpha q, new r.z -----------------------
// Joint: the last block also moves t and the border residual.
template <bool JOINT>
__global__ void k_pcg_step(Planes k, double tol, const float *__restrict__ p) {
  if (k.sc->stop || (k.sc->flags & kFlagBadInput)) return;
  TileIter it(k.W, k.H);
  const float alpha = (float)k.sc->alpha;
  float *r = k.v[0];
  const float *q = k.v[3];
  float rz = 0.0f, rr = 0.0f;
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const size_t i = (size_t)v * k.P + u;
    k.x[i] += alpha * p[i];
    const float ri = r[i] - alpha * q[i];
    r[i] = ri;
    const float d = k.diag[i];
    const float z = ri * inv_diag(d);
    rz += ri * z;
    rr += ri * ri;
  }
  double s[2] = {(double)rz, (double)rr}, out[2];
  if (grid_sum_last_block<2>(s, k.partial, &k.sc->count, out)) {
    k.sc->iters += 1;
    if (JOINT) {
      const double a = k.sc->alpha, S = k.sc->j_s;
      k.sc->t += a * k.sc->j_pt;
      const double rt = k.sc->j_rt - a * k.sc->j_qt;
      k.sc->j_rt = rt;
      out[0] += S > 0.0 ? rt * (rt / S) : 0.0;
      out[1] += rt * rt;
    }
    k.sc->rr = out[1];
    if (tol > 0.0 && sqrt(out[1]) < tol * sqrt(k.sc->bb)) {
      k.sc->stop = 1;
    } else {
      k.sc->beta = out[0] / k.sc->rho;
      k.sc->rho = out[0];
    }
  }
}

// ---- output: d = exp(x) (or x), dense H x W --------------------------------
__global__ void k_fetch(Planes k, float *out, int log_space) {
  TileIter it(k.W, k.H);
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const float xi = k.x[(size_t)v * k.P + u];
    out[(size_t)v * k.W + u] = log_space ? xi : expf(xi);
  }
}

__global__ void k_set_x(Planes k, const float *xd) {
  TileIter it(k.W, k.H);
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    k.x[(size_t)v * k.P + u] = xd[(size_t)v * k.W + u];
  }
}

__global__ void k_set_scale(Scalars *sc, double t) { sc->t = t; }

// ---- Table II's least-squares scale fit (Section III-C) -------------------
// After a scale-ambiguous solve, the log offset c minimising
// sum_i (x_i + c - mu_n,i)^2 is mean(mu_n - x); x += c and t += c keep the
// semi-dense residuals x - t - mu_s unchanged.
template <int DT>
__global__ void k_lsfit_sum(Planes k) {
  TileIter it(k.W, k.H);
  float acc = 0.0f;
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const size_t i = (size_t)v * k.P + u;
    acc += ld_cnn<DT>(k.cnn[0], i) - k.x[i];
  }
  double a[1] = {(double)acc}, out[1];
  if (grid_sum_last_block<1>(a, k.partial, &k.sc->count, out)) {
    const double c = out[0] / ((double)k.W * (double)k.H);
    k.sc->gamma = c;  // the shift, read by k_lsfit_shift
    k.sc->t += c;
  }
}

__global__ void k_lsfit_shift(Planes k) {
  TileIter it(k.W, k.H);
  const float c = (float)k.sc->gamma;
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    k.x[(size_t)v * k.P + u] += c;
  }
}

// ---- cost c(x, t) of Eq. 5 with the robust loss (FP64) --------------------
template <int DT>
__global__ void k_cost(Planes k, SolveCfg c) {
  TileIter it(k.W, k.H);
  const double t = k.sc->t;
  const double delta = c.delta;
  const size_t P = k.P;
  double acc = 0.0;
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const size_t i = (size_t)v * P + u;
    const double xi = k.x[i];
    if (c.terms & DF_TERM_SEMI) {
      const float ms = k.mu_s[i], vs = k.var_s[i];
      if (semi_valid(ms, vs)) acc += robust_rho(xi - t - ms, vs, delta, c.loss);
    }
    if (c.terms & DF_TERM_NET)
      acc += robust_rho(xi - ld_cnn<DT>(k.cnn[0], i), ld_cnn<DT>(k.cnn[1], i), delta, c.loss);
    if (c.terms & DF_TERM_GRAD) {
      if (u < k.W - 1)
        acc += robust_rho((double)k.x[i + 1] - xi - ld_cnn<DT>(k.cnn[2], i),
                          ld_cnn<DT>(k.cnn[3], i), delta, c.loss);
      if (v < k.H - 1)
        acc += robust_rho((double)k.x[i + P] - xi - ld_cnn<DT>(k.cnn[4], i),
                          ld_cnn<DT>(k.cnn[5], i), delta, c.loss);
    }
  }
  double s[1] = {acc}, out[1];
  if (grid_sum_last_block<1>(s, k.partial, &k.sc->count, out)) k.sc->cost = out[0];
}

// ---- accuracy metric of Section III-B: depth within rel_tol of the truth ---
// Counts, over the pixels with a finite ground truth g > 0, those with
// |exp(x) - g| <= rel_tol * g (decided in FP64). Counts are summed as
// doubles, exact below 2^53.
__global__ void k_accuracy(Planes k, const float *__restrict__ d_true, double rel_tol) {
  TileIter it(k.W, k.H);
  double n_in = 0.0, n_valid = 0.0;
  for (int tile = blockIdx.x; tile < it.ntiles; tile += gridDim.x) {
    int u, v;
    if (!pixel_of(tile, it.tiles_x, k.W, k.H, u, v)) continue;
    const double g = d_true[(size_t)v * k.W + u];
    if (!(g > 0.0) || !isfinite(g)) continue;
    n_valid += 1.0;
    const double d = exp((double)k.x[(size_t)v * k.P + u]);
    if (fabs(d - g) <= rel_tol * g) n_in += 1.0;
  }
  double s[2] = {n_in, n_valid}, out[2];
  if (grid_sum_last_block<2>(s, k.partial, &k.sc->count, out)) {
    k.sc->acc_in = out[0];
    k.sc->acc_valid = out[1];
  }
}

// ---- Section II-B: semi-dense depth / variance to log space ---------------
__global__ void k_semi_to_log(const float *d, const float *vd, float *mu, float *var,
                              int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float di = d[i], vi = vd[i];
    if (isfinite(di) && di > 0.0f && isfinite(vi) && vi > 0.0f) {
      mu[i] = logf(di);
      var[i] = vi / (di * di);
    } else {
      mu[i] = 0.0f;
      var[i] = 0.0f;
    }
  }
}

int g_num_sms = 0;

}  // namespace

int launch_grid(int tiles) {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  int cap = g_num_sms * 8;
  if (cap > kMaxPartialBlocks) cap = kMaxPartialBlocks;
  return tiles < cap ? (tiles < 1 ? 1 : tiles) : cap;
}

static int tiles_of(const Planes &k) {
  return ((k.W + TX - 1) / TX) * ((k.H + TY - 1) / TY);
}

#define DF_DISPATCH_DT(dt, KERNEL, ...)                          \
  do {                                                           \
    if ((dt) == DF_BF16)                                         \
      KERNEL<DF_BF16><<<__VA_ARGS__>>>;                          \
    else if ((dt) == DF_F16)                                     \
      KERNEL<DF_F16><<<__VA_ARGS__>>>;                           \
    else                                                         \
      KERNEL<DF_F32><<<__VA_ARGS__>>>;                           \
  } while (0)

cudaError_t launch_init_state(const Planes &k, cudaStream_t s) {
  count_launches(1);
  const dim3 blk(TX, TY), grd(launch_grid(tiles_of(k)));
  if (k.dtype == DF_BF16)
    k_init_state<DF_BF16><<<grd, blk, 0, s>>>(k);
  else if (k.dtype == DF_F16)
    k_init_state<DF_F16><<<grd, blk, 0, s>>>(k);
  else
    k_init_state<DF_F32><<<grd, blk, 0, s>>>(k);
  return cudaGetLastError();
}

cudaError_t launch_check_inputs(const Planes &k, cudaStream_t s) {
  count_launches(1);
  const dim3 blk(TX, TY), grd(launch_grid(tiles_of(k)));
  if (k.dtype == DF_BF16)
    k_check_inputs<DF_BF16><<<grd, blk, 0, s>>>(k);
  else if (k.dtype == DF_F16)
    k_check_inputs<DF_F16><<<grd, blk, 0, s>>>(k);
  else
    k_check_inputs<DF_F32><<<grd, blk, 0, s>>>(k);
  return cudaGetLastError();
}

template <bool JOINT>
static void solve_launches(const Planes &k, const SolveCfg &c, int n_gn, int n_pcg, bool scale,
                           dim3 grd, dim3 blk, cudaStream_t s) {
  for (int g = 0; g < n_gn; ++g) {
    if (scale) k_scale<<<grd, blk, 0, s>>>(k, c);
    if (k.dtype == DF_BF16)
      k_assemble<DF_BF16, JOINT><<<grd, blk, 0, s>>>(k, c);
    else if (k.dtype == DF_F16)
      k_assemble<DF_F16, JOINT><<<grd, blk, 0, s>>>(k, c);
    else
      k_assemble<DF_F32, JOINT><<<grd, blk, 0, s>>>(k, c);
    for (int j = 0; j < n_pcg; ++j) {
      float *p_old = k.v[1 + (j & 1)];
      float *p_new = k.v[1 + ((j + 1) & 1)];
      k_pcg_dir<JOINT><<<grd, blk, 0, s>>>(k, j == 0, p_old, p_new);
      k_pcg_step<JOINT><<<grd, blk, 0, s>>>(k, c.tol, p_new);
    }
  }
}

cudaError_t launch_solve_launches(const Planes &k, const SolveCfg &c, int n_gn, int n_pcg,
                                  cudaStream_t s) {
  const dim3 blk(TX, TY), grd(launch_grid(tiles_of(k)));
  const bool semi = (c.terms & DF_TERM_SEMI) != 0;
  const bool joint = semi && c.scale_step == DF_SCALE_JOINT;
  const bool scale = semi && c.scale_step == DF_SCALE_ALTERNATE;
  count_launches((unsigned)(n_gn * ((scale ? 2 : 1) + 2 * n_pcg)));
  if (joint)
    solve_launches<true>(k, c, n_gn, n_pcg, scale, grd, blk, s);
  else
    solve_launches<false>(k, c, n_gn, n_pcg, scale, grd, blk, s);
  return cudaGetLastError();
}

cudaError_t launch_fetch(const Planes &k, float *out, int log_space, cudaStream_t s) {
  count_launches(1);
  k_fetch<<<launch_grid(tiles_of(k)), dim3(TX, TY), 0, s>>>(k, out, log_space);
  return cudaGetLastError();
}

cudaError_t launch_set_x(const Planes &k, const float *xd, cudaStream_t s) {
  count_launches(1);
  k_set_x<<<launch_grid(tiles_of(k)), dim3(TX, TY), 0, s>>>(k, xd);
  return cudaGetLastError();
}

cudaError_t launch_set_scale(const Planes &k, double t, cudaStream_t s) {
  count_launches(1);
  k_set_scale<<<1, 1, 0, s>>>(k.sc, t);
  return cudaGetLastError();
}

cudaError_t launch_ls_scale_fit(const Planes &k, cudaStream_t s) {
  count_launches(2);
  const dim3 blk(TX, TY), grd(launch_grid(tiles_of(k)));
  if (k.dtype == DF_BF16)
    k_lsfit_sum<DF_BF16><<<grd, blk, 0, s>>>(k);
  else if (k.dtype == DF_F16)
    k_lsfit_sum<DF_F16><<<grd, blk, 0, s>>>(k);
  else
    k_lsfit_sum<DF_F32><<<grd, blk, 0, s>>>(k);
  k_lsfit_shift<<<grd, blk, 0, s>>>(k);
  return cudaGetLastError();
}

cudaError_t launch_accuracy(const Planes &k, const float *d_true, double rel_tol,
                            cudaStream_t s) {
  count_launches(1);
  const dim3 blk(TX, TY), grd(launch_grid(tiles_of(k)));
  k_accuracy<<<grd, blk, 0, s>>>(k, d_true, rel_tol);
  return cudaGetLastError();
}

cudaError_t launch_cost(const Planes &k, const SolveCfg &c, cudaStream_t s) {
  count_launches(1);
  const dim3 blk(TX, TY), grd(launch_grid(tiles_of(k)));
  if (k.dtype == DF_BF16)
    k_cost<DF_BF16><<<grd, blk, 0, s>>>(k, c);
  else if (k.dtype == DF_F16)
    k_cost<DF_F16><<<grd, blk, 0, s>>>(k, c);
  else
    k_cost<DF_F32><<<grd, blk, 0, s>>>(k, c);
  return cudaGetLastError();
}

cudaError_t launch_semi_to_log(const float *d, const float *vd, float *mu, float *var,
                               int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  const int cap = launch_grid(1 << 30);
  if (blocks > cap) blocks = cap;
  count_launches(1);
  k_semi_to_log<<<(int)blocks, 256, 0, s>>>(d, vd, mu, var, n);
  return cudaGetLastError();
}

}  // namespace df
