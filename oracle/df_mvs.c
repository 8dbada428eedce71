/*
 * Semi-dense depth from two views -- FP64 CPU ORACLE (test infrastructure).
 *
 * Only the tests, the smoke check and the benchmark's CPU legs load this
 * file; the product path never calls it and shares no code with it.
 *
 * What it computes (paper Section II-B, "Semi-Dense Estimation", which follows
 * the per-pixel stereo of LSD-SLAM's semi-dense mapping): for every keyframe
 * pixel with enough texture, the depth along its ray that best explains a
 * reference image, and the variance of that measurement, then the Gaussian
 * fusion of the measurement with the pixel's current estimate.
 *
 *  - Photometric error (Eq. 2): e = I_1(pi(K T_ref<-key rho(x, d))) - I_0(x).
 *    Five equally spaced keyframe points x + s e0 (s = -2..2, 1 px apart
 *    along the keyframe's epipolar line at x) are compared with their
 *    projections into the reference image at the candidate depth d, giving
 *    the 5-vector e(d) and SSD(d) = e.e.
 *  - Search: with a current estimate (d, sigma^2) the depths in
 *    [d - k sigma, d + k sigma] (k = 2 in the paper), else [d_min, d_max];
 *    the interval's ends project to the reference image, and the segment
 *    between them is walked in 1-pixel steps q_j = P_lo + j u (u the unit
 *    direction), j = 0 .. floor(L) with L the segment's length. Each step's
 *    depth is the one whose projection is q_j (closed form below).
 *  - Sub-pixel step: from the best step a and its better neighbour b (steps
 *    a - 1 and a + 1, evaluated even just beyond the interval), the error is
 *    linearised between them, e(s) = e_a + s (e_b - e_a), and minimised over
 *    s in [0, 1]: d = d_a + s (d_b - d_a).
 *  - Variance (Eqs. 3, 4): J = (e_b - e_a) / (d_b - d_a), sigma^2 =
 *    photo_var (J^T J)^-1 with photo_var = 1 in the paper's formula.
 *  - Fusion with the current estimate (Gaussian product): var' = var var_o /
 *    (var + var_o), d' = (d var_o + d_o var) / (var + var_o).
 *
 * Readings where the paper is silent are listed in the design notes: the
 * texture test (central-difference gradient magnitude >= grad_min), the
 * reference samples (the keyframe samples projected at the candidate depth),
 * the tie rules (first minimum; equal neighbours take a - 1), the rejection
 * rules (status codes below) and bilinear interpolation of both images.
 *
 * Besides the result, each pixel gets a status, its best step and a
 * decision margin: the smallest normalised distance of any decision taken
 * for it (threshold tests, the argmin, the neighbour choice, the step count,
 * image-border tests) from flipping; tests compare a reduced-precision
 * implementation with this one decision by decision only where the margin
 * is clear.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#ifndef ORC_MUTANT
#define ORC_MUTANT 0 /* >0 only in the tests' planted-mistake builds */
#endif

typedef struct {
  double fx, fy, cx, cy;
} orc_camera;

typedef struct {
  double R[9]; /* row-major: X_ref = R X_key + t */
  double t[3];
} orc_pose;

typedef struct {
  double grad_min;    /* texture: |grad I_0| (central differences) >= grad_min */
  double d_min, d_max;/* search range without an estimate */
  double sigma_range; /* interval half-width in sigmas with an estimate (2) */
  double ssd_max;     /* a best SSD above this gives no measurement */
  double photo_var;   /* image noise variance in sigma^2 = photo_var (J^T J)^-1 */
  int32_t max_steps;  /* a segment of more steps gives no measurement */
} orc_mvs_params;

enum {
  MVS_OK = 0,        /* measured (and fused) */
  MVS_FLAT = 1,      /* image border or too little texture */
  MVS_INTERVAL = 2,  /* empty search interval */
  MVS_LINE = 3,      /* degenerate or too long epipolar segment, samples outside */
  MVS_NOSTEP = 4,    /* no step with all samples inside the reference image */
  MVS_SSD = 5,       /* best SSD above ssd_max */
  MVS_NEIGHBOUR = 6  /* no usable neighbour step for the sub-pixel fit */
};

static double dmin(double a, double b) { return a < b ? a : b; }

/* Bilinear sample of I (H x W, row-major) at (x, y); 0 if outside
 * [0, W-1] x [0, H-1]. *edge tracks the smallest distance of any sample to
 * that boundary (for the decision margin). */
static int bilinear(const float *I, int W, int H, double x, double y, double *out, double *edge) {
  const double dist = dmin(dmin(x, (double)(W - 1) - x), dmin(y, (double)(H - 1) - y));
  *edge = dmin(*edge, fabs(dist));
  if (!(x >= 0.0 && y >= 0.0 && x <= (double)(W - 1) && y <= (double)(H - 1))) return 0;
  int x0 = (int)floor(x), y0 = (int)floor(y);
  if (x0 > W - 2) x0 = W - 2;
  if (y0 > H - 2) y0 = H - 2;
  if (x0 < 0) x0 = 0;
  if (y0 < 0) y0 = 0;
  const double ax = x - x0, ay = y - y0;
  const int x1 = W > 1 ? x0 + 1 : x0, y1 = H > 1 ? y0 + 1 : y0;
  const double top = (1.0 - ax) * I[(size_t)y0 * W + x0] + ax * I[(size_t)y0 * W + x1];
  const double bot = (1.0 - ax) * I[(size_t)y1 * W + x0] + ax * I[(size_t)y1 * W + x1];
  *out = (1.0 - ay) * top + ay * bot;
  return 1;
}

/* Projection into the reference image of keyframe point (u, v) at depth d. */
static int project(const orc_camera *c, const orc_pose *T, double u, double v, double d,
                   double *pu, double *pv) {
  const double X[3] = {d * (u - c->cx) / c->fx, d * (v - c->cy) / c->fy, d};
  double Y[3];
  for (int r = 0; r < 3; ++r)
    Y[r] = T->R[3 * r] * X[0] + T->R[3 * r + 1] * X[1] + T->R[3 * r + 2] * X[2] + T->t[r];
  if (!(Y[2] > 0.0)) return 0;
  *pu = c->fx * Y[0] / Y[2] + c->cx;
  *pv = c->fy * Y[1] / Y[2] + c->cy;
  return 1;
}

/* Photometric error vector and SSD of step j (depth *dj): 1 if every sample
 * is inside the reference image and the depth is positive. */
static int step_error(const float *I1, int W, int H, const orc_camera *c, const orc_pose *T,
                      double u, double v, const double e0[2], const double key[5],
                      const double a[3], int use_x, const double P0[2], const double dir[2],
                      int j, double e[5], double *ssd, double *dj, double *edge) {
  const double qx = P0[0] + j * dir[0], qy = P0[1] + j * dir[1];
  /* depth whose projection is q: with Y = d a + t (a = R K^-1 [u v 1]^T),
   * q~ = Y_x / Y_z gives d (q~ a_z - a_x) = t_x - q~ t_z (or the y row) */
  double d;
  if (use_x) {
    const double qt = (qx - c->cx) / c->fx;
    d = (T->t[0] - qt * T->t[2]) / (qt * a[2] - a[0]);
  } else {
    const double qt = (qy - c->cy) / c->fy;
    d = (T->t[1] - qt * T->t[2]) / (qt * a[2] - a[1]);
  }
  if (!(d > 0.0) || !isfinite(d)) return 0;
  double s2 = 0.0;
  for (int s = -2; s <= 2; ++s) {
    double pu, pv, val;
    if (!project(c, T, u + s * e0[0], v + s * e0[1], d, &pu, &pv)) return 0;
    if (!bilinear(I1, W, H, pu, pv, &val, edge)) return 0;
    e[s + 2] = val - key[s + 2];
    s2 += e[s + 2] * e[s + 2];
  }
  *ssd = s2;
  *dj = d;
  return 1;
}

/* One stereo update of the keyframe's semi-dense estimate (in place).
 * img_key, img_ref: H x W intensities. depth, var: the current estimate
 * (var <= 0 or non-finite: none), replaced by the fused one where a
 * measurement was made. status, best_step, margin: per-pixel diagnostics
 * (may be NULL). Returns the number of measured pixels. */
int64_t orc_semi_dense(int32_t W, int32_t H, const float *img_key, const float *img_ref,
                       const orc_camera *cam, const orc_pose *T, const orc_mvs_params *prm,
                       double *depth, double *var, int32_t *status, int32_t *best_step,
                       double *margin) {
  /* reference camera centre in keyframe coordinates: C = -R^T t */
  double C[3];
  for (int r = 0; r < 3; ++r)
    C[r] = -(T->R[r] * T->t[0] + T->R[3 + r] * T->t[1] + T->R[6 + r] * T->t[2]);
  int64_t measured = 0;
  for (int v = 0; v < H; ++v) {
    for (int u = 0; u < W; ++u) {
      const size_t i = (size_t)v * W + u;
      int st = MVS_FLAT, bk = -1;
      double mg = INFINITY;
      double edge = INFINITY;
      do {
        if (u < 1 || u > W - 2 || v < 1 || v > H - 2) break;
        const double gx = 0.5 * ((double)img_key[i + 1] - img_key[i - 1]);
        const double gy = 0.5 * ((double)img_key[i + W] - img_key[i - W]);
        const double g = sqrt(gx * gx + gy * gy);
        mg = dmin(mg, fabs(g - prm->grad_min) / (prm->grad_min > 0.0 ? prm->grad_min : 1.0));
        if (g < prm->grad_min) break;
        /* search interval */
        const double dp = depth[i], vp = var[i];
        const int has = dp > 0.0 && isfinite(dp) && vp > 0.0 && isfinite(vp);
        double lo = prm->d_min, hi = prm->d_max;
        if (has) {
          const double sp = sqrt(vp);
          lo = dp - prm->sigma_range * sp;
          hi = dp + prm->sigma_range * sp;
          if (lo < prm->d_min) lo = prm->d_min;
          if (hi > prm->d_max) hi = prm->d_max;
        }
        st = MVS_INTERVAL;
        if (!(lo < hi)) break;
        st = MVS_LINE;
        double P0[2], P1[2];
        if (!project(cam, T, u, v, lo, &P0[0], &P0[1]) || !project(cam, T, u, v, hi, &P1[0], &P1[1]))
          break;
        const double dx = P1[0] - P0[0], dy = P1[1] - P0[1];
        const double L = sqrt(dx * dx + dy * dy);
        if (!(L > 0.0)) break;
        const double fl = floor(L);
        mg = dmin(mg, dmin(L - fl, fl + 1.0 - L));
        const int n = (int)fl + 1;
        if (n > prm->max_steps) break;
        const double dir[2] = {dx / L, dy / L};
        const int use_x = fabs(dir[0]) >= fabs(dir[1]);  /* either row gives d; the larger is better conditioned */
        /* the keyframe's epipolar direction at (u, v): x - epipole, scaled by C_z */
        double e0[2] = {C[2] * (u - cam->cx) - cam->fx * C[0], C[2] * (v - cam->cy) - cam->fy * C[1]};
        const double ne = sqrt(e0[0] * e0[0] + e0[1] * e0[1]);
        if (!(ne > 0.0)) break;
        e0[0] /= ne;
        e0[1] /= ne;
        double key[5];
        int inside = 1;
        for (int s = -2; s <= 2 && inside; ++s)
          inside = bilinear(img_key, W, H, u + s * e0[0], v + s * e0[1], &key[s + 2], &edge);
        if (!inside) break;
        const double r[3] = {(u - cam->cx) / cam->fx, (v - cam->cy) / cam->fy, 1.0};
        double a[3];
        for (int k = 0; k < 3; ++k) a[k] = T->R[3 * k] * r[0] + T->R[3 * k + 1] * r[1] + T->R[3 * k + 2] * r[2];
        /* the walk: best step over j = 0 .. n-1 (first minimum) */
        int best = -1;
        double b1 = INFINITY, b2 = INFINITY;
        for (int j = 0; j < n; ++j) {
          double e[5], ssd, dj;
          if (!step_error(img_ref, W, H, cam, T, u, v, e0, key, a, use_x, P0, dir, j, e, &ssd, &dj, &edge))
            continue;
          if (ssd < b1) {
            b2 = b1;
            b1 = ssd;
            best = j;
          } else if (ssd < b2) {
            b2 = ssd;
          }
        }
        st = MVS_NOSTEP;
        if (best < 0) break;
        bk = best;
        if (isfinite(b2)) mg = dmin(mg, (b2 - b1) / (b1 > 1.0 ? b1 : 1.0));
        mg = dmin(mg, fabs(b1 - prm->ssd_max) / (prm->ssd_max > 1.0 ? prm->ssd_max : 1.0));
        st = MVS_SSD;
        if (b1 > prm->ssd_max) break;
        /* sub-pixel fit between the best step and its better neighbour */
        double ea[5], da, sa, em[5], dm, sm, ep[5], dq, sq;
        step_error(img_ref, W, H, cam, T, u, v, e0, key, a, use_x, P0, dir, best, ea, &sa, &da, &edge);
        const int okm = step_error(img_ref, W, H, cam, T, u, v, e0, key, a, use_x, P0, dir, best - 1, em, &sm, &dm, &edge);
        const int okp = step_error(img_ref, W, H, cam, T, u, v, e0, key, a, use_x, P0, dir, best + 1, ep, &sq, &dq, &edge);
        st = MVS_NEIGHBOUR;
        if (!okm && !okp) break;
        if (okm && okp) mg = dmin(mg, fabs(sm - sq) / dmin(sm > 1.0 ? sm : 1.0, sq > 1.0 ? sq : 1.0));
        const int take_m = okm && (!okp || sm <= sq);
        const double *eb = take_m ? em : ep;
        const double db = take_m ? dm : dq;
        double de[5], D2 = 0.0, ade = 0.0;
        for (int s = 0; s < 5; ++s) {
          de[s] = eb[s] - ea[s];
          D2 += de[s] * de[s];
          ade += ea[s] * de[s];
        }
        if (!(D2 > 0.0)) break;
#if ORC_MUTANT == 12
        double sstar = ade / D2;
#else
        double sstar = -ade / D2;
#endif
        if (sstar < 0.0) sstar = 0.0;
        if (sstar > 1.0) sstar = 1.0;
        const double dd = db - da;
        const double d_obs = da + sstar * dd;
#if ORC_MUTANT == 11
        const double v_obs = prm->photo_var * fabs(dd) / D2;
#else
        const double v_obs = prm->photo_var * dd * dd / D2;
#endif
        if (!(v_obs > 0.0) || !isfinite(v_obs)) break;
        if (has) {
          depth[i] = (dp * v_obs + d_obs * vp) / (vp + v_obs);
          var[i] = vp * v_obs / (vp + v_obs);
        } else {
          depth[i] = d_obs;
          var[i] = v_obs;
        }
        st = MVS_OK;
        ++measured;
      } while (0);
      if (st != MVS_FLAT || isfinite(edge)) mg = dmin(mg, edge);
      if (status) status[i] = st;
      if (best_step) best_step[i] = bk;
      if (margin) margin[i] = mg;
    }
  }
  return measured;
}
