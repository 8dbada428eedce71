/*
 * deepfusion.h -- C ABI of the GB300 (sm_103a) keyframe depth optimiser.
 *
 * The library solves, for each new frame, the fused keyframe log-depth
 * problem of DeepFusion (Laidlow, Czarnowski, Leutenegger; Section II-C,
 * "Optimisation"):
 *
 *   c(d, s) = c_semi(d, s) + c_net(d) + c_grad(d)                  (Eq. 5)
 *
 * over the per-pixel log-depth x_i = ln d_i and the log scale correction
 * t = ln s, with the semi-dense unary term (Eq. 6), the network unary term
 * (Eq. 7) and the network log-depth-gradient pairwise term (Eq. 8), each
 * whitened by its variance and robustified by the Huber loss, by Gauss-Newton
 * iterations that alternate between the scale and the depth (10 in the
 * paper). The depth half solves the 5-point normal equations by
 * Jacobi-preconditioned conjugate gradients.
 *
 * Conventions for every entry point:
 *   - Images are H x W, row-major, dense (row stride = width elements);
 *     pixel i = v * W + u (column u, row v), as in Eq. 8.
 *   - 'ptrs_on_device' != 0: the buffers are device pointers on the current
 *     CUDA device; otherwise host pointers (pinned memory gives asynchronous
 *     copies, pageable memory is copied synchronously by the driver).
 *   - 'stream' is a cudaStream_t (NULL = the legacy default stream). All work
 *     is stream-ordered: the caller keeps ownership of its buffers and must
 *     not modify or free them until the stream has passed the call.
 *   - Every call returns a df_status; none aborts the process. On error the
 *     keyframe is left as it was before the call and df_last_error() gives a
 *     thread-local message.
 *   - The library owns each keyframe's device memory (allocated at create,
 *     released at destroy) and counts it against a process-wide budget.
 */
#ifndef DEEPFUSION_H
#define DEEPFUSION_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DF_OK = 0,
  DF_EINVAL = 1,    /* bad argument or invalid input values */
  DF_ENOMEM = 2,    /* device allocation failed */
  DF_EBUDGET = 3,   /* the memory budget would be exceeded */
  DF_ECUDA = 4,     /* a CUDA runtime call failed */
  DF_ETIMEOUT = 5,  /* a device-side wait gave up (the solve was abandoned) */
  DF_ESTATE = 6,    /* the keyframe is in an unusable state */
  DF_ENOTSUP = 7    /* not supported on this device / build */
} df_status;

/* Storage type of the six network planes (Section II-A outputs). */
typedef enum { DF_F32 = 0, DF_BF16 = 1, DF_F16 = 2 } df_dtype;

/* Cost terms (Eq. 5). Leaving some out gives the ablations of Tables II
 * (semi + gradient, scale fitted afterwards) and III (no pairwise term). */
enum { DF_TERM_SEMI = 1, DF_TERM_NET = 2, DF_TERM_GRAD = 4, DF_TERMS_ALL = 7 };

/* Robust loss on every term: Huber (Section II-C) or Tukey's biweight
 * (named as an alternative in Section IV). */
enum { DF_LOSS_HUBER = 0, DF_LOSS_TUKEY = 1 };

/* Which kernel schedule runs the solve. AUTO picks the fused persistent
 * kernel when it fits, else the per-phase launches. */
enum { DF_SOLVER_AUTO = 0, DF_SOLVER_LAUNCHES = 1, DF_SOLVER_FUSED = 2 };

typedef struct {
  int32_t width;      /* W >= 1 */
  int32_t height;     /* H >= 1 */
  int32_t cnn_dtype;  /* df_dtype of the six network planes */
} df_keyframe_desc;

/* df_solve_params.scale_step: how the log scale t = ln s is solved.
 *  DF_SCALE_FIXED     t is kept (Table II's scale-ambiguous solve);
 *  DF_SCALE_ALTERNATE each GN iteration first solves t with x fixed, then
 *                     x with t fixed (Section II-C, last paragraph: the
 *                     paper's alternation);
 *  DF_SCALE_JOINT     each GN iteration runs Jacobi-PCG on the bordered
 *                     normal equations in (x, t)
 *                       [A, -ws; -ws^T, sum ws] [x; t] = [b - ws t; -ws.mu_s]
 *                     (A, b: the depth step's 5-point system; ws: the
 *                     semi-dense weights), preconditioned by diag(A) and
 *                     sum ws. Not in the paper: a solver variant that needs
 *                     no alternation. Runs on the launch solver and, with a
 *                     fixed iteration count (tol = 0), on the fused solver:
 *                     the shared-memory resident kernel, or the streaming
 *                     kernel with 4 pixels per lane and n_pcg >= 1; other
 *                     launch shapes make DF_SOLVER_AUTO take the launch
 *                     solver and DF_SOLVER_FUSED return DF_ENOTSUP. Batches
 *                     are solved keyframe by keyframe. */
#define DF_SCALE_FIXED 0
#define DF_SCALE_ALTERNATE 1
#define DF_SCALE_JOINT 2

typedef struct {
  int32_t n_gn;       /* Gauss-Newton iterations; 10 in Section II-C */
  int32_t n_pcg;      /* PCG iterations per depth step (>= 0) */
  float delta;        /* robust threshold on whitened residuals;
                         <= 0 or +inf gives plain least squares */
  int32_t loss;       /* DF_LOSS_* */
  int32_t terms;      /* DF_TERM_* bits; must include NET or GRAD */
  int32_t scale_step; /* DF_SCALE_*: how t is solved (see below) */
  int32_t solver;     /* DF_SOLVER_* */
  double tol;         /* > 0: end a depth step once ||r|| < tol ||b||;
                         0: fixed iteration count */
  int32_t warm_gn;    /* the first warm_gn GN iterations use the Huber loss
                         with threshold warm_delta, the remaining ones 'loss'
                         with 'delta': Tukey's biweight (Section IV) is not
                         convex, so it is started from Huber iterations;
                         0: every iteration uses 'loss' */
  float warm_delta;   /* Huber threshold of the warm iterations (<= 0 or +inf:
                         least squares) */
} df_solve_params;

typedef struct {
  double scale_log;    /* t = ln s after the solve */
  double res_norm;     /* ||r|| of the last depth step's PCG residual */
  int32_t iters_done;  /* PCG iterations executed, summed over GN iterations */
  int32_t flags;       /* device-side status bits (0 = clean) */
} df_solve_report;

typedef struct df_keyframe df_keyframe; /* opaque; owns its device memory */

/* Fill 'p' with the paper's schedule: n_gn = 10 (Section II-C), n_pcg = 3,
 * Huber with delta = 1.345, all terms, scale step on, AUTO solver, tol = 0,
 * no warm start (warm_gn = 0, warm_delta = 1.345). */
void df_default_params(df_solve_params *p);

/* Create a keyframe from the network's per-keyframe outputs (Section II:
 * the CNN runs once per keyframe; Section II-A lists its outputs):
 *   mu_net  = ln d_net (Eq. 7b),  var_net = R_net (Eq. 7a),
 *   gx, var_gx = x-gradient of the log-depth and its variance (Eq. 8b),
 *   gy, var_gy = y-gradient and its variance (Eq. 8c).
 * Each is H x W of desc->cnn_dtype. gx in column W-1 and gy in row H-1 are
 * ignored (those pairwise terms have no partner pixel). The state starts at
 * x = mu_net, t = 0; there is no semi-dense term until df_frame_update.
 * Variances must be finite and > 0 and means finite: with host pointers a
 * violation returns DF_EINVAL and allocates nothing; with device pointers it
 * is detected on the device, the keyframe is marked invalid (solves leave it
 * unchanged) and df_keyframe_check() returns DF_EINVAL.
 * Errors: DF_EINVAL (null/size/dtype), DF_EBUDGET, DF_ENOMEM, DF_ECUDA. */
df_status df_keyframe_create(const df_keyframe_desc *desc, const void *mu_net,
                             const void *var_net, const void *gx, const void *var_gx,
                             const void *gy, const void *var_gy, int ptrs_on_device,
                             void *stream, df_keyframe **out);

/* Re-initialise an existing keyframe with new network outputs (same size and
 * dtype): as df_keyframe_create, without allocating. */
df_status df_keyframe_reset(df_keyframe *kf, const void *mu_net, const void *var_net,
                            const void *gx, const void *var_gx, const void *gy,
                            const void *var_gy, int ptrs_on_device, void *stream);

/* Replace the semi-dense measurements of the current frame (Sections II and
 * II-B: updated with every new frame, already in log space):
 *   mu_semi = ln d_semi (Eq. 6b), var_semi = R_semi (Eq. 6a), both H x W f32.
 * A pixel without a measurement has var_semi <= 0 or a non-finite value.
 * Ordered on 'stream' like every call; the buffers are read before the
 * stream passes the call. Host buffers (ptrs_on_device = 0) are uploaded on
 * the keyframe's own copy stream into a staging pair of the keyframe, so
 * that the upload overlaps the work 'stream' runs before the call (the
 * previous frame's solve); 'stream' then waits for it and moves the planes
 * into place. Host buffers must therefore hold the frame's data when the
 * call is made (as host planes must for df_keyframe_create / _reset, which
 * check them on the host): a copy into them still pending on a stream is
 * not waited for. Under stream capture the upload goes on 'stream' itself.
 * Errors: DF_EINVAL (null kf/pointers), DF_ECUDA. */
df_status df_frame_update(df_keyframe *kf, const float *mu_semi, const float *var_semi,
                          int ptrs_on_device, void *stream);

/* Run one frame's solve (Section II-C): params->n_gn iterations of
 * { scale step; re-weighting; n_pcg Jacobi-PCG iterations on the depth },
 * warm-started from the keyframe's current (x, t). 'params' NULL = defaults.
 * 'report' NULL: fully asynchronous. Otherwise the call synchronises the
 * stream and fills the report.
 * Errors: DF_EINVAL (params out of range), DF_ESTATE (invalid keyframe),
 * DF_ETIMEOUT (fused solver's device-side wait gave up), DF_ECUDA. */
df_status df_optimise(df_keyframe *kf, const df_solve_params *params, void *stream,
                      df_solve_report *report);

/* Solve n keyframes of possibly different sizes together (one fused launch
 * per group that fits the device). Each keyframe's result is the one
 * df_optimise would give it alone. 'reports' may be NULL or hold n entries
 * (then the call synchronises). Errors as df_optimise. */
df_status df_optimise_batch(df_keyframe *const *kfs, int32_t n,
                            const df_solve_params *params, void *stream,
                            df_solve_report *reports);

/* Prepare a keyframe list for repeated batched solves and for capture in a
 * CUDA graph: builds the fused solver's launch plans for exactly this list
 * (in this order) and the current tuning, and keeps them on the device
 * (synchronises 'stream'). df_optimise_batch on the same list then uses
 * them with no host work or allocation; a batched solve under stream capture
 * requires them (DF_ENOTSUP otherwise). Plans live until df_batch_release
 * names one of their keyframes or one of them is destroyed; graphs that
 * captured a solve must not be replayed after that. Lists of one keyframe
 * need nothing (each keyframe keeps its own plan). Not in the paper: launch
 * management. Errors: DF_EINVAL (NULL / repeated / cross-device keyframes),
 * DF_ENOTSUP (no fused solver on this device). */
df_status df_batch_prepare(df_keyframe *const *kfs, int32_t n, void *stream);
df_status df_batch_release(df_keyframe *const *kfs, int32_t n);

/* The per-frame bookkeeping of many keyframes at once, in one or two device
 * passes per 24 keyframes instead of one copy or launch per plane and
 * keyframe (paper counterpart: none; the same work as the single-keyframe
 * calls it names). kfs: n distinct keyframes on one device (DF_EINVAL
 * otherwise, before anything runs). Stream-ordered; the caller keeps its
 * buffers and must not modify them until the stream has passed the call.
 * With device pointers nothing is uploaded and the calls can be captured in
 * a CUDA graph. Host pointers into page-locked (pinned) memory are treated
 * like device pointers: the kernels read and write them directly over the
 * host link (so the reset's input check runs on the device and flags a
 * keyframe rather than returning DF_EINVAL). Other host pointers go through
 * the single-keyframe calls.
 *
 * df_keyframe_reset_batch: df_keyframe_reset of keyframe j from
 *   planes[6j .. 6j+5] = mu_net, var_net, gx, var_gx, gy, var_gy (each
 *   dense row-major in keyframe j's cnn_dtype): the planes are copied in,
 *   x = mu_n and t = 0 (Section II: a keyframe starts from the network's
 *   prediction), the semi-dense variance is cleared, and the inputs are
 *   checked (pageable host pointers: all before any keyframe is touched,
 *   DF_EINVAL; device and pinned host pointers: on the device, flagging the
 *   keyframe as df_keyframe_reset does with device pointers).
 * df_frame_update_batch: df_frame_update of keyframe j from mu_semi[j],
 *   var_semi[j] (dense f32, log space, Section II-B).
 * df_fetch_depth_batch: df_fetch_depth of keyframe j into out[j] (dense f32:
 *   d = exp(x), or x when log_space). */
df_status df_keyframe_reset_batch(df_keyframe *const *kfs, int32_t n, const void *const *planes,
                                  int ptrs_on_device, void *stream);
df_status df_frame_update_batch(df_keyframe *const *kfs, int32_t n, const float *const *mu_semi,
                                const float *const *var_semi, int ptrs_on_device, void *stream);
df_status df_fetch_depth_batch(df_keyframe *const *kfs, int32_t n, float *const *out,
                               int log_space, int ptrs_on_device, void *stream);

/* Write the keyframe's depth map d = exp(x) (Eq. 5's d; log_space != 0
 * writes x = ln d instead) as H x W f32 into 'out'. */
df_status df_fetch_depth(df_keyframe *kf, float *out, int log_space, int ptr_on_device,
                         void *stream);

/* Read / overwrite the solver state (log-depth x as H x W f32, log scale t).
 * Used to checkpoint and resume a keyframe and to start a solve from a
 * chosen point. 't_out' is written when the stream reaches the call (host
 * pointer: the call synchronises). */
df_status df_keyframe_get_state(df_keyframe *kf, float *x_out, double *t_out,
                                int ptrs_on_device, void *stream);
df_status df_keyframe_set_state(df_keyframe *kf, const float *x, double t,
                                int ptrs_on_device, void *stream);

/* Evaluate the robust cost c(x, t) of Eq. 5 at the current state with the
 * given terms/loss/delta (FP64 reduction). Synchronises the stream. */
df_status df_cost(df_keyframe *kf, const df_solve_params *params, void *stream,
                  double *cost_out);

/* The scale estimate of the ablation of Table II (Section III-C, "Scale
 * Optimisation Evaluation"): after a scale-ambiguous solve (terms =
 * SEMI | GRAD, scale_step = 0), fit the scale to the network prediction by
 * least squares in log space: c = mean(mu_n - x), then x += c and t += c
 * (the semi-dense residuals x - t - mu_s are unchanged). Asynchronous. */
df_status df_scale_fit_ls(df_keyframe *kf, void *stream);

/* Accuracy metric of Section III-B (the measure of Tables I-III): counts
 * the pixels whose estimated depth d = exp(x) lies within rel_tol of the
 * ground truth, |d - d_true| <= rel_tol * d_true (rel_tol = 0.1 in the
 * paper), among the pixels with a finite d_true > 0 (*n_valid); the paper's
 * percentage is 100 * n_within / n_valid. depth_true: dense row-major H x W
 * FP32 metric depth, host or device (ptr_on_device), caller-owned, read
 * before return. The within decision is taken in FP64. Synchronous.
 * Errors: DF_EINVAL for NULL pointers or a negative / non-finite rel_tol. */
df_status df_depth_accuracy(df_keyframe *kf, const float *depth_true, int ptr_on_device,
                            double rel_tol, void *stream, int64_t *n_within, int64_t *n_valid);

/* Synchronise 'stream' and return DF_EINVAL if device-side input checks
 * flagged the keyframe, DF_ETIMEOUT if a fused solve gave up, else DF_OK. */
df_status df_keyframe_check(df_keyframe *kf, void *stream);

/* Size / dtype of a keyframe and the device bytes it holds. */
df_status df_keyframe_info(const df_keyframe *kf, df_keyframe_desc *desc,
                           size_t *device_bytes);

/* Release a keyframe (NULL-safe). Waits for the keyframe's pending work. */
void df_keyframe_destroy(df_keyframe *kf);

/* Device bytes a keyframe of this size and dtype will hold (for admission). */
size_t df_keyframe_bytes(int32_t width, int32_t height, int32_t cnn_dtype);

/* Process-wide device-memory budget for keyframes (0 = unlimited) and the
 * bytes currently held. */
df_status df_set_memory_budget(size_t bytes);
size_t df_memory_in_use(void);

/* ---- semi-dense two-view depth (Section II-B) -----------------------------
 *
 * The step that produces the optimisation's semi-dense input each frame:
 * for every keyframe pixel with enough texture, a search along its epipolar
 * line in a reference image for the depth that minimises the SSD of five
 * equally spaced points (Eq. 2), a sub-pixel fit between the best 1-pixel
 * step and its better neighbour, the measurement variance
 * sigma^2 = photo_var (J^T J)^-1 with J the finite-difference Jacobian of the
 * 5-vector error along the depth (Eqs. 3, 4), and the Gaussian fusion of the
 * measurement with the pixel's current estimate. Details the paper leaves
 * open are fixed as follows:
 *  - texture: central-difference gradient magnitude of the keyframe image
 *    >= grad_min (the image border is never measured);
 *  - search interval: [d - sigma_range sigma, d + sigma_range sigma] with a
 *    current estimate (sigma_range = 2 in the paper), else [d_min, d_max],
 *    clipped to [d_min, d_max]; the projections of its ends span a segment of
 *    length L in the reference image, walked in floor(L) + 1 steps of 1 px
 *    from the near end (segments of more than max_steps steps are skipped);
 *  - samples: keyframe points x + s e0 (s = -2..2, e0 the unit direction of
 *    the keyframe's epipolar line at x), each compared with its projection
 *    into the reference image at the step's depth; bilinear interpolation;
 *    a step with any sample outside the image is invalid;
 *  - the first minimum wins; the neighbour is the step before or after the
 *    best one (evaluated even just beyond the interval) with the smaller SSD,
 *    the one before on ties; the error is linearised between the two and
 *    minimised over the segment between them;
 *  - no measurement when the best SSD exceeds ssd_max. */
typedef struct {
  float fx, fy, cx, cy; /* pinhole intrinsics, pixels (both images) */
} df_camera;

typedef struct {
  float R[9]; /* row-major rotation, keyframe camera -> reference camera */
  float t[3]; /* X_ref = R X_key + t (metres) */
} df_pose;

typedef struct {
  float grad_min;    /* texture threshold, intensity units per pixel (default 20) */
  float d_min, d_max;/* search range without an estimate (default 0.3, 10 m) */
  float sigma_range; /* half-width of the interval in sigmas (default 2) */
  float ssd_max;     /* largest accepted best SSD (default 5 * 20^2) */
  float photo_var;   /* image noise variance in sigma^2 (default 1) */
  int32_t max_steps; /* longest walk, steps (default 512) */
} df_mvs_params;

/* per-pixel outcome codes of df_mvs_update's status plane */
#define DF_MVS_OK 0        /* measured and fused */
#define DF_MVS_FLAT 1      /* border pixel or too little texture */
#define DF_MVS_INTERVAL 2  /* empty search interval */
#define DF_MVS_LINE 3      /* degenerate / too long segment, keyframe samples outside */
#define DF_MVS_NOSTEP 4    /* no step with all samples inside the reference image */
#define DF_MVS_SSD 5       /* best SSD above ssd_max */
#define DF_MVS_NEIGHBOUR 6 /* no usable neighbour for the sub-pixel fit */

typedef struct df_mvs df_mvs;

void df_mvs_default_params(df_mvs_params *p);

/* Work space for images of width x height (a device list of candidate
 * pixels and a counter), on the current device. */
df_status df_mvs_create(int32_t width, int32_t height, df_mvs **out);
void df_mvs_destroy(df_mvs *m); /* NULL-safe */

/* One stereo update of a keyframe's semi-dense estimate, asynchronous on
 * 'stream'. img_key, img_ref: dense row-major H x W FP32 intensities on the
 * device. depth, var: dense H x W FP32 device planes holding the current
 * estimate (metres, metres^2; var <= 0 or non-finite: no estimate), updated
 * in place where a measurement is made. status, best_step: optional dense
 * H x W int32 device planes (NULL to skip) receiving DF_MVS_* and the best
 * step index (-1 when there was none). All buffers are caller-owned and
 * must not be written until the stream has passed the call. The result goes
 * to log space with df_semi_to_log and into the solve with df_frame_update.
 * Errors: DF_EINVAL for NULL required pointers, a size other than the
 * context's, or invalid parameters (d_min <= 0, d_max <= d_min, max_steps <
 * 1, negative thresholds). */
df_status df_mvs_update(df_mvs *m, const float *img_key, const float *img_ref,
                        const df_camera *cam, const df_pose *key_to_ref,
                        const df_mvs_params *params, float *depth, float *var,
                        int32_t *status, int32_t *best_step, void *stream);

/* Epipolar steps the last df_mvs_update evaluated (each walked step plus
 * the three steps recomputed for the sub-pixel fit, summed over pixels):
 * the work count of the update. Synchronises 'stream'. */
df_status df_mvs_last_steps(df_mvs *m, void *stream, uint64_t *steps);

/* Section II-B, last sentence: semi-dense depth d and its variance
 * sigma_d^2 to log space, to first order: mu = ln d, var = sigma_d^2 / d^2.
 * Invalid inputs (d <= 0, variance <= 0, non-finite) give mu = 0, var = 0.
 * n elements; all four arrays on the same side (device or host). */
df_status df_semi_to_log(const float *depth, const float *var_depth, float *mu_semi,
                         float *var_semi, int64_t n, int ptrs_on_device, void *stream);

/* ---- serving: many camera streams, continuous batching --------------------
 *
 * A server keeps one keyframe per camera stream resident on the device
 * (Section II: the keyframe is re-optimised with every new frame) and
 * solves the frame updates that callers submit. Streams are admitted
 * against the memory budget; submitted frames queue per stream; every
 * df_server_progress call retires the batches that have finished and, in
 * batching mode, launches ONE batched solve (df_optimise_batch) over every
 * stream that has a frame waiting and is not already on the GPU. Batches run
 * on a pool of CUDA streams, so frames that arrive while others are being
 * solved are admitted at the next call and overlap on the device. With
 * batching = 0 every frame is solved by its own df_optimise launch in
 * arrival order (the plain baseline). In batching mode each launch slot
 * owns a device and a pinned host buffer for a batched launch's plan (room
 * for max_batch keyframes), made by df_server_create, and a tick's frame
 * updates go through df_frame_update_batch when all are device buffers, so
 * a tick allocates nothing. Not thread-safe: one host thread drives a
 * server. Paper counterpart: none (a serving layer of this library). */
typedef struct df_server df_server;

typedef struct {
  size_t memory_budget;   /* device bytes for the streams' keyframes; 0 = unlimited */
  int32_t max_batch;      /* keyframes per batched launch, 1..256 */
  int32_t max_inflight;   /* launches in flight at once (CUDA streams), 1..16 */
  int32_t batching;       /* 1: continuous batching; 0: one launch per frame */
  int32_t pad;
  df_solve_params params; /* solve of every frame */
} df_server_config;

/* One finished frame update. Times are host steady-clock nanoseconds. */
typedef struct {
  uint64_t tag;          /* the caller's tag from df_server_submit */
  int32_t stream_id;
  int32_t status;        /* df_status of the solve */
  int64_t t_submit_ns;   /* df_server_submit returned */
  int64_t t_launch_ns;   /* its batch was launched */
  int64_t t_done_ns;     /* its batch was seen finished */
  int32_t batch_size;    /* keyframes in its launch */
  int32_t pad;
} df_completion;

df_status df_server_create(const df_server_config *cfg, df_server **out);
/* Waits for all work, releases every stream. NULL-safe. */
void df_server_destroy(df_server *srv);
/* Admit a camera stream: create its keyframe from the network planes as
 * df_keyframe_create does. DF_EBUDGET when the budget cannot hold it. */
df_status df_server_open_stream(df_server *srv, const df_keyframe_desc *desc,
                                const void *mu_net, const void *var_net, const void *gx,
                                const void *var_gx, const void *gy, const void *var_gy,
                                int ptrs_on_device, int32_t *stream_id);
/* Release a stream (waits for its pending work); its memory returns to the
 * budget. */
df_status df_server_close_stream(df_server *srv, int32_t stream_id);
/* Queue a frame update (semi-dense log-depth / variance, H x W f32, as
 * df_frame_update). The buffers must stay valid and unchanged until the
 * frame's completion has been returned. */
df_status df_server_submit(df_server *srv, int32_t stream_id, const float *mu_semi,
                           const float *var_semi, int ptrs_on_device, uint64_t tag);
/* Non-blocking scheduler step: retire finished launches, start new ones,
 * write up to 'cap' completions to 'out' and their number to *n_out. */
df_status df_server_progress(df_server *srv, df_completion *out, int32_t cap, int32_t *n_out);
/* Frames submitted but not yet returned by df_server_progress. */
int32_t df_server_pending(const df_server *srv);
/* The stream's current depth (as df_fetch_depth; synchronises). */
df_status df_server_fetch_depth(df_server *srv, int32_t stream_id, float *out, int log_space,
                                int ptr_on_device);
/* The stream's current state (as df_keyframe_get_state: the log-depth x,
 * H x W f32, and the log scale t of Eq. 5, either may be NULL; waits for
 * the server's launches and synchronises). */
df_status df_server_get_state(df_server *srv, int32_t stream_id, float *x_out, double *t_out,
                              int ptrs_on_device);

/* Largest keyframe (in pixels) df_optimise_noalloc accepts: 196608, i.e.
 * 512 x 384, or four times the 256 x 192 resolution of Section II-A. */
#define DF_NOALLOC_MAX_PIXELS 196608

/* The per-frame solve of df_optimise for callers that cannot allocate device
 * memory. Some callers may not call cudaMalloc at all: a real-time loop whose
 * rules forbid allocation after start-up (an allocation can block on the
 * driver for milliseconds), a plugin inside a host program whose device
 * memory is owned by that program's own allocator (which may hold nearly all
 * of it), or a process that runs under a fixed device-memory quota. The
 * paper has no counterpart; this is an interface of this library.
 *
 * Arguments: H x W = height x width (at most DF_NOALLOC_MAX_PIXELS pixels),
 * dense row-major f32 DEVICE buffers owned by the caller: the six network
 * planes as in df_keyframe_create, the semi-dense planes as in
 * df_frame_update (both NULL = no semi-dense term), the log-depth x (read as
 * the warm start, overwritten with the result) and the log scale t (one
 * device double, read and overwritten). params: as df_optimise (NULL =
 * defaults; the solver field is ignored: this always runs the per-phase
 * launch schedule). Inputs are not checked on the device.
 *
 * It allocates nothing: its working memory (the solver vectors, FP64 partial
 * sums and scalars) is one static device array of the library of 5,701,824
 * bytes (5.70 MB, 5.44 MiB) that every GPU which loads the library holds
 * until the process exits. All calls on a device share that array and it
 * keeps the last call's contents (the scalars are cleared at the start of
 * each call), so calls whose work overlaps on the GPU (other streams, other
 * host threads) race with each other: serialise them. The first call on
 * each device looks the array's device address up (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream
 * capture. Asynchronous on 'stream'.
 * Errors: DF_EINVAL (sizes above the limit, NULL pointers, parameters),
 * DF_ENOTSUP (the joint (x, t) variant with the semi-dense term, whose extra
 * scratch plane the array does not hold; without the semi-dense term the
 * joint variant leaves t in place and runs as the depth step with t fixed;
 * a device index beyond 63), DF_ECUDA. */
df_status df_optimise_noalloc(int32_t width, int32_t height, const float *mu_net,
                              const float *var_net, const float *gx, const float *var_gx,
                              const float *gy, const float *var_gy, const float *mu_semi,
                              const float *var_semi, float *x_inout, double *scale_log_inout,
                              const df_solve_params *params, void *stream);

/* Launch shape of the fused solver (process-wide; paper counterpart: none,
 * this is how the GB300 kernels are cut). A field of 0 means "choose from
 * the problem size". Keyframes pick up a new setting at their next solve.
 *   mode      0 auto (resident when the state fits in shared memory,
 *             else streaming), 1 streaming only, 2 resident only
 *   vec       streaming kernel: pixels per lane along a row, 1 or 4
 *   tile_rows streaming kernel: rows per warp tile (1..64)
 *   max_ctas  cap on the cooperative grid
 *   gn_per_launch  Gauss-Newton iterations per fused launch (0 = all of
 *             them in one launch); the solve is split into launches of
 *             whole GN iterations with the same result
 *   debug_skip_cta  test only: >= 0 makes that CTA of the next fused launches
 *             leave without adding its sums of the first pass (and, in
 *             the resident kernel, without raising its edge flag after
 *             the assembly), so the others' bounded waits run out
 *             (DF_ETIMEOUT); -1 = off.
 *   assembly  streaming kernel with 4 pixels per lane: where each GN
 *             iteration's weights and 5-point system are assembled.
 *             1 in a pass of the persistent kernel, 2 in an ordinary kernel
 *             of its own between two persistent launches (many warps per SM
 *             instead of 8; same arithmetic, the reductions summed per
 *             piece), 0 auto: 2 when each warp of the persistent kernel
 *             walks 56 rows or more (large batches), else 1. */
typedef struct {
  int32_t mode;
  int32_t vec;
  int32_t tile_rows;
  int32_t max_ctas;
  int32_t gn_per_launch;
  int32_t debug_skip_cta;
  int32_t assembly;
} df_tuning;

df_status df_set_tuning(const df_tuning *t); /* NULL restores the defaults */
df_status df_get_tuning(df_tuning *t);

/* Autotuner (paper counterpart: none): time the fused solver's candidate
 * launch shapes -- the resident kernel with all GN iterations in one launch
 * or one per launch; the streaming kernel with 1 or 4 pixels per lane, each
 * warp walking its whole row share or pieces of 4..64 rows, and with 1 or 2
 * GN iterations per launch -- on these keyframes (solved together as by
 * df_optimise_batch, or alone when n = 1) with 'params'. Every trial starts
 * from the keyframes' current state, which is restored at the end. The
 * fastest shape becomes the current tuning (df_set_tuning) and is written to
 * *best, its time per solve (the median of five timed solves after an
 * untimed one) to *best_ms. Synchronises; allocates a snapshot of the
 * keyframes' log-depth for the duration of the call.
 * Errors: DF_EINVAL for a NULL or repeated keyframe in the list (checked
 * before anything is allocated or changed); a failure while taking the
 * snapshot frees what was taken and leaves every keyframe and the tuning as
 * they were; DF_ENOTSUP when no shape can solve the list (the states are
 * restored and the tuning is left as it was). */
df_status df_autotune(df_keyframe *const *kfs, int32_t n, const df_solve_params *params,
                      void *stream, df_tuning *best, float *best_ms);

/* Upper bound on every device-side wait of the fused solver (the polls of
 * each keyframe's sum words and of the neighbouring bands' edge flags, the
 * waits on staged rows), in nanoseconds; a wait that runs out abandons the
 * solve and is reported as DF_ETIMEOUT. Default 2 s. */
df_status df_set_spin_limit_ns(uint64_t ns);

/* Number of kernels this library has launched in this process (all devices);
 * a diagnostic for counting device work inside a timed region. */
uint64_t df_kernel_launches(void);

const char *df_status_str(df_status s);
const char *df_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DEEPFUSION_H */
