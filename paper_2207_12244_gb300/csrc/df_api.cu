// C ABI of the keyframe optimiser: keyframe state, memory budget, copies,
// input validation and the solve driver. Declarations and the contract of
// every entry point are in include/deepfusion.h.
#include <math.h>
#include <pthread.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "df_batch_io.cuh"
#include "df_fused.cuh"
#include "df_sync.cuh"
#include "df_internal.cuh"

using df::Planes;
using df::Scalars;
using df::SolveCfg;

struct df_keyframe {
  int device;
  int W, H, P, dtype;
  size_t bytes;
  void *mem;
  Planes planes;
  float *staging;   // dense H x W plane for host-side depth reads
  // host-pointer frame updates: dense H x W mu / var staging planes, filled
  // on the keyframe's own copy stream so that the upload of a frame overlaps
  // the solve of the previous one (stream and events made on first use)
  float *semi_stage;
  cudaStream_t copy_stream;
  cudaEvent_t ev_staged, ev_free;
  void *plan;       // resident launch plan of the fused solver (single keyframe)
  size_t plan_cap;  // bytes reserved for it
  df::LaunchShape plan_shape;    // shape of the plan currently on the device (kind -1: none)
  df::FusedTuning plan_tune;
};

namespace {

thread_local std::string g_err;
std::atomic<size_t> g_in_use{0};
std::atomic<size_t> g_budget{0};
std::atomic<uint64_t> g_launches{0};
std::atomic<unsigned long long> g_spin_limit_ns{2000000000ull};
std::mutex g_tune_mu;
df::FusedTuning g_tune;

df_status fail(df_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

df_status cuda_fail(cudaError_t e, const char *what) {
  return fail(DF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define DF_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int elem_size(int dtype) { return dtype == DF_F32 ? 4 : 2; }

int pitch_of(int W) { return (int)align_up((size_t)W, df::kPitchElems); }

// Byte layout of one keyframe allocation (offsets are 256-B aligned).
struct Layout {
  size_t cnn[6], mu_s, var_s, x, diag, wx, wy, v[df::kWorkPlanes], staging, semi_stage, sc,
      partial, plan, plan_cap, total;
};

Layout layout_of(int W, int H, int dtype) {
  Layout L;
  const size_t P = (size_t)pitch_of(W);
  const size_t cnn_plane = align_up(P * H * elem_size(dtype), 256);
  const size_t f32_plane = align_up(P * H * 4, 256);
  size_t off = 0;
  for (int j = 0; j < 6; ++j) { L.cnn[j] = off; off += cnn_plane; }
  L.mu_s = off; off += f32_plane;
  L.var_s = off; off += f32_plane;
  L.x = off; off += f32_plane;
  L.diag = off; off += f32_plane;
  L.wx = off; off += f32_plane;
  L.wy = off; off += f32_plane;
  for (int j = 0; j < df::kWorkPlanes; ++j) { L.v[j] = off; off += f32_plane; }
  L.staging = off; off += align_up((size_t)W * H * 4, 256);
  L.semi_stage = off; off += 2 * align_up((size_t)W * H * 4, 256);
  L.sc = off; off += align_up(sizeof(Scalars), 256);
  L.partial = off; off += align_up(sizeof(double) * df::kMaxPartialBlocks * df::kNumQ, 256);
  L.plan = off;
  L.plan_cap = df::fused_supported() ? align_up(df::fused_plan_cap_single(), 256) : 0;
  off += L.plan_cap;
  L.total = off;
  return L;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev) {
      prev = cur;
      cudaSetDevice(dev);
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

float half_bits_to_float(uint16_t h) {
  const uint32_t sign = (uint32_t)(h >> 15) << 31;
  const int exp = (h >> 10) & 0x1f;
  uint32_t mant = h & 0x3ff;
  uint32_t bits;
  if (exp == 0x1f) {
    bits = sign | 0x7f800000u | (mant << 13);
  } else if (exp == 0) {
    if (mant == 0) {
      bits = sign;
    } else {  // subnormal: renormalise
      int e = -1;
      do { ++e; mant <<= 1; } while ((mant & 0x400) == 0);
      bits = sign | ((uint32_t)(127 - 15 - e) << 23) | ((mant & 0x3ff) << 13);
    }
  } else {
    bits = sign | ((uint32_t)(exp - 15 + 127) << 23) | (mant << 13);
  }
  float f;
  memcpy(&f, &bits, 4);
  return f;
}

float host_elem(const void *p, size_t i, int dtype) {
  if (dtype == DF_F32) return static_cast<const float *>(p)[i];
  const uint16_t h = static_cast<const uint16_t *>(p)[i];
  if (dtype == DF_BF16) {
    const uint32_t bits = (uint32_t)h << 16;
    float f;
    memcpy(&f, &bits, 4);
    return f;
  }
  return half_bits_to_float(h);
}

// ---- host worker threads for checking large host inputs --------------------
//
// A batch reloads the network planes of every keyframe each frame (hundreds
// of MB). One host thread checks ~20 GB/s; the pool spreads a check over the
// host's cores without creating threads per call. Its threads are made once,
// detached, and wait on a condition variable; one job runs at a time, and
// every worker acknowledges each job before run() returns, so no worker
// touches a finished job. A process that forks gets no pool in the child
// (the threads are not copied): there, and while another thread's job runs,
// run() declines and the caller checks on its own thread.
std::atomic<bool> g_pool_forked{false};

class CheckPool {
 public:
  static CheckPool &get() {
    static CheckPool *pool = new CheckPool();  // never destroyed: its threads live until exit
    return *pool;
  }
  // f(0) .. f(parts - 1) on the pool's threads and the caller's; false (and
  // nothing run) if the pool is unavailable or busy.
  bool run(int parts, const std::function<void(int)> &f) {
    if (g_pool_forked.load() || nthreads_ == 0) return false;
    std::unique_lock<std::mutex> job(job_mu_, std::try_to_lock);
    if (!job.owns_lock()) return false;
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &f;
      parts_ = parts;
      acked_ = 0;
      next_.store(0);
      ++gen_;
    }
    wake_.notify_all();
    for (int p = next_.fetch_add(1); p < parts; p = next_.fetch_add(1)) f(p);
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return acked_ == nthreads_; });
    return true;
  }

 private:
  CheckPool() {
    pthread_atfork(nullptr, nullptr, [] { g_pool_forked.store(true); });
    const unsigned hc = std::thread::hardware_concurrency();
    const int n = (int)std::min(15u, hc > 1 ? hc - 1 : 0u);
    for (int i = 0; i < n; ++i) {
      try {
        std::thread(&CheckPool::worker, this).detach();
      } catch (...) {
        break;
      }
      ++nthreads_;
    }
  }
  void worker() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      wake_.wait(lk, [&] { return gen_ != seen; });
      seen = gen_;
      const std::function<void(int)> *fn = fn_;
      const int parts = parts_;
      lk.unlock();
      for (int p = next_.fetch_add(1); p < parts; p = next_.fetch_add(1)) (*fn)(p);
      lk.lock();
      if (++acked_ == nthreads_) done_.notify_one();
    }
  }
  std::mutex job_mu_, mu_;
  std::condition_variable wake_, done_;
  const std::function<void(int)> *fn_ = nullptr;
  int parts_ = 0, acked_ = 0, nthreads_ = 0;
  std::atomic<int> next_{0};
  uint64_t gen_ = 0;
};

// Validity of one network plane from the bit patterns of its elements:
// finite (any sign) for a mean, finite and > 0 for a variance. Integer tests
// over whole rows, so the loop is a plain streaming pass (the caller's planes
// are megabytes and this runs before every host-pointer keyframe load).
//   float: |bits| < 0x7f800000 is finite; 0 < bits < 0x7f800000 is finite > 0
//   bf16:  the same on the upper 16 bits (0x7f80)
//   fp16:  exponent field all ones (0x7c00) is Inf / NaN
template <class T>
bool plane_ok(const T *p, int W, int rows, int cols, bool is_var, uint32_t inf_bits) {
  constexpr uint32_t kSign = sizeof(T) == 4 ? 0x80000000u : 0x8000u;
  for (int v = 0; v < rows; ++v) {
    const T *row = p + (size_t)v * W;
    uint32_t bad = 0;
    if (is_var) {
      for (int u = 0; u < cols; ++u) bad |= (uint32_t)((uint32_t)row[u] - 1u >= inf_bits - 1u);
    } else {
      for (int u = 0; u < cols; ++u) bad |= (uint32_t)(((uint32_t)row[u] & ~kSign) >= inf_bits);
    }
    if (bad) return false;
  }
  return true;
}

// Host-side check of the network planes: means finite, variances finite > 0
// (gx / var_gx in the last column and gy / var_gy in the last row ignored).
// A fast pass over each plane's bits; only when it fails does the
// element-by-element walk below look for the first bad pixel (row, column,
// then plane order) to report.
bool host_inputs_ok(const void *const cnn[6], int W, int H, int dtype, char *why, size_t n) {
  // the fast pass: row blocks of every plane, split over host threads when
  // the planes are large (a batch of keyframes reloads hundreds of MB)
  std::atomic<bool> fast_ok{true};
  auto check_rows = [&](int part, int parts) {
    for (int j = 0; j < 6 && fast_ok.load(std::memory_order_relaxed); ++j) {
      const int cols = (j == 2 || j == 3) ? W - 1 : W, rows = (j == 4 || j == 5) ? H - 1 : H;
      const int r0 = (int)((long long)rows * part / parts);
      const int r1 = (int)((long long)rows * (part + 1) / parts);
      const bool is_var = (j & 1) == 1;
      bool ok;
      if (dtype == DF_F32)
        ok = plane_ok(static_cast<const uint32_t *>(cnn[j]) + (size_t)r0 * W, W, r1 - r0, cols,
                      is_var, 0x7f800000u);
      else
        ok = plane_ok(static_cast<const uint16_t *>(cnn[j]) + (size_t)r0 * W, W, r1 - r0, cols,
                      is_var, dtype == DF_BF16 ? 0x7f80u : 0x7c00u);
      if (!ok) fast_ok.store(false, std::memory_order_relaxed);
    }
  };
  // inputs of 1 M elements and more go to the pool in row blocks
  const long long elems = 6LL * W * H;
  const int parts = std::min(H, 64);
  bool done = false;
  if (elems >= (1LL << 20) && parts > 1) {
    const std::function<void(int)> job = [&](int part) { check_rows(part, parts); };
    done = CheckPool::get().run(parts, job);
  }
  if (!done) check_rows(0, 1);
  if (fast_ok.load()) return true;
  for (int v = 0; v < H; ++v) {
    for (int u = 0; u < W; ++u) {
      const size_t i = (size_t)v * W + u;
      for (int j = 0; j < 6; ++j) {
        if ((j == 2 || j == 3) && u == W - 1) continue;
        if ((j == 4 || j == 5) && v == H - 1) continue;
        const float a = host_elem(cnn[j], i, dtype);
        const bool is_var = (j & 1) == 1;
        if (!isfinite(a) || (is_var && !(a > 0.0f))) {
          static const char *names[6] = {"mu_net", "var_net", "gx", "var_gx", "gy", "var_gy"};
          snprintf(why, n, "%s at (u=%d, v=%d) is %g", names[j], u, v, (double)a);
          return false;
        }
      }
    }
  }
  return true;
}

// The six network planes into the keyframe's pitched planes, ordered on s.
// Host planes go up as whole contiguous copies into the dense staging plane
// (one f32 plane or two 16-bit planes at a time) and then into place by
// pitched device-to-device copies: a pitched copy straight from host memory
// moves one row per transfer and ran at ~24 GB/s on GB300, a contiguous one
// at ~160 GB/s.
df_status copy_cnn(df_keyframe *kf, const void *const cnn[6], int on_device, cudaStream_t s) {
  const size_t es = elem_size(kf->dtype);
  const size_t row = (size_t)kf->W * es, pitch = (size_t)kf->P * es;
  if (on_device) {
    for (int j = 0; j < 6; ++j)
      DF_CUDA(cudaMemcpy2DAsync(const_cast<void *>(kf->planes.cnn[j]), pitch, cnn[j], row, row,
                                kf->H, cudaMemcpyDefault, s));
    return DF_OK;
  }
  const size_t plane = row * kf->H;
  const int per = (int)(((size_t)kf->W * kf->H * 4) / plane);  // planes per staging round
  char *st = reinterpret_cast<char *>(kf->staging);
  for (int j = 0; j < 6; j += per) {
    for (int q = 0; q < per && j + q < 6; ++q)
      DF_CUDA(cudaMemcpyAsync(st + q * plane, cnn[j + q], plane, cudaMemcpyDefault, s));
    for (int q = 0; q < per && j + q < 6; ++q)
      DF_CUDA(cudaMemcpy2DAsync(const_cast<void *>(kf->planes.cnn[j + q]), pitch, st + q * plane,
                                row, row, kf->H, cudaMemcpyDeviceToDevice, s));
  }
  return DF_OK;
}

df_status load_cnn(df_keyframe *kf, const void *const cnn[6], int on_device, cudaStream_t s) {
  df_status st = copy_cnn(kf, cnn, on_device, s);
  if (st != DF_OK) return st;
  DF_CUDA(cudaMemsetAsync(kf->planes.sc, 0, sizeof(Scalars), s));
  DF_CUDA(df::launch_init_state(kf->planes, s));
  if (on_device) DF_CUDA(df::launch_check_inputs(kf->planes, s));
  return DF_OK;
}

df_status check_params(const df_solve_params *p) {
  if (p->n_gn < 0 || p->n_pcg < 0) return fail(DF_EINVAL, "n_gn and n_pcg must be >= 0");
  if (p->loss != DF_LOSS_HUBER && p->loss != DF_LOSS_TUKEY)
    return fail(DF_EINVAL, "unknown loss %d", p->loss);
  if ((p->terms & ~DF_TERMS_ALL) != 0 || (p->terms & (DF_TERM_NET | DF_TERM_GRAD)) == 0)
    return fail(DF_EINVAL, "terms must be DF_TERM_* bits including NET or GRAD");
  if (p->solver < DF_SOLVER_AUTO || p->solver > DF_SOLVER_FUSED)
    return fail(DF_EINVAL, "unknown solver %d", p->solver);
  if (p->scale_step < DF_SCALE_FIXED || p->scale_step > DF_SCALE_JOINT)
    return fail(DF_EINVAL, "unknown scale_step %d", p->scale_step);
  if (!(p->tol >= 0.0) || !isfinite(p->tol)) return fail(DF_EINVAL, "tol must be finite >= 0");
  if (isnan(p->delta)) return fail(DF_EINVAL, "delta is NaN");
  if (p->warm_gn < 0) return fail(DF_EINVAL, "warm_gn must be >= 0");
  if (p->warm_gn > 0 && isnan(p->warm_delta)) return fail(DF_EINVAL, "warm_delta is NaN");
  return DF_OK;
}


SolveCfg cfg_of(const df_solve_params *p) {
  SolveCfg c;
  c.delta = p->delta;
  c.loss = p->loss;
  c.terms = p->terms;
  c.scale_step = p->scale_step;
  c.tol = p->tol;
  return c;
}

df_status read_report(df_keyframe *kf, cudaStream_t s, df_solve_report *rep) {
  Scalars h;
  DF_CUDA(cudaMemcpyAsync(&h, kf->planes.sc, sizeof h, cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  rep->scale_log = h.t;
  rep->res_norm = sqrt(h.rr);
  rep->iters_done = h.iters;
  rep->flags = h.flags;
  if (h.flags & df::kFlagBadInput) return fail(DF_ESTATE, "keyframe inputs failed the device check");
  if (h.flags & df::kFlagTimeout) return fail(DF_ETIMEOUT, "fused solve: a device-side wait gave up");
  return DF_OK;
}

}  // namespace

namespace df {
void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

df_status report(df_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

// The schedule as (at most) two phases of whole GN iterations: the warm
// start (Huber with warm_delta) and the rest (the requested loss). Each
// fused launch and each launch-solver run starts its first GN iteration
// with its own scale step, so two back-to-back solves are exactly one
// schedule whose loss changes after warm_gn iterations.
int split_schedule(const df_solve_params &p, df_solve_params ph[2]) {
  if (p.warm_gn <= 0 || p.n_gn == 0) {
    ph[0] = p;
    ph[0].warm_gn = 0;
    return 1;
  }
  const int warm = p.warm_gn < p.n_gn ? p.warm_gn : p.n_gn;
  ph[0] = p;
  ph[0].n_gn = warm;
  ph[0].loss = DF_LOSS_HUBER;
  ph[0].delta = p.warm_delta;
  ph[0].warm_gn = 0;
  if (warm == p.n_gn) return 1;
  ph[1] = p;
  ph[1].n_gn = p.n_gn - warm;
  ph[1].warm_gn = 0;
  return 2;
}

df_status check_solve_params(const df_solve_params *p) { return check_params(p); }

SolveCfg solve_cfg(const df_solve_params *p) { return cfg_of(p); }
}  // namespace df

extern "C" {

uint64_t df_kernel_launches(void) { return g_launches.load(); }

df_status df_set_tuning(const df_tuning *t) {
  df::FusedTuning n;
  if (t) {
    if (t->mode < 0 || t->mode > 2) return fail(DF_EINVAL, "tuning mode must be 0, 1 or 2");
    if (t->vec != 0 && t->vec != 1 && t->vec != 4) return fail(DF_EINVAL, "vec must be 0, 1 or 4");
    if (t->tile_rows < 0 || t->tile_rows > 64) return fail(DF_EINVAL, "tile_rows must be 0..64");
    if (t->max_ctas < 0) return fail(DF_EINVAL, "max_ctas must be >= 0");
    if (t->debug_skip_cta < -1) return fail(DF_EINVAL, "debug_skip_cta must be >= -1");
    n.mode = t->mode;
    n.vec = t->vec;
    n.tile_rows = t->tile_rows;
    n.max_ctas = t->max_ctas;
    if (t->gn_per_launch < 0) return fail(DF_EINVAL, "gn_per_launch must be >= 0");
    n.gn_per_launch = t->gn_per_launch;
    n.debug_skip_cta = t->debug_skip_cta;
    if (t->assembly < 0 || t->assembly > 2) return fail(DF_EINVAL, "assembly must be 0, 1 or 2");
    n.assembly = t->assembly;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune = n;
  return DF_OK;
}

df_status df_get_tuning(df_tuning *t) {
  if (!t) return fail(DF_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  t->mode = g_tune.mode;
  t->vec = g_tune.vec;
  t->tile_rows = g_tune.tile_rows;
  t->max_ctas = g_tune.max_ctas;
  t->gn_per_launch = g_tune.gn_per_launch;
  t->debug_skip_cta = g_tune.debug_skip_cta;
  t->assembly = g_tune.assembly;
  return DF_OK;
}

df_status df_set_spin_limit_ns(uint64_t ns) {
  if (ns == 0) return fail(DF_EINVAL, "spin limit must be > 0");
  g_spin_limit_ns.store(ns);
  return DF_OK;
}


void df_default_params(df_solve_params *p) {
  if (!p) return;
  p->n_gn = 10;
  p->n_pcg = 3;
  p->delta = 1.345f;
  p->loss = DF_LOSS_HUBER;
  p->terms = DF_TERMS_ALL;
  p->scale_step = 1;
  p->solver = DF_SOLVER_AUTO;
  p->tol = 0.0;
  p->warm_gn = 0;
  p->warm_delta = 1.345f;
}

size_t df_keyframe_bytes(int32_t width, int32_t height, int32_t cnn_dtype) {
  if (width < 1 || height < 1 || cnn_dtype < DF_F32 || cnn_dtype > DF_F16) return 0;
  return layout_of(width, height, cnn_dtype).total;
}

df_status df_set_memory_budget(size_t bytes) {
  g_budget.store(bytes);
  return DF_OK;
}

size_t df_memory_in_use(void) { return g_in_use.load(); }

df_status df_keyframe_create(const df_keyframe_desc *desc, const void *mu_net,
                             const void *var_net, const void *gx, const void *var_gx,
                             const void *gy, const void *var_gy, int ptrs_on_device,
                             void *stream, df_keyframe **out) {
  if (!out) return fail(DF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!desc) return fail(DF_EINVAL, "desc is NULL");
  const int W = desc->width, H = desc->height, dt = desc->cnn_dtype;
  if (W < 1 || H < 1) return fail(DF_EINVAL, "width and height must be >= 1");
  if ((int64_t)W * H > (int64_t)1 << 30) return fail(DF_EINVAL, "keyframe too large");
  if (dt != DF_F32 && dt != DF_BF16 && dt != DF_F16) return fail(DF_EINVAL, "bad cnn_dtype %d", dt);
  const void *cnn[6] = {mu_net, var_net, gx, var_gx, gy, var_gy};
  for (int j = 0; j < 6; ++j)
    if (!cnn[j]) return fail(DF_EINVAL, "network plane %d is NULL", j);
  if (!ptrs_on_device) {
    char why[256];
    if (!host_inputs_ok(cnn, W, H, dt, why, sizeof why))
      return fail(DF_EINVAL, "invalid network input: %s", why);
  }
  const Layout L = layout_of(W, H, dt);
  // reserve budget first
  size_t cur = g_in_use.load();
  for (;;) {
    const size_t budget = g_budget.load();
    if (budget != 0 && cur + L.total > budget)
      return fail(DF_EBUDGET, "keyframe needs %zu bytes, %zu of %zu in use", L.total, cur, budget);
    if (g_in_use.compare_exchange_weak(cur, cur + L.total)) break;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  void *mem = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&mem, L.total);
  if (e != cudaSuccess) {
    g_in_use.fetch_sub(L.total);
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? DF_ENOMEM : DF_ECUDA, "cudaMalloc(%zu): %s",
                L.total, cudaGetErrorString(e));
  }
  df_keyframe *kf = new df_keyframe();
  kf->device = dev;
  kf->W = W;
  kf->H = H;
  kf->P = pitch_of(W);
  kf->dtype = dt;
  kf->bytes = L.total;
  kf->mem = mem;
  char *base = static_cast<char *>(mem);
  Planes &k = kf->planes;
  k.W = W;
  k.H = H;
  k.P = kf->P;
  k.dtype = dt;
  for (int j = 0; j < 6; ++j) k.cnn[j] = base + L.cnn[j];
  k.mu_s = reinterpret_cast<float *>(base + L.mu_s);
  k.var_s = reinterpret_cast<float *>(base + L.var_s);
  k.x = reinterpret_cast<float *>(base + L.x);
  k.diag = reinterpret_cast<float *>(base + L.diag);
  k.wx = reinterpret_cast<float *>(base + L.wx);
  k.wy = reinterpret_cast<float *>(base + L.wy);
  for (int j = 0; j < df::kWorkPlanes; ++j) k.v[j] = reinterpret_cast<float *>(base + L.v[j]);
  k.sc = reinterpret_cast<Scalars *>(base + L.sc);
  k.partial = reinterpret_cast<double *>(base + L.partial);
  kf->staging = reinterpret_cast<float *>(base + L.staging);
  kf->semi_stage = reinterpret_cast<float *>(base + L.semi_stage);
  kf->copy_stream = nullptr;
  kf->ev_staged = kf->ev_free = nullptr;
  kf->plan = L.plan_cap ? base + L.plan : nullptr;
  kf->plan_cap = L.plan_cap;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  df_status st = DF_OK;
  e = cudaMemsetAsync(mem, 0, L.total, s);
  if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync");
  if (st == DF_OK) st = load_cnn(kf, cnn, ptrs_on_device, s);
  if (st != DF_OK) {
    cudaStreamSynchronize(s);
    cudaFree(mem);
    g_in_use.fetch_sub(L.total);
    delete kf;
    return st;
  }
  *out = kf;
  return DF_OK;
}

df_status df_keyframe_reset(df_keyframe *kf, const void *mu_net, const void *var_net,
                            const void *gx, const void *var_gx, const void *gy,
                            const void *var_gy, int ptrs_on_device, void *stream) {
  if (!kf) return fail(DF_EINVAL, "keyframe is NULL");
  const void *cnn[6] = {mu_net, var_net, gx, var_gx, gy, var_gy};
  for (int j = 0; j < 6; ++j)
    if (!cnn[j]) return fail(DF_EINVAL, "network plane %d is NULL", j);
  if (!ptrs_on_device) {
    char why[256];
    if (!host_inputs_ok(cnn, kf->W, kf->H, kf->dtype, why, sizeof why))
      return fail(DF_EINVAL, "invalid network input: %s", why);
  }
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // no semi-dense term until the next frame update
  DF_CUDA(cudaMemsetAsync((void *)kf->planes.var_s, 0, (size_t)kf->P * kf->H * 4, s));
  return load_cnn(kf, cnn, ptrs_on_device, s);
}

// The keyframe's copy stream and its two events, made on first use; false
// (and no error left pending) if the runtime cannot make them.
static bool ensure_copy_stream(df_keyframe *kf) {
  if (kf->copy_stream) return true;
  cudaStream_t cs = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreateWithFlags(&a, cudaEventDisableTiming) == cudaSuccess &&
      cudaEventCreateWithFlags(&b, cudaEventDisableTiming) == cudaSuccess) {
    kf->copy_stream = cs;
    kf->ev_staged = a;
    kf->ev_free = b;
    return true;
  }
  cudaGetLastError();
  if (b) cudaEventDestroy(b);
  if (a) cudaEventDestroy(a);
  if (cs) cudaStreamDestroy(cs);
  return false;
}

df_status df_frame_update(df_keyframe *kf, const float *mu_semi, const float *var_semi,
                          int ptrs_on_device, void *stream) {
  if (!kf) return fail(DF_EINVAL, "keyframe is NULL");
  if (!mu_semi || !var_semi) return fail(DF_EINVAL, "semi-dense plane is NULL");
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t row = (size_t)kf->W * 4, pitch = (size_t)kf->P * 4;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (!ptrs_on_device && cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
      cap == cudaStreamCaptureStatusNone && ensure_copy_stream(kf)) {
    // Upload on the copy stream once the previous update's staging has been
    // consumed; 's' waits for the upload and moves the planes into place, so
    // the call is still ordered on 's' and the host buffers are read before
    // 's' passes it. The upload itself overlaps whatever 's' runs before.
    const size_t n = (size_t)kf->W * kf->H * 4;
    float *st_mu = kf->semi_stage;
    float *st_var = reinterpret_cast<float *>(reinterpret_cast<char *>(st_mu) + align_up(n, 256));
    DF_CUDA(cudaStreamWaitEvent(kf->copy_stream, kf->ev_free, 0));
    DF_CUDA(cudaMemcpyAsync(st_mu, mu_semi, n, cudaMemcpyDefault, kf->copy_stream));
    DF_CUDA(cudaMemcpyAsync(st_var, var_semi, n, cudaMemcpyDefault, kf->copy_stream));
    DF_CUDA(cudaEventRecord(kf->ev_staged, kf->copy_stream));
    DF_CUDA(cudaStreamWaitEvent(s, kf->ev_staged, 0));
    DF_CUDA(cudaMemcpy2DAsync((void *)kf->planes.mu_s, pitch, st_mu, row, row, kf->H,
                              cudaMemcpyDeviceToDevice, s));
    DF_CUDA(cudaMemcpy2DAsync((void *)kf->planes.var_s, pitch, st_var, row, row, kf->H,
                              cudaMemcpyDeviceToDevice, s));
    DF_CUDA(cudaEventRecord(kf->ev_free, s));
    return DF_OK;
  }
  DF_CUDA(cudaMemcpy2DAsync((void *)kf->planes.mu_s, pitch, mu_semi, row, row, kf->H,
                            cudaMemcpyDefault, s));
  DF_CUDA(cudaMemcpy2DAsync((void *)kf->planes.var_s, pitch, var_semi, row, row, kf->H,
                            cudaMemcpyDefault, s));
  return DF_OK;
}

static df::FusedTuning current_tuning() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune;
}

static bool same_tuning(const df::FusedTuning &a, const df::FusedTuning &b) {
  return a.mode == b.mode && a.vec == b.vec && a.tile_rows == b.tile_rows &&
         a.max_ctas == b.max_ctas && a.debug_skip_cta == b.debug_skip_cta &&
         a.assembly == b.assembly;  // gn_per_launch
                                                                            // does not shape plans
}

static int pick_solver(const df_solve_params &p) {
  if (p.solver != DF_SOLVER_AUTO) return p.solver;
  // the joint solve with a tolerance runs on the launch solver only
  if (p.scale_step == DF_SCALE_JOINT && p.tol > 0.0) return DF_SOLVER_LAUNCHES;
  return df::fused_supported() ? DF_SOLVER_FUSED : DF_SOLVER_LAUNCHES;
}

static df_status check_joint(const df_solve_params &p) {
  if (p.scale_step == DF_SCALE_JOINT && p.solver == DF_SOLVER_FUSED && p.tol > 0.0)
    return fail(DF_ENOTSUP, "DF_SCALE_JOINT with tol > 0 runs on the launch solver only");
  return DF_OK;
}

// Fused solve of one keyframe: its launch plan lives in the keyframe's own
// allocation and is uploaded once per launch shape.
// joint: the joint (x, t) solve, which runs on a shared-memory resident
// plan, or on a streaming plan with 4 pixels per lane and at least one CG
// iteration; DF_ENOTSUP otherwise, before anything is launched.
static df_status fused_one(df_keyframe *kf, const SolveCfg &c, int n_gn, int n_pcg,
                           cudaStream_t s, bool joint = false, bool first_phase = true) {
  if (!df::fused_supported() || !kf->plan) return fail(DF_ENOTSUP, "fused solver not available on this device");
  const df::FusedTuning tune = current_tuning();
  if (kf->plan_shape.kind < 0 || !same_tuning(tune, kf->plan_tune)) {
    std::vector<char> host;
    df::LaunchShape shape;
    const Planes *one = &kf->planes;
    if (!df::fused_build_plan(&one, 1, tune, host, shape))
      return fail(DF_ENOTSUP, "fused solver: this launch shape cannot hold the keyframe");
    if (host.size() > kf->plan_cap) return fail(DF_EINVAL, "fused plan larger than reserved");
    DF_CUDA(cudaMemcpyAsync(kf->plan, host.data(), host.size(), cudaMemcpyHostToDevice, s));
    kf->plan_shape = shape;
    kf->plan_tune = tune;
  }
  if (joint && kf->plan_shape.kind != df::kPlanResident &&
      (kf->plan_shape.vec != 4 || (n_pcg < 1 && n_gn > 0)))
    return fail(DF_ENOTSUP, "the joint (x, t) solve needs a shared-memory resident plan or a "
                            "4-wide streaming plan with at least one CG iteration");
  const int chunk = tune.gn_per_launch > 0 ? tune.gn_per_launch : (n_gn > 0 ? n_gn : 1);
  for (int g0 = 0, first = 1; g0 < n_gn || first; g0 += chunk, first = 0) {
    const int m = std::min(chunk, n_gn - g0);
    DF_CUDA(df::fused_launch(kf->plan, kf->plan_shape, c, m < 0 ? 0 : m, n_pcg,
                             g_spin_limit_ns.load(), s, first && first_phase));
    if (n_gn == 0) break;
  }
  return DF_OK;
}

// Launch plans of keyframe lists prepared for repeated solves and for CUDA
// graphs (df_batch_prepare): kept on the device, keyed by the ordered
// keyframe list, the tuning and the device, and freed by df_batch_release
// or when one of their keyframes is destroyed. A list without a prepared
// plan gets a stream-ordered temporary one per solve.
struct BatchPlan {
  std::vector<df_keyframe *> kfs;
  df::FusedTuning tune;
  int device = 0;
  df::LaunchShape shape;
  void *dplan = nullptr;
};
static std::mutex g_bp_mu;
static std::vector<BatchPlan> g_bp;

static void drop_batch_plans_if(const std::vector<df_keyframe *> &any_of) {
  std::lock_guard<std::mutex> lk(g_bp_mu);
  for (size_t j = 0; j < g_bp.size();) {
    bool hit = false;
    for (df_keyframe *k : any_of)
      hit = hit || std::find(g_bp[j].kfs.begin(), g_bp[j].kfs.end(), k) != g_bp[j].kfs.end();
    if (hit) {
      cudaFree(g_bp[j].dplan);  // synchronising: no launch still reads it
      g_bp.erase(g_bp.begin() + j);
    } else {
      ++j;
    }
  }
}

static bool find_batch_plan(df_keyframe *const *kfs, int n, const df::FusedTuning &tune,
                            void **dplan, df::LaunchShape *shape) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_bp_mu);
  for (const BatchPlan &b : g_bp) {
    if (b.device == dev && (int)b.kfs.size() == n && same_tuning(b.tune, tune) &&
        std::equal(b.kfs.begin(), b.kfs.end(), kfs)) {
      *dplan = b.dplan;
      *shape = b.shape;
      return true;
    }
  }
  return false;
}

static df_status fused_launches(void *dplan, const df::LaunchShape &shape,
                                const df::FusedTuning &tune, const SolveCfg &c, int n_gn,
                                int n_pcg, cudaStream_t s, bool first_phase) {
  const int chunk = tune.gn_per_launch > 0 ? tune.gn_per_launch : (n_gn > 0 ? n_gn : 1);
  for (int g0 = 0, first = 1; g0 < n_gn || first; g0 += chunk, first = 0) {
    const int m = std::min(chunk, n_gn - g0);
    DF_CUDA(df::fused_launch(dplan, shape, c, m < 0 ? 0 : m, n_pcg, g_spin_limit_ns.load(), s,
                             first && first_phase));
    if (n_gn == 0) break;
  }
  return DF_OK;
}

// Fused solve of a list of keyframes in as few launches as the plan allows
// (a list whose tiles cannot share one grid is split in halves).
static df_status fused_many(df_keyframe *const *kfs, int n, const SolveCfg &c, int n_gn,
                            int n_pcg, cudaStream_t s, bool first_phase) {
  if (n <= 0) return DF_OK;
  if (n == 1) return fused_one(kfs[0], c, n_gn, n_pcg, s, false, first_phase);
  if (n > df::kMaxBatch) {
    df_status st = fused_many(kfs, df::kMaxBatch, c, n_gn, n_pcg, s, first_phase);
    if (st != DF_OK) return st;
    return fused_many(kfs + df::kMaxBatch, n - df::kMaxBatch, c, n_gn, n_pcg, s, first_phase);
  }
  const df::FusedTuning tune = current_tuning();
  void *dplan = nullptr;
  df::LaunchShape shape;
  if (find_batch_plan(kfs, n, tune, &dplan, &shape))
    return fused_launches(dplan, shape, tune, c, n_gn, n_pcg, s, first_phase);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs != cudaStreamCaptureStatusNone)
    return fail(DF_ENOTSUP, "batched solve under stream capture needs df_batch_prepare on "
                            "this keyframe list first");
  std::vector<const Planes *> list(n);
  for (int j = 0; j < n; ++j) list[j] = &kfs[j]->planes;
  std::vector<char> host;
  if (!df::fused_build_plan(list.data(), n, tune, host, shape)) {
    const int h = n / 2;
    df_status st = fused_many(kfs, h, c, n_gn, n_pcg, s, first_phase);
    if (st != DF_OK) return st;
    return fused_many(kfs + h, n - h, c, n_gn, n_pcg, s, first_phase);
  }
  DF_CUDA(cudaMallocAsync(&dplan, host.size(), s));
  cudaError_t e = cudaMemcpyAsync(dplan, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  df_status st = e == cudaSuccess
                     ? fused_launches(dplan, shape, tune, c, n_gn, n_pcg, s, first_phase)
                     : cuda_fail(e, "batch plan upload");
  cudaError_t e2 = cudaFreeAsync(dplan, s);
  if (st != DF_OK) return st;
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  return DF_OK;
}

// df_batch_prepare: the plans fused_many would build for this list, kept.
static df_status prepare_many(df_keyframe *const *kfs, int n, cudaStream_t s) {
  if (n <= 1) return DF_OK;  // a single keyframe keeps its own plan
  if (n > df::kMaxBatch) {
    df_status st = prepare_many(kfs, df::kMaxBatch, s);
    if (st != DF_OK) return st;
    return prepare_many(kfs + df::kMaxBatch, n - df::kMaxBatch, s);
  }
  const df::FusedTuning tune = current_tuning();
  void *dp = nullptr;
  df::LaunchShape shape;
  if (find_batch_plan(kfs, n, tune, &dp, &shape)) return DF_OK;
  std::vector<const Planes *> list(n);
  for (int j = 0; j < n; ++j) list[j] = &kfs[j]->planes;
  std::vector<char> host;
  if (!df::fused_build_plan(list.data(), n, tune, host, shape)) {
    const int h = n / 2;
    df_status st = prepare_many(kfs, h, s);
    if (st != DF_OK) return st;
    return prepare_many(kfs + h, n - h, s);
  }
  BatchPlan b;
  DF_CUDA(cudaMalloc(&b.dplan, host.size()));
  cudaError_t e = cudaMemcpyAsync(b.dplan, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(b.dplan);
    return cuda_fail(e, "batch plan upload");
  }
  b.kfs.assign(kfs, kfs + n);
  b.tune = tune;
  cudaGetDevice(&b.device);
  b.shape = shape;
  std::lock_guard<std::mutex> lk(g_bp_mu);
  g_bp.push_back(std::move(b));
  return DF_OK;
}

// One phase of a keyframe's schedule (first: the PCG iteration count of the
// report starts at zero; otherwise it continues the previous phase's).
static df_status optimise_phase(df_keyframe *kf, const df_solve_params *p, cudaStream_t s,
                                bool first) {
  const SolveCfg c = cfg_of(p);
  const bool joint = p->scale_step == DF_SCALE_JOINT;
  if (pick_solver(*p) == DF_SOLVER_FUSED) {
    df_status st = fused_one(kf, c, p->n_gn, p->n_pcg, s, joint, first);
    // the joint solve on a streaming launch shape: the launch solver serves AUTO
    if (!(joint && st == DF_ENOTSUP && p->solver == DF_SOLVER_AUTO)) return st;
  }
  if (first) DF_CUDA(cudaMemsetAsync(&kf->planes.sc->iters, 0, sizeof(int), s));
  DF_CUDA(cudaMemsetAsync(&kf->planes.sc->stop, 0, sizeof(int), s));
  DF_CUDA(df::launch_solve_launches(kf->planes, c, p->n_gn, p->n_pcg, s));
  return DF_OK;
}

static df_status optimise_one(df_keyframe *kf, const df_solve_params *p, cudaStream_t s) {
  df_solve_params ph[2];
  const int n = df::split_schedule(*p, ph);
  for (int j = 0; j < n; ++j) {
    df_status st = optimise_phase(kf, &ph[j], s, j == 0);
    if (st != DF_OK) return st;
  }
  return DF_OK;
}

df_status df_optimise(df_keyframe *kf, const df_solve_params *params, void *stream,
                      df_solve_report *report) {
  if (!kf) return fail(DF_EINVAL, "keyframe is NULL");
  df_solve_params p;
  if (params) {
    p = *params;
  } else {
    df_default_params(&p);
  }
  df_status st = check_params(&p);
  if (st == DF_OK) st = check_joint(p);
  if (st != DF_OK) return st;
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = optimise_one(kf, &p, s);
  if (st != DF_OK) return st;
  if (report) return read_report(kf, s, report);
  return DF_OK;
}

df_status df_optimise_batch(df_keyframe *const *kfs, int32_t n, const df_solve_params *params,
                            void *stream, df_solve_report *reports) {
  if (n < 0 || (n > 0 && !kfs)) return fail(DF_EINVAL, "bad keyframe list");
  df_solve_params p;
  if (params) {
    p = *params;
  } else {
    df_default_params(&p);
  }
  df_status st = check_params(&p);
  if (st == DF_OK) st = check_joint(p);
  if (st != DF_OK) return st;
  for (int j = 0; j < n; ++j) {
    if (!kfs[j]) return fail(DF_EINVAL, "keyframe %d is NULL", j);
    for (int m = 0; m < j; ++m)
      if (kfs[m] == kfs[j]) return fail(DF_EINVAL, "keyframe %d appears twice", j);
    if (kfs[j]->device != kfs[0]->device) return fail(DF_EINVAL, "keyframes on different devices");
  }
  if (n == 0) return DF_OK;
  DeviceGuard g(kfs[0]->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (pick_solver(p) == DF_SOLVER_FUSED && p.scale_step != DF_SCALE_JOINT) {
    df_solve_params ph[2];
    const int np = df::split_schedule(p, ph);
    for (int j = 0; j < np; ++j) {
      st = fused_many(kfs, n, cfg_of(&ph[j]), ph[j].n_gn, ph[j].n_pcg, s, j == 0);
      if (st != DF_OK) return st;
    }
  } else {  // the launch solver, or the joint solve (keyframe by keyframe)
    for (int j = 0; j < n; ++j) {
      st = optimise_one(kfs[j], &p, s);
      if (st != DF_OK) return st;
    }
  }
  if (reports) {
    df_status worst = DF_OK;
    for (int j = 0; j < n; ++j) {
      st = read_report(kfs[j], s, &reports[j]);
      if (st != DF_OK && worst == DF_OK) worst = st;
    }
    return worst;
  }
  return DF_OK;
}

df_status df_batch_prepare(df_keyframe *const *kfs, int32_t n, void *stream) {
  if (n < 0 || (n > 0 && !kfs)) return fail(DF_EINVAL, "bad keyframe list");
  for (int j = 0; j < n; ++j) {
    if (!kfs[j]) return fail(DF_EINVAL, "keyframe %d is NULL", j);
    for (int m = 0; m < j; ++m)
      if (kfs[m] == kfs[j]) return fail(DF_EINVAL, "keyframe %d appears twice", j);
    if (kfs[j]->device != kfs[0]->device) return fail(DF_EINVAL, "keyframes on different devices");
  }
  if (n < 2) return DF_OK;
  if (!df::fused_supported()) return fail(DF_ENOTSUP, "fused solver not available on this device");
  DeviceGuard g(kfs[0]->device);
  return prepare_many(kfs, n, static_cast<cudaStream_t>(stream));
}

df_status df_batch_release(df_keyframe *const *kfs, int32_t n) {
  if (n < 0 || (n > 0 && !kfs)) return fail(DF_EINVAL, "bad keyframe list");
  std::vector<df_keyframe *> v(kfs, kfs + n);
  drop_batch_plans_if(v);
  return DF_OK;
}

df_status df_fetch_depth(df_keyframe *kf, float *out, int log_space, int ptr_on_device,
                         void *stream) {
  if (!kf) return fail(DF_EINVAL, "keyframe is NULL");
  if (!out) return fail(DF_EINVAL, "out is NULL");
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (ptr_on_device) {
    DF_CUDA(df::launch_fetch(kf->planes, out, log_space, s));
    return DF_OK;
  }
  DF_CUDA(df::launch_fetch(kf->planes, kf->staging, log_space, s));
  DF_CUDA(cudaMemcpyAsync(out, kf->staging, (size_t)kf->W * kf->H * 4, cudaMemcpyDeviceToHost, s));
  return DF_OK;
}

// ---- batched bookkeeping of many keyframes --------------------------------

static df_status check_list(df_keyframe *const *kfs, int32_t n) {
  if (n < 0 || (n > 0 && !kfs)) return fail(DF_EINVAL, "bad keyframe list");
  for (int j = 0; j < n; ++j) {
    if (!kfs[j]) return fail(DF_EINVAL, "keyframe %d is NULL", j);
    for (int m = 0; m < j; ++m)
      if (kfs[m] == kfs[j]) return fail(DF_EINVAL, "keyframe %d appears twice", j);
    if (kfs[j]->device != kfs[0]->device) return fail(DF_EINVAL, "keyframes on different devices");
  }
  return DF_OK;
}

// A batched solve whose launch plan goes through caller-owned buffers: the
// plan is built on the host into 'hplan' (pinned), copied to 'dplan' on the
// stream and used for every phase of the schedule; no allocation. With
// one_launch (and the automatic placement) the streaming kernel keeps its
// assembly, so each phase is one cooperative launch. Lists that
// cannot use them (one keyframe, not the fused solver, the joint variant,
// more keyframes than one launch holds, a plan larger than the buffers, a
// list that must be split) take df_optimise_batch. The buffers must not be
// reused before the stream has passed this call.
extern "C++" {
namespace df {

df_status optimise_batch_buffered(df_keyframe *const *kfs, int32_t n, const df_solve_params *params,
                                  cudaStream_t s, void *dplan, size_t dcap, void *hplan,
                                  size_t hcap, bool one_launch) {
  df_solve_params p;
  if (params) {
    p = *params;
  } else {
    df_default_params(&p);
  }
  if (n <= 1 || n > df::kMaxBatch || !dplan || !hplan || check_params(&p) != DF_OK ||
      check_joint(p) != DF_OK || pick_solver(p) != DF_SOLVER_FUSED ||
      p.scale_step == DF_SCALE_JOINT || check_list(kfs, n) != DF_OK)
    return df_optimise_batch(kfs, n, params, s, nullptr);
  DeviceGuard g(kfs[0]->device);
  df::FusedTuning tune = current_tuning();
  if (one_launch && tune.assembly == 0) tune.assembly = 1;  // the assembly in the persistent kernel
  void *dp = nullptr;
  df::LaunchShape shape;
  if (!find_batch_plan(kfs, n, tune, &dp, &shape)) {
    std::vector<const Planes *> list(n);
    for (int j = 0; j < n; ++j) list[j] = &kfs[j]->planes;
    std::vector<char> host;
    if (!df::fused_build_plan(list.data(), n, tune, host, shape) || host.size() > dcap ||
        host.size() > hcap)
      return df_optimise_batch(kfs, n, params, s, nullptr);
    memcpy(hplan, host.data(), host.size());
    DF_CUDA(cudaMemcpyAsync(dplan, hplan, host.size(), cudaMemcpyHostToDevice, s));
    dp = dplan;
  }
  df_solve_params ph[2];
  const int np = df::split_schedule(p, ph);
  for (int j = 0; j < np; ++j) {
    df_status st = fused_launches(dp, shape, tune, cfg_of(&ph[j]), ph[j].n_gn, ph[j].n_pcg, s,
                                  j == 0);
    if (st != DF_OK) return st;
  }
  return DF_OK;
}

}  // namespace df
}  // extern "C++"

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Host buffers in page-locked (pinned) memory are read and written by the
// batched kernels directly: *out gets each one's device-side address. False
// (and nothing changed) if any of them is pageable.
static bool pinned_all(const void *const *p, int n, std::vector<const void *> *out) {
  out->resize(n);
  for (int j = 0; j < n; ++j) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p[j]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    (*out)[j] = a.devicePointer;
  }
  return true;
}

// Fill one launch's item table with keyframes [j0, j0 + m) of the list.
extern "C++" {
template <typename Fill>
static df_status launch_io_chunks(df_keyframe *const *kfs, int32_t n, df::IoKind kind, int check,
                                  int log_space, cudaStream_t s, Fill fill) {
  for (int j0 = 0; j0 < n; j0 += df::kIoBatch) {
    const int m = std::min(df::kIoBatch, n - j0);
    df::IoBatch b;
    memset(&b, 0, sizeof b);
    b.n = m;
    b.check = check;
    b.log_space = log_space;
    int rows = 0;
    for (int q = 0; q < m; ++q) {
      df_keyframe *kf = kfs[j0 + q];
      df::IoItem &it = b.item[q];
      it.W = kf->W;
      it.H = kf->H;
      it.P = kf->P;
      it.dtype = kf->dtype;
      it.x = kf->planes.x;
      it.var_s = const_cast<float *>(kf->planes.var_s);
      it.sc = kf->planes.sc;
      it.row0 = rows;
      rows += kf->H;
      fill(j0 + q, kf, it);
    }
    b.total = rows;
    DF_CUDA(df::launch_io(kind, b, s));
  }
  return DF_OK;
}
}  // extern "C++"

df_status df_keyframe_reset_batch(df_keyframe *const *kfs, int32_t n, const void *const *planes,
                                  int ptrs_on_device, void *stream) {
  df_status st = check_list(kfs, n);
  if (st != DF_OK) return st;
  if (n == 0) return DF_OK;
  if (!planes) return fail(DF_EINVAL, "planes is NULL");
  for (int j = 0; j < 6 * n; ++j)
    if (!planes[j]) return fail(DF_EINVAL, "network plane %d of keyframe %d is NULL", j % 6, j / 6);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<const void *> mapped;
  if (!ptrs_on_device && pinned_all(planes, 6 * n, &mapped)) {
    // pinned host planes: the kernel reads them directly and checks them on
    // the device, as it does device planes
    planes = mapped.data();
    ptrs_on_device = 1;
  }
  if (!ptrs_on_device) {
    // pageable host planes: every keyframe's inputs are checked before any is
    // touched, then each goes up through its staging plane
    for (int j = 0; j < n; ++j) {
      char why[256];
      if (!host_inputs_ok(planes + 6 * j, kfs[j]->W, kfs[j]->H, kfs[j]->dtype, why, sizeof why))
        return fail(DF_EINVAL, "invalid network input of keyframe %d: %s", j, why);
    }
    for (int j = 0; j < n; ++j) {
      DeviceGuard g(kfs[j]->device);
      df_keyframe *kf = kfs[j];
      DF_CUDA(cudaMemsetAsync((void *)kf->planes.var_s, 0, (size_t)kf->P * kf->H * 4, s));
      st = load_cnn(kf, planes + 6 * j, 0, s);
      if (st != DF_OK) return st;
    }
    return DF_OK;
  }
  DeviceGuard g(kfs[0]->device);
  return launch_io_chunks(kfs, n, df::IoKind::kReset, 1, 0, s,
                          [&](int j, df_keyframe *kf, df::IoItem &it) {
                            const size_t es = elem_size(kf->dtype);
                            bool vec = ((size_t)kf->W * es) % 16 == 0;
                            for (int q = 0; q < 6; ++q) {
                              it.src[q] = planes[6 * j + q];
                              it.dst[q] = const_cast<void *>(kf->planes.cnn[q]);
                              vec = vec && aligned16(it.src[q]);
                            }
                            it.vec = vec;
                          });
}

df_status df_frame_update_batch(df_keyframe *const *kfs, int32_t n, const float *const *mu_semi,
                                const float *const *var_semi, int ptrs_on_device, void *stream) {
  df_status st = check_list(kfs, n);
  if (st != DF_OK) return st;
  if (n == 0) return DF_OK;
  if (!mu_semi || !var_semi) return fail(DF_EINVAL, "plane list is NULL");
  for (int j = 0; j < n; ++j)
    if (!mu_semi[j] || !var_semi[j]) return fail(DF_EINVAL, "semi-dense plane of keyframe %d is NULL", j);
  std::vector<const void *> mu_m, var_m;
  if (!ptrs_on_device && pinned_all(reinterpret_cast<const void *const *>(mu_semi), n, &mu_m) &&
      pinned_all(reinterpret_cast<const void *const *>(var_semi), n, &var_m)) {
    mu_semi = reinterpret_cast<const float *const *>(mu_m.data());
    var_semi = reinterpret_cast<const float *const *>(var_m.data());
    ptrs_on_device = 1;  // pinned: read directly by the kernel
  }
  if (!ptrs_on_device) {
    // host planes: each keyframe's upload overlaps the previous solve as in
    // df_frame_update
    for (int j = 0; j < n; ++j) {
      st = df_frame_update(kfs[j], mu_semi[j], var_semi[j], 0, stream);
      if (st != DF_OK) return st;
    }
    return DF_OK;
  }
  DeviceGuard g(kfs[0]->device);
  return launch_io_chunks(kfs, n, df::IoKind::kUpdate, 0, 0, static_cast<cudaStream_t>(stream),
                          [&](int j, df_keyframe *kf, df::IoItem &it) {
                            it.src[0] = mu_semi[j];
                            it.src[1] = var_semi[j];
                            it.dst[0] = const_cast<float *>(kf->planes.mu_s);
                            it.dst[1] = const_cast<float *>(kf->planes.var_s);
                            it.vec = kf->W % 4 == 0 && aligned16(mu_semi[j]) && aligned16(var_semi[j]);
                          });
}

df_status df_fetch_depth_batch(df_keyframe *const *kfs, int32_t n, float *const *out,
                               int log_space, int ptrs_on_device, void *stream) {
  df_status st = check_list(kfs, n);
  if (st != DF_OK) return st;
  if (n == 0) return DF_OK;
  if (!out) return fail(DF_EINVAL, "output list is NULL");
  for (int j = 0; j < n; ++j)
    if (!out[j]) return fail(DF_EINVAL, "output of keyframe %d is NULL", j);
  std::vector<const void *> out_m;
  std::vector<float *> out_w;
  if (!ptrs_on_device && pinned_all(reinterpret_cast<const void *const *>(out), n, &out_m)) {
    for (const void *q : out_m) out_w.push_back(static_cast<float *>(const_cast<void *>(q)));
    out = out_w.data();
    ptrs_on_device = 1;  // pinned: written directly by the kernel
  }
  if (!ptrs_on_device) {
    for (int j = 0; j < n; ++j) {
      st = df_fetch_depth(kfs[j], out[j], log_space, 0, stream);
      if (st != DF_OK) return st;
    }
    return DF_OK;
  }
  DeviceGuard g(kfs[0]->device);
  return launch_io_chunks(kfs, n, df::IoKind::kFetch, 0, log_space ? 1 : 0,
                          static_cast<cudaStream_t>(stream),
                          [&](int j, df_keyframe *kf, df::IoItem &it) {
                            it.dst[0] = out[j];
                            it.vec = kf->W % 4 == 0 && aligned16(out[j]);
                          });
}

df_status df_keyframe_get_state(df_keyframe *kf, float *x_out, double *t_out,
                                int ptrs_on_device, void *stream) {
  if (!kf) return fail(DF_EINVAL, "keyframe is NULL");
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (x_out) {
    DF_CUDA(cudaMemcpy2DAsync(x_out, (size_t)kf->W * 4, kf->planes.x, (size_t)kf->P * 4,
                              (size_t)kf->W * 4, kf->H, cudaMemcpyDefault, s));
  }
  if (t_out) DF_CUDA(cudaMemcpyAsync(t_out, &kf->planes.sc->t, sizeof(double), cudaMemcpyDefault, s));
  if (!ptrs_on_device) DF_CUDA(cudaStreamSynchronize(s));
  return DF_OK;
}

df_status df_keyframe_set_state(df_keyframe *kf, const float *x, double t, int ptrs_on_device,
                                void *stream) {
  (void)ptrs_on_device;
  if (!kf) return fail(DF_EINVAL, "keyframe is NULL");
  if (!isfinite(t)) return fail(DF_EINVAL, "t must be finite");
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (x) {
    DF_CUDA(cudaMemcpy2DAsync(kf->planes.x, (size_t)kf->P * 4, x, (size_t)kf->W * 4,
                              (size_t)kf->W * 4, kf->H, cudaMemcpyDefault, s));
  }
  DF_CUDA(df::launch_set_scale(kf->planes, t, s));
  return DF_OK;
}

df_status df_cost(df_keyframe *kf, const df_solve_params *params, void *stream, double *cost_out) {
  if (!kf || !cost_out) return fail(DF_EINVAL, "NULL argument");
  df_solve_params p;
  if (params) {
    p = *params;
  } else {
    df_default_params(&p);
  }
  df_status st = check_params(&p);
  if (st != DF_OK) return st;
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DF_CUDA(df::launch_cost(kf->planes, cfg_of(&p), s));
  DF_CUDA(cudaMemcpyAsync(cost_out, &kf->planes.sc->cost, sizeof(double), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  return DF_OK;
}

df_status df_depth_accuracy(df_keyframe *kf, const float *depth_true, int ptr_on_device,
                            double rel_tol, void *stream, int64_t *n_within, int64_t *n_valid) {
  if (!kf || !depth_true || !n_within || !n_valid) return fail(DF_EINVAL, "NULL argument");
  if (!(rel_tol >= 0.0) || !isfinite(rel_tol)) return fail(DF_EINVAL, "rel_tol must be finite >= 0");
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float *dt = depth_true;
  if (!ptr_on_device) {
    DF_CUDA(cudaMemcpyAsync(kf->staging, depth_true, (size_t)kf->W * kf->H * 4,
                            cudaMemcpyHostToDevice, s));
    dt = kf->staging;
  }
  DF_CUDA(df::launch_accuracy(kf->planes, dt, rel_tol, s));
  double h[2];
  DF_CUDA(cudaMemcpyAsync(h, &kf->planes.sc->acc_in, sizeof h, cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  *n_within = (int64_t)h[0];
  *n_valid = (int64_t)h[1];
  return DF_OK;
}

df_status df_scale_fit_ls(df_keyframe *kf, void *stream) {
  if (!kf) return fail(DF_EINVAL, "keyframe is NULL");
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DF_CUDA(df::launch_ls_scale_fit(kf->planes, s));
  return DF_OK;
}

df_status df_keyframe_check(df_keyframe *kf, void *stream) {
  if (!kf) return fail(DF_EINVAL, "keyframe is NULL");
  DeviceGuard g(kf->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int flags = 0;
  DF_CUDA(cudaMemcpyAsync(&flags, &kf->planes.sc->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  if (flags & df::kFlagBadInput) return fail(DF_EINVAL, "network inputs failed the device check");
  if (flags & df::kFlagTimeout) return fail(DF_ETIMEOUT, "a fused solve gave up waiting");
  return DF_OK;
}

df_status df_keyframe_info(const df_keyframe *kf, df_keyframe_desc *desc, size_t *device_bytes) {
  if (!kf) return fail(DF_EINVAL, "keyframe is NULL");
  if (desc) {
    desc->width = kf->W;
    desc->height = kf->H;
    desc->cnn_dtype = kf->dtype;
  }
  if (device_bytes) *device_bytes = kf->bytes;
  return DF_OK;
}

void df_keyframe_destroy(df_keyframe *kf) {
  if (!kf) return;
  {
    DeviceGuard g(kf->device);
    drop_batch_plans_if({kf});
    // released by the runtime once their pending work is done
    if (kf->ev_staged) cudaEventDestroy(kf->ev_staged);
    if (kf->ev_free) cudaEventDestroy(kf->ev_free);
    if (kf->copy_stream) cudaStreamDestroy(kf->copy_stream);
    cudaFree(kf->mem);  // waits for the keyframe's pending work
  }
  g_in_use.fetch_sub(kf->bytes);
  delete kf;
}

df_status df_semi_to_log(const float *depth, const float *var_depth, float *mu_semi,
                         float *var_semi, int64_t n, int ptrs_on_device, void *stream) {
  if (n < 0) return fail(DF_EINVAL, "n < 0");
  if (n == 0) return DF_OK;
  if (!depth || !var_depth || !mu_semi || !var_semi) return fail(DF_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (ptrs_on_device) {
    DF_CUDA(df::launch_semi_to_log(depth, var_depth, mu_semi, var_semi, n, s));
    return DF_OK;
  }
  // host arrays: stage through stream-ordered device memory, compute on the GPU
  float *buf = nullptr;
  const size_t bytes = (size_t)n * 4;
  DF_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&buf), bytes * 4, s));
  df_status st = DF_OK;
  cudaError_t e = cudaMemcpyAsync(buf, depth, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + n, var_depth, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = df::launch_semi_to_log(buf, buf + n, buf + 2 * n, buf + 3 * n, n, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mu_semi, buf + 2 * n, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(var_semi, buf + 3 * n, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) st = cuda_fail(e, "df_semi_to_log");
  cudaFreeAsync(buf, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (st == DF_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamSynchronize");
  return st;
}

const char *df_status_str(df_status s) {
  switch (s) {
    case DF_OK: return "DF_OK";
    case DF_EINVAL: return "DF_EINVAL";
    case DF_ENOMEM: return "DF_ENOMEM";
    case DF_EBUDGET: return "DF_EBUDGET";
    case DF_ECUDA: return "DF_ECUDA";
    case DF_ETIMEOUT: return "DF_ETIMEOUT";
    case DF_ESTATE: return "DF_ESTATE";
    case DF_ENOTSUP: return "DF_ENOTSUP";
  }
  return "DF_UNKNOWN";
}

const char *df_last_error(void) { return g_err.c_str(); }

}  // extern "C"
