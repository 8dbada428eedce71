// Serving layer (include/deepfusion.h, "serving"): camera streams with
// device-resident keyframes, per-stream frame queues, and a non-blocking
// scheduler that packs every ready stream into one batched solve
// (continuous batching) or, as the baseline, solves each frame alone.
#include <algorithm>
#include <chrono>
#include <deque>
#include <vector>

#include "df_fused.cuh"
#include "df_internal.cuh"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Req {
  int32_t sid;
  const float *mu, *var;
  int on_device;
  uint64_t tag;
  int64_t t_submit;
};

struct StreamState {
  df_keyframe *kf = nullptr;
  size_t bytes = 0;
  bool busy = false;  // a frame of this stream is on the GPU
  std::deque<Req> queue;
};

struct Launch {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool active = false;
  int64_t t_launch = 0;
  std::vector<Req> reqs;
  // the slot's launch plan of a batched solve, built on the host into the
  // pinned buffer and copied to the device buffer every tick; a slot is
  // refilled only after its previous launch has finished, so both are free.
  // Each solve stays one cooperative launch (no separate assembly kernel):
  // with several slots in flight on different streams, extra ordinary
  // launches interleave with the other slots' whole-GPU launches (measured
  // at 1500 frames/s: p99 11.6 / 17.5 ms with one launch per solve against
  // 16.2 / 24.5 ms with the separate assembly, two arrival seeds)
  void *dplan = nullptr, *hplan = nullptr;
  size_t plan_cap = 0;
};

}  // namespace

struct df_server {
  df_server_config cfg;
  int device = 0;
  size_t used = 0;
  std::vector<StreamState> streams;
  std::vector<Launch> launches;
  std::deque<Req> arrivals;  // every queued frame in arrival order (plain mode)
  std::deque<df_completion> done;
  int32_t pending = 0;
};

namespace {

df_status retire(df_server *s) {
  for (Launch &L : s->launches) {
    if (!L.active) continue;
    const cudaError_t q = cudaEventQuery(L.done);
    if (q == cudaErrorNotReady) continue;
    const int64_t t = now_ns();
    df_status st = DF_OK;
    if (q != cudaSuccess) {
      cudaGetLastError();
      st = df::report(DF_ECUDA, "server launch failed: %s", cudaGetErrorString(q));
    }
    for (const Req &r : L.reqs) {
      df_completion c{};
      c.tag = r.tag;
      c.stream_id = r.sid;
      c.status = st;
      c.t_submit_ns = r.t_submit;
      c.t_launch_ns = L.t_launch;
      c.t_done_ns = t;
      c.batch_size = (int32_t)L.reqs.size();
      s->done.push_back(c);
      s->streams[r.sid].busy = false;
    }
    L.reqs.clear();
    L.active = false;
  }
  return DF_OK;
}

// Start one launch on the free slot L; returns false when nothing was ready.
df_status start_one(df_server *s, Launch &L, bool *started) {
  *started = false;
  std::vector<Req> take;
  if (s->cfg.batching) {
    // oldest waiting frame of every idle stream, oldest first, up to max_batch
    std::vector<std::pair<int64_t, int32_t>> ready;
    for (size_t i = 0; i < s->streams.size(); ++i) {
      const StreamState &st = s->streams[i];
      if (st.kf && !st.busy && !st.queue.empty()) ready.push_back({st.queue.front().t_submit, (int32_t)i});
    }
    if (ready.empty()) return DF_OK;
    std::sort(ready.begin(), ready.end());
    const size_t n = std::min(ready.size(), (size_t)s->cfg.max_batch);
    for (size_t j = 0; j < n; ++j) {
      StreamState &st = s->streams[ready[j].second];
      take.push_back(st.queue.front());
      st.queue.pop_front();
    }
  } else {
    // the oldest queued frame whose stream is idle
    for (auto it = s->arrivals.begin(); it != s->arrivals.end(); ++it) {
      StreamState &st = s->streams[it->sid];
      if (st.kf && !st.busy) {
        take.push_back(*it);
        st.queue.pop_front();  // frames of a stream leave in order
        s->arrivals.erase(it);
        break;
      }
    }
    if (take.empty()) return DF_OK;
  }
  std::vector<df_keyframe *> kfs;
  std::vector<const float *> mus, vars;
  bool all_dev = true;
  for (const Req &r : take) {
    kfs.push_back(s->streams[r.sid].kf);
    mus.push_back(r.mu);
    vars.push_back(r.var);
    all_dev = all_dev && r.on_device;
  }
  if (all_dev && take.size() > 1) {  // every frame in device memory: one launch
    df_status e = df_frame_update_batch(kfs.data(), (int32_t)kfs.size(), mus.data(), vars.data(),
                                        1, L.stream);
    if (e != DF_OK) return e;
  } else {
    for (const Req &r : take) {
      df_status e = df_frame_update(s->streams[r.sid].kf, r.mu, r.var, r.on_device, L.stream);
      if (e != DF_OK) return e;
    }
  }
  for (const Req &r : take) s->streams[r.sid].busy = true;
  df_status e = kfs.size() == 1
                    ? df_optimise(kfs[0], &s->cfg.params, L.stream, nullptr)
                    : df::optimise_batch_buffered(kfs.data(), (int32_t)kfs.size(), &s->cfg.params,
                                                  L.stream, L.dplan, L.plan_cap, L.hplan,
                                                  L.plan_cap, true);
  if (e != DF_OK) return e;
  cudaError_t ce = cudaEventRecord(L.done, L.stream);
  if (ce != cudaSuccess) return df::report(DF_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(ce));
  L.t_launch = now_ns();
  L.reqs = std::move(take);
  L.active = true;
  *started = true;
  return DF_OK;
}

}  // namespace

extern "C" {

df_status df_server_create(const df_server_config *cfg, df_server **out) {
  if (!out) return df::report(DF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return df::report(DF_EINVAL, "cfg is NULL");
  if (cfg->max_batch < 1 || cfg->max_batch > 256) return df::report(DF_EINVAL, "max_batch must be 1..256");
  if (cfg->max_inflight < 1 || cfg->max_inflight > 16)
    return df::report(DF_EINVAL, "max_inflight must be 1..16");
  df_status st = df::check_solve_params(&cfg->params);
  if (st != DF_OK) return st;
  df_server *s = new df_server();
  s->cfg = *cfg;
  if (!s->cfg.batching) s->cfg.max_batch = 1;
  cudaGetDevice(&s->device);
  s->launches.resize(cfg->max_inflight);
  // plan buffers for batched ticks: room for max_batch keyframes on the
  // largest fused grid of this device
  const size_t cap = (s->cfg.batching && s->cfg.max_batch > 1 && df::fused_supported())
                         ? df::fused_plan_bytes(s->cfg.max_batch, df::fused_max_ctas())
                         : 0;
  for (Launch &L : s->launches) {
    cudaError_t e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
    if (e == cudaSuccess && cap > 0) {
      e = cudaMalloc(&L.dplan, cap);
      if (e == cudaSuccess) e = cudaMallocHost(&L.hplan, cap);
      if (e == cudaSuccess) L.plan_cap = cap;
    }
    if (e != cudaSuccess) {
      df_server_destroy(s);
      return df::report(DF_ECUDA, "server streams: %s", cudaGetErrorString(e));
    }
  }
  *out = s;
  return DF_OK;
}

void df_server_destroy(df_server *s) {
  if (!s) return;
  for (Launch &L : s->launches) {
    if (L.stream) cudaStreamSynchronize(L.stream);
  }
  for (StreamState &st : s->streams) df_keyframe_destroy(st.kf);
  for (Launch &L : s->launches) {
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
    if (L.dplan) cudaFree(L.dplan);
    if (L.hplan) cudaFreeHost(L.hplan);
  }
  delete s;
}

df_status df_server_open_stream(df_server *s, const df_keyframe_desc *desc, const void *mu_net,
                                const void *var_net, const void *gx, const void *var_gx,
                                const void *gy, const void *var_gy, int ptrs_on_device,
                                int32_t *stream_id) {
  if (!s || !desc || !stream_id) return df::report(DF_EINVAL, "NULL argument");
  const size_t need = df_keyframe_bytes(desc->width, desc->height, desc->cnn_dtype);
  if (need == 0) return df::report(DF_EINVAL, "bad keyframe size or dtype");
  if (s->cfg.memory_budget && s->used + need > s->cfg.memory_budget)
    return df::report(DF_EBUDGET, "stream needs %zu bytes, %zu of %zu in use", need, s->used,
                      s->cfg.memory_budget);
  df_keyframe *kf = nullptr;
  df_status st = df_keyframe_create(desc, mu_net, var_net, gx, var_gx, gy, var_gy,
                                    ptrs_on_device, s->launches[0].stream, &kf);
  if (st != DF_OK) return st;
  cudaStreamSynchronize(s->launches[0].stream);
  int32_t id = -1;
  for (size_t i = 0; i < s->streams.size(); ++i) {
    if (!s->streams[i].kf) {
      id = (int32_t)i;
      break;
    }
  }
  if (id < 0) {
    id = (int32_t)s->streams.size();
    s->streams.emplace_back();
  }
  StreamState &ss = s->streams[id];
  ss.kf = kf;
  ss.bytes = need;
  ss.busy = false;
  ss.queue.clear();
  s->used += need;
  *stream_id = id;
  return DF_OK;
}

df_status df_server_close_stream(df_server *s, int32_t sid) {
  if (!s || sid < 0 || sid >= (int32_t)s->streams.size() || !s->streams[sid].kf)
    return df::report(DF_EINVAL, "no such stream");
  StreamState &ss = s->streams[sid];
  // finish its frames first: drive the scheduler until none is left
  while (!ss.queue.empty() || ss.busy) {
    int32_t n = 0;
    df_status st = df_server_progress(s, nullptr, 0, &n);
    if (st != DF_OK) return st;
  }
  df_keyframe_destroy(ss.kf);
  ss.kf = nullptr;
  s->used -= ss.bytes;
  ss.bytes = 0;
  return DF_OK;
}

df_status df_server_submit(df_server *s, int32_t sid, const float *mu_semi, const float *var_semi,
                           int ptrs_on_device, uint64_t tag) {
  if (!s || sid < 0 || sid >= (int32_t)s->streams.size() || !s->streams[sid].kf)
    return df::report(DF_EINVAL, "no such stream");
  if (!mu_semi || !var_semi) return df::report(DF_EINVAL, "semi-dense plane is NULL");
  Req r{sid, mu_semi, var_semi, ptrs_on_device, tag, now_ns()};
  s->streams[sid].queue.push_back(r);
  if (!s->cfg.batching) s->arrivals.push_back(r);
  ++s->pending;
  return DF_OK;
}

df_status df_server_progress(df_server *s, df_completion *out, int32_t cap, int32_t *n_out) {
  if (!s || !n_out) return df::report(DF_EINVAL, "NULL argument");
  *n_out = 0;
  int cur = 0;
  if (cudaGetDevice(&cur) == cudaSuccess && cur != s->device) cudaSetDevice(s->device);
  retire(s);
  for (Launch &L : s->launches) {
    if (L.active) continue;
    bool started = false;
    df_status st = start_one(s, L, &started);
    if (st != DF_OK) return st;
    if (!started) break;
  }
  int32_t n = 0;
  while (out && !s->done.empty() && n < cap) {  // undelivered completions wait for the next call
    out[n++] = s->done.front();
    s->done.pop_front();
    --s->pending;
  }
  *n_out = n;
  return DF_OK;
}

int32_t df_server_pending(const df_server *s) { return s ? s->pending : 0; }

df_status df_server_fetch_depth(df_server *s, int32_t sid, float *out, int log_space,
                                int ptr_on_device) {
  if (!s || sid < 0 || sid >= (int32_t)s->streams.size() || !s->streams[sid].kf)
    return df::report(DF_EINVAL, "no such stream");
  for (Launch &L : s->launches) cudaStreamSynchronize(L.stream);
  df_status st = df_fetch_depth(s->streams[sid].kf, out, log_space, ptr_on_device,
                                s->launches[0].stream);
  if (st != DF_OK) return st;
  cudaError_t e = cudaStreamSynchronize(s->launches[0].stream);
  if (e != cudaSuccess) return df::report(DF_ECUDA, "fetch: %s", cudaGetErrorString(e));
  return DF_OK;
}

df_status df_server_get_state(df_server *s, int32_t sid, float *x_out, double *t_out,
                              int ptrs_on_device) {
  if (!s || sid < 0 || sid >= (int32_t)s->streams.size() || !s->streams[sid].kf)
    return df::report(DF_EINVAL, "no such stream");
  for (Launch &L : s->launches) cudaStreamSynchronize(L.stream);
  df_status st = df_keyframe_get_state(s->streams[sid].kf, x_out, t_out, ptrs_on_device,
                                       s->launches[0].stream);
  if (st != DF_OK) return st;
  cudaError_t e = cudaStreamSynchronize(s->launches[0].stream);
  if (e != cudaSuccess) return df::report(DF_ECUDA, "get state: %s", cudaGetErrorString(e));
  return DF_OK;
}

}  // extern "C"
