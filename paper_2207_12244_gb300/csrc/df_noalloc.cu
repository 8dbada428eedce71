// df_optimise_noalloc: the per-frame solve for callers that cannot allocate
// device memory (see include/deepfusion.h). The solver's scratch lives in one
// file-scope device array that every GPU loading the library holds until the
// process exits; the caller passes only its inputs and outputs.
#include <mutex>

#include "df_internal.cuh"

namespace df {
namespace {

constexpr size_t kNoallocPixels = DF_NOALLOC_MAX_PIXELS;
constexpr int kNoallocPlanes = 7;  // diag, wx, wy and four solver vectors

struct NoallocScratch {
  Scalars sc;
  double partial[kMaxPartialBlocks * kNumQ];
  float planes[kNoallocPlanes][kNoallocPixels];
};

// Device scratch shared by every call on a device. In host code this name is
// only a stand-in: its device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

std::mutex g_mu;
void *g_addr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
df_status scratch_address(NoallocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(DF_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return report(DF_ENOTSUP, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return report(DF_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = static_cast<NoallocScratch *>(g_addr[dev]);
  return DF_OK;
}

}  // namespace
}  // namespace df

extern "C" df_status df_optimise_noalloc(int32_t width, int32_t height, const float *mu_net,
                                         const float *var_net, const float *gx,
                                         const float *var_gx, const float *gy,
                                         const float *var_gy, const float *mu_semi,
                                         const float *var_semi, float *x_inout,
                                         double *scale_log_inout, const df_solve_params *params,
                                         void *stream) {
  using namespace df;
  if (width < 1 || height < 1) return report(DF_EINVAL, "width and height must be >= 1");
  if ((int64_t)width * height > (int64_t)kNoallocPixels)
    return report(DF_EINVAL, "%d x %d pixels exceed the no-allocation limit of %d pixels",
                  width, height, (int)kNoallocPixels);
  if (!mu_net || !var_net || !gx || !var_gx || !gy || !var_gy || !x_inout || !scale_log_inout)
    return report(DF_EINVAL, "NULL input or output pointer");
  if ((mu_semi == nullptr) != (var_semi == nullptr))
    return report(DF_EINVAL, "mu_semi and var_semi must both be given or both be NULL");
  df_solve_params p;
  if (params) {
    p = *params;
  } else {
    df_default_params(&p);
  }
  df_status st = check_solve_params(&p);
  if (st != DF_OK) return st;
  if (!mu_semi) p.terms &= ~DF_TERM_SEMI;
  if (p.scale_step == DF_SCALE_JOINT) {
    if (p.terms & DF_TERM_SEMI)
      return report(DF_ENOTSUP, "df_optimise_noalloc has no scratch plane for DF_SCALE_JOINT");
    // without the semi-dense term the joint system's border row is empty and
    // t stays where it is: the depth step with t fixed is that solve
    p.scale_step = DF_SCALE_FIXED;
  }
  if ((p.terms & (DF_TERM_NET | DF_TERM_GRAD)) == 0)
    return report(DF_EINVAL, "terms must include NET or GRAD");
  NoallocScratch *scr = nullptr;
  st = scratch_address(&scr);
  if (st != DF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Planes k = {};
  k.W = width;
  k.H = height;
  k.P = width;  // the caller's planes are dense; the launch kernels take any pitch
  k.dtype = DF_F32;
  const float *cnn[6] = {mu_net, var_net, gx, var_gx, gy, var_gy};
  for (int j = 0; j < 6; ++j) k.cnn[j] = cnn[j];
  k.mu_s = mu_semi ? mu_semi : mu_net;  // not read when the semi-dense term is off
  k.var_s = var_semi ? var_semi : var_net;
  k.x = x_inout;
  k.diag = scr->planes[0];
  k.wx = scr->planes[1];
  k.wy = scr->planes[2];
  for (int j = 0; j < 4; ++j) k.v[j] = scr->planes[3 + j];
  k.sc = &scr->sc;
  k.partial = scr->partial;
  // the scalars (reduction counter, flags, CG state) must start at zero; the
  // planes and partial sums are fully written before they are read
  cudaError_t e = cudaMemsetAsync(&scr->sc, 0, sizeof(Scalars), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&scr->sc.t, scale_log_inout, sizeof(double), cudaMemcpyDeviceToDevice, s);
  df_solve_params ph[2];
  const int nph = split_schedule(p, ph);  // the Huber warm start, then the rest
  for (int j = 0; j < nph && e == cudaSuccess; ++j) {
    if (j > 0) e = cudaMemsetAsync(&scr->sc.stop, 0, sizeof(scr->sc.stop), s);
    if (e == cudaSuccess) e = launch_solve_launches(k, solve_cfg(&ph[j]), ph[j].n_gn, ph[j].n_pcg, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(scale_log_inout, &scr->sc.t, sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return report(DF_ECUDA, "df_optimise_noalloc: %s", cudaGetErrorString(e));
  return DF_OK;
}
