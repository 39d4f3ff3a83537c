// api.cu -- status handling, argument conversion and small entry points of libags.
#include <cmath>
#include <cstring>

#include "ags_internal.cuh"

namespace ags {

ags_status launch_status(cudaError_t e) { return e == cudaSuccess ? AGS_OK : AGS_ERR_CUDA; }

ags_status build_cams(const ags_camera* cams, int32_t views, CamBatch* out) {
  if (!cams || views < 1 || views > AGS_MAX_VIEWS) return AGS_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  for (int v = 0; v < views; v++) {
    const ags_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width != cams[0].width || c.height != cams[0].height)
      return AGS_ERR_INVALID_ARG;
    if (c.width > 65535 * AGS_TILE || c.height > 65535 * AGS_TILE) return AGS_ERR_INVALID_ARG;
    if (!(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.cx) || !std::isfinite(c.cy) || !(c.near_z > 0.f))
      return AGS_ERR_INVALID_ARG;
    for (int k = 0; k < 12; k++)
      if (!std::isfinite(c.viewmat[k])) return AGS_ERR_INVALID_ARG;
    DevCam& d = out->c[v];
    for (int r = 0; r < 3; r++) {
      for (int k = 0; k < 3; k++) d.R[r * 3 + k] = c.viewmat[r * 4 + k];
      d.t[r] = c.viewmat[r * 4 + 3];
      d.campos[r] = c.campos[r];
    }
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy; d.near_z = c.near_z;
    d.limx = 1.3f * (0.5f * (float)c.width / c.fx);
    d.limy = 1.3f * (0.5f * (float)c.height / c.fy);
    d.W = c.width; d.H = c.height;
    d.gx = (c.width + AGS_TILE - 1) / AGS_TILE;
    d.gy = (c.height + AGS_TILE - 1) / AGS_TILE;
  }
  return AGS_OK;
}

ags_status build_params(const ags_params* p, DevParams* out) {
  if (!p) return AGS_ERR_INVALID_ARG;
  if (p->scale_mode != AGS_SCALE_PLAIN && p->scale_mode != AGS_SCALE_ADAGSCALE) return AGS_ERR_INVALID_ARG;
  if (p->sh_degree < 0 || p->sh_degree > 3) return AGS_ERR_INVALID_ARG;
  if (p->lut_bins < 1 || p->lut_bins > AGS_MAX_LUT_BINS) return AGS_ERR_INVALID_ARG;
  if (p->tile_test != AGS_TILE_SQUARE && p->tile_test != AGS_TILE_ELLIPSE) return AGS_ERR_INVALID_ARG;
  if (p->blend_flags & ~(AGS_BLEND_ROWS2 | AGS_BLEND_BATCH64)) return AGS_ERR_INVALID_ARG;
  if (!(p->K >= 0.f) || !std::isfinite(p->K)) return AGS_ERR_INVALID_ARG;
  if (!(p->tau > 0.f) || !(p->t_min >= 0.f) || !(p->alpha_max > 0.f) || !(p->lut_depth_max > 0.f))
    return AGS_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->scale_mode = p->scale_mode;
  out->sh_degree = p->sh_degree;
  out->lut_bins = p->lut_bins;
  out->tile_test = p->tile_test;
  out->blend_flags = p->blend_flags;
  out->K = p->K; out->tau = p->tau; out->t_min = p->t_min; out->alpha_max = p->alpha_max;
  out->lut_scale = (float)p->lut_bins / p->lut_depth_max;
  for (int i = 0; i < AGS_MAX_LUT_BINS; i++) out->lut[i] = p->lut[i];
  for (int i = 0; i < 3; i++) out->bg[i] = p->bg[i];
  return AGS_OK;
}

}  // namespace ags

extern "C" {

ags_status ags_status_reset(int64_t* d_status, void* stream) {
  if (!d_status) return AGS_ERR_INVALID_ARG;
  return ags::launch_status(cudaMemsetAsync(d_status, 0, 4 * sizeof(int64_t), (cudaStream_t)stream));
}

ags_status ags_check(const int64_t* d_status, void* stream, int64_t* detail) {
  if (!d_status) return AGS_ERR_INVALID_ARG;
  int64_t h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(h, d_status, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  if (h[0] == 0 && h[2] != 0) {
    if (detail) *detail = h[2];
    return AGS_ERR_NUMERIC;
  }
  if (detail) *detail = h[1];
  return (ags_status)h[0];
}

const char* ags_status_string(ags_status s) {
  switch (s) {
    case AGS_OK: return "ok";
    case AGS_ERR_INVALID_ARG: return "invalid argument";
    case AGS_ERR_CAPACITY: return "pair capacity exceeded";
    case AGS_ERR_TIMEOUT: return "bounded device wait timed out";
    case AGS_ERR_CUDA: return "CUDA error";
    case AGS_ERR_NUMERIC: return "non-finite Gaussian parameters culled";
    case AGS_ERR_BOUNDS: return "index out of range (debug build check)";
  }
  return "unknown status";
}

#ifdef AGS_DEBUG
const char* ags_version(void) { return "ags 0.1 (sm_103a, AGS_DEBUG index checks)"; }
#else
const char* ags_version(void) { return "ags 0.1 (sm_103a)"; }
#endif

}  // extern "C"
