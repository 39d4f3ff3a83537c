// raster.cu -- per-tile front-to-back alpha blending (Eq. 1, Eq. 2) and the
// T_up calibration table (Sec. 3.4).
//
// One 256-thread CTA per 16x16 tile of each view, one pixel per thread.  The
// tile's depth-ordered pairs are staged in batches of 256: each thread gathers
// one splat record (two 16-byte loads and one 4-byte load from the 48-byte
// record) into shared memory, then every thread walks the batch for its pixel.
// The CTA stops as soon as every pixel has reached the transmittance floor
// (__syncthreads_count vote).  The blend always uses the conic of the original
// covariance and tau (Sec. 3.3 "dual-size strategy"): the scale mode only ever
// changed which pairs exist.
#include <algorithm>

#include "blend.cuh"

namespace ags {

__global__ void __launch_bounds__(kRasterThreads)
raster_kernel(const float4* __restrict__ splat, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
              int W, int H, int gx, int tiles_per_view, BlendConst bc, float* __restrict__ image,
              float* __restrict__ final_T, uint32_t* __restrict__ n_contrib, uint32_t* __restrict__ max_T_bits,
              unsigned long long* stats) {
  __shared__ float4 s_a[kRasterThreads];   // u v A B
  __shared__ float4 s_b[kRasterThreads];   // C opacity r g
  __shared__ float s_c[kRasterThreads];    // b
  __shared__ uint32_t s_e[kRasterThreads]; // splat index (calibration only)

  const int tile = blockIdx.x;
  const int view = tile / tiles_per_view;
  const int lt = tile - view * tiles_per_view;
  const int ty = lt / gx, tx = lt - ty * gx;
  const int tid = threadIdx.x, lane = tid & 31;
  const int px = tx * kTile + (tid & (kTile - 1));
  const int py = ty * kTile + (tid >> 4);
  const bool inside = px < W && py < H;
  const float fpx = (float)px, fpy = (float)py;
  const uint2 rg = __ldg(ranges + tile);
  const uint32_t start = rg.x, end = rg.y;

  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
  bool done = !inside;
  uint32_t last = 0, evals = 0, blends = 0;

  for (uint32_t b0 = start; b0 < end; b0 += kRasterThreads) {
    if (__syncthreads_count(done) == kRasterThreads) break;
    uint32_t idx = b0 + tid;
    if (idx < end) {
      uint32_t e = __ldg(vals + idx);
      const float4* rec = splat + (size_t)e * 3;
      s_a[tid] = __ldg(rec);
      s_b[tid] = __ldg(rec + 1);
      s_c[tid] = __ldg(reinterpret_cast<const float*>(rec + 2));
      s_e[tid] = e;
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)kRasterThreads, end - b0);
    for (int j = 0; j < nb; j++) {
      const float4 a = s_a[j];
      const float4 bq = s_b[j];
      bool blend = false;
      float Tbefore = T;
      if (!done) {
        evals++;
        float dx, dy;
        float power = splat_power(a.x, a.y, a.z, a.w, bq.x, fpx, fpy, dx, dy);
        if (power <= 0.f) {
          float alpha = fminf(bc.alpha_max, splat_alpha_raw(bq.y, power));
          if (alpha >= bc.tau) {
            float test_T = __fmul_rn(T, __fsub_rn(1.f, alpha));
            if (test_T < bc.t_min) {
              done = true;
            } else {
              float w = __fmul_rn(alpha, T);
              cr = __fmaf_rn(bq.z, w, cr);
              cg = __fmaf_rn(bq.w, w, cg);
              cb = __fmaf_rn(s_c[j], w, cb);
              T = test_T;
              last = b0 - start + j + 1;
              blend = true;
              blends++;
            }
          }
        }
      }
      if (max_T_bits) {   // calibration: per-Gaussian max T before blending (warp max, one atomic)
        uint32_t m = __reduce_max_sync(0xffffffffu, blend ? __float_as_uint(Tbefore) : 0u);
        if (lane == 0 && m) atomicMax(max_T_bits + s_e[j], m);
      }
    }
  }
  if (inside) {
    const size_t hw = (size_t)W * H;
    const size_t o = (size_t)view * 3 * hw + (size_t)py * W + px;
    image[o] = cr + T * bc.bg[0];
    image[o + hw] = cg + T * bc.bg[1];
    image[o + 2 * hw] = cb + T * bc.bg[2];
    const size_t op = (size_t)view * hw + (size_t)py * W + px;
    if (final_T) final_T[op] = T;
    if (n_contrib) n_contrib[op] = last;
  }
  if (stats) {
    unsigned long long e1 = warp_sum((unsigned long long)evals), e2 = warp_sum((unsigned long long)blends);
    if (lane == 0) {
      atomicAdd(stats, e1);
      atomicAdd(stats + 1, e2);
    }
  }
}

__global__ void lut_kernel(const float* __restrict__ max_T, const float* __restrict__ depth, int64_t count, int bins,
                           float scale, uint32_t* lut_bits) {
  __shared__ uint32_t h[AGS_MAX_LUT_BINS];
  if (threadIdx.x < AGS_MAX_LUT_BINS) h[threadIdx.x] = 0u;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    float t = max_T[i];
    if (t > 0.f) {
      int b = (int)fminf(fmaxf(depth[i], 0.f) * scale, (float)(bins - 1));
      atomicMax(&h[b], __float_as_uint(t));
    }
  }
  __syncthreads();
  if (threadIdx.x < bins && h[threadIdx.x]) atomicMax(lut_bits + threadIdx.x, h[threadIdx.x]);
}

__global__ void lut_finish_kernel(uint32_t* lut_bits, int bins) {
  int b = threadIdx.x;
  if (b < bins && lut_bits[b] == 0u) lut_bits[b] = __float_as_uint(1.0f);
}

}  // namespace ags

extern "C" ags_status ags_rasterize(const ags_projected* proj, int64_t n, const uint32_t* sorted_vals,
                                    const uint32_t* ranges, const ags_camera* cams, int32_t views,
                                    const ags_params* params, float* image, float* final_T, uint32_t* n_contrib,
                                    float* max_T, uint64_t* stats, int64_t* d_status, void* stream) {
  using namespace ags;
  if (!proj || !ranges || !image || !d_status || n < 0) return AGS_ERR_INVALID_ARG;
  CamBatch cb;
  DevParams dp;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  s = build_params(params, &dp);
  if (s != AGS_OK) return s;
  if (n > 0 && (!proj->splat || !sorted_vals)) return AGS_ERR_INVALID_ARG;
  if ((uintptr_t)proj->splat & 15u) return AGS_ERR_INVALID_ARG;
  const int tiles_per_view = cb.c[0].gx * cb.c[0].gy;
  BlendConst bc{dp.tau, dp.t_min, dp.alpha_max, {dp.bg[0], dp.bg[1], dp.bg[2]}};
  raster_kernel<<<(unsigned)(tiles_per_view * views), kRasterThreads, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const float4*>(proj->splat), sorted_vals, reinterpret_cast<const uint2*>(ranges),
      cb.c[0].W, cb.c[0].H, cb.c[0].gx, tiles_per_view, bc, image, final_T, n_contrib,
      reinterpret_cast<uint32_t*>(max_T), reinterpret_cast<unsigned long long*>(stats));
  return launch_status(cudaGetLastError());
}

extern "C" ags_status ags_calibrate_lut(const float* max_T, const float* depth, int64_t count, int32_t lut_bins,
                                        float lut_depth_max, float* lut_out, void* stream) {
  using namespace ags;
  if (!lut_out || count < 0 || lut_bins < 1 || lut_bins > AGS_MAX_LUT_BINS || !(lut_depth_max > 0.f))
    return AGS_ERR_INVALID_ARG;
  if (count > 0 && (!max_T || !depth)) return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* bits = reinterpret_cast<uint32_t*>(lut_out);
  cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)lut_bins * 4, st);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  if (count > 0) {
    int blocks = (int)std::min<int64_t>((count + 255) / 256, 1024);
    lut_kernel<<<blocks, 256, 0, st>>>(max_T, depth, count, lut_bins, (float)lut_bins / lut_depth_max, bits);
  }
  lut_finish_kernel<<<1, AGS_MAX_LUT_BINS, 0, st>>>(bits, lut_bins);
  return launch_status(cudaGetLastError());
}
