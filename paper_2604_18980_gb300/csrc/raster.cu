// raster.cu -- per-tile front-to-back alpha blending (Eq. 1, Eq. 2) and the
// T_up calibration table (Sec. 3.4).
//
// One 128-thread CTA per 16x16 tile of each view, two pixels per thread (each
// warp an 8x8 pixel block).  The tile's depth-ordered pairs are staged in
// batches of 128: each thread gathers one 48-byte splat record, converts it
// to the log2 form of Eq. 1 and computes the mask of warp blocks its
// alpha >= tau ellipse can reach; each warp then compacts the batch to the
// splats that reach its block and walks that list.  A warp leaves the batch
// once all its pixels reached the transmittance floor, the CTA once all warps
// did (__syncthreads_count vote).  The blend always uses the conic of the original
// covariance and tau (Sec. 3.3 "dual-size strategy"): the scale mode only ever
// changed which pairs exist.
#include <algorithm>

#include "blend.cuh"

namespace ags {

// 128 threads per tile, four warps of 8x8 pixels; lane l blends the two
// pixels (8*(w&1) + (l&7), 8*(w>>1) + (l>>3)) and the one 4 rows below, which
// share dx.  kStats: count evaluations and blends; kMaxT: calibration output;
// kState: track each pixel's last blended position (n_contrib, for the
// backward).  The benchmark's kernel is the <false, false, false> instance.
constexpr int kBlendThreads = 128;
constexpr int kBlendWarps = kBlendThreads / 32;

// One pixel's step over one splat, without branches: the accept test, the
// stop test T (1 - alpha) < t_min and the blend are predicates, and a pixel
// that does not blend adds exact zeros.  Returns whether it blended.
__device__ __forceinline__ bool blend_pixel(const Staged& s, float cb, float P, float Bx, float dy,
                                            const BlendConst& bc, bool& done, float& T, float& r, float& g,
                                            float& b) {
  const float q = splat_qy(s, P, Bx, dy);
  const bool ok = !done && splat_accept(q, s.b.y);
  const float alpha = fminf(bc.alpha_max, __fmul_rn(bc.tau, fast_exp2(q)));
  const float test_T = __fmul_rn(T, __fsub_rn(1.f, alpha));
  const bool stop = ok && test_T < bc.t_min;
  const bool blend = ok && !stop;
  done = done || stop;
  const float w = blend ? __fmul_rn(alpha, T) : 0.f;
  r = __fmaf_rn(s.b.z, w, r);
  g = __fmaf_rn(s.b.w, w, g);
  b = __fmaf_rn(cb, w, b);
  T = blend ? test_T : T;
  return blend;
}

template <bool kStats, bool kMaxT, bool kState>
__global__ void __launch_bounds__(kBlendThreads, kState ? 8 : 9)
raster_kernel(const float4* __restrict__ splat, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
              int W, int H, int gx, int tiles_per_view, BlendConst bc, float* __restrict__ image,
              float* __restrict__ final_T, uint32_t* __restrict__ n_contrib, uint32_t* __restrict__ max_T_bits,
              unsigned long long* stats) {
  constexpr int kB = kBlendThreads;                    // splats staged per batch
  constexpr int kPad = kB;                             // index of an always-rejected entry
  __shared__ float4 s_a[kB + 1];                       // u v a2 b2
  __shared__ float4 s_b[kB + 1];                       // c2 base r g
  __shared__ float s_c[kB + 1];                        // b
  __shared__ uint32_t s_m[kB];                         // 8x8 block mask
  __shared__ uint32_t s_e[kB + 1];                     // splat index (calibration only)
  __shared__ uint16_t s_list[kBlendWarps][kB + 4];     // per-warp entries, padded

  const int tile = blockIdx.x;
  const int view = tile / tiles_per_view;
  const int lt = tile - view * tiles_per_view;
  const int ty = lt / gx, tx = lt - ty * gx;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int px = tx * kTile + 8 * (warp & 1) + (lane & 7);
  const int py0 = ty * kTile + 8 * (warp >> 1) + (lane >> 3);
  const int py1 = py0 + 4;
  const bool in0 = px < W && py0 < H, in1 = px < W && py1 < H;
  const float fpx = (float)px, fpy0 = (float)py0, fpy1 = (float)py1;
  const uint2 rg = __ldg(ranges + tile);
  const uint32_t start = rg.x, end = rg.y;
  if (tid == 0) {   // the pad entry: far away and steep, q = -inf rejects every pixel
    s_a[kPad] = make_float4(1e30f, 1e30f, -1.f, 0.f);
    s_b[kPad] = make_float4(-1.f, -1.f, 0.f, 0.f);
    s_c[kPad] = 0.f;
    s_e[kPad] = 0u;
  }

  float T0 = 1.f, r0 = 0.f, g0 = 0.f, b0c = 0.f;
  float T1 = 1.f, r1 = 0.f, g1 = 0.f, b1c = 0.f;
  bool done0 = !in0, done1 = !in1;
  uint32_t last0 = 0, last1 = 0, evals = 0, blends = 0;

  for (uint32_t bb = start; bb < end; bb += kB) {
    if (__syncthreads_count(done0 && done1) == kBlendThreads) break;
    const uint32_t idx = bb + tid;
    if (idx < end) {
      const uint32_t e = __ldg(vals + idx);
      Staged st;
      uint32_t m;
      stage_splat<8, 8>(splat + (size_t)e * 3, tx * kTile, ty * kTile, bc.l2tau, st, m);
      s_a[tid] = st.a;
      s_b[tid] = st.b;
      s_c[tid] = st.c;
      s_m[tid] = m;
      if (kMaxT) s_e[tid] = e;
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)kB, end - bb);
    // this warp's entries of the batch, in depth order, padded to a multiple of 4
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kB / 32; k++) {
      const int j = k * 32 + lane;
      const bool hit = j < nb && ((s_m[j] >> warp) & 1u);
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) s_list[warp][cnt + __popc(bal & lanemask_lt())] = (uint16_t)j;
      cnt += __popc(bal);
    }
    if (lane < 4) s_list[warp][cnt + lane] = (uint16_t)kPad;
    __syncwarp();
    if (__all_sync(0xffffffffu, done0 && done1)) continue;
    for (int t = 0; t < cnt; t += 4) {
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int j = s_list[warp][t + u];
        Staged s;
        s.a = s_a[j];
        s.b = s_b[j];
        const float dx = __fsub_rn(s.a.x, fpx);
        float P, Bx;
        splat_qx(s, dx, P, Bx);
        const float cb = s_c[j];
        const float Tb0 = T0, Tb1 = T1;
        if (kStats) evals += (j != kPad) * ((done0 ? 0u : 1u) + (done1 ? 0u : 1u));
        const bool bl0 = blend_pixel(s, cb, P, Bx, __fsub_rn(s.a.y, fpy0), bc, done0, T0, r0, g0, b0c);
        const bool bl1 = blend_pixel(s, cb, P, Bx, __fsub_rn(s.a.y, fpy1), bc, done1, T1, r1, g1, b1c);
        if (kStats) blends += (bl0 ? 1u : 0u) + (bl1 ? 1u : 0u);
        if (kState) {
          const uint32_t pos1 = bb - start + j + 1;
          last0 = bl0 ? pos1 : last0;
          last1 = bl1 ? pos1 : last1;
        }
        if (kMaxT) {   // calibration: per-Gaussian max T before blending (warp max, one atomic)
          const uint32_t mine = max(bl0 ? __float_as_uint(Tb0) : 0u, bl1 ? __float_as_uint(Tb1) : 0u);
          const uint32_t m = __reduce_max_sync(0xffffffffu, mine);
          if (lane == 0 && m) atomicMax(max_T_bits + s_e[j], m);
        }
      }
      if (__all_sync(0xffffffffu, done0 && done1)) break;
    }
  }
  const size_t hw = (size_t)W * H;
  if (in0) {
    const size_t o = (size_t)view * 3 * hw + (size_t)py0 * W + px;
    image[o] = r0 + T0 * bc.bg[0];
    image[o + hw] = g0 + T0 * bc.bg[1];
    image[o + 2 * hw] = b0c + T0 * bc.bg[2];
    const size_t op = (size_t)view * hw + (size_t)py0 * W + px;
    if (final_T) final_T[op] = T0;
    if (kState) n_contrib[op] = last0;
  }
  if (in1) {
    const size_t o = (size_t)view * 3 * hw + (size_t)py1 * W + px;
    image[o] = r1 + T1 * bc.bg[0];
    image[o + hw] = g1 + T1 * bc.bg[1];
    image[o + 2 * hw] = b1c + T1 * bc.bg[2];
    const size_t op = (size_t)view * hw + (size_t)py1 * W + px;
    if (final_T) final_T[op] = T1;
    if (kState) n_contrib[op] = last1;
  }
  if (kStats) {
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
  BlendConst bc = make_blend_const(dp);
  auto kern = n_contrib ? (stats ? (max_T ? raster_kernel<true, true, true> : raster_kernel<true, false, true>)
                                 : (max_T ? raster_kernel<false, true, true> : raster_kernel<false, false, true>))
                       : (stats ? (max_T ? raster_kernel<true, true, false> : raster_kernel<true, false, false>)
                                : (max_T ? raster_kernel<false, true, false> : raster_kernel<false, false, false>));
  kern<<<(unsigned)(tiles_per_view * views), kBlendThreads, 0, (cudaStream_t)stream>>>(
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
