// diag.cu -- peripheral-score diagnostics (Sec. 2.2 Eq. 3 and Fig. 4a, Sec. 3.1
// Eq. 4, Sec. 3.2 Eq. 6-9 and Fig. 5).
//
// Three replays of the plain blend of a pair list, with the blend's own
// per-pixel decisions (the same log2-form alpha, accept test and transmittance
// stop as raster_kernel, so the set of blends is bit-identical to the image's):
//
//   scores   the exact peripheral score of every Gaussian-view at its
//            AdaGScale level Th (Eq. 4 with x = Th of Eq. 10), the max T
//            statistic of Eq. 6 and the pixel sum of alpha; a finishing pass
//            forms Eq. 6, Eq. 7 and Eq. 9 from them;
//   hist     a histogram of the contribution of every blend under one ranking
//            (alpha T of Eq. 3, max T alpha of Eq. 6, T_up(depth) alpha of Eq. 7);
//   skip     the image with every blend whose contribution is below a
//            threshold skipped (no colour, no occlusion), the unskipped T still
//            ranking and stopping as in the plain blend.
//
// One 128-thread CTA per tile as in raster_kernel (two pixels per thread, four
// 8x8 warp blocks, batches of 128 staged splats compacted per warp by the
// alpha >= tau block mask).  Per-Gaussian sums are reduced over the warp
// before one atomic per (warp, splat).
#include "blend.cuh"

namespace ags {

enum DiagMode { kDiagScores = 0, kDiagHist = 1, kDiagSkip = 2 };

constexpr int kDiagThreads = 128;
constexpr int kDiagWarps = kDiagThreads / 32;
constexpr int kScoreRows = 7;
constexpr int kHistBins = AGS_CONTRIB_HIST_BINS;   // contribution bits >> 16 (positive floats order as their bits)

struct DiagArgs {
  const float* depth;
  const uint8_t* flags;
  const float* max_T;        // rule 1 weights (nullable otherwise)
  float* scores;             // [7][count] (scores mode)
  uint32_t* hist;            // [kHistBins] (hist mode)
  unsigned long long* counts;   // [2] blends, skipped (skip mode)
  float* image;              // [views][3][H][W] (skip mode)
  int64_t count;             // views * n
  int rule;
  float thr;
};

// T_up of a depth (Sec. 3.4), binned as the preprocess bins it.
__device__ __forceinline__ float lut_of_depth(const DevParams& P, float depth) {
  const int bin = (int)fminf(depth * P.lut_scale, (float)(P.lut_bins - 1));
  return P.lut[bin];
}

// Th of Eq. 10 from a splat record: det of the dilated covariance is
// Sigma_yy / A (the conic's A is Sigma_yy / det), so no cancellation.
__device__ __forceinline__ float splat_th(const DevParams& P, float4 r0, float4 r2, float depth, float& tup,
                                          float& sdet) {
  tup = lut_of_depth(P, depth);
  sdet = sqrtf(r2.w / r0.z);
  if (!(tup > 0.f)) return __int_as_float(0x7f800000);
  return P.K / (tup * 6.2831853f * sdet) + P.tau;
}

template <int kMode>
__global__ void __launch_bounds__(kDiagThreads)
diag_kernel(const float4* __restrict__ splat, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
            int W, int H, int gx, int tiles_per_view, BlendConst bc, const __grid_constant__ DevParams P,
            DiagArgs a) {
  constexpr int kB = kDiagThreads;
  constexpr int kPad = kB;
  __shared__ float4 s_a[kB + 1];
  __shared__ float4 s_b[kB + 1];
  __shared__ float s_c[kB + 1];
  __shared__ float s_x[kB + 1];                        // level Th (scores) or ranking weight
  __shared__ uint32_t s_m[kB];
  __shared__ uint32_t s_e[kB + 1];
  __shared__ uint16_t s_list[kDiagWarps][kB + 4];

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
  if (tid == 0) {
    s_a[kPad] = make_float4(1e30f, 1e30f, -1.f, 0.f);
    s_b[kPad] = make_float4(-1.f, -1e30f, 0.f, 0.f);
    s_c[kPad] = 0.f;
    s_x[kPad] = 0.f;
    s_e[kPad] = 0u;
  }
  float T0 = 1.f, T1 = 1.f, S0 = 1.f, S1 = 1.f;          // plain and image transmittance
  float r0 = 0.f, g0 = 0.f, b0 = 0.f, r1 = 0.f, g1 = 0.f, b1 = 0.f;
  bool done0 = !in0, done1 = !in1;
  uint32_t nblend = 0, nskip = 0;

  for (uint32_t bb = start; bb < end; bb += kB) {
    if (__syncthreads_count(done0 && done1) == kDiagThreads) break;
    const uint32_t idx = bb + tid;
    if (idx < end) {
      const uint32_t e = __ldg(vals + idx);
      Staged st;
      uint32_t m;
      const float4* rec = splat + (size_t)e * 3;
      stage_splat<8, 8>(rec, tx * kTile, ty * kTile, bc.l2tau, st, m);
      s_a[tid] = st.a;
      s_b[tid] = st.b;
      s_c[tid] = st.c;
      s_m[tid] = m;
      s_e[tid] = e;
      float x = 0.f;
      if (kMode == kDiagScores) {
        float tup, sdet;
        x = splat_th(P, __ldg(rec), __ldg(rec + 2), __ldg(a.depth + e), tup, sdet);
      } else if (a.rule == 1) {
        x = __ldg(a.max_T + e);
      } else if (a.rule == 2) {
        x = lut_of_depth(P, __ldg(a.depth + e));
      }
      s_x[tid] = x;
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)kB, end - bb);
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kB / 32; k++) {
      const int j = k * 32 + lane;
      const bool hit = j < nb && ((s_m[j] >> warp) & 1u);
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) s_list[warp][cnt + __popc(bal & lanemask_lt())] = (uint16_t)j;
      cnt += __popc(bal);
    }
    __syncwarp();
    if (!__all_sync(0xffffffffu, done0 && done1)) {
      for (int t = 0; t < cnt; t++) {
        const int j = s_list[warp][t];
        Staged s;
        s.a = s_a[j];
        s.b = s_b[j];
        const float dx = __fsub_rn(s.a.x, fpx);
        float P0, Bx;
        splat_qx(s, dx, P0, Bx);
        const float cb = s_c[j], x = s_x[j];
        float al[2], Tb[2];
        bool bl[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
          bool& done = h ? done1 : done0;
          float& T = h ? T1 : T0;
          const float q = splat_qy(s, P0, Bx, __fsub_rn(s.a.y, h ? fpy1 : fpy0));
          const bool ok = !done && splat_accept(q, bc.l2tau);
          float raw;
          const float alpha = splat_alpha(q, bc.alpha_max, raw);
          const float test_T = transmit(alpha, T);
          const bool stop = ok && test_T < bc.t_min;
          const bool blend = ok && !stop;
          done = done || stop;
          al[h] = alpha;
          Tb[h] = T;
          bl[h] = blend;
          if (kMode == kDiagHist && blend) {
            const float c = a.rule == 0 ? __fmul_rn(alpha, T) : __fmul_rn(x, alpha);
            atomicAdd(a.hist + min(__float_as_uint(c) >> 16, (uint32_t)kHistBins - 1u), 1u);   // negative: last bin
          }
          if (kMode == kDiagSkip && blend) {
            const float c = a.rule == 0 ? __fmul_rn(alpha, T) : __fmul_rn(x, alpha);
            float& S = h ? S1 : S0;
            nblend++;
            if (c < a.thr) {
              nskip++;
            } else {
              const float w = __fmul_rn(alpha, S);
              float& rr = h ? r1 : r0;
              float& gg = h ? g1 : g0;
              float& bbc = h ? b1 : b0;
              rr = __fmaf_rn(s.b.z, w, rr);
              gg = __fmaf_rn(s.b.w, w, gg);
              bbc = __fmaf_rn(cb, w, bbc);
              S = transmit(alpha, S);
            }
          }
          T = blend ? test_T : T;
        }
        if (kMode == kDiagScores && __any_sync(0xffffffffu, bl[0] || bl[1])) {
          float ps = 0.f, sa = 0.f;
          uint32_t mt = 0u;
#pragma unroll
          for (int h = 0; h < 2; h++) {
            if (bl[h]) {
              if (al[h] < x) {
                ps += __fmul_rn(al[h], Tb[h]);
                sa += al[h];
              }
              mt = max(mt, __float_as_uint(Tb[h]));
            }
          }
          ps = warp_sum(ps);
          sa = warp_sum(sa);
          mt = __reduce_max_sync(0xffffffffu, mt);
          if (lane == 0) {
            const uint32_t e = s_e[j];
            if (ps > 0.f) atomicAdd(a.scores + 1 * a.count + e, ps);
            if (sa > 0.f) atomicAdd(a.scores + 6 * a.count + e, sa);
            atomicMax(reinterpret_cast<uint32_t*>(a.scores + 5 * a.count) + e, mt);
          }
        }
      }
    }
  }
  if (kMode == kDiagSkip) {
    const size_t hw = (size_t)W * H;
    if (in0) {
      const size_t o = (size_t)view * 3 * hw + (size_t)py0 * W + px;
      a.image[o] = r0 + S0 * bc.bg[0];
      a.image[o + hw] = g0 + S0 * bc.bg[1];
      a.image[o + 2 * hw] = b0 + S0 * bc.bg[2];
    }
    if (in1) {
      const size_t o = (size_t)view * 3 * hw + (size_t)py1 * W + px;
      a.image[o] = r1 + S1 * bc.bg[0];
      a.image[o + hw] = g1 + S1 * bc.bg[1];
      a.image[o + 2 * hw] = b1 + S1 * bc.bg[2];
    }
    const unsigned long long sb = warp_sum((unsigned long long)nblend), ss = warp_sum((unsigned long long)nskip);
    if (lane == 0) {
      atomicAdd(a.counts, sb);
      atomicAdd(a.counts + 1, ss);
    }
  }
}

// Rows 0 (Th), 2 (Eq. 6), 3 (Eq. 7) and 4 (Eq. 9) from the accumulated rows 1
// (Eq. 4), 5 (max T) and 6 (sum of alpha); culled Gaussian-views keep zeros.
__global__ void scores_finish_kernel(const float4* __restrict__ splat, const __grid_constant__ DevParams P,
                                     DiagArgs a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.count || (__ldg(a.flags + e) & kFlagCulled)) return;
  const float4* rec = splat + e * 3;
  const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2);
  float tup, sdet;
  const float th = splat_th(P, r0, r2, __ldg(a.depth + e), tup, sdet);
  const float mt = a.scores[5 * a.count + e], sa = a.scores[6 * a.count + e];
  a.scores[e] = th;
  a.scores[2 * a.count + e] = mt * sa;
  a.scores[3 * a.count + e] = tup * sa;
  a.scores[4 * a.count + e] = tup * 6.2831853f * sdet * (fminf(th, r1.y) - P.tau);
}

static ags_status diag_prepare(const ags_projected* proj, int64_t n, const uint32_t* sorted_vals,
                               const uint32_t* ranges, const ags_camera* cams, int32_t views,
                               const ags_params* params, CamBatch* cb, DevParams* dp) {
  if (!proj || !ranges || n < 0) return AGS_ERR_INVALID_ARG;
  if ((uintptr_t)ranges & 7u) return AGS_ERR_INVALID_ARG;       // read as 8-byte (start, end) pairs
  ags_status s = build_cams(cams, views, cb);
  if (s != AGS_OK) return s;
  s = build_params(params, dp);
  if (s != AGS_OK) return s;
  if ((int64_t)views * n >= ((int64_t)1 << 32)) return AGS_ERR_INVALID_ARG;
  if (n > 0 && (!proj->splat || !proj->depth || !proj->flags || !sorted_vals)) return AGS_ERR_INVALID_ARG;
  if ((uintptr_t)proj->splat & 15u) return AGS_ERR_INVALID_ARG;
  return AGS_OK;
}

template <int kMode>
static ags_status diag_launch(const ags_projected* proj, const uint32_t* sorted_vals, const uint32_t* ranges,
                              const CamBatch& cb, int views, const DevParams& dp, const DiagArgs& a,
                              cudaStream_t st) {
  const int tiles_per_view = cb.c[0].gx * cb.c[0].gy;
  diag_kernel<kMode><<<(unsigned)(tiles_per_view * views), kDiagThreads, 0, st>>>(
      reinterpret_cast<const float4*>(proj->splat), sorted_vals, reinterpret_cast<const uint2*>(ranges),
      cb.c[0].W, cb.c[0].H, cb.c[0].gx, tiles_per_view, make_blend_const(dp), dp, a);
  return launch_status(cudaGetLastError());
}

}  // namespace ags

extern "C" ags_status ags_peripheral_scores(const ags_projected* proj, int64_t n, const uint32_t* sorted_vals,
                                            const uint32_t* ranges, const ags_camera* cams, int32_t views,
                                            const ags_params* params, float* scores, void* stream) {
  using namespace ags;
  CamBatch cb;
  DevParams dp;
  ags_status s = diag_prepare(proj, n, sorted_vals, ranges, cams, views, params, &cb, &dp);
  if (s != AGS_OK) return s;
  if (!scores || ((uintptr_t)scores & 3u)) return AGS_ERR_INVALID_ARG;
  const int64_t count = n * (int64_t)views;
  cudaStream_t st = (cudaStream_t)stream;
  if (count == 0) return AGS_OK;
  if (cudaMemsetAsync(scores, 0, sizeof(float) * kScoreRows * (size_t)count, st) != cudaSuccess) return AGS_ERR_CUDA;
  DiagArgs a{proj->depth, proj->flags, nullptr, scores, nullptr, nullptr, nullptr, count, 0, 0.f};
  s = diag_launch<kDiagScores>(proj, sorted_vals, ranges, cb, views, dp, a, st);
  if (s != AGS_OK) return s;
  scores_finish_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const float4*>(proj->splat), dp, a);
  return launch_status(cudaGetLastError());
}

extern "C" ags_status ags_contribution_hist(const ags_projected* proj, int64_t n, const uint32_t* sorted_vals,
                                            const uint32_t* ranges, const ags_camera* cams, int32_t views,
                                            const ags_params* params, int32_t rule, const float* max_T,
                                            uint32_t* hist, void* stream) {
  using namespace ags;
  CamBatch cb;
  DevParams dp;
  ags_status s = diag_prepare(proj, n, sorted_vals, ranges, cams, views, params, &cb, &dp);
  if (s != AGS_OK) return s;
  if (!hist || rule < 0 || rule > 2 || (rule == 1 && n > 0 && !max_T)) return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kHistBins, st) != cudaSuccess) return AGS_ERR_CUDA;
  if (n == 0) return AGS_OK;
  DiagArgs a{proj->depth, proj->flags, max_T, nullptr, hist, nullptr, nullptr, n * (int64_t)views, rule, 0.f};
  return diag_launch<kDiagHist>(proj, sorted_vals, ranges, cb, views, dp, a, st);
}

extern "C" ags_status ags_render_skip(const ags_projected* proj, int64_t n, const uint32_t* sorted_vals,
                                      const uint32_t* ranges, const ags_camera* cams, int32_t views,
                                      const ags_params* params, int32_t rule, const float* max_T, float thr,
                                      float* image, uint64_t* counts, void* stream) {
  using namespace ags;
  CamBatch cb;
  DevParams dp;
  ags_status s = diag_prepare(proj, n, sorted_vals, ranges, cams, views, params, &cb, &dp);
  if (s != AGS_OK) return s;
  if (!image || !counts || rule < 0 || rule > 2 || (rule == 1 && n > 0 && !max_T) || !(thr >= 0.f))
    return AGS_ERR_INVALID_ARG;
  DiagArgs a{proj->depth, proj->flags, max_T, nullptr, nullptr, reinterpret_cast<unsigned long long*>(counts),
             image, n * (int64_t)views, rule, thr};
  return diag_launch<kDiagSkip>(proj, sorted_vals, ranges, cb, views, dp, a, (cudaStream_t)stream);
}
