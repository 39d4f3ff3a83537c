// raster.cu -- per-tile front-to-back alpha blending (Eq. 1, Eq. 2) and the
// T_up calibration table (Sec. 3.4).
//
// One 64-thread CTA per 16x16 tile of each view: two warps, each an 8x16
// pixel block, each lane one column and four rows (y, y+4, y+8, y+12) that
// share the splat's dx terms (ags_params.blend_flags selects 8x8 blocks --
// four warps, two rows a lane -- and 64-splat batches instead, for the
// autotuner).  The warps run independently (no CTA barrier):
// a warp stages its tile's depth-ordered pairs 32 at a time, one per lane --
// gather of the 48-byte splat record (the next 32 are already in flight),
// conversion to the log2 form of Eq. 1, and the exact test whether the
// alpha >= tau ellipse reaches the warp's block -- then walks the splats that
// do.  A pixel's whole state is its transmittance T, which turns negative
// when the pixel stops (T (1 - alpha) < 1e-4, Eq. 2): a stopped pixel
// accepts nothing more, and |T| is its final transmittance.  A warp leaves
// once all its pixels stopped.  The blend always uses the conic of the
// original covariance and tau (Sec. 3.3 "dual-size strategy"): the scale mode
// only ever changed which pairs exist.
#include <algorithm>

#include "blend.cuh"

namespace ags {

// One pixel's step over one splat, in PTX so that the updates stay
// predicated FMAs: ok = (T > 0 and q >= log2 tau); T' = fma(-alpha, T, T);
// stop = ok and T' < t_min (T becomes -T: the pixel is done); blend = ok and
// not stop (colour += alpha T c, T = T').  kClamp: alpha = min(alpha_max,
// 2^q); without it alpha = 2^q (the splat's opacity is below alpha_max with
// margin, so the minimum would never bind).
template <bool kClamp>
__device__ __forceinline__ void blend_step(float q, float l2tau, float amax, float tmin, float cr, float cg,
                                           float cb, float& T, float& r, float& g, float& b) {
  if (kClamp) {
    asm("{\n\t"
        ".reg .pred tp, ok, st, bl;\n\t"
        ".reg .f32 e, a, na, tt, w;\n\t"
        "setp.gt.f32 tp, %0, 0f00000000;\n\t"
        "setp.ge.and.f32 ok, %4, %5, tp;\n\t"
        "ex2.approx.ftz.f32 e, %4;\n\t"
        "min.f32 a, e, %6;\n\t"
        "neg.f32 na, a;\n\t"
        "fma.rn.f32 tt, na, %0, %0;\n\t"
        "setp.lt.and.f32 st|bl, tt, %7, ok;\n\t"
        "mul.rn.f32 w, a, %0;\n\t"
        "@bl fma.rn.f32 %1, %8, w, %1;\n\t"
        "@bl fma.rn.f32 %2, %9, w, %2;\n\t"
        "@bl fma.rn.f32 %3, %10, w, %3;\n\t"
        "@bl fma.rn.f32 %0, na, %0, %0;\n\t"
        "@st mul.rn.f32 %0, %0, 0fBF800000;\n\t"
        "}"
        : "+f"(T), "+f"(r), "+f"(g), "+f"(b)
        : "f"(q), "f"(l2tau), "f"(amax), "f"(tmin), "f"(cr), "f"(cg), "f"(cb));
  } else {
    asm("{\n\t"
        ".reg .pred tp, ok, st, bl;\n\t"
        ".reg .f32 a, na, tt, w;\n\t"
        "setp.gt.f32 tp, %0, 0f00000000;\n\t"
        "setp.ge.and.f32 ok, %4, %5, tp;\n\t"
        "ex2.approx.ftz.f32 a, %4;\n\t"
        "neg.f32 na, a;\n\t"
        "fma.rn.f32 tt, na, %0, %0;\n\t"
        "setp.lt.and.f32 st|bl, tt, %7, ok;\n\t"
        "mul.rn.f32 w, a, %0;\n\t"
        "@bl fma.rn.f32 %1, %8, w, %1;\n\t"
        "@bl fma.rn.f32 %2, %9, w, %2;\n\t"
        "@bl fma.rn.f32 %3, %10, w, %3;\n\t"
        "@bl fma.rn.f32 %0, na, %0, %0;\n\t"
        "@st mul.rn.f32 %0, %0, 0fBF800000;\n\t"
        "}"
        : "+f"(T), "+f"(r), "+f"(g), "+f"(b)
        : "f"(q), "f"(l2tau), "f"(amax), "f"(tmin), "f"(cr), "f"(cg), "f"(cb));
  }
}

// The same step returning its decisions (blended, stopped: 0 or 1) for the
// instances that count, calibrate or record the blend state: the same
// instructions plus two selects.
template <bool kClamp>
__device__ __forceinline__ void blend_step_rec(float q, const BlendConst& bc, float cr, float cg, float cb, float& T,
                                               float& r, float& g, float& b, uint32_t& blended, uint32_t& stopped) {
  if (kClamp) {
    asm("{\n\t"
        ".reg .pred tp, ok, st, bl;\n\t"
        ".reg .f32 e, a, na, tt, w;\n\t"
        "setp.gt.f32 tp, %0, 0f00000000;\n\t"
        "setp.ge.and.f32 ok, %6, %7, tp;\n\t"
        "ex2.approx.ftz.f32 e, %6;\n\t"
        "min.f32 a, e, %8;\n\t"
        "neg.f32 na, a;\n\t"
        "fma.rn.f32 tt, na, %0, %0;\n\t"
        "setp.lt.and.f32 st|bl, tt, %9, ok;\n\t"
        "mul.rn.f32 w, a, %0;\n\t"
        "@bl fma.rn.f32 %1, %10, w, %1;\n\t"
        "@bl fma.rn.f32 %2, %11, w, %2;\n\t"
        "@bl fma.rn.f32 %3, %12, w, %3;\n\t"
        "@bl fma.rn.f32 %0, na, %0, %0;\n\t"
        "@st mul.rn.f32 %0, %0, 0fBF800000;\n\t"
        "selp.u32 %4, 1, 0, bl;\n\t"
        "selp.u32 %5, 1, 0, st;\n\t"
        "}"
        : "+f"(T), "+f"(r), "+f"(g), "+f"(b), "=r"(blended), "=r"(stopped)
        : "f"(q), "f"(bc.l2tau), "f"(bc.alpha_max), "f"(bc.t_min), "f"(cr), "f"(cg), "f"(cb));
  } else {
    asm("{\n\t"
        ".reg .pred tp, ok, st, bl;\n\t"
        ".reg .f32 a, na, tt, w;\n\t"
        "setp.gt.f32 tp, %0, 0f00000000;\n\t"
        "setp.ge.and.f32 ok, %6, %7, tp;\n\t"
        "ex2.approx.ftz.f32 a, %6;\n\t"
        "neg.f32 na, a;\n\t"
        "fma.rn.f32 tt, na, %0, %0;\n\t"
        "setp.lt.and.f32 st|bl, tt, %9, ok;\n\t"
        "mul.rn.f32 w, a, %0;\n\t"
        "@bl fma.rn.f32 %1, %10, w, %1;\n\t"
        "@bl fma.rn.f32 %2, %11, w, %2;\n\t"
        "@bl fma.rn.f32 %3, %12, w, %3;\n\t"
        "@bl fma.rn.f32 %0, na, %0, %0;\n\t"
        "@st mul.rn.f32 %0, %0, 0fBF800000;\n\t"
        "selp.u32 %4, 1, 0, bl;\n\t"
        "selp.u32 %5, 1, 0, st;\n\t"
        "}"
        : "+f"(T), "+f"(r), "+f"(g), "+f"(b), "=r"(blended), "=r"(stopped)
        : "f"(q), "f"(bc.l2tau), "f"(bc.alpha_max), "f"(bc.t_min), "f"(cr), "f"(cg), "f"(cb));
  }
}

// The step for the instance that records the blend state for the backward:
// the pixel's last blended position becomes pos1 under the blend predicate.
template <bool kClamp>
__device__ __forceinline__ void blend_step_state(float q, const BlendConst& bc, float cr, float cg, float cb,
                                                 float& T, float& r, float& g, float& b, uint32_t& last,
                                                 uint32_t pos1) {
  if (kClamp) {
    asm("{\n\t"
        ".reg .pred tp, ok, st, bl;\n\t"
        ".reg .f32 e, a, na, tt, w;\n\t"
        "setp.gt.f32 tp, %0, 0f00000000;\n\t"
        "setp.ge.and.f32 ok, %6, %7, tp;\n\t"
        "ex2.approx.ftz.f32 e, %6;\n\t"
        "min.f32 a, e, %8;\n\t"
        "neg.f32 na, a;\n\t"
        "fma.rn.f32 tt, na, %0, %0;\n\t"
        "setp.lt.and.f32 st|bl, tt, %9, ok;\n\t"
        "mul.rn.f32 w, a, %0;\n\t"
        "@bl fma.rn.f32 %1, %10, w, %1;\n\t"
        "@bl fma.rn.f32 %2, %11, w, %2;\n\t"
        "@bl fma.rn.f32 %3, %12, w, %3;\n\t"
        "@bl fma.rn.f32 %0, na, %0, %0;\n\t"
        "@bl mov.u32 %4, %5;\n\t"
        "@st mul.rn.f32 %0, %0, 0fBF800000;\n\t"
        "}"
        : "+f"(T), "+f"(r), "+f"(g), "+f"(b), "+r"(last)
        : "r"(pos1), "f"(q), "f"(bc.l2tau), "f"(bc.alpha_max), "f"(bc.t_min), "f"(cr), "f"(cg), "f"(cb));
  } else {
    asm("{\n\t"
        ".reg .pred tp, ok, st, bl;\n\t"
        ".reg .f32 a, na, tt, w;\n\t"
        "setp.gt.f32 tp, %0, 0f00000000;\n\t"
        "setp.ge.and.f32 ok, %6, %7, tp;\n\t"
        "ex2.approx.ftz.f32 a, %6;\n\t"
        "neg.f32 na, a;\n\t"
        "fma.rn.f32 tt, na, %0, %0;\n\t"
        "setp.lt.and.f32 st|bl, tt, %9, ok;\n\t"
        "mul.rn.f32 w, a, %0;\n\t"
        "@bl fma.rn.f32 %1, %10, w, %1;\n\t"
        "@bl fma.rn.f32 %2, %11, w, %2;\n\t"
        "@bl fma.rn.f32 %3, %12, w, %3;\n\t"
        "@bl fma.rn.f32 %0, na, %0, %0;\n\t"
        "@bl mov.u32 %4, %5;\n\t"
        "@st mul.rn.f32 %0, %0, 0fBF800000;\n\t"
        "}"
        : "+f"(T), "+f"(r), "+f"(g), "+f"(b), "+r"(last)
        : "r"(pos1), "f"(q), "f"(bc.l2tau), "f"(bc.alpha_max), "f"(bc.t_min), "f"(cr), "f"(cg), "f"(cb));
  }
}

// The pair value at `v` and its 48-byte splat record.  A debug build checks
// the value against the record count first; a value out of range becomes an
// empty record of Gaussian-view 0 (opacity 0: it reaches no pixel).
__device__ __forceinline__ void gather_record(const float4* __restrict__ splat, const uint32_t* v, uint32_t n_splats,
                                              int64_t* status, uint32_t& e, float4& r0, float4& r1, float4& r2) {
  e = __ldg(v);
  if (AGS_DCHECK(e < n_splats, status, AGS_CHECK_BLEND_VALUE)) {
    const float4* rec = splat + (size_t)e * 3;
    r0 = __ldg(rec); r1 = __ldg(rec + 1); r2 = __ldg(rec + 2);
  } else {
    e = 0u;
    r0 = r1 = r2 = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// kStats: count evaluations and blends; kMaxT: calibration output; kState:
// each pixel's final T and last blended position (for the backward).  The
// shape: kRows rows per lane (4: 8x16-pixel warp blocks, two warps a tile;
// 2: 8x8 blocks, four warps) and kBatch splats staged per lane and round (the
// warp's tile batch is 32 kBatch splats, the next batch in flight meanwhile).
// The benchmark's kernel is the <false, false, false, 4, 1> instance.
template <bool kStats, bool kMaxT, bool kState, int kRows, int kBatch>
__global__ void __launch_bounds__(256 / kRows)
raster_kernel(const float4* __restrict__ splat, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
              int W, int H, int gx, int tiles_per_view, BlendConst bc, float* __restrict__ image,
              float* __restrict__ final_T, uint32_t* __restrict__ n_contrib, uint32_t* __restrict__ max_T_bits,
              unsigned long long* stats, uint32_t n_splats, int64_t* status) {
  constexpr bool kRec = kStats || kMaxT || kState;
  constexpr int kWarps = 8 / kRows;
  constexpr int kBH = 4 * kRows;                 // warp block: 8 columns x kBH rows
  constexpr int kStage = 32 * kBatch;
  __shared__ float4 s_a[kWarps][kStage];    // u v a2 b2
  __shared__ float4 s_b[kWarps][kStage];    // c2 log2(opacity) r g
  __shared__ float s_c[kWarps][kStage];     // b
  __shared__ uint32_t s_e[kWarps][kMaxT ? kStage : 1];

  const int tile = blockIdx.x;
  const int view = tile / tiles_per_view;
  const int lt = tile - view * tiles_per_view;
  const int ty = lt / gx, tx = lt - ty * gx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bx0 = tx * kTile + 8 * (warp & 1), by0 = ty * kTile + kBH * (warp >> 1);
  const int px = bx0 + (lane & 7);
  const int py = by0 + (lane >> 3);
  const float fpx = (float)px;
  float fpy[kRows], T[kRows], cr[kRows], cg[kRows], cb[kRows];
  uint32_t last[kRows], stop_at[kRows];
#pragma unroll
  for (int k = 0; k < kRows; k++) {
    fpy[k] = (float)(py + 4 * k);
    T[k] = (px < W && py + 4 * k < H) ? 1.f : -1.f;      // negative: nothing to blend
    cr[k] = cg[k] = cb[k] = 0.f;
    last[k] = 0u;
    stop_at[k] = 0u;
  }
  const uint2 rg = __ldg(ranges + tile);
  const uint32_t start = rg.x;
  const uint32_t end = AGS_DCHECK(rg.x <= rg.y, status, AGS_CHECK_BLEND_RANGE) ? rg.y : rg.x;
  float4* sa = s_a[warp];
  float4* sb = s_b[warp];
  float* sc = s_c[warp];
  const float l2clamp = __log2f(bc.alpha_max) - 1e-3f;   // opacities above this take the clamped step
  uint32_t blends = 0u, walked_total = 0u;

  // the first batch in flight
  float4 n0[kBatch], n1[kBatch], n2[kBatch];
  uint32_t ne[kBatch];
#pragma unroll
  for (int i = 0; i < kBatch; i++) {
    n0[i] = n1[i] = n2[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    ne[i] = 0u;
    if (start + 32 * i + lane < end)
      gather_record(splat, vals + start + 32 * i + lane, n_splats, status, ne[i], n0[i], n1[i], n2[i]);
  }
  for (uint32_t bb = start; bb < end; bb += kStage) {
    bool alive = false;
#pragma unroll
    for (int k = 0; k < kRows; k++) alive = alive || T[k] > 0.f;
    if (!__any_sync(0xffffffffu, alive)) break;
    unsigned m[kBatch];
#pragma unroll
    for (int i = 0; i < kBatch; i++) {
      bool hit = false;
      if (bb + 32 * i + lane < end) {
        const float4 r0 = n0[i], r1 = n1[i], r2 = n2[i];
        Staged st;
        stage_record(r0, r1, r2, st);
        sa[32 * i + lane] = st.a;
        sb[32 * i + lane] = st.b;
        sc[32 * i + lane] = st.c;
        if (kMaxT) s_e[warp][32 * i + lane] = ne[i];
        hit = ellipse_reaches(r0.x - (float)bx0, r0.y - (float)by0, 7.f, (float)(kBH - 1),
                              reach_r2n(st.b.y, bc.l2tau), r2.z, r2.w, r0.z, r0.w, r1.x);
      }
      m[i] = __ballot_sync(0xffffffffu, hit);
    }
#pragma unroll
    for (int i = 0; i < kBatch; i++) {   // the next batch, in flight while this one is blended
      if (bb + kStage + 32 * i + lane < end)
        gather_record(splat, vals + bb + kStage + 32 * i + lane, n_splats, status, ne[i], n0[i], n1[i], n2[i]);
    }
    __syncwarp();
    int walked = 0;
    bool done = false;
#pragma unroll
    for (int i = 0; i < kBatch; i++) {
      unsigned mask = m[i];
      if (kStats) walked_total += (uint32_t)__popc(mask);
      while (mask) {
        const int j = 32 * i + __ffs(mask) - 1;
        mask &= mask - 1;
        Staged s;
        s.a = sa[j];
        s.b = sb[j];
        const float cbl = sc[j];
        const float dx = __fsub_rn(s.a.x, fpx);
        float P, Bx;
        splat_qx(s, dx, P, Bx);
        const bool clamp = s.b.y > l2clamp;
        if (!kRec) {
          if (clamp) {
#pragma unroll
            for (int k = 0; k < kRows; k++)
              blend_step<true>(splat_qy(s, P, Bx, __fsub_rn(s.a.y, fpy[k])), bc.l2tau, bc.alpha_max, bc.t_min,
                               s.b.z, s.b.w, cbl, T[k], cr[k], cg[k], cb[k]);
          } else {
#pragma unroll
            for (int k = 0; k < kRows; k++)
              blend_step<false>(splat_qy(s, P, Bx, __fsub_rn(s.a.y, fpy[k])), bc.l2tau, bc.alpha_max, bc.t_min,
                                s.b.z, s.b.w, cbl, T[k], cr[k], cg[k], cb[k]);
          }
        } else if (kState && !kStats && !kMaxT) {   // the backward's forward: last blended position only
          const uint32_t pos1 = bb - start + (uint32_t)j + 1u;
          if (clamp) {
#pragma unroll
            for (int k = 0; k < kRows; k++)
              blend_step_state<true>(splat_qy(s, P, Bx, __fsub_rn(s.a.y, fpy[k])), bc, s.b.z, s.b.w, cbl, T[k],
                                     cr[k], cg[k], cb[k], last[k], pos1);
          } else {
#pragma unroll
            for (int k = 0; k < kRows; k++)
              blend_step_state<false>(splat_qy(s, P, Bx, __fsub_rn(s.a.y, fpy[k])), bc, s.b.z, s.b.w, cbl, T[k],
                                      cr[k], cg[k], cb[k], last[k], pos1);
          }
        } else {
          const uint32_t pos1 = bb - start + (uint32_t)j + 1u;    // 1-based position in the tile's list
          uint32_t mt = 0u;
#pragma unroll
          for (int k = 0; k < kRows; k++) {
            const float Tb = T[k];
            const float q = splat_qy(s, P, Bx, __fsub_rn(s.a.y, fpy[k]));
            uint32_t bl, stp;
            if (clamp)
              blend_step_rec<true>(q, bc, s.b.z, s.b.w, cbl, T[k], cr[k], cg[k], cb[k], bl, stp);
            else
              blend_step_rec<false>(q, bc, s.b.z, s.b.w, cbl, T[k], cr[k], cg[k], cb[k], bl, stp);
            if (kStats) {
              blends += bl;
              stop_at[k] = stp ? pos1 : stop_at[k];
            }
            if (kState) last[k] = bl ? pos1 : last[k];
            if (kMaxT) mt = max(mt, bl ? __float_as_uint(Tb) : 0u);
          }
          if (kMaxT) {   // calibration: per-Gaussian max T before blending (warp max, one atomic)
            const uint32_t mx = __reduce_max_sync(0xffffffffu, mt);
            if (lane == 0 && mx) atomicMax(max_T_bits + s_e[warp][j], mx);
          }
        }
        if ((++walked & 3) == 0) {
          bool al = false;
#pragma unroll
          for (int k = 0; k < kRows; k++) al = al || T[k] > 0.f;
          if (!__any_sync(0xffffffffu, al)) {
            if (kStats) walked_total -= (uint32_t)__popc(mask);    // not walked
            done = true;
            break;
          }
        }
      }
      if (done) break;     // the later masks of this batch were never counted
    }
    __syncwarp();
  }
  const size_t hw = (size_t)W * H;
  unsigned long long evals = 0ull;
#pragma unroll
  for (int k = 0; k < kRows; k++) {
    const int y = py + 4 * k;
    if (px < W && y < H) {
      const float Tf = fabsf(T[k]);
      const size_t o = (size_t)view * 3 * hw + (size_t)y * W + px;
      image[o] = cr[k] + Tf * bc.bg[0];
      image[o + hw] = cg[k] + Tf * bc.bg[1];
      image[o + 2 * hw] = cb[k] + Tf * bc.bg[2];
      const size_t op = (size_t)view * hw + (size_t)y * W + px;
      if (final_T) final_T[op] = Tf;
      if (kState) n_contrib[op] = last[k];
      // Eq. 1-2 evaluations of this pixel: its tile's pairs up to the one it stopped at
      if (kStats) evals += stop_at[k] ? stop_at[k] : (end - start);
    }
  }
  if (kStats) {
    const unsigned long long e1 = warp_sum(evals), e2 = warp_sum((unsigned long long)blends);
    if (lane == 0) {
      atomicAdd(stats, e1);
      atomicAdd(stats + 1, e2);
      // pixel-pair slots the kernel walked: each walked splat against the warp's 8 x kBH pixels
      atomicAdd(stats + 2, (unsigned long long)walked_total * (8ull * kBH));
    }
  }
}

typedef void (*RasterFn)(const float4*, const uint32_t*, const uint2*, int, int, int, int, BlendConst, float*, float*,
                         uint32_t*, uint32_t*, unsigned long long*, uint32_t, int64_t*);

template <int kRows, int kBatch>
RasterFn pick_raster(bool st, bool mt, bool state) {
  if (state)
    return st ? (mt ? raster_kernel<true, true, true, kRows, kBatch> : raster_kernel<true, false, true, kRows, kBatch>)
              : (mt ? raster_kernel<false, true, true, kRows, kBatch>
                    : raster_kernel<false, false, true, kRows, kBatch>);
  return st ? (mt ? raster_kernel<true, true, false, kRows, kBatch> : raster_kernel<true, false, false, kRows, kBatch>)
            : (mt ? raster_kernel<false, true, false, kRows, kBatch>
                  : raster_kernel<false, false, false, kRows, kBatch>);
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
  if ((uintptr_t)ranges & 7u) return AGS_ERR_INVALID_ARG;       // read as 8-byte (start, end) pairs
  CamBatch cb;
  DevParams dp;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  s = build_params(params, &dp);
  if (s != AGS_OK) return s;
  if (n > 0 && (!proj->splat || !sorted_vals)) return AGS_ERR_INVALID_ARG;
  if ((uintptr_t)proj->splat & 15u) return AGS_ERR_INVALID_ARG;
  if (n * (int64_t)views > (int64_t)UINT32_MAX) return AGS_ERR_INVALID_ARG;   // pair values are 32-bit
  const int tiles_per_view = cb.c[0].gx * cb.c[0].gy;
  BlendConst bc = make_blend_const(dp);
  const bool st = stats != nullptr, mt = max_T != nullptr, state = n_contrib != nullptr;
  RasterFn kern;
  switch (dp.blend_flags) {
    case AGS_BLEND_ROWS2: kern = pick_raster<2, 1>(st, mt, state); break;
    case AGS_BLEND_BATCH64: kern = pick_raster<4, 2>(st, mt, state); break;
    case AGS_BLEND_ROWS2 | AGS_BLEND_BATCH64: kern = pick_raster<2, 2>(st, mt, state); break;
    default: kern = pick_raster<4, 1>(st, mt, state); break;
  }
  const unsigned threads = (dp.blend_flags & AGS_BLEND_ROWS2) ? 128u : 64u;   // 256 / rows per lane
  kern<<<(unsigned)(tiles_per_view * views), threads, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const float4*>(proj->splat), sorted_vals, reinterpret_cast<const uint2*>(ranges),
      cb.c[0].W, cb.c[0].H, cb.c[0].gx, tiles_per_view, bc, image, final_T, n_contrib,
      reinterpret_cast<uint32_t*>(max_T), reinterpret_cast<unsigned long long*>(stats), (uint32_t)(n * views),
      d_status);
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
