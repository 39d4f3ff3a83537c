// blend.cuh -- per-pixel alpha of one splat (Eq. 1), shared by the blend and
// its adjoint so that both take bit-identical decisions.
#pragma once

#include "ags_internal.cuh"

namespace ags {

constexpr int kRasterThreads = kTile * kTile;

struct BlendConst {
  float tau, t_min, alpha_max;
  float bg[3];
};

// p = -(A dx^2 + C dy^2)/2 - B dx dy with dx = u - px, dy = v - py, every
// operation rounded explicitly (no contraction freedom for the compiler).
__device__ __forceinline__ float splat_power(float u, float v, float A, float B, float C, float px, float py,
                                             float& dx, float& dy) {
  dx = __fsub_rn(u, px);
  dy = __fsub_rn(v, py);
  float q = __fadd_rn(__fmul_rn(__fmul_rn(A, dx), dx), __fmul_rn(__fmul_rn(C, dy), dy));
  return __fsub_rn(__fmul_rn(-0.5f, q), __fmul_rn(__fmul_rn(B, dx), dy));
}

// opacity * e^p before the alpha_max clamp.
__device__ __forceinline__ float splat_alpha_raw(float opacity, float power) {
  return __fmul_rn(opacity, __expf(power));
}

}  // namespace ags
