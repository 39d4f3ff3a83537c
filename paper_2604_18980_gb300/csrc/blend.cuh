// blend.cuh -- per-pixel alpha of one splat (Eq. 1) as the blend, its adjoint
// and the diagnostics evaluate it, shared so all take bit-identical decisions.
//
// The exponent is carried in log2 units:
//   a2 = -A log2(e)/2, b2 = -B log2(e), c2 = -C log2(e)/2,
//   q  = a2 dx^2 + b2 dx dy + c2 dy^2 + log2(opacity) = log2(opacity e^p),
// so Eq. 1 is alpha = min(alpha_max, 2^q) and alpha >= tau is q >= log2(tau):
// the threshold test runs before the exponential.  The transmittance after a
// blended splat is fma(-alpha, T, T), T (1 - alpha) rounded once.
//
// For every staged splat the loading thread also computes which blocks of
// the 16x16 tile can hold a pixel with alpha >= tau: its ellipse
// p >= ln(tau/opacity) must reach the block's rectangle of pixel centres -- a
// bounding-box test (half-widths sqrt(2 ln(opacity/tau) Sigma_xx),
// sqrt(2 ln(opacity/tau) Sigma_yy)) and then the exact minimum of the
// quadratic form over the rectangle, both with a slack far above fp32
// rounding.  A block whose bit is clear would have rejected the splat with
// alpha < tau at every pixel, so skipping it leaves the result unchanged.
#pragma once

#include <cmath>

#include "ags_internal.cuh"

namespace ags {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

struct BlendConst {
  float tau, t_min, alpha_max, l2tau;   // l2tau = log2(tau)
  float bg[3];
};

// Host-side constants of the blend from the parameter block.
inline BlendConst make_blend_const(const DevParams& dp) {
  BlendConst bc;
  bc.tau = dp.tau;
  bc.t_min = dp.t_min;
  bc.alpha_max = dp.alpha_max;
  bc.l2tau = (float)std::log2((double)dp.tau);
  for (int i = 0; i < 3; i++) bc.bg[i] = dp.bg[i];
  return bc;
}

struct Staged {
  float4 a;      // u, v, a2, b2
  float4 b;      // c2, log2(opacity), r, g
  float c;       // b
};

// Does the alpha >= tau ellipse of a splat reach the rectangle of pixel
// centres [x0, x0 + w] x [y0, y0 + h]?  (cu, cv): the splat centre relative to
// (x0, y0); r2n: 2 ln(opacity / tau) plus slack; Sxx, Syy: the covariance
// diagonal (half-widths of the ellipse's bounding box); A, B, C: the conic.
__device__ __forceinline__ bool ellipse_reaches(float cu, float cv, float w, float h, float r2n, float Sxx, float Syy,
                                                float A, float B, float C);

// Minimum over the rectangle [xl,xh] x [yl,yh] of A x^2 + 2 B x y + C y^2 for a
// positive-definite (A B; B C): zero when the rectangle holds the origin,
// otherwise attained on an edge, where the 1-D minimiser is clamped to it.
__device__ __forceinline__ float rect_min_quad(float A, float B, float C, float xl, float xh, float yl, float yh) {
  if (xl <= 0.f && xh >= 0.f && yl <= 0.f && yh >= 0.f) return 0.f;
  const float iA = 1.f / A, iC = 1.f / C;
  float m = 3.402823466e38f;
  const float xs[2] = {xl, xh}, ys[2] = {yl, yh};
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const float x = xs[k];
    const float y = fminf(fmaxf(-B * x * iC, yl), yh);
    m = fminf(m, fmaf(A * x, x, fmaf(2.f * B * x, y, C * y * y)));
    const float y2 = ys[k];
    const float x2 = fminf(fmaxf(-B * y2 * iA, xl), xh);
    m = fminf(m, fmaf(A * x2, x2, fmaf(2.f * B * x2, y2, C * y2 * y2)));
  }
  return m;
}

__device__ __forceinline__ bool ellipse_reaches(float cu, float cv, float w, float h, float r2n, float Sxx, float Syy,
                                                float A, float B, float C) {
  if (!(r2n > 0.f)) return false;
  const float hx = sqrtf(r2n * Sxx) * 1.0001f + 0.01f;
  const float hy = sqrtf(r2n * Syy) * 1.0001f + 0.01f;
  return cu + hx >= 0.f && cu - hx <= w && cv + hy >= 0.f && cv - hy <= h &&
         rect_min_quad(A, B, C, -cu, w - cu, -cv, h - cv) <= r2n * 1.0001f;
}

// The staged form of a splat record (48 bytes: u v A B | C opacity r g | b Th Sxx Syy).
__device__ __forceinline__ void stage_record(const float4& r0, const float4& r1, const float4& r2, Staged& s) {
  s.a = make_float4(r0.x, r0.y, -0.5f * kLog2e * r0.z, -kLog2e * r0.w);
  s.b = make_float4(-0.5f * kLog2e * r1.x, __log2f(r1.y), r1.z, r1.w);
  s.c = r2.x;
}

// 2 ln(opacity / tau) + slack: the squared Mahalanobis radius of the alpha >= tau ellipse.
__device__ __forceinline__ float reach_r2n(float l2s, float l2tau) { return 2.f * kLn2 * (l2s - l2tau) + 1e-3f; }

// Mask bit w: the ellipse can reach block w of the tile, blocks being
// BW x BH pixels in row-major order of (16/BW) x (16/BH).
template <int BW, int BH>
__device__ __forceinline__ void stage_splat(const float4* rec, int tx0, int ty0, float l2tau, Staged& s,
                                            uint32_t& mask) {
  const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2);
  stage_record(r0, r1, r2, s);
  mask = 0u;
  const float r2n = reach_r2n(s.b.y, l2tau);
  constexpr int NBX = kTile / BW, NBY = kTile / BH;
  const float cu = r0.x - (float)tx0, cv = r0.y - (float)ty0;    // tile-relative centre
#pragma unroll
  for (int w = 0; w < NBX * NBY; w++) {
    const float cx0 = (float)(BW * (w % NBX)), ry0 = (float)(BH * (w / NBX));
    if (ellipse_reaches(cu - cx0, cv - ry0, (float)(BW - 1), (float)(BH - 1), r2n, r2.z, r2.w, r0.z, r0.w, r1.x))
      mask |= 1u << w;
  }
}

// The splat is blended at a pixel iff alpha >= tau: q >= log2(tau).  (p <= 0
// holds exactly for a positive-definite conic; a q rounded a hair above
// log2(opacity) only gives an alpha a hair above the opacity.)
__device__ __forceinline__ bool splat_accept(float q, float l2tau) { return q >= l2tau; }

__device__ __forceinline__ float fast_exp2(float x);

// Eq. 1: alpha = min(alpha_max, 2^q); also the unclamped value.
__device__ __forceinline__ float splat_alpha(float q, float alpha_max, float& raw) {
  raw = fast_exp2(q);
  return fminf(alpha_max, raw);
}

// Eq. 2: the transmittance behind a blended splat, T (1 - alpha) rounded once.
__device__ __forceinline__ float transmit(float alpha, float T) { return __fmaf_rn(-alpha, T, T); }

// q = (a2 dx^2 + log2 opacity) + dy (b2 dx + c2 dy), split so that pixels
// sharing a column share the dx terms: splat_qx gives (P, Bx), splat_qy
// finishes q with dy = v - y (one rounding).
__device__ __forceinline__ void splat_qx(const Staged& s, float dx, float& P, float& Bx) {
  P = __fmaf_rn(__fmul_rn(s.a.z, dx), dx, s.b.y);
  Bx = __fmul_rn(s.a.w, dx);
}

__device__ __forceinline__ float splat_qy(const Staged& s, float P, float Bx, float dy) {
  return __fmaf_rn(dy, __fmaf_rn(s.b.x, dy, Bx), P);
}

__device__ __forceinline__ float splat_q(const Staged& s, float px, float py, float& dx, float& dy) {
  dx = __fsub_rn(s.a.x, px);
  dy = __fsub_rn(s.a.y, py);
  float P, Bx;
  splat_qx(s, dx, P, Bx);
  return splat_qy(s, P, Bx, dy);
}

// Eigenframe of a conic (A B; B C): e_a = (ca, sa) maximises the quadratic
// form (the splat's minor axis), e_b = (-sa, ca).  Shared by the blend adjoint
// and the preprocess adjoint so both use the same frame.
__device__ __forceinline__ void conic_frame(float A, float B, float C, float& ca, float& sa) {
  const float th = 0.5f * atan2f(2.f * B, A - C);
  sincosf(th, &sa, &ca);
}

__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

}  // namespace ags
