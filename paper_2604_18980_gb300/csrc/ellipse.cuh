// ellipse.cuh -- the ellipse tile test (tile_test AGS_TILE_ELLIPSE): which
// tiles of a Gaussian's square footprint the ellipse alpha >= Th reaches.
//
// With the blending conic (A B; B C) and q = A dx^2 + 2 B dx dy + C dy^2, the
// ellipse is q <= Q, Q = 2 ln(opacity / Th) (Th = tau in plain mode, Eq. 10 in
// AdaGScale mode).  A tile is kept when the ellipse meets the rectangle spanned
// by the tile's pixel centres (clipped to the image): the minimum of q over
// that rectangle is <= Q.  The preprocess counts the kept tiles and the
// emission enumerates them with the same functions on the same fp32 inputs,
// so both see the same tiles.
#pragma once

#include "blend.cuh"

namespace ags {

struct EllipseTiles {
  float u, v, A, B, C, Q;    // centre, conic, level
  int x0, x1;                // tile columns [x0, x1) of the square footprint
  int W, H;                  // image size
};

// Q from the stored opacity and threshold (the same expression everywhere).
__device__ __forceinline__ float ellipse_level(float opacity, float th) { return 2.f * logf(opacity / th); }

// A tile is kept when the minimum of q over its pixel-centre rectangle is at
// most Q plus a relative 1e-5: a margin far above the fp32 rounding of the
// blend's own alpha >= tau test, so that in plain mode no tile holding an
// accepted pixel is ever dropped.
__device__ __forceinline__ float ellipse_keep_level(float Q) { return Q + 1e-5f * fmaxf(Q, 1.f); }

__device__ __forceinline__ float tile_min_q(const EllipseTiles& E, int tx, int ty) {
  const float xl = (float)(kTile * tx) - E.u, xh = (float)min(kTile * tx + kTile - 1, E.W - 1) - E.u;
  const float yl = (float)(kTile * ty) - E.v, yh = (float)min(kTile * ty + kTile - 1, E.H - 1) - E.v;
  return rect_min_quad(E.A, E.B, E.C, xl, xh, yl, yh);
}

__device__ __forceinline__ bool tile_kept(const EllipseTiles& E, float Qk, int tx, int ty) {
  return tile_min_q(E, tx, ty) <= Qk;
}

// First kept column in [a, b] when column b is kept (the kept columns of a row
// are contiguous).  `guess` is tried first with short walks, then bisection.
__device__ __forceinline__ int first_kept(const EllipseTiles& E, float Qk, int ty, int a, int b, int guess) {
  int g = min(max(guess, a), b);
  if (tile_kept(E, Qk, g, ty)) {
    if (g == a || !tile_kept(E, Qk, g - 1, ty)) return g;
    b = g - 1;                                  // kept; the first one is in [a, g - 1]
  } else {
    if (tile_kept(E, Qk, g + 1, ty)) return g + 1;
    a = g + 2;                                  // [g + 2, b], b kept
    if (a > b) return b;
  }
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (tile_kept(E, Qk, mid, ty)) b = mid; else a = mid + 1;
  }
  return a;
}

// Last kept column in [a, b] when column a is kept.
__device__ __forceinline__ int last_kept(const EllipseTiles& E, float Qk, int ty, int a, int b, int guess) {
  int g = min(max(guess, a), b);
  if (tile_kept(E, Qk, g, ty)) {
    if (g == b || !tile_kept(E, Qk, g + 1, ty)) return g;
    a = g + 1;
  } else {
    if (tile_kept(E, Qk, g - 1, ty)) return g - 1;
    b = g - 2;
    if (a > b) return a;
  }
  while (a < b) {
    const int mid = (a + b + 1) >> 1;
    if (tile_kept(E, Qk, mid, ty)) a = mid; else b = mid - 1;
  }
  return a;
}

// Kept tiles [lo, hi] of tile row ty (lo > hi when none).  The minimum of q
// over a tile rectangle is a convex function of the tile's position, so the
// kept tiles of a row are contiguous around the column where the row band's
// minimum of q lies; that column (or its neighbour across the gap between
// tiles) decides whether the row has any.  The ends start from the closed-form
// x-range of the ellipse over the band -- the section of a conic, whose
// extreme points lie at dy = -+B sqrt(Q / (det C)) -- and are settled by the
// per-tile test.
__device__ __forceinline__ void ellipse_row_span(const EllipseTiles& E, int ty, int& lo, int& hi) {
  lo = 1;
  hi = 0;
  if (!(E.Q >= 0.f) || E.x0 >= E.x1) return;
  const float Qk = ellipse_keep_level(E.Q);
  const float yl = (float)(kTile * ty) - E.v, yh = (float)min(kTile * ty + kTile - 1, E.H - 1) - E.v;
  // the band's lowest q: dy closest to 0, then dx = -B dy / A
  const float dyc = fminf(fmaxf(0.f, yl), yh);
  const float xc = E.u - E.B * dyc / E.A;
  const float fc = floorf(fminf(fmaxf(xc, -1e9f), 1e9f) / (float)kTile);
  int tc = min(max((int)fc, E.x0), E.x1 - 1);
  int tb = tc;
  float mb = tile_min_q(E, tc, ty);
  if (xc - (float)(kTile * tc) > (float)(kTile - 1) && tc + 1 < E.x1) {   // minimiser in the gap after tc
    const float m = tile_min_q(E, tc + 1, ty);
    if (m < mb) { mb = m; tb = tc + 1; }
  }
  if (xc < (float)(kTile * tc) && tc > E.x0) {                              // clamped from the left
    const float m = tile_min_q(E, tc - 1, ty);
    if (m < mb) { mb = m; tb = tc - 1; }
  }
  if (!(mb <= Qk)) return;
  // closed-form x-range of the ellipse over the band (a guess: fp32, thin ellipses lose digits)
  int gl = E.x0, gh = E.x1 - 1;
  const float det = E.A * E.C - E.B * E.B;
  if (det > 0.f) {
    const float ymax = sqrtf(E.A * E.Q / det);
    const float bl = fmaxf(yl, -ymax), bh = fminf(yh, ymax);
    if (bl <= bh) {
      const float ds = E.B * sqrtf(E.Q / (det * E.C));
      const float d1 = fminf(fmaxf(ds, bl), bh), d2 = fminf(fmaxf(-ds, bl), bh);
      const float xl = E.u + (-E.B * d1 - sqrtf(fmaxf(E.A * E.Q - det * d1 * d1, 0.f))) / E.A;
      const float xr = E.u + (-E.B * d2 + sqrtf(fmaxf(E.A * E.Q - det * d2 * d2, 0.f))) / E.A;
      gl = (int)fminf(fmaxf(ceilf((xl - (float)(kTile - 1)) / (float)kTile), -1e6f), 1e6f);
      gh = (int)fminf(fmaxf(floorf(xr / (float)kTile), -1e6f), 1e6f);
    }
  }
  lo = first_kept(E, Qk, ty, E.x0, tb, gl);
  hi = last_kept(E, Qk, ty, tb, E.x1 - 1, gh);
}

}  // namespace ags

namespace ags {

// Enumeration of one Gaussian-view's kept tiles in row-major order (the
// emission order), starting at its r-th kept tile.  Reads the square from the
// rectangle record and the centre, conic, opacity and Th from the splat record.
struct EllipseWalk {
  EllipseTiles E;
  int ty, y1, lo, hi, tx;
  uint32_t vbase;              // view * tiles_per_view

  __device__ __forceinline__ void start(const float4* __restrict__ splat, const uint2* __restrict__ rect, uint32_t e,
                                        uint32_t n, uint32_t tiles_per_view, int W, int H, uint32_t r) {
    const uint2 rc = __ldg(rect + e);
    const int x0 = (int)(rc.x & 0xffffu), y0 = (int)(rc.x >> 16);
    E.x0 = x0;
    E.x1 = (int)(rc.y & 0xffffu);
    y1 = (int)(rc.y >> 16);
    const float4 s0 = __ldg(splat + (size_t)e * 3), s1 = __ldg(splat + (size_t)e * 3 + 1);
    const float th = __ldg(reinterpret_cast<const float*>(splat + (size_t)e * 3 + 2) + 1);
    E.u = s0.x; E.v = s0.y; E.A = s0.z; E.B = s0.w; E.C = s1.x;
    E.Q = ellipse_level(s1.y, th);
    E.W = W; E.H = H;
    vbase = (e / n) * tiles_per_view;
    ty = y0;
    ellipse_row_span(E, ty, lo, hi);
    while (true) {
      const uint32_t cnt = lo <= hi ? (uint32_t)(hi - lo + 1) : 0u;
      if (r < cnt || ty + 1 >= y1) break;
      r -= cnt;
      ++ty;
      ellipse_row_span(E, ty, lo, hi);
    }
    tx = lo + (int)r;
  }

  __device__ __forceinline__ uint32_t tile(uint32_t gx) const { return vbase + (uint32_t)ty * gx + (uint32_t)tx; }

  __device__ __forceinline__ void next() {
    if (++tx <= hi) return;
    do {
      if (++ty >= y1) return;
      ellipse_row_span(E, ty, lo, hi);
    } while (lo > hi);
    tx = lo;
  }
};

}  // namespace ags
