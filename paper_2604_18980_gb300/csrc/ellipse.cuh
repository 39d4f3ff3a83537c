// ellipse.cuh -- the ellipse tile test (tile_test AGS_TILE_ELLIPSE): which
// tiles of a Gaussian's square footprint the ellipse alpha >= Th reaches.
//
// With the blending conic (A B; B C) and q = A dx^2 + 2 B dx dy + C dy^2, the
// ellipse is q <= Q, Q = 2 ln(opacity / Th) (Th = tau in plain mode, Eq. 10 in
// AdaGScale mode).  A tile is kept when the ellipse meets the rectangle spanned
// by the tile's pixel centres (clipped to the image): the minimum of q over
// that rectangle is <= Q.  The preprocess counts the kept tiles and the
// emission enumerates them with the same functions on the same fp32 inputs
// (the splat record), so both see the same tiles.
#pragma once

#include "blend.cuh"

namespace ags {

struct EllipseTiles {
  float u, v, A, B, C, Q;    // centre, conic, level
  int x0, x1;                // tile columns [x0, x1) of the square footprint
  int W, H;                  // image size
  float iA, iC;              // 1/A, 1/C (set by prepare)
};

__device__ __forceinline__ void ellipse_prepare(EllipseTiles& E) {
  E.iA = 1.f / E.A;
  E.iC = 1.f / E.C;
}

// rect_min_quad with the conic's diagonal reciprocals given.
__device__ __forceinline__ float rect_min_quad_r(float A, float B, float C, float iA, float iC, float xl, float xh,
                                                 float yl, float yh) {
  if (xl <= 0.f && xh >= 0.f && yl <= 0.f && yh >= 0.f) return 0.f;
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

// Q from the stored opacity and threshold (the same expression everywhere).
__device__ __forceinline__ float ellipse_level(float opacity, float th) { return 2.f * logf(opacity / th); }

// A tile of row ty is kept when the minimum of q over its pixel-centre
// rectangle is at most Q plus a margin far above the fp32 rounding of both
// that minimum and the blend's own alpha >= tau test: 1e-5 of Q, plus 1e-6 of
// S = A X^2 + 2|B| X Y + C Y^2, X and Y the largest |dx| and |dy| of the row's
// part of the square, which bounds the terms of q before they cancel (thin,
// tilted ellipses far across a large image).  So in plain mode no tile holding
// an accepted pixel is ever dropped.
__device__ __forceinline__ float ellipse_row_keep_level(const EllipseTiles& E, int ty) {
  const float X = fmaxf(fabsf((float)(kTile * E.x0) - E.u), fabsf((float)min(kTile * E.x1 - 1, E.W - 1) - E.u));
  const float Y = fmaxf(fabsf((float)(kTile * ty) - E.v), fabsf((float)min(kTile * ty + kTile - 1, E.H - 1) - E.v));
  const float S = E.A * X * X + 2.f * fabsf(E.B) * X * Y + E.C * Y * Y;
  return E.Q + 1e-5f * fmaxf(E.Q, 1.f) + 1e-6f * S;
}

__device__ __forceinline__ float tile_min_q(const EllipseTiles& E, int tx, int ty) {
  const float xl = (float)(kTile * tx) - E.u, xh = (float)min(kTile * tx + kTile - 1, E.W - 1) - E.u;
  const float yl = (float)(kTile * ty) - E.v, yh = (float)min(kTile * ty + kTile - 1, E.H - 1) - E.v;
  return rect_min_quad_r(E.A, E.B, E.C, E.iA, E.iC, xl, xh, yl, yh);
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

// Right edge of tile t's pixel-centre span (the last tile is clipped to the image).
__device__ __forceinline__ float tile_right(const EllipseTiles& E, int t) {
  return (float)min(kTile * t + kTile - 1, E.W - 1);
}

// The exact search: the kept tiles of a row are contiguous around the column
// where the row band's minimum of q lies (the minimum of q over a tile
// rectangle is convex in the tile's position); that column, or its neighbour
// across the gap between tiles, decides whether the row has any, and the two
// ends are found with the per-tile test from the guesses gl, gh.
__device__ __forceinline__ void ellipse_row_search(const EllipseTiles& E, float Qk, int ty, float yl, float yh,
                                                   int gl, int gh, int& lo, int& hi) {
  const float dyc = fminf(fmaxf(0.f, yl), yh);      // the band's lowest q: dy closest to 0, dx = -B dy / A
  const float xc = E.u - E.B * dyc * E.iA;
  const float fc = floorf(fminf(fmaxf(xc, -1e9f), 1e9f) / (float)kTile);
  const int tc = min(max((int)fc, E.x0), E.x1 - 1);
  int tb = tc;
  float mb = tile_min_q(E, tc, ty);
  if (xc - (float)(kTile * tc) > (float)(kTile - 1) && tc + 1 < E.x1) {   // minimiser in the gap after tc
    const float m = tile_min_q(E, tc + 1, ty);
    if (m < mb) { mb = m; tb = tc + 1; }
  }
  if (!(mb <= Qk)) return;
  lo = first_kept(E, Qk, ty, E.x0, tb, gl);
  hi = last_kept(E, Qk, ty, tb, E.x1 - 1, gh);
}

// Kept tiles [lo, hi] of tile row ty (lo > hi when none).  A tile is kept when
// its pixel-centre x-span meets the x-range [xl, xr] of the ellipse over the
// row's band of pixel-centre rows, so the closed form of that range (the
// section of a conic, extreme points at dy = -+B sqrt(Q / (det C))) decides
// every tile whose span ends lie clear of xl and xr.  Where an end lies within
// a small margin of a tile edge, or the conic is too ill-conditioned for the
// closed form, the per-tile test decides (ellipse_row_search); both give the
// per-tile test's answer, the closed form only where fp32 cannot tell them apart.
__device__ __forceinline__ void ellipse_row_span(const EllipseTiles& E, int ty, int& lo, int& hi) {
  lo = 1;
  hi = 0;
  if (!(E.Q >= 0.f) || E.x0 >= E.x1) return;
  const float Qk = ellipse_row_keep_level(E, ty);
  const float yl = (float)(kTile * ty) - E.v, yh = (float)min(kTile * ty + kTile - 1, E.H - 1) - E.v;
  // det = AC - B^2 to about an ulp however thin the ellipse (Kahan's fma
  // form: the rounding error of B^2 is recovered exactly and subtracted)
  const float bb = E.B * E.B;
  const float det = __fmaf_rn(E.A, E.C, -bb) - __fmaf_rn(E.B, E.B, -bb);
  if (!(det > 0.f)) {                                // degenerate: search
    ellipse_row_search(E, Qk, ty, yl, yh, E.x0, E.x1 - 1, lo, hi);
    return;
  }
  const float ymax = sqrtf(E.A * Qk / det);         // the ellipse's half-height at the keep level
  const float xmax = sqrtf(E.C * Qk / det);         // and half-width
  // the closed form's fp32 error grows with the ellipse (square roots of
  // differences near its extreme rows); the margin covers it with room to spare
  const float kMargin = 0.02f + 2e-3f * (xmax + ymax);
  const float bl = fmaxf(yl, -ymax), bh = fminf(yh, ymax);
  if (bl > bh + kMargin) return;                     // band clear of the ellipse
  if (bl > bh - kMargin) {                           // band grazes its top or bottom
    ellipse_row_search(E, Qk, ty, yl, yh, E.x0, E.x1 - 1, lo, hi);
    return;
  }
  const float ds = E.B * sqrtf(Qk * E.iC / det);
  const float d1 = fminf(fmaxf(ds, bl), bh), d2 = fminf(fmaxf(-ds, bl), bh);
  const float xl = E.u + (-E.B * d1 - sqrtf(fmaxf(E.A * Qk - det * d1 * d1, 0.f))) * E.iA;
  const float xr = E.u + (-E.B * d2 + sqrtf(fmaxf(E.A * Qk - det * d2 * d2, 0.f))) * E.iA;
  // first tile whose span reaches xl, last whose span starts at or before xr
  int gl = (int)fminf(fmaxf(ceilf((xl - (float)(kTile - 1)) / (float)kTile), -1e6f), 1e6f);
  int gh = (int)fminf(fmaxf(floorf(xr / (float)kTile), -1e6f), 1e6f);
  gl = max(gl, E.x0);
  gh = min(gh, E.x1 - 1);
  if (gl > gh) {                                     // in a gap between spans or outside the square: rare
    ellipse_row_search(E, Qk, ty, yl, yh, E.x0, E.x1 - 1, lo, hi);
    return;
  }
  // a decision is certain when xl, xr lie clear of the span edges around them
  const bool sure_l = gl == E.x0 ? (tile_right(E, gl) - xl > kMargin || xl < (float)(kTile * gl))
                                 : (xl - tile_right(E, gl - 1) > kMargin && tile_right(E, gl) - xl > kMargin);
  const bool sure_h = gh == E.x1 - 1 ? (xr - (float)(kTile * gh) > kMargin || xr > tile_right(E, gh))
                                     : ((float)(kTile * (gh + 1)) - xr > kMargin && xr - (float)(kTile * gh) > kMargin);
  if (sure_l && sure_h) {
    lo = gl;
    hi = gh;
    return;
  }
  ellipse_row_search(E, Qk, ty, yl, yh, gl, gh, lo, hi);
}

}  // namespace ags

namespace ags {

// Kept tiles of the 32 Gaussian-views of a warp (one per lane: E, the first
// row y0 and the number of rows h, h = 0 for none).  Called by the whole warp.
// The rows of all 32 are spread over the lanes, one row per lane per step, the
// owner found by bisection over the warp's row prefix, so that the work does
// not diverge with the Gaussians' sizes.  k_run: 32 words of shared memory.
__device__ __forceinline__ uint32_t warp_ellipse_count(const EllipseTiles& E, int y0, uint32_t h, int lane,
                                                       uint32_t* k_run) {
  uint32_t incl = h;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t start = incl - h, R = __shfl_sync(0xffffffffu, incl, 31);
  k_run[lane] = 0u;
  __syncwarp();
  for (uint32_t k0 = 0; k0 < R; k0 += 32) {
    const uint32_t k = k0 + (uint32_t)lane;
    int own = 0;                                   // the last lane whose rows start at or before k
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      const uint32_t s = __shfl_sync(0xffffffffu, start, own + step);
      if (s <= k) own += step;
    }
    const EllipseTiles Eo{__shfl_sync(0xffffffffu, E.u, own), __shfl_sync(0xffffffffu, E.v, own),
                          __shfl_sync(0xffffffffu, E.A, own), __shfl_sync(0xffffffffu, E.B, own),
                          __shfl_sync(0xffffffffu, E.C, own), __shfl_sync(0xffffffffu, E.Q, own),
                          __shfl_sync(0xffffffffu, E.x0, own), __shfl_sync(0xffffffffu, E.x1, own), E.W, E.H,
                          __shfl_sync(0xffffffffu, E.iA, own), __shfl_sync(0xffffffffu, E.iC, own)};
    const int ty = __shfl_sync(0xffffffffu, y0, own) + (int)(k - __shfl_sync(0xffffffffu, start, own));
    if (k < R) {
      int lo, hi;
      ellipse_row_span(Eo, ty, lo, hi);
      if (lo <= hi) atomicAdd(&k_run[own], (uint32_t)(hi - lo + 1));
    }
  }
  __syncwarp();
  const uint32_t c = k_run[lane];
  __syncwarp();
  return c;
}

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
    ellipse_prepare(E);
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
