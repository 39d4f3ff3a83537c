/*
 * ags_oracle.c -- FP64 CPU oracle of the AdaGScale 3D Gaussian Splatting path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant with the CUDA library; it is a plain, slow restatement of what the
 * paper (AdaGScale, arXiv 2604.18980) and the 3D-GS pipeline it modifies
 * compute, in double precision:
 *
 *   preprocess  (Sec. 2.1: cull, project to 2D mean/covariance, colour, depth)
 *   AdaGScale   (Eq. 9-10 threshold Th, Sec. 3.3 cull when Th > opacity,
 *                adjusted intersection test; Sec. 3.4 T_up look-up table)
 *   tile lists  (Sec. 2.1 pair generation + sort by tile, then depth); the
 *                tiles are those of the square footprint, or (tile_test 1)
 *                those of it that the alpha >= Th ellipse reaches
 *   blending    (Eq. 1 alpha, Eq. 2 front-to-back accumulation with tau and the
 *                1e-4 transmittance stop; always with the original covariance,
 *                Sec. 3.3 "dual-size strategy")
 *   backward    (not in the paper: exact adjoint of the blend with the pair
 *                lists frozen, chained to the raw parameters by forward-mode
 *                jets, i.e. derivatives carried alongside every value)
 *   diagnostics (Eq. 3 contributions, the exact peripheral score of Eq. 4 with
 *                the max-T statistic of Eq. 6, and the contribution-skip
 *                render behind Fig. 4a and Fig. 5)
 *
 * Details the paper leaves to the original 3D-GS (near plane 0.2, EWA Jacobian
 * with the 1.3 tan(fov/2) clamp, +0.3 low-pass, eigenvalue guard 0.1, colour =
 * SH + 0.5 clamped at 0, real SH with the Condon-Shortley phase, alpha clamp
 * 0.99) follow that pipeline.  The SH basis is computed here from the general
 * real-SH formula (Legendre polynomials), not from tabulated constants.
 *
 * Parity pins: see the oracle tests (closed forms, Eq. 9 quadrature, SH
 * orthonormality, brute force vs tiled, invariants, finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_TILE 16
#define NJ 11          /* jet directions: mean 0-2, log_scale 3-5, quat 6-9, logit 10 */

/* ------------------------------------------------------------------------ */
/* Public structures (mirrored by oracle/__init__.py with ctypes).           */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t width, height;
  double fx, fy, cx, cy;
  double R[9];      /* row-major world->camera rotation */
  double t[3];      /* world->camera translation */
  double campos[3];
  double near_z;
} oc_camera;

typedef struct {
  int32_t scale_mode;     /* 0 plain 3-sigma, 1 AdaGScale */
  int32_t sh_degree;      /* 0..3 */
  int32_t lut_bins;       /* <= 32 */
  int32_t tile_test;      /* 0 square footprint, 1 square and ellipse */
  double K, tau, t_min, alpha_max;
  double lut_depth_max;
  double lut[32];
  double bg[3];
  double edge_rel;        /* relative width of the discrete-decision edge class */
  double pos_err;         /* absolute pixel-position error allowed for alpha-vs-tau edges */
} oc_params;

/* Per-Gaussian double outputs. */
enum {
  F_U = 0, F_V, F_A, F_B, F_C, F_OPAC, F_R, F_G, F_BL, F_DEPTH, F_TH, F_DET, F_LAMBDA,
  F_COVA, F_COVB, F_COVC, F_DEPTH32, F_RARG,
  F_QELL,   /* ellipse level Q = 2 ln(opacity / Th) of the tile test, NaN for the square test */
  OC_NF
};
/* Per-Gaussian integer outputs. */
enum { I_RADIUS = 0, I_X0, I_Y0, I_X1, I_Y1, I_TOUCHED, I_CULL, I_EDGE, I_CLAMP,
       I_GEDGE,   /* decisions that change only the derivatives (bits below) */
       OC_NI };

/* cull reasons */
#define CULL_NONE 0
#define CULL_NEAR 1
#define CULL_DET 2
#define CULL_TH 3
#define CULL_TUP 4
#define CULL_NONFINITE 5
#define CULL_EMPTY 6   /* radius 0 or empty rectangle: no pairs */

/* edge-class bits */
#define EDGE_NEAR 1
#define EDGE_DET 2
#define EDGE_TH 4
#define EDGE_CEIL 8
#define EDGE_RECT 16
#define EDGE_LUT 32
#define EDGE_ELLIPSE 64

/* gradient-only edge bits (I_GEDGE): the image is continuous across these
 * decisions, its derivative is not */
#define GEDGE_FRUSTUM 1   /* x/z or y/z within eps of the 1.3 tan(fov/2) clamp */
#define GEDGE_COLOUR 2    /* a colour channel within eps of the clamp at 0 */

/* ------------------------------------------------------------------------ */
/* Jets: value plus NJ partial derivatives.                                   */
/* ------------------------------------------------------------------------ */
typedef struct { double v; double d[NJ]; } jet;

static jet jc(double x) { jet r; r.v = x; memset(r.d, 0, sizeof r.d); return r; }
static jet jvar(double x, int k) { jet r = jc(x); r.d[k] = 1.0; return r; }
static jet jadd(jet a, jet b) { jet r; r.v = a.v + b.v; for (int k = 0; k < NJ; k++) r.d[k] = a.d[k] + b.d[k]; return r; }
static jet jsub(jet a, jet b) { jet r; r.v = a.v - b.v; for (int k = 0; k < NJ; k++) r.d[k] = a.d[k] - b.d[k]; return r; }
static jet jmul(jet a, jet b) {
  jet r; r.v = a.v * b.v;
  for (int k = 0; k < NJ; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
static jet jscale(jet a, double s) { jet r; r.v = a.v * s; for (int k = 0; k < NJ; k++) r.d[k] = a.d[k] * s; return r; }
static jet jaddc(jet a, double c) { a.v += c; return a; }
static jet jdiv(jet a, jet b) {
  jet r; r.v = a.v / b.v;
  for (int k = 0; k < NJ; k++) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
  return r;
}
static jet jsqrt(jet a) {
  jet r; r.v = sqrt(a.v);
  for (int k = 0; k < NJ; k++) r.d[k] = a.d[k] / (2.0 * r.v);
  return r;
}
static jet jexp(jet a) { jet r; r.v = exp(a.v); for (int k = 0; k < NJ; k++) r.d[k] = a.d[k] * r.v; return r; }

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics from the general formula.                        */
/*   Y_l^0  = K_l^0 P_l(z)                                                   */
/*   Y_l^m  = sqrt2 K_l^m (-1)^m P_l^(m)(z) Re((x+iy)^m)      m > 0         */
/*   Y_l^-m = sqrt2 K_l^m (-1)^m P_l^(m)(z) Im((x+iy)^m)      m > 0         */
/* with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) and P_l^(m) the m-th       */
/* derivative of the Legendre polynomial; (-1)^m is the Condon-Shortley      */
/* phase.  Coefficient index: l*l + l + m.                                   */
/* ------------------------------------------------------------------------ */
static double factorial(int n) { double f = 1; for (int i = 2; i <= n; i++) f *= i; return f; }
static double binom(int n, int k) { return factorial(n) / (factorial(k) * factorial(n - k)); }

/* coefficients c[j] of z^j in d^m/dz^m P_l(z) */
static void legendre_deriv_coeffs(int l, int m, double* c) {
  double p[8] = {0};
  for (int k = 0; 2 * k <= l; k++)
    p[l - 2 * k] = ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l) / ldexp(1.0, l);
  for (int it = 0; it < m; it++) {
    for (int j = 0; j < 7; j++) p[j] = p[j + 1] * (j + 1);
    p[7] = 0;
  }
  for (int j = 0; j < 8; j++) c[j] = p[j];
}

static void sh_basis_jet(int degree, jet x, jet y, jet z, jet* Y) {
  for (int l = 0; l <= degree; l++) {
    for (int m = 0; m <= l; m++) {
      double c[8];
      legendre_deriv_coeffs(l, m, c);
      jet pz = jc(0.0), zp = jc(1.0);
      for (int j = 0; j <= l; j++) { pz = jadd(pz, jscale(zp, c[j])); zp = jmul(zp, z); }
      double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
      if (m == 0) { Y[l * l + l] = jscale(pz, K); continue; }
      jet re = jc(1.0), im = jc(0.0);
      for (int j = 0; j < m; j++) {   /* (re + i im) *= (x + i y) */
        jet nre = jsub(jmul(re, x), jmul(im, y));
        jet nim = jadd(jmul(re, y), jmul(im, x));
        re = nre; im = nim;
      }
      double s = sqrt(2.0) * K * ((m & 1) ? -1.0 : 1.0);
      Y[l * l + l + m] = jscale(jmul(pz, re), s);
      Y[l * l + l - m] = jscale(jmul(pz, im), s);
    }
  }
}

/* Plain-double SH basis for a direction (exposed for the orthonormality pin). */
void oracle_sh_basis(int degree, double x, double y, double z, double* out) {
  jet Y[16];
  sh_basis_jet(degree, jc(x), jc(y), jc(z), Y);
  int nc = (degree + 1) * (degree + 1);
  for (int i = 0; i < nc; i++) out[i] = Y[i].v;
}

/* ------------------------------------------------------------------------ */
/* Preprocess of one Gaussian, all quantities as jets.                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  jet u, v, A, B, C, opac, rgb[3];
  jet Y[16];         /* SH basis at the view direction */
  int clamp[3];
} gjet;

static int all_finite(const double* p, int64_t n, int64_t i, int rows) {
  for (int r = 0; r < rows; r++) if (!isfinite((double)p[r * n + i])) return 0;
  return 1;
}

/* Tiles [t0,t1) covering the pixel centres in [lo, hi] of an axis of `len`
 * pixels.  Returns 1 when the answer changes if lo and hi move by +-slack
 * (the edge class of this decision). */
static void span_tiles_exact(double lo, double hi, int len, int* t0, int* t1) {
  double plo = ceil(lo), phi = floor(hi);
  if (plo < 0) plo = 0;
  if (phi > len - 1) phi = len - 1;
  if (plo > phi) { *t0 = 0; *t1 = 0; return; }
  *t0 = (int)plo / OC_TILE;
  *t1 = (int)phi / OC_TILE + 1;
}
static int span_tiles(double lo, double hi, int len, double slack, int* t0, int* t1) {
  int a0, a1, b0, b1, c0, c1, d0, d1;
  span_tiles_exact(lo, hi, len, t0, t1);
  span_tiles_exact(lo - slack, hi - slack, len, &a0, &a1);
  span_tiles_exact(lo + slack, hi + slack, len, &b0, &b1);
  span_tiles_exact(lo - slack, hi + slack, len, &c0, &c1);
  span_tiles_exact(lo + slack, hi - slack, len, &d0, &d1);
  return !(a0 == *t0 && a1 == *t1 && b0 == *t0 && b1 == *t1 && c0 == *t0 && c1 == *t1 && d0 == *t0 && d1 == *t1);
}

/* edge test: is |a - b| within rel * scale ? */
static int near_edge(double a, double b, double rel, double scale) {
  return fabs(a - b) <= rel * scale;
}

/* Minimum of the conic's quadratic form q(x, y) = A x^2 + 2 B x y + C y^2
 * (positive definite) over the rectangle [xl, xh] x [yl, yh] of offsets from
 * the Gaussian's centre.  Zero when the rectangle holds the centre; otherwise
 * the minimum of a convex function over a rectangle lies on its boundary, and
 * along each edge q is a parabola in the free coordinate whose vertex, clamped
 * to the edge, gives that edge's minimum. */
static double rect_min_form(double A, double B, double C, double xl, double xh, double yl, double yh) {
  if (xl <= 0.0 && xh >= 0.0 && yl <= 0.0 && yh >= 0.0) return 0.0;
  double best = INFINITY;
  const double xs[2] = {xl, xh}, ys[2] = {yl, yh};
  for (int k = 0; k < 2; k++) {
    double x = xs[k];
    double y = fmin(fmax(-B * x / C, yl), yh);          /* vertex of q(x, .) */
    best = fmin(best, A * x * x + 2.0 * B * x * y + C * y * y);
    y = ys[k];
    x = fmin(fmax(-B * y / A, xl), xh);                 /* vertex of q(., y) */
    best = fmin(best, A * x * x + 2.0 * B * x * y + C * y * y);
  }
  return best;
}

/* Ellipse tile test (the exact footprint-tile intersection the paper's
 * implementation builds on; our reading for tile_test 1): tile (tx, ty) is kept
 * when some point of the rectangle spanned by its pixel centres (clipped to
 * the image) has alpha >= Th with the blending conic, i.e. q <= Q with
 * Q = 2 ln(opacity / Th), Th = tau in plain mode.  Returns the minimum of q
 * over that rectangle. */
static double tile_min_form(const double* g, int tx, int ty, int width, int height) {
  double xl = OC_TILE * tx - g[F_U], xh = fmin(OC_TILE * tx + OC_TILE - 1, width - 1) - g[F_U];
  double yl = OC_TILE * ty - g[F_V], yh = fmin(OC_TILE * ty + OC_TILE - 1, height - 1) - g[F_V];
  return rect_min_form(g[F_A], g[F_B], g[F_C], xl, xh, yl, yh);
}

static int tile_kept(const double* g, int tx, int ty, int width, int height) {
  double Q = g[F_QELL];
  if (isnan(Q)) return 1;
  return tile_min_form(g, tx, ty, width, height) <= Q;
}

/* Returns cull reason; fills dbl[OC_NF], irec[OC_NI] and (optionally) the jets. */
static int preprocess_one(const double* mean, const double* log_scale, const double* quat,
                          const double* logit, const double* sh, int64_t n, int64_t i,
                          const oc_camera* cam, const oc_params* par, double* dbl,
                          int32_t* irec, gjet* gj) {
  memset(dbl, 0, sizeof(double) * OC_NF);
  memset(irec, 0, sizeof(int32_t) * OC_NI);
  int nc = (par->sh_degree + 1) * (par->sh_degree + 1);
  if (!all_finite(mean, n, i, 3) || !all_finite(log_scale, n, i, 3) || !all_finite(quat, n, i, 4) ||
      !all_finite(logit, n, i, 1) || !all_finite(sh, n, i, 3 * nc)) {
    irec[I_CULL] = CULL_NONFINITE;
    return CULL_NONFINITE;
  }
  const double eps = par->edge_rel;
  int edge = 0;
  jet m[3];
  for (int k = 0; k < 3; k++) m[k] = jvar(mean[k * n + i], k);

  /* view-space position t = R m + t_cam.  The edge classes take t as the
   * fp32 inputs give it exactly (a correctly rounded fp32 evaluation is within
   * one rounding of it), so each band is eps relative to the magnitudes of the
   * compared quantities themselves. */
  jet t[3];
  for (int r = 0; r < 3; r++) {
    t[r] = jc(cam->t[r]);
    for (int k = 0; k < 3; k++) t[r] = jadd(t[r], jscale(m[k], cam->R[r * 3 + k]));
  }
  if (near_edge(t[2].v, cam->near_z, eps, fmax(fabs(t[2].v), cam->near_z))) edge |= EDGE_NEAR;
  irec[I_EDGE] = edge;
  dbl[F_DEPTH] = t[2].v;
  dbl[F_DEPTH32] = (double)(float)t[2].v;
  if (!(t[2].v > cam->near_z)) { irec[I_CULL] = CULL_NEAR; return CULL_NEAR; }

  /* 3D covariance: Sigma = Rq S S Rq^T, q normalised, S = diag(exp(log_scale)) */
  jet s[3], q[4];
  for (int k = 0; k < 3; k++) s[k] = jexp(jvar(log_scale[k * n + i], 3 + k));
  for (int k = 0; k < 4; k++) q[k] = jvar(quat[k * n + i], 6 + k);
  jet qn2 = jadd(jadd(jmul(q[0], q[0]), jmul(q[1], q[1])), jadd(jmul(q[2], q[2]), jmul(q[3], q[3])));
  jet qn = jsqrt(qn2);
  jet w = jdiv(q[0], qn), x = jdiv(q[1], qn), y = jdiv(q[2], qn), z = jdiv(q[3], qn);
  jet Rq[9];
  Rq[0] = jsub(jc(1.0), jscale(jadd(jmul(y, y), jmul(z, z)), 2.0));
  Rq[1] = jscale(jsub(jmul(x, y), jmul(w, z)), 2.0);
  Rq[2] = jscale(jadd(jmul(x, z), jmul(w, y)), 2.0);
  Rq[3] = jscale(jadd(jmul(x, y), jmul(w, z)), 2.0);
  Rq[4] = jsub(jc(1.0), jscale(jadd(jmul(x, x), jmul(z, z)), 2.0));
  Rq[5] = jscale(jsub(jmul(y, z), jmul(w, x)), 2.0);
  Rq[6] = jscale(jsub(jmul(x, z), jmul(w, y)), 2.0);
  Rq[7] = jscale(jadd(jmul(y, z), jmul(w, x)), 2.0);
  Rq[8] = jsub(jc(1.0), jscale(jadd(jmul(x, x), jmul(y, y)), 2.0));
  jet S3[9];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      jet acc = jc(0.0);
      for (int k = 0; k < 3; k++) acc = jadd(acc, jmul(jmul(Rq[a * 3 + k], Rq[b * 3 + k]), jmul(s[k], s[k])));
      S3[a * 3 + b] = acc;
    }

  /* EWA: J (with the 1.3 tan(fov/2) frustum clamp on x/z, y/z), W = camera rotation */
  double limx = 1.3 * (0.5 * cam->width / cam->fx);
  double limy = 1.3 * (0.5 * cam->height / cam->fy);
  jet txtz = jdiv(t[0], t[2]), tytz = jdiv(t[1], t[2]);
  jet tx = t[0], ty = t[1];
  int fclamp = 0;
  if (near_edge(fabs(txtz.v), limx, eps, limx) || near_edge(fabs(tytz.v), limy, eps, limy))
    irec[I_GEDGE] |= GEDGE_FRUSTUM;
  if (txtz.v > limx) { tx = jscale(t[2], limx); fclamp |= 8; }
  else if (txtz.v < -limx) { tx = jscale(t[2], -limx); fclamp |= 8; }
  if (tytz.v > limy) { ty = jscale(t[2], limy); fclamp |= 16; }
  else if (tytz.v < -limy) { ty = jscale(t[2], -limy); fclamp |= 16; }
  jet iz = jdiv(jc(1.0), t[2]);
  jet iz2 = jmul(iz, iz);
  jet J[6];
  J[0] = jscale(iz, cam->fx); J[1] = jc(0.0); J[2] = jscale(jmul(tx, iz2), -cam->fx);
  J[3] = jc(0.0); J[4] = jscale(iz, cam->fy); J[5] = jscale(jmul(ty, iz2), -cam->fy);
  jet T[6];   /* T = J W */
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 3; b++) {
      jet acc = jc(0.0);
      for (int k = 0; k < 3; k++) acc = jadd(acc, jscale(J[a * 3 + k], cam->R[k * 3 + b]));
      T[a * 3 + b] = acc;
    }
  jet S2[4];  /* T S3 T^T */
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++) {
      jet acc = jc(0.0);
      for (int k = 0; k < 3; k++)
        for (int l = 0; l < 3; l++) acc = jadd(acc, jmul(jmul(T[a * 3 + k], S3[k * 3 + l]), T[b * 3 + l]));
      S2[a * 2 + b] = acc;
    }
  jet ca = jaddc(S2[0], 0.3), cb = S2[1], cc = jaddc(S2[3], 0.3);
  jet det = jsub(jmul(ca, cc), jmul(cb, cb));
  dbl[F_COVA] = ca.v; dbl[F_COVB] = cb.v; dbl[F_COVC] = cc.v; dbl[F_DET] = det.v;
  if (near_edge(det.v, 0.0, eps, fabs(ca.v * cc.v) + cb.v * cb.v)) edge |= EDGE_DET;
  irec[I_EDGE] = edge;
  if (!(det.v > 0.0)) { irec[I_CULL] = CULL_DET; return CULL_DET; }
  jet A = jdiv(cc, det), B = jscale(jdiv(cb, det), -1.0), C = jdiv(ca, det);

  /* largest eigenvalue with the 0.1 guard, and the plain 3-sigma radius */
  double mid = 0.5 * (ca.v + cc.v);
  double lam1 = mid + sqrt(fmax(0.1, mid * mid - det.v));
  dbl[F_LAMBDA] = lam1;

  /* 2D mean (unclamped projection), depth */
  jet u = jaddc(jscale(jmul(t[0], iz), cam->fx), cam->cx);
  jet v = jaddc(jscale(jmul(t[1], iz), cam->fy), cam->cy);
  double uscale = fabs(cam->fx * t[0].v / t[2].v) + fabs(cam->cx);
  double vscale = fabs(cam->fy * t[1].v / t[2].v) + fabs(cam->cy);

  /* opacity */
  jet opac = jdiv(jc(1.0), jaddc(jexp(jscale(jvar(logit[i], 10), -1.0)), 1.0));

  /* colour: SH evaluated at the world-space direction from the camera */
  jet dx = jaddc(m[0], -cam->campos[0]), dy = jaddc(m[1], -cam->campos[1]), dz = jaddc(m[2], -cam->campos[2]);
  jet dn = jsqrt(jadd(jadd(jmul(dx, dx), jmul(dy, dy)), jmul(dz, dz)));
  jet Y[16];
  sh_basis_jet(par->sh_degree, jdiv(dx, dn), jdiv(dy, dn), jdiv(dz, dn), Y);
  jet rgb[3];
  int clampbits = fclamp;
  for (int c = 0; c < 3; c++) {
    jet acc = jc(0.5);
    double mag = 0.5;
    for (int k = 0; k < nc; k++) {
      acc = jadd(acc, jscale(Y[k], sh[(k * 3 + c) * n + i]));
      mag += fabs(Y[k].v * sh[(k * 3 + c) * n + i]);
    }
    if (fabs(acc.v) <= eps * mag) irec[I_GEDGE] |= GEDGE_COLOUR;
    if (acc.v < 0.0) { acc = jc(0.0); clampbits |= 1 << c; }
    rgb[c] = acc;
  }

  /* AdaGScale threshold (Eq. 10) and adjusted radius, or the plain 3-sigma radius */
  double th = par->tau;
  double rarg, rarg_lo, rarg_hi;
  int radius;
  if (par->scale_mode == 1) {
    double binw = par->lut_depth_max / par->lut_bins;
    double fb = t[2].v / binw;
    int bin = (int)floor(fb);
    if (bin > par->lut_bins - 1) bin = par->lut_bins - 1;
    if (bin < 0) bin = 0;
    double fr = floor(fb + 0.5);
    if (fr >= 1.0 && fr <= par->lut_bins - 1 && near_edge(fb, fr, eps, fmax(fabs(fb), 1.0))) edge |= EDGE_LUT;
    double tup = par->lut[bin];
    if (!(tup > 0.0)) {
      irec[I_EDGE] = edge; irec[I_CULL] = CULL_TUP; dbl[F_TH] = INFINITY; return CULL_TUP;
    }
    double sd = sqrt(det.v);
    th = par->K / (tup * 2.0 * M_PI * sd) + par->tau;
    dbl[F_TH] = th;
    if (near_edge(th, opac.v, eps, fmax(th, opac.v))) edge |= EDGE_TH;
    if (th > opac.v) { irec[I_EDGE] = edge; irec[I_CULL] = CULL_TH; return CULL_TH; }
    rarg = sqrt(lam1) * fmin(3.0, sqrt(2.0 * log(opac.v / th)));
    /* same decision with every input nudged by eps in each direction */
    double thl = par->K / (tup * 2.0 * M_PI * sd * (1 + eps)) + par->tau;
    double thh = par->K / (tup * 2.0 * M_PI * sd * (1 - eps)) + par->tau;
    double ol = opac.v * (1 - eps), oh = opac.v * (1 + eps);
    rarg_hi = sqrt(lam1 * (1 + eps)) * fmin(3.0, sqrt(2.0 * log(fmax(oh / thl, 1.0))));
    rarg_lo = sqrt(lam1 * (1 - eps)) * fmin(3.0, sqrt(2.0 * log(fmax(ol / thh, 1.0))));
  } else {
    dbl[F_TH] = th;
    rarg = 3.0 * sqrt(lam1);
    rarg_hi = 3.0 * sqrt(lam1 * (1 + eps));
    rarg_lo = 3.0 * sqrt(lam1 * (1 - eps));
  }
  radius = (int)ceil(rarg);
  if ((int)ceil(rarg_hi) != (int)ceil(rarg_lo)) edge |= EDGE_CEIL;
  dbl[F_RARG] = rarg;

  /* Tile rectangle [x0,x1) x [y0,y1): every tile that holds a pixel centre
   * (integer coordinates) inside the square [u-r, u+r] x [v-r, v+r]. */
  int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
  double su = eps * uscale, sv = eps * vscale;
  if (span_tiles(u.v - radius, u.v + radius, cam->width, su, &x0, &x1)) edge |= EDGE_RECT;
  if (span_tiles(v.v - radius, v.v + radius, cam->height, sv, &y0, &y1)) edge |= EDGE_RECT;

  dbl[F_U] = u.v; dbl[F_V] = v.v; dbl[F_A] = A.v; dbl[F_B] = B.v; dbl[F_C] = C.v;
  dbl[F_OPAC] = opac.v; dbl[F_R] = rgb[0].v; dbl[F_G] = rgb[1].v; dbl[F_BL] = rgb[2].v;
  irec[I_RADIUS] = radius;
  irec[I_X0] = x0; irec[I_Y0] = y0; irec[I_X1] = x1; irec[I_Y1] = y1;
  irec[I_CLAMP] = clampbits;
  irec[I_EDGE] = edge;
  if (gj) {
    gj->u = u; gj->v = v; gj->A = A; gj->B = B; gj->C = C; gj->opac = opac;
    for (int c = 0; c < 3; c++) { gj->rgb[c] = rgb[c]; gj->clamp[c] = (clampbits >> c) & 1; }
    for (int k = 0; k < nc; k++) gj->Y[k] = Y[k];
  }
  int64_t area = (int64_t)(x1 - x0) * (y1 - y0);
  dbl[F_QELL] = NAN;
  if (par->tile_test == 1 && radius > 0 && area > 0) {
    /* keep the tiles of the square that the alpha >= Th ellipse reaches; a
     * decision within the edge width of Q marks the Gaussian an edge case
     * (its conic and position carry fp32 rounding on the GPU: Q's relative
     * width plus the position error times |grad q| = 2 sqrt(q * lambda)) */
    double Q = 2.0 * log(opac.v / th);
    dbl[F_QELL] = Q;
    int64_t kept = 0;
    for (int ty = y0; ty < y1; ty++) {
      /* the GPU's keep margin grows with S, the size of q's terms over the
       * row's part of the square before they cancel (thin, tilted ellipses):
       * decisions within 2e-6 S of Q are edge cases too */
      double X = fmax(fabs(OC_TILE * x0 - u.v), fabs(fmin(OC_TILE * x1 - 1, cam->width - 1) - u.v));
      double Y = fmax(fabs(OC_TILE * ty - v.v), fabs(fmin(OC_TILE * ty + OC_TILE - 1, cam->height - 1) - v.v));
      double S = A.v * X * X + 2.0 * fabs(B.v) * X * Y + C.v * Y * Y;
      for (int tx = x0; tx < x1; tx++) {
        double m = tile_min_form(dbl, tx, ty, cam->width, cam->height);
        if (m <= Q) kept++;
        double tol = eps * fmax(Q, 1.0) + 2.0 * par->pos_err * sqrt((A.v + C.v) * fmax(fmax(Q, m), 0.0)) + 2e-6 * S;
        if (fabs(m - Q) <= tol) edge |= EDGE_ELLIPSE;
      }
    }
    irec[I_EDGE] = edge;
    area = kept;
  }
  if (radius <= 0 || area <= 0) { irec[I_CULL] = CULL_EMPTY; return CULL_EMPTY; }
  irec[I_TOUCHED] = (int32_t)area;
  return CULL_NONE;
}

void oracle_preprocess(const double* mean, const double* log_scale, const double* quat,
                       const double* logit, const double* sh, int64_t n,
                       const oc_camera* cam, const oc_params* par, double* dbl, int32_t* irec) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; i++)
    preprocess_one(mean, log_scale, quat, logit, sh, n, i, cam, par, dbl + i * OC_NF, irec + i * OC_NI, NULL);
}

/* ------------------------------------------------------------------------ */
/* Tile lists: every Gaussian (in id order) appends itself to every tile of  */
/* its rectangle (row-major), then each tile's list is sorted by the fp32     */
/* depth and Gaussian id.  Two calls: counts (ids == NULL), then fill.        */
/* ------------------------------------------------------------------------ */
typedef struct { float depth; int32_t id; } oc_pair;

static int cmp_pair(const void* a, const void* b) {
  const oc_pair* x = (const oc_pair*)a;
  const oc_pair* y = (const oc_pair*)b;
  if (x->depth < y->depth) return -1;
  if (x->depth > y->depth) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* tile_start has num_tiles+1 entries; returns the number of pairs.  tile_mask
 * (nullable, [num_tiles]) restricts the lists to the selected tiles (the
 * others stay empty), so large scenes can be checked on a sample of tiles. */
int64_t oracle_tile_lists(int64_t n, const double* dbl, const int32_t* irec, int32_t width,
                          int32_t height, const uint8_t* tile_mask, int64_t* tile_start, int32_t* ids) {
  int gx = (width + OC_TILE - 1) / OC_TILE, gy = (height + OC_TILE - 1) / OC_TILE;
  int64_t nt = (int64_t)gx * gy;
  int64_t* cnt = (int64_t*)calloc(nt, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) {
    const int32_t* r = irec + i * OC_NI;
    if (r[I_TOUCHED] <= 0) continue;
    for (int ty = r[I_Y0]; ty < r[I_Y1]; ty++)
      for (int tx = r[I_X0]; tx < r[I_X1]; tx++) {
        int64_t t = (int64_t)ty * gx + tx;
        if ((!tile_mask || tile_mask[t]) && tile_kept(dbl + i * OC_NF, tx, ty, width, height)) cnt[t]++;
      }
  }
  tile_start[0] = 0;
  for (int64_t t = 0; t < nt; t++) tile_start[t + 1] = tile_start[t] + cnt[t];
  int64_t total = tile_start[nt];
  if (ids) {
    oc_pair* pairs = (oc_pair*)malloc(sizeof(oc_pair) * (total > 0 ? total : 1));
    memset(cnt, 0, sizeof(int64_t) * nt);
    for (int64_t i = 0; i < n; i++) {
      const int32_t* r = irec + i * OC_NI;
      if (r[I_TOUCHED] <= 0) continue;
      float d = (float)dbl[i * OC_NF + F_DEPTH];
      for (int ty = r[I_Y0]; ty < r[I_Y1]; ty++)
        for (int tx = r[I_X0]; tx < r[I_X1]; tx++) {
          int64_t t = (int64_t)ty * gx + tx;
          if (tile_mask && !tile_mask[t]) continue;
          if (!tile_kept(dbl + i * OC_NF, tx, ty, width, height)) continue;
          oc_pair* p = &pairs[tile_start[t] + cnt[t]++];
          p->depth = d;
          p->id = (int32_t)i;
        }
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++)
      qsort(pairs + tile_start[t], (size_t)(tile_start[t + 1] - tile_start[t]), sizeof(oc_pair), cmp_pair);
    for (int64_t k = 0; k < total; k++) ids[k] = pairs[k].id;
    free(pairs);
  }
  free(cnt);
  return total;
}

/* ------------------------------------------------------------------------ */
/* Blending of one pixel over one depth-ordered list (Eq. 1, Eq. 2).          */
/* ------------------------------------------------------------------------ */
typedef struct {
  double col[3];
  double T;
  int32_t n_contrib;     /* 1-based position of the last blended entry */
  int32_t n_blend;       /* number of blended entries */
  int32_t n_clamp;       /* number of blended entries with alpha clamped at alpha_max */
  int32_t n_eval;        /* entries evaluated: up to and including the one it stopped at, else all */
  double budget;         /* bound on the change a near-threshold flip can cause */
} oc_pix;

static void blend_pixel(double px, double py, const int32_t* list, int64_t len, const double* dbl,
                        const oc_params* par, double cmax, double* maxT, oc_pix* out) {
  double T = 1.0, col[3] = {0, 0, 0}, budget = 0.0;
  int32_t last = 0, nb = 0, ncl = 0, nev = (int32_t)len;
  for (int64_t k = 0; k < len; k++) {
    const double* g = dbl + (int64_t)list[k] * OC_NF;
    double dx = g[F_U] - px, dy = g[F_V] - py;
    double p = -0.5 * (g[F_A] * dx * dx + g[F_C] * dy * dy) - g[F_B] * dx * dy;
    double araw = g[F_OPAC] * exp(p);
    double alpha = fmin(par->alpha_max, araw);
    /* edge class: alpha within (edge_rel + fp32 position error x |grad ln alpha|) of tau */
    double gl = fabs(g[F_A] * dx + g[F_B] * dy) + fabs(g[F_B] * dx + g[F_C] * dy);
    double tol = par->edge_rel + par->pos_err * gl;
    if (araw > 0.0 && fabs(log(araw / par->tau)) <= tol) budget += 2.0 * par->tau * T * cmax;
    if (fabs(p) <= par->edge_rel && g[F_OPAC] >= par->tau) budget += 2.0 * g[F_OPAC] * T * cmax;
    if (p > 0.0) continue;
    if (alpha < par->tau) continue;
    double test_T = T * (1.0 - alpha);
    if (test_T < par->t_min) { nev = (int32_t)(k + 1); break; }
    col[0] += g[F_R] * alpha * T;
    col[1] += g[F_G] * alpha * T;
    col[2] += g[F_BL] * alpha * T;
    if (maxT) {   /* per-Gaussian max transmittance before blending (T_up calibration) */
      uint64_t* slot = (uint64_t*)&maxT[list[k]];
      uint64_t expect = __atomic_load_n(slot, __ATOMIC_RELAXED), desired;
      double cur;
      memcpy(&cur, &expect, 8);
      memcpy(&desired, &T, 8);
      while (T > cur) {
        if (__atomic_compare_exchange_n(slot, &expect, desired, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED))
          break;
        memcpy(&cur, &expect, 8);
      }
    }
    T = test_T;
    last = (int32_t)(k + 1);
    nb++;
    ncl += araw > par->alpha_max;
  }
  for (int c = 0; c < 3; c++) out->col[c] = col[c] + T * par->bg[c];
  out->T = T;
  out->n_contrib = last;
  out->n_blend = nb;
  out->n_clamp = ncl;
  out->n_eval = nev;
  out->budget = budget;
}

static double color_max(int64_t n, const double* dbl, const oc_params* par) {
  double cm = 1.0;
  for (int c = 0; c < 3; c++) cm = fmax(cm, par->bg[c]);
  for (int64_t i = 0; i < n; i++)
    for (int c = 0; c < 3; c++) cm = fmax(cm, dbl[i * OC_NF + F_R + c]);
  return cm;
}

/* Tiled render.  tile_mask (nullable, [num_tiles]) selects the tiles to blend;
 * image [3][H][W], final_T [H][W], n_contrib [H][W], budget [H][W] (nullable),
 * maxT [n] (nullable; zero it first), state (nullable). */
void oracle_rasterize(int64_t n, const double* dbl, const int64_t* tile_start, const int32_t* ids,
                      int32_t width, int32_t height, const oc_params* par, const uint8_t* tile_mask,
                      double* image, double* final_T, int32_t* n_contrib, double* budget, double* maxT,
                      int32_t* state /* [H][W][3] nullable: blended, clamped and evaluated counts */) {
  int gx = (width + OC_TILE - 1) / OC_TILE, gy = (height + OC_TILE - 1) / OC_TILE;
  int64_t nt = (int64_t)gx * gy;
  int64_t hw = (int64_t)width * height;
  double cmax = color_max(n, dbl, par);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < nt; t++) {
    if (tile_mask && !tile_mask[t]) continue;
    int tx = (int)(t % gx), ty = (int)(t / gx);
    for (int y = ty * OC_TILE; y < ty * OC_TILE + OC_TILE && y < height; y++)
      for (int x = tx * OC_TILE; x < tx * OC_TILE + OC_TILE && x < width; x++) {
        oc_pix pix;
        blend_pixel((double)x, (double)y, ids + tile_start[t], tile_start[t + 1] - tile_start[t], dbl, par,
                    cmax, maxT, &pix);
        int64_t o = (int64_t)y * width + x;
        for (int c = 0; c < 3; c++) image[c * hw + o] = pix.col[c];
        if (final_T) final_T[o] = pix.T;
        if (n_contrib) n_contrib[o] = pix.n_contrib;
        if (budget) budget[o] = pix.budget;
        if (state) { state[3 * o] = pix.n_blend; state[3 * o + 1] = pix.n_clamp; state[3 * o + 2] = pix.n_eval; }
      }
  }
}

/* Brute force: no tile lists and no key sort.  Every pixel takes every
 * Gaussian whose rectangle holds the pixel's tile (and whose ellipse reaches
 * it, with tile_test 1), orders them globally by (fp32 depth, id) and blends. */
void oracle_render_bruteforce(int64_t n, const double* dbl, const int32_t* irec, int32_t width,
                              int32_t height, const oc_params* par, double* image) {
  oc_pair* all = (oc_pair*)malloc(sizeof(oc_pair) * (n > 0 ? n : 1));
  int64_t m = 0;
  for (int64_t i = 0; i < n; i++) {
    if (irec[i * OC_NI + I_TOUCHED] <= 0) continue;
    all[m].depth = (float)dbl[i * OC_NF + F_DEPTH];
    all[m].id = (int32_t)i;
    m++;
  }
  qsort(all, (size_t)m, sizeof(oc_pair), cmp_pair);
  int64_t hw = (int64_t)width * height;
  double cmax = color_max(n, dbl, par);
#pragma omp parallel for schedule(dynamic, 4)
  for (int y = 0; y < height; y++) {
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (m > 0 ? m : 1));
    for (int x = 0; x < width; x++) {
      int tx = x / OC_TILE, ty = y / OC_TILE;
      int64_t len = 0;
      for (int64_t k = 0; k < m; k++) {
        const int32_t* r = irec + (int64_t)all[k].id * OC_NI;
        if (tx >= r[I_X0] && tx < r[I_X1] && ty >= r[I_Y0] && ty < r[I_Y1] &&
            tile_kept(dbl + (int64_t)all[k].id * OC_NF, tx, ty, width, height))
          list[len++] = all[k].id;
      }
      oc_pix pix;
      blend_pixel((double)x, (double)y, list, len, dbl, par, cmax, NULL, &pix);
      for (int c = 0; c < 3; c++) image[c * hw + (int64_t)y * width + x] = pix.col[c];
    }
    free(list);
  }
  free(all);
}

static void atomic_add_double(double* p, double v) {
#pragma omp atomic
  *p += v;
}

static void atomic_max_double(double* p, double v) {
#pragma omp critical(oc_max)
  if (v > *p) *p = v;
}

/* ------------------------------------------------------------------------ */
/* Peripheral-score diagnostics (Sec. 2.2 Eq. 3, Sec. 3.1 Eq. 4, Sec. 3.2     */
/* Eq. 6-7, Fig. 4a and Fig. 5).                                              */
/*                                                                            */
/* Both functions replay the blend of the given (plain) tile lists pixel by   */
/* pixel, with the decisions of blend_pixel: Gaussian i is blended at pixel k */
/* when alpha >= tau and p <= 0, before the stop T (1 - alpha) < t_min.  Its  */
/* contribution there is alpha * T (Eq. 3), T the transmittance before it.    */
/* ------------------------------------------------------------------------ */

/* Eq. 4 at the level x_i = level[i]: ps[i] = sum of alpha * T over the pixels
 * where i is blended with alpha < level[i]; sum_alpha[i] = sum of alpha over
 * the same pixels; max_T[i] = max of T over all pixels where i is blended.
 * edge[i] collects the alpha * T of the blends whose alpha lies within the
 * edge width (edge_rel + pos_err |grad ln alpha| + level_rel) of level[i], and
 * 2 tau T for alpha within the edge width of tau: a fp32 evaluation may count
 * them on the other side.  All arrays [n], zeroed by the caller. */
void oracle_peripheral(int64_t n, const double* dbl, const int64_t* tile_start, const int32_t* ids,
                       int32_t width, int32_t height, const oc_params* par, const double* level,
                       double level_rel, double* ps, double* sum_alpha, double* max_T, double* edge) {
  int gx = (width + OC_TILE - 1) / OC_TILE, gy = (height + OC_TILE - 1) / OC_TILE;
  int64_t nt = (int64_t)gx * gy;
  (void)n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < nt; t++) {
    int tx = (int)(t % gx), ty = (int)(t / gx);
    const int32_t* list = ids + tile_start[t];
    int64_t len = tile_start[t + 1] - tile_start[t];
    for (int y = ty * OC_TILE; y < ty * OC_TILE + OC_TILE && y < height; y++)
      for (int x = tx * OC_TILE; x < tx * OC_TILE + OC_TILE && x < width; x++) {
        double T = 1.0;
        for (int64_t k = 0; k < len; k++) {
          int32_t i = list[k];
          const double* g = dbl + (int64_t)i * OC_NF;
          double dx = g[F_U] - x, dy = g[F_V] - y;
          double p = -0.5 * (g[F_A] * dx * dx + g[F_C] * dy * dy) - g[F_B] * dx * dy;
          double araw = g[F_OPAC] * exp(p);
          double alpha = fmin(par->alpha_max, araw);
          double gl = fabs(g[F_A] * dx + g[F_B] * dy) + fabs(g[F_B] * dx + g[F_C] * dy);
          double tol = par->edge_rel + par->pos_err * gl;
          if (araw > 0.0 && fabs(log(araw / par->tau)) <= tol) atomic_add_double(&edge[i], 2.0 * par->tau * T);
          if (p > 0.0 || alpha < par->tau) continue;
          double test_T = T * (1.0 - alpha);
          if (test_T < par->t_min) break;
          double c = alpha * T;
          if (alpha < level[i]) {
            atomic_add_double(&ps[i], c);
            atomic_add_double(&sum_alpha[i], alpha);
          }
          if (isfinite(level[i]) && fabs(log(alpha / level[i])) <= tol + level_rel) atomic_add_double(&edge[i], c);
          atomic_max_double(&max_T[i], T);
          T = test_T;
        }
      }
  }
}

/* Contribution-skip render: the blends of the plain render, each skipped when
 * its contribution c < thr, with c = alpha * T (rule 0, Eq. 3), or
 * weight[i] * alpha (rule 1: weight = max T_i, Eq. 6; rule 2: weight =
 * T_up(depth_i), Eq. 7).  A skipped blend adds no colour and leaves the
 * image's transmittance Ts unchanged; T, which ranks rule 0 and decides the
 * stop, advances as in the plain render, so every rule and threshold works on
 * the same set of blends.  image [3][H][W] = colour + Ts bg; counts[0] =
 * blends, counts[1] = skipped; budget [H][W] (nullable) bounds the change a
 * near-threshold decision (alpha vs tau, p vs 0, c vs thr within thr_rel)
 * can cause. */
void oracle_render_skip(int64_t n, const double* dbl, const int64_t* tile_start, const int32_t* ids,
                        int32_t width, int32_t height, const oc_params* par, int rule, const double* weight,
                        double thr, double thr_rel, double* image, int64_t* counts, double* budget) {
  int gx = (width + OC_TILE - 1) / OC_TILE, gy = (height + OC_TILE - 1) / OC_TILE;
  int64_t nt = (int64_t)gx * gy, hw = (int64_t)width * height;
  double cmax = color_max(n, dbl, par);
  int64_t tot = 0, skipped = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : tot, skipped)
  for (int64_t t = 0; t < nt; t++) {
    int tx = (int)(t % gx), ty = (int)(t / gx);
    const int32_t* list = ids + tile_start[t];
    int64_t len = tile_start[t + 1] - tile_start[t];
    for (int y = ty * OC_TILE; y < ty * OC_TILE + OC_TILE && y < height; y++)
      for (int x = tx * OC_TILE; x < tx * OC_TILE + OC_TILE && x < width; x++) {
        double T = 1.0, Ts = 1.0, col[3] = {0, 0, 0}, bud = 0.0;
        for (int64_t k = 0; k < len; k++) {
          const double* g = dbl + (int64_t)list[k] * OC_NF;
          double dx = g[F_U] - x, dy = g[F_V] - y;
          double p = -0.5 * (g[F_A] * dx * dx + g[F_C] * dy * dy) - g[F_B] * dx * dy;
          double araw = g[F_OPAC] * exp(p);
          double alpha = fmin(par->alpha_max, araw);
          double gl = fabs(g[F_A] * dx + g[F_B] * dy) + fabs(g[F_B] * dx + g[F_C] * dy);
          double tol = par->edge_rel + par->pos_err * gl;
          if (araw > 0.0 && fabs(log(araw / par->tau)) <= tol) bud += 2.0 * par->tau * T * cmax;
          if (fabs(p) <= par->edge_rel && g[F_OPAC] >= par->tau) bud += 2.0 * g[F_OPAC] * T * cmax;
          if (p > 0.0 || alpha < par->tau) continue;
          double test_T = T * (1.0 - alpha);
          if (test_T < par->t_min) break;
          double c = rule == 0 ? alpha * T : weight[list[k]] * alpha;
          if (fabs(c - thr) <= (tol + thr_rel) * thr) bud += 2.0 * alpha * Ts * cmax;
          tot++;
          if (c < thr) {
            skipped++;
          } else {
            col[0] += g[F_R] * alpha * Ts;
            col[1] += g[F_G] * alpha * Ts;
            col[2] += g[F_BL] * alpha * Ts;
            Ts *= 1.0 - alpha;
          }
          T = test_T;
        }
        int64_t o = (int64_t)y * width + x;
        for (int c = 0; c < 3; c++) image[c * hw + o] = col[c] + Ts * par->bg[c];
        if (budget) budget[o] = bud;
      }
  }
  counts[0] = tot;
  counts[1] = skipped;
}

/* ------------------------------------------------------------------------ */
/* Backward with frozen tile lists.                                          */
/* Per pixel: forward products give T_i; the colour behind entry i,         */
/*   R_i = sum_{j>i} c_j a_j prod_{i<k<j}(1-a_k) + bg prod_{k>i}(1-a_k),      */
/* obeys R_{i-1} = c_i a_i + (1-a_i) R_i with R_last = bg, so                 */
/*   dL/da_i = sum_ch g_ch T_i (c_i,ch - R_i,ch)  and  dL/dc_i = g a_i T_i    */
/* without any division.  The feature gradients are chained to the raw       */
/* parameters through the jets of the preprocess.                            */
/* ------------------------------------------------------------------------ */

void oracle_backward(const double* mean, const double* log_scale, const double* quat, const double* logit,
                     const double* sh, int64_t n, const oc_camera* cam, const oc_params* par,
                     const int64_t* tile_start, const int32_t* ids, const double* dL_dimage,
                     double* g_mean, double* g_log_scale, double* g_quat, double* g_logit,
                     double* g_sh, double* g_feat /* [n][9] nullable: u v A B C opac r g b */,
                     double* g_edge /* [n] nullable: near-threshold pixel decisions per Gaussian */,
                     double* g_budget /* [n][NJ + 48] nullable: flip budget of each raw gradient */) {
  int nc = (par->sh_degree + 1) * (par->sh_degree + 1);
  double* dbl = (double*)malloc(sizeof(double) * OC_NF * (n > 0 ? n : 1));
  int32_t* irec = (int32_t*)malloc(sizeof(int32_t) * OC_NI * (n > 0 ? n : 1));
  gjet* gj = (gjet*)malloc(sizeof(gjet) * (n > 0 ? n : 1));
  double* G = (double*)calloc((size_t)(9 * (n > 0 ? n : 1)), sizeof(double));
  /* flip budget per feature: what a near-threshold decision of another entry
   * at a shared pixel can change in this Gaussian's terms there */
  double* Gb = g_budget ? (double*)calloc((size_t)(9 * (n > 0 ? n : 1)), sizeof(double)) : NULL;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; i++)
    preprocess_one(mean, log_scale, quat, logit, sh, n, i, cam, par, dbl + i * OC_NF, irec + i * OC_NI, gj + i);
  double cmax = color_max(n, dbl, par);

  int width = cam->width, height = cam->height;
  int gx = (width + OC_TILE - 1) / OC_TILE, gy = (height + OC_TILE - 1) / OC_TILE;
  int64_t nt = (int64_t)gx * gy, hw = (int64_t)width * height;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < nt; t++) {
    int tx = (int)(t % gx), ty = (int)(t / gx);
    int64_t len = tile_start[t + 1] - tile_start[t];
    const int32_t* list = ids + tile_start[t];
    int32_t* who = (int32_t*)malloc(sizeof(int32_t) * (len > 0 ? len : 1));
    double* al = (double*)malloc(sizeof(double) * (len > 0 ? len : 1));
    double* Ti = (double*)malloc(sizeof(double) * (len > 0 ? len : 1));
    int* clampa = (int*)malloc(sizeof(int) * (len > 0 ? len : 1));
    double* ep = (double*)malloc(sizeof(double) * (len > 0 ? len : 1));
    double* dxs = (double*)malloc(sizeof(double) * (len > 0 ? len : 1));
    double* dys = (double*)malloc(sizeof(double) * (len > 0 ? len : 1));
    for (int y = ty * OC_TILE; y < ty * OC_TILE + OC_TILE && y < height; y++)
      for (int x = tx * OC_TILE; x < tx * OC_TILE + OC_TILE && x < width; x++) {
        int64_t o = (int64_t)y * width + x;
        double g[3] = {dL_dimage[o], dL_dimage[hw + o], dL_dimage[2 * hw + o]};
        /* forward: collect the blended entries and their transmittance */
        double T = 1.0;
        int64_t m = 0;
        /* entries with a near-threshold decision that can change the other
         * entries' terms: position (blended entries before it), whether it is
         * blended, the weight of its change to the colour behind the entries
         * in front of it (alpha T, or T for the stop), and the relative change
         * of the transmittance of the entries behind it (a / (1 - a)) */
        enum { MAXF = 16 };
        int64_t fpos[MAXF];
        int fbl[MAXF];
        double fw[MAXF], frho[MAXF];
        int nflip = 0, foverflow = 0;
        for (int64_t k = 0; k < len; k++) {
          const double* f = dbl + (int64_t)list[k] * OC_NF;
          double dx = f[F_U] - x, dy = f[F_V] - y;
          double p = -0.5 * (f[F_A] * dx * dx + f[F_C] * dy * dy) - f[F_B] * dx * dy;
          double e = exp(p);
          double araw = f[F_OPAC] * e;
          double a = fmin(par->alpha_max, araw);
          if (g_edge || Gb) {
            /* decisions within their edge band at this pixel: alpha vs tau (the
             * image's band), alpha vs its clamp, p vs 0, and the stop test
             * (T carries one rounding per blend before it) */
            double gl = fabs(f[F_A] * dx + f[F_B] * dy) + fabs(f[F_B] * dx + f[F_C] * dy);
            double tol = par->edge_rel + par->pos_err * gl;
            /* inclusion decisions (alpha vs tau, p vs 0) add or drop the entry;
             * the clamp decision changes only its own derivative */
            int incl = (araw > 0.0 && fabs(log(araw / par->tau)) <= tol) || fabs(p) <= par->edge_rel;
            int clampd = araw > 0.0 && fabs(log(araw / par->alpha_max)) <= tol;
            int stopd = 0;
            if (!incl && p <= 0.0 && a >= par->tau) {
              double tt = T * (1.0 - a);
              stopd = fabs(log(tt / par->t_min)) <= par->edge_rel + (double)(m + 1) * 1.2e-7 + tol;
            }
            if (incl || clampd || stopd) {
              if (g_edge) atomic_add_double(&g_edge[list[k]], 1.0);
              if (incl || stopd) {
                if (nflip < MAXF) {
                  fpos[nflip] = m;
                  fbl[nflip] = p <= 0.0 && a >= par->tau && T * (1.0 - a) >= par->t_min;
                  fw[nflip] = stopd ? T : a * T;
                  frho[nflip] = stopd ? 0.0 : a / (1.0 - a);
                  nflip++;
                } else {
                  foverflow = 1;
                }
              }
            }
          }
          if (p > 0.0) continue;
          if (a < par->tau) continue;
          double test_T = T * (1.0 - a);
          if (test_T < par->t_min) break;
          who[m] = list[k]; al[m] = a; Ti[m] = T; clampa[m] = araw > par->alpha_max; ep[m] = e;
          dxs[m] = dx; dys[m] = dy;
          m++;
          T = test_T;
        }
        /* backward recursion on R */
        double R[3] = {par->bg[0], par->bg[1], par->bg[2]};
        for (int64_t j = m - 1; j >= 0; j--) {
          const double* f = dbl + (int64_t)who[j] * OC_NF;
          double c[3] = {f[F_R], f[F_G], f[F_BL]};
          double dLda = 0.0;
          for (int ch = 0; ch < 3; ch++) {
            dLda += g[ch] * Ti[j] * (c[ch] - R[ch]);
            atomic_add_double(&G[who[j] * 9 + 6 + ch], g[ch] * al[j] * Ti[j]);
          }
          if (Gb && (nflip > 0 || foverflow)) {
            /* a flipping entry f in front of this one changes T before it by
             * the factor (1 - a_f)^(-+1) (relatively by rho); one behind it
             * changes the colour behind it by at most 2 c_max w_f / T_(j+1)
             * (w_f <= T_(j+1): f lies behind) */
            double rho = 0.0, dR = 0.0;
            double Tn = Ti[j] * (1.0 - al[j]);
            for (int q = 0; q < nflip; q++) {
              if (fbl[q] ? fpos[q] < j : fpos[q] <= j) rho += frho[q];
              else if (fpos[q] > j) dR += 2.0 * cmax * fw[q] / Tn;
            }
            if (foverflow) { rho += 1.0; dR += 2.0 * cmax; }   /* too many to track: a coarse bound */
            double bda = 0.0;
            for (int ch = 0; ch < 3; ch++) {
              bda += fabs(g[ch]) * Ti[j] * (rho * fabs(c[ch] - R[ch]) + dR);
              atomic_add_double(&Gb[who[j] * 9 + 6 + ch], fabs(g[ch]) * al[j] * Ti[j] * rho);
            }
            if (!clampa[j]) {
              double dx = dxs[j], dy = dys[j];
              atomic_add_double(&Gb[who[j] * 9 + 5], bda * ep[j]);
              atomic_add_double(&Gb[who[j] * 9 + 0], bda * al[j] * fabs(f[F_A] * dx + f[F_B] * dy));
              atomic_add_double(&Gb[who[j] * 9 + 1], bda * al[j] * fabs(f[F_C] * dy + f[F_B] * dx));
              atomic_add_double(&Gb[who[j] * 9 + 2], bda * al[j] * 0.5 * dx * dx);
              atomic_add_double(&Gb[who[j] * 9 + 3], bda * al[j] * fabs(dx * dy));
              atomic_add_double(&Gb[who[j] * 9 + 4], bda * al[j] * 0.5 * dy * dy);
            }
          }
          for (int ch = 0; ch < 3; ch++) R[ch] = c[ch] * al[j] + (1.0 - al[j]) * R[ch];
          if (clampa[j]) continue;   /* alpha = alpha_max: no dependence on opacity or power */
          double dLdp = dLda * al[j];
          double dx = dxs[j], dy = dys[j];
          atomic_add_double(&G[who[j] * 9 + 5], dLda * ep[j]);
          atomic_add_double(&G[who[j] * 9 + 0], dLdp * (-(f[F_A] * dx + f[F_B] * dy)));
          atomic_add_double(&G[who[j] * 9 + 1], dLdp * (-(f[F_C] * dy + f[F_B] * dx)));
          atomic_add_double(&G[who[j] * 9 + 2], dLdp * (-0.5 * dx * dx));
          atomic_add_double(&G[who[j] * 9 + 3], dLdp * (-dx * dy));
          atomic_add_double(&G[who[j] * 9 + 4], dLdp * (-0.5 * dy * dy));
        }
      }
    free(who); free(al); free(Ti); free(clampa); free(ep); free(dxs); free(dys);
  }

  /* chain to raw parameters */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    double gr[NJ] = {0};
    const double* Gi = G + i * 9;
    if (g_feat) for (int k = 0; k < 9; k++) g_feat[i * 9 + k] = Gi[k];
    int live = irec[i * OC_NI + I_CULL] == CULL_NONE;
    if (live) {
      const gjet* q = gj + i;
      const jet* fj[9] = {&q->u, &q->v, &q->A, &q->B, &q->C, &q->opac, &q->rgb[0], &q->rgb[1], &q->rgb[2]};
      for (int f = 0; f < 9; f++)
        for (int k = 0; k < NJ; k++) gr[k] += Gi[f] * fj[f]->d[k];
    }
    for (int k = 0; k < 3; k++) g_mean[k * n + i] = gr[k];
    for (int k = 0; k < 3; k++) g_log_scale[k * n + i] = gr[3 + k];
    for (int k = 0; k < 4; k++) g_quat[k * n + i] = gr[6 + k];
    g_logit[i] = gr[10];
    for (int k = 0; k < nc; k++)
      for (int ch = 0; ch < 3; ch++)
        g_sh[(k * 3 + ch) * n + i] = (live && !gj[i].clamp[ch]) ? Gi[6 + ch] * gj[i].Y[k].v : 0.0;
    if (Gb) {   /* the feature budgets through the absolute derivatives */
      double* bo = g_budget + i * (NJ + 48);
      const double* Bi = Gb + i * 9;
      memset(bo, 0, sizeof(double) * (NJ + 48));
      if (live) {
        const gjet* q = gj + i;
        const jet* fj[9] = {&q->u, &q->v, &q->A, &q->B, &q->C, &q->opac, &q->rgb[0], &q->rgb[1], &q->rgb[2]};
        for (int f = 0; f < 9; f++)
          for (int k = 0; k < NJ; k++) bo[k] += Bi[f] * fabs(fj[f]->d[k]);
        for (int k = 0; k < nc; k++)
          for (int ch = 0; ch < 3; ch++) bo[NJ + k * 3 + ch] = gj[i].clamp[ch] ? 0.0 : Bi[6 + ch] * fabs(gj[i].Y[k].v);
      }
    }
  }
  free(dbl); free(irec); free(gj); free(G); free(Gb);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
