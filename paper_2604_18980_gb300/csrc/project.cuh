// project.cuh -- per-Gaussian projection math shared by the preprocess kernel
// and its adjoint (device code only).
//
// 3D covariance  Sigma = Rq S S^T Rq^T, Rq from the normalised quaternion
//                (w,x,y,z), S = diag(exp(log_scale)).
// EWA            Sigma2D = T Sigma T^T + 0.3 I with T = J W, J the Jacobian of
//                the perspective map at the view-space mean with x/z and y/z
//                clamped to 1.3 tan(fov/2), W the camera rotation.
// We form V = T Rq S (2x3) so that Sigma2D - 0.3 I = V V^T; then
//   a = |v0|^2, b = v0.v1, c = |v1|^2 and det(V V^T) = |v0 x v1|^2,
// which keeps the dilated determinant free of cancellation:
//   det = |v0 x v1|^2 + 0.3 (a + c) + 0.09.
// Colour: real spherical harmonics (Condon-Shortley phase, index l*l+l+m)
// evaluated at the unit direction from the camera centre to the mean, + 0.5,
// clamped at 0.
#pragma once

#include "ags_internal.cuh"

namespace ags {

// Real SH normalisation constants (textbook closed forms):
constexpr float kSH0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kSH1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kSH2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kSH2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kSH2c = 0.5462742152960396f;   // sqrt(15/pi)/4
constexpr float kSH3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
constexpr float kSH3b = 2.890611442640554f;    // sqrt(105/pi)/2
constexpr float kSH3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
constexpr float kSH3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kSH3e = 1.445305721320277f;    // sqrt(105/pi)/4

// Basis values Y[0..15] at unit direction (x,y,z), degrees 0..deg.
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
  Y[0] = kSH0;
  if (deg < 1) return;
  Y[1] = -kSH1 * y;
  Y[2] = kSH1 * z;
  Y[3] = -kSH1 * x;
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kSH2a * x * y;
  Y[5] = -kSH2a * y * z;
  Y[6] = kSH2b * (3.f * zz - 1.f);
  Y[7] = -kSH2a * x * z;
  Y[8] = kSH2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -kSH3a * y * (3.f * xx - yy);
  Y[10] = kSH3b * x * y * z;
  Y[11] = -kSH3c * y * (5.f * zz - 1.f);
  Y[12] = kSH3d * z * (5.f * zz - 3.f);
  Y[13] = -kSH3c * x * (5.f * zz - 1.f);
  Y[14] = kSH3e * z * (xx - yy);
  Y[15] = -kSH3a * x * (xx - 3.f * yy);
}

// Gradient sum_k w[k] dY_k/d(x,y,z) of the polynomial forms above.
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, const float* w,
                                              float& gx, float& gy, float& gz) {
  gx = gy = gz = 0.f;
  if (deg < 1) return;
  gy += -kSH1 * w[1];
  gz += kSH1 * w[2];
  gx += -kSH1 * w[3];
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  gx += kSH2a * y * w[4];            gy += kSH2a * x * w[4];
  gy += -kSH2a * z * w[5];           gz += -kSH2a * y * w[5];
  gz += 6.f * kSH2b * z * w[6];
  gx += -kSH2a * z * w[7];           gz += -kSH2a * x * w[7];
  gx += 2.f * kSH2c * x * w[8];      gy += -2.f * kSH2c * y * w[8];
  if (deg < 3) return;
  gx += -6.f * kSH3a * x * y * w[9];  gy += -3.f * kSH3a * (xx - yy) * w[9];
  gx += kSH3b * y * z * w[10];        gy += kSH3b * x * z * w[10];  gz += kSH3b * x * y * w[10];
  gy += -kSH3c * (5.f * zz - 1.f) * w[11];  gz += -10.f * kSH3c * y * z * w[11];
  gz += kSH3d * (15.f * zz - 3.f) * w[12];
  gx += -kSH3c * (5.f * zz - 1.f) * w[13];  gz += -10.f * kSH3c * x * z * w[13];
  gx += 2.f * kSH3e * x * z * w[14];  gy += -2.f * kSH3e * y * z * w[14];  gz += kSH3e * (xx - yy) * w[14];
  gx += -3.f * kSH3a * (xx - yy) * w[15];  gy += 6.f * kSH3a * x * y * w[15];
}

// a0 b0 + a1 b1 + a2 b2 + c, accurate to about one fp32 rounding: the "Dot2"
// compensated dot product of Ogita, Rump and Oishi (SIAM J. Sci. Comput.
// 26(6), 2005): products split exactly with FMA, sums with TwoSum, errors
// accumulated and added back once.  Intrinsics keep the compiler from
// contracting or reassociating the error-free transformations.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  float z = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ float dot3_plus(float a0, float b0, float a1, float b1, float a2, float b2, float c) {
  float p = __fmul_rn(a0, b0);
  float e = __fmaf_rn(a0, b0, -p);
  float h, q, s, t;
  h = __fmul_rn(a1, b1);
  q = __fmaf_rn(a1, b1, -h);
  two_sum(p, h, s, t);
  p = s;
  e = __fadd_rn(e, __fadd_rn(q, t));
  h = __fmul_rn(a2, b2);
  q = __fmaf_rn(a2, b2, -h);
  two_sum(p, h, s, t);
  p = s;
  e = __fadd_rn(e, __fadd_rn(q, t));
  two_sum(p, c, s, t);
  return __fadd_rn(s, __fadd_rn(e, t));
}

// View-independent quantities of one Gaussian.
struct Frame {
  float s[3];          // exp(log_scale)
  float qn[4];         // normalised quaternion
  float qinv;          // 1 / |q|
  float Rq[9];         // rotation matrix
  float M[9];          // Rq S
  float opac;          // sigmoid(logit)
};

__device__ __forceinline__ void make_frame(const float ls[3], const float q[4], float logit, Frame& F) {
#pragma unroll
  for (int k = 0; k < 3; k++) F.s[k] = expf(ls[k]);
  const float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  F.qinv = rsqrtf(qq);
  const float w = q[0] * F.qinv, x = q[1] * F.qinv, y = q[2] * F.qinv, z = q[3] * F.qinv;
  F.qn[0] = w; F.qn[1] = x; F.qn[2] = y; F.qn[3] = z;
  F.Rq[0] = 1.f - 2.f * (y * y + z * z); F.Rq[1] = 2.f * (x * y - w * z);       F.Rq[2] = 2.f * (x * z + w * y);
  F.Rq[3] = 2.f * (x * y + w * z);       F.Rq[4] = 1.f - 2.f * (x * x + z * z); F.Rq[5] = 2.f * (y * z - w * x);
  F.Rq[6] = 2.f * (x * z - w * y);       F.Rq[7] = 2.f * (y * z + w * x);       F.Rq[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int k = 0; k < 3; k++) F.M[r * 3 + k] = F.Rq[r * 3 + k] * F.s[k];
  F.opac = 1.0f / (1.0f + expf(-logit));
}

// Everything the forward computes for one Gaussian in one view.
struct Proj {
  float t[3];          // view-space mean
  float iz;            // 1 / t_z
  float ctx, cty;      // x/z and y/z after the frustum clamp
  int fclamp;          // bit3 x clamped, bit4 y clamped
  float Tm[6];         // T = J W (2x3)
  float V[6];          // V = T Rq S (2x3)
  float a, b, c;       // V V^T (undilated)
  float det;           // det(V V^T + 0.3 I)
  float A, B, C;       // conic
  float lam1;          // largest eigenvalue of the dilated covariance
  float u, v;          // 2D mean
};

// Projection of Gaussian (m, F) for camera C.  Returns false when the
// Gaussian is culled (near plane or degenerate).
// The view-space mean, the frustum clamp, T = J W and the 2D mean: the first
// half of project_view (false behind the near plane).
__device__ __forceinline__ bool project_mean(const DevCam& C, const float m[3], Proj& P);
// The second half: V, the dilated 2D covariance, its conic and largest
// eigenvalue (false when the determinant is not positive).
__device__ __forceinline__ bool project_cov(const Frame& F, Proj& P);

__device__ __forceinline__ bool project_view(const DevCam& C, const float m[3], const Frame& F, Proj& P) {
  return project_mean(C, m, P) && project_cov(F, P);
}

// Can the footprint of a Gaussian whose mean passed project_mean touch a
// pixel of the W x H image?  A bound taken before the covariance: the radius
// of either scale mode is at most ceil(3 sqrt(lam1)); lam1 <= tr + 0.3163 for
// the dilated covariance (trace tr, the eigenvalue's max(0.1, .) floor
// included); tr = |T Rq S|_F^2 + 0.6 <= |T|_F^2 s_max^2 + 0.6.  With relative
// slack far above fp32 rounding and a pixel of absolute slack, a false answer
// means the full projection would find no tile (tile_span of u +- rf, v +- rf
// is empty), so skipping it changes no output.  NaN bounds answer true.
__device__ __forceinline__ bool footprint_may_reach(const Proj& P, float smax2, int W, int H) {
  float tn2 = 0.f;
#pragma unroll
  for (int k = 0; k < 6; k++) tn2 = fmaf(P.Tm[k], P.Tm[k], tn2);
  const float lam = fmaf(tn2 * smax2, 1.001f, 0.92f);
  const float R = 3.003f * sqrtf(lam) + 2.f;
  return !(P.u + R < 0.f || P.u - R > (float)(W - 1) || P.v + R < 0.f || P.v - R > (float)(H - 1));
}

__device__ __forceinline__ bool project_mean(const DevCam& C, const float m[3], Proj& P) {
  // view transform t = R m + t_cam (compensated: depth keys and the near-plane
  // test see the correctly rounded value up to an ulp)
#pragma unroll
  for (int r = 0; r < 3; r++)
    P.t[r] = dot3_plus(C.R[r * 3 + 0], m[0], C.R[r * 3 + 1], m[1], C.R[r * 3 + 2], m[2], C.t[r]);
  if (!(P.t[2] > C.near_z)) return false;
  P.iz = 1.0f / P.t[2];
  const float txtz = P.t[0] * P.iz, tytz = P.t[1] * P.iz;
  P.fclamp = 0;
  P.ctx = txtz;
  P.cty = tytz;
  if (txtz > C.limx) { P.ctx = C.limx; P.fclamp |= 8; }
  else if (txtz < -C.limx) { P.ctx = -C.limx; P.fclamp |= 8; }
  if (tytz > C.limy) { P.cty = C.limy; P.fclamp |= 16; }
  else if (tytz < -C.limy) { P.cty = -C.limy; P.fclamp |= 16; }

  // T = J W: row 0 = fx/tz (W0 - ctx W2), row 1 = fy/tz (W1 - cty W2)
  const float jx = C.fx * P.iz, jy = C.fy * P.iz;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    P.Tm[k] = jx * fmaf(-P.ctx, C.R[6 + k], C.R[k]);
    P.Tm[3 + k] = jy * fmaf(-P.cty, C.R[6 + k], C.R[3 + k]);
  }
  P.u = fmaf(C.fx, P.t[0] * P.iz, C.cx);
  P.v = fmaf(C.fy, P.t[1] * P.iz, C.cy);
  return true;
}

__device__ __forceinline__ bool project_cov(const Frame& F, Proj& P) {
  // V = T (Rq S)
#pragma unroll
  for (int r = 0; r < 2; r++)
#pragma unroll
    for (int k = 0; k < 3; k++)
      P.V[r * 3 + k] = P.Tm[r * 3 + 0] * F.M[0 * 3 + k] + P.Tm[r * 3 + 1] * F.M[1 * 3 + k] +
                       P.Tm[r * 3 + 2] * F.M[2 * 3 + k];
  const float* v0 = P.V;
  const float* v1 = P.V + 3;
  P.a = v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2];
  P.b = v0[0] * v1[0] + v0[1] * v1[1] + v0[2] * v1[2];
  P.c = v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2];
  const float cx_ = v0[1] * v1[2] - v0[2] * v1[1];
  const float cy_ = v0[2] * v1[0] - v0[0] * v1[2];
  const float cz_ = v0[0] * v1[1] - v0[1] * v1[0];
  const float ad = P.a + 0.3f, cd = P.c + 0.3f;
  P.det = (cx_ * cx_ + cy_ * cy_ + cz_ * cz_) + 0.3f * (P.a + P.c) + 0.09f;
  if (!(P.det > 0.f)) return false;
  const float id = 1.0f / P.det;
  P.A = cd * id;
  P.B = -P.b * id;
  P.C = ad * id;
  const float half = 0.5f * (ad - cd);
  P.lam1 = 0.5f * (ad + cd) + sqrtf(fmaxf(0.1f, half * half + P.b * P.b));
  return true;
}

}  // namespace ags
