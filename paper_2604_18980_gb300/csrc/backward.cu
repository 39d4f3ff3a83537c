// backward.cu -- adjoint of the blend and of the preprocess (not in the paper;
// the AdaGScale pair selection is held fixed, i.e. Th, the footprint and the
// pair lists are treated as piecewise constant).
//
// Blend adjoint: one CTA per tile; each pixel walks its list backwards from its
// last blended pair, recovering the transmittance before pair j as
// T_j = T_{j+1} / (1 - alpha_j), and keeps R, the colour behind pair j
// (background included): R <- c_j alpha_j + (1 - alpha_j) R.  Then
//   dL/dalpha_j = T_j sum_ch g_ch (c_j,ch - R_ch),   dL/dc_j = alpha_j T_j g.
// Per-splat gradients (u, v, conic, opacity, r, g, b) are reduced across the
// warp before one atomic add per warp.  The conic gradient is accumulated in
// the splat's eigenframe (pixel offsets rotated onto its axes): in Cartesian
// components the minor-axis part of a long thin splat would be lost to fp32
// cancellation against the far larger major-axis terms.
//
// Preprocess adjoint: one thread per Gaussian, summing over views; it
// recomputes the projection with the forward's code and applies the chain
// rule through the conic inverse, V = J W Rq S, the EWA Jacobian (frustum
// clamp honoured), the quaternion normalisation, exp(log_scale), the sigmoid
// and the SH basis (colour clamp honoured).
#include <algorithm>

#include "blend.cuh"
#include "project.cuh"

namespace ags {

constexpr int kGradStride = 9;   // u v | conic gradient in the eigenframe (aa, ab, bb) | opacity r g b

// Sums v[0..8] over the warp with a transposed butterfly (16 shuffles for all
// nine sums instead of 45): after it, lane 2c (c < 9) holds the total of v[c].
__device__ __forceinline__ float warp_reduce9(const float v[9], int lane) {
  float a[16];
#pragma unroll
  for (int k = 0; k < 9; k++) a[k] = v[k];
#pragma unroll
  for (int k = 9; k < 16; k++) a[k] = 0.f;
#pragma unroll
  for (int o = 16, h = 8; o >= 2; o >>= 1, h >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < h; k++) {
      const float send = hi ? a[k] : a[k + h];
      const float keep = hi ? a[k + h] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// One pixel's step of the reverse walk over a splat it may have blended:
// recovers T before the splat, updates the colour behind it, and adds the
// pixel's share of the splat's nine gradients to acc.  Returns whether the
// splat was blended here (the forward's accept test, bit for bit).
__device__ __forceinline__ bool pixel_adjoint(const Staged& s, float cbl, const float4& o, const float2& f,
                                              const BlendConst& bc, float dx, float dy, float P, float Bx, float ga,
                                              float gb, float gc, float& T, float& Ra, float& Rb, float& Rc,
                                              float acc[9]) {
  const float q = splat_qy(s, P, Bx, dy);
  if (!splat_accept(q, bc.l2tau)) return false;
  float raw;
  const float alpha = splat_alpha(q, bc.alpha_max, raw);
  const float om = 1.f - alpha;
  T = __fdividef(T, om);                         // transmittance before this splat
  const float w = alpha * T;
  acc[6] += w * ga;
  acc[7] += w * gb;
  acc[8] += w * gc;
  const float dLda = T * (ga * (s.b.z - Ra) + gb * (s.b.w - Rb) + gc * (cbl - Rc));
  Ra = s.b.z * alpha + om * Ra;
  Rb = s.b.w * alpha + om * Rb;
  Rc = cbl * alpha + om * Rc;
  if (!(raw > bc.alpha_max)) {                   // the clamp cuts the gradient through alpha
    const float dLdp = dLda * alpha;
    acc[5] += dLdp * o.w;                        // d alpha / d opacity = alpha / opacity
    acc[0] -= dLdp * (o.x * dx + o.y * dy);
    acc[1] -= dLdp * (o.y * dx + o.z * dy);
    const float da = f.x * dx + f.y * dy, db = f.x * dy - f.y * dx;
    acc[2] -= 0.5f * dLdp * da * da;
    acc[3] -= dLdp * da * db;
    acc[4] -= 0.5f * dLdp * db * db;
  }
  return true;
}

// Blend adjoint, laid out like the forward: 128 threads per tile, warps of
// 8x8 pixels, two pixels per thread (rows y and y+4), per-warp lists of the
// splats whose alpha >= tau ellipse reaches the warp's block, walked from the
// back.  Each pixel starts from its final T and its last blended position.
__global__ void __launch_bounds__(128)
raster_backward_kernel(const float4* __restrict__ splat, const uint32_t* __restrict__ vals,
                       const uint2* __restrict__ ranges, int W, int H, int gx, int tiles_per_view, BlendConst bc,
                       const float* __restrict__ final_T, const uint32_t* __restrict__ n_contrib,
                       const float* __restrict__ dL_dimage, float* __restrict__ gsplat, uint32_t n_splats,
                       int64_t* status) {
  constexpr int kB = 128;
  __shared__ float4 s_a[kB];      // u v a2 b2
  __shared__ float4 s_b[kB];      // c2 base r g
  __shared__ float4 s_o[kB];      // A B C 1/opacity
  __shared__ float2 s_f[kB];      // eigenframe (cos, sin) of the conic
  __shared__ float s_c[kB];       // b
  __shared__ uint32_t s_m[kB];
  __shared__ uint32_t s_e[kB];
  __shared__ uint16_t s_list[4][kB];
  __shared__ uint32_t s_maxlast;

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
  const uint32_t start = rg.x;
  const uint32_t end = AGS_DCHECK(rg.x <= rg.y, status, AGS_CHECK_BACKWARD_RANGE) ? rg.y : rg.x;
  const size_t hw = (size_t)W * H;

  float T0 = 1.f, T1 = 1.f, g00 = 0.f, g01 = 0.f, g02 = 0.f, g10 = 0.f, g11 = 0.f, g12 = 0.f;
  uint32_t last0 = 0, last1 = 0;
  if (in0) {
    const size_t op = (size_t)view * hw + (size_t)py0 * W + px;
    T0 = final_T[op];
    last0 = n_contrib[op];
    const size_t o = (size_t)view * 3 * hw + (size_t)py0 * W + px;
    g00 = dL_dimage[o]; g01 = dL_dimage[o + hw]; g02 = dL_dimage[o + 2 * hw];
  }
  if (in1) {
    const size_t op = (size_t)view * hw + (size_t)py1 * W + px;
    T1 = final_T[op];
    last1 = n_contrib[op];
    const size_t o = (size_t)view * 3 * hw + (size_t)py1 * W + px;
    g10 = dL_dimage[o]; g11 = dL_dimage[o + hw]; g12 = dL_dimage[o + 2 * hw];
  }
  float R00 = bc.bg[0], R01 = bc.bg[1], R02 = bc.bg[2];
  float R10 = bc.bg[0], R11 = bc.bg[1], R12 = bc.bg[2];
  if (tid == 0) s_maxlast = 0u;
  __syncthreads();
  const uint32_t mylast = max(last0, last1);
  if (mylast) atomicMax(&s_maxlast, mylast);
  __syncthreads();
  const uint32_t maxlast = min(s_maxlast, end - start);
  const uint32_t wlast = __reduce_max_sync(0xffffffffu, mylast);   // this warp's entries end here

  for (int32_t bend = (int32_t)maxlast; bend > 0; bend -= kB) {
    const int32_t bbeg = max(0, bend - kB);
    const int nb = bend - bbeg;
    __syncthreads();
    // (a debug build skips a pair value out of range: no warp walks it)
    if (tid < nb && !AGS_DCHECK(__ldg(vals + start + bbeg + tid) < n_splats, status, AGS_CHECK_BACKWARD_VALUE)) {
      s_m[tid] = 0u;
      s_e[tid] = 0u;
    } else if (tid < nb) {
      const uint32_t e = __ldg(vals + start + bbeg + tid);
      const float4* rec = splat + (size_t)e * 3;
      Staged st;
      uint32_t m;
      stage_splat<8, 8>(rec, tx * kTile, ty * kTile, bc.l2tau, st, m);
      const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
      s_a[tid] = st.a;
      s_b[tid] = st.b;
      s_c[tid] = st.c;
      s_o[tid] = make_float4(r0.z, r0.w, r1.x, __frcp_rn(r1.y));
      float ca, sa;
      conic_frame(r0.z, r0.w, r1.x, ca, sa);
      s_f[tid] = make_float2(ca, sa);
      s_m[tid] = m;
      s_e[tid] = e;
    }
    __syncthreads();
    // this warp's entries below its last blended position, in depth order
    const int jtop = min(nb, (int)wlast - bbeg);
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kB / 32; k++) {
      const int j = k * 32 + lane;
      const bool hit = j < jtop && ((s_m[j] >> warp) & 1u);
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) s_list[warp][cnt + __popc(bal & lanemask_lt())] = (uint16_t)j;
      cnt += __popc(bal);
    }
    __syncwarp();
    for (int t = cnt - 1; t >= 0; t--) {                // back to front
      const int j = s_list[warp][t];
      const uint32_t pos = (uint32_t)(bbeg + j);         // 0-based position in the tile list
      Staged s;
      s.a = s_a[j];
      s.b = s_b[j];
      const float cbl = s_c[j];
      const float4 o = s_o[j];
      const float2 f = s_f[j];
      const float dx = __fsub_rn(s.a.x, fpx);
      float P, Bx;
      splat_qx(s, dx, P, Bx);
      float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      bool contrib = false;
      if (pos < last0)
        contrib |= pixel_adjoint(s, cbl, o, f, bc, dx, __fsub_rn(s.a.y, fpy0), P, Bx, g00, g01, g02, T0, R00, R01,
                                 R02, acc);
      if (pos < last1)
        contrib |= pixel_adjoint(s, cbl, o, f, bc, dx, __fsub_rn(s.a.y, fpy1), P, Bx, g10, g11, g12, T1, R10, R11,
                                 R12, acc);
      if (__any_sync(0xffffffffu, contrib)) {
        const float sum = warp_reduce9(acc, lane);
        if ((lane & 1) == 0 && lane < 18) atomicAdd(gsplat + (size_t)s_e[j] * kGradStride + (lane >> 1), sum);
      }
    }
  }
}

struct GradOut {
  float* mean;
  float* ls;
  float* quat;
  float* logit;
  float* sh;
};

// kOneView: a single view needs no per-Gaussian SH accumulator; its SH
// gradient is written as soon as it is known, which frees 48 registers.
template <bool kOneView>
__global__ void __launch_bounds__(128, kOneView ? 4 : 3)
preprocess_backward_kernel(const float* __restrict__ mean, const float* __restrict__ lsc, const float* __restrict__ quat,
                           const float* __restrict__ logit_in, const float* __restrict__ sh, int64_t n, int views,
                           const __grid_constant__ CamBatch cams, const __grid_constant__ DevParams P,
                           const uint8_t* __restrict__ flags, const float* __restrict__ gsplat,
                           const float* __restrict__ conic_rec, GradOut out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int deg = P.sh_degree;
  const int nc = (deg + 1) * (deg + 1);
  float m[3], ls[3], q[4];
  for (int k = 0; k < 3; k++) m[k] = __ldg(mean + k * n + i);
  for (int k = 0; k < 3; k++) ls[k] = __ldg(lsc + k * n + i);
  for (int k = 0; k < 4; k++) q[k] = __ldg(quat + k * n + i);
  const float logit = __ldg(logit_in + i);
  float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, glogit = 0.f;
  float gsh[kOneView ? 1 : 16][3];
  if constexpr (!kOneView)
    for (int k = 0; k < 16; k++) gsh[k][0] = gsh[k][1] = gsh[k][2] = 0.f;
  bool sh_written = false;
  // One view: every load of a visible Gaussian is issued up front, so that
  // they are all in flight together instead of one dependent phase at a time.
  float shv[kOneView ? 48 : 1], Gv[kOneView ? 9 : 1];
  float4 cv0 = make_float4(0.f, 0.f, 0.f, 0.f);
  float cvC = 0.f;
  uint8_t fl0 = 0;
  if constexpr (kOneView) {
    fl0 = __ldg(flags + i);
    if (!(fl0 & kFlagCulled)) {
#pragma unroll
      for (int k = 0; k < 16; k++)
#pragma unroll
        for (int ch = 0; ch < 3; ch++) shv[k * 3 + ch] = k < nc ? __ldg(sh + (int64_t)(k * 3 + ch) * n + i) : 0.f;
#pragma unroll
      for (int k = 0; k < kGradStride; k++) Gv[k] = __ldg(gsplat + (size_t)i * kGradStride + k);
      cv0 = __ldg(reinterpret_cast<const float4*>(conic_rec + (size_t)i * kSplatFloats));
      cvC = __ldg(conic_rec + (size_t)i * kSplatFloats + 4);
    }
  }
  Frame F;
  make_frame(ls, q, logit, F);

  for (int view = 0; view < views; view++) {
    const int64_t e = (int64_t)view * n + i;
    const uint8_t fl = kOneView ? fl0 : __ldg(flags + e);
    if (fl & kFlagCulled) continue;
    const float* G = gsplat + (size_t)e * kGradStride;
    float Gl[kGradStride];
#pragma unroll
    for (int k = 0; k < kGradStride; k++) Gl[k] = kOneView ? Gv[k] : __ldg(G + k);
    const float gu = Gl[0], gv = Gl[1], gA = Gl[2], gB = Gl[3], gC = Gl[4], gO = Gl[5];
    const float gcol[3] = {(fl & 1) ? 0.f : Gl[6], (fl & 2) ? 0.f : Gl[7], (fl & 4) ? 0.f : Gl[8]};
    const DevCam& C = cams.c[view];
    Proj pj;
    if (!project_view(C, m, F, pj)) continue;

    // colour: rgb_ch = sum_k sh[k][ch] Y_k(dir) + 0.5
    float dx = m[0] - C.campos[0], dy = m[1] - C.campos[1], dz = m[2] - C.campos[2];
    float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    float dir[3] = {dx * il, dy * il, dz * il};
    float Y[16];
    sh_basis(deg, dir[0], dir[1], dir[2], Y);
    float wk[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
      wk[k] = 0.f;
      if (k < nc) {
        const float s0 = kOneView ? shv[k * 3 + 0] : __ldg(sh + (int64_t)(k * 3 + 0) * n + i),
                    s1 = kOneView ? shv[k * 3 + 1] : __ldg(sh + (int64_t)(k * 3 + 1) * n + i),
                    s2 = kOneView ? shv[k * 3 + 2] : __ldg(sh + (int64_t)(k * 3 + 2) * n + i);
        wk[k] = gcol[0] * s0 + gcol[1] * s1 + gcol[2] * s2;
        if constexpr (kOneView) {
          out.sh[(int64_t)(k * 3 + 0) * n + i] = gcol[0] * Y[k];
          out.sh[(int64_t)(k * 3 + 1) * n + i] = gcol[1] * Y[k];
          out.sh[(int64_t)(k * 3 + 2) * n + i] = gcol[2] * Y[k];
        } else {
          gsh[k][0] += gcol[0] * Y[k];
          gsh[k][1] += gcol[1] * Y[k];
          gsh[k][2] += gcol[2] * Y[k];
        }
      }
    }
    sh_written = true;
    float gd0, gd1, gd2;
    sh_basis_grad(deg, dir[0], dir[1], dir[2], wk, gd0, gd1, gd2);
    float dot = gd0 * dir[0] + gd1 * dir[1] + gd2 * dir[2];
    gm[0] += (gd0 - dot * dir[0]) * il;
    gm[1] += (gd1 - dot * dir[1]) * il;
    gm[2] += (gd2 - dot * dir[2]) * il;

    // opacity
    glogit += gO * F.opac * (1.f - F.opac);

    // conic M = Sigma^-1 of the dilated covariance: dL/dSigma = -M (dL/dM) M,
    // evaluated in the eigenframe (e_a minor axis, e_b major axis) where
    // M = diag(1/lambda_min, 1/lambda_max) and dL/dM = (gA gB/2; gB/2 gC)
    // as accumulated by the blend adjoint, then rotated back.
    const float4 c0 = kOneView ? cv0 : __ldg(reinterpret_cast<const float4*>(conic_rec + (size_t)e * kSplatFloats));
    const float cC = kOneView ? cvC : __ldg(conic_rec + (size_t)e * kSplatFloats + 4);
    float ca, sa;
    conic_frame(c0.z, c0.w, cC, ca, sa);
    const float ad = pj.a + 0.3f, cd = pj.c + 0.3f;
    const float half = 0.5f * (ad - cd);
    const float lmax = 0.5f * (ad + cd) + sqrtf(half * half + pj.b * pj.b);
    const float ma = lmax / pj.det, mb = 1.f / lmax;               // 1/lambda_min, 1/lambda_max
    const float eaa = -ma * ma * gA, eab = -ma * mb * 0.5f * gB, ebb = -mb * mb * gC;
    // Cartesian dL/d(a, b, c) of Sigma = R E R^T with R = (e_a e_b)
    const float ga = ca * ca * eaa - 2.f * ca * sa * eab + sa * sa * ebb;
    const float g12 = ca * sa * eaa + (ca * ca - sa * sa) * eab - ca * sa * ebb;
    const float gc = sa * sa * eaa + 2.f * ca * sa * eab + ca * ca * ebb;
    const float gbb = 2.f * g12;
    // a = |v0|^2, b = v0.v1, c = |v1|^2
    float gV[6];
    for (int k = 0; k < 3; k++) {
      gV[k] = 2.f * ga * pj.V[k] + gbb * pj.V[3 + k];
      gV[3 + k] = gbb * pj.V[k] + 2.f * gc * pj.V[3 + k];
    }
    // V_rk = Wm_rk s_k with Wm = T Rq
    float gT[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gR[9];
    for (int k = 0; k < 9; k++) gR[k] = 0.f;
    for (int k = 0; k < 3; k++) {
      float gs = 0.f;
      for (int r = 0; r < 2; r++) {
        float wm = pj.Tm[r * 3 + 0] * F.Rq[k] + pj.Tm[r * 3 + 1] * F.Rq[3 + k] + pj.Tm[r * 3 + 2] * F.Rq[6 + k];
        gs += gV[r * 3 + k] * wm;
        float gw = gV[r * 3 + k] * F.s[k];
        for (int j = 0; j < 3; j++) {
          gT[r * 3 + j] += gw * F.Rq[j * 3 + k];
          gR[j * 3 + k] += pj.Tm[r * 3 + j] * gw;
        }
      }
      gls[k] += gs * F.s[k];
    }
    // rotation matrix -> normalised quaternion (w, x, y, z)
    const float w = F.qn[0], x = F.qn[1], y = F.qn[2], z = F.qn[3];
    float gw_ = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    float gx_ = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] -
                       2.f * x * gR[8]);
    float gy_ = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] -
                       2.f * y * gR[8]);
    float gz_ = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] +
                       x * gR[6] + y * gR[7]);
    float qd = gw_ * w + gx_ * x + gy_ * y + gz_ * z;
    gq[0] += (gw_ - qd * w) * F.qinv;
    gq[1] += (gx_ - qd * x) * F.qinv;
    gq[2] += (gy_ - qd * y) * F.qinv;
    gq[3] += (gz_ - qd * z) * F.qinv;

    // T = J W: row 0 = fx/tz (W0 - ctx W2), row 1 = fy/tz (W1 - cty W2)
    float gt[3] = {0.f, 0.f, 0.f};
    const float iz = pj.iz, iz2 = iz * iz;
    for (int k = 0; k < 3; k++) {
      const float W0 = C.R[k], W1 = C.R[3 + k], W2 = C.R[6 + k];
      if (pj.fclamp & 8) {
        gt[2] += gT[k] * (-pj.Tm[k] * iz);
      } else {
        gt[0] += gT[k] * (-C.fx * W2 * iz2);
        gt[2] += gT[k] * (-C.fx * W0 * iz2 + 2.f * C.fx * pj.t[0] * W2 * iz2 * iz);
      }
      if (pj.fclamp & 16) {
        gt[2] += gT[3 + k] * (-pj.Tm[3 + k] * iz);
      } else {
        gt[1] += gT[3 + k] * (-C.fy * W2 * iz2);
        gt[2] += gT[3 + k] * (-C.fy * W1 * iz2 + 2.f * C.fy * pj.t[1] * W2 * iz2 * iz);
      }
    }
    // 2D mean u = fx tx/tz + cx, v = fy ty/tz + cy
    gt[0] += gu * C.fx * iz;
    gt[1] += gv * C.fy * iz;
    gt[2] += -(gu * C.fx * pj.t[0] + gv * C.fy * pj.t[1]) * iz2;
    // t = R m + t_cam
    for (int k = 0; k < 3; k++) gm[k] += C.R[k] * gt[0] + C.R[3 + k] * gt[1] + C.R[6 + k] * gt[2];
  }
  for (int k = 0; k < 3; k++) out.mean[k * n + i] = gm[k];
  for (int k = 0; k < 3; k++) out.ls[k * n + i] = gls[k];
  for (int k = 0; k < 4; k++) out.quat[k * n + i] = gq[k];
  out.logit[i] = glogit;
  if constexpr (kOneView) {
    if (!sh_written)
      for (int k = 0; k < nc; k++)
        for (int ch = 0; ch < 3; ch++) out.sh[(int64_t)(k * 3 + ch) * n + i] = 0.f;
  } else {
    for (int k = 0; k < nc; k++)
      for (int ch = 0; ch < 3; ch++) out.sh[(int64_t)(k * 3 + ch) * n + i] = gsh[k][ch];
  }
}

}  // namespace ags

extern "C" size_t ags_backward_workspace_bytes(int64_t n, int32_t views) {
  if (n < 0 || views < 1) return 0;
  return (size_t)n * (size_t)views * ags::kGradStride * sizeof(float);
}

extern "C" ags_status ags_rasterize_backward(const ags_gaussians* g, const ags_camera* cams, int32_t views,
                                             const ags_params* params, const ags_projected* proj,
                                             const uint32_t* sorted_vals, const uint32_t* ranges,
                                             const float* final_T, const uint32_t* n_contrib,
                                             const float* dL_dimage, float* g_mean, float* g_log_scale,
                                             float* g_quat, float* g_opacity_logit, float* g_sh, int64_t* d_status,
                                             void* ws, size_t ws_bytes, void* stream) {
  using namespace ags;
  if (!g || !proj || !ranges || !final_T || !n_contrib || !dL_dimage || !d_status) return AGS_ERR_INVALID_ARG;
  if ((uintptr_t)ranges & 7u) return AGS_ERR_INVALID_ARG;       // read as 8-byte (start, end) pairs
  if (!g_mean || !g_log_scale || !g_quat || !g_opacity_logit || !g_sh) return AGS_ERR_INVALID_ARG;
  if (g->n < 0 || g->n > (int64_t)1 << 31) return AGS_ERR_INVALID_ARG;
  CamBatch cb;
  DevParams dp;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  s = build_params(params, &dp);
  if (s != AGS_OK) return s;
  if (g->n * (int64_t)views > (int64_t)UINT32_MAX) return AGS_ERR_INVALID_ARG;   // pair values are 32-bit
  if (g->n == 0) return AGS_OK;
  if (!ws || ws_bytes < ags_backward_workspace_bytes(g->n, views) || ((uintptr_t)ws & 3u)) return AGS_ERR_INVALID_ARG;
  if (!proj->splat || !proj->flags || !sorted_vals || ((uintptr_t)proj->splat & 15u)) return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float* gs = reinterpret_cast<float*>(ws);
  cudaError_t e = cudaMemsetAsync(gs, 0, ags_backward_workspace_bytes(g->n, views), st);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  const int tiles_per_view = cb.c[0].gx * cb.c[0].gy;
  BlendConst bc = make_blend_const(dp);
  raster_backward_kernel<<<(unsigned)(tiles_per_view * views), 128, 0, st>>>(
      reinterpret_cast<const float4*>(proj->splat), sorted_vals, reinterpret_cast<const uint2*>(ranges), cb.c[0].W,
      cb.c[0].H, cb.c[0].gx, tiles_per_view, bc, final_T, n_contrib, dL_dimage, gs, (uint32_t)(g->n * views),
      d_status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  GradOut go{g_mean, g_log_scale, g_quat, g_opacity_logit, g_sh};
  const unsigned grid = (unsigned)((g->n + 127) / 128);
  if (views == 1)
    preprocess_backward_kernel<true><<<grid, 128, 0, st>>>(g->mean, g->log_scale, g->quat, g->opacity_logit, g->sh,
                                                           g->n, views, cb, dp, proj->flags, gs, proj->splat, go);
  else
    preprocess_backward_kernel<false><<<grid, 128, 0, st>>>(g->mean, g->log_scale, g->quat, g->opacity_logit, g->sh,
                                                            g->n, views, cb, dp, proj->flags, gs, proj->splat, go);
  return launch_status(cudaGetLastError());
}
