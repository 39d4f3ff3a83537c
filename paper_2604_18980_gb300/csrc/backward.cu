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

__global__ void __launch_bounds__(kRasterThreads)
raster_backward_kernel(const float4* __restrict__ splat, const uint32_t* __restrict__ vals,
                       const uint2* __restrict__ ranges, int W, int H, int gx, int tiles_per_view, BlendConst bc,
                       const float* __restrict__ final_T, const uint32_t* __restrict__ n_contrib,
                       const float* __restrict__ dL_dimage, float* __restrict__ gsplat) {
  __shared__ float4 s_a[kRasterThreads];    // u v a2 b2
  __shared__ float4 s_b[kRasterThreads];    // c2 l2s r g
  __shared__ float4 s_o[kRasterThreads];    // A B C opacity (original units, for the gradients)
  __shared__ float2 s_f[kRasterThreads];    // eigenframe (cos, sin) of the conic
  __shared__ float s_c[kRasterThreads];
  __shared__ uint32_t s_m[kRasterThreads];
  __shared__ uint32_t s_e[kRasterThreads];
  __shared__ uint32_t s_maxlast;

  const int tile = blockIdx.x;
  const int view = tile / tiles_per_view;
  const int lt = tile - view * tiles_per_view;
  const int ty = lt / gx, tx = lt - ty * gx;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int lx, ly;
  tile_pixel(tid, lx, ly);
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  const bool inside = px < W && py < H;
  const float fpx = (float)px, fpy = (float)py;
  const uint2 rg = __ldg(ranges + tile);
  const uint32_t start = rg.x, end = rg.y;

  const size_t hw = (size_t)W * H;
  float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  uint32_t last = 0;
  if (inside) {
    const size_t op = (size_t)view * hw + (size_t)py * W + px;
    T = final_T[op];
    last = n_contrib[op];
    const size_t o = (size_t)view * 3 * hw + (size_t)py * W + px;
    g0 = dL_dimage[o];
    g1 = dL_dimage[o + hw];
    g2 = dL_dimage[o + 2 * hw];
  }
  float R0 = bc.bg[0], R1 = bc.bg[1], R2 = bc.bg[2];
  if (tid == 0) s_maxlast = 0u;
  __syncthreads();
  if (last) atomicMax(&s_maxlast, last);
  __syncthreads();
  const uint32_t maxlast = min(s_maxlast, end - start);
  // the warp walks only the positions below its own largest "last"
  const uint32_t wlast = __reduce_max_sync(0xffffffffu, last);

  for (int32_t bend = (int32_t)maxlast; bend > 0; bend -= kRasterThreads) {
    const int32_t bbeg = max(0, bend - kRasterThreads);
    const int nb = bend - bbeg;
    __syncthreads();
    if (tid < nb) {
      const uint32_t e = __ldg(vals + start + bbeg + tid);
      const float4* rec = splat + (size_t)e * 3;
      Staged st;
      uint32_t m;
      stage_splat<8, 4>(rec, tx * kTile, ty * kTile, bc.l2tau, st, m);
      const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
      s_a[tid] = st.a;
      s_b[tid] = st.b;
      s_c[tid] = st.c;
      s_o[tid] = make_float4(r0.z, r0.w, r1.x, r1.y);
      float ca, sa;
      conic_frame(r0.z, r0.w, r1.x, ca, sa);
      s_f[tid] = make_float2(ca, sa);
      s_m[tid] = m;
      s_e[tid] = e;
    }
    __syncthreads();
    const int jtop = min(nb, (int)wlast - bbeg);
    for (int j = jtop - 1; j >= 0; j--) {
      if (!((s_m[j] >> warp) & 1u)) continue;         // warp-uniform skip, as in the forward
      const uint32_t pos = (uint32_t)(bbeg + j);       // 0-based position in the tile list
      Staged s;
      s.a = s_a[j];
      s.b = s_b[j];
      const float cbl = s_c[j];
      float gu = 0.f, gv = 0.f, gA = 0.f, gB = 0.f, gC = 0.f, gO = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
      bool contrib = false;
      if (pos < last) {
        float dx, dy;
        const float q = splat_q(s, fpx, fpy, dx, dy);
        if (splat_accept(q, s.b.y)) {
          const float raw = __fmul_rn(bc.tau, fast_exp2(q));
          const float alpha = fminf(bc.alpha_max, raw);
          contrib = true;
          const float4 o = s_o[j];
          const float om = 1.f - alpha;
          T = T / om;
          const float w = alpha * T;
          gr = w * g0;
          gg = w * g1;
          gb = w * g2;
          const float dLda = T * (g0 * (s.b.z - R0) + g1 * (s.b.w - R1) + g2 * (cbl - R2));
          R0 = s.b.z * alpha + om * R0;
          R1 = s.b.w * alpha + om * R1;
          R2 = cbl * alpha + om * R2;
          if (!(raw > bc.alpha_max)) {
            const float dLdp = dLda * alpha;
            gO = dLda * (alpha / o.w);
            gu = -dLdp * (o.x * dx + o.y * dy);
            gv = -dLdp * (o.y * dx + o.z * dy);
            const float2 f = s_f[j];
            const float da = f.x * dx + f.y * dy, db = f.x * dy - f.y * dx;
            gA = -0.5f * dLdp * da * da;
            gB = -dLdp * da * db;
            gC = -0.5f * dLdp * db * db;
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        gu = warp_sum(gu); gv = warp_sum(gv); gA = warp_sum(gA); gB = warp_sum(gB); gC = warp_sum(gC);
        gO = warp_sum(gO); gr = warp_sum(gr); gg = warp_sum(gg); gb = warp_sum(gb);
        if (lane == 0) {
          float* G = gsplat + (size_t)s_e[j] * kGradStride;
          atomicAdd(G + 0, gu); atomicAdd(G + 1, gv); atomicAdd(G + 2, gA); atomicAdd(G + 3, gB);
          atomicAdd(G + 4, gC); atomicAdd(G + 5, gO); atomicAdd(G + 6, gr); atomicAdd(G + 7, gg);
          atomicAdd(G + 8, gb);
        }
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

__global__ void __launch_bounds__(128)
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
  for (int k = 0; k < 3; k++) m[k] = mean[k * n + i];
  for (int k = 0; k < 3; k++) ls[k] = lsc[k * n + i];
  for (int k = 0; k < 4; k++) q[k] = quat[k * n + i];
  const float logit = logit_in[i];
  float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, glogit = 0.f;
  float gsh[16][3];
  for (int k = 0; k < 16; k++) gsh[k][0] = gsh[k][1] = gsh[k][2] = 0.f;
  Frame F;
  make_frame(ls, q, logit, F);

  for (int view = 0; view < views; view++) {
    const int64_t e = (int64_t)view * n + i;
    const uint8_t fl = flags[e];
    if (fl & kFlagCulled) continue;
    const float* G = gsplat + (size_t)e * kGradStride;
    const float gu = G[0], gv = G[1], gA = G[2], gB = G[3], gC = G[4], gO = G[5];
    const float gcol[3] = {(fl & 1) ? 0.f : G[6], (fl & 2) ? 0.f : G[7], (fl & 4) ? 0.f : G[8]};
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
    for (int k = 0; k < nc; k++) {
      float s0 = sh[(int64_t)(k * 3 + 0) * n + i], s1 = sh[(int64_t)(k * 3 + 1) * n + i],
            s2 = sh[(int64_t)(k * 3 + 2) * n + i];
      wk[k] = gcol[0] * s0 + gcol[1] * s1 + gcol[2] * s2;
      gsh[k][0] += gcol[0] * Y[k];
      gsh[k][1] += gcol[1] * Y[k];
      gsh[k][2] += gcol[2] * Y[k];
    }
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
    const float4 c0 = __ldg(reinterpret_cast<const float4*>(conic_rec + (size_t)e * kSplatFloats));
    const float cC = conic_rec[(size_t)e * kSplatFloats + 4];
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
  for (int k = 0; k < nc; k++)
    for (int ch = 0; ch < 3; ch++) out.sh[(int64_t)(k * 3 + ch) * n + i] = gsh[k][ch];
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
  if (!g_mean || !g_log_scale || !g_quat || !g_opacity_logit || !g_sh) return AGS_ERR_INVALID_ARG;
  if (g->n < 0 || g->n > (int64_t)1 << 31) return AGS_ERR_INVALID_ARG;
  CamBatch cb;
  DevParams dp;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  s = build_params(params, &dp);
  if (s != AGS_OK) return s;
  if (g->n == 0) return AGS_OK;
  if (!ws || ws_bytes < ags_backward_workspace_bytes(g->n, views) || ((uintptr_t)ws & 3u)) return AGS_ERR_INVALID_ARG;
  if (!proj->splat || !proj->flags || !sorted_vals || ((uintptr_t)proj->splat & 15u)) return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float* gs = reinterpret_cast<float*>(ws);
  cudaError_t e = cudaMemsetAsync(gs, 0, ags_backward_workspace_bytes(g->n, views), st);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  const int tiles_per_view = cb.c[0].gx * cb.c[0].gy;
  BlendConst bc = make_blend_const(dp);
  raster_backward_kernel<<<(unsigned)(tiles_per_view * views), kRasterThreads, 0, st>>>(
      reinterpret_cast<const float4*>(proj->splat), sorted_vals, reinterpret_cast<const uint2*>(ranges), cb.c[0].W,
      cb.c[0].H, cb.c[0].gx, tiles_per_view, bc, final_T, n_contrib, dL_dimage, gs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  GradOut go{g_mean, g_log_scale, g_quat, g_opacity_logit, g_sh};
  preprocess_backward_kernel<<<(unsigned)((g->n + 127) / 128), 128, 0, st>>>(
      g->mean, g->log_scale, g->quat, g->opacity_logit, g->sh, g->n, views, cb, dp, proj->flags, gs, proj->splat, go);
  return launch_status(cudaGetLastError());
}
