// preprocess.cu -- per-Gaussian preprocess with the AdaGScale threshold.
//
// Paper: AdaGScale (arXiv 2604.18980).  Sec. 2.1 (preprocessing: cull,
// projected 2D mean and covariance, colour, depth), Eq. 10 (Th), Sec. 3.3
// (cull when Th > opacity; Th shrinks only the footprint used by the tile
// test), Sec. 3.4 (T_up from a depth look-up table).
//
// One thread per Gaussian, looping over all views of the batch: the
// structure-of-arrays geometry is read once (coalesced) whatever the number of
// views; the 48 SH floats are read only for views in which the Gaussian
// survives and touches a tile (from DRAM the first time, then from cache), by
// a block-wide colour pass over the queued survivors.  Outputs per view and
// survivor: a 48-byte splat record (three 16-byte stores), depth, the tile
// rectangle (one 8-byte store), the tile count, a flag byte and the depth key.
#include "ellipse.cuh"
#include "project.cuh"

namespace ags {

struct PreIn {
  const float* mean;
  const float* ls;
  const float* quat;
  const float* logit;
  const float* sh;
};

struct PreOut {
  float* splat;
  float* depth;
  uint16_t* rect;
  uint32_t* touched;
  uint8_t* flags;
  uint32_t* dkey;
};

__device__ __forceinline__ void write_culled(const PreOut& o, int64_t e) {
  reinterpret_cast<uint2*>(o.rect)[e] = make_uint2(0u, 0u);
  if (o.touched) o.touched[e] = 0u;
  o.flags[e] = kFlagCulled;
  if (o.dkey) o.dkey[e] = 0xffffffffu;
}

// Tiles [t0, t1) holding a pixel centre in [lo, hi] on an axis of `len` pixels.
__device__ __forceinline__ void tile_span(float lo, float hi, int len, int& t0, int& t1) {
  float plo = fmaxf(ceilf(lo), 0.f);
  float phi = fminf(floorf(hi), (float)(len - 1));
  if (!(plo <= phi)) { t0 = t1 = 0; return; }
  t0 = (int)plo >> 4;
  t1 = ((int)phi >> 4) + 1;
}

constexpr int kPreThreads = 256;
constexpr int kPreWarps = kPreThreads / 32;
constexpr int kShFloats = 48;                       // SH coefficients x channels of one Gaussian, degree 3
constexpr size_t kPreShBytes = (size_t)kPreWarps * kShFloats * 32 * sizeof(float);

// Colour of one queued survivor (SH at the world-space direction from the
// camera centre, + 0.5, clamped at 0) and the rest of its splat record.  The
// Gaussian's mean and opacity arrive from its lane by shuffles (all lanes call
// this; only `go` lanes write).
__device__ __forceinline__ void colour_job(bool go, float4 jb, uint32_t tg, int64_t iw, int64_t n, const float m[3],
                                           float opac, const CamBatch& cams, const DevParams& P, const float* wsh,
                                           const PreOut& out, int64_t* status) {
  const int gl = (int)(tg & 31u), gv = (int)((tg >> 8) & 0xffu);
  const float mx = __shfl_sync(0xffffffffu, m[0], gl), my = __shfl_sync(0xffffffffu, m[1], gl),
              mz = __shfl_sync(0xffffffffu, m[2], gl), op = __shfl_sync(0xffffffffu, opac, gl);
  if (!go) return;
  const int64_t gi = iw + gl, ge = (int64_t)gv * n + gi;
  const DevCam& C = cams.c[gv];
  const float dx = mx - C.campos[0], dy = my - C.campos[1], dz = mz - C.campos[2];
  const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
  float Y[16];
  sh_basis(P.sh_degree, dx * il, dy * il, dz * il, Y);
  const int nc = (P.sh_degree + 1) * (P.sh_degree + 1);
  float rgb[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int c = 0; c < 16; c++) {
    if (c < nc) {
#pragma unroll
      for (int ch = 0; ch < 3; ch++) rgb[ch] = fmaf(wsh[(c * 3 + ch) * 32 + gl], Y[c], rgb[ch]);
    }
  }
  uint8_t flags = (uint8_t)(tg >> 16);
  bool bad = false;
#pragma unroll
  for (int ch = 0; ch < 3; ch++) {
    if (!isfinite(rgb[ch])) bad = true;
    if (rgb[ch] < 0.f) { rgb[ch] = 0.f; flags |= (uint8_t)(1 << ch); }
  }
  if (bad) {
    if (gv == 0) atomicAdd(reinterpret_cast<unsigned long long*>(status + 2), 1ull);
    write_culled(out, ge);
    return;
  }
  float4* sp = reinterpret_cast<float4*>(out.splat + ge * kSplatFloats);
  sp[1] = make_float4(jb.x, op, rgb[0], rgb[1]);
  sp[2] = make_float4(rgb[2], jb.y, jb.z, jb.w);
  out.flags[ge] = flags;
}

// One thread per Gaussian, looping over all views.  Per view each lane
// projects its Gaussian, computes Th and the tile rectangle and writes either
// the culled record or everything but the colour; the survivors queue up in
// the warp's shared-memory queue, and whenever 32 are waiting (and after the
// last view) the warp evaluates 32 SH colours at once, one per lane.  Culling
// leaves few survivors scattered over the lanes (a few percent of the
// Gaussian-views on city scenes, a fifth after the AdaGScale cull on object
// scenes), so evaluating the colour in the lanes that found them would run the
// SH stage, with most lanes idle, in almost every warp and view.
__global__ void __launch_bounds__(kPreThreads, 3) preprocess_kernel(PreIn in, int64_t n, int views,
                                                                     const __grid_constant__ CamBatch cams,
                                                                     const __grid_constant__ DevParams P,
                                                                     PreOut out, int64_t* status) {
  __shared__ float4 s_job[kPreWarps][64];     // conic C, Th, Sigma_xx, Sigma_yy
  __shared__ uint32_t s_tag[kPreWarps][64];   // lane | view << 8 | frustum-clamp bits << 16

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t i = (int64_t)blockIdx.x * kPreThreads + tid;
  const int64_t iw = i - lane;                // the warp's first Gaussian
  if (iw >= n) return;                        // whole warps only
  const bool active = i < n;

  // geometry: read once for all views
  float m[3] = {0.f, 0.f, 0.f}, ls[3] = {0.f, 0.f, 0.f}, q[4] = {1.f, 0.f, 0.f, 0.f}, logit = 0.f;
  if (active) {
#pragma unroll
    for (int k = 0; k < 3; k++) m[k] = __ldg(in.mean + k * n + i);
#pragma unroll
    for (int k = 0; k < 3; k++) ls[k] = __ldg(in.ls + k * n + i);
#pragma unroll
    for (int k = 0; k < 4; k++) q[k] = __ldg(in.quat + k * n + i);
    logit = __ldg(in.logit + i);
  }
  const bool finite = isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]) && isfinite(ls[0]) && isfinite(ls[1]) &&
                      isfinite(ls[2]) && isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]) &&
                      isfinite(logit);
  if (active && !finite) {
    atomicAdd(reinterpret_cast<unsigned long long*>(status + 2), 1ull);
    for (int view = 0; view < views; view++) write_culled(out, (int64_t)view * n + i);
  }
  const bool ok = active && finite;
  // the SH planes of the warp's 32 Gaussians, copied to shared memory at the
  // first view in which one of them survives, while further views are
  // projected; waited for before the first colour batch (a warp none of whose
  // Gaussians survives anywhere reads no SH)
  extern __shared__ float s_sh[];                       // [kPreWarps][48][32]
  float* wsh = s_sh + warp * kShFloats * 32;
  bool sh_issued = false, sh_ready = false;
  auto sh_issue = [&]() {     // warp-uniform
    if (!sh_issued) {
      if (active) {
        const int planes = (P.sh_degree + 1) * (P.sh_degree + 1) * 3;
        for (int c = 0; c < planes; c++) {
          const uint32_t dst = (uint32_t)__cvta_generic_to_shared(wsh + c * 32 + lane);
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(in.sh + (int64_t)c * n + i)
                       : "memory");
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      sh_issued = true;
    }
  };
  auto sh_wait = [&]() {      // warp-uniform: every lane reaches it together
    if (!sh_ready) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncwarp();
      sh_ready = true;
    }
  };
  Frame F;                    // scales, rotation, R S and opacity: once for all views
  make_frame(ls, q, logit, F);
  const float smax = fmaxf(F.s[0], fmaxf(F.s[1], F.s[2]));
  const float smax2 = smax * smax;
  float4* qj = s_job[warp];
  uint32_t* qt = s_tag[warp];
  int qn = 0;                 // queued survivors (warp-uniform)

  for (int view = 0; view < views; view++) {
    const DevCam& C = cams.c[view];
    const int64_t e = (int64_t)view * n + i;
    bool surv = false;
    float4 job = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t tag = 0u;
    if (ok) {
      Proj pj;
      // off-screen footprints leave before the covariance (same outputs: no tile)
      bool live = project_mean(C, m, pj) && footprint_may_reach(pj, smax2, C.W, C.H) && project_cov(F, pj);
      // footprint radius: plain 3-sigma, or AdaGScale (Eq. 10, Sec. 3.3)
      float th = P.tau, rf = 0.f;
      if (live) {
        if (P.scale_mode == AGS_SCALE_ADAGSCALE) {
          const int bin = (int)fminf(pj.t[2] * P.lut_scale, (float)(P.lut_bins - 1));   // depth > 0: trunc = floor
          const float tup = P.lut[bin];
          if (!(tup > 0.f)) {
            live = false;
          } else {
            th = P.K / (tup * 6.2831853f * sqrtf(pj.det)) + P.tau;
            if (th > F.opac) live = false;
            else rf = ceilf(sqrtf(pj.lam1) * fminf(3.f, sqrtf(2.f * logf(F.opac / th))));
          }
        } else {
          rf = ceilf(3.f * sqrtf(pj.lam1));
        }
      }
      int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
      if (live && rf > 0.f) {
        tile_span(pj.u - rf, pj.u + rf, C.W, x0, x1);
        tile_span(pj.v - rf, pj.v + rf, C.H, y0, y1);
      }
      const uint32_t touched = (uint32_t)(x1 - x0) * (uint32_t)(y1 - y0);
      if (!live || touched == 0u) {
        write_culled(out, e);
      } else {
        // everything but the colour now; the colour pass writes the rest
        reinterpret_cast<float4*>(out.splat + e * kSplatFloats)[0] = make_float4(pj.u, pj.v, pj.A, pj.B);
        out.depth[e] = pj.t[2];
        reinterpret_cast<uint2*>(out.rect)[e] = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16),
                                                           (uint32_t)x1 | ((uint32_t)y1 << 16));
        if (out.touched) out.touched[e] = touched;
        if (out.dkey) out.dkey[e] = __float_as_uint(pj.t[2]);
        surv = true;
        job = make_float4(pj.C, th, pj.a + 0.3f, pj.c + 0.3f);
        tag = (uint32_t)lane | ((uint32_t)view << 8) | ((uint32_t)pj.fclamp << 16);
      }
    }
    // enqueue this view's survivors behind the waiting ones
    const unsigned bal = __ballot_sync(0xffffffffu, surv);
    if (bal) sh_issue();
    if (surv) {
      const int slot = qn + __popc(bal & lanemask_lt());
      qj[slot] = job;
      qt[slot] = tag;
    }
    qn += __popc(bal);
    __syncwarp();
    if (qn >= 32) {           // a full batch: one colour per lane
      sh_wait();
      colour_job(true, qj[lane], qt[lane], iw, n, m, F.opac, cams, P, wsh, out, status);
      __syncwarp();
      if (lane < qn - 32) {
        qj[lane] = qj[lane + 32];
        qt[lane] = qt[lane + 32];
      }
      qn -= 32;
      __syncwarp();
    }
  }
  if (qn > 0) {
    const bool go = lane < qn;
    sh_wait();
    colour_job(go, go ? qj[lane] : make_float4(0.f, 0.f, 0.f, 0.f), go ? qt[lane] : 0u, iw, n, m, F.opac, cams, P,
               wsh, out, status);
  }
  // no copy into this block's shared memory may still be in flight when it exits
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Ellipse tile test (tile_test AGS_TILE_ELLIPSE): the kept tiles of every
// surviving Gaussian-view, from its splat record and square, by the same
// functions the emission enumerates them with.  One warp per 32 consecutive
// Gaussian-views (Gaussian order, so the sizes within a warp are mixed); the
// rows of the 32 are spread over the lanes.  A Gaussian-view without a kept
// tile is culled.
__global__ void __launch_bounds__(256) ellipse_count_kernel(const float4* __restrict__ splat,
                                                            const uint2* __restrict__ rect, int64_t total, int W,
                                                            int H, PreOut out) {
  __shared__ uint32_t s_run[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  EllipseTiles E{0.f, 0.f, 1.f, 0.f, 1.f, -1.f, 0, 0, W, H, 1.f, 1.f};
  int y0 = 0;
  uint32_t h = 0;
  const bool live = e < total && !(out.flags[e] & kFlagCulled);
  if (live) {
    const uint2 r = __ldg(rect + e);
    const float4 s0 = __ldg(splat + e * 3), s1 = __ldg(splat + e * 3 + 1);
    const float th = __ldg(reinterpret_cast<const float*>(splat + e * 3 + 2) + 1);
    E = EllipseTiles{s0.x, s0.y, s0.z, s0.w, s1.x, ellipse_level(s1.y, th), (int)(r.x & 0xffffu),
                     (int)(r.y & 0xffffu), W, H, 0.f, 0.f};
    ellipse_prepare(E);
    y0 = (int)(r.x >> 16);
    h = (r.y >> 16) - (uint32_t)y0;
  }
  const uint32_t c = warp_ellipse_count(E, y0, h, lane, s_run[warp]);
  if (live) {
    if (c) out.touched[e] = c;
    else write_culled(out, e);
  }
}

}  // namespace ags

extern "C" ags_status ags_preprocess(const ags_gaussians* g, const ags_camera* cams, int32_t views,
                                     const ags_params* params, const ags_projected* out, int64_t* d_status,
                                     void* stream) {
  using namespace ags;
  if (!g || !out || !d_status) return AGS_ERR_INVALID_ARG;
  if (g->n < 0 || g->n > (int64_t)1 << 31) return AGS_ERR_INVALID_ARG;
  CamBatch cb;
  DevParams dp;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  s = build_params(params, &dp);
  if (s != AGS_OK) return s;
  if ((int64_t)views * g->n >= ((int64_t)1 << 32)) return AGS_ERR_INVALID_ARG;
  if (g->n == 0) return AGS_OK;
  if (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->sh) return AGS_ERR_INVALID_ARG;
  if (!out->splat || !out->depth || !out->rect || !out->flags) return AGS_ERR_INVALID_ARG;
  if (((uintptr_t)out->splat & 15u) || ((uintptr_t)out->rect & 7u)) return AGS_ERR_INVALID_ARG;
  if (dp.tile_test == AGS_TILE_ELLIPSE && !out->tiles_touched) return AGS_ERR_INVALID_ARG;
  PreIn in{g->mean, g->log_scale, g->quat, g->opacity_logit, g->sh};
  PreOut po{out->splat, out->depth, out->rect, out->tiles_touched, out->flags, out->depth_key};
  cudaError_t ea = cudaFuncSetAttribute(preprocess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kPreShBytes);
  if (ea != cudaSuccess) return launch_status(ea);
  preprocess_kernel<<<(unsigned)((g->n + kPreThreads - 1) / kPreThreads), kPreThreads, kPreShBytes,
                      (cudaStream_t)stream>>>(in, g->n, views, cb, dp, po, d_status);
  if (dp.tile_test == AGS_TILE_ELLIPSE) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return launch_status(e);
    const int64_t total = (int64_t)views * g->n;
    ellipse_count_kernel<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(out->splat), reinterpret_cast<const uint2*>(out->rect), total, cb.c[0].W,
        cb.c[0].H, po);
  }
  return launch_status(cudaGetLastError());
}
