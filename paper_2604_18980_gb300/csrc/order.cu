// order.cu -- storage order of the Gaussians (not in the paper).
//
// The preprocess runs one thread per Gaussian and a warp's 32 Gaussians go
// through every view together.  In a large scene most Gaussian-views are
// culled (behind the camera or off the image), but when a warp's Gaussians are
// scattered over the scene almost every warp keeps a few in every view and
// pays the full projection for them.  Stored along a Morton (Z-order) curve of
// their means, a warp's Gaussians lie close together and are culled together.
//
//   ags_morton_codes       30-bit Morton code of every mean (10 bits per axis
//                          over the means' bounding box)
//   ags_gather_gaussians   every attribute array permuted: dst[k] = src[perm[k]]
//
// The permutation itself is a stable sort of the codes (ags_sort32 with
// identity values).  Rendering the permuted scene gives the same images: the
// pair lists order equal depths by index, so only Gaussians of exactly equal
// depth in one tile can swap places.
#include <algorithm>

#include "ags_internal.cuh"

namespace ags {

// Order-preserving map of a float to an unsigned key (and back).
__device__ __forceinline__ uint32_t ordered_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Bounding box of the finite means: box[0..2] minimum keys, box[3..5] maximum
// keys (box preset to all-ones and zeros).
__global__ void __launch_bounds__(256) bbox_kernel(const float* __restrict__ mean, int64_t n, uint32_t* box) {
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = __ldg(mean + i), y = __ldg(mean + n + i), z = __ldg(mean + 2 * n + i);
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) continue;
    const uint32_t k[3] = {ordered_key(x), ordered_key(y), ordered_key(z)};
#pragma unroll
    for (int a = 0; a < 3; a++) {
      lo[a] = min(lo[a], k[a]);
      hi[a] = max(hi[a], k[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
    hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      if (lo[a] != 0xffffffffu) atomicMin(box + a, lo[a]);
      if (hi[a] != 0u) atomicMax(box + 3 + a, hi[a]);
    }
  }
}

// 10 bits spread to every third bit position.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Morton code of every mean; a mean that is not finite gets the largest code.
__global__ void __launch_bounds__(256) morton_kernel(const float* __restrict__ mean, int64_t n,
                                                     const uint32_t* __restrict__ box, uint32_t* __restrict__ codes) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float m[3] = {__ldg(mean + i), __ldg(mean + n + i), __ldg(mean + 2 * n + i)};
  if (!(isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]))) {
    codes[i] = 0xffffffffu;
    return;
  }
  uint32_t c = 0u;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const float lo = ordered_float(box[a]), hi = ordered_float(box[3 + a]);
    const float ext = hi - lo;
    const float f = ext > 0.f ? (m[a] - lo) / ext : 0.f;
    const uint32_t q = (uint32_t)fminf(fmaxf(f * 1024.f, 0.f), 1023.f);
    c |= spread3(q) << a;
  }
  codes[i] = c;
}

// dst[r][k] = src[r][perm[k]] for rows r of one structure-of-arrays attribute.
__global__ void __launch_bounds__(256) gather_kernel(const float* __restrict__ src, int64_t n,
                                                     const uint32_t* __restrict__ perm, int rows,
                                                     float* __restrict__ dst) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t p = __ldg(perm + k);
  if ((int64_t)p >= n) return;
  for (int r = 0; r < rows; r++) dst[(int64_t)r * n + k] = __ldg(src + (int64_t)r * n + p);
}

}  // namespace ags

extern "C" size_t ags_morton_workspace_bytes(void) { return 256; }

extern "C" ags_status ags_morton_codes(const ags_gaussians* g, uint32_t* codes, void* ws, size_t ws_bytes,
                                       void* stream) {
  using namespace ags;
  if (!g || g->n < 0 || g->n > (int64_t)1 << 31) return AGS_ERR_INVALID_ARG;
  if (g->n == 0) return AGS_OK;
  if (!g->mean || !codes || !ws || ws_bytes < ags_morton_workspace_bytes() || ((uintptr_t)ws & 3u))
    return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* box = reinterpret_cast<uint32_t*>(ws);
  if (cudaMemsetAsync(box, 0xff, 12, st) != cudaSuccess || cudaMemsetAsync(box + 3, 0, 12, st) != cudaSuccess)
    return AGS_ERR_CUDA;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<int64_t>((g->n + 255) / 256, (int64_t)sms * 8);
  bbox_kernel<<<grid, 256, 0, st>>>(g->mean, g->n, box);
  morton_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, st>>>(g->mean, g->n, box, codes);
  return launch_status(cudaGetLastError());
}

extern "C" ags_status ags_gather_gaussians(const ags_gaussians* src, const uint32_t* perm, int32_t sh_degree,
                                           float* mean, float* log_scale, float* quat, float* opacity_logit,
                                           float* sh, void* stream) {
  using namespace ags;
  if (!src || src->n < 0 || src->n > (int64_t)1 << 31 || sh_degree < 0 || sh_degree > 3) return AGS_ERR_INVALID_ARG;
  if (src->n == 0) return AGS_OK;
  if (!perm || !src->mean || !src->log_scale || !src->quat || !src->opacity_logit || !src->sh || !mean ||
      !log_scale || !quat || !opacity_logit || !sh)
    return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned grid = (unsigned)((src->n + 255) / 256);
  const int nc = (sh_degree + 1) * (sh_degree + 1);
  gather_kernel<<<grid, 256, 0, st>>>(src->mean, src->n, perm, 3, mean);
  gather_kernel<<<grid, 256, 0, st>>>(src->log_scale, src->n, perm, 3, log_scale);
  gather_kernel<<<grid, 256, 0, st>>>(src->quat, src->n, perm, 4, quat);
  gather_kernel<<<grid, 256, 0, st>>>(src->opacity_logit, src->n, perm, 1, opacity_logit);
  gather_kernel<<<grid, 256, 0, st>>>(src->sh, src->n, perm, 3 * nc, sh);
  return launch_status(cudaGetLastError());
}
