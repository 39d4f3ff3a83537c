// visible.cu -- stable compaction of the Gaussian-views that have pairs,
// with their depth keys: the input of the depth pre-sort; and the view of each
// entry of the sorted order (ags_view_keys), the key of the one stable pass
// that groups the depth order view by view for view-major tile keys.
//
// A culled Gaussian-view (no pairs in its view, Sec. 2.1 frustum cull and
// Sec. 3.3 Th > opacity cull) never reaches a tile list, so the depth
// pre-sort needs only the others.  One pass: each 256-thread block takes 4096
// consecutive entries e (16 per thread, read as 16-byte vectors), counts the
// visible ones, scans the counts, finds its output offset with a decoupled
// look-back over the preceding blocks (bounded spin), and writes
// (float_bits(depth[e]), e) for its visible entries in increasing e -- so each
// view's entries keep increasing Gaussian index, the tie order of the sort.
#include <algorithm>

#include "ags_internal.cuh"

namespace ags {

constexpr int kVisThreads = 256;
constexpr int kVisItems = 16;
constexpr int kVisPart = kVisThreads * kVisItems;     // 4096 entries per partition
constexpr uint64_t kVisAgg = 1ull << 62;
constexpr uint64_t kVisInc = 2ull << 62;
constexpr uint64_t kVisMask = (1ull << 62) - 1;

__global__ void __launch_bounds__(kVisThreads)
visible_kernel(const uint8_t* __restrict__ flags, const float* __restrict__ depth, uint32_t total,
               uint32_t* __restrict__ keys, uint32_t* __restrict__ ids, int64_t* d_count, int64_t* status,
               uint64_t* part_status, uint32_t* counter, uint32_t num_parts) {
  __shared__ uint32_t s_warp[kVisThreads / 32];
  __shared__ uint32_t s_part;
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_part = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t part = s_part;
  const uint32_t i0 = part * kVisPart + (uint32_t)tid * kVisItems;

  // this thread's 16 entries: visibility mask and depth bits
  uint32_t vis = 0u;
  uint32_t dbits[kVisItems];
  if (i0 + kVisItems <= total) {
    const uint4 f = __ldcs(reinterpret_cast<const uint4*>(flags + i0));
    const uint32_t fw[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int k = 0; k < kVisItems; k++)
      if (!((fw[k >> 2] >> (8 * (k & 3))) & kFlagCulled)) vis |= 1u << k;
    const float4* d4 = reinterpret_cast<const float4*>(depth + i0);
#pragma unroll
    for (int q = 0; q < kVisItems / 4; q++) {
      const float4 d = __ldcs(d4 + q);
      dbits[4 * q] = __float_as_uint(d.x);
      dbits[4 * q + 1] = __float_as_uint(d.y);
      dbits[4 * q + 2] = __float_as_uint(d.z);
      dbits[4 * q + 3] = __float_as_uint(d.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < kVisItems; k++) {
      dbits[k] = 0u;
      if (i0 + k < total && !(flags[i0 + k] & kFlagCulled)) {
        vis |= 1u << k;
        dbits[k] = __float_as_uint(depth[i0 + k]);
      }
    }
  }
  const uint32_t cnt = (uint32_t)__popc(vis);

  // block scan of the counts
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0, agg = 0;
#pragma unroll
  for (int w = 0; w < kVisThreads / 32; w++) {
    const uint32_t v = s_warp[w];
    if (w < warp) wpre += v;
    agg += v;
  }

  // decoupled look-back (warp 0): 32 predecessors per poll
  if (warp == 0) {
    uint64_t excl = 0;
    if (part == 0) {
      if (lane == 0) st_relaxed_u64(part_status, kVisInc | (uint64_t)agg);
    } else {
      if (lane == 0) st_relaxed_u64(part_status + part, kVisAgg | (uint64_t)agg);
      int64_t top = (int64_t)part - 1;
      const uint64_t t0 = globaltimer_ns();
      bool timed_out = false;
      while (true) {
        const int64_t q = top - lane;
        const uint64_t sv = q >= 0 ? ld_relaxed_u64(part_status + q) : kVisInc;
        const uint32_t flag = (uint32_t)(sv >> 62);
        const unsigned inc_mask = __ballot_sync(0xffffffffu, flag == 2u);
        const unsigned none_mask = __ballot_sync(0xffffffffu, flag == 0u);
        const int first_inc = inc_mask ? __ffs(inc_mask) - 1 : 32;
        const unsigned upto = first_inc >= 31 ? 0xffffffffu : ((2u << first_inc) - 1u);
        if ((none_mask & upto) && !timed_out) {
          if (globaltimer_ns() - t0 > kWaitLimitNs) {
            timed_out = true;
            if (lane == 0) set_status(status, AGS_ERR_TIMEOUT, kStageVisible);
          }
          continue;
        }
        excl += warp_sum((lane <= first_inc && flag != 0u) ? (sv & kVisMask) : 0ull);
        if (first_inc < 32 || timed_out) break;
        top -= 32;
      }
      if (lane == 0) st_relaxed_u64(part_status + part, kVisInc | ((excl + agg) & kVisMask));
    }
    if (lane == 0) s_prefix = excl;
  }
  __syncthreads();

  // write this thread's visible entries in index order
  uint32_t o = (uint32_t)s_prefix + wpre + incl - cnt;
  uint32_t m = vis;
  while (m) {
    const int k = __ffs(m) - 1;
    m &= m - 1;
    if (o < total) {
      keys[o] = dbits[k];
      ids[o] = i0 + (uint32_t)k;
    }
    o++;
  }
  if (part == num_parts - 1 && tid == 0) *d_count = (int64_t)(s_prefix + agg);
}

static size_t vis_parts(int64_t total) { return (size_t)((total + kVisPart - 1) / kVisPart); }

}  // namespace ags

extern "C" size_t ags_compact_workspace_bytes(int64_t n, int32_t views) {
  if (n < 0 || views < 1) return 0;
  return 256 + 8 * ags::vis_parts(n * (int64_t)views);
}

extern "C" ags_status ags_compact_visible(const ags_projected* proj, int64_t n, int32_t views, uint32_t* keys,
                                          uint32_t* ids, int64_t* d_count, int64_t* d_status, void* ws,
                                          size_t ws_bytes, void* stream) {
  using namespace ags;
  if (!proj || !d_count || !d_status || n < 0 || views < 1 || views > AGS_MAX_VIEWS) return AGS_ERR_INVALID_ARG;
  const int64_t total = n * (int64_t)views;
  if (total >= ((int64_t)1 << 32) - kVisPart) return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (total == 0) return launch_status(cudaMemsetAsync(d_count, 0, sizeof(int64_t), st));
  if (!proj->flags || !proj->depth || !keys || !ids) return AGS_ERR_INVALID_ARG;
  if (((uintptr_t)proj->flags & 15u) || ((uintptr_t)proj->depth & 15u)) return AGS_ERR_INVALID_ARG;
  if (!ws || ws_bytes < ags_compact_workspace_bytes(n, views) || ((uintptr_t)ws & 7u)) return AGS_ERR_INVALID_ARG;
  const size_t parts = vis_parts(total);
  cudaError_t e = cudaMemsetAsync(ws, 0, 256 + 8 * parts, st);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws);
  uint64_t* part_status = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ws) + 256);
  visible_kernel<<<(unsigned)parts, kVisThreads, 0, st>>>(proj->flags, proj->depth, (uint32_t)total, keys, ids,
                                                          d_count, d_status, part_status, counter,
                                                          (uint32_t)parts);
  return launch_status(cudaGetLastError());
}

namespace ags {

__global__ void __launch_bounds__(256) view_keys_kernel(const uint32_t* __restrict__ order, const int64_t* d_count,
                                                        int64_t capacity, uint32_t n, uint32_t* __restrict__ keys) {
  int64_t count = *d_count;
  count = count < 0 ? 0 : (count > capacity ? capacity : count);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
    keys[k] = __ldg(order + k) / n;
}

}  // namespace ags

extern "C" ags_status ags_view_keys(const uint32_t* order, const int64_t* d_count, int64_t capacity, int64_t n,
                                    uint32_t* keys, void* stream) {
  using namespace ags;
  if (!d_count || capacity < 0 || n < 1 || n > ((int64_t)1 << 32) - 1) return AGS_ERR_INVALID_ARG;
  if (capacity == 0) return AGS_OK;
  if (!order || !keys) return AGS_ERR_INVALID_ARG;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<int64_t>((capacity + 255) / 256, (int64_t)sms * 8);
  view_keys_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(order, d_count, capacity, (uint32_t)n, keys);
  return launch_status(cudaGetLastError());
}
