// visible.cu -- stable compaction of the Gaussian-views that have pairs,
// with their depth keys: the input of the depth pre-sort; and the view of each
// entry of the sorted order (ags_view_keys), the key of the one stable pass
// that groups the depth order view by view for view-major tile keys.
//
// A culled Gaussian-view (no pairs in its view, Sec. 2.1 frustum cull and
// Sec. 3.3 Th > opacity cull) never reaches a tile list, so the depth
// pre-sort needs only the others.  Reduce, then scan, then write -- three
// launches and no block ever waits for another: (1) each 256-thread block
// counts the visible entries of one 4096-entry partition from the flags (16
// per thread, read as 16-byte vectors); (2) one block scans the partition
// counts into offsets and writes the total; (3) each block re-reads its
// partition's flags, ranks its visible entries with a block scan, reads their
// depths, stages (float_bits(depth[e]), e) in shared memory and writes them
// out coalesced at its offset -- so the entries keep increasing e and each
// view's entries increasing Gaussian index, the tie order of the sort.
#include <algorithm>

#include "ags_internal.cuh"

namespace ags {

constexpr int kVisThreads = 256;
constexpr int kVisItems = 16;
constexpr int kVisPart = kVisThreads * kVisItems;     // 4096 entries per partition
constexpr int kVisScanThreads = 1024;

// Visibility bits of this thread's 16 entries i0 .. i0+15 (bit k: entry i0+k).
__device__ __forceinline__ uint32_t visible_bits(const uint8_t* __restrict__ flags, uint32_t i0, uint32_t total) {
  uint32_t vis = 0u;
  if (i0 + kVisItems <= total) {
    const uint4 f = __ldg(reinterpret_cast<const uint4*>(flags + i0));
    const uint32_t fw[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int k = 0; k < kVisItems; k++)
      if (!((fw[k >> 2] >> (8 * (k & 3))) & kFlagCulled)) vis |= 1u << k;
  } else {
    for (int k = 0; k < kVisItems; k++)
      if (i0 + k < total && !(flags[i0 + k] & kFlagCulled)) vis |= 1u << k;
  }
  return vis;
}

// (1) visible entries per partition, and each thread's visibility bits for (3)
__global__ void __launch_bounds__(kVisThreads)
visible_count_kernel(const uint8_t* __restrict__ flags, uint32_t total, uint32_t* __restrict__ part_count,
                     uint16_t* __restrict__ masks) {
  __shared__ uint32_t s_warp[kVisThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t i0 = blockIdx.x * (uint32_t)kVisPart + (uint32_t)tid * kVisItems;
  const uint32_t vis = visible_bits(flags, i0, total);
  masks[(size_t)blockIdx.x * kVisThreads + tid] = (uint16_t)vis;
  const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(vis));
  if (lane == 0) s_warp[warp] = c;
  __syncthreads();
  if (tid == 0) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kVisThreads / 32; w++) t += s_warp[w];
    part_count[blockIdx.x] = t;
  }
}

// (2) exclusive scan of the partition counts in place (one block, chunks of
// 1024 x 16 partitions with a running carry); the total goes to *d_count
__global__ void __launch_bounds__(kVisScanThreads)
visible_scan_kernel(uint32_t* __restrict__ part, uint32_t parts, int64_t* d_count) {
  __shared__ uint32_t s_warp[kVisScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t carry = 0;
  for (uint32_t base = 0; base < parts; base += kVisScanThreads * 16u) {
    const uint32_t j0 = base + (uint32_t)tid * 16u;
    uint32_t v[16], t = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      v[k] = j0 + k < parts ? part[j0 + k] : 0u;
      t += v[k];
    }
    uint32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t wpre = 0, agg = 0;
#pragma unroll 4
    for (int w = 0; w < kVisScanThreads / 32; w++) {
      const uint32_t x = s_warp[w];
      if (w < warp) wpre += x;
      agg += x;
    }
    uint64_t run = carry + wpre + incl - t;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      if (j0 + k < parts) part[j0 + k] = (uint32_t)run;
      run += v[k];
    }
    carry += agg;
    __syncthreads();     // s_warp is reused by the next chunk
  }
  if (tid == 0) *d_count = (int64_t)carry;
}

// (3) the visible entries of one partition, written at its offset
__global__ void __launch_bounds__(kVisThreads)
visible_write_kernel(const uint16_t* __restrict__ masks, const float* __restrict__ depth,
                     const uint32_t* __restrict__ part_off, uint32_t* __restrict__ keys, uint32_t* __restrict__ ids) {
  __shared__ uint32_t s_key[kVisPart];
  __shared__ uint32_t s_id[kVisPart];
  __shared__ uint32_t s_warp[kVisThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t p0 = blockIdx.x * (uint32_t)kVisPart;
  const uint32_t i0 = p0 + (uint32_t)tid * kVisItems;
  const uint32_t vis = __ldg(masks + (size_t)blockIdx.x * kVisThreads + tid);
  const uint32_t cnt = (uint32_t)__popc(vis);
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  // this thread's depths (only where an entry is visible) while the scan settles
  uint32_t o = incl - cnt;
  uint32_t m = vis;
  uint32_t dk[kVisItems];
#pragma unroll
  for (int k = 0; k < kVisItems; k++) dk[k] = (m >> k) & 1u ? __float_as_uint(__ldg(depth + i0 + k)) : 0u;
  __syncthreads();
  uint32_t wpre = 0, agg = 0;
#pragma unroll
  for (int w = 0; w < kVisThreads / 32; w++) {
    const uint32_t x = s_warp[w];
    if (w < warp) wpre += x;
    agg += x;
  }
  o += wpre;
#pragma unroll
  for (int k = 0; k < kVisItems; k++) {
    if ((m >> k) & 1u) {
      s_key[o] = dk[k];
      s_id[o] = i0 + (uint32_t)k;
      o++;
    }
  }
  __syncthreads();
  const uint32_t base = __ldg(part_off + blockIdx.x);
  for (uint32_t k = (uint32_t)tid; k < agg; k += kVisThreads) {   // base + agg <= the entries
    keys[base + k] = s_key[k];
    ids[base + k] = s_id[k];
  }
}

static size_t vis_parts(int64_t total) { return (size_t)((total + kVisPart - 1) / kVisPart); }

}  // namespace ags

extern "C" size_t ags_compact_workspace_bytes(int64_t n, int32_t views) {
  if (n < 0 || views < 1) return 0;
  const size_t parts = ags::vis_parts(n * (int64_t)views);
  return 256 + 8 * parts + sizeof(uint16_t) * ags::kVisThreads * parts;   // header, counts, visibility masks
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
  uint32_t* part = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ws) + 256);
  uint16_t* masks = reinterpret_cast<uint16_t*>(reinterpret_cast<char*>(ws) + 256 + 8 * parts);
  visible_count_kernel<<<(unsigned)parts, kVisThreads, 0, st>>>(proj->flags, (uint32_t)total, part, masks);
  visible_scan_kernel<<<1, kVisScanThreads, 0, st>>>(part, (uint32_t)parts, d_count);
  visible_write_kernel<<<(unsigned)parts, kVisThreads, 0, st>>>(masks, proj->depth, part, keys, ids);
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
