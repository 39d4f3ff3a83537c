// emit.cu -- Gaussian-tile pair emission (Sec. 2.1 pair generation, Sec. 3.3).
//
// Single pass: each 256-thread block takes a partition of 1024 Gaussians
// (partition ids handed out by an atomic counter, so lower partitions are
// always running), computes the pair counts from the tile rectangles, scans
// them inside the block, obtains the global offset of the partition through a
// decoupled look-back over the preceding partitions' published sums, and then
// emits the partition's pairs load-balanced across the block: each warp takes
// chunks of 256 consecutive pairs and stages them in shared memory, so stores
// are coalesced whatever the per-Gaussian tile counts are.
//
//   64-bit keys: key = ((view * tiles_per_view + tile) << 32) | float_bits(depth)
//   32-bit keys: key = view * tiles_per_view + tile (pairs emitted in depth order)
//   val = view * n + i
//
// The look-back spins are bounded (globaltimer); on expiry the status block
// records AGS_ERR_TIMEOUT and every store stays inside `capacity`.
#include <mutex>

#include "ags_internal.cuh"

namespace ags {

constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 4;
constexpr int kEmitPart = kEmitThreads * kEmitItems;      // 1024 Gaussians per partition
constexpr int kEmitRun = 8;                               // pairs generated per lane per chunk
constexpr int kEmitChunk = 32 * kEmitRun;                 // pairs per warp chunk
constexpr int kEmitStride = kEmitRun + 1;                 // padded staging row (fewer bank conflicts)
constexpr uint64_t kAgg = 1ull << 62;
constexpr uint64_t kInc = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

// Pair key of a tile: 64-bit keys append the depth bits, 32-bit keys are the tile alone.
__device__ __forceinline__ void make_key(uint32_t tile, uint32_t dbits, uint64_t& k) {
  k = ((uint64_t)tile << 32) | dbits;
}
__device__ __forceinline__ void make_key(uint32_t tile, uint32_t, uint32_t& k) { k = tile; }

template <typename K>
__global__ void __launch_bounds__(kEmitThreads)
emit_kernel(const uint2* __restrict__ rect, const float* __restrict__ depth, const uint32_t* __restrict__ order,
            int64_t total, uint32_t n, uint32_t tiles_per_view, uint32_t gx, K* __restrict__ keys,
            uint32_t* __restrict__ vals, int64_t capacity, int64_t* d_num_pairs, int64_t* status,
            uint64_t* part_status, uint32_t* counter, uint32_t num_parts) {
  __shared__ uint32_t s_base[kEmitPart];   // key high word of the rectangle's first tile
  __shared__ uint32_t s_w[kEmitPart];      // rectangle width in tiles
  __shared__ uint32_t s_dbits[kEmitPart];  // depth bits
  __shared__ uint32_t s_idx[kEmitPart];    // splat index view*n+i
  __shared__ uint32_t s_off[kEmitPart + 1];
  __shared__ uint32_t s_warp[kEmitThreads / 32];
  __shared__ uint32_t s_part;
  __shared__ unsigned long long s_prefix;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_part = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t part = s_part;
  const int64_t base = (int64_t)part * kEmitPart;

  // 1. coalesced loads of the rectangles (striped), counts staged in s_off
#pragma unroll
  for (int k = 0; k < kEmitItems; k++) {
    int li = k * kEmitThreads + tid;
    int64_t s = base + li;
    uint32_t c = 0;
    if (s < total) {
      uint32_t e = order ? __ldg(order + s) : (uint32_t)s;
      uint2 r = __ldg(rect + e);
      uint32_t x0 = r.x & 0xffffu, y0 = r.x >> 16, x1 = r.y & 0xffffu, y1 = r.y >> 16;
      uint32_t w = x1 - x0;
      c = w * (y1 - y0);
      uint32_t view = e / n;
      s_base[li] = view * tiles_per_view + y0 * gx + x0;
      s_w[li] = w;
      if (sizeof(K) == 8) s_dbits[li] = c ? __float_as_uint(__ldg(depth + e)) : 0u;
      s_idx[li] = e;
    }
    s_off[li] = c;
  }
  __syncthreads();

  // 2. block scan: each thread owns kEmitItems consecutive entries
  uint32_t cnt[kEmitItems];
  uint32_t tsum = 0;
#pragma unroll
  for (int k = 0; k < kEmitItems; k++) {
    cnt[k] = s_off[tid * kEmitItems + k];
    tsum += cnt[k];
  }
  uint32_t incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0, agg = 0;
#pragma unroll
  for (int w = 0; w < kEmitThreads / 32; w++) {
    uint32_t v = s_warp[w];
    if (w < warp) wpre += v;
    agg += v;
  }
  uint32_t texcl = wpre + incl - tsum;

  // 3. decoupled look-back (warp 0) for the partition's global offset
  if (warp == 0) {
    uint64_t excl = 0;
    if (part == 0) {
      if (lane == 0) st_relaxed_u64(part_status, kInc | (uint64_t)agg);
    } else {
      if (lane == 0) st_relaxed_u64(part_status + part, kAgg | (uint64_t)agg);
      int64_t top = (int64_t)part - 1;
      const uint64_t t0 = globaltimer_ns();
      bool timed_out = false;
      while (true) {
        int64_t qidx = top - lane;
        uint64_t sv = qidx >= 0 ? ld_relaxed_u64(part_status + qidx) : kInc;
        uint32_t flag = (uint32_t)(sv >> 62);
        unsigned inc_mask = __ballot_sync(0xffffffffu, flag == 2u);
        unsigned inv_mask = __ballot_sync(0xffffffffu, flag == 0u);
        int first_inc = inc_mask ? __ffs(inc_mask) - 1 : 32;
        unsigned upto = first_inc >= 31 ? 0xffffffffu : ((2u << first_inc) - 1u);
        if ((inv_mask & upto) && !timed_out) {
          if (globaltimer_ns() - t0 > kWaitLimitNs) {
            timed_out = true;
            if (lane == 0) set_status(status, AGS_ERR_TIMEOUT, kStageEmit);
          }
          continue;
        }
        uint64_t v = (lane <= first_inc) ? (sv & kValMask) : 0ull;
        excl += warp_sum(v);
        if (first_inc < 32 || timed_out) break;
        top -= 32;
      }
      if (lane == 0) st_relaxed_u64(part_status + part, kInc | ((excl + agg) & kValMask));
    }
    if (lane == 0) s_prefix = excl;
  }
  // local exclusive offsets
  uint32_t run = texcl;
#pragma unroll
  for (int k = 0; k < kEmitItems; k++) {
    s_off[tid * kEmitItems + k] = run;
    run += cnt[k];
  }
  if (tid == kEmitThreads - 1) s_off[kEmitPart] = run;
  __syncthreads();
  const uint64_t prefix = s_prefix;

  // 4. load-balanced emission: warps take chunks of 256 consecutive pairs; each
  //    lane generates 8 consecutive pairs (one binary search, then walking the
  //    rectangle row by row) into a warp-private staging row, and the warp
  //    writes the chunk out with coalesced stores.
  __shared__ K s_key[kEmitThreads / 32][32 * kEmitStride];
  __shared__ uint32_t s_val[kEmitThreads / 32][32 * kEmitStride];
  for (uint32_t w0 = (uint32_t)warp * kEmitChunk; w0 < agg; w0 += (kEmitThreads / 32) * kEmitChunk) {
    const uint32_t j0 = w0 + (uint32_t)lane * kEmitRun;
    if (j0 < agg) {
      int lo = 0, hi = kEmitPart;   // invariant: s_off[lo] <= j0 < s_off[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] <= j0) lo = mid; else hi = mid;
      }
      uint32_t r = j0 - s_off[lo];
      uint32_t w = s_w[lo];
      uint32_t ry = r / w, rx = r - ry * w;
#pragma unroll
      for (int k = 0; k < kEmitRun; k++) {
        const uint32_t j = j0 + k;
        if (j >= agg) break;
        while (j >= s_off[lo + 1]) {          // next Gaussian with pairs
          lo++;
          w = s_w[lo];
          rx = 0;
          ry = 0;
        }
        const uint32_t tile = s_base[lo] + ry * gx + rx;
        make_key(tile, sizeof(K) == 8 ? s_dbits[lo] : 0u, s_key[warp][lane * kEmitStride + k]);
        s_val[warp][lane * kEmitStride + k] = s_idx[lo];
        if (++rx == w) { rx = 0; ry++; }
      }
    }
    __syncwarp();
    const uint32_t nval = min((uint32_t)kEmitChunk, agg - w0);
    for (uint32_t m = lane; m < nval; m += 32) {
      const uint64_t pos = prefix + w0 + m;
      const uint32_t si = (m / kEmitRun) * kEmitStride + (m % kEmitRun);
      if (pos < (uint64_t)capacity) {
        keys[pos] = s_key[warp][si];
        vals[pos] = s_val[warp][si];
      }
    }
    __syncwarp();
  }
  if (part == num_parts - 1 && tid == 0) {
    int64_t tot = (int64_t)(prefix + agg);
    *d_num_pairs = tot;
    if (tot > capacity) set_status(status, AGS_ERR_CAPACITY, tot);
  }
}

static size_t emit_parts(int64_t total) { return (size_t)((total + kEmitPart - 1) / kEmitPart); }

}  // namespace ags

extern "C" size_t ags_emit_workspace_bytes(int64_t n, int32_t views) {
  if (n < 0 || views < 1) return 0;
  return 256 + 8 * ags::emit_parts(n * (int64_t)views);
}

extern "C" ags_status ags_emit_pairs(const ags_projected* proj, int64_t n, int32_t views, const ags_camera* cams,
                                     const uint32_t* order, uint64_t* keys, uint32_t* vals, int64_t capacity,
                                     int64_t* d_num_pairs, int64_t* d_status, void* ws, size_t ws_bytes,
                                     void* stream) {
  using namespace ags;
  if (!proj || !d_num_pairs || !d_status || n < 0 || capacity < 0 || capacity > AGS_MAX_PAIRS)
    return AGS_ERR_INVALID_ARG;
  CamBatch cb;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  const int64_t total = n * (int64_t)views;
  if (total >= ((int64_t)1 << 32)) return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (total == 0) return launch_status(cudaMemsetAsync(d_num_pairs, 0, sizeof(int64_t), st));
  if (!proj->rect || !proj->depth || (capacity > 0 && (!keys || !vals))) return AGS_ERR_INVALID_ARG;
  if (!ws || ws_bytes < ags_emit_workspace_bytes(n, views) || ((uintptr_t)ws & 7u)) return AGS_ERR_INVALID_ARG;
  const size_t parts = emit_parts(total);
  uint32_t tiles_per_view = (uint32_t)cb.c[0].gx * (uint32_t)cb.c[0].gy;
  if ((uint64_t)tiles_per_view * (uint64_t)views >= (1ull << 32)) return AGS_ERR_INVALID_ARG;
  cudaError_t e = cudaMemsetAsync(ws, 0, 256 + 8 * parts, st);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws);
  uint64_t* part_status = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ws) + 256);
  emit_kernel<uint64_t><<<(unsigned)parts, kEmitThreads, 0, st>>>(
      reinterpret_cast<const uint2*>(proj->rect), proj->depth, order, total, (uint32_t)n, tiles_per_view,
      (uint32_t)cb.c[0].gx, keys, vals, capacity, d_num_pairs, d_status, part_status, counter, (uint32_t)parts);
  return launch_status(cudaGetLastError());
}

extern "C" ags_status ags_emit_tile_pairs(const ags_projected* proj, int64_t n, int32_t views,
                                          const ags_camera* cams, const uint32_t* order, uint32_t* keys,
                                          uint32_t* vals, int64_t capacity, int64_t* d_num_pairs, int64_t* d_status,
                                          void* ws, size_t ws_bytes, void* stream) {
  using namespace ags;
  if (!proj || !d_num_pairs || !d_status || n < 0 || capacity < 0 || capacity > AGS_MAX_PAIRS)
    return AGS_ERR_INVALID_ARG;
  CamBatch cb;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  const int64_t total = n * (int64_t)views;
  if (total >= ((int64_t)1 << 32)) return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (total == 0) return launch_status(cudaMemsetAsync(d_num_pairs, 0, sizeof(int64_t), st));
  if (!proj->rect || (capacity > 0 && (!keys || !vals))) return AGS_ERR_INVALID_ARG;
  if (!ws || ws_bytes < ags_emit_workspace_bytes(n, views) || ((uintptr_t)ws & 7u)) return AGS_ERR_INVALID_ARG;
  const size_t parts = emit_parts(total);
  uint32_t tiles_per_view = (uint32_t)cb.c[0].gx * (uint32_t)cb.c[0].gy;
  if ((uint64_t)tiles_per_view * (uint64_t)views >= (1ull << 32)) return AGS_ERR_INVALID_ARG;
  cudaError_t e = cudaMemsetAsync(ws, 0, 256 + 8 * parts, st);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws);
  uint64_t* part_status = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ws) + 256);
  emit_kernel<uint32_t><<<(unsigned)parts, kEmitThreads, 0, st>>>(
      reinterpret_cast<const uint2*>(proj->rect), proj->depth, order, total, (uint32_t)n, tiles_per_view,
      (uint32_t)cb.c[0].gx, keys, vals, capacity, d_num_pairs, d_status, part_status, counter, (uint32_t)parts);
  return launch_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Allocation-free variant of ags_emit_pairs (see include/ags.h).
//
// The look-back state lives in a library-owned device array instead of a
// caller workspace.  In host code `g_emit_scratch` names a host-side stand-in,
// not a device address, so the device address is looked up with
// cudaGetSymbolAddress once per device (with that device current) and cached.
// ---------------------------------------------------------------------------
namespace ags {

constexpr int64_t kNoAllocMaxGaussianViews = (int64_t)1 << 24;     // views * n limit
constexpr size_t kNoAllocScratchBytes = 256 + 8 * (size_t)(kNoAllocMaxGaussianViews / kEmitPart);   // 128.25 KiB

static __device__ __align__(256) unsigned char g_emit_scratch[kNoAllocScratchBytes];

static std::mutex g_scratch_mutex;
static void* g_scratch_ptr[256];          // device address per CUDA device ordinal (nullptr: not set up)

static ags_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return AGS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_emit_scratch) != cudaSuccess || !p) return AGS_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return AGS_OK;
}

}  // namespace ags

extern "C" int64_t ags_emit_pairs_noalloc_max_gaussians(void) { return ags::kNoAllocMaxGaussianViews; }

extern "C" ags_status ags_emit_pairs_noalloc(const ags_projected* proj, int64_t n, int32_t views,
                                             const ags_camera* cams, const uint32_t* order, uint64_t* keys,
                                             uint32_t* vals, int64_t capacity, int64_t* d_num_pairs,
                                             int64_t* d_status, void* stream) {
  using namespace ags;
  if (!proj || !d_num_pairs || !d_status || n < 0 || capacity < 0 || capacity > AGS_MAX_PAIRS)
    return AGS_ERR_INVALID_ARG;
  CamBatch cb;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  const int64_t total = n * (int64_t)views;
  if (total > kNoAllocMaxGaussianViews) return AGS_ERR_INVALID_ARG;   // beyond the static scratch
  cudaStream_t st = (cudaStream_t)stream;
  void* ws = nullptr;
  s = scratch_address(&ws);
  if (s != AGS_OK) return s;
  if (total == 0) return launch_status(cudaMemsetAsync(d_num_pairs, 0, sizeof(int64_t), st));
  if (!proj->rect || !proj->depth || (capacity > 0 && (!keys || !vals))) return AGS_ERR_INVALID_ARG;
  const size_t parts = emit_parts(total);
  const uint32_t tiles_per_view = (uint32_t)cb.c[0].gx * (uint32_t)cb.c[0].gy;
  if ((uint64_t)tiles_per_view * (uint64_t)views >= (1ull << 32)) return AGS_ERR_INVALID_ARG;
  // the array keeps the previous call's contents: clear the counter and look-back flags
  cudaError_t e = cudaMemsetAsync(ws, 0, 256 + 8 * parts, st);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws);
  uint64_t* part_status = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ws) + 256);
  emit_kernel<uint64_t><<<(unsigned)parts, kEmitThreads, 0, st>>>(
      reinterpret_cast<const uint2*>(proj->rect), proj->depth, order, total, (uint32_t)n, tiles_per_view,
      (uint32_t)cb.c[0].gx, keys, vals, capacity, d_num_pairs, d_status, part_status, counter, (uint32_t)parts);
  return launch_status(cudaGetLastError());
}
