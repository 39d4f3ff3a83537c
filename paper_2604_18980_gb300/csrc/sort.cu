// sort.cu -- stable LSD radix sort of the Gaussian-tile pairs (Sec. 2.1 sorting
// stage) and the per-tile ranges.
//
// "Onesweep" organisation: one pass over the keys builds the histograms of
// every digit at once; then each digit pass is a single kernel in which each
// block (256 threads x 8 keys) ranks its keys with warp-level match/ballot
// (per-warp digit counters in shared memory), publishes its digit counts,
// obtains each digit's global offset by a decoupled look-back over the
// preceding blocks (bounded spin, partition ids from an atomic counter), and
// scatters through shared memory so that global stores are contiguous runs.
// Ranking visits keys in index order (warp-major, then item, then lane), so
// every pass is stable and equal keys keep their emission (Gaussian) order.
#include <algorithm>
#include <utility>

#include "ags_internal.cuh"

namespace ags {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortPart = kSortThreads * kSortItems;     // 2048 keys per block
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadix = 256;
constexpr int kMaxPasses = 16;
constexpr uint32_t kLbAgg = 1u << 30;
constexpr uint32_t kLbInc = 2u << 30;
constexpr uint32_t kLbMask = (1u << 30) - 1u;
constexpr int kLookWindow = 8;                              // predecessors polled per round trip
constexpr size_t kSortHdr = 256;                           // pass counters
constexpr size_t kSortHistBytes = (size_t)kMaxPasses * kRadix * 4;

struct SortSmem {
  union {
    uint32_t warp_hist[kSortWarps][kRadix];                // ranking phase
    struct {
      uint64_t keys[kSortPart];
      uint32_t vals[kSortPart];
    } stage;                                               // scatter phase
  } u;
  uint32_t digit_off[kRadix];   // block-local exclusive start of each digit
  uint32_t gbase[kRadix];       // global index of block-local position 0, per digit (mod 2^32)
  uint32_t warp_tot[kSortWarps];
  uint32_t part;
};

__device__ __forceinline__ uint32_t digit_mask(int shift, int end_bit, int digit_bits) {
  int b = min(digit_bits, end_bit - shift);
  return (1u << b) - 1u;
}

// The pair count is read on the device and clamped to the buffer capacity (after
// an emission overflow it exceeds it; the status block already records that).
__device__ __forceinline__ int64_t clamped_count(const int64_t* count_ptr, int64_t capacity) {
  int64_t c = *count_ptr;
  return c < 0 ? 0 : (c > capacity ? capacity : c);
}

__global__ void __launch_bounds__(256) hist_kernel(const uint64_t* __restrict__ keys, const int64_t* count_ptr,
                                                   int64_t capacity, int begin_bit, int end_bit, int digit_bits,
                                                   int passes, uint32_t* ghist) {
  __shared__ uint32_t h[kMaxPasses][kRadix];
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) (&h[0][0])[i] = 0u;
  __syncthreads();
  const int64_t count = clamped_count(count_ptr, capacity);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = __ldg(keys + i);
    for (int p = 0; p < passes; p++) {
      int sh = begin_bit + p * digit_bits;
      atomicAdd(&h[p][(uint32_t)(k >> sh) & digit_mask(sh, end_bit, digit_bits)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    uint32_t v = (&h[0][0])[i];
    if (v) atomicAdd(ghist + i, v);
  }
}

// Exclusive scan of each pass's 256-bin histogram, in place (one block per pass).
__global__ void __launch_bounds__(kRadix) hist_scan_kernel(uint32_t* ghist) {
  __shared__ uint32_t wt[kRadix / 32];
  uint32_t* h = ghist + blockIdx.x * kRadix;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t v = h[t], incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wt[w] = incl;
  __syncthreads();
  uint32_t pre = 0;
  for (int i = 0; i < w; i++) pre += wt[i];
  h[t] = pre + incl - v;
}

__global__ void __launch_bounds__(kSortThreads, 4)
onesweep_kernel(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
                uint32_t* __restrict__ vout, const int64_t* count_ptr, int64_t capacity, int identity, int shift,
                uint32_t mask,
                const uint32_t* __restrict__ gprefix, uint32_t* lookback, uint32_t* counter, int64_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem& S = *reinterpret_cast<SortSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) S.part = atomicAdd(counter, 1u);
  for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&S.u.warp_hist[0][0])[i] = 0u;
  __syncthreads();
  const uint32_t part = S.part;
  const uint32_t count = (uint32_t)clamped_count(count_ptr, capacity);
  const uint32_t nparts = (count + kSortPart - 1) / kSortPart;
  if (part >= nparts) return;   // no block waits on a higher partition
  const uint32_t base = part * kSortPart;

  // load (warp-striped, coalesced) and rank within the warp
  uint64_t key[kSortItems];
  uint32_t val[kSortItems];
  uint32_t rank[kSortItems];
  const unsigned lt_mask = lanemask_lt();
  // all loads first (memory-level parallelism), then the ranking
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    uint32_t idx = base + warp * (32 * kSortItems) + i * 32 + lane;
    bool valid = idx < count;
    key[i] = valid ? __ldcs(kin + idx) : 0ull;
    val[i] = valid ? (identity ? idx : __ldcs(vin + idx)) : 0u;
  }
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    uint32_t idx = base + warp * (32 * kSortItems) + i * 32 + lane;
    bool valid = idx < count;
    uint32_t d = valid ? ((uint32_t)(key[i] >> shift) & mask) : (uint32_t)kRadix;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = valid ? S.u.warp_hist[warp][d] : 0u;
    __syncwarp();
    if (valid && (peers & lt_mask) == 0u) S.u.warp_hist[warp][d] = before + (uint32_t)__popc(peers);
    __syncwarp();
    rank[i] = before + (uint32_t)__popc(peers & lt_mask);
  }
  __syncthreads();

  // per digit (thread = digit): block total and per-warp exclusive prefixes
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; w++) {
    uint32_t v = S.u.warp_hist[w][tid];
    S.u.warp_hist[w][tid] = tot;
    tot += v;
  }
  uint32_t* lb = lookback + (size_t)part * kRadix;
  st_relaxed_u32(lb + tid, (part == 0 ? kLbInc : kLbAgg) | tot);
  // block-exclusive scan of the digit totals
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) S.warp_tot[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < warp; w++) wpre += S.warp_tot[w];
  S.digit_off[tid] = wpre + incl - tot;

  // decoupled look-back for this digit, kLookWindow predecessors per round trip:
  // add the aggregates back to the nearest inclusive prefix; re-poll from the
  // first predecessor that has not published yet.
  uint32_t excl = 0;
  if (part > 0) {
    int64_t p = (int64_t)part - 1;
    const uint64_t t0 = globaltimer_ns();
    bool found = false;
    while (!found) {
      uint32_t sv[kLookWindow];
#pragma unroll
      for (int k = 0; k < kLookWindow; k++)
        sv[k] = (p - k >= 0) ? ld_relaxed_u32(lookback + (size_t)(p - k) * kRadix + tid) : kLbInc;
      int used = 0;
#pragma unroll
      for (int k = 0; k < kLookWindow; k++) {
        if (found || used < k) continue;           // stop at the first unpublished entry
        const uint32_t flag = sv[k] >> 30;
        if (flag == 0u) continue;
        excl += sv[k] & kLbMask;
        used = k + 1;
        if (flag == 2u) found = true;
      }
      p -= used;
      if (!found && used < kLookWindow && globaltimer_ns() - t0 > kWaitLimitNs) {
        set_status(status, AGS_ERR_TIMEOUT, kStageSort);
        break;
      }
    }
    st_relaxed_u32(lb + tid, kLbInc | ((excl + tot) & kLbMask));
  }
  S.gbase[tid] = gprefix[tid] + excl - S.digit_off[tid];
  __syncthreads();

  // block-local sorted positions
  uint32_t pos[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    uint32_t idx = base + warp * (32 * kSortItems) + i * 32 + lane;
    uint32_t d = (uint32_t)(key[i] >> shift) & mask;
    pos[i] = idx < count ? S.digit_off[d] + S.u.warp_hist[warp][d] + rank[i] : 0xffffffffu;
  }
  __syncthreads();   // the staging area aliases the warp counters
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    if (pos[i] < (uint32_t)kSortPart) {
      S.u.stage.keys[pos[i]] = key[i];
      S.u.stage.vals[pos[i]] = val[i];
    }
  }
  __syncthreads();
  const uint32_t nvalid = min((uint32_t)kSortPart, count - base);
  for (uint32_t j = tid; j < nvalid; j += kSortThreads) {
    uint64_t k = S.u.stage.keys[j];
    uint32_t d = (uint32_t)(k >> shift) & mask;
    uint32_t dst = S.gbase[d] + j;
    if (dst < count) {
      kout[dst] = k;
      vout[dst] = S.u.stage.vals[j];
    }
  }
}

__global__ void ranges_kernel(const uint64_t* __restrict__ keys, const int64_t* count_ptr, int64_t capacity,
                              uint32_t* ranges, int64_t num_ranges) {
  const int64_t count = clamped_count(count_ptr, capacity);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t tile = keys[i] >> 32;
    if (tile >= (uint64_t)num_ranges) continue;
    if (i == 0 || (keys[i - 1] >> 32) != tile) ranges[2 * tile] = (uint32_t)i;
    if (i == count - 1 || (keys[i + 1] >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(i + 1);
  }
}

static size_t sort_parts(int64_t capacity) { return (size_t)((capacity + kSortPart - 1) / kSortPart); }

}  // namespace ags

extern "C" size_t ags_sort_workspace_bytes(int64_t capacity) {
  if (capacity < 0) return 0;
  return ags::kSortHdr + ags::kSortHistBytes + ags::sort_parts(capacity) * ags::kRadix * 4;
}

extern "C" ags_status ags_sort(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                               const int64_t* d_num_pairs, int64_t capacity, int32_t begin_bit, int32_t end_bit,
                               int32_t digit_bits, int32_t flags, uint32_t* ranges, int64_t num_ranges,
                               int32_t* result_in_alt, int64_t* d_status, void* ws, size_t ws_bytes,
                               void* stream) {
  using namespace ags;
  if (!d_num_pairs || !d_status || capacity < 0 || capacity >= AGS_MAX_PAIRS) return AGS_ERR_INVALID_ARG;
  if (begin_bit < 0 || end_bit > 64 || begin_bit > end_bit || digit_bits < 4 || digit_bits > 8)
    return AGS_ERR_INVALID_ARG;
  if (flags & ~AGS_SORT_IDENTITY_VALUES) return AGS_ERR_INVALID_ARG;
  const int passes = (end_bit - begin_bit + digit_bits - 1) / digit_bits;
  if (passes > kMaxPasses) return AGS_ERR_INVALID_ARG;
  if (ranges && num_ranges <= 0) return AGS_ERR_INVALID_ARG;
  if (capacity > 0 && (!keys || !vals || (passes > 0 && (!keys_alt || !vals_alt)))) return AGS_ERR_INVALID_ARG;
  if (!ws || ws_bytes < ags_sort_workspace_bytes(capacity) || ((uintptr_t)ws & 15u)) return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (result_in_alt) *result_in_alt = passes & 1;
  char* w = reinterpret_cast<char*>(ws);
  uint32_t* counters = reinterpret_cast<uint32_t*>(w);
  uint32_t* ghist = reinterpret_cast<uint32_t*>(w + kSortHdr);
  uint32_t* lookback = reinterpret_cast<uint32_t*>(w + kSortHdr + kSortHistBytes);
  const size_t parts = sort_parts(capacity);
  cudaError_t e = cudaSuccess;
  uint64_t* kin = keys;
  uint32_t* vin = vals;
  if (capacity > 0 && passes > 0) {
    e = cudaMemsetAsync(w, 0, kSortHdr + kSortHistBytes, st);
    if (e != cudaSuccess) return AGS_ERR_CUDA;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned hb = (unsigned)std::min<int64_t>((capacity + 255) / 256, (int64_t)sms * 4);
    hist_kernel<<<hb, 256, 0, st>>>(keys, d_num_pairs, capacity, begin_bit, end_bit, digit_bits, passes, ghist);
    hist_scan_kernel<<<passes, kRadix, 0, st>>>(ghist);
    const int smem = (int)sizeof(SortSmem);
    e = cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return AGS_ERR_CUDA;
    uint64_t* kout = keys_alt;
    uint32_t* vout = vals_alt;
    for (int p = 0; p < passes; p++) {
      e = cudaMemsetAsync(lookback, 0, parts * kRadix * 4, st);
      if (e != cudaSuccess) return AGS_ERR_CUDA;
      int sh = begin_bit + p * digit_bits;
      uint32_t mask = (1u << std::min(digit_bits, end_bit - sh)) - 1u;
      const int identity = (p == 0 && (flags & AGS_SORT_IDENTITY_VALUES)) ? 1 : 0;
      onesweep_kernel<<<(unsigned)parts, kSortThreads, smem, st>>>(kin, vin, kout, vout, d_num_pairs, capacity,
                                                                  identity, sh, mask,
                                                                  ghist + p * kRadix, lookback, counters + p,
                                                                  d_status);
      e = cudaGetLastError();
      if (e != cudaSuccess) return AGS_ERR_CUDA;
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
  }
  if (ranges) {
    e = cudaMemsetAsync(ranges, 0, (size_t)num_ranges * 2 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return AGS_ERR_CUDA;
    if (capacity > 0) {
      int blocks = (int)std::min<int64_t>((capacity + 255) / 256, 65535 * 4);
      ranges_kernel<<<blocks, 256, 0, st>>>(kin, d_num_pairs, capacity, ranges, num_ranges);
    }
  }
  return launch_status(cudaGetLastError());
}
