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

constexpr int kSortItems = 8;                             // keys per thread
constexpr int kMinPart = 256 * kSortItems;                // smallest partition (workspace sizing)
constexpr int kMaxRadix = 512;                            // digits of up to 9 bits
constexpr int kMaxPasses = 16;
constexpr uint32_t kLbAgg = 1u << 30;
constexpr uint32_t kLbInc = 2u << 30;
constexpr uint32_t kLbMask = (1u << 30) - 1u;
constexpr int kLookWindow = 32;                             // predecessors polled per round trip
constexpr size_t kSortHdr = 256;                           // pass counters
constexpr size_t kSortHistBytes = (size_t)kMaxPasses * kMaxRadix * 4;

template <int THREADS, int RADIX>
struct SortSmem {
  static constexpr int kWarps = THREADS / 32;
  static constexpr int kPart = THREADS * kSortItems;
  union {
    uint16_t warp_hist[kWarps][RADIX];                     // ranking phase (<= 256 per warp)
    struct {
      uint64_t keys[kPart];
      uint32_t vals[kPart];
    } stage;                                               // block-sorted keys, before the look-back
  } u;
  uint32_t bhist[RADIX];        // block digit counts, then the block-local exclusive digit starts
  uint32_t gbase[RADIX];        // global index of block-local position 0, per digit (mod 2^32)
  uint32_t scan_tot[kWarps];
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

// Global digit histograms of every pass in one read.  Each thread takes 16
// consecutive keys and counts runs of equal digits before adding them: the
// keys are highly clustered (pairs of one Gaussian are consecutive, the depth
// exponent byte is nearly constant), so a run costs one shared atomic instead
// of one per key, and unclustered digits do not contend anyway.
__global__ void __launch_bounds__(256) hist_kernel(const uint64_t* __restrict__ keys, const int64_t* count_ptr,
                                                   int64_t capacity, int begin_bit, int end_bit, int digit_bits,
                                                   int passes, int radix, uint32_t* ghist) {
  __shared__ uint32_t h[kMaxPasses * kMaxRadix];
  for (int i = threadIdx.x; i < passes * radix; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const int64_t count = clamped_count(count_ptr, capacity);
  constexpr int R = 16;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * R;
  for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * R; i0 < count; i0 += stride) {
    uint64_t k[R];
    if (i0 + R <= count) {
      const ulonglong2* p = reinterpret_cast<const ulonglong2*>(keys + i0);
#pragma unroll
      for (int q = 0; q < R / 2; q++) { ulonglong2 t = __ldcs(p + q); k[2 * q] = t.x; k[2 * q + 1] = t.y; }
    } else {
#pragma unroll
      for (int q = 0; q < R; q++) k[q] = (i0 + q < count) ? keys[i0 + q] : ~0ull;
    }
    const int nv = (int)min((int64_t)R, count - i0);
    for (int p = 0; p < passes; p++) {
      const int sh = begin_bit + p * digit_bits;
      const uint32_t m = digit_mask(sh, end_bit, digit_bits);
      uint32_t cur = (uint32_t)(k[0] >> sh) & m, run = 1;
#pragma unroll
      for (int q = 1; q < R; q++) {
        if (q >= nv) break;
        const uint32_t d = (uint32_t)(k[q] >> sh) & m;
        if (d == cur) { run++; } else { atomicAdd(&h[p * radix + cur], run); cur = d; run = 1; }
      }
      atomicAdd(&h[p * radix + cur], run);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * radix; i += blockDim.x) {
    uint32_t v = h[i];
    if (v) atomicAdd(ghist + i, v);
  }
}

// Exclusive scan of each pass's histogram, in place (one block per pass).
template <int RADIX>
__global__ void __launch_bounds__(RADIX) hist_scan_kernel(uint32_t* ghist) {
  __shared__ uint32_t wt[RADIX / 32];
  uint32_t* h = ghist + blockIdx.x * RADIX;
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

// One digit pass over a partition of THREADS x 8 keys.  The keys are ranked
// within each warp (match.any, index order, so the pass is stable); the
// per-warp counts give the block's digit totals, which are published to the
// look-back at once; the keys are placed in shared memory in block-sorted
// order, and only then does the block look back for each digit's global
// offset (a window of 32 predecessors per round trip), with its registers
// free.  Large partitions keep the number of look-back steps small.
template <int THREADS, int RADIX>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
onesweep_kernel(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
                uint32_t* __restrict__ vout, const int64_t* count_ptr, int64_t capacity, int identity, int shift,
                uint32_t mask, const uint32_t* __restrict__ gprefix, uint32_t* lookback, uint32_t* counter,
                int64_t* status, uint32_t* ranges, int64_t num_ranges) {
  using Sm = SortSmem<THREADS, RADIX>;
  constexpr int kWarps = Sm::kWarps;
  constexpr int kPart = Sm::kPart;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Sm& S = *reinterpret_cast<Sm*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool digit_thread = tid < RADIX;                   // threads owning one digit each
  if (tid == 0) S.part = atomicAdd(counter, 1u);
  {
    uint32_t* wh = reinterpret_cast<uint32_t*>(&S.u.warp_hist[0][0]);
    for (int i = tid; i < kWarps * RADIX / 2; i += THREADS) wh[i] = 0u;
    for (int i = tid; i < RADIX; i += THREADS) S.bhist[i] = 0u;
  }
  const uint32_t gp = digit_thread ? __ldg(gprefix + tid) : 0u;   // prefetched, used at the end
  __syncthreads();
  const uint32_t part = S.part;
  const uint32_t count = (uint32_t)clamped_count(count_ptr, capacity);
  const uint32_t nparts = (count + kPart - 1) / kPart;
  if (part >= nparts) return;   // no block waits on a higher partition
  const uint32_t base = part * kPart;

  // load (warp-striped, coalesced), all loads first
  uint64_t key[kSortItems];
  uint32_t val[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const uint32_t idx = base + warp * (32 * kSortItems) + i * 32 + lane;
    const bool valid = idx < count;
    key[i] = valid ? __ldcs(kin + idx) : 0ull;
    val[i] = valid ? (identity ? idx : __ldcs(vin + idx)) : 0u;
  }
  uint32_t* lb = lookback + (size_t)part * RADIX;
  uint32_t tot = 0;

  // rank within the warp (match.any), in index order
  uint32_t rank[kSortItems];
  const unsigned lt_mask = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const uint32_t idx = base + warp * (32 * kSortItems) + i * 32 + lane;
    const bool valid = idx < count;
    const uint32_t d = valid ? ((uint32_t)(key[i] >> shift) & mask) : (uint32_t)RADIX;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? S.u.warp_hist[warp][d] : 0u;
    __syncwarp();
    if (valid && (peers & lt_mask) == 0u) S.u.warp_hist[warp][d] = (uint16_t)(before + __popc(peers));
    __syncwarp();
    rank[i] = before + (uint32_t)__popc(peers & lt_mask);
  }
  __syncthreads();

  // per digit: per-warp exclusive prefixes and the block-exclusive digit start
  if (digit_thread) {
    uint32_t run = 0;
#pragma unroll 4
    for (int w = 0; w < kWarps; w++) {
      const uint32_t v = S.u.warp_hist[w][tid];
      S.u.warp_hist[w][tid] = (uint16_t)run;
      run += v;
    }
    tot = run;
    st_relaxed_u32(lb + tid, (part == 0 ? kLbInc : kLbAgg) | tot);
  }
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) S.scan_tot[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < warp; w++) wpre += S.scan_tot[w];
  const uint32_t doff = wpre + incl - tot;
  if (digit_thread) S.bhist[tid] = doff;                  // block-local exclusive start of digit tid
  __syncthreads();

  // block-sorted positions, then the keys go to shared memory
  uint32_t pos[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const uint32_t idx = base + warp * (32 * kSortItems) + i * 32 + lane;
    const uint32_t d = (uint32_t)(key[i] >> shift) & mask;
    pos[i] = idx < count ? S.bhist[d] + S.u.warp_hist[warp][d] + rank[i] : 0xffffffffu;
  }
  __syncthreads();   // the staging area aliases the warp counters
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    if (pos[i] < (uint32_t)kPart) {
      S.u.stage.keys[pos[i]] = key[i];
      S.u.stage.vals[pos[i]] = val[i];
    }
  }

  // decoupled look-back per digit, kLookWindow predecessors per round trip:
  // add the aggregates back to the nearest inclusive prefix; re-poll from the
  // first predecessor that has not published yet.
  if (digit_thread) {
    uint32_t excl = 0;
    if (part > 0) {
      const uint64_t t0 = globaltimer_ns();
      int64_t p = (int64_t)part - 1;
      bool found = false;
      while (!found) {
        uint32_t sv[kLookWindow];
#pragma unroll
        for (int q = 0; q < kLookWindow; q++)
          sv[q] = (p - q >= 0) ? ld_relaxed_u32(lookback + (size_t)(p - q) * RADIX + tid) : kLbInc;
        int used = 0;
#pragma unroll
        for (int q = 0; q < kLookWindow; q++) {
          if (found || used < q) continue;           // stop at the first unpublished entry
          const uint32_t flag = sv[q] >> 30;
          if (flag == 0u) continue;
          excl += sv[q] & kLbMask;
          used = q + 1;
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
    S.gbase[tid] = gp + excl - doff;
  }
  __syncthreads();
  const uint32_t nvalid = min((uint32_t)kPart, count - base);
  for (uint32_t j = tid; j < nvalid; j += THREADS) {
    const uint64_t k = S.u.stage.keys[j];
    const uint32_t d = (uint32_t)(k >> shift) & mask;
    const uint32_t dst = S.gbase[d] + j;
    if (dst < count) {
      kout[dst] = k;
      vout[dst] = S.u.stage.vals[j];
      if (ranges) {
        // last pass: the output is fully sorted and one tile's keys are consecutive
        // (equal tiles share the digit), so a tile's first and last keys in this
        // block bound its range; other blocks holding the same tile do the same.
        const uint64_t tile = k >> 32;
        if (tile < (uint64_t)num_ranges) {
          if (j == 0 || (S.u.stage.keys[j - 1] >> 32) != tile) atomicMin(ranges + 2 * tile, dst);
          if (j + 1 == nvalid || (S.u.stage.keys[j + 1] >> 32) != tile) atomicMax(ranges + 2 * tile + 1, dst + 1);
        }
      }
    }
  }
}

// Tiles no pair reached still hold the (0xffffffff, 0) of the initialisation.
__global__ void ranges_fixup_kernel(uint2* ranges, int64_t num_ranges) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < num_ranges; t += (int64_t)gridDim.x * blockDim.x) {
    const uint2 r = ranges[t];
    if (r.x > r.y) ranges[t] = make_uint2(0u, 0u);
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

static size_t sort_parts(int64_t capacity) { return (size_t)((capacity + kMinPart - 1) / kMinPart); }

template <int THREADS, int RADIX>
static cudaError_t launch_passes(uint64_t*& kin, uint32_t*& vin, uint64_t* kout, uint32_t* vout,
                                 const int64_t* d_num_pairs, int64_t capacity, int begin_bit, int end_bit,
                                 int digit_bits, int passes, int flags, uint32_t* ghist, uint32_t* lookback,
                                 uint32_t* counters, int64_t* d_status, uint32_t* ranges, int64_t num_ranges,
                                 cudaStream_t st) {
  hist_scan_kernel<RADIX><<<passes, RADIX, 0, st>>>(ghist);
  const int smem = (int)sizeof(SortSmem<THREADS, RADIX>);
  cudaError_t e = cudaFuncSetAttribute(onesweep_kernel<THREADS, RADIX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const size_t parts = (size_t)((capacity + SortSmem<THREADS, RADIX>::kPart - 1) / SortSmem<THREADS, RADIX>::kPart);
  for (int p = 0; p < passes; p++) {
    e = cudaMemsetAsync(lookback, 0, parts * RADIX * 4, st);
    if (e != cudaSuccess) return e;
    const int sh = begin_bit + p * digit_bits;
    const uint32_t mask = (1u << std::min(digit_bits, end_bit - sh)) - 1u;
    const int identity = (p == 0 && (flags & AGS_SORT_IDENTITY_VALUES)) ? 1 : 0;
    const bool last = p == passes - 1;
    onesweep_kernel<THREADS, RADIX><<<(unsigned)parts, THREADS, smem, st>>>(
        kin, vin, kout, vout, d_num_pairs, capacity, identity, sh, mask, ghist + p * RADIX, lookback, counters + p,
        d_status, last ? ranges : nullptr, num_ranges);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  return cudaSuccess;
}

}  // namespace ags

extern "C" size_t ags_sort_workspace_bytes(int64_t capacity) {
  if (capacity < 0) return 0;
  return ags::kSortHdr + ags::kSortHistBytes + ags::sort_parts(capacity) * ags::kMaxRadix * 4;
}

extern "C" ags_status ags_sort(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                               const int64_t* d_num_pairs, int64_t capacity, int32_t begin_bit, int32_t end_bit,
                               int32_t digit_bits, int32_t flags, uint32_t* ranges, int64_t num_ranges,
                               int32_t* result_in_alt, int64_t* d_status, void* ws, size_t ws_bytes,
                               void* stream) {
  using namespace ags;
  if (!d_num_pairs || !d_status || capacity < 0 || capacity >= AGS_MAX_PAIRS) return AGS_ERR_INVALID_ARG;
  if (begin_bit < 0 || end_bit > 64 || begin_bit > end_bit || digit_bits < 4 || digit_bits > 9)
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
  const int radix = digit_bits > 8 ? 512 : 256;
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
    hist_kernel<<<hb, 256, 0, st>>>(keys, d_num_pairs, capacity, begin_bit, end_bit, digit_bits, passes, radix, ghist);
    // partitions of 512 threads x 8 keys, two blocks per SM
    if (ranges) {   // start = 0xffffffff, end = 0: the last pass narrows them with atomics
      e = cudaMemset2DAsync(ranges, 8, 0xff, 4, (size_t)num_ranges, st);
      if (e == cudaSuccess) e = cudaMemset2DAsync(ranges + 1, 8, 0, 4, (size_t)num_ranges, st);
      if (e != cudaSuccess) return AGS_ERR_CUDA;
    }
    e = radix == 512 ? launch_passes<512, 512>(kin, vin, keys_alt, vals_alt, d_num_pairs, capacity, begin_bit,
                                               end_bit, digit_bits, passes, flags, ghist, lookback, counters,
                                               d_status, ranges, num_ranges, st)
                     : launch_passes<512, 256>(kin, vin, keys_alt, vals_alt, d_num_pairs, capacity, begin_bit,
                                               end_bit, digit_bits, passes, flags, ghist, lookback, counters,
                                               d_status, ranges, num_ranges, st);
    if (e != cudaSuccess) return AGS_ERR_CUDA;
  }
  if (ranges) {
    if (capacity > 0 && passes > 0) {
      const int blocks = (int)std::min<int64_t>((num_ranges + 255) / 256, 4096);
      ranges_fixup_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<uint2*>(ranges), num_ranges);
    } else {
      e = cudaMemsetAsync(ranges, 0, (size_t)num_ranges * 2 * sizeof(uint32_t), st);
      if (e != cudaSuccess) return AGS_ERR_CUDA;
      if (capacity > 0) {
        const int blocks = (int)std::min<int64_t>((capacity + 255) / 256, 65535 * 4);
        ranges_kernel<<<blocks, 256, 0, st>>>(kin, d_num_pairs, capacity, ranges, num_ranges);
      }
    }
  }
  return launch_status(cudaGetLastError());
}
