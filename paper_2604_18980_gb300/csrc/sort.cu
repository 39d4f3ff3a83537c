// sort.cu -- stable LSD radix sorts (Sec. 2.1 sorting stage) of 32- or 64-bit
// keys with 32-bit values, and the per-tile ranges of the sorted pairs.
//
// Used three ways: the depth pre-sort of the Gaussians (32-bit keys: the fp32
// depth bits), the sort of the tile keys of depth-ordered pairs (32-bit keys:
// view * tiles + tile), and the sort of full 64-bit (tile | depth) pair keys.
//
// "Onesweep" organisation: one kernel reads every key once and builds the
// histograms of all digits; then each digit pass is a single kernel in which
// each block (512 threads x 8 keys; 256 x 16 for 32-bit keys and digits of up
// to 8 bits, lean_kernel) ranks its keys with warp-level match/ballot
// (per-warp digit counters in shared memory), publishes its digit counts,
// places its keys in shared memory in block-sorted order, obtains each digit's
// global offset by a decoupled look-back over the preceding blocks (bounded
// spin, partition ids from an atomic counter), and writes runs of equal digits
// as contiguous stores.  Ranking visits keys in index order (warp-major, then
// item, then lane), so every pass is stable and equal keys keep their input
// order.
#include <algorithm>
#include <cstddef>
#include <utility>

#include "ags_internal.cuh"

namespace ags {

constexpr int kSortThreads = 512;
constexpr int kSortItems = 8;                             // keys per thread
constexpr int kSortPart = kSortThreads * kSortItems;      // 4096 keys per partition
constexpr int kMaxRadix = 512;                            // digits of up to 9 bits
constexpr int kMaxPasses = 16;
constexpr uint32_t kLbAgg = 1u << 30;
constexpr uint32_t kLbInc = 2u << 30;
constexpr uint32_t kLbMask = (1u << 30) - 1u;
constexpr int kLookWindow = 8;                           // predecessors polled per round trip
constexpr size_t kSortHdr = 256;                          // pass counters
constexpr size_t kSortHistBytes = (size_t)kMaxPasses * kMaxRadix * 4;

__device__ __forceinline__ uint32_t key_digit(uint32_t k, int shift, uint32_t mask) { return (k >> shift) & mask; }
__device__ __forceinline__ uint32_t key_digit(uint64_t k, int shift, uint32_t mask) {
  return (uint32_t)(k >> shift) & mask;
}
// Range (tile) index of a key: 32-bit keys are the index, 64-bit pair keys
// carry it in the high word.
// Range index of a key: the key itself (64-bit keys: their high word), or, for
// tile keys that carry the view above `shift` bits (view << shift | tile),
// view * per + tile.
struct RangeMap {
  uint32_t shift;   // 0: the key itself
  uint32_t per;     // ranges per view
};
__device__ __forceinline__ uint32_t key_range(uint32_t k, RangeMap m) {
  return m.shift ? (k >> m.shift) * m.per + (k & ((1u << m.shift) - 1u)) : k;
}
__device__ __forceinline__ uint32_t key_range(uint64_t k, RangeMap) { return (uint32_t)(k >> 32); }

// Staging index with one padding word per 32: keys of consecutive digits are
// staged about 4096 / RADIX words apart, which would otherwise put many lanes
// of a warp on one shared-memory bank.
__device__ __forceinline__ uint32_t stage_index(uint32_t i) { return i + (i >> 5); }
constexpr int kStageWords = kSortPart + kSortPart / 32;

template <int RADIX, typename K>
struct SortSmem {
  static constexpr int kWarps = kSortThreads / 32;
  uint32_t bhist[RADIX];        // block-local exclusive digit starts
  uint32_t gbase[RADIX];        // global index of block-local position 0, per digit (mod 2^32)
  uint32_t scan_tot[kWarps];
  uint32_t part;
  union {
    struct {
      uint16_t warp_hist[kWarps][RADIX + 2];               // ranking; slot RADIX absorbs keys past the count
      uint32_t bins[kWarps][RADIX + 1];                    // peer masks of the atomic-OR ranking (last member:
    } r;                                                   // absent from the launch when ranking by match)
    struct {
      K keys[kStageWords];
      uint32_t vals[kStageWords];
    } stage;                                               // block-sorted keys, before the look-back
  } u;
};

// Dynamic shared memory of a digit pass: the peer-mask table only when it is used.
template <int RADIX, typename K>
static size_t sort_smem_bytes(bool rank_or) {
  using Sm = SortSmem<RADIX, K>;
  if (rank_or) return sizeof(Sm);
  return offsetof(Sm, u) + std::max(sizeof(Sm::u.r.warp_hist), sizeof(Sm::u.stage));   // <= sizeof(Sm)
}

// The count is read on the device and clamped to the buffer capacity (after
// an emission overflow it exceeds it; the status block already records that).
__device__ __forceinline__ uint32_t clamped_count(const int64_t* count_ptr, int64_t capacity) {
  int64_t c = *count_ptr;
  return (uint32_t)(c < 0 ? 0 : (c > capacity ? capacity : c));
}

// Sixteen consecutive keys from a 16-byte aligned address.
__device__ __forceinline__ void load16(const uint32_t* p, uint32_t (&k)[16]) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const uint4 t = __ldcs(q + i);
    k[4 * i] = t.x; k[4 * i + 1] = t.y; k[4 * i + 2] = t.z; k[4 * i + 3] = t.w;
  }
}
__device__ __forceinline__ void load16(const uint64_t* p, uint64_t (&k)[16]) {
  const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const ulonglong2 t = __ldcs(q + i);
    k[2 * i] = t.x; k[2 * i + 1] = t.y;
  }
}

// Global digit histograms of every pass in one read.  Each thread takes 16
// consecutive keys and counts runs of equal digits before adding them: the
// keys are highly clustered (pairs of one Gaussian are consecutive, the depth
// exponent byte is nearly constant), so a run costs one shared atomic instead
// of one per key, and unclustered digits do not contend anyway.
template <typename K>
__global__ void __launch_bounds__(256) hist_kernel(const K* __restrict__ keys, const int64_t* count_ptr,
                                                   int64_t capacity, int begin_bit, int end_bit, int digit_bits,
                                                   int passes, int radix, uint32_t* ghist) {
  __shared__ uint32_t h[kMaxPasses * kMaxRadix];
  for (int i = threadIdx.x; i < passes * radix; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const uint32_t count = clamped_count(count_ptr, capacity);
  constexpr int R = 16;
  const uint32_t stride = gridDim.x * blockDim.x * R;
  for (uint32_t i0 = (blockIdx.x * blockDim.x + threadIdx.x) * R; i0 < count; i0 += stride) {
    K k[R];
    if (i0 + R <= count) {
      load16(keys + i0, k);
    } else {
#pragma unroll
      for (int q = 0; q < R; q++) k[q] = (i0 + q < count) ? keys[i0 + q] : (K)0;
    }
    const int nv = (int)min((uint32_t)R, count - i0);
    for (int p = 0; p < passes; p++) {
      const int sh = begin_bit + p * digit_bits;
      const uint32_t m = (1u << min(digit_bits, end_bit - sh)) - 1u;
      uint32_t cur = key_digit(k[0], sh, m), run = 1;
#pragma unroll
      for (int q = 1; q < R; q++) {
        if (q >= nv) break;
        const uint32_t d = key_digit(k[q], sh, m);
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

// One digit pass over a partition of 4096 keys.  The keys are ranked within
// each warp (match.any, index order, so the pass is stable); the per-warp
// counts give the block's digit totals, which are published to the look-back
// at once; the keys are placed in shared memory in block-sorted order, and
// only then does the block look back for each digit's global offset (up to
// kLookWindow predecessors per round trip, consumed front to back until the
// first inclusive prefix), with its registers free.  kout may be null (the
// last pass of a sort whose caller needs only the values); ranges, when not
// null, receive [start, end) of every range index met in this last pass.
template <int RADIX, typename K>
__global__ void __launch_bounds__(kSortThreads, sizeof(K) == 4 ? 3 : 2)
onesweep_kernel(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
                uint32_t* __restrict__ vout, const int64_t* count_ptr, int64_t capacity, int identity, int shift,
                uint32_t mask, int rank_or, const uint32_t* __restrict__ gprefix, uint32_t* lookback,
                uint32_t* counter, int64_t* status, uint32_t* ranges, uint32_t num_ranges, RangeMap rmap,
                WaitHook hook) {
  using Sm = SortSmem<RADIX, K>;
  constexpr int kWarps = Sm::kWarps;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Sm& S = *reinterpret_cast<Sm*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool digit_thread = tid < RADIX;                   // threads owning one digit each
  if (tid == 0) S.part = atomicAdd(counter, 1u);
  {
    uint32_t* wh = reinterpret_cast<uint32_t*>(&S.u.r.warp_hist[0][0]);
    for (int i = tid; i < kWarps * (RADIX + 2) / 2; i += kSortThreads) wh[i] = 0u;
    if (rank_or) {
      uint32_t* bz = &S.u.r.bins[0][0];
      for (int i = tid; i < kWarps * (RADIX + 1); i += kSortThreads) bz[i] = 0u;
    }
  }
  const uint32_t gp = digit_thread ? __ldg(gprefix + tid) : 0u;   // prefetched, used at the end
  __syncthreads();
  const uint32_t part = S.part;
  const uint32_t count = clamped_count(count_ptr, capacity);
  if (part >= (count + kSortPart - 1) / kSortPart) return;   // no block waits on a higher partition
  const uint32_t base = part * kSortPart;
  const uint32_t ibase = base + warp * (32 * kSortItems) + lane;   // item i sits at ibase + 32 i

  // load (warp-striped, coalesced), all loads first
  K key[kSortItems];
  uint32_t val[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const uint32_t idx = ibase + 32 * i;
    const bool valid = idx < count;
    key[i] = valid ? __ldcs(kin + idx) : (K)0;
    val[i] = valid ? (identity ? idx : __ldcs(vin + idx)) : 0u;
  }

  // rank within the warp (match.any), in index order; keys past the count
  // take the dummy digit RADIX
  uint16_t* wh = S.u.r.warp_hist[warp];
  uint32_t* bins = rank_or ? S.u.r.bins[warp] : nullptr;
  uint32_t rank[kSortItems];
  const unsigned lt_mask = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const uint32_t d = ibase + 32 * i < count ? key_digit(key[i], shift, mask) : (uint32_t)RADIX;
    unsigned peers;
    if (rank_or) {                      // peers by atomic OR of lane bits into the digit's word
      atomicOr(bins + d, 1u << lane);
      __syncwarp();
      peers = bins[d];
    } else {
      peers = __match_any_sync(0xffffffffu, d);
    }
    const uint32_t before = wh[d];
    const uint32_t below = (uint32_t)__popc(peers & lt_mask);
    __syncwarp();
    if (below == 0u) {
      wh[d] = (uint16_t)(before + __popc(peers));
      if (rank_or) bins[d] = 0u;
    }
    __syncwarp();
    rank[i] = before + below;
  }
  __syncthreads();

  // per digit: per-warp exclusive prefixes and the block-exclusive digit start
  uint32_t tot = 0;
  uint32_t* lb = lookback + (size_t)part * RADIX;
  if (digit_thread) {
#pragma unroll 4
    for (int w = 0; w < kWarps; w++) {
      const uint32_t v = S.u.r.warp_hist[w][tid];
      S.u.r.warp_hist[w][tid] = (uint16_t)tot;
      tot += v;
    }
    if (part != hook.withhold) st_relaxed_u32(lb + tid, (part == 0 ? kLbInc : kLbAgg) | tot);
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
    const uint32_t d = key_digit(key[i], shift, mask);
    pos[i] = ibase + 32 * i < count ? S.bhist[d] + wh[d] + rank[i] : 0xffffffffu;
  }
  __syncthreads();   // the staging area aliases the warp counters
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    if (pos[i] < (uint32_t)kSortPart) {
      const uint32_t si = stage_index(pos[i]);
      S.u.stage.keys[si] = key[i];
      S.u.stage.vals[si] = val[i];
    }
  }

  // decoupled look-back per digit: add the predecessors' aggregates back to
  // the nearest inclusive prefix; re-poll from the first one not yet published
  if (digit_thread) {
    uint32_t excl = 0;
    if (part > 0) {
      const uint64_t t0 = globaltimer_ns();
      int32_t p = (int32_t)part - 1;
      bool found = false;
      while (!found) {
        uint32_t sv[kLookWindow];
#pragma unroll
        for (int q = 0; q < kLookWindow; q++)
          sv[q] = (p - q >= 0) ? ld_relaxed_u32(lookback + (size_t)(p - q) * RADIX + tid) : kLbInc;
        int used = 0;
#pragma unroll
        for (int q = 0; q < kLookWindow; q++) {
          const uint32_t flag = sv[q] >> 30;
          if (flag == 0u) break;
          excl += sv[q] & kLbMask;
          used = q + 1;
          if (flag == 2u) { found = true; break; }
        }
        p -= used;
        if (!found && used < kLookWindow && globaltimer_ns() - t0 > hook.limit_ns) {
          set_status(status, AGS_ERR_TIMEOUT, kStageSort);
          break;
        }
      }
      if (part != hook.withhold) st_relaxed_u32(lb + tid, kLbInc | ((excl + tot) & kLbMask));
    }
    S.gbase[tid] = gp + excl - doff;
  }
  __syncthreads();

  // scatter: consecutive positions of one digit go to consecutive addresses
  const uint32_t nvalid = min((uint32_t)kSortPart, count - base);
#pragma unroll 2
  for (int t = 0; t < kSortItems; t++) {
    const uint32_t j = (uint32_t)(t * kSortThreads + tid);
    const bool v = j < nvalid;
    const K k = v ? S.u.stage.keys[stage_index(j)] : (K)0;
    const uint32_t dst = v ? S.gbase[key_digit(k, shift, mask)] + j : 0xffffffffu;
    if (dst < count) {
      if (kout) kout[dst] = k;
      vout[dst] = S.u.stage.vals[stage_index(j)];
    }
    if (ranges) {
      // last pass: the output is fully sorted, so a range index's keys are
      // consecutive here and in the output; its first and last key in this
      // block bound its range (other blocks holding it do the same)
      const uint32_t r = key_range(k, rmap);
      uint32_t rp = __shfl_up_sync(0xffffffffu, r, 1), rn = __shfl_down_sync(0xffffffffu, r, 1);
      if (lane == 0) rp = (v && j > 0) ? key_range(S.u.stage.keys[stage_index(j - 1)], rmap) : 0xffffffffu;
      if (lane == 31) rn = (j + 1 < nvalid) ? key_range(S.u.stage.keys[stage_index(j + 1)], rmap) : 0xffffffffu;
      if (j + 1 >= nvalid) rn = 0xffffffffu;
      if (j == 0) rp = 0xffffffffu;
      if (dst < count && r < num_ranges) {
        if (rp != r) atomicMin(ranges + 2 * (size_t)r, dst);
        if (rn != r) atomicMax(ranges + 2 * (size_t)r + 1, dst + 1);
      }
    }
  }
}

// Every range to (0xffffffff, 0) before the last pass narrows them (one
// 8-byte store per range; a 2D memset of 4-byte rows at an 8-byte pitch ran
// far slower over 10^5..10^6 ranges).
__global__ void ranges_init_kernel(uint2* ranges, int64_t num_ranges) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < num_ranges; t += (int64_t)gridDim.x * blockDim.x)
    ranges[t] = make_uint2(0xffffffffu, 0u);
}

// Ranges no key reached still hold the (0xffffffff, 0) of the initialisation.
__global__ void ranges_fixup_kernel(uint2* ranges, int64_t num_ranges) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < num_ranges; t += (int64_t)gridDim.x * blockDim.x) {
    const uint2 r = ranges[t];
    if (r.x > r.y) ranges[t] = make_uint2(0u, 0u);
  }
}

// Ranges of keys that are already sorted (a sort with no digit pass).
template <typename K>
__global__ void ranges_kernel(const K* __restrict__ keys, const int64_t* count_ptr, int64_t capacity,
                              uint32_t* ranges, int64_t num_ranges, RangeMap rmap) {
  const int64_t count = clamped_count(count_ptr, capacity);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t r = key_range(keys[i], rmap);
    if (r >= (uint64_t)num_ranges) continue;
    if (i == 0 || key_range(keys[i - 1], rmap) != r) ranges[2 * (size_t)r] = (uint32_t)i;
    if (i == count - 1 || key_range(keys[i + 1], rmap) != r) ranges[2 * (size_t)r + 1] = (uint32_t)(i + 1);
  }
}

// ---------------------------------------------------------------------------
// Digit pass for 32-bit keys and digits of up to 8 bits (the depth pre-sort
// and the tile-key pair sort): the same algorithm as onesweep_kernel with 256
// threads x 16 keys per 4096-key partition (fewer warps to merge per digit,
// no register spills), the ranking method fixed at compile time, and the
// tile ranges of the last pass found from each staged key's neighbours.
// ---------------------------------------------------------------------------
constexpr int kLT = 256, kLI = 16, kLW = kLT / 32;
static_assert(kLT * kLI == kSortPart, "partition size");

template <int RADIX, bool kOr>
struct LeanSmem {
  uint32_t bstart[RADIX];
  uint32_t gbase[RADIX];
  uint32_t wtot[kLW];
  uint32_t part;
  union {
    struct {
      uint16_t wh[kLW][RADIX + 2];
      uint32_t bins[kOr ? kLW : 1][RADIX + 1];
    } r;
    struct {
      uint32_t keys[kStageWords];
      uint32_t vals[kStageWords];
    } st;
  } u;
};

__device__ __forceinline__ uint32_t bfe32(uint32_t k, int shift, int bits) {
  uint32_t d;
  asm("bfe.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(k), "r"(shift), "r"(bits));
  return d;
}

template <int RADIX, bool kOr, bool kPersist>
__global__ void __launch_bounds__(kLT, 4)
lean_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
            uint32_t* __restrict__ vout, const int64_t* count_ptr, int64_t capacity, int identity, int shift,
            int bits, const uint32_t* __restrict__ gprefix, uint32_t* lookback, uint32_t* counter, int64_t* status,
            uint32_t* ranges, uint32_t num_ranges, RangeMap rmap, WaitHook hook) {
  using Sm = LeanSmem<RADIX, kOr>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Sm& S = *reinterpret_cast<Sm*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool dthread = tid < RADIX;
  const uint32_t gp = dthread ? __ldg(gprefix + tid) : 0u;
  const uint32_t count = clamped_count(count_ptr, capacity);
  const uint32_t nparts = (count + kSortPart - 1) / kSortPart;
  // one partition per block, or (persistent) partitions in ticket order until
  // none is left -- every lower ticket belongs to a block that is running or
  // done, so the look-back always makes progress
  for (;;) {
  if (tid == 0) S.part = atomicAdd(counter, 1u);
  {
    uint32_t* wz = reinterpret_cast<uint32_t*>(&S.u.r.wh[0][0]);
    for (int i = tid; i < kLW * (RADIX + 2) / 2; i += kLT) wz[i] = 0u;
    if (kOr) {
      uint32_t* bz = &S.u.r.bins[0][0];
      for (int i = tid; i < kLW * (RADIX + 1); i += kLT) bz[i] = 0u;
    }
  }
  __syncthreads();
  const uint32_t part = S.part;
  if (part >= nparts) return;
  const uint32_t base = part * kSortPart;
  const uint32_t ibase = base + (uint32_t)warp * (32u * kLI) + (uint32_t)lane;   // item i at ibase + 32 i
  const bool full = base + kSortPart <= count;

  uint32_t key[kLI], val[kLI], rank[kLI];
  if (full) {
#pragma unroll
    for (int i = 0; i < kLI; i++) key[i] = __ldcs(kin + ibase + 32 * i);
#pragma unroll
    for (int i = 0; i < kLI; i++) val[i] = identity ? ibase + 32 * i : __ldcs(vin + ibase + 32 * i);
  } else {
#pragma unroll
    for (int i = 0; i < kLI; i++) {
      const uint32_t idx = ibase + 32 * i;
      key[i] = idx < count ? __ldcs(kin + idx) : 0u;
      val[i] = idx < count ? (identity ? idx : __ldcs(vin + idx)) : 0u;
    }
  }
  uint16_t* wh = S.u.r.wh[warp];
  uint32_t* bins = kOr ? S.u.r.bins[warp] : nullptr;
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kLI; i++) {
    const uint32_t d = (full || ibase + 32 * i < count) ? bfe32(key[i], shift, bits) : (uint32_t)RADIX;
    unsigned peers;
    if (kOr) {
      atomicOr(bins + d, 1u << lane);
      __syncwarp();
      peers = bins[d];
    } else {
      peers = __match_any_sync(0xffffffffu, d);
    }
    const uint32_t before = wh[d];
    const uint32_t below = (uint32_t)__popc(peers & lt);
    __syncwarp();
    if (below == 0u) {
      wh[d] = (uint16_t)(before + __popc(peers));
      if (kOr) bins[d] = 0u;
    }
    __syncwarp();
    rank[i] = before + below;
  }
  __syncthreads();
  uint32_t tot = 0;
  if (dthread) {
#pragma unroll
    for (int w = 0; w < kLW; w++) {
      const uint32_t v = S.u.r.wh[w][tid];
      S.u.r.wh[w][tid] = (uint16_t)tot;
      tot += v;
    }
    if (part != hook.withhold) st_relaxed_u32(lookback + (size_t)part * RADIX + tid, (part == 0 ? kLbInc : kLbAgg) | tot);
  }
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) S.wtot[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0;
#pragma unroll
  for (int w = 0; w < kLW; w++) wpre += w < warp ? S.wtot[w] : 0u;
  const uint32_t doff = wpre + incl - tot;
  if (dthread) S.bstart[tid] = doff;
  __syncthreads();
  uint32_t pos[kLI];
#pragma unroll
  for (int i = 0; i < kLI; i++) {
    const uint32_t d = bfe32(key[i], shift, bits);
    pos[i] = (full || ibase + 32 * i < count) ? S.bstart[d] + wh[d] + rank[i] : 0xffffffffu;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kLI; i++) {
    if (full || pos[i] != 0xffffffffu) {
      const uint32_t si = stage_index(pos[i]);
      S.u.st.keys[si] = key[i];
      S.u.st.vals[si] = val[i];
    }
  }
  if (dthread) {
    uint32_t excl = 0;
    if (part > 0) {
      const uint64_t t0 = globaltimer_ns();
      int32_t p = (int32_t)part - 1;
      bool found = false;
      while (!found) {
        uint32_t sv[kLookWindow];
#pragma unroll
        for (int q = 0; q < kLookWindow; q++)
          sv[q] = (p - q >= 0) ? ld_relaxed_u32(lookback + (size_t)(p - q) * RADIX + tid) : kLbInc;
        int used = 0;
#pragma unroll
        for (int q = 0; q < kLookWindow; q++) {
          const uint32_t flag = sv[q] >> 30;
          if (flag == 0u) break;
          excl += sv[q] & kLbMask;
          used = q + 1;
          if (flag == 2u) { found = true; break; }
        }
        p -= used;
        if (!found && used < kLookWindow && globaltimer_ns() - t0 > hook.limit_ns) {
          set_status(status, AGS_ERR_TIMEOUT, kStageSort);
          break;
        }
      }
      if (part != hook.withhold)
        st_relaxed_u32(lookback + (size_t)part * RADIX + tid, kLbInc | ((excl + tot) & kLbMask));
    }
    S.gbase[tid] = gp + excl - doff;
  }
  __syncthreads();
  const uint32_t nvalid = full ? (uint32_t)kSortPart : count - base;
#pragma unroll 4
  for (int t = 0; t < kLI; t++) {
    const uint32_t j = (uint32_t)(t * kLT + tid);
    if (!full && j >= nvalid) break;
    const uint32_t k = S.u.st.keys[stage_index(j)];
    const uint32_t d = bfe32(k, shift, bits);
    const uint32_t dst = S.gbase[d] + j;
    if (dst >= count) continue;   // only after a look-back that gave up: stay inside the output
    if (kout) kout[dst] = k;
    vout[dst] = S.u.st.vals[stage_index(j)];
    if (ranges) {
      // the staged keys are sorted; within one digit's run here the outputs
      // are consecutive, so a range boundary inside the run is this block's
      // alone (plain stores); the ends of a run may continue in other blocks
      // (atomics against the (0xffffffff, 0) initialisation)
      const uint32_t r = key_range(k, rmap);
      const bool first = j == 0 || bfe32(S.u.st.keys[stage_index(j - 1)], shift, bits) != d;
      const bool last = j + 1 >= nvalid || bfe32(S.u.st.keys[stage_index(j + 1)], shift, bits) != d;
      if (r < num_ranges) {
        if (first) {
          atomicMin(ranges + 2 * (size_t)r, dst);
        } else {
          const uint32_t rp = key_range(S.u.st.keys[stage_index(j - 1)], rmap);
          if (rp != r) {
            ranges[2 * (size_t)r] = dst;
            if (rp < num_ranges) ranges[2 * (size_t)rp + 1] = dst;
          }
        }
        if (last) atomicMax(ranges + 2 * (size_t)r + 1, dst + 1);
      }
    }
  }
  if (!kPersist) return;
  __syncthreads();     // the staged keys are read above; the next partition overwrites them
  }
}

template <int RADIX>
static cudaError_t launch_lean(bool rank_or, dim3 grid, cudaStream_t st, const uint32_t* kin, const uint32_t* vin,
                               uint32_t* kout, uint32_t* vout, const int64_t* count_ptr, int64_t capacity, int identity,
                               int shift, int bits, const uint32_t* gprefix, uint32_t* lookback, uint32_t* counter,
                               int64_t* status, uint32_t* ranges, uint32_t num_ranges, RangeMap rmap, WaitHook hook,
                               bool persistent) {
  cudaError_t e;
  // persistent: as many blocks as are resident at once (they take the
  // partitions of the count on the device by ticket), never more than the
  // partitions of the capacity; otherwise one block per partition of the capacity
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto resident = [&](auto kern, int smem) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kLT, smem) != cudaSuccess || occ < 1) occ = 1;
    return persistent ? dim3(std::min<unsigned>(grid.x, (unsigned)(sms * occ))) : grid;
  };
  auto go = [&](auto kern, int smem) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<resident(kern, smem), kLT, smem, st>>>(kin, vin, kout, vout, count_ptr, capacity, identity, shift, bits,
                                                  gprefix, lookback, counter, status, ranges, num_ranges, rmap, hook);
    return cudaSuccess;
  };
  const int smem_or = (int)sizeof(LeanSmem<RADIX, true>), smem_m = (int)sizeof(LeanSmem<RADIX, false>);
  if (rank_or)
    e = persistent ? go(lean_kernel<RADIX, true, true>, smem_or) : go(lean_kernel<RADIX, true, false>, smem_or);
  else
    e = persistent ? go(lean_kernel<RADIX, false, true>, smem_m) : go(lean_kernel<RADIX, false, false>, smem_m);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}


static size_t sort_parts(int64_t capacity) { return (size_t)((capacity + kSortPart - 1) / kSortPart); }

template <int RADIX, typename K>
static cudaError_t launch_passes(K*& kin, uint32_t*& vin, K* kout, uint32_t* vout, const int64_t* d_num_pairs,
                                 int64_t capacity, int begin_bit, int end_bit, int digit_bits, int passes,
                                 int flags, uint32_t* ghist, uint32_t* lookback, uint32_t* counters,
                                 int64_t* d_status, uint32_t* ranges, int64_t num_ranges, RangeMap rmap,
                                 cudaStream_t st) {
  hist_scan_kernel<RADIX><<<passes, RADIX, 0, st>>>(ghist);
  const int rank_or = (flags & AGS_SORT_RANK_OR) ? 1 : 0;
  const int smem = (int)sort_smem_bytes<RADIX, K>(rank_or != 0);
  // the attribute always allows the larger layout, so that launches of either
  // ranking method (e.g. recorded together in one CUDA graph) stay valid
  cudaError_t e = cudaFuncSetAttribute(onesweep_kernel<RADIX, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sort_smem_bytes<RADIX, K>(true));
  if (e != cudaSuccess) return e;
  const size_t parts = sort_parts(capacity);
  for (int p = 0; p < passes; p++) {
    e = cudaMemsetAsync(lookback, 0, parts * RADIX * 4, st);
    if (e != cudaSuccess) return e;
    const int sh = begin_bit + p * digit_bits;
    const uint32_t mask = (1u << std::min(digit_bits, end_bit - sh)) - 1u;
    const int identity = (p == 0 && (flags & AGS_SORT_IDENTITY_VALUES)) ? 1 : 0;
    const bool last = p == passes - 1;
    K* ko = (last && (flags & AGS_SORT_DISCARD_KEYS)) ? nullptr : kout;
    if (sizeof(K) == 4 && RADIX <= 256 && !(flags & AGS_SORT_WIDE_BLOCK)) {
      e = launch_lean<RADIX <= 256 ? RADIX : 256>(rank_or != 0, dim3((unsigned)parts), st,
                                                  reinterpret_cast<const uint32_t*>(kin), vin,
                                                  reinterpret_cast<uint32_t*>(ko), vout, d_num_pairs, capacity,
                                                  identity, sh, __builtin_popcount(mask), ghist + p * RADIX,
                                                  lookback, counters + p, d_status, last ? ranges : nullptr,
                                                  (uint32_t)num_ranges, rmap, wait_hook(flags & AGS_SORT_TEST_STALL),
                                                  (flags & AGS_SORT_PERSISTENT) != 0);
      if (e != cudaSuccess) return e;
      std::swap(kin, kout);
      std::swap(vin, vout);
      continue;
    }
    onesweep_kernel<RADIX, K><<<(unsigned)parts, kSortThreads, smem, st>>>(
        kin, vin, ko, vout, d_num_pairs, capacity, identity, sh, mask, rank_or, ghist + p * RADIX, lookback,
        counters + p,
        d_status, last ? ranges : nullptr, (uint32_t)num_ranges, rmap, wait_hook(flags & AGS_SORT_TEST_STALL));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  return cudaSuccess;
}

template <typename K>
static ags_status sort_impl(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, const int64_t* d_num_pairs,
                            int64_t capacity, int32_t begin_bit, int32_t end_bit, int32_t digit_bits, int32_t flags,
                            uint32_t* ranges, int64_t num_ranges, int32_t* result_in_alt, int64_t* d_status,
                            void* ws, size_t ws_bytes, void* stream, RangeMap rmap = RangeMap{0u, 0u});

}  // namespace ags

extern "C" size_t ags_sort_workspace_bytes(int64_t capacity) {
  if (capacity < 0) return 0;
  return ags::kSortHdr + ags::kSortHistBytes + ags::sort_parts(capacity) * ags::kMaxRadix * 4;
}

namespace ags {

template <typename K>
static ags_status sort_impl(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, const int64_t* d_num_pairs,
                            int64_t capacity, int32_t begin_bit, int32_t end_bit, int32_t digit_bits, int32_t flags,
                            uint32_t* ranges, int64_t num_ranges, int32_t* result_in_alt, int64_t* d_status,
                            void* ws, size_t ws_bytes, void* stream, RangeMap rmap) {
  constexpr int kKeyBits = 8 * (int)sizeof(K);
  if (!d_num_pairs || !d_status || capacity < 0 || capacity >= AGS_MAX_PAIRS) return AGS_ERR_INVALID_ARG;
  if (begin_bit < 0 || end_bit > kKeyBits || begin_bit > end_bit || digit_bits < 4 || digit_bits > 9)
    return AGS_ERR_INVALID_ARG;
  if (flags & ~(AGS_SORT_IDENTITY_VALUES | AGS_SORT_DISCARD_KEYS | AGS_SORT_RANK_OR | AGS_SORT_WIDE_BLOCK |
                AGS_SORT_PERSISTENT | AGS_SORT_TEST_STALL))
    return AGS_ERR_INVALID_ARG;
  const int passes = (end_bit - begin_bit + digit_bits - 1) / digit_bits;
  if (passes > kMaxPasses) return AGS_ERR_INVALID_ARG;
  if (ranges && (num_ranges <= 0 || num_ranges > ((int64_t)1 << 32) - 1)) return AGS_ERR_INVALID_ARG;
  if ((uintptr_t)ranges & 7u) return AGS_ERR_INVALID_ARG;       // (start, end) pairs are 8-byte stores
  if (capacity > 0 && (!keys || !vals || (passes > 0 && (!keys_alt || !vals_alt)))) return AGS_ERR_INVALID_ARG;
  if (capacity > 0 && passes > 0 && ((uintptr_t)keys & 15u)) return AGS_ERR_INVALID_ARG;   // 16-byte key loads
  if (!ws || ws_bytes < ags_sort_workspace_bytes(capacity) || ((uintptr_t)ws & 15u)) return AGS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (result_in_alt) *result_in_alt = passes & 1;
  char* w = reinterpret_cast<char*>(ws);
  uint32_t* counters = reinterpret_cast<uint32_t*>(w);
  uint32_t* ghist = reinterpret_cast<uint32_t*>(w + kSortHdr);
  uint32_t* lookback = reinterpret_cast<uint32_t*>(w + kSortHdr + kSortHistBytes);
  // the smallest digit table that holds the digit (at least 64 entries)
  const int radix = digit_bits > 8 ? 512 : digit_bits > 7 ? 256 : digit_bits > 6 ? 128 : 64;
  cudaError_t e = cudaSuccess;
  K* kin = keys;
  uint32_t* vin = vals;
  if (capacity > 0 && passes > 0) {
    e = cudaMemsetAsync(w, 0, kSortHdr + kSortHistBytes, st);
    if (e != cudaSuccess) return AGS_ERR_CUDA;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned hb = (unsigned)std::min<int64_t>((capacity + 255) / 256, (int64_t)sms * 4);
    hist_kernel<K><<<hb, 256, 0, st>>>(keys, d_num_pairs, capacity, begin_bit, end_bit, digit_bits, passes, radix,
                                       ghist);
    if (ranges) {   // start = 0xffffffff, end = 0: the last pass narrows them with atomics
      const int blocks = (int)std::min<int64_t>((num_ranges + 255) / 256, 4096);
      ranges_init_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<uint2*>(ranges), num_ranges);
    }
    auto launch = radix == 512   ? launch_passes<512, K>
                  : radix == 256 ? launch_passes<256, K>
                  : radix == 128 ? launch_passes<128, K>
                                 : launch_passes<64, K>;
    e = launch(kin, vin, keys_alt, vals_alt, d_num_pairs, capacity, begin_bit, end_bit, digit_bits, passes, flags,
               ghist, lookback, counters, d_status, ranges, num_ranges, rmap, st);
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
        ranges_kernel<K><<<blocks, 256, 0, st>>>(kin, d_num_pairs, capacity, ranges, num_ranges, rmap);
      }
    }
  }
  return launch_status(cudaGetLastError());
}

}  // namespace ags

extern "C" ags_status ags_sort(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                               const int64_t* d_num_pairs, int64_t capacity, int32_t begin_bit, int32_t end_bit,
                               int32_t digit_bits, int32_t flags, uint32_t* ranges, int64_t num_ranges,
                               int32_t* result_in_alt, int64_t* d_status, void* ws, size_t ws_bytes,
                               void* stream) {
  return ags::sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, d_num_pairs, capacity, begin_bit, end_bit,
                                  digit_bits, flags, ranges, num_ranges, result_in_alt, d_status, ws, ws_bytes,
                                  stream);
}

extern "C" ags_status ags_sort32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                 const int64_t* d_num_pairs, int64_t capacity, int32_t begin_bit, int32_t end_bit,
                                 int32_t digit_bits, int32_t flags, uint32_t* ranges, int64_t num_ranges,
                                 int32_t* result_in_alt, int64_t* d_status, void* ws, size_t ws_bytes,
                                 void* stream) {
  return ags::sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, d_num_pairs, capacity, begin_bit, end_bit,
                                  digit_bits, flags, ranges, num_ranges, result_in_alt, d_status, ws, ws_bytes,
                                  stream);
}

extern "C" ags_status ags_sort_tiles(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                     const int64_t* d_num_pairs, int64_t capacity, int32_t tile_bits,
                                     int32_t digit_bits, int32_t flags, uint32_t* ranges, int32_t views,
                                     int32_t tiles_per_view, int32_t* result_in_alt, int64_t* d_status, void* ws,
                                     size_t ws_bytes, void* stream) {
  if (tile_bits < 1 || tile_bits > 31 || views < 1 || tiles_per_view < 1 ||
      (int64_t)tiles_per_view > ((int64_t)1 << tile_bits) || (int64_t)views << tile_bits > ((int64_t)1 << 32))
    return AGS_ERR_INVALID_ARG;
  return ags::sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, d_num_pairs, capacity, 0, tile_bits, digit_bits,
                                  flags, ranges, (int64_t)views * tiles_per_view, result_in_alt, d_status, ws,
                                  ws_bytes, stream, ags::RangeMap{(uint32_t)tile_bits, (uint32_t)tiles_per_view});
}
