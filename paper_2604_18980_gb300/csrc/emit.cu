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
//   32-bit keys: key = view * tiles_per_view + tile (pairs emitted in depth order),
//                or view << tile_bits | tile (AGS_EMIT_VIEW_SHIFT: the kernels
//                take the power of two 2^tile_bits as their view stride)
//   val = view * n + i
//
// The look-back spins are bounded (globaltimer); on expiry the status block
// records AGS_ERR_TIMEOUT and every store stays inside `capacity`.
#include <algorithm>
#include <mutex>

#include "ags_internal.cuh"
#include "ellipse.cuh"

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
constexpr int kTileChunk = 2048;                          // pairs per block of the two-pass emission
constexpr int64_t kTileChunksMax = ((int64_t)AGS_MAX_PAIRS + kTileChunk - 1) / kTileChunk + 1;

// Inputs of the ellipse tile test's enumeration; splat == nullptr means whole
// squares (the rectangle records alone decide the tiles).
struct EllipseSrc {
  const float4* splat;       // splat records (centre, conic, opacity, Th)
  const uint32_t* touched;   // kept tiles per Gaussian-view (from the preprocess)
  int W, H;
};

// Pair key of a tile: 64-bit keys append the depth bits, 32-bit keys are the tile alone.
__device__ __forceinline__ void make_key(uint32_t tile, uint32_t dbits, uint64_t& k) {
  k = ((uint64_t)tile << 32) | dbits;
}
__device__ __forceinline__ void make_key(uint32_t tile, uint32_t, uint32_t& k) { k = tile; }

template <typename K>
__global__ void __launch_bounds__(kEmitThreads)
emit_kernel(const uint2* __restrict__ rect, const float* __restrict__ depth, const uint32_t* __restrict__ order,
            int64_t total_bound, const int64_t* d_total, uint32_t n, uint32_t tiles_per_view, uint32_t gx,
            K* __restrict__ keys,
            uint32_t* __restrict__ vals, int64_t capacity, int64_t* d_num_pairs, int64_t* status,
            uint64_t* part_status, uint32_t* counter, uint4* __restrict__ recs,
            uint32_t* __restrict__ chunk_start, EllipseSrc ell, WaitHook hook) {
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
  // entries to visit: all views*n, or the count the device holds (a compacted order)
  int64_t total = total_bound;
  if (d_total) {
    const int64_t t = *d_total;
    total = t < 0 ? 0 : (t > total_bound ? total_bound : t);
  }
  const uint32_t nparts = (uint32_t)((total + kEmitPart - 1) / kEmitPart);
  if (part >= nparts) {                       // beyond the entries: no pairs, nobody waits on it
    if (part == 0 && tid == 0) *d_num_pairs = 0;
    return;
  }
  const int64_t base = (int64_t)part * kEmitPart;

  // 1. coalesced loads of the rectangles (striped), counts staged in s_off
#pragma unroll
  for (int k = 0; k < kEmitItems; k++) {
    int li = k * kEmitThreads + tid;
    int64_t s = base + li;
    uint32_t c = 0;
    if (s < total) {
      uint32_t e = order ? __ldg(order + s) : (uint32_t)s;
      if (AGS_DCHECK(e < (uint64_t)total_bound, status, AGS_CHECK_EMIT_ORDER)) {
        uint2 r = __ldg(rect + e);
        uint32_t x0 = r.x & 0xffffu, y0 = r.x >> 16, x1 = r.y & 0xffffu, y1 = r.y >> 16;
        uint32_t w = x1 - x0;
        c = ell.splat ? __ldg(ell.touched + e) : w * (y1 - y0);
        uint32_t view = e / n;
        s_base[li] = view * tiles_per_view + y0 * gx + x0;
        s_w[li] = w;
        if (sizeof(K) == 8) s_dbits[li] = c ? __float_as_uint(__ldg(depth + e)) : 0u;
        s_idx[li] = e;
      } else {     // (debug builds) an order entry out of range: no pairs, an empty record
        s_base[li] = s_w[li] = s_idx[li] = 0u;
        if (sizeof(K) == 8) s_dbits[li] = 0u;
      }
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
    const bool publish = part != hook.withhold;
    if (part == 0) {
      if (lane == 0 && publish) st_relaxed_u64(part_status, kInc | (uint64_t)agg);
    } else {
      if (lane == 0 && publish) st_relaxed_u64(part_status + part, kAgg | (uint64_t)agg);
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
          if (globaltimer_ns() - t0 > hook.limit_ns) {
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
      if (lane == 0 && publish) st_relaxed_u64(part_status + part, kInc | ((excl + agg) & kValMask));
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

  if (recs) {
    // two-phase emission: only the per-entry records {first pair, splat index,
    // first tile key, width}; the pairs come from tile_emit_kernel
#pragma unroll
    for (int k = 0; k < kEmitItems; k++) {
      const int li = k * kEmitThreads + tid;
      if (base + li < total) {
        const uint64_t off = prefix + s_off[li], end = prefix + s_off[li + 1];
        recs[base + li] = make_uint4((uint32_t)off, s_idx[li], s_base[li], s_w[li]);
        // this entry holds the first pair of every pair block starting inside it
        const uint64_t lim = end < (uint64_t)capacity ? end : (uint64_t)capacity;
        for (uint64_t c = (off + kTileChunk - 1) / kTileChunk * kTileChunk; c < lim; c += kTileChunk)
          chunk_start[c / kTileChunk] = (uint32_t)(base + li);
      }
    }
    if (part == nparts - 1 && tid == 0) {
      const int64_t tot = (int64_t)(prefix + agg);
      *d_num_pairs = tot;
      if (tot > capacity) set_status(status, AGS_ERR_CAPACITY, tot);
    }
    return;
  }

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
      if (ell.splat) {                        // the ellipse test's tiles, row by row
        EllipseWalk wk;
        wk.start(ell.splat, rect, s_idx[lo], n, tiles_per_view, ell.W, ell.H, r);
#pragma unroll 1
        for (int k = 0; k < kEmitRun; k++) {
          const uint32_t j = j0 + k;
          if (j >= agg) break;
          if (j >= s_off[lo + 1]) {           // next Gaussian with pairs
            do lo++; while (j >= s_off[lo + 1]);
            wk.start(ell.splat, rect, s_idx[lo], n, tiles_per_view, ell.W, ell.H, j - s_off[lo]);
          }
          make_key(wk.tile(gx), sizeof(K) == 8 ? s_dbits[lo] : 0u, s_key[warp][lane * kEmitStride + k]);
          s_val[warp][lane * kEmitStride + k] = s_idx[lo];
          wk.next();
        }
      } else {
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
  if (part == nparts - 1 && tid == 0) {
    int64_t tot = (int64_t)(prefix + agg);
    *d_num_pairs = tot;
    if (tot > capacity) set_status(status, AGS_ERR_CAPACITY, tot);
  }
}

// Second phase of the tile-key emission: blocks over fixed ranges of 2048
// pairs, whatever the pairs per Gaussian.  In depth order the large
// Gaussians near the camera come together, and a fused scan-and-emit over
// Gaussian partitions would leave a few blocks with most of the pairs.  The
// first pass recorded which entry holds the first pair of each block; a block
// stages the records its range touches, and its warps emit chunks of 256 pairs
// (8 per lane, one shared-memory binary search each) with coalesced stores,
// as the fused kernel does.  Entries without pairs (an order that lists culled
// views) can push the records of a block past the staging area: the block then
// continues with further windows, found by a 32-way search of the records'
// first-pair offsets.
// Pairs [p0, p1) of the ellipse tile test, enumerated by a whole warp from the
// records rec[0..m] staged in shared memory (rec[m] a sentinel).  The records
// that own these pairs are taken 32 at a time, one per lane; the rows of all
// of them are spread over the lanes (one row per lane per step, the owner found
// by bisection over the row prefix), so that every row's span is computed once
// with all lanes busy whatever the Gaussians' sizes; a segmented scan places
// each row's tiles, each lane stages its row's tiles that fall in [p0, p1)
// (at most kEmitChunk pairs) in shared memory, and the warp writes them out
// with coalesced stores.  k_run (32 words of shared memory per warp) carries
// each record's kept tiles from one step of rows to the next.
__device__ __forceinline__ void warp_emit_ellipse(const uint4* rec, int m, uint32_t p0, uint32_t p1,
                                                  const EllipseSrc& ell, const uint2* __restrict__ rect, uint32_t n,
                                                  uint32_t tiles_per_view, uint32_t gx, uint32_t* __restrict__ keys,
                                                  uint32_t* __restrict__ vals, uint32_t* k_run, uint32_t* st_key,
                                                  uint32_t* st_val, int lane) {
  int lo = 0, hi = m;                              // rec[lo].x <= p0 < rec[hi].x
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (rec[mid].x <= p0) lo = mid; else hi = mid;
  }
  for (int eb = lo; eb < m && rec[eb].x < p1;) {
    // this lane's record of the batch
    const int ek = eb + lane;
    const bool in = ek < m && rec[ek].x < p1;
    const int nb = __popc(__ballot_sync(0xffffffffu, in));   // records start in order: a prefix of the lanes
    uint32_t e = 0, off = 0, h = 0, vb = 0;
    int y0 = 0;
    EllipseTiles E{0.f, 0.f, 1.f, 0.f, 1.f, -1.f, 0, 0, ell.W, ell.H, 1.f, 1.f};
    if (in && rec[ek + 1].x > rec[ek].x) {
      e = rec[ek].y;
      off = rec[ek].x;
      const uint2 rr = __ldg(rect + e);
      y0 = (int)(rr.x >> 16);
      h = (rr.y >> 16) - (uint32_t)y0;
      const float4 s0 = __ldg(ell.splat + (size_t)e * 3), s1 = __ldg(ell.splat + (size_t)e * 3 + 1);
      const float th = __ldg(reinterpret_cast<const float*>(ell.splat + (size_t)e * 3 + 2) + 1);
      E = EllipseTiles{s0.x, s0.y, s0.z, s0.w, s1.x, ellipse_level(s1.y, th), (int)(rr.x & 0xffffu),
                       (int)(rr.y & 0xffffu), ell.W, ell.H, 0.f, 0.f};
      ellipse_prepare(E);
      vb = (e / n) * tiles_per_view;
    }
    uint32_t incl = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t rstart = incl - h, R = __shfl_sync(0xffffffffu, incl, 31);
    k_run[lane] = 0u;
    __syncwarp();
    for (uint32_t k0 = 0; k0 < R; k0 += 32) {
      const uint32_t k = k0 + (uint32_t)lane;
      int own = 0;                                 // the last lane whose rows start at or before k
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const uint32_t s = __shfl_sync(0xffffffffu, rstart, own + step);
        if (s <= k) own += step;
      }
      const EllipseTiles Eo{__shfl_sync(0xffffffffu, E.u, own), __shfl_sync(0xffffffffu, E.v, own),
                            __shfl_sync(0xffffffffu, E.A, own), __shfl_sync(0xffffffffu, E.B, own),
                            __shfl_sync(0xffffffffu, E.C, own), __shfl_sync(0xffffffffu, E.Q, own),
                            __shfl_sync(0xffffffffu, E.x0, own), __shfl_sync(0xffffffffu, E.x1, own), ell.W, ell.H,
                            __shfl_sync(0xffffffffu, E.iA, own), __shfl_sync(0xffffffffu, E.iC, own)};
      const uint32_t rs_own = __shfl_sync(0xffffffffu, rstart, own);
      const int ty = __shfl_sync(0xffffffffu, y0, own) + (int)(k - rs_own);
      int slo = 1, shi = 0;
      if (k < R) ellipse_row_span(Eo, ty, slo, shi);
      const uint32_t c = slo <= shi ? (uint32_t)(shi - slo + 1) : 0u;
      // kept index of this row's first tile within its record: the record's
      // count from earlier steps plus its earlier rows in this step
      uint32_t sc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, sc, o);
        if (lane >= o) sc += y;
      }
      const uint32_t ex = sc - c;
      const int first = (int)(max(rs_own, k0) - k0);   // first lane of this record in the step
      const uint32_t kidx = k_run[own] + ex - __shfl_sync(0xffffffffu, ex, first);
      const uint32_t pr = __shfl_sync(0xffffffffu, off, own) + kidx;   // pair index of the row's first tile
      const uint32_t t0 = __shfl_sync(0xffffffffu, vb, own) + (uint32_t)ty * gx + (uint32_t)slo;
      const uint32_t ev = __shfl_sync(0xffffffffu, e, own);
      __syncwarp();
      if (c) atomicAdd(&k_run[own], c);
      // this lane's row: stage its tiles that fall in [p0, p1)
      const uint32_t a = max(pr, p0), b = min(pr + c, p1);
      for (uint32_t q = a; q < b; q++) {
        st_key[q - p0] = t0 + (q - pr);
        st_val[q - p0] = ev;
      }
      __syncwarp();
    }
    eb += nb;
  }
  for (uint32_t q = (uint32_t)lane; q < p1 - p0; q += 32) {   // coalesced stores of the staged pairs
    keys[p0 + q] = st_key[q];
    vals[p0 + q] = st_val[q];
  }
  __syncwarp();
}

// Pass 1 of the two-pass tile-key emission: the record {first pair, splat
// index, first tile key, width} of every visited entry, the entry holding the
// first pair of every kTileChunk-pair block, and the pair total.  Partitions
// of 4096 entries per 256-thread block (a quarter of the look-backs of
// 1024-entry partitions): striped loads of the order (coalesced) with the 16
// rectangle gathers of a thread in flight together, the counts transposed
// through shared memory for a blocked scan, a decoupled look-back for the
// partition's offset.  The records go out striped (coalesced 16-byte stores)
// as soon as an entry's rectangle is known, with the count in the first-pair
// field, which the last step overwrites (still in L2), so no entry state stays
// in registers across the scan.  Same records, block starts and total as the
// fused kernel's record path.
constexpr int kScanItems = 16;
constexpr int kScanPart = kEmitThreads * kScanItems;      // 4096 entries per partition

__device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }   // conflict-free blocked reads

__global__ void __launch_bounds__(kEmitThreads)
tile_scan_kernel(const uint2* __restrict__ rect, const uint32_t* __restrict__ order, int64_t total_bound,
                 const int64_t* d_total, uint32_t n, uint32_t tiles_per_view, uint32_t gx, int64_t capacity,
                 int64_t* d_num_pairs, int64_t* status, uint64_t* part_status, uint32_t* counter,
                 uint4* __restrict__ recs, uint32_t* __restrict__ chunk_start, EllipseSrc ell, WaitHook hook) {
  __shared__ uint32_t s_c[kScanPart + kScanPart / 32];   // counts, then exclusive offsets in the partition
  __shared__ uint32_t s_warp[kEmitThreads / 32];
  __shared__ uint32_t s_part;
  __shared__ unsigned long long s_prefix;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_part = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t part = s_part;
  int64_t total = total_bound;
  if (d_total) {
    const int64_t t = *d_total;
    total = t < 0 ? 0 : (t > total_bound ? total_bound : t);
  }
  const uint32_t nparts = (uint32_t)((total + kScanPart - 1) / kScanPart);
  if (part >= nparts) {                       // beyond the entries: no pairs, nobody waits on it
    if (part == 0 && tid == 0) *d_num_pairs = 0;
    return;
  }
  const int64_t base = (int64_t)part * kScanPart;

  // 1. striped entries li = k * 256 + tid: order, rectangle, count; the record
  //    is written now with the count in place of the first pair (step 4 fixes it)
  uint32_t e[kScanItems];
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    const int64_t s = base + k * kEmitThreads + tid;
    e[k] = 0xffffffffu;
    if (s < total) {
      const uint32_t v = order ? __ldg(order + s) : (uint32_t)s;
      e[k] = AGS_DCHECK(v < (uint64_t)total_bound, status, AGS_CHECK_EMIT_ORDER) ? v : 0xffffffffu;
    }
  }
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    const int li = k * kEmitThreads + tid;
    const uint2 r = e[k] != 0xffffffffu ? __ldg(rect + e[k]) : make_uint2(0u, 0u);
    const uint32_t x0 = r.x & 0xffffu, y0 = r.x >> 16, w = (r.y & 0xffffu) - x0, h = (r.y >> 16) - y0;
    uint32_t c = w * h;
    if (ell.splat) c = c ? __ldg(ell.touched + e[k]) : 0u;
    s_c[scan_pad(li)] = c;
    if (base + li < total) {
      const uint32_t ev = e[k] == 0xffffffffu ? 0u : e[k];
      recs[base + li] = make_uint4(c, ev, (ev / n) * tiles_per_view + y0 * gx + x0, w);
    }
  }
  __syncthreads();

  // 2. blocked scan: thread t owns entries 16t .. 16t+15
  uint32_t tsum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) tsum += s_c[scan_pad(tid * kScanItems + j)];
  uint32_t incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0, agg = 0;
#pragma unroll
  for (int w = 0; w < kEmitThreads / 32; w++) {
    const uint32_t v = s_warp[w];
    if (w < warp) wpre += v;
    agg += v;
  }
  uint32_t run = wpre + incl - tsum;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    const uint32_t c = s_c[scan_pad(tid * kScanItems + j)];
    s_c[scan_pad(tid * kScanItems + j)] = run;
    run += c;
  }

  // 3. decoupled look-back (warp 0) for the partition's global offset
  if (warp == 0) {
    uint64_t excl = 0;
    const bool publish = part != hook.withhold;
    if (part == 0) {
      if (lane == 0 && publish) st_relaxed_u64(part_status, kInc | (uint64_t)agg);
    } else {
      if (lane == 0 && publish) st_relaxed_u64(part_status + part, kAgg | (uint64_t)agg);
      int64_t top = (int64_t)part - 1;
      const uint64_t t0 = globaltimer_ns();
      bool timed_out = false;
      while (true) {
        const int64_t qidx = top - lane;
        const uint64_t sv = qidx >= 0 ? ld_relaxed_u64(part_status + qidx) : kInc;
        const uint32_t flag = (uint32_t)(sv >> 62);
        const unsigned inc_mask = __ballot_sync(0xffffffffu, flag == 2u);
        const unsigned inv_mask = __ballot_sync(0xffffffffu, flag == 0u);
        const int first_inc = inc_mask ? __ffs(inc_mask) - 1 : 32;
        const unsigned upto = first_inc >= 31 ? 0xffffffffu : ((2u << first_inc) - 1u);
        if ((inv_mask & upto) && !timed_out) {
          if (globaltimer_ns() - t0 > hook.limit_ns) {
            timed_out = true;
            if (lane == 0) set_status(status, AGS_ERR_TIMEOUT, kStageEmit);
          }
          continue;
        }
        excl += warp_sum((lane <= first_inc) ? (sv & kValMask) : 0ull);
        if (first_inc < 32 || timed_out) break;
        top -= 32;
      }
      if (lane == 0 && publish) st_relaxed_u64(part_status + part, kInc | ((excl + agg) & kValMask));
    }
    if (lane == 0) s_prefix = excl;
  }
  __syncthreads();
  const uint64_t prefix = s_prefix;

  // 4. each record's first pair, and the pair blocks that start inside it
#pragma unroll 4
  for (int k = 0; k < kScanItems; k++) {
    const int li = k * kEmitThreads + tid;
    if (base + li < total) {
      const uint32_t o = s_c[scan_pad(li)];
      const uint32_t c = (li + 1 < kScanPart ? s_c[scan_pad(li + 1)] : agg) - o;
      const uint64_t off = prefix + o, end = off + c;
      recs[base + li].x = (uint32_t)off;
      const uint64_t lim = end < (uint64_t)capacity ? end : (uint64_t)capacity;
      for (uint64_t q = (off + kTileChunk - 1) / kTileChunk * kTileChunk; q < lim; q += kTileChunk)
        chunk_start[q / kTileChunk] = (uint32_t)(base + li);
    }
  }
  if (part == nparts - 1 && tid == 0) {
    const int64_t tot = (int64_t)(prefix + agg);
    *d_num_pairs = tot;
    if (tot > capacity) set_status(status, AGS_ERR_CAPACITY, tot);
  }
}

struct TileEmitSmem {
  uint4 rec[kTileChunk + 2];
  uint32_t k_run[kEmitThreads / 32][32];
  uint32_t key[kEmitThreads / 32][32 * kEmitStride];
  uint32_t val[kEmitThreads / 32][32 * kEmitStride];
  uint32_t k0;
  uint32_t k1;       // first window of a block: one past the sentinel record it needs
};

__global__ void __launch_bounds__(kEmitThreads)
tile_emit_kernel(const uint4* __restrict__ recs, const uint32_t* __restrict__ chunk_start, const int64_t* d_entries,
                 int64_t entries_bound, const int64_t* d_num_pairs, int64_t capacity, uint32_t gx,
                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, const uint2* __restrict__ rect, uint32_t n,
                 uint32_t tiles_per_view, EllipseSrc ell) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileEmitSmem& S = *reinterpret_cast<TileEmitSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int64_t ne = d_entries ? *d_entries : entries_bound;
  ne = ne < 0 ? 0 : (ne > entries_bound ? entries_bound : ne);
  int64_t np = *d_num_pairs;
  np = np < 0 ? 0 : (np > capacity ? capacity : np);
  const uint32_t nent = (uint32_t)ne, total = (uint32_t)np;
  for (uint32_t b = blockIdx.x; (uint64_t)b * kTileChunk < total; b += gridDim.x) {
    const uint32_t c0 = b * (uint32_t)kTileChunk;
    const uint32_t cend = min(c0 + (uint32_t)kTileChunk, total);
    uint32_t cs = c0;
    bool first = true;
    while (cs < cend) {
      const bool win_first = first;
      if (first) {
        // the block's records run from the one holding its first pair to the one
        // holding the next block's first pair (whose successor is the sentinel)
        if (tid == 0) {
          S.k0 = min(__ldg(chunk_start + b), nent - 1u);
          S.k1 = cend < total ? min(__ldg(chunk_start + b + 1) + 2u, nent + 1u) : nent + 1u;
        }
      } else if (warp == 0) {   // the last record whose first pair is <= cs
        uint32_t lo = 0, hi = nent;                // answer in [lo, hi); record 0 starts at pair 0
        while (hi - lo > 32) {
          const uint32_t step = (hi - lo + 31) / 32;
          const uint32_t idx = lo + (uint32_t)lane * step;
          const unsigned bal = __ballot_sync(0xffffffffu, idx < hi && __ldg(&recs[idx].x) <= cs);
          lo = lo + (uint32_t)(31 - __clz(bal)) * step;   // lane 0 probes lo itself, so bal != 0
          hi = min(hi, lo + step);
        }
        const uint32_t idx = lo + (uint32_t)lane;
        const unsigned bal = __ballot_sync(0xffffffffu, idx < hi && __ldg(&recs[idx].x) <= cs);
        if (lane == 0) S.k0 = lo + (uint32_t)(31 - __clz(bal));
      }
      first = false;
      __syncthreads();
      const uint32_t k0 = S.k0;
      const uint32_t m = min(min((uint32_t)kTileChunk + 1u, nent - k0), win_first ? S.k1 - 1u - k0 : 0xffffffffu);
      for (uint32_t q = tid; q <= m; q += kEmitThreads)
        S.rec[q] = (k0 + q < nent) ? __ldg(&recs[k0 + q]) : make_uint4(total, 0u, 0u, 1u);
      __syncthreads();
      const uint32_t wend = min(cend, S.rec[m].x);   // pairs this window covers: [cs, wend)
      const uint32_t cn = wend > cs ? wend - cs : 0u;
      for (uint32_t w0 = (uint32_t)warp * kEmitChunk; w0 < cn; w0 += (kEmitThreads / 32) * kEmitChunk) {
        if (ell.splat) {                           // ellipse tiles: the whole warp enumerates rows
          warp_emit_ellipse(S.rec, (int)m, cs + w0, min(cs + w0 + (uint32_t)kEmitChunk, wend), ell, rect, n,
                            tiles_per_view, gx, keys, vals, S.k_run[warp], S.key[warp], S.val[warp], lane);
          continue;
        }
        const uint32_t j0 = cs + w0 + (uint32_t)lane * kEmitRun;
        if (j0 < wend) {
          int lo = 0, hi = (int)m;                 // invariant: rec[lo].x <= j0 < rec[hi].x
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (S.rec[mid].x <= j0) lo = mid; else hi = mid;
          }
          uint4 rc = S.rec[lo];
          uint32_t nxt = S.rec[lo + 1].x;
          const uint32_t r = j0 - rc.x;
          {
            uint32_t ry = r / rc.w, rx = r - ry * rc.w;
#pragma unroll
            for (int k = 0; k < kEmitRun; k++) {
              const uint32_t j = j0 + k;
              if (j >= wend) break;
              while (j >= nxt) {                     // next record with pairs (j < wend <= rec[m].x)
                lo++;
                rc = S.rec[lo];
                nxt = S.rec[lo + 1].x;
                rx = 0;
                ry = 0;
              }
              S.key[warp][lane * kEmitStride + k] = rc.z + ry * gx + rx;
              S.val[warp][lane * kEmitStride + k] = rc.y;
              if (++rx == rc.w) { rx = 0; ry++; }
            }
          }
        }
        __syncwarp();
        const uint32_t nval = min((uint32_t)kEmitChunk, cn - w0);
        for (uint32_t q = lane; q < nval; q += 32) {
          const uint32_t pos = cs + w0 + q;
          const uint32_t si = (q / kEmitRun) * kEmitStride + (q % kEmitRun);
          keys[pos] = S.key[warp][si];
          vals[pos] = S.val[warp][si];
        }
        __syncwarp();
      }
      cs = wend > cs ? wend : cend;                    // always progresses on consistent records
      __syncthreads();
    }
  }
}

static size_t emit_parts(int64_t total) { return (size_t)((total + kEmitPart - 1) / kEmitPart); }

// The ellipse enumeration's inputs for AGS_EMIT_ELLIPSE (or whole squares).
static ags_status ellipse_src(const ags_projected* proj, const CamBatch& cb, int32_t flags, EllipseSrc* out) {
  *out = EllipseSrc{nullptr, nullptr, cb.c[0].W, cb.c[0].H};
  if (!(flags & AGS_EMIT_ELLIPSE)) return AGS_OK;
  if (!proj->splat || !proj->tiles_touched || ((uintptr_t)proj->splat & 15u)) return AGS_ERR_INVALID_ARG;
  out->splat = reinterpret_cast<const float4*>(proj->splat);
  out->touched = proj->tiles_touched;
  return AGS_OK;
}

}  // namespace ags

extern "C" size_t ags_emit_workspace_bytes(int64_t n, int32_t views) {
  if (n < 0 || views < 1 || n > (((int64_t)1 << 32) - 1) / views) return 0;
  return 256 + 8 * ags::emit_parts(n * (int64_t)views);
}

extern "C" ags_status ags_emit_pairs(const ags_projected* proj, int64_t n, int32_t views, const ags_camera* cams,
                                     const uint32_t* order, uint64_t* keys, uint32_t* vals, int64_t capacity,
                                     int64_t* d_num_pairs, int64_t* d_status, int32_t flags, void* ws,
                                     size_t ws_bytes, void* stream) {
  using namespace ags;
  if (!proj || !d_num_pairs || !d_status || n < 0 || capacity < 0 || capacity > AGS_MAX_PAIRS)
    return AGS_ERR_INVALID_ARG;
  CamBatch cb;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  if (n > (((int64_t)1 << 32) - 1) / views) return AGS_ERR_INVALID_ARG;   // before multiplying
  const int64_t total = n * (int64_t)views;
  cudaStream_t st = (cudaStream_t)stream;
  if (flags & ~(AGS_EMIT_ELLIPSE | AGS_EMIT_TEST_STALL)) return AGS_ERR_INVALID_ARG;
  if (total == 0) return launch_status(cudaMemsetAsync(d_num_pairs, 0, sizeof(int64_t), st));
  if (!proj->rect || !proj->depth || (capacity > 0 && (!keys || !vals))) return AGS_ERR_INVALID_ARG;
  EllipseSrc ell;
  s = ellipse_src(proj, cb, flags, &ell);
  if (s != AGS_OK) return s;
  if (!ws || ws_bytes < ags_emit_workspace_bytes(n, views) || ((uintptr_t)ws & 7u)) return AGS_ERR_INVALID_ARG;
  const size_t parts = emit_parts(total);
  uint32_t tiles_per_view = (uint32_t)cb.c[0].gx * (uint32_t)cb.c[0].gy;
  if ((uint64_t)tiles_per_view * (uint64_t)views >= (1ull << 32)) return AGS_ERR_INVALID_ARG;
  cudaError_t e = cudaMemsetAsync(ws, 0, 256 + 8 * parts, st);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws);
  uint64_t* part_status = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ws) + 256);
  emit_kernel<uint64_t><<<(unsigned)parts, kEmitThreads, 0, st>>>(
      reinterpret_cast<const uint2*>(proj->rect), proj->depth, order, total, nullptr, (uint32_t)n, tiles_per_view,
      (uint32_t)cb.c[0].gx, keys, vals, capacity, d_num_pairs, d_status, part_status, counter, nullptr, nullptr, ell,
      wait_hook(flags & AGS_EMIT_TEST_STALL));
  return launch_status(cudaGetLastError());
}

extern "C" size_t ags_emit_tile_workspace_bytes(int64_t n, int32_t views) {
  if (n < 0 || views < 1 || n > (((int64_t)1 << 32) - 1) / views) return 0;
  const int64_t total = n * (int64_t)views;
  return (256 + 8 * ags::emit_parts(total) + 15) / 16 * 16 + 16 * (size_t)total + 4 * (size_t)ags::kTileChunksMax;
}

extern "C" ags_status ags_emit_tile_pairs(const ags_projected* proj, int64_t n, int32_t views,
                                          const ags_camera* cams, const uint32_t* order,
                                          const int64_t* d_order_count, uint32_t* keys, uint32_t* vals,
                                          int64_t capacity, int64_t* d_num_pairs, int64_t* d_status,
                                          int32_t flags, void* ws, size_t ws_bytes, void* stream) {
  using namespace ags;
  if (!proj || !d_num_pairs || !d_status || n < 0 || capacity < 0 || capacity > AGS_MAX_PAIRS)
    return AGS_ERR_INVALID_ARG;
  CamBatch cb;
  ags_status s = build_cams(cams, views, &cb);
  if (s != AGS_OK) return s;
  if (n > (((int64_t)1 << 32) - 1) / views) return AGS_ERR_INVALID_ARG;   // before multiplying
  const int64_t total = n * (int64_t)views;
  cudaStream_t st = (cudaStream_t)stream;
  if (flags & ~(AGS_EMIT_SINGLE_PASS | AGS_EMIT_ELLIPSE | AGS_EMIT_VIEW_SHIFT | AGS_EMIT_TEST_STALL))
    return AGS_ERR_INVALID_ARG;
  if (total == 0) return launch_status(cudaMemsetAsync(d_num_pairs, 0, sizeof(int64_t), st));
  if (!proj->rect || (capacity > 0 && (!keys || !vals))) return AGS_ERR_INVALID_ARG;
  EllipseSrc ell;
  s = ellipse_src(proj, cb, flags, &ell);
  if (s != AGS_OK) return s;
  if (!ws || ws_bytes < ags_emit_tile_workspace_bytes(n, views) || ((uintptr_t)ws & 15u)) return AGS_ERR_INVALID_ARG;
  const size_t parts = emit_parts(total);
  // the view's part of a key: view * tiles_per_view, or view << tile_bits (AGS_EMIT_VIEW_SHIFT)
  uint32_t tiles_per_view = (uint32_t)cb.c[0].gx * (uint32_t)cb.c[0].gy;
  if (flags & AGS_EMIT_VIEW_SHIFT) {
    uint32_t stride = 2u;
    while (stride < tiles_per_view) stride <<= 1;
    tiles_per_view = stride;
  }
  if ((uint64_t)tiles_per_view * (uint64_t)views > (1ull << 32)) return AGS_ERR_INVALID_ARG;
  cudaError_t e = cudaMemsetAsync(ws, 0, 256 + 8 * parts, st);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws);
  uint64_t* part_status = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ws) + 256);
  uint4* recs = reinterpret_cast<uint4*>(reinterpret_cast<char*>(ws) + (256 + 8 * parts + 15) / 16 * 16);
  uint32_t* chunk_start = reinterpret_cast<uint32_t*>(recs + total);
  const int64_t* d_entries = order ? d_order_count : nullptr;
  if (flags & AGS_EMIT_SINGLE_PASS) {   // fused scan and emission over partitions of Gaussians
    emit_kernel<uint32_t><<<(unsigned)parts, kEmitThreads, 0, st>>>(
        reinterpret_cast<const uint2*>(proj->rect), proj->depth, order, total, d_entries, (uint32_t)n,
        tiles_per_view, (uint32_t)cb.c[0].gx, keys, vals, capacity, d_num_pairs, d_status, part_status, counter,
        nullptr, nullptr, ell, wait_hook(flags & AGS_EMIT_TEST_STALL));
    return launch_status(cudaGetLastError());
  }
  // phase 1: per-entry records and the pair count
  tile_scan_kernel<<<(unsigned)((total + kScanPart - 1) / kScanPart), kEmitThreads, 0, st>>>(
      reinterpret_cast<const uint2*>(proj->rect), order, total, d_entries, (uint32_t)n, tiles_per_view,
      (uint32_t)cb.c[0].gx, capacity, d_num_pairs, d_status, part_status, counter, recs, chunk_start, ell,
      wait_hook(flags & AGS_EMIT_TEST_STALL));
  e = cudaGetLastError();
  if (e != cudaSuccess || capacity == 0) return launch_status(e);
  // phase 2: the pairs, in blocks of kTileChunk (grid-stride over the device count)
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t chunks = (capacity + kTileChunk - 1) / kTileChunk;
  const unsigned grid = (unsigned)std::min<int64_t>(chunks, (int64_t)sms * 8);
  const int smem = (int)sizeof(TileEmitSmem);
  e = cudaFuncSetAttribute(tile_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return AGS_ERR_CUDA;
  tile_emit_kernel<<<grid, kEmitThreads, smem, st>>>(recs, chunk_start, d_entries, total, d_num_pairs, capacity,
                                                     (uint32_t)cb.c[0].gx, keys, vals,
                                                     reinterpret_cast<const uint2*>(proj->rect), (uint32_t)n,
                                                     tiles_per_view, ell);
  return launch_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Allocation-free variant of ags_emit_pairs (see include/ags.h).
//
// The look-back state lives in a library-owned device array instead of a
// caller workspace.  In host code `g_emit_scratch` names a host-side stand-in,
// not a device address, so the device address is looked up with
// cudaGetSymbolAddress (with the device current) and cached per CUDA context:
// a device reset creates a new context, whose id differs, so the address is
// looked up again there instead of reusing the old context's.
// ---------------------------------------------------------------------------
namespace ags {

constexpr int64_t kNoAllocMaxGaussianViews = (int64_t)1 << 24;     // views * n limit
constexpr size_t kNoAllocScratchBytes = 256 + 8 * (size_t)(kNoAllocMaxGaussianViews / kEmitPart);   // 128.25 KiB

static __device__ __align__(256) unsigned char g_emit_scratch[kNoAllocScratchBytes];

// The current context's unique id, through the driver entry points the
// runtime exposes (no link against the driver library).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

static bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    resolved = true;
  }
  void* ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

static std::mutex g_scratch_mutex;
static void* g_scratch_ptr[256];                  // device address per device ordinal (nullptr: not set up)
static unsigned long long g_scratch_ctx[256];     // the context it was looked up in

static ags_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return AGS_ERR_CUDA;
  unsigned long long ctx = 0;
  const bool have_ctx = current_context_id(&ctx);   // false before the runtime set up any context
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!have_ctx || !g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;   // the lookup also sets up the device's primary context if needed
    if (cudaGetSymbolAddress(&p, g_emit_scratch) != cudaSuccess || !p) return AGS_ERR_CUDA;
    if (!have_ctx && !current_context_id(&ctx)) return AGS_ERR_CUDA;
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = ctx;
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
  if (n > kNoAllocMaxGaussianViews / views) return AGS_ERR_INVALID_ARG;   // beyond the static scratch
  const int64_t total = n * (int64_t)views;
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
      reinterpret_cast<const uint2*>(proj->rect), proj->depth, order, total, nullptr, (uint32_t)n, tiles_per_view,
      (uint32_t)cb.c[0].gx, keys, vals, capacity, d_num_pairs, d_status, part_status, counter, nullptr, nullptr,
      EllipseSrc{nullptr, nullptr, cb.c[0].W, cb.c[0].H}, wait_hook(false));
  return launch_status(cudaGetLastError());
}
