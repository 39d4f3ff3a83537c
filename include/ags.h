/*
 * ags.h -- C ABI of the AdaGScale 3D Gaussian Splatting hot path for one
 * NVIDIA GB300 (sm_103a).
 *
 * The rendering pipeline (AdaGScale, arXiv 2604.18980, Sec. 2.1 and Fig. 1) has
 * four stages, one entry point each, plus the hand-written backward:
 *
 *   ags_preprocess          cull, EWA projection, SH colour, depth, and the
 *                           AdaGScale threshold Th (Eq. 10), opacity cull and
 *                           adjusted footprint (Sec. 3.3)
 *   ags_emit_pairs          Gaussian-tile pairs with 64-bit (tile | depth) keys
 *                           (Sec. 2.1, Sec. 3.3 "Gaussian-tile pair generation")
 *   ags_sort                stable LSD radix sort of the pairs (Sec. 2.1) and the
 *                           per-tile [start, end) ranges
 *
 * and the same tile lists by a shorter route: sort the Gaussians of every view
 * by depth first (ags_sort32 of depth_key), emit 32-bit tile keys in that order
 * (ags_emit_tile_pairs) and sort only those (ags_sort32) -- bit-identical
 * lists with fewer, narrower digit passes.
 *
 *   ags_rasterize           per-16x16-tile front-to-back alpha blending, Eq. 1
 *                           and Eq. 2, always with the original covariance and
 *                           tau (Sec. 3.3 "dual-size strategy")
 *   ags_rasterize_backward  adjoint of the blend and of the preprocess (not in
 *                           the paper; the pair selection is held fixed)
 *   ags_calibrate_lut       T_up(depth) look-up table from per-Gaussian maximum
 *                           transmittance (Sec. 3.4)
 *   ags_morton_codes,       storage order of the Gaussians along a Morton curve
 *   ags_gather_gaussians    (a setup step, not in the paper)
 *   ags_peripheral_scores   diagnostics: exact peripheral score (Eq. 4) at each
 *   ags_contribution_hist   Gaussian's Th beside its estimates (Eq. 6, 7, 9);
 *   ags_render_skip         the contribution distribution of a plain render and
 *                           the image with low-contribution blends skipped
 *                           (Sec. 2.2 Fig. 4a, Sec. 3.2 Fig. 5)
 *
 * Conventions (all entry points):
 *  - Every pointer is a DEVICE pointer owned by the caller unless it is marked
 *    "host".  The library allocates no memory and keeps no mutable global
 *    state -- with one exception, ags_emit_pairs_noalloc's static device
 *    scratch array and its cached device address; scratch memory
 *    ("workspace") is passed in by the caller, sized by the matching
 *    *_workspace_bytes() call.
 *  - `stream` is a cudaStream_t passed as void*.  Every call only enqueues
 *    work on that stream and returns without synchronising, so a sequence of
 *    calls can be captured in a CUDA graph.
 *  - The return value reports what the host can detect: invalid arguments
 *    (AGS_ERR_INVALID_ARG, nothing is launched) and launch failures
 *    (AGS_ERR_CUDA).  What only the device can detect -- pair capacity
 *    overflow, a bounded wait that gave up, non-finite inputs -- is written to
 *    the caller's device status block `d_status` (int64_t[4], zeroed with
 *    ags_status_reset) and read back by ags_check.  No kernel ever traps.
 *  - Arrays are structure-of-arrays fp32 unless stated; `n` Gaussians, `views`
 *    cameras of one common width and height rendered in one launch per stage.
 *  - Tiles are 16x16 pixels; pixel centres sit at integer coordinates.
 *  - Tile ranges are uint32[tiles][2] = (start, end) pairs, 8-byte aligned
 *    (every kernel reads or writes a pair in one 8-byte access).
 *  - Gaussian-tile pair counts are limited to AGS_MAX_PAIRS per sort call.
 */
#ifndef AGS_H
#define AGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AGS_TILE 16
#define AGS_MAX_VIEWS 32
#define AGS_MAX_LUT_BINS 32
#define AGS_MAX_PAIRS ((int64_t)1 << 30)   /* exclusive bound on a sort's pair count */

typedef enum {
  AGS_OK = 0,
  AGS_ERR_INVALID_ARG = 1,
  AGS_ERR_CAPACITY = 2,     /* more pairs than `capacity`; detail = pairs needed */
  AGS_ERR_TIMEOUT = 3,      /* a bounded device wait gave up; detail = stage id */
  AGS_ERR_CUDA = 4,         /* a CUDA launch or runtime call failed */
  AGS_ERR_NUMERIC = 5,      /* non-finite Gaussian parameters were culled; detail = count */
  AGS_ERR_BOUNDS = 6        /* debug builds (AGS_DEBUG) only: an index read from the inputs
                             * (a pair value, a tile range, an emission order entry) was out
                             * of range and its access skipped; detail = the first failed
                             * check's id (AGS_CHECK_*), d_status[3] = bit (1 << id) of every
                             * check that failed */
} ags_status;

/* Check ids of AGS_ERR_BOUNDS. */
#define AGS_CHECK_BLEND_RANGE 1      /* ags_rasterize: a tile range with start > end */
#define AGS_CHECK_BLEND_VALUE 2      /* ags_rasterize: a pair value >= views * n */
#define AGS_CHECK_BACKWARD_RANGE 3   /* ags_rasterize_backward: a tile range with start > end */
#define AGS_CHECK_BACKWARD_VALUE 4   /* ags_rasterize_backward: a pair value >= views * n */
#define AGS_CHECK_EMIT_ORDER 5       /* emission: an order entry >= views * n */

typedef enum { AGS_SCALE_PLAIN = 0, AGS_SCALE_ADAGSCALE = 1 } ags_scale_mode;

/* Which tiles of a Gaussian's footprint get a pair.  SQUARE: every tile of the
 * square [u-r, u+r]^2 (3D-GS; the paper's baseline).  ELLIPSE: those of them
 * that the ellipse alpha >= Th meets -- with the blending conic, q <= Q =
 * 2 ln(opacity / Th), Th = tau in plain mode and Eq. 10 in AdaGScale mode --
 * tested against the rectangle spanned by the tile's pixel centres: the exact
 * footprint-tile intersection of the FlashGS-style renderer the paper's
 * implementation builds on.  In plain mode it drops only tiles whose pixels all
 * have alpha < tau, so the image is unchanged. */
typedef enum { AGS_TILE_SQUARE = 0, AGS_TILE_ELLIPSE = 1 } ags_tile_test;

/* Pinhole camera (host struct).  viewmat is the row-major 3x4 world->camera
 * transform (+x right, +y down, +z forward): t = R m + t_cam.  The EWA
 * frustum clamp uses tan(fov/2) = 0.5*width/fx and 0.5*height/fy. */
typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
  float viewmat[12];
  float campos[3];
  float near_z;             /* 0.2 in 3D-GS */
} ags_camera;

/* Render parameters (host struct). */
typedef struct {
  int32_t scale_mode;       /* ags_scale_mode */
  int32_t sh_degree;        /* 0..3 */
  int32_t lut_bins;         /* 1..AGS_MAX_LUT_BINS; 20 in the paper (Sec. 3.4) */
  float K;                  /* peripheral-loss budget K >= 0 (Eq. 5, Eq. 10) */
  float tau;                /* alpha threshold, 1/255 (Sec. 2.1) */
  float t_min;              /* transmittance stop, 1e-4 (Sec. 2.1) */
  float alpha_max;          /* alpha clamp, 0.99 (3D-GS) */
  float lut_depth_max;      /* depth range [0, lut_depth_max] of the LUT; 100 (Sec. 3.4) */
  float lut[AGS_MAX_LUT_BINS]; /* T_up per depth bin (Sec. 3.2 Eq. 7, Sec. 3.4) */
  float bg[3];              /* background colour added with the final transmittance */
  int32_t tile_test;        /* ags_tile_test */
  int32_t blend_flags;      /* launch shape of the blend: 0 (8x16-pixel warp blocks, 32-splat
                             * batches) or AGS_BLEND_* bits; any other bit is invalid.  The
                             * image, final_T, n_contrib, max_T and stats do not depend on it. */
} ags_params;

#define AGS_BLEND_ROWS2 1     /* blend_flags: 8x8-pixel warp blocks (four warps a tile, two rows a
                               * lane) instead of 8x16 (two warps, four rows a lane) */
#define AGS_BLEND_BATCH64 2   /* blend_flags: each warp stages 64 of its tile's splats a round
                               * (two a lane) instead of 32 */

/* Gaussian parameters (pointers to device memory, SoA fp32). */
typedef struct {
  const float* mean;          /* [3][n] world position */
  const float* log_scale;     /* [3][n] log standard deviations */
  const float* quat;          /* [4][n] rotation (w,x,y,z), any non-zero norm */
  const float* opacity_logit; /* [n]    opacity = sigmoid(logit) */
  const float* sh;            /* [(sh_degree+1)^2][3][n] real SH, index l*l+l+m */
  int64_t n;
} ags_gaussians;

/* Per-view preprocess results (device memory, index e = view*n + i). */
typedef struct {
  float* splat;             /* [views*n][12], 16-byte aligned:
                               u v A B | C opacity r g | b Th Sxx Syy
                               (u,v) 2D mean in pixels, (A,B,C) conic of the
                               ORIGINAL dilated 2D covariance, (Sxx,Syy) its
                               diagonal, Th the alpha threshold (Eq. 10) */
  float* depth;             /* [views*n] view-space z */
  uint16_t* rect;           /* [views*n][4] tile rectangle x0 y0 x1 y1 (end
                               exclusive); all zero for culled Gaussians */
  uint32_t* tiles_touched;  /* [views*n] (x1-x0)*(y1-y0), nullable */
  uint8_t* flags;           /* [views*n] bit0-2 colour clamped at 0, bit3/bit4
                               EWA x/y frustum clamp, bit7 culled */
  uint32_t* depth_key;      /* [views*n] float_bits(depth) (depth > 0, so the
                               bits order as the depths do), all ones for
                               Gaussians without pairs; nullable.  A stable
                               sort of these (ags_sort32) gives an emission
                               order in which each view's Gaussians are in
                               depth order (equal depths in index order); see
                               ags_emit_tile_pairs. */
} ags_projected;

/* Device status block: int64_t[4] = {status code, detail, non-finite count,
 * failed-check bits (AGS_DEBUG builds; zero otherwise)}. */

/* ---------------------------------------------------------------------- */

/* Zero a device status block (int64_t[4]) on `stream`. */
ags_status ags_status_reset(int64_t* d_status, void* stream);

/* Synchronise `stream`, read the device status block and return its code;
 * *detail (host, nullable) receives its detail word. */
ags_status ags_check(const int64_t* d_status, void* stream, int64_t* detail);

/* Human-readable name of a status code (static string). */
const char* ags_status_string(ags_status s);

/* Preprocess (Sec. 2.1 preprocessing; Eq. 10 and Sec. 3.3 in AdaGScale mode).
 * For every view v and Gaussian i: frustum (near-plane) cull, EWA projection
 * of the 3D covariance R S S^T R^T to the dilated 2D covariance (+0.3 I), its
 * conic, 2D mean, depth, opacity = sigmoid(logit), colour = SH + 0.5 clamped
 * at 0, and the footprint radius: ceil(3 sqrt(lambda_max)) in plain mode; in
 * AdaGScale mode Th = K / (T_up(depth) 2 pi sqrt(det)) + tau (Eq. 10), culled
 * when Th > opacity, else radius ceil(sqrt(lambda_max) min(3, sqrt(2 ln(opacity/Th)))).
 * The rectangle holds every tile containing a pixel centre within the square
 * [u-r, u+r] x [v-r, v+r].  cams (host) has `views` entries of equal size.
 * Non-finite parameters are culled and counted in d_status[2]. */
ags_status ags_preprocess(const ags_gaussians* g, const ags_camera* cams, int32_t views,
                          const ags_params* params, const ags_projected* out,
                          int64_t* d_status, void* stream);

/* Scratch bytes needed by ags_emit_pairs for views*n Gaussians. */
size_t ags_emit_workspace_bytes(int64_t n, int32_t views);

/* Pair emission (Sec. 2.1, Sec. 3.3).  Exclusive prefix sum of the rectangle
 * areas (single pass, decoupled look-back) and one pair per covered tile, in
 * Gaussian order and row-major within a rectangle:
 *   key = ((view * tiles_per_view + tile) << 32) | float_bits(depth),
 *   val = view * n + i.
 * `order` (nullable, [views*n]) visits the Gaussians in that order instead
 * (a permutation of 0..views*n-1).  *d_num_pairs (device int64) receives the
 * total.  Pairs beyond `capacity` are not written; the status block then
 * holds AGS_ERR_CAPACITY and the total needed.  flags: AGS_EMIT_ELLIPSE (the
 * kept tiles of each square, row-major, instead of all of them). */
#define AGS_EMIT_ELLIPSE 2       /* emission flag: the tiles of the ellipse test (the
                                    preprocess ran with tile_test AGS_TILE_ELLIPSE; reads
                                    splat records and tiles_touched) instead of whole squares */
ags_status ags_emit_pairs(const ags_projected* proj, int64_t n, int32_t views,
                          const ags_camera* cams, const uint32_t* order,
                          uint64_t* keys, uint32_t* vals, int64_t capacity,
                          int64_t* d_num_pairs, int64_t* d_status, int32_t flags,
                          void* ws, size_t ws_bytes, void* stream);

/* Scratch bytes needed by ags_emit_tile_pairs for views*n Gaussian-views
 * (the look-back state and a 16-byte record per visited Gaussian-view). */
size_t ags_emit_tile_workspace_bytes(int64_t n, int32_t views);

/* Pair emission with 32-bit tile keys (Sec. 2.1, Sec. 3.3): ags_emit_pairs
 * with key = view * tiles_per_view + tile and no depth bits.  Pairs come out
 * in the order of `order`; when `order` is the stable depth order (a sort of
 * depth_key, or of the compacted keys of ags_compact_visible), a stable sort of
 * these keys (ags_sort32 over their bits) yields exactly the per-tile lists
 * that sorting the 64-bit (tile | depth) keys of ags_emit_pairs yields: the
 * tile, then the depth, then the Gaussian index.  d_order_count (device int64,
 * nullable; used only with `order`) is the number of entries of `order` to
 * visit, at most views*n (default views*n).  `proj->depth` is not read.
 * Two passes by default: counts, offsets and one record per visited
 * Gaussian-view, then the pairs in blocks of a fixed number of pairs (balanced
 * however the tile counts cluster in depth order); flags AGS_EMIT_SINGLE_PASS
 * selects the single fused pass of ags_emit_pairs instead.  Same pairs either
 * way.  AGS_EMIT_ELLIPSE as for ags_emit_pairs.  Workspace:
 * ags_emit_tile_workspace_bytes, 16-byte aligned. */
#define AGS_EMIT_SINGLE_PASS 1  /* ags_emit_tile_pairs flag: one fused scan-and-emit pass over
                                   partitions of Gaussian-views (faster when the tile counts
                                   are spread evenly along the order) */
#define AGS_EMIT_TEST_STALL 256 /* emission flag, for testing the bounded wait only: partition 1
                                   of the look-back never publishes its sums, so the partitions
                                   after it give up after 2 ms (instead of 200 ms), record
                                   AGS_ERR_TIMEOUT with detail 1 (emission) and finish with every
                                   store inside capacity; the pairs are then meaningless */
#define AGS_EMIT_VIEW_SHIFT 4   /* ags_emit_tile_pairs flag: key = (view << tile_bits) | tile,
                                   tile_bits = the bits of tiles_per_view - 1 (at least 1), for
                                   ags_sort_tiles; with an `order` that lists each view's
                                   Gaussian-views together (views ascending, depth order within
                                   each: a stable sort of ags_view_keys after the depth sort) */
ags_status ags_emit_tile_pairs(const ags_projected* proj, int64_t n, int32_t views,
                               const ags_camera* cams, const uint32_t* order,
                               const int64_t* d_order_count, uint32_t* keys, uint32_t* vals,
                               int64_t capacity, int64_t* d_num_pairs, int64_t* d_status,
                               int32_t flags, void* ws, size_t ws_bytes, void* stream);

/* Scratch bytes needed by ags_compact_visible for views*n Gaussian-views
 * (per 4096-entry partition: its count and offset, and 512 B of visibility bits). */
size_t ags_compact_workspace_bytes(int64_t n, int32_t views);

/* The Gaussian-views with pairs (flags bit 7 clear), in increasing index
 * e = view*n + i, with their depth keys: keys[k] = float_bits(depth[e]),
 * ids[k] = e for k < *d_count (device int64, written).  Culled views never
 * reach a tile list (Sec. 2.1 frustum cull, Sec. 3.3 Th > opacity cull), so the
 * depth pre-sort (ags_sort32 of keys with ids as values, count d_count) needs
 * only these.  Reads proj->flags and proj->depth (both 16-byte aligned);
 * keys and ids hold up to views*n entries.  Three launches -- per-partition
 * counts, one block scanning them, the writes -- with no device-side wait;
 * d_status is not written. */
ags_status ags_compact_visible(const ags_projected* proj, int64_t n, int32_t views, uint32_t* keys,
                               uint32_t* ids, int64_t* d_count, int64_t* d_status, void* ws,
                               size_t ws_bytes, void* stream);

/* View of each listed Gaussian-view: keys[k] = order[k] / n for k < *d_count
 * (device int64, clamped to [0, capacity]).  A stable sort of these keys
 * (ags_sort32, values `order`) after the depth sort lists the views one after
 * the other, each in depth order -- the order AGS_EMIT_VIEW_SHIFT expects. */
ags_status ags_view_keys(const uint32_t* order, const int64_t* d_count, int64_t capacity, int64_t n,
                         uint32_t* keys, void* stream);

/* Largest views*n that ags_emit_pairs_noalloc accepts (2^24). */
int64_t ags_emit_pairs_noalloc_max_gaussians(void);

/* ags_emit_pairs for callers that cannot allocate device memory.  The paper
 * has no counterpart: this exists for callers that own no allocator of their
 * own -- a host application that gives a plugin a fixed device-memory budget
 * and forbids it to allocate, or code calling this C ABI from a language with
 * no CUDA allocator binding -- and so cannot provide the workspace that
 * ags_emit_pairs needs.  Arguments and results are those of ags_emit_pairs
 * without `flags` (whole squares) and `ws`/`ws_bytes`; the caller still
 * passes every input and output.
 * The look-back scratch is a library-owned static device array of
 * 256 + 8 * (2^24 / 1024) bytes (about 128 KiB), held by every GPU that loads
 * the library until the process exits; views*n above
 * ags_emit_pairs_noalloc_max_gaussians() is rejected with
 * AGS_ERR_INVALID_ARG.  The first call on a device looks up that array's
 * device address (with the device current) and caches it per CUDA context, so
 * make the first call on each device before any stream capture, and again
 * first after a device reset (a reset destroys the context and its copy of the
 * array; the next call sees a new context and looks the address up anew).
 * Every call zeroes the part of the array it uses on `stream`; calls whose
 * work overlaps on the GPU (on different streams) share the array and race:
 * serialise them.  No call allocates or frees memory. */
ags_status ags_emit_pairs_noalloc(const ags_projected* proj, int64_t n, int32_t views,
                                  const ags_camera* cams, const uint32_t* order,
                                  uint64_t* keys, uint32_t* vals, int64_t capacity,
                                  int64_t* d_num_pairs, int64_t* d_status, void* stream);

/* Scratch bytes needed by ags_sort for up to `capacity` pairs. */
size_t ags_sort_workspace_bytes(int64_t capacity);

#define AGS_SORT_IDENTITY_VALUES 1   /* sort flag: values are 0..count-1; `vals` is not read */
#define AGS_SORT_DISCARD_KEYS 2      /* sort flag: the last digit pass writes no keys, so the
                                        key buffer that would hold the result is left
                                        unspecified (values and ranges only) */
#define AGS_SORT_TEST_STALL 256      /* sort flag, for testing the bounded wait only: partition 1
                                        of each digit pass's look-back never publishes, so the
                                        partitions after it give up after 2 ms, record
                                        AGS_ERR_TIMEOUT with detail 2 (sort) and write only inside
                                        the count; the order is then meaningless */
#define AGS_SORT_RANK_OR 4           /* sort flag: rank a warp's equal digits with shared-memory
                                        atomic-OR peer masks instead of warp match; same result,
                                        faster when a warp's keys mostly carry distinct digits
                                        (tile keys in emission order) */
#define AGS_SORT_WIDE_BLOCK 8        /* sort flag: the digit passes over 32-bit keys with digits of
                                        up to 8 bits use 512-thread partitions of 8 keys a thread
                                        instead of 256 threads of 16 keys (4096 keys either way);
                                        same result.  64-bit keys and 9-bit digits always take the
                                        512-thread pass. */
#define AGS_SORT_PERSISTENT 16       /* sort flag: the 256-thread digit passes launch only as many
                                        blocks as are resident at once, each taking partitions of
                                        the count on the device until none is left, instead of one
                                        block per partition of the capacity; same result, faster
                                        when the count is far below the capacity (the depth
                                        pre-sort of the visible Gaussian-views) */

/* Stable LSD radix sort of (keys, vals) by key bits [begin_bit, end_bit)
 * (Sec. 2.1 sorting stage): one global-histogram pass, then one single-pass
 * ("onesweep") scatter per digit of `digit_bits` (4..9) bits, with warp-level
 * match/ballot ranking and decoupled look-back between blocks.  The count is
 * read on the device from *d_num_pairs (clamped to capacity < AGS_MAX_PAIRS).
 * Keys already stably ordered by their bits below begin_bit stay so ordered
 * within equal [begin_bit, end_bit) fields: pairs emitted in depth order
 * need only the tile digits, with the same result as a sort of all bits.
 * flags: AGS_SORT_IDENTITY_VALUES, AGS_SORT_DISCARD_KEYS, AGS_SORT_RANK_OR, AGS_SORT_WIDE_BLOCK,
 * AGS_SORT_PERSISTENT (any other bit but AGS_SORT_TEST_STALL is invalid).  `keys` must be
 * 16-byte aligned when a digit pass runs (read 16 bytes at a time).
 * The sorted result lands in (keys, vals) when the number of digit passes is
 * even and in (keys_alt, vals_alt) when it is odd; *result_in_alt (host)
 * reports which.  If `ranges` is non-null it then receives, for each of
 * `num_ranges` tiles, [start, end) of that tile's pairs (uint32[num_ranges][2],
 * zero for empty tiles), the tile being key >> 32. */
ags_status ags_sort(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                    const int64_t* d_num_pairs, int64_t capacity, int32_t begin_bit,
                    int32_t end_bit, int32_t digit_bits, int32_t flags, uint32_t* ranges,
                    int64_t num_ranges, int32_t* result_in_alt, int64_t* d_status, void* ws,
                    size_t ws_bytes, void* stream);

/* ags_sort for 32-bit keys (end_bit <= 32): the depth pre-sort of depth_key
 * and the sort of the tile keys of ags_emit_tile_pairs.  Same arguments,
 * workspace (ags_sort_workspace_bytes), flags and results; the range index of
 * a key is the whole key.  `keys` must be 16-byte aligned when a digit pass
 * runs (it is read 16 bytes at a time), as for ags_sort. */
ags_status ags_sort32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                      const int64_t* d_num_pairs, int64_t capacity, int32_t begin_bit,
                      int32_t end_bit, int32_t digit_bits, int32_t flags, uint32_t* ranges,
                      int64_t num_ranges, int32_t* result_in_alt, int64_t* d_status, void* ws,
                      size_t ws_bytes, void* stream);

/* Sort of view-shifted tile keys (AGS_EMIT_VIEW_SHIFT): ags_sort32 over bits
 * [0, tile_bits) only, i.e. by tile, stable, so that the pairs of one tile keep
 * the emission order -- view by view, each in depth order; fewer key bits than
 * view * tiles_per_view + tile when the views outnumber the spare bits.  ranges
 * (nullable, [views * tiles_per_view][2]) are indexed by view * tiles_per_view +
 * tile, the view being the key's bits above tile_bits.  Same workspace, flags
 * and results as ags_sort32; tiles_per_view <= 2^tile_bits, views << tile_bits
 * <= 2^32. */
ags_status ags_sort_tiles(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                          const int64_t* d_num_pairs, int64_t capacity, int32_t tile_bits,
                          int32_t digit_bits, int32_t flags, uint32_t* ranges, int32_t views,
                          int32_t tiles_per_view, int32_t* result_in_alt, int64_t* d_status, void* ws,
                          size_t ws_bytes, void* stream);

/* Blending (Eq. 1, Eq. 2; Sec. 3.3 dual size).  One CTA per 16x16 tile of
 * each view; per pixel, front to back over the tile's sorted pairs:
 *   p = -(A dx^2 + C dy^2)/2 - B dx dy, skip if p > 0,
 *   alpha = min(alpha_max, opacity e^p), skip if alpha < tau,
 *   stop (without blending) when T (1 - alpha) < t_min,
 *   C += alpha T rgb, T *= 1 - alpha.
 * Always the original conic and tau, whatever the scale mode.
 * Outputs: image [views][3][H][W] = C + T bg; final_T [views][H][W] and
 * n_contrib [views][H][W] (1-based position in the tile list of the last
 * blended pair), both nullable (the backward needs them); max_T [views*n]
 * (nullable; zeroed by the caller) receives, per Gaussian, the largest T seen
 * before blending it (calibration, Sec. 3.4); stats (nullable uint64[3])
 * accumulates {evaluations of Eq. 1-2 as the method defines them -- each
 * pixel against the pairs of its tile's list up to the one at which it stops,
 * or the whole list --, blended pairs, pixel-pair slots the kernel actually
 * evaluated (its per-warp culling skips the pairs whose alpha >= tau ellipse
 * misses a warp's 8x16 block)}. */
ags_status ags_rasterize(const ags_projected* proj, int64_t n, const uint32_t* sorted_vals,
                         const uint32_t* ranges, const ags_camera* cams, int32_t views,
                         const ags_params* params, float* image, float* final_T,
                         uint32_t* n_contrib, float* max_T, uint64_t* stats,
                         int64_t* d_status, void* stream);

/* T_up look-up table (Sec. 3.4): for every Gaussian and view with
 * max_T > 0, bin its depth into lut_bins uniform intervals of
 * [0, lut_depth_max] (depths beyond go to the last bin) and take the maximum.
 * lut_out [lut_bins] fp32; bins no Gaussian reached are set to 1.0. */
ags_status ags_calibrate_lut(const float* max_T, const float* depth, int64_t count,
                             int32_t lut_bins, float lut_depth_max, float* lut_out,
                             void* stream);

/* Peripheral-score diagnostics (Sec. 3.1 Eq. 4, Sec. 3.2 Eq. 6-10).  Replays
 * the blend of ags_rasterize over the given pair lists -- normally those of a
 * PLAIN-mode preprocess, whose tiles cover the whole alpha >= tau region Eq. 4
 * sums over -- with its exact per-pixel decisions, and writes for every
 * Gaussian-view e (count = views*n), at its AdaGScale level Th_e from Eq. 10
 * (params->K and the T_up table, det Sigma2D from the splat record):
 *   scores[0][e]  Th_e (+inf where T_up = 0)
 *   scores[1][e]  Eq. 4: sum of alpha T over the pixels where e blends with alpha < Th_e
 *   scores[2][e]  Eq. 6: max T_e * sum of alpha over the same pixels
 *   scores[3][e]  Eq. 7: T_up(depth_e) * that sum
 *   scores[4][e]  Eq. 9: T_up(depth_e) 2 pi sqrt(det Sigma2D) (min(Th_e, opacity) - tau)
 *                 (alpha never exceeds the opacity; equals K where Th_e <= opacity)
 *   scores[5][e]  max T_e, the largest T before e over the pixels where it blends
 *   scores[6][e]  the sum of alpha of row 1's pixels
 * scores: fp32 [7][views*n], overwritten (culled Gaussian-views get zeros).
 * The sums are fp32 atomics (order-dependent in the last bits). */
ags_status ags_peripheral_scores(const ags_projected* proj, int64_t n, const uint32_t* sorted_vals,
                                 const uint32_t* ranges, const ags_camera* cams, int32_t views,
                                 const ags_params* params, float* scores, void* stream);

/* Contribution histogram (Sec. 2.2 Fig. 4a, Sec. 3.2 Fig. 5).  For every blend
 * of ags_rasterize over the given lists, its contribution under `rule`:
 *   0: alpha T (Eq. 3);  1: max_T[e] alpha (Eq. 6; max_T e.g. row 5 of
 *   ags_peripheral_scores);  2: T_up(depth_e) alpha (Eq. 7)
 * is counted in hist[bits(c) >> 16] (uint32 [32768], overwritten; positive
 * floats order as their bit patterns, so the bins are in contribution order;
 * a negative contribution counts in the last bin).  max_T is read only for
 * rule 1. */
#define AGS_CONTRIB_HIST_BINS 32768
ags_status ags_contribution_hist(const ags_projected* proj, int64_t n, const uint32_t* sorted_vals,
                                 const uint32_t* ranges, const ags_camera* cams, int32_t views,
                                 const ags_params* params, int32_t rule, const float* max_T,
                                 uint32_t* hist, void* stream);

/* Contribution-skip render (Sec. 2.2 Fig. 4a, Sec. 3.2 Fig. 5): the blends of
 * ags_rasterize, each skipped when its contribution under `rule` (as for
 * ags_contribution_hist) is below thr.  A skipped blend adds no colour and
 * does not occlude; the unskipped T still ranks (rule 0) and decides the stop,
 * so every rule and threshold acts on the same set of blends.  image
 * [views][3][H][W] = kept colour + (image transmittance) bg; counts (uint64[2],
 * accumulated: zero them first) += {blends, skipped}. */
ags_status ags_render_skip(const ags_projected* proj, int64_t n, const uint32_t* sorted_vals,
                           const uint32_t* ranges, const ags_camera* cams, int32_t views,
                           const ags_params* params, int32_t rule, const float* max_T, float thr,
                           float* image, uint64_t* counts, void* stream);

/* Storage order of the Gaussians (not in the paper).  The preprocess runs a
 * warp's 32 Gaussians through every view together; stored along a Morton
 * (Z-order) curve of their means, the Gaussians of a warp lie close together,
 * so the views that cull them (behind the camera, off the image) cull them
 * together and the projection work follows the visible Gaussians.  The order
 * is a stable sort (ags_sort32, AGS_SORT_IDENTITY_VALUES, bits [0, 30)) of the
 * codes below; rendering the permuted scene gives the same images (only
 * Gaussians of exactly equal depth in one tile, ordered by index, can swap).
 *
 * ags_morton_codes: codes[n] (uint32) = the 30-bit Morton code of each mean,
 * 10 bits per axis over the bounding box of the finite means (bit 3b+a holds
 * bit b of axis a); a mean that is not finite gets 0xffffffff.  Workspace:
 * ags_morton_workspace_bytes(), 4-byte aligned.
 * ags_gather_gaussians: every attribute array of the n Gaussians of `src`
 * (SH rows for sh_degree) permuted into the caller's arrays (same layouts):
 * dst[.][k] = src[.][perm[k]]; perm is a permutation of 0..n-1 (an entry >= n
 * leaves its destination column unwritten). */
size_t ags_morton_workspace_bytes(void);
ags_status ags_morton_codes(const ags_gaussians* g, uint32_t* codes, void* ws, size_t ws_bytes, void* stream);
ags_status ags_gather_gaussians(const ags_gaussians* src, const uint32_t* perm, int32_t sh_degree, float* mean,
                                float* log_scale, float* quat, float* opacity_logit, float* sh, void* stream);

/* Scratch bytes needed by ags_rasterize_backward. */
size_t ags_backward_workspace_bytes(int64_t n, int32_t views);

/* Backward of ags_rasterize and ags_preprocess with the pair lists held
 * fixed (not in the paper).  dL_dimage [views][3][H][W].  The blend adjoint
 * replays each pixel from its last blended pair backwards, recovering T by
 * division by (1 - alpha); the preprocess adjoint chains through the EWA
 * projection, the covariance, the quaternion normalisation, the sigmoid and
 * the SH basis, summing over views.  Clamped quantities (alpha at
 * alpha_max, colour at 0, the EWA frustum clamp) pass no gradient; Th and
 * the footprint pass none either.  Outputs are overwritten:
 * g_mean [3][n], g_log_scale [3][n], g_quat [4][n], g_opacity_logit [n],
 * g_sh [(sh_degree+1)^2][3][n]. */
ags_status ags_rasterize_backward(const ags_gaussians* g, const ags_camera* cams, int32_t views,
                                  const ags_params* params, const ags_projected* proj,
                                  const uint32_t* sorted_vals, const uint32_t* ranges,
                                  const float* final_T, const uint32_t* n_contrib,
                                  const float* dL_dimage, float* g_mean, float* g_log_scale,
                                  float* g_quat, float* g_opacity_logit, float* g_sh,
                                  int64_t* d_status, void* ws, size_t ws_bytes, void* stream);

/* Library version string (static). */
const char* ags_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AGS_H */
