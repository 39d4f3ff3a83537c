// ags_internal.cuh -- device-side helpers shared by the CUDA translation units
// of libags (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ags.h"

namespace ags {

constexpr int kTile = AGS_TILE;
constexpr int kSplatFloats = 12;            // u v A B | C opacity r g | b Th Sxx Syy
constexpr uint8_t kFlagCulled = 0x80;
constexpr uint64_t kWaitLimitNs = 200ull * 1000ull * 1000ull;   // bounded spin: 200 ms
constexpr uint64_t kTestWaitLimitNs = 2ull * 1000ull * 1000ull;  // with a test stall: 2 ms

// Look-back wait settings of one launch: the partition that never publishes
// its flags (test stall; 0xffffffff: none) and the spin limit.
struct WaitHook {
  uint32_t withhold;
  uint64_t limit_ns;
};
inline WaitHook wait_hook(bool test_stall) {
  return test_stall ? WaitHook{1u, kTestWaitLimitNs} : WaitHook{0xffffffffu, kWaitLimitNs};
}

// Stage ids reported as the detail word of AGS_ERR_TIMEOUT.
enum : int64_t { kStageEmit = 1, kStageSort = 2, kStageVisible = 3 };

// ---------------------------------------------------------------------------
// Camera and parameter blocks passed by value (__grid_constant__).
// ---------------------------------------------------------------------------
struct DevCam {
  float R[9];
  float t[3];
  float campos[3];
  float fx, fy, cx, cy, near_z;
  float limx, limy;          // 1.3 * tan(fov/2) per axis
  int W, H, gx, gy;
};

struct CamBatch {
  DevCam c[AGS_MAX_VIEWS];
};

struct DevParams {
  int scale_mode, sh_degree, lut_bins, tile_test, blend_flags;
  float K, tau, t_min, alpha_max, lut_scale;   // lut_scale = lut_bins / lut_depth_max
  float lut[AGS_MAX_LUT_BINS];
  float bg[3];
};

// ---------------------------------------------------------------------------
// Device status block: {code, detail, non-finite count, reserved}.
// The first error code wins; a capacity overflow keeps the largest need.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int64_t* st, int64_t code, int64_t detail) {
  unsigned long long* s = reinterpret_cast<unsigned long long*>(st);
  atomicCAS(s, 0ull, (unsigned long long)code);
  if (code == AGS_ERR_CAPACITY)
    atomicMax(reinterpret_cast<long long*>(st + 1), (long long)detail);
  else
    atomicCAS(s + 1, 0ull, (unsigned long long)detail);
}

// Index checks of AGS_DEBUG builds, on the indices that come from the inputs
// (pair values, tile ranges, emission order entries): a failed check records
// AGS_ERR_BOUNDS with its id as detail, sets bit (1 << id) in word 3 of the
// status block, and returns false so that the caller skips the access.  In
// release builds AGS_DCHECK is the constant true and the checks compile away.
__device__ __forceinline__ bool debug_check(bool ok, int64_t* st, int id) {
  if (!ok) {
    set_status(st, AGS_ERR_BOUNDS, id);
    atomicOr(reinterpret_cast<unsigned long long*>(st + 3), 1ull << id);
  }
  return ok;
}
#ifdef AGS_DEBUG
#define AGS_DCHECK(cond, st, id) (::ags::debug_check((cond), (st), (id)))
#else
#define AGS_DCHECK(cond, st, id) true
#endif

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace ags

// Host-side helpers (defined in api.cu).
namespace ags {
ags_status build_cams(const ags_camera* cams, int32_t views, CamBatch* out);
ags_status build_params(const ags_params* p, DevParams* out);
ags_status launch_status(cudaError_t e);
}  // namespace ags
