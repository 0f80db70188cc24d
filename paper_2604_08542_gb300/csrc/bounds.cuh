// Bounds checking (a build with -DSCAL3R_DEBUG_BOUNDS; compiled out otherwise).
//
// Each checked call registers the byte ranges of the tensors it was given and
// of its workspace regions.  Every plain global load or store that a checked
// kernel makes goes through in_bounds(): the access must lie entirely inside
// one registered range.  An access that does not is skipped (a load reads
// zeros) and the call's status word records SCAL3R_ERR_BOUNDS.  This is
// stricter than an allocation-level checker: a caching allocator's block
// holds many tensors, a registered range only the one.
//
// The table lives in each translation unit's constant memory.  The host
// uploads it on the call's stream before the call's kernels and uploads an
// empty table (checking off) after them, so no table outlives its call.
// TMA loads and stores are not routed through it: the tensor maps bound them
// in hardware.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/scal3r_ttt.h"

namespace scal3r {

constexpr int kMaxBoundsRanges = 24;

struct BoundsTable {
  int32_t n;        // registered ranges; 0 = checking off
  int32_t pad;
  int* status;      // the handle's status word
  uint64_t lo[kMaxBoundsRanges], hi[kMaxBoundsRanges];   // [lo, hi) in bytes
};

#ifdef SCAL3R_DEBUG_BOUNDS
static __constant__ BoundsTable c_bounds;

__device__ __forceinline__ bool in_bounds(const void* p, uint32_t bytes) {
  if (c_bounds.n == 0) return true;
  const uint64_t a = reinterpret_cast<uint64_t>(p), b = a + bytes;
  for (int i = 0; i < c_bounds.n; ++i)
    if (a >= c_bounds.lo[i] && b <= c_bounds.hi[i]) return true;
  atomicCAS(c_bounds.status, 0, SCAL3R_ERR_BOUNDS);
  return false;
}

inline cudaError_t upload_bounds_table(const BoundsTable& t, cudaStream_t st) {
  return cudaMemcpyToSymbolAsync(c_bounds, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
}
#else
__device__ __forceinline__ constexpr bool in_bounds(const void*, uint32_t) { return true; }
#endif

// Checked plain accesses: a skipped load reads zero.  In the ordinary build
// they are macros for the plain access itself, so that the compiler sees the
// same expression (and the same aliasing) as unchecked code.
#ifdef SCAL3R_DEBUG_BOUNDS
template <typename T>
__device__ __forceinline__ T ld_chk(const T* p) {
  return in_bounds(p, sizeof(T)) ? *p : T{};
}
template <typename T>
__device__ __forceinline__ void st_chk(T* p, const T& v) {
  if (in_bounds(p, sizeof(T))) *p = v;
}
__device__ __forceinline__ float4 ldg_chk(const float4* p) {
  return in_bounds(p, sizeof(float4)) ? __ldg(p) : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ float ldg_chk(const float* p) { return in_bounds(p, sizeof(float)) ? __ldg(p) : 0.f; }
#else
#define ld_chk(p) (*(p))
#define st_chk(p, v) (*(p) = (v))
#define ldg_chk(p) __ldg(p)
#endif

}  // namespace scal3r
