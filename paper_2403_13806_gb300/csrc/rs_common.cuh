// Shared device helpers of the GB300 splatting library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "radsplat.h"

namespace rs {

// Compositing constants: alpha clamp, skip threshold and early-stop transmittance of
// the 3DGS rasterizer the paper renders with (Sec. 3.2, Sec. 3.4 "default rasterization").
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;

constexpr int kNumSMs = 152;   // GB300: 2 dies x 76 SMs (grid sizing only; not a correctness input)

// 1/x by the hardware approximation (rcp.approx.ftz: within 1 ulp for normal x).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// A view found by a binary search on a sorted int64 key (item_base or tile_base).
__device__ __forceinline__ int find_view_by_item(const rs_view* views, int n_views, int64_t item) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (views[mid].item_base <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_view_by_tile(const rs_view* views, int n_views, int tile) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Records the first device-side error code (never traps).
__device__ __forceinline__ void set_status(rs_device_status* st, int code) {
  if (st) atomicCAS(&st->code, 0, code);
}

inline rs_status launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

template <typename T>
inline bool aligned(const void* p, size_t a) {
  return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Threads of a blend CTA: one warp per tile (eight pixels of a column per thread, two for
// 8x8 tiles), in the forward and the backward pass alike.
inline int blend_threads(int, int) { return 32; }

// rs_config.batch (records staged per blend batch): 0 (default) or 1, 2 or 4 per thread.
inline bool blend_batch_ok(int tile_w, int tile_h, int batch) {
  if (batch == 0) return true;
  const int nt = blend_threads(tile_w, tile_h);
  if (batch < 0 || batch % nt != 0) return false;
  const int m = batch / nt;
  return m == 1 || m == 2 || m == 4;
}

}  // namespace rs
