// Access to one Gaussian's parameters by row: means (rows 0-2), log-scales (3-5),
// quaternion w, x, y, z (6-9), opacity logit (10), then SH coefficient k, channel c at row
// 11 + 3 k + c.  Either straight from the structure-of-arrays inputs, or from a block of
// columns a CTA has staged in shared memory (stage_params: one column per thread,
// asynchronous 4-byte copies, every load of the block in flight at once and no registers
// held while they land).
#pragma once

#include <stdint.h>

#include "radsplat.h"

namespace rs {

template <int D>
struct ParamRows {
  static constexpr int value = 11 + 3 * (D + 1) * (D + 1);
};

struct GlobalParams {
  const rs_gaussians* g;
  int64_t gid;
  __device__ __forceinline__ float operator()(int i) const {
    const int64_t N = g->n;
    const float* base = i < 3 ? g->means + (int64_t)i * N
                      : i < 6 ? g->log_scales + (int64_t)(i - 3) * N
                      : i < 10 ? g->quats + (int64_t)(i - 6) * N
                      : i < 11 ? g->opacity_logit
                               : g->sh + (int64_t)(i - 11) * N;
    return __ldg(base + gid);
  }
};

// All rows of one Gaussian loaded into registers at once (every load in flight together).
template <int D>
struct RegParams {
  float p[ParamRows<D>::value];
  __device__ __forceinline__ RegParams(const GlobalParams& src) {
#pragma unroll
    for (int i = 0; i < ParamRows<D>::value; ++i) p[i] = src(i);
  }
  __device__ __forceinline__ float operator()(int i) const { return p[i]; }
};

struct SmemParams {
  const float* col;   // row i of the thread's column at col[i * stride]
  int stride;
  __device__ __forceinline__ float operator()(int i) const { return col[i * stride]; }
};

// Copies the parameter rows of Gaussian gid into column `col` (row stride `stride` floats)
// of a shared-memory block and waits for the thread's own copies.
template <int D>
__device__ __forceinline__ void stage_params(const rs_gaussians& g, int64_t gid, float* col, int stride) {
  constexpr int NC = (D + 1) * (D + 1);
  const int64_t N = g.n;
  const float* rows[5] = {g.means, g.log_scales, g.quats, g.opacity_logit, g.sh};
  const int first[5] = {0, 3, 6, 10, 11};
  const int count[5] = {3, 3, 4, 1, 3 * NC};
#pragma unroll
  for (int r = 0; r < 5; ++r) {
#pragma unroll
    for (int k = 0; k < count[r]; ++k) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(col + (first[r] + k) * stride);
      const float* src = rows[r] + (int64_t)k * N + gid;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace rs
