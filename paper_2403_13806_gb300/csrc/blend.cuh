// Blend-ready Gaussian records shared by the forward and backward blend kernels.
//
// Both kernels stage and evaluate a record with the same explicitly rounded operations
// (no compiler contraction), so the backward pass replays every skip decision of the
// forward pass bit for bit.
#pragma once

#include "rs_common.cuh"

namespace rs {

// Record of one Gaussian: g = (x, y, A, B), g2 = (C, cut, o, 0), col = (r, g, b, 0) with
// A, B, C = conic (a, b, c) times (-log2(e)/2, -log2(e), -log2(e)/2), so that
// p2 = A dx^2 + B dx dy + C dy^2 = log2(e) * power, and cut = log2(1/(255 o)) - 1e-3: below
// it alpha = o 2^p2 < 1/255 for sure, and only pairs above it take the exact test.
__device__ __forceinline__ void stage_record(const float2* xy, const float4* conic_o, const float4* rgb_d,
                                             uint32_t item, float4& g, float4& g2, float4& col) {
  const float2 p = __ldg(xy + item);
  const float4 co = __ldg(conic_o + item);
  const float4 cd = __ldg(rgb_d + item);
  g = make_float4(p.x, p.y, __fmul_rn(-0.5f * kLog2e, co.x), __fmul_rn(-kLog2e, co.y));
  g2 = make_float4(__fmul_rn(-0.5f * kLog2e, co.z), __fsub_rn(log2f(__fdiv_rn(kAlphaMin, co.w)), 1e-3f), co.w, 0.f);
  col = make_float4(cd.x, cd.y, cd.z, 0.f);
}

// p2 = log2(e) * power at pixel (fu, fv), with dx = x - u, dy = y - v.
__device__ __forceinline__ float blend_power(const float4& g, const float4& g2, float fu, float fv) {
  const float dx = __fsub_rn(g.x, fu), dy = __fsub_rn(g.y, fv);
  return __fmaf_rn(dx, __fmaf_rn(g.z, dx, __fmul_rn(g.w, dy)), __fmul_rn(__fmul_rn(g2.x, dy), dy));
}

}  // namespace rs
