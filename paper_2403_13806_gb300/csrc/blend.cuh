// Blend-ready Gaussian records and the per-pixel-pair arithmetic shared by the forward and
// backward blend kernels.
//
// Each thread owns pixels of one column, taken two at a time: the two pixels of a pair share
// the horizontal offset dx and differ in dy, so the quadratic form, the opacity product,
// the transmittance update and the colour sums run as packed two-lane FP32 instructions
// (__ffma2_rn / __fmul2_rn / __fadd2_rn, one rounding per lane, identical to the scalar
// operations).  Both kernels evaluate a record with the same explicitly rounded operations
// (no compiler contraction), so the backward pass replays every skip decision of the
// forward pass bit for bit.
#pragma once

#include "rs_common.cuh"

namespace rs {

// Record of one Gaussian in shared memory.  Every value a pixel pair uses on both lanes is
// stored twice so that a packed instruction reads it as one register pair.  A, B, C are the
// conic (a, b, c) times (-log2(e)/2, -log2(e), -log2(e)/2), so that
// p2 = A dx^2 + B dx dy + C dy^2 = log2(e) * power; cut = log2(1/(255 o)) - 1e-3: below it
// alpha = o 2^p2 < 1/255 for sure, and only pairs above it take the exact test.
//
// The clamp alpha = min(0.99, o 2^p2) is applied as alpha = 0.99 s with the saturated product
// s = sat(o' 2^p2), o' = o / 0.99 (the same function of o and p2; a saturating multiply runs
// on the FMA pipe where a minimum would take the ALU pipe).  The record holds o'; the
// forward pass composites s T with colours pre-scaled by 0.99, so it never forms alpha.
struct BlendRec {
  float4 xy;    // (x, x, y, y)
  float4 ab;    // (A, A, B, B)
  float4 co;    // (C, C, o', o')
  float4 rg;    // (r, r, g, g), times 0.99 in the forward pass
  float4 bc;    // (b, b, cut, cut), b times 0.99 in the forward pass
};

constexpr float kInvAlphaMax = 1.0f / kAlphaMax;
// alpha >= 1/255 as a test on s = alpha / 0.99
constexpr float kSMin = (float)(1.0 / (255.0 * 0.99));

// FWD: colours pre-scaled by 0.99 (the forward pass's weight is s T = alpha T / 0.99).
template <bool FWD>
__device__ __forceinline__ void stage_record(const float2* xy, const float4* conic_o, const float4* rgb_d,
                                             uint32_t item, BlendRec& r) {
  const float2 p = __ldg(xy + item);
  const float4 co = __ldg(conic_o + item);
  const float4 cd = __ldg(rgb_d + item);
  const float A = __fmul_rn(-0.5f * kLog2e, co.x), B = __fmul_rn(-kLog2e, co.y), C = __fmul_rn(-0.5f * kLog2e, co.z);
  const float cut = __fsub_rn(log2f(__fdiv_rn(kAlphaMin, co.w)), 1e-3f);
  const float os = __fmul_rn(co.w, kInvAlphaMax);
  const float cr = FWD ? __fmul_rn(kAlphaMax, cd.x) : cd.x;
  const float cg = FWD ? __fmul_rn(kAlphaMax, cd.y) : cd.y;
  const float cb = FWD ? __fmul_rn(kAlphaMax, cd.z) : cd.z;
  r.xy = make_float4(p.x, p.x, p.y, p.y);
  r.ab = make_float4(A, A, B, B);
  r.co = make_float4(C, C, os, os);
  r.rg = make_float4(cr, cr, cg, cg);
  r.bc = make_float4(cb, cb, cut, cut);
}

__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }

// 2^x by the hardware approximation (ex2.approx.ftz: relative error below 2^-22 for the
// arguments whose result decides anything here, x in [-8.1, 0] up to rounding, where the
// results are normal numbers; far below that the result flushes to 0).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// max(a, b, c) in one instruction; a NaN operand is ignored unless all three are NaN.
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// The largest p2 of a thread's pixels, NaN (a done or not-yet-live pixel) ignored: it is at
// least the cut exactly when some pixel's p2 is, so the warp-level support pre-test takes one
// comparison per thread instead of one per pixel.
template <int NP>
__device__ __forceinline__ float max_p2(const float2 (&p2)[NP]) {
  float m = fmaxf(p2[0].x, p2[0].y);
#pragma unroll
  for (int q = 1; q < NP; ++q) m = max3f(m, p2[q].x, p2[q].y);
  return m;
}

// (x - u, x - u) for the thread's column u (nu = (-u, -u)).
__device__ __forceinline__ float2 pair_dx(const BlendRec& r, float2 nu) { return __fadd2_rn(lo2(r.xy), nu); }

// (y - v0, y - v1) for a pixel pair in rows v0, v1 (nv = (-v0, -v1)).
__device__ __forceinline__ float2 pair_dy(const BlendRec& r, float2 nv) { return __fadd2_rn(hi2(r.xy), nv); }

// A thread's pixels share one column, hence one dx per record: the terms A dx^2 and B dx of
// p2 = A dx^2 + dy (B dx + C dy) are computed once per record for all its pixel pairs.
struct ColTerms {
  float2 adx2;   // (A dx^2, A dx^2)
  float2 bdx;    // (B dx, B dx)
};

__device__ __forceinline__ ColTerms col_terms(const BlendRec& r, float2 dx) {
  ColTerms c;
  c.adx2 = __fmul2_rn(__fmul2_rn(lo2(r.ab), dx), dx);
  c.bdx = __fmul2_rn(hi2(r.ab), dx);
  return c;
}

// p2 = log2(e) * power for both pixels of a pair: A dx^2 + dy (B dx + C dy).
__device__ __forceinline__ float2 pair_power(const BlendRec& r, const ColTerms& c, float2 dy) {
  return __ffma2_rn(dy, __ffma2_rn(lo2(r.co), dy, c.bdx), c.adx2);
}

// x y rounded and clamped to [0, 1] (a NaN product gives 0), on the FMA pipe.
__device__ __forceinline__ float mul_sat(float x, float y) {
  float r;
  asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(y));
  return r;
}

// Per-pixel outcome of the blend rule's tests on one record.
//
// The rule skips pairs with power > 0 or alpha < 1/255.  Sigma' is positive definite (the
// 2D covariance plus eps I), so power <= 0 holds exactly; a positive FP32 p2 is a rounding
// artefact of a power near 0 (at the centre, or along the long axis of a needle-thin
// Gaussian, where the rounding of the three terms exceeds the true value) and is composited
// at its rounded value, which lies closer to the exact alpha than skipping the pair would.
// The test reduces to alpha >= 1/255.
struct PairAlpha {
  float2 ex;      // min(2^p2, 1) (CLAMP) or 2^p2
  float2 s;       // sat(o' 2^p2) = alpha / 0.99; s = 1 exactly where the 0.99 clamp is active
  bool in0, in1;  // alpha >= 1/255
};

// CLAMP: keep ex finite for every pair, NaN (gated) p2 included (the backward multiplies it;
// min(NaN, 1) = 1); the forward only uses s, where sat() already maps a large or NaN product
// to 1 or 0.  Both passes take s from the unclamped 2^p2, so they make the same decisions.
template <bool CLAMP = true>
__device__ __forceinline__ PairAlpha pair_alpha(const BlendRec& r, float2 p2) {
  PairAlpha a;
  const float2 e = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
  a.ex = CLAMP ? make_float2(fminf(e.x, 1.f), fminf(e.y, 1.f)) : e;
  a.s = make_float2(mul_sat(r.co.z, e.x), mul_sat(r.co.w, e.y));
  // alpha >= 1/255 implies p2 >= cut (the cut's 1e-3 margin exceeds the rounding of
  // 2^p2, o' 2^p2 and the cut itself), so the exact test needs no cut comparison; the cut
  // only serves the warp-level pre-test of the kernels
  a.in0 = a.s.x >= kSMin;
  a.in1 = a.s.y >= kSMin;
  return a;
}

// The test s >= kSMin as an exact factor 1 or 0 on the FMA pipe: sat(s 2^31 + (1 - kSMin 2^31)).
// kSMin lies in [2^-8, 2^-7), where floats are spaced 2^-31, so kSMin 2^31 is an integer below
// 2^24 (the constant is exact) and every s < kSMin is at most kSMin - 2^-31 (smaller s are
// below 2^-8, further still): the fused product-sum is <= 0 exactly when s < kSMin and >= 1
// otherwise, which rounding preserves.  s is never NaN (it comes from sat()).
constexpr float kInC = 1.0f - kSMin * 0x1p31f;
static_assert(kSMin >= 0x1p-8f && kSMin < 0x1p-7f, "spacing of floats near kSMin");
__device__ __forceinline__ float in_factor(float s) {
  float r;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(s), "f"(0x1p31f), "f"(kInC));
  return r;
}

// 1 - alpha = 1 - 0.99 s on both lanes (one rounding); the forward and backward passes both
// form it this way, so the backward divides by the forward's factors exactly.
__device__ __forceinline__ float2 one_minus_alpha(float2 s) {
  return __ffma2_rn(s, make_float2(-kAlphaMax, -kAlphaMax), make_float2(1.f, 1.f));
}

}  // namespace rs
