// The optimisation step around the hot path (Sec. 3.2, Sec. 3.3):
//
// rs_adam_step -- one Adam step (Kingma & Ba, Algorithm 1) over up to eight parameter
//   arrays with their own learning rates, in one launch: m <- b1 m + (1 - b1) g,
//   v <- b2 v + (1 - b2) g^2, p <- p - lr (m / bc1) / (sqrt(v / bc2) + eps) with
//   bc = 1 - b^t.  Every element is read once (p, g, m, v) and written once (p, m, v):
//   28 bytes, HBM-bound.  Each CTA owns a contiguous run of one group (CTAs are dealt to
//   the groups in proportion to their sizes on the host, so no thread searches for its
//   group); threads take four consecutive elements (16-byte loads when all four arrays of
//   the group are 16-byte aligned), two such units in flight per thread.
// rs_gather_columns -- the compaction after pruning: for every structure-of-arrays
//   parameter (and optimiser moment) dst[r][k] = src[r][idx[k]] for k < count, count and
//   idx being the device outputs of rs_filter (the survivors, ascending).  One thread per
//   surviving column k walks every row of every array, so idx is read once; the stores of
//   a warp are contiguous and its loads follow the ascending indices.
#include <math.h>

#include "profile.cuh"
#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {

constexpr int kMaxAdamGroups = 8;
constexpr int kMaxGather = 16;

struct AdamArgs {
  float* p[kMaxAdamGroups];
  const float* g[kMaxAdamGroups];
  float* m[kMaxAdamGroups];
  float* v[kMaxAdamGroups];
  int64_t n[kMaxAdamGroups];
  int32_t cta0[kMaxAdamGroups + 1];    // first CTA of each group
  float lr[kMaxAdamGroups];
  int32_t vec[kMaxAdamGroups];         // 1: 16-byte loads and stores
  int32_t n_groups;
  float b1, b2, eps, ibc1, ibc2;   // ibc = 1 / (1 - b^t), rounded once on the host
};

// (the bias corrections multiply by host-rounded reciprocals and the step's ratio uses the
// fast division: within a few ulps of the correctly rounded operations, far inside what
// FP32 parameters resolve)
__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float lr, const AdamArgs& a) {
  m = __fmaf_rn(a.b1, m, __fmul_rn(1.f - a.b1, g));
  v = __fmaf_rn(a.b2, v, __fmul_rn(__fmul_rn(1.f - a.b2, g), g));
  const float mhat = __fmul_rn(m, a.ibc1);
  const float vhat = __fmul_rn(v, a.ibc2);
  p = __fsub_rn(p, __fdividef(__fmul_rn(lr, mhat), __fadd_rn(__fsqrt_rn(vhat), a.eps)));
}

// One 4-element unit (16-byte accesses when vec) at element e of group gi.
__device__ __forceinline__ void adam_unit(const AdamArgs& a, int gi, int64_t e) {
  const int64_t n = a.n[gi];
  const float lr = a.lr[gi];
  if (a.vec[gi] && e + 4 <= n) {
    float4 p = *reinterpret_cast<const float4*>(a.p[gi] + e);
    const float4 g = __ldcs(reinterpret_cast<const float4*>(a.g[gi] + e));
    float4 m = *reinterpret_cast<const float4*>(a.m[gi] + e);
    float4 v = *reinterpret_cast<const float4*>(a.v[gi] + e);
    adam_one(p.x, g.x, m.x, v.x, lr, a);
    adam_one(p.y, g.y, m.y, v.y, lr, a);
    adam_one(p.z, g.z, m.z, v.z, lr, a);
    adam_one(p.w, g.w, m.w, v.w, lr, a);
    *reinterpret_cast<float4*>(a.p[gi] + e) = p;
    *reinterpret_cast<float4*>(a.m[gi] + e) = m;
    *reinterpret_cast<float4*>(a.v[gi] + e) = v;
  } else {
    for (int64_t k = e; k < e + 4 && k < n; ++k) {
      float p = a.p[gi][k], m = a.m[gi][k], v = a.v[gi][k];
      adam_one(p, a.g[gi][k], m, v, lr, a);
      a.p[gi][k] = p;
      a.m[gi][k] = m;
      a.v[gi][k] = v;
    }
  }
}

__global__ void __launch_bounds__(256) k_adam(AdamArgs a) {
  int gi = 0;   // the CTA's group (uniform)
  while (gi + 1 < a.n_groups && (int)blockIdx.x >= a.cta0[gi + 1]) ++gi;
  const int64_t ctas = a.cta0[gi + 1] - a.cta0[gi];
  const int64_t units = (a.n[gi] + 3) / 4;
  const int64_t stride = ctas * 256;
  const int64_t n = a.n[gi];
  const float lr = a.lr[gi];
  // two units per thread and round: all eight 16-byte loads are issued before any store
  for (int64_t u = (int64_t)(blockIdx.x - a.cta0[gi]) * 256 + threadIdx.x; u < units; u += 2 * stride) {
    const int64_t e1 = 4 * u, e2 = 4 * (u + stride);
    if (a.vec[gi] && e2 + 4 <= n) {
      float4 p[2], m[2], v[2], g[2];
      const int64_t e[2] = {e1, e2};
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        p[k] = *reinterpret_cast<const float4*>(a.p[gi] + e[k]);
        g[k] = __ldcs(reinterpret_cast<const float4*>(a.g[gi] + e[k]));
        m[k] = *reinterpret_cast<const float4*>(a.m[gi] + e[k]);
        v[k] = *reinterpret_cast<const float4*>(a.v[gi] + e[k]);
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        adam_one(p[k].x, g[k].x, m[k].x, v[k].x, lr, a);
        adam_one(p[k].y, g[k].y, m[k].y, v[k].y, lr, a);
        adam_one(p[k].z, g[k].z, m[k].z, v[k].z, lr, a);
        adam_one(p[k].w, g[k].w, m[k].w, v[k].w, lr, a);
        *reinterpret_cast<float4*>(a.p[gi] + e[k]) = p[k];
        *reinterpret_cast<float4*>(a.m[gi] + e[k]) = m[k];
        *reinterpret_cast<float4*>(a.v[gi] + e[k]) = v[k];
      }
    } else {
      adam_unit(a, gi, e1);
      if (u + stride < units) adam_unit(a, gi, e2);
    }
  }
}

struct GatherArgs {
  const float* src[kMaxGather];
  float* dst[kMaxGather];
  int64_t rows[kMaxGather];
  int64_t src_stride[kMaxGather];
  int64_t dst_stride[kMaxGather];
  int32_t n_desc;
};

__global__ void __launch_bounds__(256) k_gather_columns(GatherArgs a, const uint32_t* __restrict__ idx,
                                                        const uint32_t* __restrict__ count, int64_t max_count) {
  const int64_t cnt = min((int64_t)*count, max_count);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx[k];
    for (int d = 0; d < a.n_desc; ++d) {
      const float* s = a.src[d] + i;
      float* o = a.dst[d] + k;
      const int64_t rows = a.rows[d], ss = a.src_stride[d], ds = a.dst_stride[d];
      // eight rows' loads in flight before their stores (source and destination may not
      // be told apart by the compiler, so it would not reorder them itself)
      int64_t r = 0;
      for (; r + 8 <= rows; r += 8) {
        float t[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = __ldg(s + (r + j) * ss);
#pragma unroll
        for (int j = 0; j < 8; ++j) o[(r + j) * ds] = t[j];
      }
      for (; r < rows; ++r) o[r * ds] = __ldg(s + r * ss);
    }
  }
}

// The inverse placement: dst column idx[k] of every row receives src column k.
__global__ void __launch_bounds__(256) k_scatter_columns(GatherArgs a, const uint32_t* __restrict__ idx,
                                                         const uint32_t* __restrict__ count, int64_t max_count) {
  const int64_t cnt = min((int64_t)*count, max_count);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx[k];
    for (int d = 0; d < a.n_desc; ++d) {
      const float* s = a.src[d] + k;
      float* o = a.dst[d] + i;
      const int64_t rows = a.rows[d], ss = a.src_stride[d], ds = a.dst_stride[d];
      int64_t r = 0;
      for (; r + 8 <= rows; r += 8) {
        float t[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = __ldg(s + (r + j) * ss);
#pragma unroll
        for (int j = 0; j < 8; ++j) o[(r + j) * ds] = t[j];
      }
      for (; r < rows; ++r) o[r * ds] = __ldg(s + r * ss);
    }
  }
}

// out[i] = 1 where some row of column i is non-zero (the Gaussians a gradient reaches).
__global__ void __launch_bounds__(256) k_touched_columns(const float* __restrict__ src, int64_t rows, int64_t n,
                                                         float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    bool any = false;
    for (int64_t r = 0; r < rows && !any; ++r) any = __ldcs(src + r * n + i) != 0.f;
    out[i] = any ? 1.f : 0.f;
  }
}

}  // namespace rs

using namespace rs;

extern "C" rs_status rs_adam_step(const rs_adam_group* groups, int32_t n_groups, float beta1, float beta2, float eps,
                                  int32_t step, void* stream) {
  if (!groups || n_groups < 1 || n_groups > kMaxAdamGroups || step < 1) return RS_ERR_INVALID_ARG;
  if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f)) return RS_ERR_INVALID_ARG;
  AdamArgs a{};
  a.n_groups = n_groups;
  a.b1 = beta1;
  a.b2 = beta2;
  a.eps = eps;
  a.ibc1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)step)));
  a.ibc2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)step)));
  int64_t units = 0;
  for (int32_t i = 0; i < n_groups; ++i) {
    const rs_adam_group& g = groups[i];
    if (g.n < 0 || (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v))) return RS_ERR_INVALID_ARG;
    a.p[i] = g.param;
    a.g[i] = g.grad;
    a.m[i] = g.m;
    a.v[i] = g.v;
    a.n[i] = g.n;
    a.lr[i] = g.lr;
    a.vec[i] = aligned<float4>(g.param, 16) && aligned<float4>(g.grad, 16) && aligned<float4>(g.m, 16) &&
               aligned<float4>(g.v, 16);
    units += (g.n + 3) / 4;
  }
  if (units == 0) return RS_OK;
  // CTAs dealt to the groups in proportion to their units (at least one each, at most one
  // per 256 units), about 16 per SM in total
  const int64_t budget = 16 * kNumSMs;
  int32_t total = 0;
  for (int32_t i = 0; i < n_groups; ++i) {
    a.cta0[i] = total;
    const int64_t u = (groups[i].n + 3) / 4;
    int64_t c = (u * budget + units - 1) / units;
    const int64_t cmax = (u + 255) / 256;
    c = c < 1 ? 1 : (c > cmax ? (cmax > 0 ? cmax : 1) : c);
    total += (int32_t)c;
  }
  a.cta0[n_groups] = total;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  prof::Scope ps("k_adam", s);
  k_adam<<<(unsigned)total, 256, 0, s>>>(a);
  return launch_status();
}

extern "C" rs_status rs_gather_columns(const rs_gather_desc* descs, int32_t n_desc, const uint32_t* idx,
                                       const uint32_t* count, int64_t max_count, void* stream) {
  if (!descs || n_desc < 1 || n_desc > kMaxGather || !idx || !count || max_count < 0) return RS_ERR_INVALID_ARG;
  GatherArgs a{};
  a.n_desc = n_desc;
  for (int32_t d = 0; d < n_desc; ++d) {
    const rs_gather_desc& g = descs[d];
    if (!g.src || !g.dst || g.rows < 0 || g.dst_stride < max_count || g.src_stride < 0) return RS_ERR_INVALID_ARG;
    a.src[d] = g.src;
    a.dst[d] = g.dst;
    a.rows[d] = g.rows;
    a.src_stride[d] = g.src_stride;
    a.dst_stride[d] = g.dst_stride;
  }
  if (max_count == 0) return RS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t blocks = (max_count + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 8 * kNumSMs ? blocks : 8 * kNumSMs);
  prof::Scope ps("k_gather_columns", s);
  k_gather_columns<<<grid, 256, 0, s>>>(a, idx, count, max_count);
  return launch_status();
}

extern "C" rs_status rs_scatter_columns(const rs_gather_desc* descs, int32_t n_desc, const uint32_t* idx,
                                        const uint32_t* count, int64_t max_count, void* stream) {
  if (!descs || n_desc < 1 || n_desc > kMaxGather || !idx || !count || max_count < 0) return RS_ERR_INVALID_ARG;
  GatherArgs a{};
  a.n_desc = n_desc;
  for (int32_t d = 0; d < n_desc; ++d) {
    const rs_gather_desc& g = descs[d];
    if (!g.src || !g.dst || g.rows < 0 || g.src_stride < max_count || g.dst_stride < 0) return RS_ERR_INVALID_ARG;
    a.src[d] = g.src;
    a.dst[d] = g.dst;
    a.rows[d] = g.rows;
    a.src_stride[d] = g.src_stride;
    a.dst_stride[d] = g.dst_stride;
  }
  if (max_count == 0) return RS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t blocks = (max_count + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 8 * kNumSMs ? blocks : 8 * kNumSMs);
  prof::Scope ps("k_scatter_columns", s);
  k_scatter_columns<<<grid, 256, 0, s>>>(a, idx, count, max_count);
  return launch_status();
}

extern "C" rs_status rs_touched_columns(const float* src, int64_t rows, int64_t n, float* out, void* stream) {
  if ((!src && rows > 0 && n > 0) || !out || rows < 0 || n < 0) return RS_ERR_INVALID_ARG;
  if (n == 0) return RS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t blocks = (n + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 8 * kNumSMs ? blocks : 8 * kNumSMs);
  prof::Scope ps("k_touched_columns", s);
  k_touched_columns<<<grid, 256, 0, s>>>(src, rows, n, out);
  return launch_status();
}
