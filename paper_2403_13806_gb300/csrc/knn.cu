// rs_nn_distance: the distance from every point to its nearest other point, the scale
// initialisation of Sec. 3.2 (s_i = min over p != p_i of |p_i - p|).
//
// Point sets such as a dense object inside a sparse background make a uniform grid either
// too coarse for the dense part or too fine for the sparse part, so the search uses an
// implicit octree: the points sorted by a 30-bit Morton code (10 bits per axis over the
// bounding cube), in which every octree cell of level L (edge h 2^L) is a contiguous range.
//   k_bbox, k_grid_params  -- bounding cube (origin, h = edge / 1024);
//   k_morton               -- Morton code of every point;
//   radix_tiles            -- points sorted by code (stable);
//   k_sorted_points        -- coordinates in sorted order;
//   k_nn                   -- per point: an upper bound R from its 16 neighbours in Morton
//                             order; the smallest level whose cell edge is >= 2R (at most two
//                             cells per axis then cover the ball of radius R around the
//                             point); the start and end of each of those <= 8 cells (a table
//                             of the first index per 18-bit code prefix leaves at most a short
//                             search inside one prefix bucket); the minimum over their points.
// Exactness: the cell index floor((v - o)/h) is monotone in v, so every point within R of the
// query on each axis (a superset of the ball) lies in a cell of the quantised range.
// Distances are FP32 ((dx^2 + dy^2) + dz^2 with every operation rounded; square root
// correctly rounded); a point with a non-finite coordinate gets +inf.
#include <math.h>

#include "profile.cuh"
#include "radix_tiles.cuh"
#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {

constexpr int kBBoxBlocks = 1024;
constexpr int kMortonBits = 10;   // per axis
constexpr int kWindow = 8;        // Morton neighbours on each side for the first bound
constexpr int kPrefixShift = 12;  // index table over the top 18 code bits (octree level 4 cells)
constexpr int kPrefixes = 1 << (3 * kMortonBits - kPrefixShift);

struct CubeParams {
  float ox, oy, oz, h, inv_h;
  uint32_t n;   // the point count, as the sort's device count
};

struct NNWs {
  CubeParams* params;
  float* partial;       // [6][kBBoxBlocks]
  uint32_t* keys[2];
  uint32_t* vals[2];
  uint32_t* scratch;
  float4* spts;         // [n]
  uint32_t* first;      // [kPrefixes + 1]: first sorted index whose code has a prefix >= p
  size_t bytes;
};

static NNWs nn_ws_layout(void* base, int64_t n) {
  NNWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? static_cast<char*>(base) + off : nullptr;
    off += align_up(bytes > 0 ? bytes : 1, 256);
    return p;
  };
  const size_t nn = (size_t)(n > 0 ? n : 1);
  w.params = reinterpret_cast<CubeParams*>(take(sizeof(CubeParams)));
  w.partial = reinterpret_cast<float*>(take(6 * kBBoxBlocks * 4));
  for (int i = 0; i < 2; ++i) w.keys[i] = reinterpret_cast<uint32_t*>(take(nn * 4));
  for (int i = 0; i < 2; ++i) w.vals[i] = reinterpret_cast<uint32_t*>(take(nn * 4));
  w.scratch = reinterpret_cast<uint32_t*>(take(tiles::scratch_words(n) * 4));
  w.spts = reinterpret_cast<float4*>(take(nn * 16));
  w.first = reinterpret_cast<uint32_t*>(take((size_t)(kPrefixes + 1) * 4));
  w.bytes = off;
  return w;
}

__global__ void __launch_bounds__(256) k_bbox(const float* __restrict__ m, int64_t n, float* __restrict__ partial) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float v = m[a * n + i];
      lo[a] = fminf(lo[a], v);
      hi[a] = fmaxf(hi[a], v);
    }
  }
  __shared__ float s[6][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
    if (lane == 0) {
      s[a][warp] = lo[a];
      s[3 + a][warp] = hi[a];
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float v = s[threadIdx.x][0];
    for (int w = 1; w < 8; ++w) v = threadIdx.x < 3 ? fminf(v, s[threadIdx.x][w]) : fmaxf(v, s[threadIdx.x][w]);
    partial[threadIdx.x * kBBoxBlocks + blockIdx.x] = v;
  }
}

__global__ void k_grid_params(const float* __restrict__ partial, int nblk, int64_t n, CubeParams* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float lo[3], hi[3];
  double emax = 0.0;
  for (int a = 0; a < 3; ++a) {
    lo[a] = INFINITY;
    hi[a] = -INFINITY;
    for (int b = 0; b < nblk; ++b) {
      lo[a] = fminf(lo[a], partial[a * kBBoxBlocks + b]);
      hi[a] = fmaxf(hi[a], partial[(3 + a) * kBBoxBlocks + b]);
    }
    emax = fmax(emax, (double)hi[a] - (double)lo[a]);
  }
  if (!(emax > 0.0) || !isfinite(emax)) emax = 1.0;
  // cube edge 1024 h, slightly larger than the box so the largest coordinate maps below 1024
  const double h = emax * (1.0 + 1e-6) / (double)(1 << kMortonBits) + 1e-30;
  out->ox = lo[0];
  out->oy = lo[1];
  out->oz = lo[2];
  out->h = (float)h;
  out->inv_h = (float)(1.0 / h);
  out->n = (uint32_t)n;
}

__device__ __forceinline__ int quant(float v, float o, float inv_h) {
  const float f = floorf(__fmul_rn(__fsub_rn(v, o), inv_h));
  if (!(f >= 0.f)) return 0;   // also NaN
  return f > (float)((1 << kMortonBits) - 1) ? (1 << kMortonBits) - 1 : (int)f;
}

// bits of x (< 2^kMortonBits) spread to every third position
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
  uint32_t r = 0;
#pragma unroll
  for (int b = 0; b < kMortonBits; ++b) r |= ((x >> b) & 1u) << (3 * b);
  return r;
}

__device__ __forceinline__ uint32_t morton(int x, int y, int z) {
  return spread3((uint32_t)x) | (spread3((uint32_t)y) << 1) | (spread3((uint32_t)z) << 2);
}

__global__ void __launch_bounds__(256) k_morton(const float* __restrict__ m, int64_t n,
                                                const CubeParams* __restrict__ cp, uint32_t* __restrict__ keys,
                                                uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const CubeParams p = *cp;
  keys[i] = morton(quant(m[i], p.ox, p.inv_h), quant(m[n + i], p.oy, p.inv_h), quant(m[2 * n + i], p.oz, p.inv_h));
  vals[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(256) k_sorted_points(const float* __restrict__ m, int64_t n,
                                                       const uint32_t* __restrict__ sv, float4* __restrict__ spts) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t i = sv[j];
  spts[j] = make_float4(m[i], m[n + i], m[2 * n + i], 0.f);
}

__device__ __forceinline__ float dist2(const float4& a, const float4& b) {
  const float d0 = __fsub_rn(a.x, b.x), d1 = __fsub_rn(a.y, b.y), d2 = __fsub_rn(a.z, b.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
}

// first index in sorted codes [0, n) with code >= key
__device__ __forceinline__ int64_t lower_bound(const uint32_t* __restrict__ sk, int64_t n, uint32_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (sk[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// first[p] = lower_bound(codes, p << kPrefixShift) for every prefix p (and first[kPrefixes] = n)
__global__ void __launch_bounds__(256) k_prefix_table(const uint32_t* __restrict__ sk, int64_t n,
                                                      uint32_t* __restrict__ first) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kPrefixes) return;
  first[p] = p == kPrefixes ? (uint32_t)n : (uint32_t)lower_bound(sk, n, (uint32_t)p << kPrefixShift);
}

// lower_bound through the prefix table: a search only inside one prefix bucket
__device__ __forceinline__ int64_t lower_bound_t(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ first,
                                                 uint32_t key) {
  const uint32_t p = key >> kPrefixShift;
  int64_t lo = first[p], hi = first[p + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (sk[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_nn(const float4* __restrict__ spts, const uint32_t* __restrict__ sk,
                                            const uint32_t* __restrict__ sv, int64_t n,
                                            const CubeParams* __restrict__ cp, const uint32_t* __restrict__ first,
                                            float* __restrict__ dist) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const CubeParams p = *cp;
  const float4 q = spts[j];
  if (!(isfinite(q.x) && isfinite(q.y) && isfinite(q.z))) {
    dist[sv[j]] = INFINITY;   // a non-finite point has no nearest neighbour
    return;
  }
  float best = INFINITY;
  for (int64_t k = max(j - kWindow, (int64_t)0); k <= min(j + kWindow, n - 1); ++k)
    if (k != j) best = fminf(best, dist2(q, spts[k]));
  // per-axis half width covering the ball of radius sqrt(best), with a margin for rounding
  const float R = __fsqrt_rn(best) * (1.f + 1e-5f) + 1e-30f;
  int L = 0;
  while (L < kMortonBits && (double)p.h * (double)(1 << L) < 2.0 * (double)R) ++L;
  const int side = 1 << (kMortonBits - L);
  const int x0 = quant(__fsub_rn(q.x, R), p.ox, p.inv_h) >> L;
  const int x1 = min(quant(__fadd_rn(q.x, R), p.ox, p.inv_h) >> L, side - 1);
  const int y0 = quant(__fsub_rn(q.y, R), p.oy, p.inv_h) >> L;
  const int y1 = min(quant(__fadd_rn(q.y, R), p.oy, p.inv_h) >> L, side - 1);
  const int z0 = quant(__fsub_rn(q.z, R), p.oz, p.inv_h) >> L;
  const int z1 = min(quant(__fadd_rn(q.z, R), p.oz, p.inv_h) >> L, side - 1);
  for (int z = z0; z <= z1; ++z)
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) {
        const uint32_t c0 = morton(x, y, z) << (3 * L);
        const uint64_t c1 = (uint64_t)c0 + ((uint64_t)1 << (3 * L));   // exclusive
        const int64_t k0 = lower_bound_t(sk, first, c0);
        const int64_t k1 = c1 >= ((uint64_t)1 << (3 * kMortonBits)) ? n : lower_bound_t(sk, first, (uint32_t)c1);
        for (int64_t k = k0; k < k1; ++k)
          if (k != j) best = fminf(best, dist2(q, spts[k]));
      }
  dist[sv[j]] = __fsqrt_rn(best);
}

}  // namespace rs

using namespace rs;

extern "C" size_t rs_nn_workspace_size(int64_t n) {
  if (n < 2) return 0;
  return nn_ws_layout(nullptr, n).bytes;
}

extern "C" rs_status rs_nn_distance(const float* means, int64_t n, float* dist, void* ws, size_t ws_bytes,
                                    void* stream) {
  if (!means || !dist || n < 2 || n >= ((int64_t)1 << 31)) return RS_ERR_INVALID_ARG;
  const NNWs w = nn_ws_layout(ws, n);
  if (!ws || ws_bytes < w.bytes || !aligned<float4>(ws, 256)) return RS_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t blocks = (n + 255) / 256;
  const int nblk = (int)(blocks < kBBoxBlocks ? blocks : kBBoxBlocks);
  {
    prof::Scope ps("k_bbox", s);
    k_bbox<<<nblk, 256, 0, s>>>(means, n, w.partial);
  }
  {
    prof::Scope ps("k_grid_params", s);
    k_grid_params<<<1, 32, 0, s>>>(w.partial, nblk, n, w.params);
  }
  {
    prof::Scope ps("k_morton", s);
    k_morton<<<(unsigned)blocks, 256, 0, s>>>(means, n, w.params, w.keys[0], w.vals[0]);
  }
  const int cur = tiles::sort_pairs<uint32_t>(w.keys[0], w.vals[0], w.keys[1], w.vals[1], &w.params->n, n,
                                              3 * kMortonBits, w.scratch, s, true,
                                              {"k_morton_sort_hist", "k_morton_sort_scan", "k_morton_sort"});
  {
    prof::Scope ps("k_sorted_points", s);
    k_sorted_points<<<(unsigned)blocks, 256, 0, s>>>(means, n, w.vals[cur], w.spts);
  }
  {
    prof::Scope ps("k_prefix_table", s);
    k_prefix_table<<<(kPrefixes + 256) / 256, 256, 0, s>>>(w.keys[cur], n, w.first);
  }
  prof::Scope ps("k_nn", s);
  k_nn<<<(unsigned)blocks, 256, 0, s>>>(w.spts, w.keys[cur], w.vals[cur], n, w.params, w.first, dist);
  return launch_status();
}
