// rs_filter: pruning mask (Sec. 3.3) / visibility indicator (Eq. importance-score-vis) with
// stream compaction to an ascending index list; rs_filter_nearest: nearest cluster centre
// for test cameras (Sec. 3.4).
//
// rs_filter is three HBM-bound kernels over h: per-block counts of the predicate (and the
// byte mask), one exclusive scan of the block counts, and an order-preserving scatter of
// the indices (block-local scan with warp ballots).  The block counts are the only
// scratch memory (4 bytes per 4096 elements).

#include "profile.cuh"
#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {

constexpr int kFiltThreads = 256;
constexpr int kFiltItems = 16;
constexpr int kFiltTile = kFiltThreads * kFiltItems;

__device__ __forceinline__ bool filter_pred(float h, float t, int mode) {
  return mode == 0 ? (h < t) : mode == 1 ? (h > t) : !(h < t);
}

// Per block: mask bytes and the number of selected elements in its tile (warp-striped).
__global__ void __launch_bounds__(kFiltThreads) k_filter_count(const float* __restrict__ h, int64_t n, float t,
                                                               int mode, uint8_t* __restrict__ mask,
                                                               uint32_t* __restrict__ bcount) {
  __shared__ uint32_t s[kFiltThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kFiltTile;
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < kFiltItems; ++i) {
    const int64_t k = base + i * kFiltThreads + threadIdx.x;
    if (k < n) {
      const bool on = filter_pred(__ldcs(h + k), t, mode);
      c += on;
      if (mask) mask[k] = (uint8_t)on;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < kFiltThreads / 32; ++w) tot += s[w];
    bcount[blockIdx.x] = tot;
  }
}

// Exclusive scan of the block counts in place (one block of 1024 threads); total to *count.
__global__ void __launch_bounds__(1024) k_filter_scan(uint32_t* __restrict__ bcount, int64_t nblk,
                                                      uint32_t* __restrict__ count) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0u;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nblk; b0 += 1024) {
    const int64_t b = b0 + threadIdx.x;
    const uint32_t v = b < nblk ? bcount[b] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_w[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_w[lane] = w;
    }
    __syncthreads();
    const uint32_t carry = s_carry;
    if (b < nblk) bcount[b] = carry + (warp ? s_w[warp - 1] : 0u) + x - v;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = carry + s_w[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = s_carry;
}

// Order-preserving scatter of the selected indices.  Element order inside a tile is
// (item, thread): each item row is a contiguous run of kFiltThreads elements.
__global__ void __launch_bounds__(kFiltThreads) k_filter_scatter(const float* __restrict__ h, int64_t n, float t,
                                                                 int mode, const uint32_t* __restrict__ bpre,
                                                                 uint32_t* __restrict__ idx) {
  __shared__ uint32_t s_w[kFiltThreads / 32];
  __shared__ uint32_t s_row;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kFiltTile;
  uint32_t run = bpre[blockIdx.x];
  for (int i = 0; i < kFiltItems; ++i) {
    const int64_t k = base + i * kFiltThreads + threadIdx.x;
    const bool on = k < n && filter_pred(__ldcs(h + k), t, mode);
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    if (lane == 0) s_w[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, row = 0;
#pragma unroll
    for (int w = 0; w < kFiltThreads / 32; ++w) {
      const uint32_t c = s_w[w];
      before += (w < warp) ? c : 0u;
      row += c;
    }
    if (on) idx[run + before + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)k;
    run += row;
    __syncthreads();
  }
  (void)s_row;
}

__global__ void k_nearest(const float* __restrict__ centres, int k, const float* __restrict__ cams, int n,
                          int32_t* __restrict__ out) {
  extern __shared__ float s_c[];
  for (int i = threadIdx.x; i < 3 * k; i += blockDim.x) s_c[i] = centres[i];
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const float x0 = cams[3 * c], x1 = cams[3 * c + 1], x2 = cams[3 * c + 2];
  int best = 0;
  float bd = 0.f;
  for (int j = 0; j < k; ++j) {
    const float d0 = __fsub_rn(x0, s_c[3 * j]);
    const float d1 = __fsub_rn(x1, s_c[3 * j + 1]);
    const float d2 = __fsub_rn(x2, s_c[3 * j + 2]);
    // ((d0^2 + d1^2) + d2^2), each product rounded: no fused multiply-add
    const float d = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
    if (j == 0 || d < bd) {
      best = j;
      bd = d;
    }
  }
  out[c] = best;
}

size_t filter_ws_bytes(int64_t n) {
  const int64_t nblk = (n + kFiltTile - 1) / kFiltTile;
  return align_up((size_t)(nblk > 0 ? nblk : 1) * sizeof(uint32_t), 256);
}

rs_status filter_launch(const float* h, int64_t n, float t, int mode, uint8_t* mask, uint32_t* idx,
                        uint32_t* count, uint32_t* bcount, cudaStream_t s) {
  const int64_t nblk = (n + kFiltTile - 1) / kFiltTile;
  if (nblk > 0x7fffffffLL) return RS_ERR_INVALID_ARG;
  if (n == 0) {
    if (cudaMemsetAsync(count, 0, sizeof(uint32_t), s) != cudaSuccess) return RS_ERR_CUDA;
    return RS_OK;
  }
  { prof::Scope ps("k_filter_count", s);
  k_filter_count<<<(unsigned)nblk, kFiltThreads, 0, s>>>(h, n, t, mode, mask, bcount); }
  { prof::Scope ps("k_filter_scan", s);
  k_filter_scan<<<1, 1024, 0, s>>>(bcount, nblk, count); }
  if (idx) {
    prof::Scope ps("k_filter_scatter", s);
    k_filter_scatter<<<(unsigned)nblk, kFiltThreads, 0, s>>>(h, n, t, mode, bcount, idx);
  }
  return launch_status();
}

}  // namespace rs

using namespace rs;

extern "C" rs_status rs_filter(const float* h, int64_t n, float t, rs_filter_mode mode, uint8_t* mask,
                               uint32_t* idx, uint32_t* count, void* ws, size_t ws_bytes, void* stream) {
  if ((!h && n > 0) || !count || n < 0 || n >= ((int64_t)1 << 32)) return RS_ERR_INVALID_ARG;
  if (mode != RS_PRUNE_BELOW && mode != RS_KEEP_ABOVE && mode != RS_PRUNE_KEEP) return RS_ERR_INVALID_ARG;
  if (!ws || ws_bytes < filter_ws_bytes(n)) return RS_ERR_WORKSPACE;
  return filter_launch(h, n, t, (int)mode, mask, idx, count, static_cast<uint32_t*>(ws),
                       reinterpret_cast<cudaStream_t>(stream));
}

extern "C" rs_status rs_filter_nearest(const float* centres, int32_t k, const float* cam_centres, int32_t n_cams,
                                       int32_t* out, void* stream) {
  if (!centres || !cam_centres || !out || k <= 0 || n_cams < 0 || k > 4096) return RS_ERR_INVALID_ARG;
  if (n_cams == 0) return RS_OK;
  const int threads = 128;
  prof::Scope ps("k_nearest", reinterpret_cast<cudaStream_t>(stream));
  k_nearest<<<(n_cams + threads - 1) / threads, threads, (size_t)k * 3 * sizeof(float),
              reinterpret_cast<cudaStream_t>(stream)>>>(centres, k, cam_centres, n_cams, out);
  return launch_status();
}

// ---------------------------------------------------------------------------------------
// rs_filter_noalloc: the same kernels with their per-block counts in a fixed device array.

namespace rs {

constexpr int64_t kNoallocMaxBlocks = (RS_FILTER_NOALLOC_MAX_N + kFiltTile - 1) / kFiltTile;   // 16384 words
static __device__ __align__(256) uint32_t g_filter_scratch[kNoallocMaxBlocks];

// Device address of g_filter_scratch on the current device.  (In host code the array's name
// is only a host-side stand-in, never a device address.)  Looked up on every call: the
// lookup allocates nothing and stays right after a device reset reloads the module.
static rs_status noalloc_scratch(uint32_t** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_filter_scratch) != cudaSuccess || !p) return RS_ERR_CUDA;
  *out = static_cast<uint32_t*>(p);
  return RS_OK;
}

}  // namespace rs

extern "C" rs_status rs_filter_noalloc(const float* h, int64_t n, float t, rs_filter_mode mode, uint8_t* mask,
                                       uint32_t* idx, uint32_t* count, void* stream) {
  if ((!h && n > 0) || !count || n < 0) return RS_ERR_INVALID_ARG;
  if (n > RS_FILTER_NOALLOC_MAX_N) return RS_ERR_INVALID_ARG;
  if (mode != RS_PRUNE_BELOW && mode != RS_KEEP_ABOVE && mode != RS_PRUNE_KEEP) return RS_ERR_INVALID_ARG;
  uint32_t* scratch = nullptr;
  const rs_status st = noalloc_scratch(&scratch);
  if (st != RS_OK) return st;
  // every block of k_filter_count writes its own count before the scan reads it: the array
  // needs no clearing between calls
  return filter_launch(h, n, t, (int)mode, mask, idx, count, scratch, reinterpret_cast<cudaStream_t>(stream));
}
