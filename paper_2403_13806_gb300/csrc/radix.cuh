// Stable LSD radix sort of (uint32 key, uint32 value) pairs, reduce-then-scan form.
//
// A pass over digit [shift, shift + rbits) (rbits <= 8) is three kernels on a fixed grid of
// `grid` blocks, each owning one contiguous range of the input:
//   upsweep   -- per-block digit histogram, hist[grid][R];
//   hist scan -- one block per digit: exclusive prefix of that digit over the blocks, and
//                the digit's total;
//   downsweep -- every block adds the digit bases (exclusive prefix of the totals) to its
//                per-digit offsets, then walks its range in tiles of 2048 keys: a stable
//                in-tile rank (warp match + per-warp digit counters), a shared-memory reorder
//                by digit, and coalesced stores of each digit run.
// There are no inter-block waits.  The element count may live in device memory (produced
// by an earlier kernel of the same stream): the grid is sized for an upper bound and each
// block clamps to the actual count.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "profile.cuh"

namespace rs {
namespace radix {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                       // keys per thread per tile
constexpr int kTile = kThreads * kItems;        // 2048
constexpr int kMaxR = 256;
constexpr int kMaxGrid = 4 * 152;

struct Range {
  int64_t begin, end;
};

__device__ __forceinline__ int64_t load_count(int64_t n_host, const uint32_t* n_dev) {
  return n_dev ? (int64_t)*n_dev : n_host;
}

// Contiguous range of block b: whole tiles, so every block but the last processes full tiles.
__device__ __forceinline__ Range block_range(int64_t n, int grid, int b) {
  const int64_t tiles = (n + kTile - 1) / kTile;
  const int64_t per = (tiles + grid - 1) / grid;
  Range r;
  r.begin = min((int64_t)b * per * kTile, n);
  r.end = min((int64_t)(b + 1) * per * kTile, n);
  return r;
}

// Exclusive scan of v over the block (kThreads values, one per thread); the block total is
// written to *total (shared).  Contains barriers: every thread must call it.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kWarps ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kWarps) s_warp[lane] = w;   // inclusive warp prefix
    if (lane == kWarps - 1) *total = w;
  }
  __syncthreads();
  const uint32_t wbase = warp ? s_warp[warp - 1] : 0u;
  const uint32_t r = wbase + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThreads) k_upsweep(const uint32_t* __restrict__ keys, int64_t n_host,
                                                      const uint32_t* __restrict__ n_dev, int shift, int rbits,
                                                      uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[kWarps][kMaxR];
  const int R = 1 << rbits;
  const uint32_t mask = (uint32_t)R - 1u;
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * kMaxR; i += kThreads) (&s_hist[0][0])[i] = 0u;
  __syncthreads();
  const int64_t n = load_count(n_host, n_dev);
  const Range r = block_range(n, gridDim.x, blockIdx.x);
  // 16-byte loads over the aligned body (range starts are multiples of 2048 keys)
  const int64_t body_end = r.begin + ((r.end - r.begin) & ~(int64_t)3);
  const uint4* k4 = reinterpret_cast<const uint4*>(keys + r.begin);
  const int64_t n4 = (body_end - r.begin) >> 2;
  for (int64_t i = threadIdx.x; i < n4; i += kThreads) {
    const uint4 k = __ldcs(k4 + i);
    atomicAdd(&s_hist[warp][(k.x >> shift) & mask], 1u);
    atomicAdd(&s_hist[warp][(k.y >> shift) & mask], 1u);
    atomicAdd(&s_hist[warp][(k.z >> shift) & mask], 1u);
    atomicAdd(&s_hist[warp][(k.w >> shift) & mask], 1u);
  }
  for (int64_t i = body_end + threadIdx.x; i < r.end; i += kThreads)
    atomicAdd(&s_hist[warp][(keys[i] >> shift) & mask], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < R; d += kThreads) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) c += s_hist[w][d];
    hist[(int64_t)blockIdx.x * R + d] = c;
  }
}

// One block per digit d: off[b][d] = sum of hist[b'][d] for b' < b; tot[d] = sum over all b.
__global__ void __launch_bounds__(kThreads) k_hist_scan(const uint32_t* __restrict__ hist, int grid, int rbits,
                                                        uint32_t* __restrict__ off, uint32_t* __restrict__ tot) {
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_total;
  const int R = 1 << rbits;
  const int d = blockIdx.x;
  uint32_t carry = 0;
  for (int b0 = 0; b0 < grid; b0 += kThreads) {
    const int b = b0 + threadIdx.x;
    const uint32_t v = b < grid ? hist[(int64_t)b * R + d] : 0u;
    const uint32_t ex = block_excl_scan(v, s_warp, &s_total);
    if (b < grid) off[(int64_t)b * R + d] = carry + ex;
    carry += s_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[d] = carry;
}

__global__ void __launch_bounds__(kThreads) k_downsweep(const uint32_t* __restrict__ keys_in,
                                                        const uint32_t* __restrict__ vals_in,
                                                        uint32_t* __restrict__ keys_out,
                                                        uint32_t* __restrict__ vals_out, int64_t n_host,
                                                        const uint32_t* __restrict__ n_dev, int shift, int rbits,
                                                        const uint32_t* __restrict__ off,
                                                        const uint32_t* __restrict__ tot) {
  __shared__ uint32_t s_keys[kTile];
  __shared__ uint32_t s_vals[kTile];
  __shared__ uint32_t s_whist[kWarps][kMaxR];     // per-warp digit counts, then prefixes
  __shared__ uint32_t s_off[kMaxR];               // global position of the next key of digit d
  __shared__ uint32_t s_lstart[kMaxR];            // tile-local start of digit d
  __shared__ uint32_t s_cnt[kMaxR];
  __shared__ uint32_t s_scan[kWarps];
  __shared__ uint32_t s_total;

  const int R = 1 << rbits;
  const uint32_t mask = (uint32_t)R - 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = load_count(n_host, n_dev);
  const Range r = block_range(n, gridDim.x, blockIdx.x);
  if (r.begin >= r.end) return;    // uniform per block

  {
    const int d = threadIdx.x;
    const uint32_t base = block_excl_scan(d < R ? tot[d] : 0u, s_scan, &s_total);
    if (d < R) s_off[d] = base + off[(int64_t)blockIdx.x * R + d];
  }
  __syncthreads();

  const unsigned lt_mask = (1u << lane) - 1u;
  for (int64_t t0 = r.begin; t0 < r.end; t0 += kTile) {
    const int tn = (int)min((int64_t)kTile, r.end - t0);
    for (int i = threadIdx.x; i < kWarps * kMaxR; i += kThreads) (&s_whist[0][0])[i] = 0u;
    __syncthreads();
    uint32_t k[kItems], v[kItems], rank[kItems];
    int dg[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int li = warp * (kItems * 32) + i * 32 + lane;     // warp-striped: coalesced loads
      if (li < tn) {
        k[i] = __ldcs(keys_in + t0 + li);
        v[i] = __ldcs(vals_in + t0 + li);
        dg[i] = (int)((k[i] >> shift) & mask);
      } else {
        k[i] = 0u;
        v[i] = 0u;
        dg[i] = R;      // sentinel digit, never counted
      }
    }
    // stable rank within the warp, in (item, lane) order
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const unsigned peers = __match_any_sync(0xffffffffu, dg[i]);
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if (dg[i] < R) base = s_whist[warp][dg[i]];
      rank[i] = base + __popc(peers & lt_mask);
      __syncwarp();
      if (lane == leader && dg[i] < R) s_whist[warp][dg[i]] = base + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {
      const int d = threadIdx.x;
      uint32_t c = 0;
      if (d < R) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          const uint32_t x = s_whist[w][d];
          s_whist[w][d] = c;
          c += x;
        }
        s_cnt[d] = c;
      }
      const uint32_t st = block_excl_scan(d < R ? c : 0u, s_scan, &s_total);
      if (d < R) s_lstart[d] = st;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      if (dg[i] < R) {
        const uint32_t p = s_lstart[dg[i]] + s_whist[warp][dg[i]] + rank[i];
        s_keys[p] = k[i];
        s_vals[p] = v[i];
      }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < tn; p += kThreads) {
      const uint32_t key = s_keys[p];
      const int d = (int)((key >> shift) & mask);
      const uint32_t g = s_off[d] + (uint32_t)p - s_lstart[d];
      if (keys_out) keys_out[g] = key;
      vals_out[g] = s_vals[p];
    }
    __syncthreads();
    if (threadIdx.x < R) s_off[threadIdx.x] += s_cnt[threadIdx.x];
    __syncthreads();
  }
}

inline int grid_for(int64_t n_max, int max_grid = kMaxGrid) {
  int64_t tiles = (n_max + kTile - 1) / kTile;
  if (tiles < 1) tiles = 1;
  return (int)(tiles < max_grid ? tiles : max_grid);
}

// Scratch of a sort with this grid: hist and off (grid x 256 each) and the digit totals.
inline size_t scratch_words(int grid) { return (size_t)2 * grid * kMaxR + kMaxR; }

inline int sort_passes(int bits) { return bits < 1 ? 1 : (bits + 7) / 8; }

// Sorts on bits [0, bits) of the keys.  Buffers ping-pong between (k0, v0) and (k1, v1);
// returns 0 if the result is in (k0, v0), 1 if in (k1, v1).  The last pass writes keys
// only if write_last_keys.
inline int sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n_host,
                      const uint32_t* n_dev, int bits, uint32_t* scratch, int grid, cudaStream_t s,
                      bool write_last_keys = true) {
  const int passes = sort_passes(bits);
  const int rbits = (bits + passes - 1) / passes;
  uint32_t* hist = scratch;
  uint32_t* off = scratch + (size_t)grid * kMaxR;
  uint32_t* tot = off + (size_t)grid * kMaxR;
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * rbits;
    const int rb = (shift + rbits <= bits) ? rbits : bits - shift;
    uint32_t* ki = cur ? k1 : k0;
    uint32_t* vi = cur ? v1 : v0;
    uint32_t* ko = cur ? k0 : k1;
    uint32_t* vo = cur ? v0 : v1;
    { ::rs::prof::Scope ps("k_upsweep", s);
    k_upsweep<<<grid, kThreads, 0, s>>>(ki, n_host, n_dev, shift, rb, hist); }
    { ::rs::prof::Scope ps("k_hist_scan", s);
    k_hist_scan<<<1 << rb, kThreads, 0, s>>>(hist, grid, rb, off, tot); }
    const bool last = (p == passes - 1);
    ::rs::prof::Scope ps("k_downsweep", s);
    k_downsweep<<<grid, kThreads, 0, s>>>(ki, vi, (last && !write_last_keys) ? nullptr : ko, vo, n_host, n_dev,
                                          shift, rb, off, tot);
    cur ^= 1;
  }
  return cur;
}

}  // namespace radix
}  // namespace rs
