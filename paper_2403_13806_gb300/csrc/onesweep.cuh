// Single-pass-per-digit stable radix sort of (uint32 key, uint32 value) pairs with
// decoupled look-back (for large inputs, such as the duplicated tile instances).
//
//   k_digit_hist  -- one read of the keys: the histogram of every digit of every pass.
//   k_onesweep    -- one launch per pass.  Each CTA claims the next tile of 4096 keys from an
//                    atomic counter (so every earlier tile belongs to a CTA that is already
//                    running), ranks its keys stably (warp match + per-warp counters),
//                    publishes its per-digit counts, and looks back over the earlier tiles'
//                    published words until it meets an inclusive prefix.  A status word packs
//                    a 2-bit flag (0 not ready, 1 tile count, 2 inclusive prefix) with a
//                    30-bit count, so the data travels with the flag and relaxed loads and
//                    stores suffice.  Keys then go to digit base + prefix + local rank through
//                    a shared-memory reorder, so each digit run is stored contiguously.
// Every wait is bounded: a CTA that gives up records RS_ERR_TIMEOUT in the device status and
// goes on with the partial prefix (its positions stay below the true ones, so every store
// stays inside the output), and never hangs.  Counts must stay below 2^30.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "radix.cuh"
#include "radsplat.h"

namespace rs {
namespace onesweep {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // 4096
constexpr int kR = 256;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr int kMaxPasses = 4;
constexpr int kSpinLimit = 1 << 20;   // polls of one predecessor word before giving up

// Histograms of `passes` digits of rbits bits each over the first n keys (n in device memory).
__global__ void __launch_bounds__(256) k_digit_hist(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_dev,
                                                    int passes, int rbits, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t s[kMaxPasses * kR];
  for (int i = threadIdx.x; i < kMaxPasses * kR; i += blockDim.x) s[i] = 0u;
  __syncthreads();
  const int64_t n = *n_dev;
  const uint32_t mask = (1u << rbits) - 1u;
  const int64_t n4 = n >> 2;
  const uint4* k4 = reinterpret_cast<const uint4*>(keys);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 k = __ldcs(k4 + i);
    for (int p = 0; p < passes; ++p) {
      const int sh = p * rbits;
      atomicAdd(&s[p * kR + ((k.x >> sh) & mask)], 1u);
      atomicAdd(&s[p * kR + ((k.y >> sh) & mask)], 1u);
      atomicAdd(&s[p * kR + ((k.z >> sh) & mask)], 1u);
      atomicAdd(&s[p * kR + ((k.w >> sh) & mask)], 1u);
    }
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&s[p * kR + ((k >> (p * rbits)) & mask)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kR; i += blockDim.x)
    if (s[i]) atomicAdd(ghist + i, s[i]);
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Exclusive scan over the CTA (one value per thread); total to *total.
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
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
    if (lane < kWarps) s_warp[lane] = w;
    if (lane == kWarps - 1) *total = w;
  }
  __syncthreads();
  const uint32_t r = (warp ? s_warp[warp - 1] : 0u) + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThreads, 2) k_onesweep(const uint32_t* __restrict__ keys_in,
                                                          const uint32_t* __restrict__ vals_in,
                                                          uint32_t* __restrict__ keys_out,
                                                          uint32_t* __restrict__ vals_out,
                                                          const uint32_t* __restrict__ n_dev, int shift, int rbits,
                                                          const uint32_t* __restrict__ ghist, uint32_t* status,
                                                          uint32_t* tile_counter, rs_device_status* st) {
  __shared__ uint32_t s_keys[kTile];
  __shared__ uint32_t s_vals[kTile];
  __shared__ uint16_t s_whist[kWarps][kR];     // per-warp digit counts (<= 256), then prefixes (<= 4096)
  __shared__ uint32_t s_gpos[kR];      // global position of the first key of digit d in this tile
  __shared__ uint32_t s_lstart[kR];
  __shared__ uint32_t s_scan[kWarps];
  __shared__ uint32_t s_total;
  __shared__ int s_tile;

  const int R = 1 << rbits;
  const uint32_t mask = (uint32_t)R - 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = *n_dev;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_counter, 1u);
  for (int i = threadIdx.x; i < kWarps * kR; i += kThreads) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t t0 = (int64_t)tile * kTile;
  if (t0 >= n) return;   // uniform per CTA; no later tile waits on this one
  const int tn = (int)min((int64_t)kTile, n - t0);

  uint32_t k[kItems], v[kItems], rank[kItems];
  int dg[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int li = warp * (kItems * 32) + i * 32 + lane;
    if (li < tn) {
      k[i] = __ldcs(keys_in + t0 + li);
      v[i] = __ldcs(vals_in + t0 + li);
      dg[i] = (int)((k[i] >> shift) & mask);
    } else {
      k[i] = 0u;
      v[i] = 0u;
      dg[i] = R;
    }
  }
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const unsigned peers = __match_any_sync(0xffffffffu, dg[i]);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (dg[i] < R) base = s_whist[warp][dg[i]];
    rank[i] = base + __popc(peers & lt_mask);
    __syncwarp();
    if (lane == leader && dg[i] < R) s_whist[warp][dg[i]] = (uint16_t)(base + __popc(peers));
    __syncwarp();
  }
  __syncthreads();

  // per digit: warp prefixes, tile count; publish the count, look back, publish the prefix
  const int d = threadIdx.x;
  uint32_t cnt = 0;
  if (d < R) {
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t x = s_whist[w][d];
      s_whist[w][d] = (uint16_t)cnt;
      cnt += x;
    }
    uint32_t* my = status + (int64_t)tile * kR + d;
    if (tile == 0) {
      st_relaxed(my, kFlagInc | cnt);
    } else {
      st_relaxed(my, kFlagAgg | cnt);
    }
  }
  uint32_t excl = 0;
  if (d < R && tile > 0) {
    int t = tile - 1;
    int spins = 0;
    while (t >= 0) {
      const uint32_t w = ld_relaxed(status + (int64_t)t * kR + d);
      const uint32_t f = w & ~kValMask;
      if (f == 0u) {
        if (++spins > kSpinLimit) {
          if (st) atomicCAS(&st->code, 0, (int)RS_ERR_TIMEOUT);
          break;
        }
        if (spins > 32) __nanosleep(128);
        continue;
      }
      spins = 0;
      excl += w & kValMask;
      if (f == kFlagInc) break;
      --t;
    }
    st_relaxed(status + (int64_t)tile * kR + d, kFlagInc | ((excl + cnt) & kValMask));
  }
  // digit base from the global histogram
  const uint32_t base = cta_excl_scan(d < R ? ghist[d] : 0u, s_scan, &s_total);
  const uint32_t lstart = cta_excl_scan(d < R ? cnt : 0u, s_scan, &s_total);
  if (d < R) {
    s_gpos[d] = base + excl;
    s_lstart[d] = lstart;
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
    const int dd = (int)((key >> shift) & mask);
    const uint32_t g = s_gpos[dd] + (uint32_t)p - s_lstart[dd];
    if (keys_out) keys_out[g] = key;
    vals_out[g] = s_vals[p];
  }
}

inline int64_t tiles_for(int64_t n) { return (n + kTile - 1) / kTile; }

// Scratch words: digit histograms, one tile counter per pass, status words of the largest pass.
inline size_t scratch_words(int64_t n_max) { return (size_t)kMaxPasses * kR + 64 + (size_t)tiles_for(n_max) * kR; }

// Stable sort of the first n (device count) pairs on bits [0, bits), bits <= 32.  Buffers
// ping-pong between (k0, v0) and (k1, v1); returns 0 if the result is in (k0, v0), 1 if in
// (k1, v1).  n_max bounds the count (grid size and scratch).
inline int sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* n_dev, int64_t n_max,
                      int bits, uint32_t* scratch, rs_device_status* st, cudaStream_t s, bool write_last_keys = true) {
  const int passes = radix::sort_passes(bits);
  const int rbits = (bits + passes - 1) / passes;
  uint32_t* ghist = scratch;
  uint32_t* counters = scratch + kMaxPasses * kR;
  uint32_t* status = counters + 64;
  const int64_t tiles = tiles_for(n_max);
  cudaMemsetAsync(scratch, 0, (kMaxPasses * kR + 64) * sizeof(uint32_t), s);
  k_digit_hist<<<4 * 152, 256, 0, s>>>(k0, n_dev, passes, rbits, ghist);
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * rbits;
    const int rb = (shift + rbits <= bits) ? rbits : bits - shift;
    uint32_t* ki = cur ? k1 : k0;
    uint32_t* vi = cur ? v1 : v0;
    uint32_t* ko = cur ? k0 : k1;
    uint32_t* vo = cur ? v0 : v1;
    cudaMemsetAsync(status, 0, (size_t)tiles * kR * sizeof(uint32_t), s);
    const bool last = (p == passes - 1);
    k_onesweep<<<(unsigned)(tiles > 0 ? tiles : 1), kThreads, 0, s>>>(
        ki, vi, (last && !write_last_keys) ? nullptr : ko, vo, n_dev, shift, rb, ghist + p * kR, status,
        counters + p, st);
    cur ^= 1;
  }
  return cur;
}

}  // namespace onesweep
}  // namespace rs
