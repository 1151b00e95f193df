// Stable LSD radix sort of (key, uint32 value) pairs -- the items by depth and the
// super-tile instances by super-tile id: CTAs work on tiles of 2048 keys in every kernel,
// with no waits between CTAs.  Keys are 16-bit when every key fits (fewer bytes per pass),
// else 32-bit (all-ones is reserved as the padding sentinel; a 32-bit key equal to it is
// never counted nor written, so a caller can drop pairs by giving them that key).
//
// A pass over one digit (<= 8 bits) is three kernels:
//   k_tile_hist  -- per tile: its digit histogram, stored digit-major cnt[d][tile];
//   k_tile_scan  -- one CTA per digit: exclusive prefix of cnt[d][.] over the tiles (in
//                   place) and the digit's total;
//   k_tile_sort  -- per tile: digit bases (exclusive prefix of the totals) plus the tile's
//                   prefixes give the global position of its first key of each digit; the
//                   tile's keys are ranked stably (warp match and per-warp counters),
//                   reordered by digit in shared memory, and each digit run is stored
//                   contiguously.
// The per-tile counters cost 2 x 1 KB per 2048 keys of extra traffic per pass and make
// every tile independent, so the scatter runs at full occupancy.  The count lives on the
// device; the histogram and scatter kernels stride over its tiles with grids capped at a
// few waves, and the scan covers only its tiles, so a generous bound n_max (the instance
// capacity) costs no empty work.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "profile.cuh"
#include "rs_common.cuh"

namespace rs {
namespace tiles {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // 2048
constexpr int kR = 256;

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

// Passes of at most 8 bits for a sort on `bits` key bits.
__host__ __device__ inline int sort_passes(int bits) { return bits < 1 ? 1 : (bits + 7) / 8; }

template <typename KeyT, int TILE = kTile>
__global__ void __launch_bounds__(kThreads) k_tile_hist(const KeyT* __restrict__ keys, const uint32_t* __restrict__ n_dev,
                                                        int shift, int rbits, const int32_t* __restrict__ dig,
                                                        int64_t n_tiles_max, uint32_t* __restrict__ cnt) {
  if (dig) {   // the pass's digit from the device (shift, bits)
    shift = dig[0];
    rbits = dig[1];
  }
  __shared__ uint32_t s[kWarps][kR];
  const int warp = threadIdx.x >> 5;
  const int64_t n = *n_dev;
  const int64_t n_tiles = (n + TILE - 1) / TILE;
  const uint32_t mask = (1u << rbits) - 1u;
  // grid-stride over the tiles the device count needs (the grid is sized for the bound)
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    for (int i = threadIdx.x; i < kWarps * kR; i += kThreads) (&s[0][0])[i] = 0u;
    __syncthreads();
    const int64_t t0 = tile * TILE;
    const int tn = (int)min((int64_t)TILE, n - t0);
    constexpr int kVec = 16 / sizeof(KeyT);
    if (tn == TILE) {
      const uint4* kv = reinterpret_cast<const uint4*>(keys + t0);
      for (int i = threadIdx.x; i < TILE / kVec; i += kThreads) {
        const uint4 w = __ldcs(kv + i);
        const KeyT* k = reinterpret_cast<const KeyT*>(&w);
#pragma unroll
        for (int j = 0; j < kVec; ++j)
          if ((uint32_t)k[j] != 0xffffffffu) atomicAdd(&s[warp][((uint32_t)k[j] >> shift) & mask], 1u);
      }
    } else {
      for (int i = threadIdx.x; i < tn; i += kThreads) {
        const uint32_t kk = (uint32_t)keys[t0 + i];
        if (kk != 0xffffffffu) atomicAdd(&s[warp][(kk >> shift) & mask], 1u);
      }
    }
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) c += s[w][d];
    cnt[(int64_t)d * n_tiles_max + tile] = c;
    __syncthreads();
  }
}

// One CTA per digit d: exclusive prefix of cnt[d][0 .. n_tiles) in place, n_tiles the
// tiles of the device count (rows have stride n_tiles_max); tot[d] = total.
template <int TILE>
__global__ void __launch_bounds__(1024) k_tile_scan(uint32_t* __restrict__ cnt, const uint32_t* __restrict__ n_dev,
                                                    const int32_t* __restrict__ dig, int64_t n_tiles_max,
                                                    uint32_t* __restrict__ tot) {
  if (dig && (int)blockIdx.x >= (1 << dig[1])) return;   // a digit value the device digit cannot take
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n_tiles = ((int64_t)*n_dev + TILE - 1) / TILE;
  uint32_t* row = cnt + (int64_t)blockIdx.x * n_tiles_max;
  if (threadIdx.x == 0) s_carry = 0u;
  __syncthreads();
  constexpr int PER = 4;   // consecutive entries per thread
  for (int64_t b0 = 0; b0 < n_tiles; b0 += PER * 1024) {
    const int64_t b = b0 + PER * (int64_t)threadIdx.x;
    uint32_t v[PER], sum = 0u;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      v[j] = (b + j < n_tiles) ? row[b + j] : 0u;
      sum += v[j];
    }
    uint32_t x = sum;
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
    uint32_t run = s_carry + (warp ? s_w[warp - 1] : 0u) + x - sum;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      if (b + j < n_tiles) row[b + j] = run;
      run += v[j];
    }
    __syncthreads();
    if (threadIdx.x == 1023) s_carry += s_w[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = s_carry;
}

template <typename KeyT, int ITEMS = kItems>
__global__ void __launch_bounds__(kThreads, ITEMS <= 8 ? 4 : 3) k_tile_sort(const KeyT* __restrict__ keys_in,
                                                           const uint32_t* __restrict__ vals_in,
                                                           const uint8_t* __restrict__ aux_in,
                                                           KeyT* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                           uint8_t* __restrict__ aux_out,
                                                           const uint32_t* __restrict__ n_dev, int shift, int rbits,
                                                           const int32_t* __restrict__ dig,
                                                           const uint32_t* __restrict__ cnt, int64_t n_tiles_max,
                                                           const uint32_t* __restrict__ tot,
                                                           uint32_t* __restrict__ n_out) {
  constexpr int TILE = kThreads * ITEMS;
  static_assert(kWarps * kR * 2 == kThreads * 16, "one 16-byte store per thread clears the counters");
  __shared__ KeyT s_keys[TILE];
  __shared__ uint32_t s_vals[TILE];
  __shared__ uint8_t s_aux[TILE];                      // optional byte payload (aux_in non-null)
  __shared__ __align__(16) uint16_t s_whist[kWarps][kR];   // per-warp digit counts, then each
                                                           // (warp, digit)'s tile-local start
  __shared__ uint32_t s_gpos[kR];            // global position of local position 0 of digit d
  __shared__ uint32_t s_scan[kWarps];
  __shared__ uint32_t s_total;

  if (dig) {
    shift = dig[0];
    rbits = dig[1];
  }
  const int R = 1 << rbits;
  const uint32_t mask = (uint32_t)R - 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = *n_dev;
  const int64_t n_tiles = (n + TILE - 1) / TILE;
  // global position of the first key of digit d over all tiles (exclusive prefix of totals);
  // their sum is the number of keys that are not the padding sentinel, which CTA 0 reports
  const int d = threadIdx.x;
  const uint32_t dbase = block_excl_scan(d < R ? tot[d] : 0u, s_scan, &s_total);
  if (n_out && blockIdx.x == 0 && threadIdx.x == 0) *n_out = s_total;
  if ((int64_t)blockIdx.x >= n_tiles) return;   // uniform per CTA
  const unsigned lt_mask = (1u << lane) - 1u;

  // grid-stride over the tiles the device count needs (the grid is sized for the bound)
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t t0 = tile * TILE;
    const int tn = (int)min((int64_t)TILE, n - t0);
    __syncthreads();   // the previous tile's shared-memory reads are done
    reinterpret_cast<uint4*>(&s_whist[0][0])[threadIdx.x] = make_uint4(0u, 0u, 0u, 0u);

    uint32_t k[ITEMS], v[ITEMS];
    uint8_t x[ITEMS];
    uint32_t rank2[(ITEMS + 1) / 2];   // 16-bit ranks, two per register
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int li = warp * (ITEMS * 32) + i * 32 + lane;
      x[i] = 0;
      if (li < tn) {
        k[i] = (uint32_t)__ldcs(keys_in + t0 + li);
        v[i] = __ldcs(vals_in + t0 + li);
        if (aux_in) x[i] = __ldcs(aux_in + t0 + li);
      } else {
        k[i] = 0xffffffffu;   // sentinel: digit R, never counted
        v[i] = 0u;
      }
    }
    // global position of this tile's first key of digit d
    const uint32_t gfirst = d < R ? dbase + cnt[(int64_t)d * n_tiles_max + tile] : 0u;
    __syncthreads();   // counters zeroed

#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int dg = k[i] == 0xffffffffu ? R : (int)((k[i] >> shift) & mask);
      // lanes with the same digit: one match instruction for low-entropy digits (16-bit
      // tile keys repeat a lot), rbits + 1 ballots for high-entropy ones (32-bit depth and
      // Morton keys), where the match instruction's cost grows with the distinct values
      unsigned peers;
      if (sizeof(KeyT) == 2) {
        peers = __match_any_sync(0xffffffffu, dg);
      } else {
        peers = 0xffffffffu;
        for (int b = 0; b <= rbits; ++b) {   // bit rbits separates the padding digit R
          const bool bit = (dg >> b) & 1;
          const unsigned bal = __ballot_sync(0xffffffffu, bit);
          peers &= bit ? bal : ~bal;
        }
      }
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if (dg < R) base = s_whist[warp][dg];
      const uint32_t rk = base + __popc(peers & lt_mask);
      rank2[i / 2] = (i & 1) ? (rank2[i / 2] | (rk << 16)) : rk;
      __syncwarp();
      if (lane == leader && dg < R) s_whist[warp][dg] = (uint16_t)(base + __popc(peers));
      __syncwarp();
    }
    __syncthreads();
    // per digit: the warps' counts (kept in registers), the digit's tile-local start from a
    // block scan of the totals, then each (warp, digit)'s start = digit start + the counts of
    // the earlier warps (positions < TILE fit the 16-bit counters)
    uint32_t cw[kWarps], c = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      cw[w] = d < R ? s_whist[w][d] : 0u;
      c += cw[w];
    }
    const uint32_t lstart = block_excl_scan(d < R ? c : 0u, s_scan, &s_total);   // (barriers inside)
    const int tv = (int)s_total;   // the tile's keys that are not the sentinel (all of them but padding)
    if (d < R) {
      uint32_t run = lstart;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        s_whist[w][d] = (uint16_t)run;
        run += cw[w];
      }
      s_gpos[d] = gfirst - lstart;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (k[i] != 0xffffffffu) {
        const int dg = (int)((k[i] >> shift) & mask);
        const uint32_t p = s_whist[warp][dg] + ((rank2[i / 2] >> (16 * (i & 1))) & 0xffffu);
        s_keys[p] = (KeyT)k[i];
        s_vals[p] = v[i];
        if (aux_in) s_aux[p] = x[i];
      }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < tv; p += kThreads) {
      const KeyT key = s_keys[p];
      const int dd = (int)(((uint32_t)key >> shift) & mask);
      const uint32_t g = s_gpos[dd] + (uint32_t)p;
      if (keys_out) keys_out[g] = key;
      vals_out[g] = s_vals[p];
      if (aux_in) aux_out[g] = s_aux[p];
    }
  }
}

inline int64_t tiles_for(int64_t n, int tile = kTile) { return (n + tile - 1) / tile; }

// Scratch words: per-tile digit counters and the digit totals.
inline size_t scratch_words(int64_t n_max, int tile = kTile) {
  const int64_t nt = tiles_for(n_max, tile);
  return (size_t)kR * (size_t)(nt > 0 ? nt : 1) + kR;
}

// Stable sort of the first n (device count) pairs on bits [0, bits).  Buffers ping-pong
// between (k0, v0[, aux0]) and (k1, v1[, aux1]); returns 0 if the result is in the first
// set, 1 if in the second.
// n_max bounds the count (grid sizes and scratch).
// Names under which the launch tracer records the three kernels of a use of the sort.
struct SortNames {
  const char* hist;
  const char* scan;
  const char* sort;
};

// aux0 / aux1 (optional, both or neither): a byte payload that travels with each pair.
// dev_digits (optional): a device array of (shift, bits) per pass that replaces the host's
// digit plan when the kernels run (keys known on the device to need fewer bits); each pass's
// device bits must not exceed the host plan's bits for that pass.
// n_kept (optional): keys equal to the all-ones sentinel (32-bit keys) are dropped by the
// first pass, which writes the count of the others here; the later passes sort that many.
template <typename KeyT, int ITEMS = kItems>
inline int sort_pairs(KeyT* k0, uint32_t* v0, KeyT* k1, uint32_t* v1, const uint32_t* n_dev, int64_t n_max, int bits,
                      uint32_t* scratch, cudaStream_t s, bool write_last_keys, const SortNames& names,
                      uint8_t* aux0 = nullptr, uint8_t* aux1 = nullptr, const int32_t* dev_digits = nullptr,
                      uint32_t* n_kept = nullptr) {
  constexpr int TILE = kThreads * ITEMS;
  const int passes = sort_passes(bits);
  const int rbits = (bits + passes - 1) / passes;
  const int64_t nt = tiles_for(n_max, TILE) > 0 ? tiles_for(n_max, TILE) : 1;
  uint32_t* cnt = scratch;
  uint32_t* tot = scratch + (size_t)kR * nt;
  // grids sized for the bound n_max but capped at a few waves: the kernels stride over the
  // tiles of the device count, so an over-provisioned bound costs no empty CTAs
  const unsigned grid_hist = (unsigned)(nt < 8 * kNumSMs ? nt : 8 * kNumSMs);
  const unsigned grid_sort = (unsigned)(nt < 4 * kNumSMs ? nt : 4 * kNumSMs);
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * rbits;
    const int rb = (shift + rbits <= bits) ? rbits : bits - shift;
    KeyT* ki = cur ? k1 : k0;
    uint32_t* vi = cur ? v1 : v0;
    KeyT* ko = cur ? k0 : k1;
    uint32_t* vo = cur ? v0 : v1;
    const uint8_t* ai = aux0 ? (cur ? aux1 : aux0) : nullptr;
    uint8_t* ao = aux0 ? (cur ? aux0 : aux1) : nullptr;
    const bool last = (p == passes - 1);
    const int32_t* dig = dev_digits ? dev_digits + 2 * p : nullptr;
    const uint32_t* np = (n_kept && p > 0) ? n_kept : n_dev;
    {
      prof::Scope ps(names.hist, s);
      k_tile_hist<KeyT, TILE><<<grid_hist, kThreads, 0, s>>>(ki, np, shift, rb, dig, nt, cnt);
    }
    {
      prof::Scope ps(names.scan, s);
      k_tile_scan<TILE><<<1 << rb, 1024, 0, s>>>(cnt, np, dig, nt, tot);
    }
    prof::Scope ps(names.sort, s);
    k_tile_sort<KeyT, ITEMS><<<grid_sort, kThreads, 0, s>>>(
        ki, vi, ai, (last && !write_last_keys) ? nullptr : ko, vo, ao, np, shift, rb, dig, cnt, nt, tot,
        p == 0 ? n_kept : nullptr);
    cur ^= 1;
  }
  return cur;
}

}  // namespace tiles
}  // namespace rs
