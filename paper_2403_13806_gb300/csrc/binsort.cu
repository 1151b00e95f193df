// rs_bin_sort: duplicated (tile | depth) keys and a device radix sort.
//
// The 64-bit key of an instance is (global tile id) << 32 | float bits of the item's depth.
// An LSD radix sort processes the least significant digits first; the low 32 bits depend
// on the item only, so their passes are run over the N items before duplication (four
// 8-bit passes), and the expansion then emits every item's tiles in that depth order.  The
// remaining passes sort the K instances stably on the tile id alone, over only the
// ceil(log2(tiles)) significant bits.  The result -- permutation and keys -- is exactly
// that of a stable sort of the 64-bit keys emitted in item order.
//
// Pipeline (one stream, no host synchronisation; K lives in device memory):
//   k_depth_keys -> 4 depth passes (reduce-then-scan radix over the N items)
//   -> k_count_blocks -> k_count_top (K, capacity check)
//   -> k_emit (warp-cooperative expansion, coalesced stores)
//   -> tile passes (per-tile histogram, per-digit scan, per-tile stable scatter, per 8-bit digit)
//   -> memset(ranges) -> k_ranges -> [k_keys]
#include "radix_tiles.cuh"
#include "radix.cuh"
#include "profile.cuh"
#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {

constexpr int kEmitThreads = 256;

struct BinWs {
  uint32_t* dkeys[2];
  uint32_t* dvals[2];
  unsigned long long* bsum;   // per emission block: instances, then exclusive prefix
  char* tkeys[2];
  uint32_t* tvals;
  uint32_t* hist;
  uint32_t* sweep;            // per-tile digit counters of the instance sort
  uint32_t* counters;         // [0] = instances written (min(K, capacity))
  int grid_depth, grid_tile;
  size_t bytes;
};

static BinWs bin_ws_layout(void* base, int64_t n_items, int64_t capacity) {
  BinWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? static_cast<char*>(base) + off : nullptr;
    off += align_up(bytes, 256);
    return p;
  };
  const size_t ni = (size_t)(n_items > 0 ? n_items : 1);
  const size_t cap = (size_t)(capacity > 0 ? capacity : 1);
  const int64_t nblk = (n_items + kEmitThreads - 1) / kEmitThreads;
  w.grid_depth = radix::grid_for(n_items);
  w.grid_tile = radix::grid_for(capacity);
  const int hist_grid = w.grid_depth > w.grid_tile ? w.grid_depth : w.grid_tile;
  for (int i = 0; i < 2; ++i) w.dkeys[i] = reinterpret_cast<uint32_t*>(take(ni * 4));
  for (int i = 0; i < 2; ++i) w.dvals[i] = reinterpret_cast<uint32_t*>(take(ni * 4));
  w.bsum = reinterpret_cast<unsigned long long*>(take((size_t)(nblk > 0 ? nblk : 1) * 8));
  for (int i = 0; i < 2; ++i) w.tkeys[i] = take(cap * 4);   // uint16 or uint32 tile ids
  w.tvals = reinterpret_cast<uint32_t*>(take(cap * 4));
  w.hist = reinterpret_cast<uint32_t*>(take(radix::scratch_words(hist_grid) * 4));
  w.sweep = reinterpret_cast<uint32_t*>(take(tiles::scratch_words(capacity) * 4));
  w.counters = reinterpret_cast<uint32_t*>(take(64));
  w.bytes = off;
  return w;
}

__global__ void k_depth_keys(const float4* __restrict__ rgb_d, int64_t n, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = __float_as_uint(rgb_d[i].w);
  vals[i] = (uint32_t)i;
}

// Instances per block of kEmitThreads depth-sorted items.
__global__ void __launch_bounds__(kEmitThreads) k_count_blocks(const uint32_t* __restrict__ order, int64_t n,
                                                               const uint32_t* __restrict__ n_tiles,
                                                               unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long s[kEmitThreads / 32];
  const int64_t i = (int64_t)blockIdx.x * kEmitThreads + threadIdx.x;
  unsigned long long c = i < n ? (unsigned long long)n_tiles[order[i]] : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kEmitThreads / 32; ++w) t += s[w];
    bsum[blockIdx.x] = t;
  }
}

// Exclusive prefix over the block counts (one block), the instance total K, and the
// capacity check.
__global__ void __launch_bounds__(1024) k_count_top(unsigned long long* __restrict__ bsum, int64_t nblk,
                                                    int64_t capacity, uint32_t* __restrict__ counters,
                                                    rs_device_status* st) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0ull;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nblk; b0 += 1024) {
    const int64_t b = b0 + threadIdx.x;
    const unsigned long long v = b < nblk ? bsum[b] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = s_w[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_w[lane] = w;
    }
    __syncthreads();
    const unsigned long long carry = s_carry;
    const unsigned long long excl = carry + (warp ? s_w[warp - 1] : 0ull) + x - v;
    if (b < nblk) bsum[b] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = carry + s_w[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long K = s_carry;
    const unsigned long long written = K < (unsigned long long)capacity ? K : (unsigned long long)capacity;
    counters[0] = (uint32_t)written;
    if (st) {
      atomicMax(reinterpret_cast<unsigned long long*>(&st->required), K);
      st->n_instances = (int64_t)written;
      if (K > (unsigned long long)capacity) atomicCAS(&st->code, 0, (int)RS_ERR_CAPACITY);
    }
  }
}

// Expansion: each warp takes 32 consecutive depth-sorted items and writes their
// instances contiguously (tile ids row-major inside each rect); lanes locate the item of
// their instance by a binary search over the warp's inclusive prefix.
template <typename KeyT>
__global__ void __launch_bounds__(kEmitThreads) k_emit(const uint32_t* __restrict__ order, int64_t n,
                                                       const uint32_t* __restrict__ n_tiles,
                                                       const ushort4* __restrict__ rect,
                                                       const rs_view* __restrict__ views, int n_views,
                                                       const unsigned long long* __restrict__ bpre,
                                                       int64_t capacity, KeyT* __restrict__ tkeys,
                                                       uint32_t* __restrict__ tvals) {
  __shared__ uint32_t s_wtot[kEmitThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kEmitThreads + threadIdx.x;
  uint32_t item = 0, cnt = 0;
  ushort4 rc = make_ushort4(0, 0, 0, 0);
  int tile_base = 0, tiles_x = 0;
  if (i < n) {
    item = order[i];
    cnt = n_tiles[item];
    if (cnt) {
      rc = rect[item];
      const int v = find_view_by_item(views, n_views, (int64_t)item);
      tile_base = views[v].tile_base;
      tiles_x = views[v].tiles_x;
    }
  }
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
  if (lane == 0) s_wtot[warp] = wtot;
  __syncthreads();
  unsigned long long wbase = bpre[blockIdx.x];
  for (int w = 0; w < warp; ++w) wbase += s_wtot[w];
  const uint32_t excl = incl - cnt;
  const int rw = (int)rc.z - (int)rc.x;
  for (uint32_t e0 = 0; e0 < wtot; e0 += 32) {
    const uint32_t e = e0 + lane;
    int lo = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      const uint32_t v = __shfl_sync(0xffffffffu, incl, lo + s - 1);
      if (v <= e) lo += s;
    }
    const int owner = lo < 31 ? lo : 31;
    const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, owner);
    const int o_rw = __shfl_sync(0xffffffffu, rw, owner);
    const int o_x0 = __shfl_sync(0xffffffffu, (int)rc.x, owner);
    const int o_y0 = __shfl_sync(0xffffffffu, (int)rc.y, owner);
    const int o_tb = __shfl_sync(0xffffffffu, tile_base, owner);
    const int o_tx = __shfl_sync(0xffffffffu, tiles_x, owner);
    const uint32_t o_item = __shfl_sync(0xffffffffu, item, owner);
    if (e < wtot) {
      const uint32_t r = e - o_excl;
      const uint32_t ty = r / (uint32_t)o_rw;
      const uint32_t tx = r - ty * (uint32_t)o_rw;
      const unsigned long long pos = wbase + e;
      if (pos < (unsigned long long)capacity) {
        tkeys[pos] = (KeyT)((uint32_t)o_tb + (uint32_t)(o_y0 + (int)ty) * (uint32_t)o_tx + (uint32_t)(o_x0 + (int)tx));
        tvals[pos] = o_item;
      }
    }
  }
}

// Tile boundaries of the sorted tile ids: each thread owns 4 consecutive keys (one 16-byte
// load) and compares across its neighbours.  A key outside [0, n_tiles) can only come from
// a rect outside its view's tile grid and is ignored.
template <typename KeyT>
__global__ void k_ranges(const KeyT* __restrict__ tkeys, const uint32_t* __restrict__ counters,
                         uint32_t n_tiles, uint32_t* __restrict__ ranges) {
  constexpr int V = 16 / sizeof(KeyT);   // keys per 16-byte load
  const int64_t K = counters[0];
  const int64_t nq = (K + V - 1) / V;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k0 = V * q;
    uint32_t t[V];
    if (k0 + V - 1 < K) {
      const uint4 w = *reinterpret_cast<const uint4*>(tkeys + k0);
      const KeyT* kk = reinterpret_cast<const KeyT*>(&w);
#pragma unroll
      for (int j = 0; j < V; ++j) t[j] = kk[j];
    } else {
      for (int j = 0; j < V; ++j) t[j] = (k0 + j < K) ? (uint32_t)tkeys[k0 + j] : 0xffffffffu;
    }
    uint32_t prev = k0 > 0 ? (uint32_t)tkeys[k0 - 1] : 0xffffffffu;
    const uint32_t next = (k0 + V < K) ? (uint32_t)tkeys[k0 + V] : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int64_t k = k0 + j;
      if (k >= K) break;
      const uint32_t nx = (j < V - 1) ? ((k + 1 < K) ? t[j + 1] : 0xffffffffu) : next;
      if (t[j] < n_tiles) {
        if (k == 0 || prev != t[j]) ranges[2 * (int64_t)t[j]] = (uint32_t)k;
        if (k == K - 1 || nx != t[j]) ranges[2 * (int64_t)t[j] + 1] = (uint32_t)(k + 1);
      }
      prev = t[j];
    }
  }
}

template <typename KeyT>
__global__ void k_keys(const KeyT* __restrict__ tkeys, const uint32_t* __restrict__ vals,
                       const float4* __restrict__ rgb_d, const uint32_t* __restrict__ counters,
                       unsigned long long* __restrict__ keys) {
  const int64_t K = counters[0];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x)
    keys[k] = ((unsigned long long)tkeys[k] << 32) | (unsigned long long)__float_as_uint(rgb_d[vals[k]].w);
}

static int bits_for(int64_t n) {
  int b = 1;
  while (b < 32 && ((int64_t)1 << b) < n) ++b;
  return b;
}

size_t bin_sort_ws_bytes(int64_t n_items, int64_t capacity) { return bin_ws_layout(nullptr, n_items, capacity).bytes; }

// Expansion, stable sort of the instances on the tile id, ranges and optional keys, with
// tile ids held as KeyT (16-bit whenever every tile id fits).
template <typename KeyT>
static void sort_instances(const BinWs& w, const uint32_t* order, int64_t n, const rs_projected* proj,
                           const rs_view_batch* batch, const rs_bins* bins, int64_t cap, int64_t nblk,
                           uint32_t* v_first, uint32_t* v_second, rs_device_status* status, cudaStream_t s) {
  KeyT* k0 = reinterpret_cast<KeyT*>(w.tkeys[0]);
  KeyT* k1 = reinterpret_cast<KeyT*>(w.tkeys[1]);
  { prof::Scope ps("k_emit", s);
  k_emit<KeyT><<<(unsigned)nblk, kEmitThreads, 0, s>>>(order, n, proj->n_tiles,
                                                       reinterpret_cast<const ushort4*>(proj->rect), batch->views,
                                                       batch->n_views, w.bsum, cap, k0, v_first); }
  const int tbits = bits_for(batch->n_tiles);
  const int cur = tiles::sort_pairs<KeyT>(k0, v_first, k1, v_second, w.counters, cap, tbits, w.sweep, s, true);
  const KeyT* tk = cur ? k1 : k0;
  const int rgrid = 4 * kNumSMs;
  { prof::Scope ps("k_ranges", s);
  k_ranges<KeyT><<<rgrid, 256, 0, s>>>(tk, w.counters, (uint32_t)batch->n_tiles, bins->ranges); }
  prof::Scope ps("k_keys", s);
  if (bins->keys)
    k_keys<KeyT><<<rgrid, 256, 0, s>>>(tk, bins->vals, reinterpret_cast<const float4*>(proj->rgb_d), w.counters,
                                       reinterpret_cast<unsigned long long*>(bins->keys));
}

}  // namespace rs

using namespace rs;

extern "C" rs_status rs_bin_sort(const rs_projected* proj, const rs_view_batch* batch, const rs_bins* bins,
                                 void* ws, size_t ws_bytes, rs_device_status* status, void* stream) {
  if (!proj || !batch || !bins) return RS_ERR_INVALID_ARG;
  if (!bins->vals || !bins->ranges || bins->capacity <= 0 || bins->capacity >= ((int64_t)1 << 32))
    return RS_ERR_INVALID_ARG;
  if (batch->n_items < 0 || batch->n_items >= ((int64_t)1 << 32) || batch->n_tiles <= 0 || !batch->views)
    return RS_ERR_INVALID_ARG;
  if (!proj->rgb_d || !proj->rect || !proj->n_tiles) return RS_ERR_INVALID_ARG;
  const BinWs w = bin_ws_layout(ws, batch->n_items, bins->capacity);
  if (!ws || ws_bytes < w.bytes || !aligned<uint4>(ws, 256)) return RS_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = batch->n_items;
  const int64_t cap = bins->capacity;
  const float4* rgb_d = reinterpret_cast<const float4*>(proj->rgb_d);

  if (cudaMemsetAsync(w.counters, 0, 64, s) != cudaSuccess) return RS_ERR_CUDA;
  if (cudaMemsetAsync(bins->ranges, 0, (size_t)batch->n_tiles * 2 * sizeof(uint32_t), s) != cudaSuccess)
    return RS_ERR_CUDA;
  if (n == 0) {
    k_count_top<<<1, 1024, 0, s>>>(w.bsum, 0, cap, w.counters, status);
    return launch_status();
  }
  // 1) items by depth (four 8-bit passes; even count leaves the result in buffer 0)
  { prof::Scope ps("k_depth_keys", s);
  k_depth_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rgb_d, n, w.dkeys[0], w.dvals[0]); }
  radix::sort_pairs(w.dkeys[0], w.dvals[0], w.dkeys[1], w.dvals[1], n, nullptr, 32, w.hist, w.grid_depth, s, false);
  const uint32_t* order = w.dvals[0];
  // 2) instance offsets in depth order and K
  const int64_t nblk = (n + kEmitThreads - 1) / kEmitThreads;
  { prof::Scope ps("k_count_blocks", s);
  k_count_blocks<<<(unsigned)nblk, kEmitThreads, 0, s>>>(order, n, proj->n_tiles, w.bsum); }
  { prof::Scope ps("k_count_top", s);
  k_count_top<<<1, 1024, 0, s>>>(w.bsum, nblk, cap, w.counters, status); }
  // 3) expansion; the tile passes then ping-pong so that the final values land in bins->vals
  const int tbits = bits_for(batch->n_tiles);
  const int passes = radix::sort_passes(tbits);
  uint32_t* v_first = (passes % 2 == 0) ? bins->vals : w.tvals;
  uint32_t* v_second = (passes % 2 == 0) ? w.tvals : bins->vals;
  if (batch->n_tiles <= 65536)
    sort_instances<uint16_t>(w, order, n, proj, batch, bins, cap, nblk, v_first, v_second, status, s);
  else
    sort_instances<uint32_t>(w, order, n, proj, batch, bins, cap, nblk, v_first, v_second, status, s);
  return launch_status();
}
