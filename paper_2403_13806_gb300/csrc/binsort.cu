// rs_bin_sort: tile binning by duplicated 64-bit (tile | depth) keys and a device radix sort.
//
// The order to produce, per tile, is that of a stable sort of the keys
// (global tile id) << 32 | float bits of the item's depth, emitted item by item.  It is an
// LSD radix sort taken in three groups of digits:
//   1. the low 32 bits (the depth) are constant per item, so their four 8-bit passes run
//      over the N items before any duplication;
//   2. the tile id is split into a coarse digit -- the super-tile of 4 x 4 tiles that holds
//      the tile -- and a fine one.  Items are duplicated once per super-tile their rect
//      touches (about 7x fewer instances than tiles at the workload sizes) and those
//      instances are radix-sorted stably on the super-tile id (one pass per 8 bits); each
//      carries one byte, the part of the super-tile's 4 x 4 tiles its rect covers, so the
//      fine kernels below read their lists sequentially and gather nothing;
//   3. the fine digit is one stable counting pass per super-tile: each super-tile's
//      depth-ordered list is cut into segments of kSegLen entries (work in proportion to the
//      list, however unevenly the items fall on the super-tiles), and a CTA per segment
//      keeps, for each of the 4 x 4 tiles, the items whose rect covers that tile -- once to
//      count them (exclusive scans over the segments and over all tiles then give every tile
//      its range and every segment its first position in it), once to write them,
//      contiguously and in order.
// Every tile's list therefore holds its items by depth, ties to the lower item: exactly the
// order of the stable 64-bit sort.  The 64-bit keys are written only on request.
//
// Pipeline (one stream, no host synchronisation; counts live in device memory):
//   k_super_layout (super-tile bases per view); k_depth_keys, 4 depth passes over the items
//   (radix_tiles, 31-bit keys);
//   k_count_blocks, k_count_top (super total); k_emit (super instances); super passes
//   (radix_tiles); k_ranges (super ranges); k_fine_layout (segments); k_fine_count;
//   k_fine_seg_scan; k_fine_scan (ranges, K, capacity check); k_fine_scatter (vals,
//   optional keys).
#include "front_cut.cuh"
#include "profile.cuh"
#include "radix_tiles.cuh"
#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {

constexpr int kEmitThreads = 256;
// Blocks of the super-instance counting and emission: the first nb8 hold 64 depth-ranked
// items (8 per warp), the rest 256 (32 per warp).  With the occlusion cut nb8 covers the
// cut's window, so that the nearest items -- the largest, ranked first -- spread over four
// times as many warps (a warp walks all the super cells of its items); whole lists use
// nb8 = 0.
__host__ __device__ inline int64_t block_start(int64_t blk, int64_t nb8) {
  return blk < nb8 ? blk * 64 : nb8 * 64 + (blk - nb8) * 256;
}
__host__ __device__ inline int block_ipw(int64_t blk, int64_t nb8) { return blk < nb8 ? 8 : 32; }
// Blocks for n items with nb8 small blocks.
inline int64_t block_count(int64_t n, int64_t nb8) {
  return nb8 + (n > nb8 * 64 ? (n - nb8 * 64 + 255) / 256 : 0);
}
constexpr int kSuper = 4;           // tiles per super-tile side
constexpr int kFineThreads = 256;   // threads of a fine-binning CTA
constexpr int kSegLen = 3840;       // super-list entries per fine work item (segment; 15 per thread)
constexpr int kTileBlock = 256;     // tiles per CTA of the per-tile scans
constexpr int kCountChunk = 256;    // emission blocks per CTA of the block-count scan
constexpr int kNF = kSuper * kSuper;
constexpr int64_t kFrontItemsPerTile = 32;   // rs_bin_sort_front: below this, whole lists
constexpr int kCounterWords = 32;   // the device counters block (see BinWs::counters)

struct BinWs {
  uint32_t* dkeys[2];
  uint32_t* dvals[2];
  unsigned long long* bsum;   // per emission block: super instances, then exclusive prefix
  unsigned long long* csum;   // per chunk of kCountChunk emission blocks: super instances
  char* skeys[2];             // super-tile ids (uint16 or uint32)
  uint32_t* svals[2];         // items
  uint8_t* saux[2];           // covered part of the super-tile (cover byte)
  uint32_t* hist;             // per-tile digit counters of the item (depth) sort
  uint32_t* sweep;            // per-tile digit counters of the super-instance sort
  uint32_t* sranges;          // [n_tiles][2]: super-tile ranges (super-tiles never outnumber tiles)
  uint32_t* super_base;       // [n_views + 1]
  uint32_t* fine_tot;         // [n_tiles]: instances per tile, then first position
  unsigned long long* tile_blk;   // [ceil(n_tiles / kTileBlock)]: instances per block of tiles
  uint32_t* seg_off;          // [n_tiles + 1]: first segment of every super-tile, then the total
  uint32_t* work_s;           // [n_work_max]: super-tile of every segment
  uint32_t* seg_cnt;          // [n_work_max][16]: per (segment, tile) counts, then prefixes
  int64_t n_work_max;         // segments: at most capacity / kSegLen + one per super-tile
  uint32_t* cut_acc;          // [kCutBuckets][n_tiles]: occlusion bound sums (rs_bin_sort_front);
                              // cut_s follows it directly (zeroed together)
  uint32_t* cut_s;            // [n_tiles]: rank cut of every super-tile (rs_bin_sort_front)
  uint32_t* wsum;             // [blocks][kEmitThreads / 32]: kept super instances per warp (front)
  uint32_t* counters;         // [0] super instances written, [2] instances written,
                              // [4], [5] work counters of the fine count and scatter,
                              // [6] item count (the depth sort's device count), [7] segments,
                              // [8..15] the super-tile sort's digits (shift, bits) of up to
                              // four passes, [16] items the depth sort kept (those with
                              // instances), [17] the largest tile cut (rs_bin_sort_front);
                              // kCounterWords words in all
  size_t bytes;
};

static BinWs bin_ws_layout(void* base, int64_t n_items, int64_t capacity, int n_tiles, int n_views) {
  BinWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? static_cast<char*>(base) + off : nullptr;
    off += align_up(bytes > 0 ? bytes : 1, 256);
    return p;
  };
  const size_t ni = (size_t)(n_items > 0 ? n_items : 1);
  const size_t cap = (size_t)(capacity > 0 ? capacity : 1);   // super instances <= instances
  const int64_t nblk = (n_items + 63) / 64 + 2;   // at least block_count for any nb8
  for (int i = 0; i < 2; ++i) w.dkeys[i] = reinterpret_cast<uint32_t*>(take(ni * 4));
  for (int i = 0; i < 2; ++i) w.dvals[i] = reinterpret_cast<uint32_t*>(take(ni * 4));
  w.bsum = reinterpret_cast<unsigned long long*>(take((size_t)(nblk > 0 ? nblk : 1) * 8));
  w.csum = reinterpret_cast<unsigned long long*>(take((size_t)((nblk > 0 ? nblk : 1) + kCountChunk - 1) / kCountChunk * 8));
  for (int i = 0; i < 2; ++i) w.skeys[i] = take(cap * 4);
  for (int i = 0; i < 2; ++i) w.svals[i] = reinterpret_cast<uint32_t*>(take(cap * 4));
  for (int i = 0; i < 2; ++i) w.saux[i] = reinterpret_cast<uint8_t*>(take(cap));
  w.hist = reinterpret_cast<uint32_t*>(take(tiles::scratch_words(n_items) * 4));
  w.sweep = reinterpret_cast<uint32_t*>(take(tiles::scratch_words(capacity) * 4));
  w.sranges = reinterpret_cast<uint32_t*>(take((size_t)(n_tiles > 0 ? n_tiles : 1) * 8));
  w.super_base = reinterpret_cast<uint32_t*>(take((size_t)(n_views + 1) * 4));
  w.fine_tot = reinterpret_cast<uint32_t*>(take((size_t)(n_tiles > 0 ? n_tiles : 1) * 4));
  w.tile_blk = reinterpret_cast<unsigned long long*>(
      take((size_t)((n_tiles > 0 ? n_tiles : 1) + kTileBlock - 1) / kTileBlock * 8));
  w.n_work_max = (int64_t)(cap / kSegLen) + (n_tiles > 0 ? n_tiles : 1) + 1;
  w.seg_off = reinterpret_cast<uint32_t*>(take((size_t)((n_tiles > 0 ? n_tiles : 1) + 1) * 4));
  w.work_s = reinterpret_cast<uint32_t*>(take((size_t)w.n_work_max * 4));
  w.seg_cnt = reinterpret_cast<uint32_t*>(take((size_t)w.n_work_max * kNF * 4));
  w.counters = reinterpret_cast<uint32_t*>(take(kCounterWords * 4));
  w.cut_acc = reinterpret_cast<uint32_t*>(take((size_t)(n_tiles > 0 ? n_tiles : 1) * kCutBuckets * 4));
  w.cut_s = reinterpret_cast<uint32_t*>(take((size_t)(n_tiles > 0 ? n_tiles : 1) * 4));
  w.wsum = reinterpret_cast<uint32_t*>(take((size_t)(nblk > 0 ? nblk : 1) * (kEmitThreads / 32) * 4));
  w.bytes = off;
  return w;
}

__device__ __forceinline__ int super_w(const rs_view& v) { return (v.tiles_x + kSuper - 1) / kSuper; }
__device__ __forceinline__ int super_h(const rs_view& v) { return (v.tiles_y + kSuper - 1) / kSuper; }

// Depth sort keys: the FP32 depth bits with the sign bit cleared.  Every item that emits
// instances has depth > near_plane > 0, whose bits order like the value and are unchanged,
// and no such key equals the sort's all-ones sentinel.  Items that emit nothing (culled, or
// off the image: n_tiles = 0) get the sentinel, which the first sort pass drops, so the
// later passes and the emission order only the items that have instances.
// For rs_bin_sort_front the grid also zeroes the occlusion cut's bound sums and super-tile
// cuts (z, nz 16-byte words; nullptr / 0 otherwise), which the cut kernels use next.
__global__ void k_depth_keys(const float4* __restrict__ rgb_d, const uint32_t* __restrict__ n_tiles, int64_t n,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint4* __restrict__ z,
                             int64_t nz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t k = i; k < nz; k += (int64_t)gridDim.x * blockDim.x) z[k] = make_uint4(0u, 0u, 0u, 0u);
  if (i >= n) return;
  keys[i] = n_tiles[i] ? (__float_as_uint(rgb_d[i].w) & 0x7fffffffu) : 0xffffffffu;
  vals[i] = (uint32_t)i;
}

// First super-tile id of every view (exclusive prefix of the views' super-tile counts), the
// item count as the depth sort's device count, and the digits of the super-tile sort.  The
// host plans its passes for a bound on the ids (host_bits, from the tile count): P passes
// of tiles::sort_passes' widths.  The ids actually need b <= host_bits bits; the device
// digits are as even as the host widths allow (each at most ceil(b / P) and at most the
// host's width for that pass, any shortfall added to the earliest passes with room), so
// they cover the b bits and the host's launch grids cover every digit value.
// A batch whose n_tiles is below its views' tile count (only a hand-built rs_view_batch can
// be) would need more tiles and super-tiles than the per-tile arrays, ranges and segment
// tables hold: it is reported as RS_ERR_INVALID_ARG in the device status and binned as if no
// view had a super-tile (no fine work items, every tile list empty), with every access in
// bounds.
__global__ void k_super_layout(const rs_view* __restrict__ views, int n_views, uint32_t* __restrict__ super_base,
                               int64_t n_items, uint32_t* __restrict__ n_dev, int host_bits,
                               int32_t* __restrict__ digits, int64_t n_tiles, rs_device_status* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  *n_dev = (uint32_t)n_items;
  uint64_t run = 0, tiles = 0;
  for (int v = 0; v < n_views; ++v) {
    super_base[v] = (uint32_t)run;
    run += (uint64_t)super_w(views[v]) * (uint64_t)super_h(views[v]);
    tiles += (uint64_t)views[v].tiles_x * (uint64_t)views[v].tiles_y;
  }
  if (tiles > (uint64_t)n_tiles) {   // (super-tiles never outnumber tiles)
    if (st) atomicCAS(&st->code, 0, (int)RS_ERR_INVALID_ARG);
    for (int v = 0; v < n_views; ++v) super_base[v] = 0;
    run = 0;
  }
  super_base[n_views] = (uint32_t)run;
  int b = 1;
  while (b < 32 && (1u << b) < run) ++b;
  const int P = tiles::sort_passes(host_bits);   // at most 4
  const int rh = (host_bits + P - 1) / P;
  int width[4], dv[4], used = 0;
  for (int p = 0; p < P; ++p) {
    width[p] = (p * rh + rh <= host_bits) ? rh : host_bits - p * rh;
    dv[p] = min(width[p], (b + P - 1) / P);
    used += dv[p];
  }
  for (int p = 0; p < P && used < b; ++p) {
    const int add = min(b - used, width[p] - dv[p]);
    dv[p] += add;
    used += add;
  }
  for (int p = 0, shift = 0; p < P; ++p) {
    digits[2 * p] = shift;
    digits[2 * p + 1] = dv[p];
    shift += dv[p];
  }
}

// Super-tile rect of an item's tile rect (both half-open).
__device__ __forceinline__ ushort4 super_rect(ushort4 r) {
  if (r.z <= r.x || r.w <= r.y) return make_ushort4(0, 0, 0, 0);
  return make_ushort4(r.x / kSuper, r.y / kSuper, (r.z - 1) / kSuper + 1, (r.w - 1) / kSuper + 1);
}

// Cover byte: the tiles of a super-tile that an item's tile rect covers, as the first and
// last covered column (bits 0-1, 2-3) and row (bits 4-5, 6-7) inside its 4 x 4 block.  The
// rect touches the super-tile and lies inside the view's tile grid, so every field is in
// 0..3; k_emit writes one per super instance.
// Bit (fy * kSuper + fx) set for every tile of the block that a cover byte covers.
__device__ __forceinline__ uint32_t cover_mask(uint32_t c) {
  const int x0 = c & 3, x1 = (c >> 2) & 3, y0 = (c >> 4) & 3, y1 = c >> 6;
  const uint32_t row = (2u << x1) - (1u << x0);                      // bits x0 .. x1
  const uint32_t rep = 0x1111u >> (kSuper * (kSuper - 1 - (y1 - y0)));   // y1 - y0 + 1 rows, one bit each
  return (row * rep) << (kSuper * y0);                               // row repeated on rows y0 .. y1
}

// Per-lane data of one depth-ranked item for its expansion into super instances.
struct SuperItem {
  uint32_t item = 0;
  uint32_t cnt = 0;     // cells of its super rect (0: no item)
  uint32_t sbase = 0;   // the view's first super-tile id
  uint32_t org = 0;     // super rect origin: x | y << 16
  uint32_t dims = 1;    // super rect width | view's super-tile row length << 16
  uint32_t edge = 0;    // cover fields of the rect's first/last super column and row | rows << 8
};

__device__ __forceinline__ SuperItem super_item(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect,
                                                const rs_view* __restrict__ views, int n_views,
                                                const uint32_t* __restrict__ super_base, int64_t i, bool live) {
  SuperItem s;
  if (!live) return s;
  s.item = order[i];
  const ushort4 tr = rect[s.item];
  const ushort4 sr = super_rect(tr);
  s.cnt = (uint32_t)(sr.z - sr.x) * (uint32_t)(sr.w - sr.y);
  if (s.cnt) {
    const int v = find_view_by_item(views, n_views, (int64_t)s.item);
    s.sbase = super_base[v];
    s.org = (uint32_t)sr.x | ((uint32_t)sr.y << 16);
    s.dims = (uint32_t)(sr.z - sr.x) | ((uint32_t)super_w(views[v]) << 16);
    // first covered column inside the first super column, last inside the last one, etc.
    const uint32_t fx0 = tr.x - kSuper * sr.x, fx1 = tr.z - 1 - kSuper * (sr.z - 1);
    const uint32_t fy0 = tr.y - kSuper * sr.y, fy1 = tr.w - 1 - kSuper * (sr.w - 1);
    s.edge = fx0 | (fx1 << 2) | (fy0 << 4) | (fy1 << 6) | ((uint32_t)(sr.w - sr.y) << 8);
  }
  return s;
}

// Cell e of a warp's expansion: the lane whose item owns it (a binary search over the
// warp's inclusive prefix of cell counts), and its super-tile id and place in the owner's
// super rect.  The owner's data travels in shuffles (packed 16-bit fields); the row inside
// the rect comes from a float reciprocal with an exact integer correction.  Every lane of
// the warp must call it; the result is meaningful for e < the warp's total only.
struct SuperCell {
  int owner;
  uint32_t item, sid, tx, ty, rw, edge;
};

__device__ __forceinline__ SuperCell super_cell(const SuperItem& s, uint32_t incl, uint32_t excl, uint32_t e) {
  SuperCell c;
  int lo = 0;
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1) {
    const uint32_t v = __shfl_sync(0xffffffffu, incl, lo + sh - 1);
    if (v <= e) lo += sh;
  }
  c.owner = lo < 31 ? lo : 31;
  const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, c.owner);
  c.item = __shfl_sync(0xffffffffu, s.item, c.owner);
  const uint32_t o_sb = __shfl_sync(0xffffffffu, s.sbase, c.owner);
  const uint32_t o_org = __shfl_sync(0xffffffffu, s.org, c.owner);
  const uint32_t o_dims = __shfl_sync(0xffffffffu, s.dims, c.owner);
  c.edge = __shfl_sync(0xffffffffu, s.edge, c.owner);
  const uint32_t r = e - o_excl;
  c.rw = o_dims & 0xffffu;   // >= 1
  // ty = r / rw: the float estimate is within one of the quotient, then corrected
  uint32_t ty = (uint32_t)(((float)r + 0.5f) * rcp_approx((float)c.rw));
  if (ty * c.rw > r) --ty;
  if ((ty + 1u) * c.rw <= r) ++ty;
  c.ty = ty;
  c.tx = r - ty * c.rw;
  c.sid = o_sb + ((o_org >> 16) + ty) * (o_dims >> 16) + (o_org & 0xffffu) + c.tx;
  return c;
}

// With the occlusion cut: whether super instance (item of depth rank `rank`, super-tile
// sid) is kept, i.e. the super-tile's rank cut lies beyond the item.
__device__ __forceinline__ bool super_kept(uint32_t sid, uint32_t rank, uint32_t n_super, const uint32_t* cut_s) {
  return sid < n_super && rank < cut_s[sid];   // n_super is 0 for a rejected batch
}

// The super-tiles' rank cuts as the keep tests read them: a copy in shared memory (s) when
// they fit, else the global array.  Contains a barrier: every thread of the CTA calls it.
constexpr uint32_t kCutSmem = 8192;
__device__ __forceinline__ const uint32_t* stage_cuts(const uint32_t* __restrict__ cut_s, uint32_t n_super,
                                                      uint32_t* s) {
  if (n_super > kCutSmem) return cut_s;
  for (uint32_t k = threadIdx.x; k < n_super; k += blockDim.x) s[k] = cut_s[k];
  __syncthreads();
  return s;
}

// Super instances per block of depth-sorted items (block_start, block_ipw), also added into
// the total of the block's chunk of kCountChunk blocks (csum, zeroed by the caller).  CUT:
// only the instances that k_emit keeps (super_kept), counted by a warp-wide walk over the
// cells of the warp's items, per warp into wsum as well; blocks whose items all lie beyond
// the largest cut end at once.
template <bool CUT>
__global__ void __launch_bounds__(kEmitThreads) k_count_blocks(const uint32_t* __restrict__ order,
                                                               const uint32_t* __restrict__ n_dev,
                                                               const ushort4* __restrict__ rect,
                                                               const rs_view* __restrict__ views, int n_views,
                                                               const uint32_t* __restrict__ super_base,
                                                               const uint32_t* __restrict__ cut_s,
                                                               const uint32_t* __restrict__ cut_max, int64_t nb8,
                                                               unsigned long long* __restrict__ bsum,
                                                               unsigned long long* __restrict__ csum,
                                                               uint32_t* __restrict__ wsum) {
  __shared__ unsigned long long s[kEmitThreads / 32];
  __shared__ uint32_t s_cut[CUT ? kCutSmem : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = *n_dev;   // the items the depth sort kept (those with instances)
  const int64_t lim = CUT ? min(n, (int64_t)*cut_max) : n;
  const int64_t blk = blockIdx.x;
  // CUT: a block at or beyond the largest cut keeps nothing (k_count_top reads its count as 0)
  if (CUT && block_start(blk, nb8) >= lim) return;   // uniform per CTA
  const uint32_t ns = CUT ? super_base[n_views] : 0u;
  const uint32_t* cuts = CUT ? stage_cuts(cut_s, ns, s_cut) : cut_s;
  const int ipw = block_ipw(blk, nb8);
  {
    const int64_t first = block_start(blk, nb8) + warp * ipw;   // the warp's first item (rank)
    const int64_t i = first + lane;                             // this lane's item, for lane < ipw
    unsigned long long c = 0;
    if (!CUT) {
      if (i < n) {   // (nb8 = 0: 32 items per warp, i = block start + threadIdx.x)
        const ushort4 sr = super_rect(rect[order[i]]);
        c = (unsigned long long)(sr.z - sr.x) * (unsigned long long)(sr.w - sr.y);
      }
    } else {
      const SuperItem si = super_item(order, rect, views, n_views, super_base, i, lane < ipw && i < lim);
      uint32_t incl = si.cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t excl = incl - si.cnt;
      const uint32_t first_rank = (uint32_t)first;
      uint32_t kept = 0;
      for (uint32_t e0 = 0; e0 < wtot; e0 += 32) {   // uniform per warp
        const SuperCell sc = super_cell(si, incl, excl, e0 + lane);
        const bool keep = e0 + lane < wtot && super_kept(sc.sid, first_rank + (uint32_t)sc.owner, ns, cuts);
        kept += (uint32_t)__popc(__ballot_sync(0xffffffffu, keep));
      }
      if (lane == 0) wsum[blk * (kEmitThreads / 32) + warp] = kept;
      c = lane == 0 ? kept : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) s[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kEmitThreads / 32; ++w) t += s[w];
      bsum[blk] = t;
      if (t) atomicAdd(csum + blk / kCountChunk, t);
    }
  }
}

// Sum of one value per thread over a 256-thread CTA (every thread receives it).
__device__ __forceinline__ unsigned long long block_sum256_u64(unsigned long long v, unsigned long long* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  unsigned long long t = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += s_w[w];
  __syncthreads();
  return t;
}

// Exclusive prefix of the chunk totals csum[0 .. n_chunks) in place (one CTA, 4 entries
// per thread per round, a carry between rounds).
__global__ void __launch_bounds__(1024) k_count_chunks(unsigned long long* __restrict__ csum, int64_t n_chunks) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0ull;
  __syncthreads();
  for (int64_t c0 = 0; c0 < n_chunks; c0 += 4 * 1024) {
    const int64_t c = c0 + 4 * (int64_t)threadIdx.x;
    unsigned long long v[4], sum = 0ull;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = c + j < n_chunks ? csum[c + j] : 0ull;
      sum += v[j];
    }
    unsigned long long x = sum;
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
    unsigned long long run = s_carry + (warp ? s_w[warp - 1] : 0ull) + x - sum;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (c + j < n_chunks) csum[c + j] = run;
      run += v[j];
    }
    __syncthreads();
    if (threadIdx.x == 1023) s_carry += s_w[31];
    __syncthreads();
  }
}

// Exclusive prefix over the block counts, one CTA per chunk of kCountChunk blocks: the
// chunk's base is the scanned total of the earlier chunks, the blocks' places inside it a
// CTA scan.  The CTA of the last block writes the super-instance total.
// (With the occlusion cut, blocks starting at or beyond the device limit min(*n_dev,
// *cut_max) count 0 -- k_count_blocks leaves them; csum holds the chunks' exclusive
// prefix, from k_count_chunks.)
__global__ void __launch_bounds__(kCountChunk) k_count_top(unsigned long long* __restrict__ bsum,
                                                           const unsigned long long* __restrict__ csum, int64_t nblk,
                                                           int64_t capacity, uint32_t* __restrict__ counters,
                                                           rs_device_status* st, const uint32_t* __restrict__ n_dev,
                                                           const uint32_t* __restrict__ cut_max, int64_t nb8) {
  static_assert(kCountChunk == 256, "one thread per block of the chunk");
  __shared__ unsigned long long s_w[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long base = csum[blockIdx.x];
  const int64_t lim = cut_max ? min((int64_t)*n_dev, (int64_t)*cut_max) : INT64_MAX;
  const int64_t b = (int64_t)blockIdx.x * kCountChunk + threadIdx.x;
  const unsigned long long v = (b < nblk && block_start(b, nb8) < lim) ? bsum[b] : 0ull;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  unsigned long long wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += s_w[w];
  const unsigned long long run = base + wpre + x - v;
  if (b < nblk) bsum[b] = run;
  if (b == nblk - 1) {
    // super instances never outnumber instances: more than the capacity means the instances
    // overflow too (k_fine_scan records the required count)
    const unsigned long long Ks = run + v;
    counters[0] = (uint32_t)(Ks < (unsigned long long)capacity ? Ks : (unsigned long long)capacity);
    if (st && Ks > (unsigned long long)capacity) atomicCAS(&st->code, 0, (int)RS_ERR_CAPACITY);
  }
}

// Expansion into super instances: each warp takes 8 or 32 consecutive depth-sorted items
// (block_start, block_ipw) and
// writes their super-tile ids, items and cover bytes contiguously (row-major inside each
// super rect), 32 cells per round (super_cell); the cover byte comes from the four edge
// offsets of the rect (inner super-tiles are covered whole).  CUT: only the kept instances
// (super_kept) are written, packed in the same order by a warp ballot per round, from the
// warp's base given by k_count_blocks' per-warp counts.
template <typename KeyT, bool CUT>
__global__ void __launch_bounds__(kEmitThreads) k_emit(const uint32_t* __restrict__ order,
                                                       const uint32_t* __restrict__ n_dev,
                                                       const ushort4* __restrict__ rect,
                                                       const rs_view* __restrict__ views, int n_views,
                                                       const uint32_t* __restrict__ super_base,
                                                       const uint32_t* __restrict__ cut_s,
                                                       const uint32_t* __restrict__ cut_max, int64_t nb8,
                                                       const unsigned long long* __restrict__ bpre, int64_t capacity,
                                                       const uint32_t* __restrict__ wsum,
                                                       KeyT* __restrict__ skeys, uint32_t* __restrict__ svals,
                                                       uint8_t* __restrict__ saux) {
  __shared__ uint32_t s_wtot[kEmitThreads / 32];
  __shared__ uint32_t s_cut[CUT ? kCutSmem : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = *n_dev;   // the items the depth sort kept (those with instances)
  const int64_t lim = CUT ? min(n, (int64_t)*cut_max) : n;
  const int64_t blk = blockIdx.x;
  if (CUT && block_start(blk, nb8) >= lim) return;   // uniform per CTA: nothing kept
  const uint32_t ns = CUT ? super_base[n_views] : 0u;
  const uint32_t* cuts = CUT ? stage_cuts(cut_s, ns, s_cut) : nullptr;
  const int ipw = block_ipw(blk, nb8);
  {
    const int64_t first = block_start(blk, nb8) + warp * ipw;   // the warp's first item (rank)
    const int64_t i = first + lane;                             // this lane's item, for lane < ipw
    const SuperItem si = super_item(order, rect, views, n_views, super_base, i, lane < ipw && i < lim);
    uint32_t incl = si.cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - si.cnt;
    const uint32_t first_rank = (uint32_t)first;
    if (lane == 0) s_wtot[warp] = CUT ? wsum[blk * (kEmitThreads / 32) + warp] : wtot;
    __syncthreads();
    unsigned long long wbase = bpre[blk];
    for (int w = 0; w < warp; ++w) wbase += s_wtot[w];
    uint32_t run = 0;   // CUT: instances the warp wrote in earlier rounds
    for (uint32_t e0 = 0; e0 < wtot; e0 += 32) {
      const uint32_t e = e0 + lane;
      const SuperCell sc = super_cell(si, incl, excl, e);
      const bool keep = e < wtot && (!CUT || super_kept(sc.sid, first_rank + (uint32_t)sc.owner, ns, cuts));
      unsigned long long pos = wbase + e;
      if (CUT) {
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        pos = wbase + run + (uint32_t)__popc(bal & ((1u << lane) - 1u));
        run += (uint32_t)__popc(bal);
      }
      if (keep && pos < (unsigned long long)capacity) {
        skeys[pos] = (KeyT)sc.sid;
        svals[pos] = sc.item;
        const uint32_t rh = sc.edge >> 8;
        const uint32_t lx0 = sc.tx == 0 ? (sc.edge & 3u) : 0u;
        const uint32_t lx1 = sc.tx == sc.rw - 1 ? ((sc.edge >> 2) & 3u) : 3u;
        const uint32_t ly0 = sc.ty == 0 ? ((sc.edge >> 4) & 3u) : 0u;
        const uint32_t ly1 = sc.ty == rh - 1 ? ((sc.edge >> 6) & 3u) : 3u;
        saux[pos] = (uint8_t)(lx0 | (lx1 << 2) | (ly0 << 4) | (ly1 << 6));
      }
    }
  }
}

// Range of every key value of a sorted key array (16-byte loads; keys >= n_keys ignored).
template <typename KeyT>
__global__ void k_ranges(const KeyT* __restrict__ tkeys, const uint32_t* __restrict__ counters, uint32_t n_keys,
                         uint32_t* __restrict__ ranges) {
  constexpr int V = 16 / sizeof(KeyT);
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
      if (t[j] < n_keys) {
        if (k == 0 || prev != t[j]) ranges[2 * (int64_t)t[j]] = (uint32_t)k;
        if (k == K - 1 || nx != t[j]) ranges[2 * (int64_t)t[j] + 1] = (uint32_t)(k + 1);
      }
      prev = t[j];
    }
  }
}

// The super-tile a CTA works on: its view, its first tile, the extent of its block of tiles
// (up to kSuper x kSuper), and its range of sorted super instances.
struct SuperTile {
  int v;
  int tx0, ty0, nx, ny;
  uint32_t s0, s1;
  bool valid;
};

__device__ __forceinline__ SuperTile super_tile(uint32_t S, const rs_view* views, int n_views,
                                                const uint32_t* super_base, const uint32_t* sranges) {
  SuperTile t;
  t.valid = S < super_base[n_views];
  if (!t.valid) return t;
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (super_base[mid] <= S) lo = mid; else hi = mid - 1;
  }
  t.v = lo;
  const rs_view& cam = views[t.v];
  const int local = (int)(S - super_base[t.v]);
  const int sw = super_w(cam);
  const int sy = local / sw, sx = local - sy * sw;
  t.tx0 = sx * kSuper;
  t.ty0 = sy * kSuper;
  t.nx = min(kSuper, cam.tiles_x - t.tx0);
  t.ny = min(kSuper, cam.tiles_y - t.ty0);
  t.s0 = sranges[2 * (int64_t)S];
  t.s1 = sranges[2 * (int64_t)S + 1];
  return t;
}

// Segment j of super-tile S's list: entries [s0 + j kSegLen, s0 + (j + 1) kSegLen) of it.
__device__ __forceinline__ void segment(const SuperTile& t, uint32_t j, uint32_t& a, uint32_t& b) {
  a = min(t.s0 + j * (uint32_t)kSegLen, t.s1);
  b = min(a + (uint32_t)kSegLen, t.s1);
}

// Segments of the super-tile lists (one CTA): seg_off[S] = first segment of super-tile S
// (exclusive prefix of ceil(len / kSegLen)), seg_off[n_super] = the total, work_s[w] = the
// super-tile of segment w, counters[7] = the number of segments (the fine work items).
__global__ void __launch_bounds__(1024) k_fine_layout(const uint32_t* __restrict__ super_base, int n_views,
                                                      const uint32_t* __restrict__ sranges,
                                                      uint32_t* __restrict__ seg_off, uint32_t* __restrict__ work_s,
                                                      int64_t n_work_max, uint32_t* __restrict__ counters) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_super = (int)super_base[n_views];
  if (threadIdx.x == 0) s_carry = 0u;
  __syncthreads();
  for (int b0 = 0; b0 < n_super; b0 += 4 * 1024) {
    const int b = b0 + 4 * (int)threadIdx.x;
    uint32_t v[4], sum = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = (b + j < n_super) ? (sranges[2 * (b + j) + 1] - sranges[2 * (b + j)] + kSegLen - 1) / kSegLen : 0u;
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
    for (int j = 0; j < 4; ++j) {
      if (b + j < n_super) {
        seg_off[b + j] = run;
        for (uint32_t k = 0; k < v[j]; ++k)
          if ((int64_t)(run + k) < n_work_max) work_s[run + k] = (uint32_t)(b + j);
      }
      run += v[j];
    }
    __syncthreads();
    if (threadIdx.x == 1023) s_carry += s_w[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    seg_off[n_super] = s_carry;
    counters[7] = (uint32_t)min((int64_t)s_carry, n_work_max);
  }
}

// Work items of the fine kernels are the segments, handed out in order from a device counter
// to a grid of at most a few CTAs per SM (their number is only known on the device).  Every
// thread of the CTA receives the same item.
__device__ __forceinline__ uint32_t next_work(uint32_t* ctr, uint32_t* s_slot) {
  __syncthreads();   // the previous item's use of shared memory is over
  if (threadIdx.x == 0) *s_slot = atomicAdd(ctr, 1u);
  __syncthreads();
  return *s_slot;
}

// Instances per (segment, tile): each work item reads the cover bytes of one segment of a
// super-tile's depth-ordered list once and counts, for each of the 4 x 4 tiles, the items
// covering it.  A thread keeps its counts as 16 four-bit fields in two words (it sees at
// most kSegLen / kFineThreads < 16 entries of a segment) and adds one shared-memory table
// row per entry -- the cover byte's tiles as ones in their fields -- so an entry costs a
// load and two adds; the fields are unpacked and summed over the CTA once per segment.
static_assert(kSegLen / kFineThreads < 16, "four-bit per-thread tile counts");

__global__ void __launch_bounds__(kFineThreads) k_fine_count(const uint8_t* __restrict__ saux,
                                                             const rs_view* __restrict__ views, int n_views,
                                                             const uint32_t* __restrict__ super_base,
                                                             const uint32_t* __restrict__ sranges,
                                                             const uint32_t* __restrict__ seg_off,
                                                             const uint32_t* __restrict__ work_s,
                                                             const uint32_t* __restrict__ n_work_dev,
                                                             uint32_t* __restrict__ seg_cnt, uint32_t* __restrict__ ctr) {
  constexpr int NW = kFineThreads / 32;
  __shared__ uint2 s_tab[256];   // cover byte -> (tiles 0-7, tiles 8-15) as four-bit ones
  __shared__ uint32_t s_cnt[NW][kNF];
  __shared__ uint32_t s_w;
  for (int c = threadIdx.x; c < 256; c += kFineThreads) {
    const uint32_t m = cover_mask((uint32_t)c);
    uint32_t lo = 0u, hi = 0u;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      lo |= ((m >> f) & 1u) << (4 * f);
      hi |= ((m >> (f + 8)) & 1u) << (4 * f);
    }
    s_tab[c] = make_uint2(lo, hi);
  }
  const uint32_t n_work = *n_work_dev;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t wi = next_work(ctr, &s_w); wi < n_work; wi = next_work(ctr, &s_w)) {
    const uint32_t S = work_s[wi];
    const uint32_t j = wi - seg_off[S];
    const SuperTile t = super_tile(S, views, n_views, super_base, sranges);
    uint32_t a, b;
    segment(t, j, a, b);
    uint32_t lo = 0u, hi = 0u;
    constexpr int U = kSegLen / kFineThreads;   // every load of the segment in flight at once
    uint32_t cb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t e = a + u * kFineThreads + threadIdx.x;
      cb[u] = e < b ? (uint32_t)__ldcs(saux + e) : 0x100u;   // 0x100: past the segment
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (cb[u] < 0x100u) {
        const uint2 r = s_tab[cb[u]];
        lo += r.x;
        hi += r.y;
      }
    }
    uint32_t mine = 0u;
#pragma unroll
    for (int f = 0; f < kNF; ++f) {
      const uint32_t v = ((f < 8 ? lo : hi) >> (4 * (f & 7))) & 15u;
      const uint32_t tot = __reduce_add_sync(0xffffffffu, v);
      mine = (lane == f) ? tot : mine;
    }
    if (lane < kNF) s_cnt[warp][lane] = mine;
    __syncthreads();
    if (threadIdx.x < kNF) {
      uint32_t tot = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) tot += s_cnt[w][threadIdx.x];
      seg_cnt[(int64_t)wi * kNF + threadIdx.x] = tot;
    }
  }
}

static_assert(kTileBlock == 256, "the per-tile scans use the 256-thread CTA sum");

// One thread per tile: exclusive prefix of its counts over its super-tile's segments (in
// place, four segments' loads at a time), the tile's total, and the total of each block of
// kTileBlock tiles.
__global__ void __launch_bounds__(kTileBlock) k_fine_seg_scan(uint32_t* __restrict__ seg_cnt,
                                                              const rs_view* __restrict__ views, int n_views,
                                                              const uint32_t* __restrict__ super_base,
                                                              const uint32_t* __restrict__ seg_off, int n_tiles,
                                                              uint32_t* __restrict__ fine_tot,
                                                              unsigned long long* __restrict__ tile_blk) {
  __shared__ unsigned long long s_w[kTileBlock / 32];
  const int T = blockIdx.x * kTileBlock + threadIdx.x;
  uint32_t run = 0;
  if (T < n_tiles) {
    const int v = find_view_by_tile(views, n_views, T);
    const rs_view& cam = views[v];
    const int local = T - cam.tile_base;
    const int ty = local / cam.tiles_x, tx = local - ty * cam.tiles_x;
    const uint32_t S = super_base[v] + (uint32_t)((ty / kSuper) * super_w(cam) + tx / kSuper);
    const int f = (ty % kSuper) * kSuper + tx % kSuper;
    // (S is below the super-tile count unless k_super_layout rejected the batch)
    const bool ok = S < super_base[n_views];
    const uint32_t w0 = ok ? seg_off[S] : 0u, w1 = ok ? seg_off[S + 1] : 0u;
    for (uint32_t w = w0; w < w1; w += 4) {
      uint32_t x[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = w + k < w1 ? seg_cnt[(int64_t)(w + k) * kNF + f] : 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (w + k < w1) seg_cnt[(int64_t)(w + k) * kNF + f] = run;
        run += x[k];
      }
    }
    fine_tot[T] = run;
  }
  const unsigned long long b = block_sum256_u64(run, s_w);
  if (threadIdx.x == 0) tile_blk[blockIdx.x] = b;
}

// Exclusive scan of the per-tile totals, one CTA per block of kTileBlock tiles: the block's
// base is the sum of the earlier blocks' totals (read by the whole CTA), the tiles' places
// inside it a block scan.  Writes every tile's first position (in place, saturated to 32
// bits) and its range clamped to the capacity; the CTA of the last tile writes K and
// checks the capacity.
__global__ void __launch_bounds__(kTileBlock) k_fine_scan(uint32_t* __restrict__ tot,
                                                          const unsigned long long* __restrict__ tile_blk,
                                                          int n_tiles, int64_t capacity, uint32_t* __restrict__ ranges,
                                                          uint32_t* __restrict__ counters, rs_device_status* st) {
  __shared__ unsigned long long s_w[kTileBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long cap = (unsigned long long)capacity;
  unsigned long long pre = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += kTileBlock) pre += tile_blk[b];
  const unsigned long long base = block_sum256_u64(pre, s_w);
  const int T = blockIdx.x * kTileBlock + threadIdx.x;
  const unsigned long long v = T < n_tiles ? tot[T] : 0ull;
  // exclusive scan of v over the CTA
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  unsigned long long wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += s_w[w];
  const unsigned long long run = base + wpre + x - v, e = run + v;
  if (T < n_tiles) {
    tot[T] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
    ranges[2 * (int64_t)T] = (uint32_t)(run < cap ? run : cap);
    ranges[2 * (int64_t)T + 1] = (uint32_t)(e < cap ? e : cap);
  }
  if (T == n_tiles - 1) {
    const unsigned long long K = e;
    counters[2] = (uint32_t)(K < cap ? K : cap);
    if (st) {
      atomicMax(reinterpret_cast<unsigned long long*>(&st->required), K);
      st->n_instances = (int64_t)(K < cap ? K : cap);
      if (K > cap) atomicCAS(&st->code, 0, (int)RS_ERR_CAPACITY);
    }
  }
}

// Every tile's items, in its super-tile list order, written contiguously: each CTA takes one
// segment of a super-tile's list and writes, for each of its tiles, the covering items from
// that tile's first position plus the counts of the earlier segments.  Per chunk of
// kFineThreads entries, an entry's rank among the warp's entries covering tile f is byte f of
// a warp-wide exclusive scan of 16-byte vectors (a shared-memory table row per cover byte:
// byte f = 1 if the entry covers tile f; no byte exceeds 32), the warps' totals give each
// (warp, tile) its first position, and each entry then stores its item once per tile it
// covers.  KEYS: also write the 64-bit (tile << 32 | depth bits) keys.
template <bool KEYS>
__global__ void __launch_bounds__(kFineThreads) k_fine_scatter(const uint32_t* __restrict__ svals,
                                                               const uint8_t* __restrict__ saux,
                                                               const float4* __restrict__ rgb_d,
                                                               const rs_view* __restrict__ views, int n_views,
                                                               const uint32_t* __restrict__ super_base,
                                                               const uint32_t* __restrict__ sranges,
                                                               const uint32_t* __restrict__ fine_start,
                                                               const uint32_t* __restrict__ seg_off,
                                                               const uint32_t* __restrict__ work_s,
                                                               const uint32_t* __restrict__ n_work_dev,
                                                               const uint32_t* __restrict__ seg_pre, int64_t capacity,
                                                               uint32_t* __restrict__ vals,
                                                               unsigned long long* __restrict__ keys,
                                                               uint32_t* __restrict__ ctr) {
  constexpr int NW = kFineThreads / 32;
  __shared__ uint4 s_tab[256];                       // cover byte -> byte f = covers tile f
  __shared__ uint4 s_wtot[NW];                       // per warp: covering entries per tile (bytes)
  __shared__ __align__(16) uint32_t s_base[NW][kNF];   // first position of each (warp, tile) in this chunk
  __shared__ uint32_t s_run[kNF];                    // next position of each tile
  __shared__ uint32_t s_tile[kNF];                   // global id of each tile
  __shared__ uint32_t s_w;
  for (int c = threadIdx.x; c < 256; c += kFineThreads) {
    const uint32_t m = cover_mask((uint32_t)c);
    uint32_t wd[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int f = 0; f < kNF; ++f) wd[f >> 2] |= ((m >> f) & 1u) << (8 * (f & 3));
    s_tab[c] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
  }
  const uint32_t n_work = *n_work_dev;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t cap = (uint32_t)(capacity < 0xffffffffLL ? capacity : 0xffffffffLL);
  for (uint32_t wi = next_work(ctr, &s_w); wi < n_work; wi = next_work(ctr, &s_w)) {
    const uint32_t S = work_s[wi];
    const uint32_t j = wi - seg_off[S];
    const SuperTile t = super_tile(S, views, n_views, super_base, sranges);
    uint32_t a, b;
    segment(t, j, a, b);
    if (threadIdx.x < kNF) {
      const int f = threadIdx.x, fx = f % kSuper, fy = f / kSuper;
      const rs_view& cam = views[t.v];
      const bool in = fx < t.nx && fy < t.ny;
      const uint32_t T = in ? (uint32_t)(cam.tile_base + (t.ty0 + fy) * cam.tiles_x + t.tx0 + fx) : 0u;
      s_tile[f] = T;
      s_run[f] = in ? fine_start[T] + seg_pre[(int64_t)wi * kNF + f] : 0u;
    }
    // the next chunk's item and cover byte are fetched while the current one is placed
    uint32_t n_item = 0, n_cb = 0x100u;   // 0x100: past the segment, covers nothing
    if (a + threadIdx.x < b) {
      n_item = __ldcs(svals + a + threadIdx.x);
      n_cb = __ldcs(saux + a + threadIdx.x);
    }
    for (uint32_t e0 = a; e0 < b; e0 += kFineThreads) {
      const uint32_t item = n_item;
      const uint32_t cb = n_cb;
      const uint32_t en = e0 + kFineThreads + threadIdx.x;
      n_item = 0;
      n_cb = 0x100u;
      if (en < b) {
        n_item = __ldcs(svals + en);
        n_cb = __ldcs(saux + en);
      }
      const uint4 own = cb < 0x100u ? s_tab[cb] : make_uint4(0u, 0u, 0u, 0u);
      uint4 x = own;   // inclusive byte-wise scan over the warp
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y0 = __shfl_up_sync(0xffffffffu, x.x, o), y1 = __shfl_up_sync(0xffffffffu, x.y, o);
        const uint32_t y2 = __shfl_up_sync(0xffffffffu, x.z, o), y3 = __shfl_up_sync(0xffffffffu, x.w, o);
        if (lane >= o) {
          x.x += y0;
          x.y += y1;
          x.z += y2;
          x.w += y3;
        }
      }
      if (lane == 31) s_wtot[warp] = x;
      // exclusive ranks (no byte borrows: the inclusive bytes are at least the own ones)
      const uint32_t ex[4] = {x.x - own.x, x.y - own.y, x.z - own.z, x.w - own.w};
      const uint32_t ow[4] = {own.x, own.y, own.z, own.w};
      __syncthreads();
      if (threadIdx.x < kNF) {
        // per tile: warp offsets inside this chunk, then advance the tile's run
        const int f = threadIdx.x;
        uint32_t r = s_run[f];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          s_base[w][f] = r;
          const uint4 tw = s_wtot[w];
          const uint32_t word = (f >> 2) == 0 ? tw.x : (f >> 2) == 1 ? tw.y : (f >> 2) == 2 ? tw.z : tw.w;
          r += (word >> (8 * (f & 3))) & 0xffu;
        }
        s_run[f] = r;
      }
      __syncthreads();
      if (cb < 0x100u) {
        uint32_t db = 0u;
        if (KEYS) db = __float_as_uint(rgb_d[item].w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 bq = *reinterpret_cast<const uint4*>(&s_base[warp][4 * q]);
          const uint32_t bs[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if ((ow[q] >> (8 * k)) & 1u) {
              const uint32_t pos = bs[k] + ((ex[q] >> (8 * k)) & 0xffu);
              if (pos < cap) {
                vals[pos] = item;
                if (KEYS) keys[pos] = ((unsigned long long)s_tile[4 * q + k] << 32) | db;
              }
            }
          }
        }
      }
      // (the next chunk rewrites s_wtot before its first barrier and s_base after it: both
      // are read only between this chunk's two barriers or after the second by their writer)
    }
  }
}

static int bits_for(int64_t n) {
  int b = 1;
  while (b < 32 && ((int64_t)1 << b) < n) ++b;
  return b;
}

size_t bin_sort_ws_bytes(const rs_view_batch* b, int64_t capacity) {
  return bin_ws_layout(nullptr, b->n_items, capacity, b->n_tiles, b->n_views).bytes;
}

// Super instances: expansion, stable sort on the super-tile id (KeyT-wide), ranges.
// Returns which buffer set (0 or 1) holds the sorted items and cover bytes.
template <typename KeyT, bool CUT>
static int super_instances(const BinWs& w, const uint32_t* order, const uint32_t* n_kept, const rs_projected* proj,
                           const rs_view_batch* batch, int64_t cap, int64_t nblk, int64_t nb8, int n_super_max,
                           cudaStream_t s) {
  KeyT* k0 = reinterpret_cast<KeyT*>(w.skeys[0]);
  KeyT* k1 = reinterpret_cast<KeyT*>(w.skeys[1]);
  {
    prof::Scope ps("k_emit", s);
    k_emit<KeyT, CUT><<<(unsigned)nblk, kEmitThreads, 0, s>>>(
        order, n_kept, reinterpret_cast<const ushort4*>(proj->rect), batch->views, batch->n_views, w.super_base,
        w.cut_s, w.counters + 17, nb8, w.bsum, cap, w.wsum, k0, w.svals[0], w.saux[0]);
  }
  const int cur = tiles::sort_pairs<KeyT>(k0, w.svals[0], k1, w.svals[1], w.counters, cap, bits_for(n_super_max),
                                          w.sweep, s, true,
                                          {"k_super_sort_hist", "k_super_sort_scan", "k_super_sort"}, w.saux[0],
                                          w.saux[1], reinterpret_cast<const int32_t*>(w.counters + 8));
  const KeyT* sk = cur ? k1 : k0;
  prof::Scope ps("k_ranges", s);
  k_ranges<KeyT><<<4 * kNumSMs, 256, 0, s>>>(sk, w.counters, (uint32_t)n_super_max, w.sranges);
  return cur;
}

template <bool CUT>
static int super_stage(const BinWs& w, const uint32_t* order, const uint32_t* n_kept, const rs_projected* proj,
                       const rs_view_batch* batch, int64_t cap, int64_t nblk, int64_t nb8, int n_super_max,
                       cudaStream_t s) {
  return (n_super_max <= 65536)
             ? super_instances<uint16_t, CUT>(w, order, n_kept, proj, batch, cap, nblk, nb8, n_super_max, s)
             : super_instances<uint32_t, CUT>(w, order, n_kept, proj, batch, cap, nblk, nb8, n_super_max, s);
}

static rs_status bin_sort_impl(const rs_projected* proj, const rs_view_batch* batch, const rs_bins* bins, void* ws,
                               size_t ws_bytes, rs_device_status* status, cudaStream_t s, bool front) {
  if (!proj || !batch || !bins) return RS_ERR_INVALID_ARG;
  if (!bins->vals || !bins->ranges || bins->capacity <= 0 || bins->capacity >= ((int64_t)1 << 32))
    return RS_ERR_INVALID_ARG;
  if (batch->n_items < 0 || batch->n_items >= ((int64_t)1 << 32) || batch->n_tiles <= 0 || !batch->views ||
      batch->n_views <= 0)
    return RS_ERR_INVALID_ARG;
  if (!proj->rgb_d || !proj->rect || !proj->n_tiles) return RS_ERR_INVALID_ARG;
  if (front && (!proj->xy || !proj->conic_o || batch->tile_w <= 0 || batch->tile_h <= 0)) return RS_ERR_INVALID_ARG;
  // with fewer than kFrontItemsPerTile items per tile on average the lists are too short for
  // the occlusion cut to pay for its passes: whole lists (the same results)
  if (front && batch->n_items < kFrontItemsPerTile * (int64_t)batch->n_tiles) front = false;
  const BinWs w = bin_ws_layout(ws, batch->n_items, bins->capacity, batch->n_tiles, batch->n_views);
  if (!ws || ws_bytes < w.bytes || !aligned<uint4>(ws, 256)) return RS_ERR_WORKSPACE;
  const int64_t n = batch->n_items;
  const int64_t cap = bins->capacity;
  const float4* rgb_d = reinterpret_cast<const float4*>(proj->rgb_d);
  const ushort4* rect = reinterpret_cast<const ushort4*>(proj->rect);
  // super-tiles never outnumber tiles: a bound for the super-tile key width and ranges
  const int n_super_max = batch->n_tiles;

  if (cudaMemsetAsync(w.counters, 0, kCounterWords * 4, s) != cudaSuccess) return RS_ERR_CUDA;
  if (cudaMemsetAsync(w.sranges, 0, (size_t)n_super_max * 8, s) != cudaSuccess) return RS_ERR_CUDA;
  {
    prof::Scope ps("k_super_layout", s);
    k_super_layout<<<1, 32, 0, s>>>(batch->views, batch->n_views, w.super_base, n, w.counters + 6,
                                    bits_for(n_super_max), reinterpret_cast<int32_t*>(w.counters + 8), batch->n_tiles,
                                    status);
  }
  int scur = 0;   // buffer set of the sorted super instances
  if (n > 0) {
    // 1) items by depth (four 8-bit passes; an even count leaves the result in buffer 0)
    {
      prof::Scope ps("k_depth_keys", s);
      // front: the bound sums and the super-tile cuts, adjacent in the workspace, are zeroed
      // here (their reserved bytes are whole multiples of 256)
      const int64_t nz = front ? (int64_t)((reinterpret_cast<char*>(w.cut_s) - reinterpret_cast<char*>(w.cut_acc)) +
                                           align_up((size_t)n_super_max * 4, 256)) / 16
                               : 0;
      k_depth_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rgb_d, proj->n_tiles, n, w.dkeys[0], w.dvals[0],
                                                             front ? reinterpret_cast<uint4*>(w.cut_acc) : nullptr, nz);
    }
    // the first pass drops the items without instances; counters[16] = the items kept
    uint32_t* n_kept = w.counters + 16;
    const int dcur = tiles::sort_pairs<uint32_t>(w.dkeys[0], w.dvals[0], w.dkeys[1], w.dvals[1], w.counters + 6, n, 31,
                                                 w.hist, s, false,
                                                 {"k_depth_sort_hist", "k_depth_sort_scan", "k_depth_sort"}, nullptr,
                                                 nullptr, nullptr, n_kept);
    const uint32_t* order = w.dvals[dcur];
    if (front) {
      // occlusion cut: bound sums over the nearest items, then a rank cut per super-tile
      const int64_t wmax = (n + kCutWindowDiv - 1) / kCutWindowDiv;   // window bound (ranks)
      {
        prof::Scope ps("k_cut_accumulate", s);
        // one warp per group of kCutGroup window items, striding: at most 8 CTAs of 8 warps per SM
        const int64_t groups = (wmax + kCutGroup - 1) / kCutGroup;
        const int64_t cgrid = (groups + 7) / 8 < 8 * kNumSMs ? (groups + 7) / 8 : 8 * kNumSMs;
        k_cut_accumulate<<<(unsigned)cgrid, 256, 0, s>>>(
            order, n_kept, reinterpret_cast<const float2*>(proj->xy), reinterpret_cast<const float4*>(proj->conic_o),
            rect, batch->views, batch->n_views, batch->tile_w, batch->tile_h, batch->n_tiles, w.cut_acc);
      }
      {
        prof::Scope ps("k_cut_tiles", s);
        k_cut_tiles<<<(unsigned)((batch->n_tiles + 127) / 128), 128, 0, s>>>(
            w.cut_acc, n_kept, batch->views, batch->n_views, w.super_base, batch->n_tiles, w.cut_s, w.counters + 17);
      }
    }
    // 2) super instances in depth order, sorted stably on the super-tile id
    // front: the cut's window (at most ceil(n / 32) ranks) in blocks of 64 items
    const int64_t nb8 = front ? ((n + kCutWindowDiv - 1) / kCutWindowDiv + 63) / 64 : 0;
    const int64_t nblk = block_count(n, nb8);
    if (cudaMemsetAsync(w.csum, 0, (size_t)((nblk + kCountChunk - 1) / kCountChunk) * 8, s) != cudaSuccess)
      return RS_ERR_CUDA;
    {
      prof::Scope ps("k_count_blocks", s);
      if (front)
        k_count_blocks<true><<<(unsigned)nblk, kEmitThreads, 0, s>>>(order, n_kept, rect, batch->views, batch->n_views,
                                                                     w.super_base, w.cut_s, w.counters + 17, nb8,
                                                                     w.bsum, w.csum, w.wsum);
      else
        k_count_blocks<false><<<(unsigned)nblk, kEmitThreads, 0, s>>>(order, n_kept, rect, batch->views,
                                                                      batch->n_views, w.super_base, nullptr, nullptr,
                                                                      0, w.bsum, w.csum, nullptr);
    }
    {
      const int64_t n_chunks = (nblk + kCountChunk - 1) / kCountChunk;
      {
        prof::Scope pc("k_count_chunks", s);
        k_count_chunks<<<1, 1024, 0, s>>>(w.csum, n_chunks);
      }
      prof::Scope ps("k_count_top", s);
      k_count_top<<<(unsigned)n_chunks, kCountChunk, 0, s>>>(w.bsum, w.csum, nblk, cap, w.counters, status, n_kept,
                                                             front ? w.counters + 17 : nullptr, nb8);
    }
    scur = front ? super_stage<true>(w, order, n_kept, proj, batch, cap, nblk, nb8, n_super_max, s)
                 : super_stage<false>(w, order, n_kept, proj, batch, cap, nblk, nb8, n_super_max, s);
  }
  const uint32_t* svals = w.svals[scur];
  const uint8_t* saux = w.saux[scur];
  // 3) per tile: count (per super-tile segment), scans (ranges and K), scatter
  // at most 8 resident CTAs per SM; the work items (super-tiles x segments) come from a
  // device counter, so a generous bound on the number of super-tiles costs nothing
  const unsigned fgrid = (unsigned)(w.n_work_max < 8 * kNumSMs ? w.n_work_max : 8 * kNumSMs);
  {
    prof::Scope ps("k_fine_layout", s);
    k_fine_layout<<<1, 1024, 0, s>>>(w.super_base, batch->n_views, w.sranges, w.seg_off, w.work_s, w.n_work_max,
                                     w.counters);
  }
  {
    prof::Scope ps("k_fine_count", s);
    k_fine_count<<<fgrid, kFineThreads, 0, s>>>(saux, batch->views, batch->n_views, w.super_base, w.sranges,
                                                 w.seg_off, w.work_s, w.counters + 7, w.seg_cnt, w.counters + 4);
  }
  {
    prof::Scope ps("k_fine_seg_scan", s);
    k_fine_seg_scan<<<(unsigned)((batch->n_tiles + kTileBlock - 1) / kTileBlock), kTileBlock, 0, s>>>(
        w.seg_cnt, batch->views, batch->n_views, w.super_base, w.seg_off, batch->n_tiles, w.fine_tot, w.tile_blk);
  }
  {
    prof::Scope ps("k_fine_scan", s);
    k_fine_scan<<<(unsigned)((batch->n_tiles + kTileBlock - 1) / kTileBlock), kTileBlock, 0, s>>>(
        w.fine_tot, w.tile_blk, batch->n_tiles, cap, bins->ranges, w.counters, status);
  }
  {
    prof::Scope ps("k_fine_scatter", s);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(bins->keys);
    if (keys)
      k_fine_scatter<true><<<fgrid, kFineThreads, 0, s>>>(svals, saux, rgb_d, batch->views, batch->n_views,
                                                          w.super_base, w.sranges, w.fine_tot, w.seg_off, w.work_s,
                                                          w.counters + 7, w.seg_cnt, cap, bins->vals, keys,
                                                          w.counters + 5);
    else
      k_fine_scatter<false><<<fgrid, kFineThreads, 0, s>>>(svals, saux, rgb_d, batch->views, batch->n_views,
                                                           w.super_base, w.sranges, w.fine_tot, w.seg_off, w.work_s,
                                                           w.counters + 7, w.seg_cnt, cap, bins->vals, nullptr,
                                                           w.counters + 5);
  }
  return launch_status();
}

}  // namespace rs

using namespace rs;

extern "C" rs_status rs_bin_sort(const rs_projected* proj, const rs_view_batch* batch, const rs_bins* bins,
                                 void* ws, size_t ws_bytes, rs_device_status* status, void* stream) {
  return bin_sort_impl(proj, batch, bins, ws, ws_bytes, status, reinterpret_cast<cudaStream_t>(stream), false);
}

extern "C" rs_status rs_bin_sort_front(const rs_projected* proj, const rs_view_batch* batch, const rs_bins* bins,
                                       void* ws, size_t ws_bytes, rs_device_status* status, void* stream) {
  return bin_sort_impl(proj, batch, bins, ws, ws_bytes, status, reinterpret_cast<cudaStream_t>(stream), true);
}
