// Occlusion cut of the tile lists (rs_bin_sort_front): for every tile, a depth rank beyond
// which no pixel of the tile composites or even reads a list entry, so that binning only
// produces the front of each list that the blend of Eq. render-gs can reach.
//
// The bound.  Blending stops a pixel before the first entry whose T (1 - alpha) falls below
// 1e-4, and T only decreases.  Take an item whose alpha stays at or above some alpha_lb
// >= kCutAlphaMin > 1/255 at every pixel centre of a tile (so the blend's skip test never
// drops it there): at each such entry the pixel either composites it, which
// multiplies T by at most 1 - alpha_lb, or has already stopped.  Once the product of
// (1 - alpha_lb) over the items ranked before some point is below 1e-4 (with a factor 2 to
// spare for the kernels' rounding of T), every pixel of the tile has stopped by then.
// The power -(a dx^2 + c dy^2)/2 - b dx dy is a concave quadratic of the pixel position
// (the conic is positive definite), so over the rectangle of a tile's pixel centres it is
// smallest at one of the four corners: the corners give alpha_lb for the whole tile.
//
// Rounding.  The blend evaluates p2 = log2(e) * power in FP32 from the rounded
// coefficients A, B, C and the rounded offsets dx, dy; the bound evaluates the same form at
// the corners and subtracts a margin of 2^-19 times the magnitude of its terms there, far
// above the few roundings either side makes.  The blend tests p2 <= 0, so the bound takes
// only items whose rounded quadratic form is well away from singular (smallest eigenvalue
// above 2^-14 of the coefficients' size), for which the FP32 p2 cannot turn positive.
// alpha_lb carries a relative margin of 2^-12 for the hardware 2^x and the products;
// -log2(1 - alpha_lb) is accumulated in fixed point (x 4096, rounded down, less 2^-10), so
// sums are exact integers and the decision does not depend on the order of the atomics.
//
// Where.  The accumulation looks at the nearest items only (a window of the first
// ceil(n / 32) depth ranks), in kCutBuckets rank buckets that widen with the rank (bucket b
// ends at rank ceil(W (b + 1)^2 / 16^2)): a tile's cut is the end of the first bucket at
// which its prefix sum passes the threshold.  A tile that is not saturated within the
// window gets no cut (its list stays whole), and a super-tile's cut is the largest of its
// tiles' cuts, so every tile list is a prefix of the full list that holds every entry the
// blend reads.
//
// Hardware approximations.  2^x and log2 come from the MUFU approximations (ex2.approx,
// lg2.approx): their documented errors (a few units in the last place of 2^x; for log2 an
// absolute 2^-22 on [0.5, 2) and two ulps elsewhere) are far inside the relative margins
// 2^-12 on alpha_lb and 2^-10 on -log2(1 - alpha_lb), whose smallest value here is
// -log2(1 - kCutAlphaMin) ~ 0.074.  The per-item filters (opacity above kCutAlphaMin,
// region wide enough for a tile, the column spans) only choose which pairs are evaluated:
// a pair they leave out gives no bound, which can only delay a cut.
#pragma once

#include "blend.cuh"
#include "rs_common.cuh"

namespace rs {

constexpr int kCutBuckets = 16;         // rank buckets of the window
constexpr uint32_t kCutWindowDiv = 32;  // window: the nearest ceil(n_kept / 32) items
constexpr float kCutScale = 4096.f;     // fixed point of -log2(1 - alpha_lb)
// prefix sums at or above this give a product of (1 - alpha_lb) <= 2^-14.307 < 5e-5
constexpr uint32_t kCutThreshold = 58600u;
constexpr uint32_t kNoCut = 0xffffffffu;
constexpr int kCutGroup = 8;            // window items per warp and group in k_cut_accumulate
// Only pairs with alpha_lb >= kCutAlphaMin add to the sums (a pair left out only delays a
// cut): in the dense headline scene this evaluates 2.4x fewer pairs than alpha_lb >= 1/255
// for 12% more listed instances.
constexpr float kCutAlphaMin = 0.05f;

// The window's ranks [0, W); bucket b holds the ranks [E(b), E(b + 1)) with
// E(b) = ceil(W b^2 / 16^2): narrow buckets at the front, where the tiles of a dense scene
// saturate, so that the cut (the end of a bucket) lies close to the saturating rank.
__device__ __forceinline__ uint32_t cut_window(uint32_t n_kept) { return (n_kept + kCutWindowDiv - 1) / kCutWindowDiv; }

__device__ __forceinline__ uint32_t cut_bucket_start(uint32_t W, uint32_t b) {
  return (uint32_t)(((uint64_t)W * b * b + (uint64_t)(kCutBuckets * kCutBuckets - 1)) /
                    (uint64_t)(kCutBuckets * kCutBuckets));
}

// The bucket of rank r < W: the largest b with E(b) <= r (a float estimate, then corrected
// in integers).
__device__ __forceinline__ uint32_t cut_bucket(uint32_t W, uint32_t r) {
  uint32_t b = (uint32_t)sqrtf((float)r * (float)(kCutBuckets * kCutBuckets) / (float)W);
  b = min(b, (uint32_t)kCutBuckets - 1u);
  while (b + 1u < (uint32_t)kCutBuckets && cut_bucket_start(W, b + 1u) <= r) ++b;
  while (b > 0u && cut_bucket_start(W, b) > r) --b;
  return b;
}

// Per item of the window, the data its (item, tile) pairs read.
struct CutItem {
  float x, y;      // mean (pixels)
  float A, B, C;   // p2 = A dx^2 + B dx dy + C dy^2, rounded as the blend rounds them
  float o;         // opacity
};

// Fixed-point -log2(1 - alpha_lb) of one (item, tile) pair, 0 if the pair gives no bound.
// Pixel centres of the tile: u in [u0, u1], v in [v0, v1] (inside the image).
__device__ __forceinline__ uint32_t cut_contribution(const CutItem& it, float u0, float u1, float v0, float v1) {
  const float dx0 = it.x - u0, dx1 = it.x - u1, dy0 = it.y - v0, dy1 = it.y - v1;
  auto p2 = [&](float dx, float dy) { return fmaf(dy, fmaf(it.C, dy, it.B * dx), it.A * dx * dx); };
  const float pmin = fminf(fminf(p2(dx0, dy0), p2(dx0, dy1)), fminf(p2(dx1, dy0), p2(dx1, dy1)));
  const float ax = fmaxf(fabsf(dx0), fabsf(dx1)), ay = fmaxf(fabsf(dy0), fabsf(dy1));
  const float mag = fabsf(it.A) * ax * ax + fabsf(it.B) * ax * ay + fabsf(it.C) * ay * ay;
  const float L = pmin - fmaf(mag, 0x1p-19f, 0x1p-40f);
  const float a_lb = fminf(kAlphaMax, it.o * ex2_approx(fmaxf(L, -126.f))) * (1.f - 0x1p-12f);
  if (!(a_lb >= kCutAlphaMin)) return 0u;
  const float l = -__log2f(1.f - a_lb) * (kCutScale * (1.f - 0x1p-10f));
  return (uint32_t)l;   // truncation: rounded down
}

// Per-item part of the bound: the form's coefficients as the blend rounds them and whether
// the item can give a bound at all (positive definite and well conditioned, opacity above
// kCutAlphaMin, and an alpha >= kCutAlphaMin region wide enough to hold a whole tile: its
// semi-minor axis^2 must reach (min(tile_w, tile_h) - 1)^2 / 4).
__device__ __forceinline__ bool cut_item(const float4 co, const ushort4 tr, int tile_w, int tile_h, CutItem& it) {
  const float A = __fmul_rn(-0.5f * kLog2e, co.x), B = __fmul_rn(-kLog2e, co.y), C = __fmul_rn(-0.5f * kLog2e, co.z);
  // eigenvalues of -[[A, B/2], [B/2, C]] (A, C < 0 for a positive definite conic)
  const float h = 0.5f * (A - C);
  const float rt = sqrtf(h * h + 0.25f * B * B);
  const float lam = -0.5f * (A + C) - rt, lam_max = -0.5f * (A + C) + rt;
  const float size = fabsf(A) + fabsf(B) + fabsf(C);
  const float lvl = __log2f(co.w * (1.f / kCutAlphaMin));   // > 0 iff o > kCutAlphaMin (a filter)
  const float s = 0.5f * (float)(min(tile_w, tile_h) - 1);
  it.A = A;
  it.B = B;
  it.C = C;
  it.o = co.w;
  return A < 0.f && C < 0.f && lam > 0x1p-14f * size && lvl > 0.f && lvl >= 0.9f * s * s * lam_max &&
         tr.z > tr.x && tr.w > tr.y;
}

// Tile columns [c0, c1] of tile row gy (pixel rows v0..v1) whose four corner pixel centres
// all lie in the item's region p2 >= lv, a convex set (the power is concave), so that the
// whole tile does: the chord of the region at each of the two rows, intersected.  Only an
// enumeration filter: the bound of every enumerated pair is recomputed by
// cut_contribution, and a tile it leaves out only gives no bound.
__device__ __forceinline__ void cut_row_span(const CutItem& it, float lv, float v0, float v1, int tile_w,
                                            float inv_tw, int width, int gx0, int gx1, int& c0, int& c1) {
  float xlo = -3.0e38f, xhi = 3.0e38f;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float dy = it.y - (k ? v1 : v0);
    // A dx^2 + (B dy) dx + (C dy^2 - lv) >= 0 with A < 0: dx between the two roots
    const float b = it.B * dy, c = fmaf(it.C * dy, dy, -lv);
    const float disc = fmaf(b, b, -4.f * it.A * c);
    if (!(disc >= 0.f)) {
      xlo = 1.f;
      xhi = 0.f;
      continue;
    }
    const float q = sqrtf(disc), inv = 0.5f / it.A;   // inv < 0
    const float d_hi = (-b - q) * inv, d_lo = (-b + q) * inv;   // d_lo <= d_hi
    // dx = x_mean - u  =>  u in [x_mean - d_hi, x_mean - d_lo]; half a pixel of slack
    xlo = fmaxf(xlo, it.x - d_hi - 0.5f);
    xhi = fminf(xhi, it.x - d_lo + 0.5f);
  }
  c0 = gx0;
  c1 = gx0 - 1;
  if (!(xlo <= xhi)) return;
  // first column whose left pixel column u0 = gx tile_w is >= xlo; last whose right pixel
  // column min(u0 + tile_w, width) - 1 is <= xhi
  const float fl = ceilf(xlo * inv_tw);
  const float fh = xhi >= (float)(width - 1) ? 3.0e38f : floorf((xhi + 1.f) * inv_tw) - 1.f;
  c0 = fl <= (float)gx0 ? gx0 : (fl > (float)gx1 ? gx1 + 1 : (int)fl);
  c1 = fh >= (float)gx1 ? gx1 : (fh < (float)gx0 ? gx0 - 1 : (int)fh);
}

// What the pairs of one window item read, staged in shared memory by its lane.
struct CutSlot {
  CutItem it;
  float lv;                   // p2 >= lv  <=>  o 2^p2 >= kCutAlphaMin
  int gx0, gx1, gy0;          // tile rect: columns gx0..gx1, first row gy0
  int width, height, tiles_x;
  uint32_t tile_base;
  uint32_t bucket;            // the rank's bucket: the item's row of the accumulator
};

// Accumulation over the window.  Each warp takes a group of kCutGroup ranks g, g + G,
// g + 2G, ... (G = ceil(W / kCutGroup) groups, so the large near items spread over the
// groups), one per lane of the first kCutGroup: the lane stages its item's data.  The warp then walks the group's (item, tile row) pairs
// 32 at a time, each lane finding the span of columns of its row that can give a bound,
// and then those spans' tiles 32 at a time; lanes find their row, and rows their item, by
// binary searches over the warp's prefixes.  acc[b * n_tiles + t] += the pair's
// contribution, b = the rank's bucket.
__global__ void __launch_bounds__(256) k_cut_accumulate(const uint32_t* __restrict__ order,
                                                        const uint32_t* __restrict__ n_kept,
                                                        const float2* __restrict__ xy,
                                                        const float4* __restrict__ conic_o,
                                                        const ushort4* __restrict__ rect,
                                                        const rs_view* __restrict__ views, int n_views, int tile_w,
                                                        int tile_h, int n_tiles, uint32_t* __restrict__ acc) {
  __shared__ CutSlot s_slot[8][kCutGroup];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  CutSlot* slot = s_slot[warp];
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t W = cut_window(*n_kept);
  const uint32_t G = (W + kCutGroup - 1u) / kCutGroup;
  const float inv_tw = 1.f / (float)tile_w;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {   // warp-uniform
    const uint32_t r = g + (uint32_t)lane * G;
    uint32_t rows = 0;
    CutSlot sl{};
    if (lane < kCutGroup && r < W) {
      const uint32_t item = order[r];
      const ushort4 tr = rect[item];
      const float4 co = conic_o[item];
      if (cut_item(co, tr, tile_w, tile_h, sl.it)) {
        const float2 p = xy[item];
        sl.it.x = p.x;
        sl.it.y = p.y;
        sl.lv = -__log2f(co.w * (1.f / kCutAlphaMin));
        const rs_view& cam = views[find_view_by_item(views, n_views, (int64_t)item)];
        sl.gx0 = tr.x;
        sl.gx1 = (int)tr.z - 1;
        sl.gy0 = tr.y;
        sl.width = cam.width;
        sl.height = cam.height;
        sl.tiles_x = cam.tiles_x;
        sl.tile_base = (uint32_t)cam.tile_base;
        sl.bucket = cut_bucket(W, r);
        rows = (uint32_t)(tr.w - tr.y);
      }
    }
    __syncwarp();   // the previous group's reads of the slots are done
    if (lane < kCutGroup) slot[lane] = sl;
    __syncwarp();
    uint32_t rincl = rows;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, rincl, o);
      if (lane >= o) rincl += y;
    }
    const uint32_t rtot = __shfl_sync(0xffffffffu, rincl, 31);
    const uint32_t rexcl = rincl - rows;
    for (uint32_t q0 = 0; q0 < rtot; q0 += 32) {
      // this lane's (item, row): item = the lane whose row range holds q
      const uint32_t q = q0 + lane;
      int oi = 0;
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, rincl, oi + sh - 1);
        if (v <= q) oi += sh;
      }
      oi = oi < 31 ? oi : 31;
      const uint32_t o_rexcl = __shfl_sync(0xffffffffu, rexcl, oi);
      int c0 = 0, c1 = -1, gy = 0;
      if (q < rtot) {
        const CutSlot& S = slot[oi];
        gy = S.gy0 + (int)(q - o_rexcl);
        const int v0 = gy * tile_h, v1 = min(v0 + tile_h, S.height) - 1;
        cut_row_span(S.it, S.lv, (float)v0, (float)v1, tile_w, inv_tw, S.width, S.gx0, S.gx1, c0, c1);
      }
      const uint32_t cnt = c1 >= c0 ? (uint32_t)(c1 - c0 + 1) : 0u;
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t excl = incl - cnt;
      for (uint32_t e0 = 0; e0 < tot; e0 += 32) {
        const uint32_t e = e0 + lane;
        int lo = 0;
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
          const uint32_t v = __shfl_sync(0xffffffffu, incl, lo + sh - 1);
          if (v <= e) lo += sh;
        }
        const int owner = lo < 31 ? lo : 31;
        const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, owner);
        const int o_c0 = __shfl_sync(0xffffffffu, c0, owner);
        const int o_gy = __shfl_sync(0xffffffffu, gy, owner);
        const int o_it = __shfl_sync(0xffffffffu, oi, owner);
        if (e < tot) {
          const CutSlot& S = slot[o_it];
          const int tx = o_c0 + (int)(e - o_excl);
          const int u0 = tx * tile_w, v0 = o_gy * tile_h;
          const int u1 = min(u0 + tile_w, S.width) - 1, v1 = min(v0 + tile_h, S.height) - 1;
          const uint32_t c = cut_contribution(S.it, (float)u0, (float)u1, (float)v0, (float)v1);
          const int64_t t = (int64_t)S.tile_base + (int64_t)o_gy * S.tiles_x + tx;
          // (a batch whose views need more tiles than n_tiles is rejected)
          if (c && t < n_tiles) atomicAdd(acc + (int64_t)S.bucket * n_tiles + t, c);
        }
      }
    }
  }
}

// One thread per tile: the first bucket at which the tile's prefix sum reaches the
// threshold gives its cut (the end rank of that bucket; kNoCut if none); each super-tile
// takes the largest cut of its tiles (cut_s zeroed by the caller), and cut_max the largest
// over all tiles.
__global__ void __launch_bounds__(128) k_cut_tiles(const uint32_t* __restrict__ acc,
                                                   const uint32_t* __restrict__ n_kept,
                                                   const rs_view* __restrict__ views, int n_views,
                                                   const uint32_t* __restrict__ super_base, int n_tiles,
                                                   uint32_t* __restrict__ cut_s, uint32_t* __restrict__ cut_max) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const int v = find_view_by_tile(views, n_views, t);
  const rs_view& cam = views[v];
  const int local = t - cam.tile_base;
  if (local < 0 || local >= cam.tiles_x * cam.tiles_y) return;
  const uint32_t W = cut_window(*n_kept);
  // a cell can only come out low if its atomics wrapped, which delays the cut: never unsafe;
  // 16 loads in flight at a time (consecutive threads read consecutive words of a bucket row)
  uint64_t run = 0;
  uint32_t cut = kNoCut;
  for (int b0 = 0; b0 < kCutBuckets && cut == kNoCut; b0 += 16) {
    uint32_t a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = acc[(int64_t)(b0 + j) * n_tiles + t];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      run += a[j];
      if (cut == kNoCut && run >= kCutThreshold) cut = cut_bucket_start(W, (uint32_t)(b0 + j) + 1u);
    }
  }
  const int ty = local / cam.tiles_x, tx = local - ty * cam.tiles_x;
  const int sw = (cam.tiles_x + 3) / 4;
  atomicMax(cut_s + super_base[v] + (ty / 4) * sw + tx / 4, cut);
  atomicMax(cut_max, cut);
}

}  // namespace rs
