// rs_render / rs_importance: per-tile front-to-back compositing, Eq. (render-gs), with the
// importance max of Eq. (importance-score) fused in.
//
// One CTA per (view, tile); each thread owns two vertically adjacent pixels, so every
// Gaussian record read from shared memory serves two pixel evaluations.  The tile's sorted
// list is consumed in batches of two records per thread, staged into shared memory in
// blend-ready form (conic pre-scaled to the log2 domain), so the inner loop per
// (pixel, Gaussian) pair is FP32 arithmetic plus one ex2.  A CTA stops fetching batches
// once every pixel is done (__syncthreads_count), and a warp leaves a batch early once all
// of its pixels are done.
// Importance: composited alpha*T values are max-reduced across the warp (redux.sync on the
// float bits, which order like the values for non-negative floats), then across the CTA in
// shared memory, then one global atomicMax per (tile, Gaussian).
#include <math.h>

#include "blend.cuh"
#include "profile.cuh"
#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {

struct RenderArgs {
  const float2* xy;
  const float4* conic_o;
  const float4* rgb_d;
  const uint32_t* vals;
  const uint2* ranges;
  const rs_view* views;
  const uint32_t* subset;
  int32_t n_views;
  float bg0, bg1, bg2;
  float* image;
  float* T_final;
  int32_t* last;
  uint32_t* importance;
  int64_t n_gaussians;
};

struct PixelState {
  float T, c0, c1, c2;
  int last;
  bool done;
};

// One (pixel, Gaussian) step of the blend rule; returns the composited weight alpha*T
// (0 if the entry was skipped or compositing stopped here).
__device__ __forceinline__ float blend_step(PixelState& s, const float4& g, const float4& g2, const float4& col,
                                            float fu, float fv, int pos) {
  if (s.done) return 0.f;
  const float p2 = blend_power(g, g2, fu, fv);
  if (!(p2 <= 0.f && p2 >= g2.y)) return 0.f;
  const float alpha = fminf(kAlphaMax, __fmul_rn(g2.z, exp2f(p2)));
  if (alpha < kAlphaMin) return 0.f;
  const float Tn = s.T * (1.f - alpha);
  if (Tn < kTMin) {
    s.done = true;
    return 0.f;
  }
  const float w = alpha * s.T;
  s.c0 = fmaf(w, col.x, s.c0);
  s.c1 = fmaf(w, col.y, s.c1);
  s.c2 = fmaf(w, col.z, s.c2);
  s.T = Tn;
  s.last = pos + 1;
  return w;
}

template <int TW, int TH, bool IMAGE, bool IMPORTANCE>
__global__ void __launch_bounds__(TW* TH / 2) k_render(RenderArgs a) {
  constexpr int NT = TW * TH / 2;   // threads; each owns pixels (x, 2r) and (x, 2r + 1)
  constexpr int NB = 2 * NT;        // records per batch
  __shared__ float4 s_geo[NB];
  __shared__ float4 s_geo2[NB];
  __shared__ float4 s_col[NB];
  __shared__ uint32_t s_h[IMPORTANCE ? NB : 1];
  __shared__ uint32_t s_gid[IMPORTANCE ? NB : 1];

  const int tile = blockIdx.x;
  const int v = find_view_by_tile(a.views, a.n_views, tile);
  const rs_view& cam = a.views[v];
  const int local = tile - cam.tile_base;
  const int tyi = local / cam.tiles_x;
  const int txi = local - tyi * cam.tiles_x;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int pu = txi * TW + (tid % TW);
  const int pv0 = tyi * TH + 2 * (tid / TW);
  const bool in0 = pu < cam.width && pv0 < cam.height;
  const bool in1 = pu < cam.width && pv0 + 1 < cam.height;
  const float fu = (float)pu, fv0 = (float)pv0, fv1 = (float)(pv0 + 1);
  const uint2 rg = a.ranges[tile];
  const uint32_t start = rg.x, end = rg.y;

  PixelState s0{1.f, 0.f, 0.f, 0.f, 0, !in0};
  PixelState s1{1.f, 0.f, 0.f, 0.f, 0, !in1};

  for (uint32_t b0 = start; b0 < end; b0 += NB) {
    if (__syncthreads_count(!(s0.done && s1.done)) == 0) break;
    const int nb = (int)min((uint32_t)NB, end - b0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int slot = tid + k * NT;
      if (slot < nb) {
        const uint32_t item = __ldg(a.vals + b0 + slot);
        stage_record(a.xy, a.conic_o, a.rgb_d, item, s_geo[slot], s_geo2[slot], s_col[slot]);
        if (IMPORTANCE) {
          s_h[slot] = 0u;
          s_gid[slot] = a.subset ? __ldg(a.subset + item) : (uint32_t)((int64_t)item - cam.item_base);
        }
      }
    }
    __syncthreads();
    const int base = (int)(b0 - start);
    for (int j = 0; j < nb; ++j) {
      const float4 g = s_geo[j];
      const float4 g2 = s_geo2[j];
      const float4 col = s_col[j];
      const float w0 = blend_step(s0, g, g2, col, fu, fv0, base + j);
      const float w1 = blend_step(s1, g, g2, col, fu, fv1, base + j);
      if (IMPORTANCE) {
        const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(w0, w1)));
        if (lane == 0 && m) atomicMax(&s_h[j], m);
      }
      if (__all_sync(0xffffffffu, s0.done && s1.done)) break;
    }
    __syncthreads();
    if (IMPORTANCE) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int slot = tid + k * NT;
        if (slot < nb) {
          const uint32_t m = s_h[slot];
          if (m && (int64_t)s_gid[slot] < a.n_gaussians) atomicMax(a.importance + s_gid[slot], m);
        }
      }
    }
  }

  const int64_t HW = (int64_t)cam.width * cam.height;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const PixelState& s = k ? s1 : s0;
    if (k ? !in1 : !in0) continue;
    const int64_t pix = (int64_t)(pv0 + k) * cam.width + pu;
    if (IMAGE) {
      float* img = a.image + 3 * cam.pixel_base;
      img[pix] = s.c0 + s.T * a.bg0;
      img[HW + pix] = s.c1 + s.T * a.bg1;
      img[2 * HW + pix] = s.c2 + s.T * a.bg2;
    }
    if (a.T_final) a.T_final[cam.pixel_base + pix] = s.T;
    if (a.last) a.last[cam.pixel_base + pix] = s.last;
  }
}

template <int TW, int TH>
static void launch_render(const RenderArgs& a, int n_tiles, bool image, bool imp, cudaStream_t s) {
  constexpr int NT = TW * TH / 2;
  prof::Scope ps(imp ? "k_render_importance" : "k_render", s);
  if (image && imp) k_render<TW, TH, true, true><<<n_tiles, NT, 0, s>>>(a);
  else if (image) k_render<TW, TH, true, false><<<n_tiles, NT, 0, s>>>(a);
  else if (imp) k_render<TW, TH, false, true><<<n_tiles, NT, 0, s>>>(a);
  else k_render<TW, TH, false, false><<<n_tiles, NT, 0, s>>>(a);
}

rs_status render_dispatch(const rs_projected* proj, const rs_bins* bins, const rs_view_batch* batch,
                          const rs_config* cfg, float* image, float* T_final, int32_t* last, uint32_t* importance,
                          int64_t n_gaussians, cudaStream_t s) {
  RenderArgs a;
  a.xy = reinterpret_cast<const float2*>(proj->xy);
  a.conic_o = reinterpret_cast<const float4*>(proj->conic_o);
  a.rgb_d = reinterpret_cast<const float4*>(proj->rgb_d);
  a.vals = bins->vals;
  a.ranges = reinterpret_cast<const uint2*>(bins->ranges);
  a.views = batch->views;
  a.subset = batch->subset_idx;
  a.n_views = batch->n_views;
  a.bg0 = cfg->bg[0];
  a.bg1 = cfg->bg[1];
  a.bg2 = cfg->bg[2];
  a.image = image;
  a.T_final = T_final;
  a.last = last;
  a.importance = importance;
  a.n_gaussians = n_gaussians;
  const bool img = image != nullptr, imp = importance != nullptr;
  if (batch->tile_w == 16 && batch->tile_h == 16) launch_render<16, 16>(a, batch->n_tiles, img, imp, s);
  else if (batch->tile_w == 32 && batch->tile_h == 8) launch_render<32, 8>(a, batch->n_tiles, img, imp, s);
  else if (batch->tile_w == 8 && batch->tile_h == 8) launch_render<8, 8>(a, batch->n_tiles, img, imp, s);
  else return RS_ERR_UNSUPPORTED;
  return launch_status();
}

static rs_status check_render_args(const rs_projected* proj, const rs_bins* bins, const rs_view_batch* batch,
                                   const rs_config* cfg) {
  if (!proj || !bins || !batch || !cfg) return RS_ERR_INVALID_ARG;
  if (!proj->xy || !proj->conic_o || !proj->rgb_d || !bins->vals || !bins->ranges || !batch->views)
    return RS_ERR_INVALID_ARG;
  if (batch->n_tiles < 0 || batch->n_views <= 0) return RS_ERR_INVALID_ARG;
  if (!aligned<float4>(proj->conic_o, 16) || !aligned<float4>(proj->rgb_d, 16) || !aligned<float2>(proj->xy, 8) ||
      !aligned<uint2>(bins->ranges, 8))
    return RS_ERR_INVALID_ARG;
  return RS_OK;
}

}  // namespace rs

using namespace rs;

extern "C" rs_status rs_render(const rs_projected* proj, const rs_bins* bins, const rs_view_batch* batch,
                               const rs_config* cfg, float* image, float* T_final, int32_t* last,
                               uint32_t* importance, int64_t n_gaussians, void* stream) {
  rs_status st = check_render_args(proj, bins, batch, cfg);
  if (st != RS_OK) return st;
  if (importance && n_gaussians <= 0) return RS_ERR_INVALID_ARG;
  if (batch->n_tiles == 0) return RS_OK;
  return render_dispatch(proj, bins, batch, cfg, image, T_final, last, importance, n_gaussians,
                         reinterpret_cast<cudaStream_t>(stream));
}

extern "C" rs_status rs_importance(const rs_projected* proj, const rs_bins* bins, const rs_view_batch* batch,
                                   const rs_config* cfg, uint32_t* importance, int64_t n_gaussians,
                                   void* stream) {
  rs_status st = check_render_args(proj, bins, batch, cfg);
  if (st != RS_OK) return st;
  if (!importance || n_gaussians <= 0) return RS_ERR_INVALID_ARG;
  if (batch->n_tiles == 0) return RS_OK;
  return render_dispatch(proj, bins, batch, cfg, nullptr, nullptr, nullptr, importance, n_gaussians,
                         reinterpret_cast<cudaStream_t>(stream));
}
