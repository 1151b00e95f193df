// rs_render / rs_importance: per-tile front-to-back compositing, Eq. (render-gs), with the
// importance max of Eq. (importance-score) fused in.
//
// One CTA per (view, tile), one thread per pixel.  The tile's sorted list is consumed in
// batches of one record per thread, staged into shared memory in blend-ready form
// (conic pre-scaled to the log2 domain), so that the inner loop per (pixel, Gaussian) pair
// is FP32 arithmetic plus one ex2.  A CTA stops fetching batches once every pixel is done
// (__syncthreads_count), and a warp leaves a batch early once all of its lanes are done.
// Importance: composited alpha*T values are max-reduced across the warp (redux.sync on the
// float bits, which order like the values for non-negative floats), then across the CTA in
// shared memory, then one global atomicMax per (tile, Gaussian).
#include <math.h>

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

template <int TW, int TH, bool IMAGE, bool IMPORTANCE>
__global__ void __launch_bounds__(TW* TH) k_render(RenderArgs a) {
  constexpr int NT = TW * TH;
  __shared__ float4 s_geo[NT];     // (x, y, A, B)   A,B,C: conic times -log2(e)/2, -log2(e), -log2(e)/2
  __shared__ float4 s_geo2[NT];    // (C, cut, o, 0) cut: below it alpha < 1/255 for sure
  __shared__ float4 s_col[NT];     // (r, g, b, 0)
  __shared__ uint32_t s_h[IMPORTANCE ? NT : 1];
  __shared__ uint32_t s_gid[IMPORTANCE ? NT : 1];

  const int tile = blockIdx.x;
  const int v = find_view_by_tile(a.views, a.n_views, tile);
  const rs_view& cam = a.views[v];
  const int local = tile - cam.tile_base;
  const int tyi = local / cam.tiles_x;
  const int txi = local - tyi * cam.tiles_x;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int pu = txi * TW + (tid % TW);
  const int pv = tyi * TH + (tid / TW);
  const bool inside = pu < cam.width && pv < cam.height;
  const float fu = (float)pu, fv = (float)pv;
  const uint2 rg = a.ranges[tile];
  const uint32_t start = rg.x, end = rg.y;

  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  int last = 0;
  bool done = !inside;

  for (uint32_t b0 = start; b0 < end; b0 += NT) {
    if (__syncthreads_count(!done) == 0) break;
    const int nb = (int)min((uint32_t)NT, end - b0);
    if (tid < nb) {
      const uint32_t item = __ldg(a.vals + b0 + tid);
      const float2 p = __ldg(a.xy + item);
      const float4 co = __ldg(a.conic_o + item);
      const float4 cd = __ldg(a.rgb_d + item);
      const float A = -0.5f * kLog2e * co.x, B = -kLog2e * co.y, C = -0.5f * kLog2e * co.z;
      // alpha = o 2^p2 < 1/255  <=>  p2 < log2(1/(255 o)); the cut sits a little below so
      // that only surely-skipped pairs avoid the exact test
      const float cut = log2f(kAlphaMin / co.w) - 1e-3f;
      s_geo[tid] = make_float4(p.x, p.y, A, B);
      s_geo2[tid] = make_float4(C, cut, co.w, 0.f);
      s_col[tid] = make_float4(cd.x, cd.y, cd.z, 0.f);
      if (IMPORTANCE) {
        s_h[tid] = 0u;
        s_gid[tid] = a.subset ? __ldg(a.subset + item) : (uint32_t)((int64_t)item - cam.item_base);
      }
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
      float w = 0.f;
      if (!done) {
        const float4 g = s_geo[j];
        const float4 g2 = s_geo2[j];
        const float dx = g.x - fu, dy = g.y - fv;
        const float p2 = dx * fmaf(g.z, dx, g.w * dy) + g2.x * dy * dy;
        if (p2 <= 0.f && p2 >= g2.y) {
          const float alpha = fminf(kAlphaMax, g2.z * exp2f(p2));
          if (alpha >= kAlphaMin) {
            const float Tn = T * (1.f - alpha);
            if (Tn < kTMin) {
              done = true;
            } else {
              w = alpha * T;
              const float4 col = s_col[j];
              c0 = fmaf(w, col.x, c0);
              c1 = fmaf(w, col.y, c1);
              c2 = fmaf(w, col.z, c2);
              T = Tn;
              last = (int)(b0 - start) + j + 1;
            }
          }
        }
      }
      if (IMPORTANCE) {
        const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(w));
        if (lane == 0 && m) atomicMax(&s_h[j], m);
      }
      if (__all_sync(0xffffffffu, done)) break;
    }
    __syncthreads();
    if (IMPORTANCE && tid < nb) {
      const uint32_t m = s_h[tid];
      if (m && (int64_t)s_gid[tid] < a.n_gaussians) atomicMax(a.importance + s_gid[tid], m);
    }
  }

  if (inside) {
    const int64_t HW = (int64_t)cam.width * cam.height;
    const int64_t pix = (int64_t)pv * cam.width + pu;
    if (IMAGE) {
      float* img = a.image + 3 * cam.pixel_base;
      img[pix] = c0 + T * a.bg0;
      img[HW + pix] = c1 + T * a.bg1;
      img[2 * HW + pix] = c2 + T * a.bg2;
    }
    if (a.T_final) a.T_final[cam.pixel_base + pix] = T;
    if (a.last) a.last[cam.pixel_base + pix] = last;
  }
}

template <int TW, int TH>
static void launch_render(const RenderArgs& a, int n_tiles, bool image, bool imp, cudaStream_t s) {
  if (image && imp) k_render<TW, TH, true, true><<<n_tiles, TW * TH, 0, s>>>(a);
  else if (image) k_render<TW, TH, true, false><<<n_tiles, TW * TH, 0, s>>>(a);
  else if (imp) k_render<TW, TH, false, true><<<n_tiles, TW * TH, 0, s>>>(a);
  else k_render<TW, TH, false, false><<<n_tiles, TW * TH, 0, s>>>(a);
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
