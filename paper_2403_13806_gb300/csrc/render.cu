// rs_render / rs_importance: per-tile front-to-back compositing, Eq. (render-gs), with the
// importance max of Eq. (importance-score) fused in.
//
// One warp per (view, tile); each thread owns PX vertically adjacent pixels of one column
// (PX = 8 for 16x16 and 32x8 tiles, 2 for 8x8), evaluated as PX/2 pixel pairs with packed
// two-lane FP32 instructions, so every Gaussian record read from shared memory serves PX
// pixel evaluations and each thread carries PX/2 independent chains through a record.  The
// tile's sorted list is consumed in batches of NBM records per thread (rs_config.batch =
// NBM x threads with NBM one of 1, 2, 4; the autotuner picks it), staged into shared memory
// in blend-ready form (conic pre-scaled to the log2 domain, opacity divided by 0.99, colours
// multiplied by 0.99); the per-pixel decisions are predicated or exact 0/1 factors, not
// branches.  A warp skips a record that none of its pixels' alpha-support tests accept,
// leaves a batch once all of its pixels are done, and the CTA stops fetching batches once
// every pixel is done (__syncthreads_count).
// Importance: the composited weights s T = alpha T / 0.99 are max-reduced across the warp
// (redux.sync on the float bits, which order like the values for non-negative floats),
// scaled by 0.99, combined across the CTA in shared memory, then one global atomicMax per
// (tile, Gaussian).
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

template <int TW, int TH, int PX, int NBM, bool IMPORTANCE>
__global__ void __launch_bounds__(TW* TH / PX) k_render(RenderArgs a) {
  constexpr int NT = TW * TH / PX;   // threads; each owns pixels (x, PX r + k), k < PX
  constexpr int NP = PX / 2;         // pixel pairs per thread
  constexpr int NB = NBM * NT;       // records per batch (NBM per thread)
  __shared__ BlendRec s_rec[NB];
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
  const int pv0 = tyi * TH + PX * (tid / TW);
  const float2 nu = make_float2(-(float)pu, -(float)pu);
  const uint2 rg = a.ranges[tile];
  const uint32_t start = rg.x, end = rg.y;

  // A pixel that is done (outside the image, or stopped by T(1 - alpha) < 1e-4) carries a NaN
  // row offset: its p2 is NaN, every test on it is false, and it needs no flag of its own.
  float2 nv[NP], T[NP], cr[NP], cg[NP], cb[NP];
  int last[PX];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const bool in0 = pu < cam.width && pv0 + 2 * q < cam.height;
    const bool in1 = pu < cam.width && pv0 + 2 * q + 1 < cam.height;
    nv[q] = make_float2(in0 ? -(float)(pv0 + 2 * q) : __int_as_float(0x7fc00000),
                        in1 ? -(float)(pv0 + 2 * q + 1) : __int_as_float(0x7fc00000));
    T[q] = make_float2(1.f, 1.f);
    cr[q] = cg[q] = cb[q] = make_float2(0.f, 0.f);
    last[2 * q] = last[2 * q + 1] = 0;
  }
  auto all_done = [&]() {
    bool d = true;
#pragma unroll
    for (int q = 0; q < NP; ++q) d = d && isnan(nv[q].x) && isnan(nv[q].y);
    return d;
  };
  bool my_done = all_done();

  for (uint32_t b0 = start; b0 < end; b0 += NB) {
    if (__syncthreads_count(!my_done) == 0) break;
    const int nb = (int)min((uint32_t)NB, end - b0);
#pragma unroll
    for (int k = 0; k < NBM; ++k) {
      const int slot = tid + k * NT;
      if (slot < nb) {
        const uint32_t item = __ldg(a.vals + b0 + slot);
        stage_record<true>(a.xy, a.conic_o, a.rgb_d, item, s_rec[slot]);
        if (IMPORTANCE) {
          s_h[slot] = 0u;
          s_gid[slot] = a.subset ? __ldg(a.subset + item) : (uint32_t)((int64_t)item - cam.item_base);
        }
      }
    }
    __syncthreads();
    const int base = (int)(b0 - start);
    for (int j = 0; j < nb; ++j) {
      const BlendRec r = s_rec[j];
      const ColTerms ct = col_terms(r, pair_dx(r, nu));
      float2 p2[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) p2[q] = pair_power(r, ct, pair_dy(r, nv[q]));
      // skip the record when no pixel of the warp is in its support; NaN (done) pixels drop
      // out of the maximum, and all done gives NaN, which compares false
      if (!__any_sync(0xffffffffu, max_p2(p2) >= r.bc.z)) continue;
      float m = 0.f;
      // An entry outside a pixel's support gets s = 0: weight 0 and T(1 - 0) = T exactly.
      // A live pixel keeps T >= 1e-4, so T(1 - alpha) < 1e-4 holds exactly for the pixels
      // whose stop rule fires on this entry; one comparison per pixel finds them, and the rare
      // stopping thread takes their s back to 0 and retires them before compositing.
      float2 s_in[NP], Tn[NP];
      bool stop = false;
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const PairAlpha al = pair_alpha<false>(r, p2[q]);
        // s where alpha >= 1/255, else 0 (the same decision as al.in0, al.in1, taken on the FMA pipe)
        s_in[q] = __fmul2_rn(al.s, make_float2(in_factor(al.s.x), in_factor(al.s.y)));
        Tn[q] = __fmul2_rn(T[q], one_minus_alpha(s_in[q]));
        stop = stop || Tn[q].x < kTMin || Tn[q].y < kTMin;
      }
      if (stop) {   // rare: retire the stopped pixels, their entry not composited
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          if (Tn[q].x < kTMin) {
            s_in[q].x = 0.f;
            Tn[q].x = T[q].x;
            nv[q].x = __int_as_float(0x7fc00000);
          }
          if (Tn[q].y < kTMin) {
            s_in[q].y = 0.f;
            Tn[q].y = T[q].y;
            nv[q].y = __int_as_float(0x7fc00000);
          }
        }
        my_done = all_done();
      }
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        // weight s T = alpha T / 0.99 against colours pre-scaled by 0.99
        const float2 w = __fmul2_rn(s_in[q], T[q]);
        T[q] = Tn[q];
        cr[q] = __ffma2_rn(w, lo2(r.rg), cr[q]);
        cg[q] = __ffma2_rn(w, hi2(r.rg), cg[q]);
        cb[q] = __ffma2_rn(w, lo2(r.bc), cb[q]);
        last[2 * q] = s_in[q].x > 0.f ? base + j + 1 : last[2 * q];
        last[2 * q + 1] = s_in[q].y > 0.f ? base + j + 1 : last[2 * q + 1];
        if (IMPORTANCE) m = max3f(m, w.x, w.y);
      }
      if (IMPORTANCE) {
        // the largest s T of the warp; alpha T = 0.99 s T (rounding is monotone, so scaling
        // the maximum equals the maximum of the scaled values)
        const uint32_t mm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
        if (lane == 0 && mm) atomicMax(&s_h[j], __float_as_uint(__fmul_rn(kAlphaMax, __uint_as_float(mm))));
      }
      if (__all_sync(0xffffffffu, my_done)) break;
    }
    __syncthreads();
    if (IMPORTANCE) {
#pragma unroll
      for (int k = 0; k < NBM; ++k) {
        const int slot = tid + k * NT;
        if (slot < nb) {
          const uint32_t mm = s_h[slot];
          if (mm && (int64_t)s_gid[slot] < a.n_gaussians) atomicMax(a.importance + s_gid[slot], mm);
        }
      }
    }
  }

  const int64_t HW = (int64_t)cam.width * cam.height;
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    if (!(pu < cam.width && pv0 + k < cam.height)) continue;
    const int q = k >> 1;
    const bool hi = k & 1;
    const float Tk = hi ? T[q].y : T[q].x;
    const int64_t pix = (int64_t)(pv0 + k) * cam.width + pu;
    if (a.image) {
      float* img = a.image + 3 * cam.pixel_base;
      img[pix] = (hi ? cr[q].y : cr[q].x) + Tk * a.bg0;
      img[HW + pix] = (hi ? cg[q].y : cg[q].x) + Tk * a.bg1;
      img[2 * HW + pix] = (hi ? cb[q].y : cb[q].x) + Tk * a.bg2;
    }
    if (a.T_final) a.T_final[cam.pixel_base + pix] = Tk;
    if (a.last) a.last[cam.pixel_base + pix] = last[k];
  }
}

template <int TW, int TH, int PX, int NBM>
static void launch_render(const RenderArgs& a, int n_tiles, bool imp, cudaStream_t s) {
  constexpr int NT = TW * TH / PX;
  prof::Scope ps(imp ? "k_render_importance" : "k_render", s);
  if (imp) k_render<TW, TH, PX, NBM, true><<<n_tiles, NT, 0, s>>>(a);
  else k_render<TW, TH, PX, NBM, false><<<n_tiles, NT, 0, s>>>(a);
}

// Records staged per thread and batch: cfg->batch / threads, one of 1, 2, 4 (0: 2).
template <int TW, int TH, int PX>
static rs_status launch_render_nb(const RenderArgs& a, int n_tiles, bool imp, int batch, cudaStream_t s) {
  constexpr int NT = TW * TH / PX;
  const int m = batch == 0 ? 2 : (batch % NT == 0 ? batch / NT : 0);
  if (m == 1) launch_render<TW, TH, PX, 1>(a, n_tiles, imp, s);
  else if (m == 2) launch_render<TW, TH, PX, 2>(a, n_tiles, imp, s);
  else if (m == 4) launch_render<TW, TH, PX, 4>(a, n_tiles, imp, s);
  else return RS_ERR_UNSUPPORTED;
  return RS_OK;
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
  const bool imp = importance != nullptr;
  rs_status st = RS_ERR_UNSUPPORTED;
  if (batch->tile_w == 16 && batch->tile_h == 16)
    st = launch_render_nb<16, 16, 8>(a, batch->n_tiles, imp, cfg->batch, s);
  else if (batch->tile_w == 32 && batch->tile_h == 8)
    st = launch_render_nb<32, 8, 8>(a, batch->n_tiles, imp, cfg->batch, s);
  else if (batch->tile_w == 8 && batch->tile_h == 8)
    st = launch_render_nb<8, 8, 2>(a, batch->n_tiles, imp, cfg->batch, s);
  if (st != RS_OK) return st;
  return launch_status();
}

static rs_status check_render_args(const rs_projected* proj, const rs_bins* bins, const rs_view_batch* batch,
                                   const rs_config* cfg) {
  if (!proj || !bins || !batch || !cfg) return RS_ERR_INVALID_ARG;
  if (!proj->xy || !proj->conic_o || !proj->rgb_d || !bins->vals || !bins->ranges || !batch->views)
    return RS_ERR_INVALID_ARG;
  if (batch->n_tiles < 0 || batch->n_views <= 0) return RS_ERR_INVALID_ARG;
  if (!blend_batch_ok(batch->tile_w, batch->tile_h, cfg->batch)) return RS_ERR_UNSUPPORTED;
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
