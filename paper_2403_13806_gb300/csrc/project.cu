// rs_project: EWA projection of every (view, Gaussian) item (Sec. 3.2 "Gaussian Splatting").
//
// Dense batches: one thread per Gaussian over all views (its parameters read from HBM once);
// visibility-list batches: one thread per item.  Reads are coalesced structure-of-arrays
// loads of the Gaussian parameters (236 B per Gaussian at SH degree 3); writes are one
// float2, two float4, one ushort4 and one uint32 per item.  The kernel is bound by HBM
// bandwidth.
#include <math.h>

#include "params.cuh"
#include "profile.cuh"
#include "radsplat.h"
#include "rs_common.cuh"
#include "sh.cuh"

namespace rs {

struct ProjectArgs {
  rs_gaussians g;
  const rs_view* views;
  const uint32_t* subset;
  int64_t n_items;
  int32_t n_views, tile_w, tile_h;
  int32_t tw_shift, th_shift;   // log2 of the tile sides (8, 16 or 32)
  float eps2d, near_plane;
  float2* xy;
  float4* conic_o;
  float4* rgb_d;
  ushort4* rect;
  uint32_t* n_tiles;
  rs_device_status* status;
};

// sqrt(x) by the hardware approximation (sqrt.approx.ftz, within a few ulps).
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// View-independent part of a Gaussian: rotation, scales and opacity (identical operations
// whichever view uses them).  Parameter rows as in params.cuh.
struct GaussLocal {
  float R[3][3];
  float s[3];
  float o;
  float q;    // 2 ln(255 o) clamped at 0: the support ellipse is d^T Sigma'^-1 d <= q
  bool fin;   // every parameter finite
  bool ok;    // finite, non-zero quaternion and o >= 1/255 (else the item is culled)
};

template <int D, typename P>
__device__ __forceinline__ GaussLocal gauss_local(const P& prm) {
  constexpr int NC = (D + 1) * (D + 1);
  GaussLocal gl;
  const float px = prm(0), py = prm(1), pz = prm(2);
  const float l0 = prm(3), l1 = prm(4), l2 = prm(5);
  const float qw = prm(6), qx = prm(7), qy = prm(8), qz = prm(9);
  const float lg = prm(10);
  bool fin = isfinite(px) && isfinite(py) && isfinite(pz) && isfinite(l0) && isfinite(l1) && isfinite(l2) &&
             isfinite(qw) && isfinite(qx) && isfinite(qy) && isfinite(qz) && isfinite(lg);
#pragma unroll
  for (int k = 0; k < 3 * NC; ++k) fin = fin && isfinite(prm(11 + k));
  gl.fin = fin;
  const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
  const float qi = rsqrtf(qn2);
  const float w = qw * qi, x = qx * qi, y = qy * qi, z = qz * qi;
  gl.R[0][0] = 1.f - 2.f * (y * y + z * z);
  gl.R[0][1] = 2.f * (x * y - w * z);
  gl.R[0][2] = 2.f * (x * z + w * y);
  gl.R[1][0] = 2.f * (x * y + w * z);
  gl.R[1][1] = 1.f - 2.f * (x * x + z * z);
  gl.R[1][2] = 2.f * (y * z - w * x);
  gl.R[2][0] = 2.f * (x * z - w * y);
  gl.R[2][1] = 2.f * (y * z + w * x);
  gl.R[2][2] = 1.f - 2.f * (x * x + y * y);
  gl.s[0] = expf(l0);
  gl.s[1] = expf(l1);
  gl.s[2] = expf(l2);
  gl.o = 1.f / (1.f + expf(-lg));
  gl.q = fmaxf(2.f * logf(255.f * gl.o), 0.f);
  gl.ok = fin && qn2 > 0.f && !(gl.o < kAlphaMin);
  return gl;
}

// One item: Gaussian gid (parameters prm, view-independent part gl) seen from view cam,
// written at row `item`.
template <int D, typename P>
__device__ __forceinline__ void project_view(const ProjectArgs& a, const rs_view& cam, const P& prm,
                                             const GaussLocal& gl, int64_t item) {
  constexpr int NC = (D + 1) * (D + 1);
  const float* W = cam.viewmat;
  const float px = prm(0), py = prm(1), pz = prm(2);
  // FP32 order key, written with an explicit fma chain so that any IEEE FP32 host
  // reproduces it bit for bit.
  const float depth = __fmaf_rn(W[8], px, __fmaf_rn(W[9], py, __fmaf_rn(W[10], pz, W[11])));

  float2 o_xy = make_float2(0.f, 0.f);
  float4 o_co = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 o_rgbd = make_float4(0.f, 0.f, 0.f, depth);
  ushort4 o_rect = make_ushort4(0, 0, 0, 0);
  uint32_t o_n = 0;

  do {
    if (!gl.fin) {
      if (a.status) atomicAdd(&a.status->nonfinite, 1);
      break;
    }
    if (!(depth > a.near_plane)) break;
    if (!gl.ok) break;

    const float tz = depth;
    const float tx = __fmaf_rn(W[0], px, __fmaf_rn(W[1], py, __fmaf_rn(W[2], pz, W[3])));
    const float ty = __fmaf_rn(W[4], px, __fmaf_rn(W[5], py, __fmaf_rn(W[6], pz, W[7])));
    const float ux = tx / tz, uy = ty / tz;
    const float uxc = fminf(fmaxf(ux, -cam.lim_x), cam.lim_x);
    const float uyc = fminf(fmaxf(uy, -cam.lim_y), cam.lim_y);
    // T = J M: row0 = fx/tz (M0 - uxc M2), row1 = fy/tz (M1 - uyc M2)
    // (the image mean above uses correctly rounded quotients; J and the conic below take the
    // hardware reciprocal: they feed only the blend, which tolerates their ulps)
    const float itz = rcp_approx(tz);
    const float jx = cam.fx * itz, jy = cam.fy * itz;
    float T[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T[0][c] = jx * (W[c] - uxc * W[8 + c]);
      T[1][c] = jy * (W[4 + c] - uyc * W[8 + c]);
    }
    // Sigma' = (T R S)(T R S)^T: positive semi-definite by construction
    float Mm[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        Mm[r][k] = (T[r][0] * gl.R[0][k] + T[r][1] * gl.R[1][k] + T[r][2] * gl.R[2][k]) * gl.s[k];
    const float s00 = Mm[0][0] * Mm[0][0] + Mm[0][1] * Mm[0][1] + Mm[0][2] * Mm[0][2];
    const float s01 = Mm[0][0] * Mm[1][0] + Mm[0][1] * Mm[1][1] + Mm[0][2] * Mm[1][2];
    const float s11 = Mm[1][0] * Mm[1][0] + Mm[1][1] * Mm[1][1] + Mm[1][2] * Mm[1][2];
    // det(M M^T) = |M0 x M1|^2 (Lagrange identity): no cancellation for thin Gaussians
    const float c0 = Mm[0][1] * Mm[1][2] - Mm[0][2] * Mm[1][1];
    const float c1 = Mm[0][2] * Mm[1][0] - Mm[0][0] * Mm[1][2];
    const float c2 = Mm[0][0] * Mm[1][1] - Mm[0][1] * Mm[1][0];
    const float det0 = c0 * c0 + c1 * c1 + c2 * c2;
    const float ea = s00 + a.eps2d, ec = s11 + a.eps2d;
    const float det = det0 + a.eps2d * (s00 + s11) + a.eps2d * a.eps2d;
    if (!(det > 0.f)) break;
    const float idet = rcp_approx(det);
    const float o = gl.o;

    const float mx = __fmaf_rn(cam.fx, ux, cam.cx);
    const float my = __fmaf_rn(cam.fy, uy, cam.cy);

    // support: alpha >= 1/255  <=>  d^T Sigma'^-1 d <= 2 ln(255 o); bounding box of that
    // ellipse, widened by a relative 2^-12 and 2^-10 px to stay a superset under rounding
    const float q = gl.q;
    const float ex = sqrt_approx(q * ea) * (1.f + 0x1p-12f) + 0x1p-10f;   // (margin >> its error)
    const float ey = sqrt_approx(q * ec) * (1.f + 0x1p-12f) + 0x1p-10f;
    const float u0 = fmaxf(ceilf(mx - ex), 0.f), u1 = fminf(floorf(mx + ex), (float)(cam.width - 1));
    const float v0 = fmaxf(ceilf(my - ey), 0.f), v1 = fminf(floorf(my + ey), (float)(cam.height - 1));

    // colour from SH along camera centre -> point
    float dx = px - cam.campos[0], dy = py - cam.campos[1], dz = pz - cam.campos[2];
    const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= dn;
    dy *= dn;
    dz *= dn;
    float Y[NC];
    sh::basis<D>(dx, dy, dz, Y);
    float col[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float acc = 0.5f;
#pragma unroll
      for (int k = 0; k < NC; ++k) acc = fmaf(prm(11 + 3 * k + c), Y[k], acc);
      col[c] = fmaxf(acc, 0.f);
    }

    o_xy = make_float2(mx, my);
    o_co = make_float4(ec * idet, -s01 * idet, ea * idet, o);
    o_rgbd = make_float4(col[0], col[1], col[2], depth);
    if (u0 <= u1 && v0 <= v1) {
      const int iu0 = (int)u0, iu1 = (int)u1, iv0 = (int)v0, iv1 = (int)v1;
      o_rect = make_ushort4((unsigned short)(iu0 >> a.tw_shift), (unsigned short)(iv0 >> a.th_shift),
                            (unsigned short)((iu1 >> a.tw_shift) + 1), (unsigned short)((iv1 >> a.th_shift) + 1));
      o_n = (uint32_t)(o_rect.z - o_rect.x) * (uint32_t)(o_rect.w - o_rect.y);
    }
  } while (false);

  a.xy[item] = o_xy;
  a.conic_o[item] = o_co;
  a.rgb_d[item] = o_rgbd;
  a.rect[item] = o_rect;
  a.n_tiles[item] = o_n;
}

// Visibility-list batches: one thread per item.
template <int D>
__global__ void __launch_bounds__(256) k_project(ProjectArgs a) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= a.n_items) return;
  const int v = find_view_by_item(a.views, a.n_views, item);
  const rs_view& cam = a.views[v];
  const int64_t gid = a.subset ? (int64_t)__ldg(a.subset + item) : item - cam.item_base;
  const RegParams<D> prm(GlobalParams{&a.g, gid});
  const GaussLocal gl = gauss_local<D>(prm);
  project_view<D>(a, cam, prm, gl, item);
}

// Dense batches (every view lists every Gaussian): one thread per Gaussian walks the views.
// The CTA's parameter block (one column per thread, 11 + 3 (D+1)^2 rows) is copied into
// shared memory with asynchronous 4-byte copies -- every load of the block in flight at
// once, no registers held -- so the 236 bytes of a Gaussian come from HBM once; rotation,
// scales and opacity are computed once for all views.
constexpr int kProjDenseThreads = 128;

template <int D>
__global__ void __launch_bounds__(kProjDenseThreads) k_project_dense(ProjectArgs a) {
  __shared__ float s_p[ParamRows<D>::value][kProjDenseThreads];
  const int64_t gid = (int64_t)blockIdx.x * kProjDenseThreads + threadIdx.x;
  if (gid >= a.g.n) return;   // no barrier below: each thread reads only its own column
  stage_params<D>(a.g, gid, &s_p[0][threadIdx.x], kProjDenseThreads);
  const SmemParams prm{&s_p[0][threadIdx.x], kProjDenseThreads};
  const GaussLocal gl = gauss_local<D>(prm);
#pragma unroll 1
  for (int v = 0; v < a.n_views; ++v) {
    const rs_view& cam = a.views[v];
    project_view<D>(a, cam, prm, gl, cam.item_base + gid);
  }
}

}  // namespace rs

using namespace rs;

extern "C" rs_status rs_project(const rs_gaussians* g, const rs_view_batch* batch, const rs_config* cfg,
                                const rs_projected* out, rs_device_status* status, void* stream) {
  if (!g || !batch || !cfg || !out) return RS_ERR_INVALID_ARG;
  if (g->sh_degree < 0 || g->sh_degree > 3) return RS_ERR_UNSUPPORTED;
  if (batch->n_items < 0 || batch->n_views < 0) return RS_ERR_INVALID_ARG;
  if (batch->n_items == 0) return RS_OK;
  if (!batch->views || batch->n_views == 0) return RS_ERR_INVALID_ARG;
  if (!g->means || !g->log_scales || !g->quats || !g->opacity_logit || !g->sh || g->n <= 0) return RS_ERR_INVALID_ARG;
  if (!batch->subset_idx && batch->n_items != (int64_t)batch->n_views * g->n) return RS_ERR_INVALID_ARG;
  if (!out->xy || !out->conic_o || !out->rgb_d || !out->rect || !out->n_tiles) return RS_ERR_INVALID_ARG;
  if (!aligned<float2>(out->xy, 8) || !aligned<float4>(out->conic_o, 16) || !aligned<float4>(out->rgb_d, 16) ||
      !aligned<ushort4>(out->rect, 8) || !aligned<uint32_t>(out->n_tiles, 4))
    return RS_ERR_INVALID_ARG;
  ProjectArgs a;
  a.g = *g;
  a.views = batch->views;
  a.subset = batch->subset_idx;
  a.n_items = batch->n_items;
  a.n_views = batch->n_views;
  a.tile_w = batch->tile_w;
  a.tile_h = batch->tile_h;
  if (!((a.tile_w == 8 || a.tile_w == 16 || a.tile_w == 32) && (a.tile_h == 8 || a.tile_h == 16)))
    return RS_ERR_UNSUPPORTED;
  a.tw_shift = a.tile_w == 8 ? 3 : a.tile_w == 16 ? 4 : 5;
  a.th_shift = a.tile_h == 8 ? 3 : 4;
  a.eps2d = cfg->eps2d;
  a.near_plane = cfg->near_plane;
  a.xy = reinterpret_cast<float2*>(out->xy);
  a.conic_o = reinterpret_cast<float4*>(out->conic_o);
  a.rgb_d = reinterpret_cast<float4*>(out->rgb_d);
  a.rect = reinterpret_cast<ushort4*>(out->rect);
  a.n_tiles = out->n_tiles;
  a.status = status;
  // one thread per Gaussian pays off once its parameters serve several views
  const bool dense = !batch->subset_idx && batch->n_views > 1;
  const int threads = dense ? kProjDenseThreads : 256;
  const int64_t blocks = ((dense ? g->n : batch->n_items) + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return RS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  prof::Scope ps("k_project", s);
  switch (g->sh_degree) {
    case 0: dense ? k_project_dense<0><<<(unsigned)blocks, threads, 0, s>>>(a)
                  : k_project<0><<<(unsigned)blocks, threads, 0, s>>>(a); break;
    case 1: dense ? k_project_dense<1><<<(unsigned)blocks, threads, 0, s>>>(a)
                  : k_project<1><<<(unsigned)blocks, threads, 0, s>>>(a); break;
    case 2: dense ? k_project_dense<2><<<(unsigned)blocks, threads, 0, s>>>(a)
                  : k_project<2><<<(unsigned)blocks, threads, 0, s>>>(a); break;
    default: dense ? k_project_dense<3><<<(unsigned)blocks, threads, 0, s>>>(a)
                   : k_project<3><<<(unsigned)blocks, threads, 0, s>>>(a); break;
  }
  return launch_status();
}
