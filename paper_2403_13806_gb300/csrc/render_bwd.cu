// rs_render_backward: derivative of Eq. (render-gs) (training loss of Sec. 3.2), in two
// kernels.
//
// k_render_bwd -- one CTA per (view, tile), two pixels per thread, the tile list walked back
//   to front from the largest `last` of the tile.  Each pixel recovers T_j = T_{j+1}/(1-a_j)
//   from its T_final and accumulates, per composited entry j,
//     dL/dc_j     = a_j T_j dL/dC
//     dL/da_j     = T_j (c_j . dL/dC) - (S_j . dL/dC + T_final bg . dL/dC) / (1 - a_j)
//   (S_j: colour composited behind j), and through a = o exp(power) (no gradient where the
//   0.99 clamp is active) the image-space gradients of the mean, conic and opacity.  The
//   nine values of a thread's two pixels are summed in registers, across the warp by
//   recursive halving (16 shuffles, only for entries some lane composited), across the
//   CTA through per-warp shared-memory slots, and added to per-item buffers with two
//   float4 and one float atomic per (tile, entry).
// k_project_bwd -- one thread per Gaussian (all views of the Gaussian summed in registers)
//   or, for visibility-list batches, one thread per item with atomic adds; chains the
//   image-space gradients through the inverse 2x2 conic, Sigma' = (T R S)(T R S)^T + eps I,
//   R(q/|q|), s = exp(log s), o = sigmoid(logit), the image mean and the SH colour
//   (including the view-direction term of the mean).
#include <math.h>

#include "profile.cuh"
#include "radsplat.h"
#include "blend.cuh"
#include "rs_common.cuh"
#include "sh.cuh"

namespace rs {

struct Grad2D {
  float4* ga;   // (d/dx, d/dy, d/da, d/db) of mean2d and conic (a, b, c)
  float4* gb;   // (d/dc, d/do, d/dr, d/dg)
  float* gc;    // d/db(lue)
};

struct BwdBlendArgs {
  const float2* xy;
  const float4* conic_o;
  const float4* rgb_d;
  const uint32_t* vals;
  const uint2* ranges;
  const rs_view* views;
  int32_t n_views;
  float bg0, bg1, bg2;
  const float* T_final;
  const int32_t* last;
  const float* dL_dimage;
  Grad2D g;
};

// Per-pixel state of the back-to-front walk.
struct BwdPixel {
  float T;      // transmittance after the current entry (T_final at the start)
  float G0, G1, G2;
  float bgG;    // T_final * (bg . dL/dC)
  float SG;     // (colour composited behind the current entry) . dL/dC
  int last;     // entries at positions >= last were not composited
};

// Adds the nine image-space gradient terms of entry e of one pixel into r (slots 0..8:
// d/dx, d/dy, d/da, d/db, d/dc, d/do, d/dr, d/dg, d/db(lue)); returns whether the entry was
// composited for this pixel.  The skip decisions replay the forward ones exactly.
__device__ __forceinline__ bool bwd_step(BwdPixel& p, const float4& g, const float4& g2, const float4& col, float fu,
                                         float fv, int e, float* r) {
  if (e >= p.last) return false;
  const float p2 = blend_power(g, g2, fu, fv);
  if (!(p2 <= 0.f && p2 >= g2.y)) return false;
  const float ex = exp2f(p2);
  const float raw = __fmul_rn(g2.z, ex);
  const float alpha = fminf(kAlphaMax, raw);
  if (alpha < kAlphaMin) return false;
  const float inv = __fdividef(1.f, 1.f - alpha);
  const float Tj = p.T * inv;
  const float w = alpha * Tj;
  const float cG = col.x * p.G0 + col.y * p.G1 + col.z * p.G2;
  const float dLda = Tj * cG - (p.SG + p.bgG) * inv;
  r[6] += w * p.G0;
  r[7] += w * p.G1;
  r[8] += w * p.G2;
  if (raw < kAlphaMax) {
    const float dLdpow = dLda * alpha;          // d alpha / d power = alpha
    r[5] += dLda * ex;                          // d alpha / d o = exp(power)
    // power = p2 ln 2, p2 = A dx^2 + B dx dy + C dy^2 with dx = mean - pixel
    const float dx = g.x - fu, dy = g.y - fv;
    const float k = dLdpow * 0.6931471805599453f;
    r[0] += k * (2.f * g.z * dx + g.w * dy);
    r[1] += k * (g.w * dx + 2.f * g2.x * dy);
    r[2] += -0.5f * dLdpow * dx * dx;
    r[3] += -dLdpow * dx * dy;
    r[4] += -0.5f * dLdpow * dy * dy;
  }
  p.SG = fmaf(w, cG, p.SG);
  p.T = Tj;
  return true;
}

// Sums v[0..15] over the warp by recursive halving: at each step a lane keeps half of its
// values and trades the other half with its partner, so the 16 sums take 16 shuffles.
// On return lanes 2c and 2c + 1 hold the warp total of component c.
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = hi ? v[i] : v[i + h];
      const float keep = hi ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW* TH / 2) k_render_bwd(BwdBlendArgs a) {
  constexpr int NT = TW * TH / 2;   // threads; each owns pixels (x, 2r) and (x, 2r + 1)
  constexpr int NW = NT / 32;
  constexpr int NB = NT;            // records per batch (one per thread: keeps shared memory < 48 KB)
  constexpr int PS = NB + 1;        // padded stride: the nine components land in distinct banks
  __shared__ float4 s_geo[NB];
  __shared__ float4 s_geo2[NB];
  __shared__ float4 s_col[NB];
  __shared__ uint32_t s_item[NB];
  __shared__ float s_part[NW][9 * PS];
  __shared__ int s_maxlast[NW];

  const int tile = blockIdx.x;
  const int v = find_view_by_tile(a.views, a.n_views, tile);
  const rs_view& cam = a.views[v];
  const int local = tile - cam.tile_base;
  const int tyi = local / cam.tiles_x;
  const int txi = local - tyi * cam.tiles_x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pu = txi * TW + (tid % TW);
  const int pv0 = tyi * TH + 2 * (tid / TW);
  const float fu = (float)pu;
  const uint2 rg = a.ranges[tile];
  const uint32_t start = rg.x;

  BwdPixel px[2];
  const int64_t HW = (int64_t)cam.width * cam.height;
  const float* gi = a.dL_dimage + 3 * cam.pixel_base;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    BwdPixel& p = px[k];
    p.T = 1.f;
    p.G0 = p.G1 = p.G2 = p.bgG = p.SG = 0.f;
    p.last = 0;
    if (pu < cam.width && pv0 + k < cam.height) {
      const int64_t pix = (int64_t)(pv0 + k) * cam.width + pu;
      p.G0 = gi[pix];
      p.G1 = gi[HW + pix];
      p.G2 = gi[2 * HW + pix];
      p.T = a.T_final[cam.pixel_base + pix];
      p.last = a.last[cam.pixel_base + pix];
      p.bgG = p.T * (a.bg0 * p.G0 + a.bg1 * p.G1 + a.bg2 * p.G2);
    }
  }
  const int my_last = max(px[0].last, px[1].last);
  int wl = my_last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
  if (lane == 0) s_maxlast[warp] = wl;
  __syncthreads();
  int max_last = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) max_last = max(max_last, s_maxlast[w]);

  for (int hi = max_last; hi > 0; hi -= NB) {
    const int lo = max(hi - NB, 0);
    const int nb = hi - lo;
    __syncthreads();
    if (tid < nb) {
      const uint32_t item = __ldg(a.vals + start + lo + tid);
      stage_record(a.xy, a.conic_o, a.rgb_d, item, s_geo[tid], s_geo2[tid], s_col[tid]);
      s_item[tid] = item;
    }
    __syncthreads();
    float* part = s_part[warp];
    for (int j = nb - 1; j >= 0; --j) {
      const int e = lo + j;
      if (!__any_sync(0xffffffffu, e < my_last)) {
        if (lane < 9) part[lane * PS + j] = 0.f;
        continue;
      }
      const float4 g = s_geo[j];
      const float4 g2 = s_geo2[j];
      const float4 col = s_col[j];
      float r[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) r[c] = 0.f;
      bool act = bwd_step(px[0], g, g2, col, fu, (float)pv0, e, r);
      act |= bwd_step(px[1], g, g2, col, fu, (float)(pv0 + 1), e, r);
      if (__any_sync(0xffffffffu, act)) {
        const float tot = warp_transpose_sum16(r);
        if ((lane & 1) == 0 && lane < 18) part[(lane >> 1) * PS + j] = tot;
      } else if (lane < 9) {
        part[lane * PS + j] = 0.f;
      }
    }
    __syncthreads();
    {
      const int slot = tid;
      if (slot < nb) {
        float c[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          float acc = 0.f;
#pragma unroll
          for (int w = 0; w < NW; ++w) acc += s_part[w][q * PS + slot];
          c[q] = acc;
        }
        bool nz = false;
#pragma unroll
        for (int q = 0; q < 9; ++q) nz |= (c[q] != 0.f);
        if (nz) {
          const uint32_t item = s_item[slot];
          atomicAdd(a.g.ga + item, make_float4(c[0], c[1], c[2], c[3]));
          atomicAdd(a.g.gb + item, make_float4(c[4], c[5], c[6], c[7]));
          atomicAdd(a.g.gc + item, c[8]);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ projection backward

struct BwdProjArgs {
  rs_gaussians g;
  const rs_view* views;
  const uint32_t* subset;
  int64_t n_items;
  int32_t n_views;
  float eps2d, near_plane;
  const float4* ga;
  const float4* gb;
  const float* gc;
  rs_gaussian_grads out;
};

template <int D>
struct ParamGrad {
  float m[3], ls[3], q[4], lg;
  float sh[(D + 1) * (D + 1)][3];
};

// Adds the parameter gradient of one item (view `cam`, Gaussian gid) into pg.
template <int D>
__device__ __forceinline__ void item_backward(const BwdProjArgs& a, const rs_view& cam, int64_t gid, float4 ga,
                                              float4 gb, float gcb, ParamGrad<D>& pg) {
  constexpr int NC = (D + 1) * (D + 1);
  const int64_t N = a.g.n;
  const float* W = cam.viewmat;
  const float px = __ldg(a.g.means + gid), py = __ldg(a.g.means + N + gid), pz = __ldg(a.g.means + 2 * N + gid);
  const float l0 = __ldg(a.g.log_scales + gid), l1 = __ldg(a.g.log_scales + N + gid),
              l2 = __ldg(a.g.log_scales + 2 * N + gid);
  const float qw = __ldg(a.g.quats + gid), qx = __ldg(a.g.quats + N + gid), qy = __ldg(a.g.quats + 2 * N + gid),
              qz = __ldg(a.g.quats + 3 * N + gid);
  const float lg = __ldg(a.g.opacity_logit + gid);

  // ---- forward recomputation (same formulas as the projection kernel)
  const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
  const float qi = rsqrtf(qn2);
  const float w = qw * qi, x = qx * qi, y = qy * qi, z = qz * qi;
  const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                         {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                         {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
  const float s[3] = {expf(l0), expf(l1), expf(l2)};
  const float tz = __fmaf_rn(W[8], px, __fmaf_rn(W[9], py, __fmaf_rn(W[10], pz, W[11])));
  const float tx = __fmaf_rn(W[0], px, __fmaf_rn(W[1], py, __fmaf_rn(W[2], pz, W[3])));
  const float ty = __fmaf_rn(W[4], px, __fmaf_rn(W[5], py, __fmaf_rn(W[6], pz, W[7])));
  const float ux = tx / tz, uy = ty / tz;
  const bool clx = !(ux > -cam.lim_x && ux < cam.lim_x), cly = !(uy > -cam.lim_y && uy < cam.lim_y);
  const float uxc = fminf(fmaxf(ux, -cam.lim_x), cam.lim_x);
  const float uyc = fminf(fmaxf(uy, -cam.lim_y), cam.lim_y);
  const float jx = cam.fx / tz, jy = cam.fy / tz;
  float T[2][3], Ebase[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Ebase[0][c] = W[c] - uxc * W[8 + c];
    Ebase[1][c] = W[4 + c] - uyc * W[8 + c];
    T[0][c] = jx * Ebase[0][c];
    T[1][c] = jy * Ebase[1][c];
  }
  float U[2][3], Mm[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      U[r][k] = T[r][0] * R[0][k] + T[r][1] * R[1][k] + T[r][2] * R[2][k];
      Mm[r][k] = U[r][k] * s[k];
    }
  const float s00 = Mm[0][0] * Mm[0][0] + Mm[0][1] * Mm[0][1] + Mm[0][2] * Mm[0][2];
  const float s01 = Mm[0][0] * Mm[1][0] + Mm[0][1] * Mm[1][1] + Mm[0][2] * Mm[1][2];
  const float s11 = Mm[1][0] * Mm[1][0] + Mm[1][1] * Mm[1][1] + Mm[1][2] * Mm[1][2];
  const float c0 = Mm[0][1] * Mm[1][2] - Mm[0][2] * Mm[1][1];
  const float c1 = Mm[0][2] * Mm[1][0] - Mm[0][0] * Mm[1][2];
  const float c2 = Mm[0][0] * Mm[1][1] - Mm[0][1] * Mm[1][0];
  const float det0 = c0 * c0 + c1 * c1 + c2 * c2;
  const float ea = s00 + a.eps2d, ec = s11 + a.eps2d;
  const float det = det0 + a.eps2d * (s00 + s11) + a.eps2d * a.eps2d;
  const float idet = 1.f / det;
  const float Qa = ec * idet, Qb = -s01 * idet, Qc = ea * idet;   // conic
  const float o = 1.f / (1.f + expf(-lg));

  // ---- conic -> Sigma':  G_Sigma = -Q G_Q Q with G_Q = [[ga, gb/2], [gb/2, gc]]
  const float gQa = ga.z, gQb = 0.5f * ga.w, gQc = gb.x;
  // P = Q G_Q
  const float P00 = Qa * gQa + Qb * gQb, P01 = Qa * gQb + Qb * gQc;
  const float P10 = Qb * gQa + Qc * gQb, P11 = Qb * gQb + Qc * gQc;
  const float GS00 = -(P00 * Qa + P01 * Qb);
  const float GS01 = -(P00 * Qb + P01 * Qc);
  const float GS11 = -(P10 * Qb + P11 * Qc);
  // ---- Sigma' = Mm Mm^T + eps I:  dL/dMm = 2 G_Sigma Mm
  float gM[2][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gM[0][k] = 2.f * (GS00 * Mm[0][k] + GS01 * Mm[1][k]);
    gM[1][k] = 2.f * (GS01 * Mm[0][k] + GS11 * Mm[1][k]);
  }
  // ---- Mm = U diag(s), U = T R
  float gU[2][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float gs = gM[0][k] * U[0][k] + gM[1][k] * U[1][k];
    pg.ls[k] += gs * s[k];
    gU[0][k] = gM[0][k] * s[k];
    gU[1][k] = gM[1][k] * s[k];
  }
  float gT[2][3], gR[3][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int i = 0; i < 3; ++i) gT[r][i] = gU[r][0] * R[i][0] + gU[r][1] * R[i][1] + gU[r][2] * R[i][2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) gR[i][k] = T[0][i] * gU[0][k] + T[1][i] * gU[1][k];
  // ---- R(q/|q|)
  {
    const float gw = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
    const float gx = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.f * x * gR[1][1] - w * gR[1][2] +
                            z * gR[2][0] + w * gR[2][1] - 2.f * x * gR[2][2]);
    const float gy = 2.f * (-2.f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                            w * gR[2][0] + z * gR[2][1] - 2.f * y * gR[2][2]);
    const float gz = 2.f * (-2.f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.f * z * gR[1][1] +
                            y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
    const float dotq = w * gw + x * gx + y * gy + z * gz;
    pg.q[0] += (gw - w * dotq) * qi;
    pg.q[1] += (gx - x * dotq) * qi;
    pg.q[2] += (gy - y * dotq) * qi;
    pg.q[3] += (gz - z * dotq) * qi;
  }
  // ---- T = [jx (W0 - uxc W2); jy (W1 - uyc W2)], jx = fx/tz, jy = fy/tz
  float gjx = 0.f, gjy = 0.f, guxc = 0.f, guyc = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gjx += gT[0][c] * Ebase[0][c];
    gjy += gT[1][c] * Ebase[1][c];
    guxc -= gT[0][c] * jx * W[8 + c];
    guyc -= gT[1][c] * jy * W[8 + c];
  }
  float gux = ga.x * cam.fx + (clx ? 0.f : guxc);
  float guy = ga.y * cam.fy + (cly ? 0.f : guyc);
  const float gtx = gux / tz, gty = guy / tz;
  const float gtz = -(gux * ux + guy * uy) / tz - (gjx * jx + gjy * jy) / tz;
  float gp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) gp[c] = W[c] * gtx + W[4 + c] * gty + W[8 + c] * gtz;

  // ---- colour: max(0, 0.5 + sum k Y(d)), d = normalise(p - campos)
  float dx = px - cam.campos[0], dy = py - cam.campos[1], dz = pz - cam.campos[2];
  const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
  dx *= dn;
  dy *= dn;
  dz *= dn;
  float Y[NC];
  sh::basis<D>(dx, dy, dz, Y);
  const float grgb[3] = {gb.z, gb.w, gcb};
  float gcol[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float acc = 0.5f;
#pragma unroll
    for (int k = 0; k < NC; ++k) acc = fmaf(__ldg(a.g.sh + (int64_t)(k * 3 + c) * N + gid), Y[k], acc);
    gcol[c] = acc > 0.f ? grgb[c] : 0.f;
  }
  float gY[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pg.sh[k][c] += gcol[c] * Y[k];
      t += gcol[c] * __ldg(a.g.sh + (int64_t)(k * 3 + c) * N + gid);
    }
    gY[k] = t;
  }
  if (D > 0) {
    float gdx, gdy, gdz;
    sh::basis_grad<D>(dx, dy, dz, gY, gdx, gdy, gdz);
    const float rad = gdx * dx + gdy * dy + gdz * dz;
    gp[0] += (gdx - rad * dx) * dn;
    gp[1] += (gdy - rad * dy) * dn;
    gp[2] += (gdz - rad * dz) * dn;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) pg.m[c] += gp[c];
  // ---- o = sigmoid(logit)
  pg.lg += gb.y * o * (1.f - o);
}

__device__ __forceinline__ bool any_grad(float4 ga, float4 gb, float gc) {
  return ga.x != 0.f || ga.y != 0.f || ga.z != 0.f || ga.w != 0.f || gb.x != 0.f || gb.y != 0.f || gb.z != 0.f ||
         gb.w != 0.f || gc != 0.f;
}

// Dense batches: item of Gaussian gid in view v is item_base[v] + gid; all views summed in
// registers, one read-modify-write of the parameter gradients.
template <int D>
__global__ void __launch_bounds__(128) k_project_bwd_dense(BwdProjArgs a) {
  constexpr int NC = (D + 1) * (D + 1);
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t N = a.g.n;
  if (gid >= N) return;
  ParamGrad<D> pg;
#pragma unroll
  for (int c = 0; c < 3; ++c) pg.m[c] = pg.ls[c] = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c) pg.q[c] = 0.f;
  pg.lg = 0.f;
#pragma unroll
  for (int k = 0; k < NC; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) pg.sh[k][c] = 0.f;
  bool touched = false;
  for (int v = 0; v < a.n_views; ++v) {
    const rs_view& cam = a.views[v];
    const int64_t item = cam.item_base + gid;
    const float4 ga = a.ga[item], gb = a.gb[item];
    const float gc = a.gc[item];
    if (!any_grad(ga, gb, gc)) continue;
    touched = true;
    item_backward<D>(a, cam, gid, ga, gb, gc, pg);
  }
  if (!touched) return;
  for (int c = 0; c < 3; ++c) {
    a.out.means[c * N + gid] += pg.m[c];
    a.out.log_scales[c * N + gid] += pg.ls[c];
  }
  for (int c = 0; c < 4; ++c) a.out.quats[c * N + gid] += pg.q[c];
  a.out.opacity_logit[gid] += pg.lg;
#pragma unroll
  for (int k = 0; k < NC; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) a.out.sh[(int64_t)(k * 3 + c) * N + gid] += pg.sh[k][c];
}

// Visibility-list batches: one thread per item, atomic adds (items of one Gaussian can sit
// in several views).
template <int D>
__global__ void __launch_bounds__(128) k_project_bwd_subset(BwdProjArgs a) {
  constexpr int NC = (D + 1) * (D + 1);
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= a.n_items) return;
  const float4 ga = a.ga[item], gb = a.gb[item];
  const float gc = a.gc[item];
  if (!any_grad(ga, gb, gc)) return;
  const int v = find_view_by_item(a.views, a.n_views, item);
  const int64_t gid = a.subset[item];
  const int64_t N = a.g.n;
  ParamGrad<D> pg;
#pragma unroll
  for (int c = 0; c < 3; ++c) pg.m[c] = pg.ls[c] = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c) pg.q[c] = 0.f;
  pg.lg = 0.f;
#pragma unroll
  for (int k = 0; k < NC; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) pg.sh[k][c] = 0.f;
  item_backward<D>(a, a.views[v], gid, ga, gb, gc, pg);
  for (int c = 0; c < 3; ++c) {
    atomicAdd(a.out.means + c * N + gid, pg.m[c]);
    atomicAdd(a.out.log_scales + c * N + gid, pg.ls[c]);
  }
  for (int c = 0; c < 4; ++c) atomicAdd(a.out.quats + c * N + gid, pg.q[c]);
  atomicAdd(a.out.opacity_logit + gid, pg.lg);
#pragma unroll
  for (int k = 0; k < NC; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(a.out.sh + (int64_t)(k * 3 + c) * N + gid, pg.sh[k][c]);
}

struct BwdWs {
  float4* ga;
  float4* gb;
  float* gc;
  size_t bytes;
};

static BwdWs bwd_ws_layout(void* base, int64_t n_items) {
  BwdWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? static_cast<char*>(base) + off : nullptr;
    off += align_up(bytes, 256);
    return p;
  };
  const size_t ni = (size_t)(n_items > 0 ? n_items : 1);
  w.ga = reinterpret_cast<float4*>(take(ni * 16));
  w.gb = reinterpret_cast<float4*>(take(ni * 16));
  w.gc = reinterpret_cast<float*>(take(ni * 4));
  w.bytes = off;
  return w;
}

size_t backward_ws_bytes(const rs_view_batch* batch) { return bwd_ws_layout(nullptr, batch->n_items).bytes; }

template <int TW, int TH>
static void launch_bwd_blend(const BwdBlendArgs& a, int n_tiles, cudaStream_t s) {
  prof::Scope ps("k_render_bwd", s);
  k_render_bwd<TW, TH><<<n_tiles, TW * TH / 2, 0, s>>>(a);
}

}  // namespace rs

using namespace rs;

extern "C" rs_status rs_render_backward(const rs_gaussians* g, const rs_view_batch* batch, const rs_config* cfg,
                                        const rs_projected* proj, const rs_bins* bins, const float* T_final,
                                        const int32_t* last, const float* dL_dimage,
                                        const rs_gaussian_grads* grads, void* ws, size_t ws_bytes, void* stream) {
  if (!g || !batch || !cfg || !proj || !bins || !T_final || !last || !dL_dimage || !grads) return RS_ERR_INVALID_ARG;
  if (g->sh_degree < 0 || g->sh_degree > 3) return RS_ERR_UNSUPPORTED;
  if (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logit || !grads->sh)
    return RS_ERR_INVALID_ARG;
  if (!batch->views || batch->n_views <= 0 || batch->n_items < 0 || g->n <= 0) return RS_ERR_INVALID_ARG;
  if (!batch->subset_idx && batch->n_items != (int64_t)batch->n_views * g->n) return RS_ERR_INVALID_ARG;
  const BwdWs w = bwd_ws_layout(ws, batch->n_items);
  if (!ws || ws_bytes < w.bytes || !aligned<float4>(ws, 256)) return RS_ERR_WORKSPACE;
  if (batch->n_items == 0 || batch->n_tiles == 0) return RS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(ws, 0, w.bytes, s) != cudaSuccess) return RS_ERR_CUDA;

  BwdBlendArgs b;
  b.xy = reinterpret_cast<const float2*>(proj->xy);
  b.conic_o = reinterpret_cast<const float4*>(proj->conic_o);
  b.rgb_d = reinterpret_cast<const float4*>(proj->rgb_d);
  b.vals = bins->vals;
  b.ranges = reinterpret_cast<const uint2*>(bins->ranges);
  b.views = batch->views;
  b.n_views = batch->n_views;
  b.bg0 = cfg->bg[0];
  b.bg1 = cfg->bg[1];
  b.bg2 = cfg->bg[2];
  b.T_final = T_final;
  b.last = last;
  b.dL_dimage = dL_dimage;
  b.g.ga = w.ga;
  b.g.gb = w.gb;
  b.g.gc = w.gc;
  if (batch->tile_w == 16 && batch->tile_h == 16) launch_bwd_blend<16, 16>(b, batch->n_tiles, s);
  else if (batch->tile_w == 32 && batch->tile_h == 8) launch_bwd_blend<32, 8>(b, batch->n_tiles, s);
  else if (batch->tile_w == 8 && batch->tile_h == 8) launch_bwd_blend<8, 8>(b, batch->n_tiles, s);
  else return RS_ERR_UNSUPPORTED;

  BwdProjArgs p;
  p.g = *g;
  p.views = batch->views;
  p.subset = batch->subset_idx;
  p.n_items = batch->n_items;
  p.n_views = batch->n_views;
  p.eps2d = cfg->eps2d;
  p.near_plane = cfg->near_plane;
  p.ga = w.ga;
  p.gb = w.gb;
  p.gc = w.gc;
  p.out = *grads;
  const int threads = 128;
  prof::Scope ps("k_project_bwd", s);
  if (!batch->subset_idx) {
    const unsigned blocks = (unsigned)((g->n + threads - 1) / threads);
    switch (g->sh_degree) {
      case 0: k_project_bwd_dense<0><<<blocks, threads, 0, s>>>(p); break;
      case 1: k_project_bwd_dense<1><<<blocks, threads, 0, s>>>(p); break;
      case 2: k_project_bwd_dense<2><<<blocks, threads, 0, s>>>(p); break;
      default: k_project_bwd_dense<3><<<blocks, threads, 0, s>>>(p); break;
    }
  } else {
    const unsigned blocks = (unsigned)((batch->n_items + threads - 1) / threads);
    switch (g->sh_degree) {
      case 0: k_project_bwd_subset<0><<<blocks, threads, 0, s>>>(p); break;
      case 1: k_project_bwd_subset<1><<<blocks, threads, 0, s>>>(p); break;
      case 2: k_project_bwd_subset<2><<<blocks, threads, 0, s>>>(p); break;
      default: k_project_bwd_subset<3><<<blocks, threads, 0, s>>>(p); break;
    }
  }
  return launch_status();
}
