// rs_render_backward: derivative of Eq. (render-gs) (training loss of Sec. 3.2), in two
// kernels.
//
// k_render_bwd -- one warp per (view, tile): eight pixels of a column per thread (two for 8x8
//   tiles) evaluated as pixel pairs with packed FP32 instructions, the tile list walked back
//   to front from the largest `last` of the tile.  Each pixel recovers T_j = T_{j+1}/(1-a_j)
//   from its T_final and accumulates, per composited entry j,
//     dL/dc_j     = a_j T_j dL/dC
//     dL/da_j     = T_j (c_j . dL/dC) - (S_j . dL/dC + T_final bg . dL/dC) / (1 - a_j)
//   (S_j: colour composited behind j), and through a = o exp(power) (no gradient where the
//   0.99 clamp is active) the image-space gradients of the mean, conic and opacity.  The
//   nine values of a thread's pixels are summed in registers, across the warp by
//   recursive halving (14 shuffles, only for entries some lane composited), across the
//   CTA through per-warp shared-memory slots, and added to per-item buffers with two
//   float4 and one float atomic per (tile, entry).
// k_project_bwd -- one thread per Gaussian (all views of the Gaussian summed in registers)
//   or, for visibility-list batches, one thread per item with atomic adds; chains the
//   image-space gradients through the inverse 2x2 conic, Sigma' = (T R S)(T R S)^T + eps I,
//   R(q/|q|), s = exp(log s), o = sigmoid(logit), the image mean and the SH colour
//   (including the view-direction term of the mean).
#include <math.h>

#include "params.cuh"
#include "profile.cuh"
#include "radsplat.h"
#include "blend.cuh"
#include "rs_common.cuh"
#include "sh.cuh"

namespace rs {

struct Grad2D {
  float4* ga;         // (d/dx, d/dy, d/da, d/db) of mean2d and conic (a, b, c)
  float4* gb;         // (d/dc, d/do, d/dr, d/dg)
  float* gc;          // d/db(lue)
  uint8_t* touched;   // 1 for every item the blend added to
};

// The backward workspace's state word after a completed call (xor the item count).
constexpr unsigned long long kBwdClean = 0x52534277734c6e21ull;

// Before the blend: zero the image-space gradients and flags of the items the previous call
// on this workspace touched, or of every item if the workspace is not in that call's clean
// state (first use, another item count, an interrupted call).
// In the clean state a thread reads the flags of 16 consecutive items as one 16-byte word
// (the flags start 256-byte aligned) and touches nothing more unless one is set; otherwise
// one thread per item zeroes everything, coalesced.
__global__ void k_bwd_prepare(Grad2D g, const unsigned long long* __restrict__ state, int64_t n) {
  const bool clean = *state == (kBwdClean ^ (unsigned long long)n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  auto zero = [&](int64_t i) {
    g.ga[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    g.gb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    g.gc[i] = 0.f;
    g.touched[i] = 0;
  };
  if (!clean) {
    for (int64_t i = t; i < n; i += stride) zero(i);
    return;
  }
  const int64_t n16 = n >> 4;
  uint4* flags = reinterpret_cast<uint4*>(g.touched);
  for (int64_t b = t; b < n16; b += stride) {
    const uint4 f = flags[b];
    if ((f.x | f.y | f.z | f.w) == 0u) continue;
    const uint32_t w[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if ((w[k >> 2] >> (8 * (k & 3))) & 0xffu) zero(16 * b + k);
  }
  for (int64_t i = 16 * n16 + t; i < n; i += stride)
    if (g.touched[i]) zero(i);
}

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

// Sums v[0..7] and s over the warp: v by recursive halving over lane bits 16, 8, 4 (7
// shuffles) and then plain butterflies over bits 2, 1; s by a plain butterfly (5 shuffles).
// On return lanes 4c .. 4c + 3 hold the warp total of v[c] (the return value) and every lane
// holds the total of s.
__device__ __forceinline__ float warp_transpose_sum8_plus1(float (&v)[8], float& s) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 4, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = hi ? v[i] : v[i + h];
      const float keep = hi ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  float t = v[0];
#pragma unroll
  for (int o = 2; o >= 1; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o);
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return t;
}

__device__ __forceinline__ float2 sel2(bool a, bool b, float2 x) {
  return make_float2(a ? x.x : 0.f, b ? x.y : 0.f);
}

// Back-to-front walk of one tile.  Per pixel pair q (lanes = the two pixels): T[q] is the
// transmittance after the current entry (T_final at the start), G*[q] = dL/dC per channel,
// SG[q] = (everything composited behind the current entry, the background's T_final bg
// included) . dL/dC -- it starts at T_final (bg . dL/dC); entries at positions >= last[k]
// were not composited for pixel k.  Per entry e the thread's pixels add up, with
// a = alpha_e and T_e = T/(1 - a):
//   d/dcolour = a T_e dL/dC,  dL/da = T_e (c . dL/dC) - SG/(1 - a),
// and, unless the 0.99 clamp was active, d/do = dL/da 2^p2 and with q = dL/da * a (the
// derivative with respect to the power) the moments sum(q), sum(q dy), sum(q dy^2); the
// column's common dx turns them into the mean and conic gradients.
template <int TW, int TH, int PX, int NBM>
__global__ void __launch_bounds__(TW* TH / PX, 16) k_render_bwd(BwdBlendArgs a) {
  constexpr int NT = TW * TH / PX;  // threads; each owns pixels (x, PX r + k), k < PX
  constexpr int NP = PX / 2;
  constexpr int NW = NT / 32;
  constexpr int NB = NBM * NT;      // records per batch (NBM per thread)
  constexpr int PS = NB + 1;        // padded stride: the nine components land in distinct banks
  __shared__ BlendRec s_rec[NB];
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
  const int pv0 = tyi * TH + PX * (tid / TW);
  const float2 nu = make_float2(-(float)pu, -(float)pu);
  const uint2 rg = a.ranges[tile];
  const uint32_t start = rg.x;

  float2 nv[NP], T[NP], Gr[NP], Gg[NP], Gb[NP], SG[NP];
  int last[PX];
  const int64_t HW = (int64_t)cam.width * cam.height;
  const float* gi = a.dL_dimage + 3 * cam.pixel_base;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    nv[q] = make_float2(-(float)(pv0 + 2 * q), -(float)(pv0 + 2 * q + 1));
    float t[2] = {1.f, 1.f}, g0[2] = {0.f, 0.f}, g1[2] = {0.f, 0.f}, g2[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * q + h;
      last[k] = 0;
      if (pu < cam.width && pv0 + k < cam.height) {
        const int64_t pix = (int64_t)(pv0 + k) * cam.width + pu;
        g0[h] = gi[pix];
        g1[h] = gi[HW + pix];
        g2[h] = gi[2 * HW + pix];
        t[h] = a.T_final[cam.pixel_base + pix];
        last[k] = a.last[cam.pixel_base + pix];
      }
    }
    T[q] = make_float2(t[0], t[1]);
    Gr[q] = make_float2(g0[0], g0[1]);
    Gg[q] = make_float2(g1[0], g1[1]);
    Gb[q] = make_float2(g2[0], g2[1]);
    SG[q] = make_float2(t[0] * (a.bg0 * g0[0] + a.bg1 * g1[0] + a.bg2 * g2[0]),
                        t[1] * (a.bg0 * g0[1] + a.bg1 * g1[1] + a.bg2 * g2[1]));
  }
  int my_last = 0;
#pragma unroll
  for (int k = 0; k < PX; ++k) my_last = max(my_last, last[k]);
  // gate[q] = (0 or NaN) per pixel: NaN until the walk reaches the pixel's last composited
  // entry (entry e is live for pixel k when e < last[k]); p2 + gate makes every test on a
  // pixel that is not live false without a per-pixel comparison of e.  next_live is the
  // largest entry at which a pixel still to be woken becomes live (-1: none).
  const float kNaN = __int_as_float(0x7fc00000);
  float2 gate[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) gate[q] = make_float2(kNaN, kNaN);
  int next_live = my_last - 1;
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
#pragma unroll
    for (int k = 0; k < NBM; ++k) {
      const int slot = tid + k * NT;
      if (slot < nb) {
        const uint32_t item = __ldg(a.vals + start + lo + slot);
        stage_record<false>(a.xy, a.conic_o, a.rgb_d, item, s_rec[slot]);
        s_item[slot] = item;
      }
    }
    __syncthreads();
    float* part = s_part[warp];
    for (int j = nb - 1; j >= 0; --j) {
      const int e = lo + j;
      if (e <= next_live) {   // rare: wake the pixels whose walk starts here
        int nl = -1;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          if (e < last[2 * q]) gate[q].x = 0.f; else nl = max(nl, last[2 * q] - 1);
          if (e < last[2 * q + 1]) gate[q].y = 0.f; else nl = max(nl, last[2 * q + 1] - 1);
        }
        next_live = nl;
      }
      const BlendRec r = s_rec[j];
      const float2 dx = pair_dx(r, nu);
      const ColTerms ct = col_terms(r, dx);
      float2 dy[NP], p2[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        dy[q] = pair_dy(r, nv[q]);
        p2[q] = __fadd2_rn(pair_power(r, ct, dy[q]), gate[q]);
      }
      // NaN (not live) pixels drop out of the maximum; none live gives NaN, which compares false
      if (!__any_sync(0xffffffffu, max_p2(p2) >= r.bc.z)) {
        if (lane < 9) part[lane * PS + j] = 0.f;
        continue;
      }
      float2 acc_r = make_float2(0.f, 0.f), acc_g = acc_r, acc_b = acc_r, acc_o = acc_r;
      float2 acc_q = acc_r, acc_qy = acc_r, acc_qyy = acc_r;
      bool act = false;
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const PairAlpha al = pair_alpha(r, p2[q]);
        act |= al.in0 || al.in1;
        // a skipped entry gets alpha 0: its weight is 0 and T_j = T exactly (1/(1 - 0) = 1)
        const float2 s_eff = sel2(al.in0, al.in1, al.s);
        const float2 om = one_minus_alpha(s_eff);
        const float2 a_eff = __fmul2_rn(make_float2(kAlphaMax, kAlphaMax), s_eff);
        // 1 / (1 - alpha) with alpha <= 0.99: the hardware reciprocal
        const float2 inv = make_float2(rcp_approx(om.x), rcp_approx(om.y));
        const float2 Tj = __fmul2_rn(T[q], inv);
        const float2 w = __fmul2_rn(a_eff, Tj);
        const float2 cG = __ffma2_rn(lo2(r.rg), Gr[q], __ffma2_rn(hi2(r.rg), Gg[q], __fmul2_rn(lo2(r.bc), Gb[q])));
        const float2 X = __fmul2_rn(SG[q], inv);
        const float2 dLda = __ffma2_rn(Tj, cG, make_float2(-X.x, -X.y));
        const float2 dl = sel2(al.in0 && al.s.x < 1.f, al.in1 && al.s.y < 1.f, dLda);
        acc_r = __ffma2_rn(w, Gr[q], acc_r);
        acc_g = __ffma2_rn(w, Gg[q], acc_g);
        acc_b = __ffma2_rn(w, Gb[q], acc_b);
        acc_o = __ffma2_rn(dl, al.ex, acc_o);
        const float2 qp = __fmul2_rn(dl, a_eff);   // d alpha / d power = alpha (dl = 0 off the support)
        const float2 qy = __fmul2_rn(qp, dy[q]);
        acc_q = __fadd2_rn(acc_q, qp);
        acc_qy = __fadd2_rn(acc_qy, qy);
        acc_qyy = __ffma2_rn(qy, dy[q], acc_qyy);
        SG[q] = __ffma2_rn(w, cG, SG[q]);
        T[q] = Tj;
      }
      if (__any_sync(0xffffffffu, act)) {
        // power = p2 ln 2, p2 = A dx^2 + B dx dy + C dy^2 with dx = x - u, dy = y - v
        const float Q = acc_q.x + acc_q.y, Qy = acc_qy.x + acc_qy.y, Qyy = acc_qyy.x + acc_qyy.y;
        const float d = dx.x;
        const float A = r.ab.x, B = r.ab.z, C = r.co.x;
        const float kl = 0.6931471805599453f;
        float rr[8];
        rr[0] = kl * (2.f * A * d * Q + B * Qy);
        rr[1] = kl * (B * d * Q + 2.f * C * Qy);
        rr[2] = -0.5f * d * d * Q;
        rr[3] = -d * Qy;
        rr[4] = -0.5f * Qyy;
        rr[5] = acc_o.x + acc_o.y;
        rr[6] = acc_r.x + acc_r.y;
        rr[7] = acc_g.x + acc_g.y;
        float r8 = acc_b.x + acc_b.y;
        const float tot = warp_transpose_sum8_plus1(rr, r8);
        if ((lane & 3) == 0) part[(lane >> 2) * PS + j] = tot;
        if (lane == 1) part[8 * PS + j] = r8;
      } else if (lane < 9) {
        part[lane * PS + j] = 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NBM; ++k) {
      const int slot = tid + k * NT;
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
          a.g.touched[item] = 1;
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
  const uint8_t* touched;         // items the blend gave a gradient (the others' are zero)
  unsigned long long* state;      // set to the clean state by the first thread
  const float4* rgb_d;   // forward colours: a clamped channel (max(0, .) = 0) has no gradient
  rs_gaussian_grads out;
  int32_t overwrite;     // dense kernel: store the sums instead of adding them
};

template <int D>
struct ParamGrad {
  float m[3], ls[3], q[4], lg;
  float sh[(D + 1) * (D + 1)][3];
};

// Adds the parameter gradient of one item (view `cam`, Gaussian gid) into pg.
// Where an item's SH gradient goes: the thread's registers (one item per thread), or a
// per-thread column of a shared-memory array (all views of a Gaussian summed there, which
// keeps 48 accumulators out of the registers).
template <int D>
struct RegSH {
  ParamGrad<D>& pg;
  __device__ __forceinline__ void add(int k, int c, float v) { pg.sh[k][c] += v; }
};
struct SmemSH {
  float* col;   // element (k, c) at col[(3 k + c) * stride]
  int stride;
  __device__ __forceinline__ void add(int k, int c, float v) { col[(3 * k + c) * stride] += v; }
};

template <int D, typename SH, typename P>
__device__ __forceinline__ void item_backward(const BwdProjArgs& a, const rs_view& cam, const P& prm, int64_t item,
                                              float4 ga, float4 gb, float gcb, ParamGrad<D>& pg, SH& shg) {
  constexpr int NC = (D + 1) * (D + 1);
  const float* W = cam.viewmat;
  const float px = prm(0), py = prm(1), pz = prm(2);
  const float l0 = prm(3), l1 = prm(4), l2 = prm(5);
  const float qw = prm(6), qx = prm(7), qy = prm(8), qz = prm(9);
  const float lg = prm(10);

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
  const float itz = rcp_approx(tz);   // as the projection: J and the conic from the reciprocal
  const float jx = cam.fx * itz, jy = cam.fy * itz;
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
  const float idet = rcp_approx(det);
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
  const float gtx = gux * itz, gty = guy * itz;
  const float gtz = -((gux * ux + guy * uy) + (gjx * jx + gjy * jy)) * itz;
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
  // the forward stored max(0, 0.5 + sum k Y): a channel it clamped to 0 gets no gradient
  const float4 fc = __ldg(a.rgb_d + item);
  const float gcol[3] = {fc.x > 0.f ? gb.z : 0.f, fc.y > 0.f ? gb.w : 0.f, fc.z > 0.f ? gcb : 0.f};
  float gY[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      shg.add(k, c, gcol[c] * Y[k]);
      t += gcol[c] * prm(11 + 3 * k + c);
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

constexpr int kProjBwdThreads = 128;

// Dense batches: item of Gaussian gid in view v is item_base[v] + gid; all views summed in
// registers, one read-modify-write of the parameter gradients.
template <int D>
__global__ void __launch_bounds__(kProjBwdThreads) k_project_bwd_dense(BwdProjArgs a) {
  constexpr int NC = (D + 1) * (D + 1);
  __shared__ float s_gsh[3 * NC][kProjBwdThreads];
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t N = a.g.n;
  if (gid >= N) return;   // no barrier below: each thread owns its column
  // the workspace is clean once this call completes (read only by the next call's prepare)
  if (gid == 0) *a.state = kBwdClean ^ (unsigned long long)a.n_items;
  ParamGrad<D> pg;
#pragma unroll
  for (int c = 0; c < 3; ++c) pg.m[c] = pg.ls[c] = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c) pg.q[c] = 0.f;
  pg.lg = 0.f;
#pragma unroll
  for (int k = 0; k < 3 * NC; ++k) s_gsh[k][threadIdx.x] = 0.f;
  SmemSH shg{&s_gsh[0][threadIdx.x], kProjBwdThreads};
  // (parameters straight from HBM: a Gaussian no view has a gradient for reads none, and
  // later views find them in L1; staging them in shared memory measured slower)
  const GlobalParams prm{&a.g, gid};
  bool touched = false;
  for (int v = 0; v < a.n_views; ++v) {
    const rs_view& cam = a.views[v];
    const int64_t item = cam.item_base + gid;
    if (!a.touched[item]) continue;   // 1 byte instead of the 36 of a zero gradient
    const float4 ga = a.ga[item], gb = a.gb[item];
    const float gc = a.gc[item];
    if (!any_grad(ga, gb, gc)) continue;
    touched = true;
    item_backward<D>(a, cam, prm, item, ga, gb, gc, pg, shg);
  }
  if (a.overwrite) {   // every Gaussian's row is written (zeros where no view touched it)
    for (int c = 0; c < 3; ++c) {
      a.out.means[c * N + gid] = pg.m[c];
      a.out.log_scales[c * N + gid] = pg.ls[c];
    }
    for (int c = 0; c < 4; ++c) a.out.quats[c * N + gid] = pg.q[c];
    a.out.opacity_logit[gid] = pg.lg;
#pragma unroll
    for (int k = 0; k < 3 * NC; ++k) a.out.sh[(int64_t)k * N + gid] = s_gsh[k][threadIdx.x];
    return;
  }
  if (!touched) return;
  // The old values are read a group at a time before the group's writes: the compiler cannot
  // tell the rows' addresses apart, so a plain += per row would chain every read behind the
  // previous write (one memory round trip per row instead of one per group).
  {
    float o[11];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      o[c] = a.out.means[c * N + gid];
      o[3 + c] = a.out.log_scales[c * N + gid];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) o[6 + c] = a.out.quats[c * N + gid];
    o[10] = a.out.opacity_logit[gid];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a.out.means[c * N + gid] = o[c] + pg.m[c];
      a.out.log_scales[c * N + gid] = o[3 + c] + pg.ls[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) a.out.quats[c * N + gid] = o[6 + c] + pg.q[c];
    a.out.opacity_logit[gid] = o[10] + pg.lg;
  }
#pragma unroll
  for (int k0 = 0; k0 < 3 * NC; k0 += 8) {
    float o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k0 + j < 3 * NC) o[j] = a.out.sh[(int64_t)(k0 + j) * N + gid];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k0 + j < 3 * NC) a.out.sh[(int64_t)(k0 + j) * N + gid] = o[j] + s_gsh[k0 + j][threadIdx.x];
  }
}

// Visibility-list batches: one thread per item, atomic adds (items of one Gaussian can sit
// in several views).
template <int D>
__global__ void __launch_bounds__(128) k_project_bwd_subset(BwdProjArgs a) {
  constexpr int NC = (D + 1) * (D + 1);
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= a.n_items) return;
  if (item == 0) *a.state = kBwdClean ^ (unsigned long long)a.n_items;
  if (!a.touched[item]) return;
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
  RegSH<D> shg{pg};
  const GlobalParams prm{&a.g, gid};
  item_backward<D>(a, a.views[v], prm, item, ga, gb, gc, pg, shg);
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

// Workspace: a state word, then the per-item image-space gradients and touched flags.  A
// completed call leaves state = kBwdClean ^ n_items and every gradient of an item without
// its flag zero, so the next call on the same workspace zeroes only the flagged items; any
// other state (first use, another item count, an interrupted call) zeroes everything.
struct BwdWs {
  unsigned long long* state;
  float4* ga;
  float4* gb;
  float* gc;
  uint8_t* touched;
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
  w.state = reinterpret_cast<unsigned long long*>(take(8));
  w.ga = reinterpret_cast<float4*>(take(ni * 16));
  w.gb = reinterpret_cast<float4*>(take(ni * 16));
  w.gc = reinterpret_cast<float*>(take(ni * 4));
  w.touched = reinterpret_cast<uint8_t*>(take(ni));
  w.bytes = off;
  return w;
}

size_t backward_ws_bytes(const rs_view_batch* batch) { return bwd_ws_layout(nullptr, batch->n_items).bytes; }

}  // namespace rs

extern "C" rs_status rs_backward_image_grads(const rs_view_batch* batch, void* ws, size_t ws_bytes,
                                             rs_image_grads* out) {
  if (!batch || !ws || !out || batch->n_items < 0) return RS_ERR_INVALID_ARG;
  const rs::BwdWs w = rs::bwd_ws_layout(ws, batch->n_items);
  if (ws_bytes < w.bytes) return RS_ERR_WORKSPACE;
  out->g_xy_ab = reinterpret_cast<const float*>(w.ga);
  out->g_c_o_rg = reinterpret_cast<const float*>(w.gb);
  out->g_b = w.gc;
  return RS_OK;
}

namespace rs {

// One warp per tile (PX = 8 pixels per thread for 16x16 and 32x8 tiles, 2 for 8x8): the
// per-entry warp reduction serves 256 (64) pixels and no cross-warp partials are needed.
// Records staged per batch: cfg->batch (the same count as the forward stages), i.e.
// cfg->batch / 32 per thread, one of 1, 2, 4, 8 (0: 64 records).
template <int TW, int TH, int PX>
static rs_status launch_bwd_blend(const BwdBlendArgs& a, int n_tiles, int batch, cudaStream_t s) {
  constexpr int NT = TW * TH / PX;
  static_assert(NT == 32, "one warp per tile");
  const int m = batch == 0 ? 2 : (batch % NT == 0 ? batch / NT : 0);
  if (m != 1 && m != 2 && m != 4 && m != 8) return RS_ERR_UNSUPPORTED;
  prof::Scope ps("k_render_bwd", s);
  if (m == 1) k_render_bwd<TW, TH, PX, 1><<<n_tiles, NT, 0, s>>>(a);
  else if (m == 2) k_render_bwd<TW, TH, PX, 2><<<n_tiles, NT, 0, s>>>(a);
  else if (m == 4) k_render_bwd<TW, TH, PX, 4><<<n_tiles, NT, 0, s>>>(a);
  else k_render_bwd<TW, TH, PX, 8><<<n_tiles, NT, 0, s>>>(a);
  return RS_OK;
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
  if (!blend_batch_ok(batch->tile_w, batch->tile_h, cfg->batch)) return RS_ERR_UNSUPPORTED;
  const BwdWs w = bwd_ws_layout(ws, batch->n_items);
  if (!ws || ws_bytes < w.bytes || !aligned<float4>(ws, 256)) return RS_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool overwrite = cfg->grad_overwrite != 0;
  // overwrite with the atomic (visibility-list) kernel, or with nothing to add: zero first
  if (overwrite && (batch->subset_idx || batch->n_items == 0 || batch->n_tiles == 0)) {
    const size_t nb = (size_t)g->n * sizeof(float);
    const size_t nsh = (size_t)3 * (g->sh_degree + 1) * (g->sh_degree + 1);
    if (cudaMemsetAsync(grads->means, 0, 3 * nb, s) != cudaSuccess ||
        cudaMemsetAsync(grads->log_scales, 0, 3 * nb, s) != cudaSuccess ||
        cudaMemsetAsync(grads->quats, 0, 4 * nb, s) != cudaSuccess ||
        cudaMemsetAsync(grads->opacity_logit, 0, nb, s) != cudaSuccess ||
        cudaMemsetAsync(grads->sh, 0, nsh * nb, s) != cudaSuccess)
      return RS_ERR_CUDA;
  }
  if (batch->n_items == 0 || batch->n_tiles == 0) return RS_OK;
  const Grad2D g2{w.ga, w.gb, w.gc, w.touched};
  {
    prof::Scope ps("k_bwd_prepare", s);
    // (the clean path covers 16 items per thread; a grid of a few waves strides over the rest)
    const int64_t pg = (batch->n_items / 16 + 255) / 256 + 1;
    k_bwd_prepare<<<(unsigned)(pg < 8 * kNumSMs ? pg : 8 * kNumSMs), 256, 0, s>>>(g2, w.state, batch->n_items);
  }

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
  b.g = g2;
  rs_status bst = RS_ERR_UNSUPPORTED;
  if (batch->tile_w == 16 && batch->tile_h == 16) bst = launch_bwd_blend<16, 16, 8>(b, batch->n_tiles, cfg->batch, s);
  else if (batch->tile_w == 32 && batch->tile_h == 8) bst = launch_bwd_blend<32, 8, 8>(b, batch->n_tiles, cfg->batch, s);
  else if (batch->tile_w == 8 && batch->tile_h == 8) bst = launch_bwd_blend<8, 8, 2>(b, batch->n_tiles, cfg->batch, s);
  if (bst != RS_OK) return bst;

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
  p.touched = w.touched;
  p.state = w.state;
  p.rgb_d = reinterpret_cast<const float4*>(proj->rgb_d);
  p.out = *grads;
  p.overwrite = (overwrite && !batch->subset_idx) ? 1 : 0;
  const int threads = 128;
  prof::Scope ps("k_project_bwd", s);
  if (!batch->subset_idx) {
    const int dt = kProjBwdThreads;
    const unsigned blocks = (unsigned)((g->n + dt - 1) / dt);
    switch (g->sh_degree) {
      case 0: k_project_bwd_dense<0><<<blocks, dt, 0, s>>>(p); break;
      case 1: k_project_bwd_dense<1><<<blocks, dt, 0, s>>>(p); break;
      case 2: k_project_bwd_dense<2><<<blocks, dt, 0, s>>>(p); break;
      default: k_project_bwd_dense<3><<<blocks, dt, 0, s>>>(p); break;
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
