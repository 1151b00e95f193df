// rs_ssim_loss: the training loss of Sec. 3.2, L = (1 - lambda) mean((x - y)^2) +
// lambda (1 - mean SSIM(x, y)), and its gradient with respect to the rendered image x, for
// planes [n_planes][H][W] (the channels of one or more same-sized views).
//
// SSIM per plane and pixel p uses the normalised 11 x 11 Gaussian window (sigma 1.5) over
// the zero-padded planes; with mu = w * x etc. and C1 = 0.01^2, C2 = 0.03^2,
//   SSIM_p = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)).
// Its derivative is dSSIM_p/dx(q) = w(p - q)(a(p) + b(p) x(q) + c(p) y(q)) with per-pixel
// maps a, b, c (the chain rule through mu_x, E[x^2], E[xy]), so
//   dL/dx(q) = (1 - lambda) 2 (x - y)(q)/n - lambda/n ((w * a)(q) + x(q)(w * b)(q) + y(q)(w * c)(q)).
//
// Two kernels, each on 32 x 32-pixel tiles of one plane with a 5-pixel halo in shared memory
// and the window applied as two 11-tap passes (rows, then columns; the window is separable:
// the outer product of the normalised 1D Gaussian):
//   k_ssim_stats -- the five window moments, SSIM, the maps a, b, c (to the workspace) and the
//                   block sums of SSIM and of the squared error (double atomics);
//   k_ssim_grad  -- the three filtered maps and the gradient; the first block also writes L.
// Recomputing the moments over the halo instead (one fused kernel) would cost ~2.5 x the
// arithmetic to save 24 bytes of traffic per value; at GB300's balance the maps are cheaper.
#include <math.h>

#include "profile.cuh"
#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {

constexpr int kSR = 5;                 // window radius
constexpr int kTaps = 2 * kSR + 1;
constexpr int kST = 32;                // output tile: kST x kST
constexpr int kSH = kST + 2 * kSR;     // tile with the halo: 42 x 42
constexpr int kSThreads = 256;
constexpr int kRowOut = 8;             // row pass: adjacent outputs per task
constexpr int kColOut = 4;             // column pass: adjacent outputs per task
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;
constexpr int kSlots = 64;             // block sums go to 64 addresses (no single hot atomic)

struct SsimArgs {
  const float* x;
  const float* y;
  float* maps;          // [3][planes][H][W]
  double* sums;         // [2][kSlots]: sums of SSIM and of squared errors, spread over slots
  float* grad;
  double* loss;
  int W, H, planes;
  float lambda;
  float w[kTaps];       // normalised 1D Gaussian, sigma 1.5
};


// Halo tile rows are loaded by columns: thread t < 252 takes column t % 42 of rows
// t / 42 + 6 p (p < 7), so the index arithmetic is done once per thread.
constexpr int kLoadRows = kSThreads / kSH;   // 6 rows per round
constexpr int kLoadRounds = kSH / kLoadRows; // 7 rounds
static_assert(kLoadRows * kLoadRounds == kSH, "halo rows per load round");

// Shared-memory layouts interleave what a tap reads together (x with y; the five moments
// as a float4 plus a float), the row pass produces 8 adjacent outputs and the column pass 4
// per task from values loaded once, and row pitches keep 8-lane phases of 16-byte accesses
// on distinct bank groups.
__global__ void __launch_bounds__(kSThreads) k_ssim_stats(SsimArgs a) {
  __shared__ __align__(16) float2 sxy[kSH][kSH];         // (x, y) with the halo
  __shared__ __align__(16) float4 hq[kSH][kST + 1];      // row-filtered (mu_x, mu_y, E[x^2], E[y^2])
  __shared__ float hxy[kSH][kST + 1];                    // row-filtered E[xy]
  __shared__ float2 s_w2[kTaps];
  __shared__ float red[2][kSThreads / 32];
  const int x0 = blockIdx.x * kST, y0 = blockIdx.y * kST, pl = blockIdx.z;
  const int64_t plane = (int64_t)a.W * a.H;
  const float* X = a.x + pl * plane;
  const float* Y = a.y + pl * plane;
  const int t = threadIdx.x;
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < kTaps; ++k) s_w2[k] = make_float2(a.w[k], a.w[k]);   // (static indices)
  }
  if (t < kLoadRows * kSH) {
    const int c = t % kSH, r0 = t / kSH;
    const int gx = x0 + c - kSR;
    const bool cin = gx >= 0 && gx < a.W;
    float2 v[kLoadRounds];
#pragma unroll
    for (int p = 0; p < kLoadRounds; ++p) {
      const int gy = y0 + r0 + kLoadRows * p - kSR;
      const int64_t o = (int64_t)gy * a.W + gx;
      v[p] = (cin && gy >= 0 && gy < a.H) ? make_float2(__ldg(X + o), __ldg(Y + o)) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int p = 0; p < kLoadRounds; ++p) sxy[r0 + kLoadRows * p][c] = v[p];
  }
  __syncthreads();
  // the window weights as (w, w) register pairs for the packed FP32 instructions, read once
  // per thread from shared memory (so they stay in registers across the unrolled passes)
  float2 w2[kTaps];
#pragma unroll
  for (int k = 0; k < kTaps; ++k) w2[k] = s_w2[k];
  // rows: kRowOut adjacent outputs per task, kSH rows x (kST / kRowOut) groups
  if (t < kSH * (kST / kRowOut)) {
    const int r = t % kSH, c0 = kRowOut * (t / kSH);
    // (mu_x, mu_y) and (E[x^2], E[y^2]) advance as packed pairs, E[xy] alone
    float2 m1[kRowOut], m2[kRowOut];
    float m3[kRowOut];
#pragma unroll
    for (int j = 0; j < kRowOut; ++j) {
      m1[j] = m2[j] = make_float2(0.f, 0.f);
      m3[j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kRowOut + 2 * kSR; k += 2) {
      const float4 q = *reinterpret_cast<const float4*>(&sxy[r][c0 + k]);
      const float2 vv[2] = {make_float2(q.x, q.y), make_float2(q.z, q.w)};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 v = vv[h];
        const float2 sq = __fmul2_rn(v, v);
        const float xy = v.x * v.y;
#pragma unroll
        for (int j = 0; j < kRowOut; ++j) {
          const int tap = k + h - j;
          if (tap < 0 || tap >= kTaps) continue;   // resolved at compile time
          m1[j] = __ffma2_rn(w2[tap], v, m1[j]);
          m2[j] = __ffma2_rn(w2[tap], sq, m2[j]);
          m3[j] = fmaf(w2[tap].x, xy, m3[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kRowOut; ++j) {
      hq[r][c0 + j] = make_float4(m1[j].x, m1[j].y, m2[j].x, m2[j].y);
      hxy[r][c0 + j] = m3[j];
    }
  }
  __syncthreads();
  // columns: kColOut adjacent rows per task, kST columns x (kST / kColOut) groups (one warp
  // per group, a lane per column)
  const int64_t total = plane * a.planes;
  float s_sum = 0.f, e_sum = 0.f;
  {
    const int c = t % kST, r0 = kColOut * (t / kST);
    float2 m1[kColOut], m2[kColOut];
    float m3[kColOut];
#pragma unroll
    for (int j = 0; j < kColOut; ++j) {
      m1[j] = m2[j] = make_float2(0.f, 0.f);
      m3[j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kColOut + 2 * kSR; ++k) {
      const float4 hv = hq[r0 + k][c];
      const float hz = hxy[r0 + k][c];
      const float2 h01 = make_float2(hv.x, hv.y), h23 = make_float2(hv.z, hv.w);
#pragma unroll
      for (int j = 0; j < kColOut; ++j) {
        const int tap = k - j;
        if (tap < 0 || tap >= kTaps) continue;
        m1[j] = __ffma2_rn(w2[tap], h01, m1[j]);
        m2[j] = __ffma2_rn(w2[tap], h23, m2[j]);
        m3[j] = fmaf(w2[tap].x, hz, m3[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kColOut; ++j) {
      const int r = r0 + j;
      const int gy = y0 + r, gx = x0 + c;
      if (gx >= a.W || gy >= a.H) continue;
      const float mx = m1[j].x, my = m1[j].y, exx = m2[j].x, eyy = m2[j].y, exy = m3[j];
      const float sxx = exx - mx * mx, syy = eyy - my * my, sxy_ = exy - mx * my;
      const float ln = 2.f * mx * my + kC1, ld = mx * mx + my * my + kC1;
      const float cn = 2.f * sxy_ + kC2, cd = sxx + syy + kC2;
      // two reciprocals give all four: 1/ln = ld q1, 1/ld = ln q1, 1/cn = cd q2, 1/cd = cn q2
      // (the hardware approximation: the products are normal, positive numbers)
      const float q1 = rcp_approx(ln * ld), q2 = rcp_approx(cn * cd);
      const float s = (ln * ln * q1) * (cn * cn * q2);
      const float d_mx = s * (2.f * my * ld - 2.f * mx * ln) * q1;
      const float d_sxx = -s * cn * q2;
      const float d_sxy = 2.f * s * cd * q2;
      const int64_t o = pl * plane + (int64_t)gy * a.W + gx;
      a.maps[o] = d_mx - 2.f * mx * d_sxx - my * d_sxy;
      a.maps[total + o] = 2.f * d_sxx;
      a.maps[2 * total + o] = d_sxy;
      s_sum += s;
      const float2 xy = sxy[r + kSR][c + kSR];
      const float d = xy.x - xy.y;
      e_sum = fmaf(d, d, e_sum);
    }
  }
  // block sums -> one double atomic each
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s_sum += __shfl_xor_sync(0xffffffffu, s_sum, o);
    e_sum += __shfl_xor_sync(0xffffffffu, e_sum, o);
  }
  const int warp = t >> 5, lane = t & 31;
  if (lane == 0) {
    red[0][warp] = s_sum;
    red[1][warp] = e_sum;
  }
  __syncthreads();
  if (t == 0) {
    double ss = 0.0, e = 0.0;
    for (int w = 0; w < kSThreads / 32; ++w) {
      ss += red[0][w];
      e += red[1][w];
    }
    const int slot = (blockIdx.x + 7 * blockIdx.y + 13 * blockIdx.z) % kSlots;
    atomicAdd(&a.sums[slot], ss);
    atomicAdd(&a.sums[kSlots + slot], e);
  }
}

__global__ void __launch_bounds__(kSThreads) k_ssim_grad(SsimArgs a) {
  __shared__ __align__(16) float2 sab[kSH][kSH];     // (a, b) with the halo
  __shared__ float sc[kSH][kSH + 1];                 // c with the halo (odd row pitch)
  __shared__ __align__(16) float2 hab[kSH][kST + 1]; // row-filtered (a, b)
  __shared__ float hc[kSH][kST + 1];                 // row-filtered c
  __shared__ float2 s_w2[kTaps];
  const int x0 = blockIdx.x * kST, y0 = blockIdx.y * kST, pl = blockIdx.z;
  const int64_t plane = (int64_t)a.W * a.H;
  const int64_t total = plane * a.planes;
  const int t = threadIdx.x;
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < kTaps; ++k) s_w2[k] = make_float2(a.w[k], a.w[k]);   // (static indices)
  }
  if (t < kLoadRows * kSH) {
    const int c = t % kSH, r0 = t / kSH;
    const int gx = x0 + c - kSR;
    const bool cin = gx >= 0 && gx < a.W;
    float2 vab[kLoadRounds];
    float vc[kLoadRounds];
#pragma unroll
    for (int p = 0; p < kLoadRounds; ++p) {
      const int gy = y0 + r0 + kLoadRows * p - kSR;
      const int64_t o = pl * plane + (int64_t)gy * a.W + gx;
      const bool in = cin && gy >= 0 && gy < a.H;
      vab[p] = in ? make_float2(__ldg(a.maps + o), __ldg(a.maps + total + o)) : make_float2(0.f, 0.f);
      vc[p] = in ? __ldg(a.maps + 2 * total + o) : 0.f;
    }
#pragma unroll
    for (int p = 0; p < kLoadRounds; ++p) {
      sab[r0 + kLoadRows * p][c] = vab[p];
      sc[r0 + kLoadRows * p][c] = vc[p];
    }
  }
  __syncthreads();
  // the window weights as (w, w) register pairs for the packed FP32 instructions, read once
  // per thread from shared memory (so they stay in registers across the unrolled passes)
  float2 w2[kTaps];
#pragma unroll
  for (int k = 0; k < kTaps; ++k) w2[k] = s_w2[k];
  if (t < kSH * (kST / kRowOut)) {
    const int r = t % kSH, c0 = kRowOut * (t / kSH);
    float2 mab[kRowOut];
    float mc[kRowOut];
#pragma unroll
    for (int j = 0; j < kRowOut; ++j) {
      mab[j] = make_float2(0.f, 0.f);
      mc[j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kRowOut + 2 * kSR; k += 2) {
      const float4 q = *reinterpret_cast<const float4*>(&sab[r][c0 + k]);
      const float2 vv[2] = {make_float2(q.x, q.y), make_float2(q.z, q.w)};
      const float cc[2] = {sc[r][c0 + k], sc[r][c0 + k + 1]};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int j = 0; j < kRowOut; ++j) {
          const int tap = k + h - j;
          if (tap < 0 || tap >= kTaps) continue;
          mab[j] = __ffma2_rn(w2[tap], vv[h], mab[j]);
          mc[j] = fmaf(w2[tap].x, cc[h], mc[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kRowOut; ++j) {
      hab[r][c0 + j] = mab[j];
      hc[r][c0 + j] = mc[j];
    }
  }
  __syncthreads();
  const float n = (float)total;
  const float k_mse = (1.f - a.lambda) * 2.f / n, k_ssim = a.lambda / n;
  {
    const int c = t % kST, r0 = kColOut * (t / kST);
    const int gx = x0 + c;
    float xv[kColOut], yv[kColOut];
#pragma unroll
    for (int j = 0; j < kColOut; ++j) {
      const int gy = y0 + r0 + j;
      const bool in = gx < a.W && gy < a.H;
      const int64_t o = pl * plane + (int64_t)gy * a.W + gx;
      xv[j] = in ? __ldg(a.x + o) : 0.f;
      yv[j] = in ? __ldg(a.y + o) : 0.f;
    }
    float2 mab[kColOut];
    float mc[kColOut];
#pragma unroll
    for (int j = 0; j < kColOut; ++j) {
      mab[j] = make_float2(0.f, 0.f);
      mc[j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kColOut + 2 * kSR; ++k) {
      const float2 v = hab[r0 + k][c];
      const float vcc = hc[r0 + k][c];
#pragma unroll
      for (int j = 0; j < kColOut; ++j) {
        const int tap = k - j;
        if (tap < 0 || tap >= kTaps) continue;
        mab[j] = __ffma2_rn(w2[tap], v, mab[j]);
        mc[j] = fmaf(w2[tap].x, vcc, mc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kColOut; ++j) {
      const int gy = y0 + r0 + j;
      if (gx >= a.W || gy >= a.H) continue;
      const int64_t o = pl * plane + (int64_t)gy * a.W + gx;
      a.grad[o] = k_mse * (xv[j] - yv[j]) - k_ssim * (mab[j].x + xv[j] * mab[j].y + yv[j] * mc[j]);
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && t == 0 && a.loss) {
    double ss = 0.0, se = 0.0;
    for (int k = 0; k < kSlots; ++k) {
      ss += a.sums[k];
      se += a.sums[kSlots + k];
    }
    const double nn = (double)total;
    *a.loss = (1.0 - (double)a.lambda) * se / nn + (double)a.lambda * (1.0 - ss / nn);
  }
}

}  // namespace rs

using namespace rs;

extern "C" size_t rs_ssim_workspace_size(int32_t width, int32_t height, int32_t n_planes) {
  if (width <= 0 || height <= 0 || n_planes <= 0) return 0;
  return 1024 + align_up((size_t)3 * n_planes * (size_t)width * height * 4, 256);
}

extern "C" rs_status rs_ssim_loss(const float* image, const float* target, int32_t width, int32_t height,
                                  int32_t n_planes, float lambda, float* dL_dimage, double* loss, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (!image || !target || !dL_dimage || width <= 0 || height <= 0 || n_planes <= 0) return RS_ERR_INVALID_ARG;
  if (!(lambda >= 0.f && lambda <= 1.f)) return RS_ERR_INVALID_ARG;
  if ((int64_t)height > 65535 * (int64_t)kST || n_planes > 65535) return RS_ERR_INVALID_ARG;
  const size_t need = rs_ssim_workspace_size(width, height, n_planes);
  if (!ws || ws_bytes < need || !aligned<double>(ws, 256)) return RS_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SsimArgs a{};
  a.x = image;
  a.y = target;
  a.sums = static_cast<double*>(ws);
  a.maps = reinterpret_cast<float*>(static_cast<char*>(ws) + 1024);
  a.grad = dL_dimage;
  a.loss = loss;
  a.W = width;
  a.H = height;
  a.planes = n_planes;
  a.lambda = lambda;
  double g[kTaps], tot = 0.0;
  for (int k = -kSR; k <= kSR; ++k) tot += (g[k + kSR] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5)));
  for (int k = 0; k < kTaps; ++k) a.w[k] = (float)(g[k] / tot);
  if (cudaMemsetAsync(ws, 0, 2 * kSlots * sizeof(double), s) != cudaSuccess) return RS_ERR_CUDA;
  const dim3 grid((unsigned)((width + kST - 1) / kST), (unsigned)((height + kST - 1) / kST), (unsigned)n_planes);
  {
    prof::Scope ps("k_ssim_stats", s);
    k_ssim_stats<<<grid, kSThreads, 0, s>>>(a);
  }
  prof::Scope ps("k_ssim_grad", s);
  k_ssim_grad<<<grid, kSThreads, 0, s>>>(a);
  return launch_status();
}
