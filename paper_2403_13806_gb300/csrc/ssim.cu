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
// Two kernels, each on 32 x 16-pixel tiles of one plane with a 5-pixel halo in shared memory
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
constexpr int kSTX = 32, kSTY = 16;    // output tile
constexpr int kSHX = kSTX + 2 * kSR, kSHY = kSTY + 2 * kSR;
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
  float w[2 * kSR + 1];   // normalised 1D Gaussian, sigma 1.5
};

// Shared-memory layouts interleave what a tap reads together (x with y; the five moments
// as a float4 plus a float; the three maps as a float4), and every thread produces four
// adjacent outputs of the row pass and two of the column pass from values it loaded once,
// so the load/store unit (the bound of a naive stencil) carries ~5x fewer instructions.
__global__ void __launch_bounds__(256) k_ssim_stats(SsimArgs a) {
  __shared__ __align__(16) float2 sxy[kSHY][kSHX];     // (x, y) with the halo
  __shared__ __align__(16) float4 hq[kSHY][kSTX + 1];  // row-filtered (mu_x, mu_y, E[x^2], E[y^2])
  __shared__ float hxy[kSHY][kSTX + 1];                // row-filtered E[xy]
  __shared__ float red[2][8];
  const int x0 = blockIdx.x * kSTX, y0 = blockIdx.y * kSTY, pl = blockIdx.z;
  const int64_t plane = (int64_t)a.W * a.H;
  const float* X = a.x + pl * plane;
  const float* Y = a.y + pl * plane;
  {
    // every load of the halo tile is issued before the first shared-memory store
    constexpr int NL = (kSHX * kSHY + 255) / 256;
    float2 v[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int i = threadIdx.x + 256 * j;
      const int r = i / kSHX, c = i % kSHX;
      const int gy = y0 + r - kSR, gx = x0 + c - kSR;
      const bool in = i < kSHX * kSHY && gx >= 0 && gx < a.W && gy >= 0 && gy < a.H;
      const int64_t o = (int64_t)gy * a.W + gx;
      v[j] = in ? make_float2(__ldg(X + o), __ldg(Y + o)) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int i = threadIdx.x + 256 * j;
      if (i < kSHX * kSHY) sxy[i / kSHX][i % kSHX] = v[j];
    }
  }
  __syncthreads();
  // rows: 4 adjacent outputs per task, (kSHY rows) x (kSTX / 4 column groups) tasks
  {
    // 8 consecutive lanes take 8 rows of one column group: with the odd row pitches their
    // 16-byte loads and stores fall in 8 distinct bank groups
    const int t = threadIdx.x;
    const int r = (t & 7) + 8 * (t >> 6), c0 = 4 * ((t >> 3) & 7);
    if (r < kSHY) {
    float2 v[4 + 2 * kSR];
#pragma unroll
    for (int k = 0; k < 4 + 2 * kSR; k += 2) {
      const float4 q = *reinterpret_cast<const float4*>(&sxy[r][c0 + k]);
      v[k] = make_float2(q.x, q.y);
      v[k + 1] = make_float2(q.z, q.w);
    }
    // (mu_x, mu_y) and (E[x^2], E[y^2]) advance as packed pairs, E[xy] alone
    float2 m1[4], m2[4];
    float m3[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      m1[j] = m2[j] = make_float2(0.f, 0.f);
      m3[j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4 + 2 * kSR; ++k) {
      const float2 sq = __fmul2_rn(v[k], v[k]);
      const float xy = v[k].x * v[k].y;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int tap = k - j;
        if (tap < 0 || tap > 2 * kSR) continue;   // resolved at compile time
        const float2 w2 = make_float2(a.w[tap], a.w[tap]);
        m1[j] = __ffma2_rn(w2, v[k], m1[j]);
        m2[j] = __ffma2_rn(w2, sq, m2[j]);
        m3[j] = fmaf(a.w[tap], xy, m3[j]);
      }
    }
    float m[4][5];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      m[j][0] = m1[j].x;
      m[j][1] = m1[j].y;
      m[j][2] = m2[j].x;
      m[j][3] = m2[j].y;
      m[j][4] = m3[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      hq[r][c0 + j] = make_float4(m[j][0], m[j][1], m[j][2], m[j][3]);
      hxy[r][c0 + j] = m[j][4];
    }
    }
  }
  __syncthreads();
  // columns: 2 adjacent rows per task, kSTX x (kSTY / 2) tasks
  const int64_t total = plane * a.planes;
  float s_sum = 0.f, e_sum = 0.f;
  for (int t = threadIdx.x; t < kSTX * (kSTY / 2); t += blockDim.x) {
    const int c = t % kSTX, r0 = 2 * (t / kSTX);
    float2 m1[2], m2[2];
    float m3[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      m1[j] = m2[j] = make_float2(0.f, 0.f);
      m3[j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 2 + 2 * kSR; ++k) {
      const float4 hv = hq[r0 + k][c];
      const float hz = hxy[r0 + k][c];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int tap = k - j;
        if (tap < 0 || tap > 2 * kSR) continue;
        const float2 w2 = make_float2(a.w[tap], a.w[tap]);
        m1[j] = __ffma2_rn(w2, make_float2(hv.x, hv.y), m1[j]);
        m2[j] = __ffma2_rn(w2, make_float2(hv.z, hv.w), m2[j]);
        m3[j] = fmaf(a.w[tap], hz, m3[j]);
      }
    }
    float m[2][5];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      m[j][0] = m1[j].x;
      m[j][1] = m1[j].y;
      m[j][2] = m2[j].x;
      m[j][3] = m2[j].y;
      m[j][4] = m3[j];
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = r0 + j;
      const int gy = y0 + r, gx = x0 + c;
      if (gx >= a.W || gy >= a.H) continue;
      const float mx = m[j][0], my = m[j][1], exx = m[j][2], eyy = m[j][3], exy = m[j][4];
      const float sxx = exx - mx * mx, syy = eyy - my * my, sxy_ = exy - mx * my;
      const float ln = 2.f * mx * my + kC1, ld = mx * mx + my * my + kC1;
      const float cn = 2.f * sxy_ + kC2, cd = sxx + syy + kC2;
      // two reciprocals give all four: 1/ln = ld q1, 1/ld = ln q1, 1/cn = cd q2, 1/cd = cn q2
      const float q1 = __frcp_rn(ln * ld), q2 = __frcp_rn(cn * cd);
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
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][warp] = s_sum;
    red[1][warp] = e_sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, e = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s += red[0][w];
      e += red[1][w];
    }
    const int slot = (blockIdx.x + 7 * blockIdx.y + 13 * blockIdx.z) % kSlots;
    atomicAdd(&a.sums[slot], s);
    atomicAdd(&a.sums[kSlots + slot], e);
  }
}

__global__ void __launch_bounds__(256) k_ssim_grad(SsimArgs a) {
  __shared__ __align__(16) float4 sm[kSHY][kSHX + 1];   // (a, b, c, 0) with the halo (odd row pitch)
  __shared__ __align__(16) float4 hm[kSHY][kSTX + 1];   // row-filtered maps
  const int x0 = blockIdx.x * kSTX, y0 = blockIdx.y * kSTY, pl = blockIdx.z;
  const int64_t plane = (int64_t)a.W * a.H;
  const int64_t total = plane * a.planes;
  {
    constexpr int NL = (kSHX * kSHY + 255) / 256;
    float4 v[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int i = threadIdx.x + 256 * j;
      const int r = i / kSHX, c = i % kSHX;
      const int gy = y0 + r - kSR, gx = x0 + c - kSR;
      const bool in = i < kSHX * kSHY && gx >= 0 && gx < a.W && gy >= 0 && gy < a.H;
      const int64_t o = pl * plane + (int64_t)gy * a.W + gx;
      v[j] = in ? make_float4(__ldg(a.maps + o), __ldg(a.maps + total + o), __ldg(a.maps + 2 * total + o), 0.f)
                : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int i = threadIdx.x + 256 * j;
      if (i < kSHX * kSHY) sm[i / kSHX][i % kSHX] = v[j];
    }
  }
  __syncthreads();
  {
    const int t = threadIdx.x;
    const int r = (t & 7) + 8 * (t >> 6), c0 = 4 * ((t >> 3) & 7);
    if (r < kSHY) {
    float2 mab[4];
    float mc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      mab[j] = make_float2(0.f, 0.f);
      mc[j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4 + 2 * kSR; ++k) {
      const float4 v = sm[r][c0 + k];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int tap = k - j;
        if (tap < 0 || tap > 2 * kSR) continue;
        mab[j] = __ffma2_rn(make_float2(a.w[tap], a.w[tap]), make_float2(v.x, v.y), mab[j]);
        mc[j] = fmaf(a.w[tap], v.z, mc[j]);
      }
    }
    float m[4][3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      m[j][0] = mab[j].x;
      m[j][1] = mab[j].y;
      m[j][2] = mc[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) hm[r][c0 + j] = make_float4(m[j][0], m[j][1], m[j][2], 0.f);
    }
  }
  __syncthreads();
  const float n = (float)total;
  const float k_mse = (1.f - a.lambda) * 2.f / n, k_ssim = a.lambda / n;
  for (int t = threadIdx.x; t < kSTX * (kSTY / 2); t += blockDim.x) {
    const int c = t % kSTX, r0 = 2 * (t / kSTX);
    float xv[2], yv[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gy = y0 + r0 + j, gx = x0 + c;
      const bool in = gx < a.W && gy < a.H;
      const int64_t o = pl * plane + (int64_t)gy * a.W + gx;
      xv[j] = in ? __ldg(a.x + o) : 0.f;
      yv[j] = in ? __ldg(a.y + o) : 0.f;
    }
    float2 mab[2];
    float mc[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      mab[j] = make_float2(0.f, 0.f);
      mc[j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 2 + 2 * kSR; ++k) {
      const float4 v = hm[r0 + k][c];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int tap = k - j;
        if (tap < 0 || tap > 2 * kSR) continue;
        mab[j] = __ffma2_rn(make_float2(a.w[tap], a.w[tap]), make_float2(v.x, v.y), mab[j]);
        mc[j] = fmaf(a.w[tap], v.z, mc[j]);
      }
    }
    float m[2][3];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      m[j][0] = mab[j].x;
      m[j][1] = mab[j].y;
      m[j][2] = mc[j];
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gy = y0 + r0 + j, gx = x0 + c;
      if (gx >= a.W || gy >= a.H) continue;
      const int64_t o = pl * plane + (int64_t)gy * a.W + gx;
      a.grad[o] = k_mse * (xv[j] - yv[j]) - k_ssim * (m[j][0] + xv[j] * m[j][1] + yv[j] * m[j][2]);
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && a.loss) {
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
  if ((int64_t)height > 65535 * (int64_t)kSTY || n_planes > 65535) return RS_ERR_INVALID_ARG;
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
  double g[2 * kSR + 1], tot = 0.0;
  for (int k = -kSR; k <= kSR; ++k) tot += (g[k + kSR] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5)));
  for (int k = 0; k < 2 * kSR + 1; ++k) a.w[k] = (float)(g[k] / tot);
  if (cudaMemsetAsync(ws, 0, 2 * kSlots * sizeof(double), s) != cudaSuccess) return RS_ERR_CUDA;
  const dim3 grid((unsigned)((width + kSTX - 1) / kSTX), (unsigned)((height + kSTY - 1) / kSTY), (unsigned)n_planes);
  {
    prof::Scope ps("k_ssim_stats", s);
    k_ssim_stats<<<grid, 256, 0, s>>>(a);
  }
  prof::Scope ps("k_ssim_grad", s);
  k_ssim_grad<<<grid, 256, 0, s>>>(a);
  return launch_status();
}
