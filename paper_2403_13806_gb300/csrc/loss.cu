// rs_l1_loss: mean absolute error and its gradient (one HBM-bound pass).
#include "profile.cuh"
#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {

__global__ void __launch_bounds__(256) k_l1(const float4* __restrict__ img, const float4* __restrict__ tgt, int64_t n4,
                                            const float* __restrict__ img1, const float* __restrict__ tgt1, int64_t n,
                                            float inv_n, float4* __restrict__ g4, float* __restrict__ g1,
                                            double* __restrict__ loss) {
  __shared__ double s[8];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 a = __ldcs(img + i), b = __ldcs(tgt + i);
    const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
    acc += (double)(fabsf(d0) + fabsf(d1)) + (double)(fabsf(d2) + fabsf(d3));
    float4 g;
    g.x = d0 > 0.f ? inv_n : (d0 < 0.f ? -inv_n : 0.f);
    g.y = d1 > 0.f ? inv_n : (d1 < 0.f ? -inv_n : 0.f);
    g.z = d2 > 0.f ? inv_n : (d2 < 0.f ? -inv_n : 0.f);
    g.w = d3 > 0.f ? inv_n : (d3 < 0.f ? -inv_n : 0.f);
    __stcs(g4 + i, g);
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float d = img1[i] - tgt1[i];
    acc += (double)fabsf(d);
    g1[i] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s[w];
    atomicAdd(loss, t * (double)inv_n);
  }
}

}  // namespace rs

using namespace rs;

extern "C" rs_status rs_l1_loss(const float* image, const float* target, int64_t n, float* dL_dimage, double* loss,
                                void* stream) {
  if (!image || !target || !dL_dimage || !loss || n < 0) return RS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return RS_ERR_CUDA;
  if (n == 0) return RS_OK;
  const bool vec = aligned<float4>(image, 16) && aligned<float4>(target, 16) && aligned<float4>(dL_dimage, 16);
  const int64_t n4 = vec ? n / 4 : 0;
  const int grid = 4 * kNumSMs;
  prof::Scope ps("k_l1", s);
  k_l1<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(image), reinterpret_cast<const float4*>(target), n4,
                            image, target, n, 1.0f / (float)n, reinterpret_cast<float4*>(dL_dimage), dL_dimage, loss);
  return launch_status();
}
