// rs_kmeans: Lloyd's k-means on camera positions, the clustering step of Sec. 3.4
// ("we run k-means clustering on the input camera locations ... and assign the input
// cameras to the respective cluster centers").
//
// One CTA of 1024 threads runs every iteration (camera sets are small: thousands of points
// and k = 64 in the paper): the centres live in shared memory; the assignment step gives
// each thread a strided share of the points and applies the nearest-centre rule of
// rs_filter_nearest (FP32 ((d0^2 + d1^2) + d2^2) with every operation rounded, ties to the
// lower index); the update step gives each warp whole clusters: its lanes sum their members
// in FP64, a shuffle tree adds the lanes, and the centre becomes the FP32 rounding of
// sum / count (a cluster without members keeps its centre).  A last assignment with the
// final centres is written out.
#include "profile.cuh"
#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {

constexpr int kKmeansThreads = 1024;
constexpr int kKmeansMaxK = 256;

__device__ __forceinline__ int nearest_centre(const float* c, int k, float x0, float x1, float x2) {
  int best = 0;
  float bd = 0.f;
  for (int j = 0; j < k; ++j) {
    const float d0 = __fsub_rn(x0, c[3 * j]);
    const float d1 = __fsub_rn(x1, c[3 * j + 1]);
    const float d2 = __fsub_rn(x2, c[3 * j + 2]);
    const float d = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
    if (j == 0 || d < bd) {
      best = j;
      bd = d;
    }
  }
  return best;
}

__global__ void __launch_bounds__(kKmeansThreads) k_kmeans(const float* __restrict__ pts, int n,
                                                           float* __restrict__ centres, int k, int iterations,
                                                           int32_t* __restrict__ assign) {
  __shared__ float s_c[3 * kKmeansMaxK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kKmeansThreads / 32;
  for (int i = threadIdx.x; i < 3 * k; i += blockDim.x) s_c[i] = centres[i];
  __syncthreads();
  for (int it = 0; it <= iterations; ++it) {
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      assign[i] = nearest_centre(s_c, k, pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    if (it == iterations) break;   // the final assignment
    __syncthreads();
    // update: warp w owns clusters w, w + 32, ...
    for (int j = warp; j < k; j += NW) {
      double sx = 0.0, sy = 0.0, sz = 0.0;
      int cnt = 0;
      for (int i = lane; i < n; i += 32) {
        if (assign[i] == j) {
          sx += (double)pts[3 * i];
          sy += (double)pts[3 * i + 1];
          sz += (double)pts[3 * i + 2];
          ++cnt;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      }
      if (lane == 0 && cnt > 0) {
        s_c[3 * j] = (float)(sx / (double)cnt);
        s_c[3 * j + 1] = (float)(sy / (double)cnt);
        s_c[3 * j + 2] = (float)(sz / (double)cnt);
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * k; i += blockDim.x) centres[i] = s_c[i];
}

}  // namespace rs

using namespace rs;

extern "C" rs_status rs_kmeans(const float* points, int32_t n, float* centres, int32_t k, int32_t iterations,
                               int32_t* assign, void* stream) {
  if (!points || !centres || !assign || n <= 0 || k <= 0 || k > kKmeansMaxK || iterations < 0)
    return RS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  prof::Scope ps("k_kmeans", s);
  k_kmeans<<<1, kKmeansThreads, 0, s>>>(points, n, centres, k, iterations, assign);
  return launch_status();
}
