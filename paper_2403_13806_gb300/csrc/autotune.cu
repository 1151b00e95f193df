// rs_autotune: picks the tile shape, the records staged per shared-memory batch of the
// blend kernels and the number of views per launch for a set of views by timing the
// library's own pipeline on them, and caches the choice.
//
// Stage 1 crosses the tile shapes 16x16, 32x8 and 8x8 with 1, 2 and 4 staged records per
// thread, all of the first min(n_views, 16) views in one launch; stage 2 keeps the winner
// and tries 1, 2, 4, ... and n_views views per launch (the views taken in order in
// consecutive chunks) over the first min(n_views, max(views per launch, 16)) views; with
// RS_TUNE_FRONT stage 3 times that choice on whole lists as well and keeps the faster.  Each
// candidate runs project -> bin_sort (front lists with RS_TUNE_FRONT) -> render (image,
// T_final, last, importance) and, with RS_TUNE_BACKWARD, render_backward: one untimed pass (which also sizes the instance
// capacity), then three timed passes bracketed by CUDA events on the caller's stream.
// The score is milliseconds per view.  A candidate whose chunks would need 2^32 or more
// instances, or whose buffers cannot be allocated, is skipped.
//
// The cache maps the workload (view sizes, item counts, Gaussian count, SH degree,
// subset use, flags, configuration) to the choice; a host mutex guards it.  Tuning
// allocates and frees device memory with cudaMalloc / cudaFree and synchronises the
// stream, so it is a setup call, not part of a captured or timed step.
#include <cuda_runtime.h>
#include <string.h>

#include <map>
#include <mutex>
#include <vector>

#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {
namespace {

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  bool ensure(size_t bytes) {
    bytes = bytes < 256 ? 256 : bytes;
    if (bytes <= n) return true;
    release();
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    n = bytes;
    return true;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  ~DevBuf() { release(); }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

std::mutex g_mu;
std::map<std::vector<int64_t>, rs_tune_result> g_cache;

struct Chunk {
  rs_view_batch batch;
};

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" int32_t rs_autotune_candidates(int32_t n_views) {
  if (n_views <= 0) return 0;
  int32_t nb = 0;
  for (int32_t b = 1; b < n_views; b *= 2) ++nb;
  return 9 + nb + 1;
}

extern "C" void rs_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
}

extern "C" rs_status rs_autotune(const rs_gaussians* g, const rs_camera* cams, int32_t n_views,
                                 const int64_t* n_items, const uint32_t* subset_idx, const rs_config* cfg,
                                 int32_t flags, rs_tune_result* out, float* cand_ms, void* stream) {
  if (!g || !cams || !n_items || !cfg || !out || n_views <= 0 || g->n <= 0) return RS_ERR_INVALID_ARG;
  if (g->sh_degree < 0 || g->sh_degree > 3) return RS_ERR_UNSUPPORTED;
  if (flags & ~(RS_TUNE_BACKWARD | RS_TUNE_FORCE | RS_TUNE_FRONT)) return RS_ERR_INVALID_ARG;
  const bool bwd = (flags & RS_TUNE_BACKWARD) != 0;
  const bool front = (flags & RS_TUNE_FRONT) != 0;
  bool use_front = front;   // the binning the candidates run (stage 3 tries whole lists too)
  int32_t cfg_bits[5];
  memcpy(cfg_bits, cfg, sizeof(cfg_bits));   // eps2d, near_plane, bg (batch excluded)
  std::vector<int64_t> key = {n_views, g->n, g->sh_degree, bwd ? 1 : 0, subset_idx ? 1 : 0, front ? 1 : 0};
  for (int i = 0; i < 5; ++i) key.push_back(cfg_bits[i]);
  std::vector<int64_t> item_off(n_views + 1, 0);
  for (int32_t v = 0; v < n_views; ++v) {
    if (n_items[v] < 0 || (!subset_idx && n_items[v] != g->n)) return RS_ERR_INVALID_ARG;
    key.push_back(cams[v].width);
    key.push_back(cams[v].height);
    key.push_back(n_items[v]);
    item_off[v + 1] = item_off[v] + n_items[v];
  }
  if (!(flags & RS_TUNE_FORCE)) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *out = it->second;
      out->cached = 1;
      out->n_candidates = 0;
      return RS_OK;
    }
  }

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int32_t shapes[3][2] = {{16, 16}, {32, 8}, {8, 8}};
  const int32_t per_thread[3] = {1, 2, 4};
  std::vector<int32_t> batches;
  for (int32_t b = 1; b < n_views; b *= 2) batches.push_back(b);
  batches.push_back(n_views);
  const int32_t n_cand = 9 + (int32_t)batches.size();
  if (cand_ms)
    for (int32_t c = 0; c < n_cand; ++c) cand_ms[c] = -1.f;
  const int32_t B1 = n_views < 16 ? n_views : 16;   // views per launch in stage 1

  // buffers sized for the largest chunk (all views), grown on demand
  int64_t pixels_all = 0;
  for (int32_t v = 0; v < n_views; ++v) pixels_all += (int64_t)cams[v].width * cams[v].height;
  const int64_t items_all = item_off[n_views];
  const int nc = (g->sh_degree + 1) * (g->sh_degree + 1) * 3;
  DevBuf views_d, xy, co, rgbd, rect, ntile, img, T, last, dL, imp, grads, status, sort_ws, bwd_ws, vals, ranges;
  const int64_t mi = items_all > 0 ? items_all : 1;
  if (!views_d.ensure((size_t)n_views * sizeof(rs_view)) || !xy.ensure(mi * 8) || !co.ensure(mi * 16) ||
      !rgbd.ensure(mi * 16) || !rect.ensure(mi * 8) || !ntile.ensure(mi * 4) || !img.ensure(pixels_all * 12) ||
      !T.ensure(pixels_all * 4) || !last.ensure(pixels_all * 4) || !imp.ensure(g->n * 4) ||
      !status.ensure(sizeof(rs_device_status)) ||
      (bwd && (!dL.ensure(pixels_all * 12) || !grads.ensure((size_t)g->n * (11 + nc) * 4))))
    return RS_ERR_CUDA;
  if (bwd && cudaMemsetAsync(dL.p, 0, pixels_all * 12, s) != cudaSuccess) return RS_ERR_CUDA;
  rs_projected proj{xy.as<float>(), co.as<float>(), rgbd.as<float>(), rect.as<uint16_t>(), ntile.as<uint32_t>()};
  rs_gaussian_grads gr{};
  if (bwd) {
    float* base = grads.as<float>();
    gr.means = base;
    gr.log_scales = base + 3 * g->n;
    gr.quats = base + 6 * g->n;
    gr.opacity_logit = base + 10 * g->n;
    gr.sh = base + 11 * g->n;
  }
  rs_device_status* st = status.as<rs_device_status>();
  int64_t capacity = 0;
  std::vector<rs_view> host(n_views);

  rs_tune_result best{};
  best.ms_per_view = -1.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return RS_ERR_CUDA;
  }
  rs_status err = RS_OK;
  int32_t timed = 0;
  rs_config c_cfg = *cfg;
  // measures one candidate; returns RS_OK with ms < 0 when it does not fit
  auto measure = [&](int32_t tw, int32_t th, int32_t smem, int32_t B, float& per_view) -> rs_status {
    per_view = -1.f;
    c_cfg.batch = smem;
    const int32_t cover = n_views < (B > 16 ? B : 16) ? n_views : (B > 16 ? B : 16);
    std::vector<Chunk> chunks;
    for (int32_t s0 = 0; s0 < cover; s0 += B) {
      const int32_t nv = (n_views - s0) < B ? (n_views - s0) : B;
      Chunk c{};
      const rs_status r = rs_views_prepare(cams + s0, nv, n_items + s0, tw, th, host.data() + s0, &c.batch);
      if (r != RS_OK) return r;
      c.batch.views = views_d.as<rs_view>() + s0;
      c.batch.subset_idx = subset_idx ? subset_idx + item_off[s0] : nullptr;
      chunks.push_back(c);
    }
    const int32_t n_timed_views = (int32_t)((chunks.size() - 1) * (size_t)B) + chunks.back().batch.n_views;
    if (cudaMemcpyAsync(views_d.p, host.data(), (size_t)n_timed_views * sizeof(rs_view), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
      return RS_ERR_CUDA;
    bool alloc_failed = false;
    auto grow = [&](DevBuf& b, size_t bytes) {
      if (b.ensure(bytes)) return true;
      alloc_failed = true;
      return false;
    };
    // one pass over every chunk; with `sizing`, reads the device status afterwards and,
    // when an instance count exceeded the capacity, grows it and repeats
    auto run = [&](bool sizing) -> rs_status {
      for (;;) {
        if (capacity == 0) capacity = (int64_t)1 << 22;
        if (!grow(vals, (size_t)capacity * 4)) return RS_ERR_CUDA;
        if (cudaMemsetAsync(st, 0, sizeof(rs_device_status), s) != cudaSuccess) return RS_ERR_CUDA;
        for (const Chunk& c : chunks) {
          const size_t wsb = rs_workspace_size(RS_STAGE_BIN_SORT, &c.batch, capacity);
          if (!grow(sort_ws, wsb) || !grow(ranges, (size_t)(c.batch.n_tiles > 0 ? c.batch.n_tiles : 1) * 8))
            return RS_ERR_CUDA;
          const size_t bwb = bwd ? rs_workspace_size(RS_STAGE_BACKWARD, &c.batch, 0) : 0;
          if (bwd && !grow(bwd_ws, bwb)) return RS_ERR_CUDA;
          rs_bins bins{nullptr, vals.as<uint32_t>(), ranges.as<uint32_t>(), capacity};
          rs_status r = rs_project(g, &c.batch, &c_cfg, &proj, st, s);
          if (r == RS_OK)
            r = use_front ? rs_bin_sort_front(&proj, &c.batch, &bins, sort_ws.p, sort_ws.n, st, s)
                      : rs_bin_sort(&proj, &c.batch, &bins, sort_ws.p, sort_ws.n, st, s);
          if (r == RS_OK)
            r = rs_render(&proj, &bins, &c.batch, &c_cfg, img.as<float>(), T.as<float>(), last.as<int32_t>(),
                          imp.as<uint32_t>(), g->n, s);
          if (r == RS_OK && bwd)
            r = rs_render_backward(g, &c.batch, &c_cfg, &proj, &bins, T.as<float>(), last.as<int32_t>(),
                                   dL.as<float>(), &gr, bwd_ws.p, bwd_ws.n, s);
          if (r != RS_OK) return r;
        }
        if (!sizing) return RS_OK;
        rs_device_status h{};
        if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          return RS_ERR_CUDA;
        if (h.code == RS_OK) return RS_OK;
        if (h.code != RS_ERR_CAPACITY) return (rs_status)h.code;
        const int64_t need = h.required + h.required / 8 + 4096;
        if (need >= ((int64_t)1 << 32) - 1) return RS_ERR_CAPACITY;
        capacity = need;
      }
    };
    rs_status r = run(true);
    if (r == RS_ERR_CAPACITY || (r == RS_ERR_CUDA && alloc_failed)) {
      cudaGetLastError();
      return RS_OK;   // does not fit: not measured
    }
    if (r != RS_OK) return r;
    if (cudaEventRecord(e0, s) != cudaSuccess) return RS_ERR_CUDA;
    for (int rep = 0; rep < 3 && r == RS_OK; ++rep) r = run(false);
    if (r != RS_OK) return r;
    float ms = 0.f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return RS_ERR_CUDA;
    per_view = ms / (3.f * (float)n_timed_views);
    ++timed;
    return RS_OK;
  };
  // stage 1: tile shape x staging batch, B1 views per launch
  for (int si = 0; si < 3 && err == RS_OK; ++si) {
    for (int pi = 0; pi < 3 && err == RS_OK; ++pi) {
      const int32_t smem = per_thread[pi] * blend_threads(shapes[si][0], shapes[si][1]);
      float ms = -1.f;
      err = measure(shapes[si][0], shapes[si][1], smem, B1, ms);
      if (cand_ms) cand_ms[si * 3 + pi] = ms;
      if (err == RS_OK && ms >= 0.f && (best.ms_per_view < 0.f || ms < best.ms_per_view)) {
        best.tile_w = shapes[si][0];
        best.tile_h = shapes[si][1];
        best.smem_batch = smem;
        best.views_per_launch = B1;
        best.ms_per_view = ms;
      }
    }
  }
  // stage 2: views per launch with the stage-1 choice
  if (err == RS_OK && best.ms_per_view >= 0.f) {
    const rs_tune_result s1 = best;
    best.ms_per_view = -1.f;
    for (size_t bi = 0; bi < batches.size() && err == RS_OK; ++bi) {
      float ms = -1.f;
      err = measure(s1.tile_w, s1.tile_h, s1.smem_batch, batches[bi], ms);
      if (cand_ms) cand_ms[9 + bi] = ms;
      if (err == RS_OK && ms >= 0.f && (best.ms_per_view < 0.f || ms < best.ms_per_view)) {
        best.views_per_launch = batches[bi];
        best.ms_per_view = ms;
      }
    }
    if (best.ms_per_view < 0.f) best = s1;
  }
  // stage 3 (RS_TUNE_FRONT): the choice again on whole lists; the faster binning is kept
  best.front_lists = front ? 1 : 0;
  if (err == RS_OK && front && best.ms_per_view >= 0.f) {
    use_front = false;
    float ms = -1.f;
    err = measure(best.tile_w, best.tile_h, best.smem_batch, best.views_per_launch, ms);
    if (err == RS_OK && ms >= 0.f && ms < best.ms_per_view) {
      best.ms_per_view = ms;
      best.front_lists = 0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != RS_OK) return err;
  if (timed == 0) return RS_ERR_CAPACITY;
  best.cached = 0;
  best.n_candidates = timed;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = best;
  }
  *out = best;
  return RS_OK;
}
