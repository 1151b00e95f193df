// Host-side helpers of the C ABI: versions, status names, defaults, view descriptors and
// workspace sizes.  No device work here.
#include <math.h>
#include <string.h>

#include "radsplat.h"
#include "rs_common.cuh"

namespace rs {
size_t bin_sort_ws_bytes(const rs_view_batch* batch, int64_t capacity);
size_t filter_ws_bytes(int64_t n);
size_t backward_ws_bytes(const rs_view_batch* batch);
}  // namespace rs

using namespace rs;

extern "C" int32_t rs_abi_version(void) { return RS_ABI_VERSION; }

extern "C" const char* rs_status_str(rs_status s) {
  switch (s) {
    case RS_OK: return "ok";
    case RS_ERR_INVALID_ARG: return "invalid argument";
    case RS_ERR_WORKSPACE: return "workspace too small or misaligned";
    case RS_ERR_UNSUPPORTED: return "unsupported option";
    case RS_ERR_CUDA: return "CUDA error";
    case RS_ERR_CAPACITY: return "instance capacity exceeded";
    case RS_ERR_TIMEOUT: return "bounded wait timed out";
  }
  return "unknown status";
}

extern "C" rs_config rs_config_default(void) {
  rs_config c;
  memset(&c, 0, sizeof(c));
  c.eps2d = 0.3f;
  c.near_plane = 0.2f;
  return c;
}

extern "C" rs_status rs_views_prepare(const rs_camera* cams, int32_t n_views, const int64_t* n_items,
                                      int32_t tile_w, int32_t tile_h, rs_view* out_views, rs_view_batch* batch) {
  if (!cams || !n_items || !out_views || !batch || n_views <= 0) return RS_ERR_INVALID_ARG;
  if (!((tile_w == 16 && tile_h == 16) || (tile_w == 32 && tile_h == 8) || (tile_w == 8 && tile_h == 8)))
    return RS_ERR_UNSUPPORTED;
  int64_t tiles = 0, pixels = 0, items = 0;
  for (int32_t v = 0; v < n_views; ++v) {
    const rs_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || n_items[v] < 0) return RS_ERR_INVALID_ARG;
    if (!(c.fx > 0.f) || !(c.fy > 0.f)) return RS_ERR_INVALID_ARG;
    const int64_t tx = (c.width + tile_w - 1) / tile_w, ty = (c.height + tile_h - 1) / tile_h;
    if (tx > 65535 || ty > 65535) return RS_ERR_INVALID_ARG;
    rs_view& o = out_views[v];
    memset(&o, 0, sizeof(o));
    memcpy(o.viewmat, c.viewmat, sizeof(o.viewmat));
    o.fx = c.fx;
    o.fy = c.fy;
    o.cx = c.cx;
    o.cy = c.cy;
    for (int k = 0; k < 3; ++k) {
      double acc = 0.0;
      for (int r = 0; r < 3; ++r) acc += (double)c.viewmat[r * 4 + k] * (double)c.viewmat[r * 4 + 3];
      o.campos[k] = (float)(-acc);
    }
    o.lim_x = (float)(1.3 * (0.5 * c.width / (double)c.fx));
    o.lim_y = (float)(1.3 * (0.5 * c.height / (double)c.fy));
    o.width = c.width;
    o.height = c.height;
    o.tiles_x = (int32_t)tx;
    o.tiles_y = (int32_t)ty;
    o.tile_base = (int32_t)tiles;
    o.pixel_base = pixels;
    o.item_base = items;
    o.n_items = n_items[v];
    tiles += tx * ty;
    pixels += (int64_t)c.width * c.height;
    items += n_items[v];
    if (tiles >= ((int64_t)1 << 31)) return RS_ERR_INVALID_ARG;
  }
  batch->n_views = n_views;
  batch->n_tiles = (int32_t)tiles;
  batch->n_items = items;
  batch->n_pixels = pixels;
  batch->tile_w = tile_w;
  batch->tile_h = tile_h;
  return RS_OK;
}

extern "C" size_t rs_workspace_size(rs_stage stage, const rs_view_batch* batch, int64_t capacity) {
  if (!batch) return 0;
  switch (stage) {
    case RS_STAGE_PROJECT: return 0;
    case RS_STAGE_BIN_SORT: return bin_sort_ws_bytes(batch, capacity);
    case RS_STAGE_RENDER: return 0;
    case RS_STAGE_BACKWARD: return backward_ws_bytes(batch);
    case RS_STAGE_FILTER: return filter_ws_bytes(batch->n_items);
  }
  return 0;
}

extern "C" int32_t rs_struct_sizes(int64_t* out, int32_t n) {
  const int64_t s[] = {(int64_t)sizeof(rs_gaussians),  (int64_t)sizeof(rs_camera),         (int64_t)sizeof(rs_view),
                       (int64_t)sizeof(rs_view_batch), (int64_t)sizeof(rs_config),         (int64_t)sizeof(rs_projected),
                       (int64_t)sizeof(rs_bins),       (int64_t)sizeof(rs_gaussian_grads), (int64_t)sizeof(rs_device_status),
                       (int64_t)sizeof(rs_tune_result), (int64_t)sizeof(rs_adam_group),
                       (int64_t)sizeof(rs_gather_desc), (int64_t)sizeof(rs_image_grads)};
  const int32_t k = (int32_t)(sizeof(s) / sizeof(s[0]));
  int32_t w = 0;
  for (; w < k && w < n; ++w) out[w] = s[w];
  return w;
}
