/*
 * radsplat.h -- C ABI of the GB300 (sm_103a) tile-based Gaussian-splatting hot path
 * of RadSplat (arXiv 2403.13806).
 *
 * The library renders a set of 3D Gaussians (Sec. 3.2 "Gaussian Splatting") into one
 * or many views, scores every Gaussian by its largest ray contribution alpha*T
 * (Eq. importance-score, Sec. 3.3), turns those scores into pruning / visibility
 * masks (Sec. 3.3 "Pruning", Eq. importance-score-vis), picks the nearest camera
 * cluster for a test view (Sec. 3.4 "Visibility List-Based Rendering"), and
 * differentiates the rendered images for optimisation (Sec. 3.2 "Radiance
 * Field-based Supervision").
 *
 * Conventions shared by every entry point
 *   - Ownership: the caller owns every buffer.  Device pointers point to device
 *     memory (e.g. PyTorch tensors); host pointers are marked HOST.  No entry point
 *     allocates device memory; temporary storage is the caller's workspace, sized by
 *     rs_workspace_size().  Inputs are const and never written.  Outputs are written
 *     and not read, except the accumulators named below (importance, gradients),
 *     which the caller zeroes once and which calls then accumulate into.
 *   - Streams: every call enqueues work on `stream` and returns without waiting for
 *     the device (no host synchronisation), so a whole pipeline can be captured in a
 *     CUDA graph.  `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream.
 *   - Errors: the return value reports argument, workspace and launch errors at call
 *     time.  Conditions only the device can see (instance capacity overflow, a
 *     bounded wait that gave up, culled non-finite inputs) are written to the
 *     caller's rs_device_status block, which the caller reads after synchronising.
 *     Kernels never trap: on overflow they clamp their writes and record the status.
 *   - Layouts: parameters are FP32 structure-of-arrays; images are planar
 *     [3][H][W] FP32 per view; world-to-camera matrices are row-major 3x4 with
 *     OpenCV axes (x right, y down, z forward); pixel (u, v) samples image point (u, v).
 *   - Alignment: every float4-typed array (documented as [n][4]) must be 16-byte
 *     aligned, every [n][2] float array 8-byte aligned; PyTorch allocations satisfy this.
 */
#ifndef RADSPLAT_H
#define RADSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RS_ABI_VERSION 1

typedef enum rs_status {
  RS_OK = 0,
  RS_ERR_INVALID_ARG = 1,  /* a pointer, size or option is out of range */
  RS_ERR_WORKSPACE = 2,    /* ws_bytes below rs_workspace_size() */
  RS_ERR_UNSUPPORTED = 3,  /* e.g. sh_degree > 3, tile shape not in the supported set */
  RS_ERR_CUDA = 4,         /* a CUDA launch or runtime call failed */
  RS_ERR_CAPACITY = 5,     /* device-reported: more (tile, Gaussian) instances than capacity */
  RS_ERR_TIMEOUT = 6       /* device-reported: a bounded wait gave up */
} rs_status;

/* Device-side status block (device memory, caller-owned, zeroed by the caller before
 * the first call of a sequence).  Fields only ever grow; `code` keeps the first error. */
typedef struct rs_device_status {
  int32_t code;          /* RS_OK, RS_ERR_CAPACITY, RS_ERR_TIMEOUT, or RS_ERR_INVALID_ARG
                            (rs_bin_sort: the batch's n_tiles is below its views' tile count;
                            the tile lists are then left empty) */
  int32_t nonfinite;     /* projected items culled for non-finite parameters */
  int64_t required;      /* largest instance count any rs_bin_sort needed */
  int64_t n_instances;   /* instances the last rs_bin_sort produced (<= capacity) */
  int64_t reserved;
} rs_device_status;

/* Gaussian parameters, Sec. 3.2: position p, scale s (stored as log s), rotation q
 * (w, x, y, z; normalised inside the library), opacity o (stored as the logit of o),
 * SH coefficients k of degree sh_degree <= 3.  All device, FP32, SoA:
 *   means[3][n], log_scales[3][n], quats[4][n], opacity_logit[n],
 *   sh[(sh_degree+1)^2 * 3][n]  with row = coefficient * 3 + channel. */
typedef struct rs_gaussians {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logit;
  const float* sh;
  int64_t n;
  int32_t sh_degree;
  int32_t reserved;
} rs_gaussians;

/* Pinhole camera (HOST struct): world-to-camera [R|t] (row-major 3x4) and intrinsics. */
typedef struct rs_camera {
  float viewmat[12];
  float fx, fy, cx, cy;
  int32_t width, height;
} rs_camera;

/* Per-view descriptor as the kernels read it (128 bytes).  rs_views_prepare() fills
 * an array of these on the host; the caller copies it to device memory and passes
 * that copy in rs_view_batch.views. */
typedef struct rs_view {
  float viewmat[12];     /* world -> camera */
  float fx, fy, cx, cy;
  float campos[3];       /* camera centre -R^T t in world space */
  float lim_x, lim_y;    /* 1.3 * (W/2)/fx, 1.3 * (H/2)/fy: clamp of x/z, y/z inside J */
  int32_t width, height;
  int32_t tiles_x, tiles_y;
  int32_t tile_base;     /* first global tile id of the view */
  int64_t pixel_base;    /* first pixel of the view in the T_final / last buffers */
  int64_t item_base;     /* first projected item of the view */
  int64_t n_items;       /* projected items of the view */
} rs_view;

/* A batch of views rendered together.  Items are (view, Gaussian) pairs: view v owns
 * items [item_base, item_base + n_items).  If subset_idx is NULL, item i of view v is
 * Gaussian (i - item_base) and n_items equals the number of Gaussians; otherwise it is
 * Gaussian subset_idx[i] (a visibility list, Sec. 3.4; ascending within each view). */
typedef struct rs_view_batch {
  const rs_view* views;        /* DEVICE [n_views] */
  const uint32_t* subset_idx;  /* DEVICE [n_items] or NULL */
  int32_t n_views;
  int32_t n_tiles;             /* total tiles over all views */
  int64_t n_items;             /* total items */
  int64_t n_pixels;            /* total pixels (sum of W*H) */
  int32_t tile_w, tile_h;      /* tile shape: 16x16, 32x8 or 8x8 */
} rs_view_batch;

/* Rasterizer options.  rs_config_default() gives the readings the library uses for
 * what the paper leaves to the 3DGS renderer it cites (Sec. 3.2, Sec. 3.4). */
typedef struct rs_config {
  float eps2d;           /* dilation added to the diagonal of Sigma' (px^2), default 0.3 */
  float near_plane;      /* cull if the FP32 camera depth <= near_plane, default 0.2 */
  float bg[3];           /* background colour composited with T_final, default 0 */
  int32_t batch;         /* Gaussian records staged in shared memory per batch of the blend
                            kernels: 0 (default: 64) or 32, 64 or 128 (1, 2 or 4 per thread);
                            both blend kernels run one warp per tile (eight pixels of a column
                            per thread, two for 8x8 tiles); other values give
                            RS_ERR_UNSUPPORTED */
  int32_t grad_overwrite;  /* rs_render_backward: 0 (default) adds the call's parameter
                            gradients into the caller's arrays (which the caller zeroes);
                            1 writes them over the arrays (zero where the call gives none),
                            so no zeroing is needed */
  int32_t reserved[1];
} rs_config;

/* Projected items (all device, [n_items] rows):
 *   xy[n][2]       image-space mean
 *   conic_o[n][4]  (a, b, c, o): inverse of Sigma' = [[a, b], [b, c]] and the opacity
 *   rgb_d[n][4]    (r, g, b, depth): SH colour and the FP32 front-to-back order key
 *   rect[n][4]     uint16 tiles (x0, y0, x1, y1), half-open, covering every pixel whose
 *                  alpha can reach 1/255; all zero for a culled item
 *   n_tiles[n]     (x1-x0)*(y1-y0), 0 for a culled item */
typedef struct rs_projected {
  float* xy;
  float* conic_o;
  float* rgb_d;
  uint16_t* rect;
  uint32_t* n_tiles;
} rs_projected;

/* Tile lists.  After rs_bin_sort, vals[ranges[2t] .. ranges[2t+1]) are the items that
 * touch global tile t, front to back (by the FP32 depth key, ties to the lower item); an
 * empty tile has ranges[2t] == ranges[2t+1] (the place its list would start).
 * keys (optional, may be NULL) receive the 64-bit sort keys (tile << 32 | depth bits)
 * in the same order.  The instance count is written to the device status block. */
typedef struct rs_bins {
  uint64_t* keys;        /* DEVICE [capacity] or NULL */
  uint32_t* vals;        /* DEVICE [capacity] */
  uint32_t* ranges;      /* DEVICE [n_tiles][2] */
  int64_t capacity;      /* rows of keys/vals, < 2^32 */
} rs_bins;

/* Gradient accumulators (device, FP32, same layouts as rs_gaussians; accumulated). */
typedef struct rs_gaussian_grads {
  float* means;
  float* log_scales;
  float* quats;
  float* opacity_logit;
  float* sh;
} rs_gaussian_grads;

typedef enum rs_filter_mode {
  RS_PRUNE_BELOW = 0,    /* mask = h < t: points the pruning step removes (Sec. 3.3) */
  RS_KEEP_ABOVE = 1,     /* mask = h > t: points active for a cluster (Eq. importance-score-vis) */
  RS_PRUNE_KEEP = 2      /* mask = h >= t: the points pruning keeps (1 - RS_PRUNE_BELOW), whose
                            ascending list drives rs_gather_columns (Sec. 3.3) */
} rs_filter_mode;

typedef enum rs_stage {
  RS_STAGE_PROJECT = 0,
  RS_STAGE_BIN_SORT = 1,
  RS_STAGE_RENDER = 2,
  RS_STAGE_BACKWARD = 3,
  RS_STAGE_FILTER = 4
} rs_stage;

/* ---- host helpers (no device work) ---------------------------------------------- */

/* Library ABI version (RS_ABI_VERSION). */
int32_t rs_abi_version(void);

/* Human-readable name of a status code (static string). */
const char* rs_status_str(rs_status s);

/* Default options: eps2d 0.3, near 0.2, bg 0, batch 0 (auto). */
rs_config rs_config_default(void);

/* Fill n_views descriptors (HOST out_views[n_views]) from HOST cameras and per-view item
 * counts (HOST n_items[n_views]), and the sizes of `batch` (views and subset_idx are left
 * for the caller to set).  Tile shape must be 16x16, 32x8 or 8x8.
 * Errors: RS_ERR_INVALID_ARG (null pointer, empty or oversized view, total tiles >= 2^31),
 * RS_ERR_UNSUPPORTED (tile shape). */
rs_status rs_views_prepare(const rs_camera* cams, int32_t n_views, const int64_t* n_items,
                           int32_t tile_w, int32_t tile_h, rs_view* out_views,
                           rs_view_batch* batch);

/* Workspace bytes a stage needs for this batch (capacity = instance rows of rs_bins). */
size_t rs_workspace_size(rs_stage stage, const rs_view_batch* batch, int64_t capacity);

/* Sizes of the ABI structs, for bindings that mirror them: writes up to n entries in the
 * order rs_gaussians, rs_camera, rs_view, rs_view_batch, rs_config, rs_projected, rs_bins,
 * rs_gaussian_grads, rs_device_status, rs_tune_result, rs_adam_group, rs_gather_desc,
 * rs_image_grads;
 * returns how many it wrote. */
int32_t rs_struct_sizes(int64_t* out, int32_t n);

/* ---- hot path ---------------------------------------------------------------------- */

/* rs_project -- Sec. 3.2 "Gaussian Splatting": for every item (view v, Gaussian i),
 * Sigma = R S S^T R^T, Sigma' = J M Sigma M^T J^T + eps2d*I (M the view rotation, J the
 * Jacobian of the perspective projection at the camera-space mean, x/z and y/z clamped
 * to lim_x/lim_y inside J), the conic (Sigma')^-1, the image mean, o = sigmoid(logit),
 * the colour max(0, 0.5 + sum k_lm Y_lm(d)) from degree-sh_degree SH along
 * d = normalise(p - campos), the FP32 order key
 *   depth = fmaf(M20, px, fmaf(M21, py, fmaf(M22, pz, t2))),
 * and the tile rectangle of the bounding box of {alpha >= 1/255}.  Items whose depth
 * <= near_plane, whose parameters are not finite (counted in status->nonfinite), whose
 * quaternion is zero, whose opacity is below 1/255 or whose support misses the image
 * get n_tiles = 0.
 * ws: unused (pass NULL, 0).  Errors: RS_ERR_INVALID_ARG, RS_ERR_UNSUPPORTED
 * (sh_degree), RS_ERR_CUDA. */
rs_status rs_project(const rs_gaussians* g, const rs_view_batch* batch, const rs_config* cfg,
                     const rs_projected* out, rs_device_status* status, void* stream);

/* rs_bin_sort -- tile binning with duplicated 64-bit (tile | depth) keys and a device
 * radix sort (the front-to-back order Eq. render-gs needs, per tile).  Every item is
 * duplicated once per tile of its rect; the instances come out sorted by
 * key = (global tile id) << 32 | float bits of depth, stably with respect to item order.
 * The sort runs in levels that give exactly that order: the items by depth (radix), their
 * instances per 4 x 4-tile super-tile by super-tile id (stable radix), then each
 * super-tile list partitioned in order into its tile lists.  Writes vals, ranges, and
 * keys if non-NULL.  Reads proj->rgb_d (depth in .w), proj->rect and proj->n_tiles as
 * rs_project writes them; rects given by other means must lie inside their view's tile
 * grid.
 * If the instance count K exceeds bins->capacity, status->code = RS_ERR_CAPACITY,
 * status->required = K, and only the first capacity instances are written (the lists
 * are then incomplete; re-run with capacity >= required).
 * ws: rs_workspace_size(RS_STAGE_BIN_SORT, batch, capacity) bytes of device memory.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_WORKSPACE, RS_ERR_CUDA. */
rs_status rs_bin_sort(const rs_projected* proj, const rs_view_batch* batch,
                      const rs_bins* bins, void* ws, size_t ws_bytes,
                      rs_device_status* status, void* stream);

/* rs_bin_sort_front -- rs_bin_sort restricted to the front of every tile list that the
 * blend of Eq. render-gs can reach (the paper has no counterpart; rs_render,
 * rs_importance and rs_render_backward give the same results on either lists).
 * Blending stops a pixel before the first entry whose T(1 - alpha) falls below 1e-4.  For
 * every tile, the items among the nearest ceil(n / 32) in depth order whose alpha is at
 * least some alpha_lb >= 0.05 at every pixel centre of the tile (the smallest over the
 * tile's four corner pixels, the power being concave; with margins for FP32 rounding)
 * bound T from above by the product of their (1 - alpha_lb); the depth rank by which that
 * product provably falls below 5e-5 (rounded up to the end of one of 16 rank buckets,
 * narrower at the front) is the tile's cut, and every super-tile of 4 x 4 tiles takes its
 * tiles' largest cut (a tile without one keeps its whole list, and so does its
 * super-tile).  vals[ranges[2t] .. ranges[2t+1]) is then the first part of rs_bin_sort's
 * list for tile t: the items ranked before the cut, in the same order; every entry the
 * blend composites or tests lies in it.  keys, capacity and status as in rs_bin_sort (the
 * instance count is that of the shortened lists).
 * A batch with fewer than 32 items per tile on average (n_items < 32 n_tiles) gets whole
 * lists, as from rs_bin_sort: its lists are too short for the cut to pay for its passes.
 * Reads proj->xy and proj->conic_o besides what rs_bin_sort reads, and batch->tile_w /
 * tile_h (the pixel rectangle of every tile).
 * ws: rs_workspace_size(RS_STAGE_BIN_SORT, batch, capacity) bytes (the same workspace).
 * Errors: RS_ERR_INVALID_ARG (also for NULL xy or conic_o), RS_ERR_WORKSPACE, RS_ERR_CUDA. */
rs_status rs_bin_sort_front(const rs_projected* proj, const rs_view_batch* batch,
                            const rs_bins* bins, void* ws, size_t ws_bytes,
                            rs_device_status* status, void* stream);

/* rs_render -- Eq. (render-gs): per pixel, walk its tile's list front to back with
 * alpha = min(0.99, o exp(power)), power = -(a dx^2 + c dy^2)/2 - b dx dy; skip entries
 * with power > 0 or alpha < 1/255; stop before the first entry whose T(1-alpha) < 1e-4;
 * C = sum c_j alpha_j T_j + T_final * bg.
 * Outputs (device; any may be NULL to skip it): image [3 * n_pixels] planar per view
 * (view v's channel c starts at 3*pixel_base + c*H*W), T_final [n_pixels],
 * last [n_pixels] (1 + position in the tile list of the last composited entry, 0 if none).
 * importance (may be NULL): uint32 [n_gaussians] holding the float bits of
 * h_i = max alpha_i T_i over composited entries (Eq. importance-score), max-accumulated
 * across calls; zero it before the first view.  n_gaussians is the length of importance
 * (the Gaussian ids are item - item_base, or subset_idx[item]).
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_CUDA. */
rs_status rs_render(const rs_projected* proj, const rs_bins* bins, const rs_view_batch* batch,
                    const rs_config* cfg, float* image, float* T_final, int32_t* last,
                    uint32_t* importance, int64_t n_gaussians, void* stream);

/* rs_importance -- Eq. (importance-score) over every view of the batch: rs_render with
 * no image outputs; importance (required) as in rs_render. */
rs_status rs_importance(const rs_projected* proj, const rs_bins* bins,
                        const rs_view_batch* batch, const rs_config* cfg,
                        uint32_t* importance, int64_t n_gaussians, void* stream);

/* rs_filter -- Sec. 3.3 pruning mask m_i = 1(h_i < t) (RS_PRUNE_BELOW) or the
 * visibility indicator 1(h_i > t) of Eq. (importance-score-vis) (RS_KEEP_ABOVE) for
 * h (device float [n]); mask (device uint8 [n], may be NULL), idx (device uint32 [n],
 * may be NULL: the indices with mask 1 in ascending order), count (device uint32 [1]).
 * ws: rs_workspace_size(RS_STAGE_FILTER, ...) with batch->n_items = n.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_WORKSPACE, RS_ERR_CUDA. */
rs_status rs_filter(const float* h, int64_t n, float t, rs_filter_mode mode, uint8_t* mask,
                    uint32_t* idx, uint32_t* count, void* ws, size_t ws_bytes, void* stream);

/* rs_filter_noalloc -- rs_filter for callers that cannot allocate device memory at all
 * (the paper has no counterpart).  Some hosts own every byte of device memory and forbid
 * allocation after start-up -- real-time renderers with a fixed budget, engine plug-ins,
 * embedded runtimes -- so they can neither call cudaMalloc nor hand this library a
 * workspace.  This entry point computes exactly what rs_filter computes, but keeps the
 * compaction's scratch (one 32-bit count per 4096 elements) in a fixed array inside the
 * library, RS_FILTER_NOALLOC_MAX_N / 4096 words (64 KB) that every GPU loading the library
 * holds until the process exits.  Nothing is allocated: no cudaMalloc, no cudaFree, no
 * allocating library call.  The caller still passes h, mask, idx and count.
 * Every call looks up that array's device address on the current device (a lookup that
 * allocates nothing and stays valid across a device reset); the first call on a device may
 * load the library's device code there, so make it before capturing a stream into a CUDA
 * graph.  Every call shares the one array, and each call overwrites all of the scratch it
 * reads before reading it (the per-block counts), so nothing from an earlier call leaks
 * into a later one; but calls that overlap on the GPU (other streams, other threads) race
 * on it, so serialise them.  n > RS_FILTER_NOALLOC_MAX_N returns RS_ERR_INVALID_ARG without
 * launching anything.  Other arguments and errors as rs_filter. */
#define RS_FILTER_NOALLOC_MAX_N (1LL << 26)
rs_status rs_filter_noalloc(const float* h, int64_t n, float t, rs_filter_mode mode, uint8_t* mask,
                            uint32_t* idx, uint32_t* count, void* stream);

/* rs_filter_nearest -- Sec. 3.4: for each of n_cams camera centres (device float [n][3]),
 * the nearest of k cluster centres (device float [k][3]) by the FP32 squared distance
 * ((x0-c0)^2 + (x1-c1)^2) + (x2-c2)^2, ties to the lower index; out device int32 [n].
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_CUDA. */
rs_status rs_filter_nearest(const float* centres, int32_t k, const float* cam_centres,
                            int32_t n_cams, int32_t* out, void* stream);

/* rs_nn_distance -- Sec. 3.2 "Radiance Field-based Initialization": the isotropic initial
 * scale s_i = min over the other points p of |p_i - p|_2, for every point of means (device
 * float [3][n], the rs_gaussians layout); dist (device float [n]) receives it (0 for a
 * duplicated point, +inf for a point with a non-finite coordinate).  Exact nearest
 * neighbour over an implicit octree (points sorted by 30-bit Morton code); FP32 distances.
 * ws: rs_nn_workspace_size(n) bytes of device memory, 256-byte aligned.  No host
 * synchronisation.  Errors: RS_ERR_INVALID_ARG (n < 2 or n >= 2^31, null pointers),
 * RS_ERR_WORKSPACE, RS_ERR_CUDA. */
rs_status rs_nn_distance(const float* means, int64_t n, float* dist, void* ws, size_t ws_bytes, void* stream);
size_t rs_nn_workspace_size(int64_t n);

/* rs_kmeans -- Sec. 3.4 "Input Camera Clustering": Lloyd's k-means on the n camera
 * locations (device float [n][3]) with k <= 256 initial centres (device float [k][3], the
 * caller's choice; overwritten with the result) for `iterations` steps of: assign every
 * point to its nearest centre (the rule of rs_filter_nearest), then move every centre that
 * has points to their mean (summed in FP64, rounded to FP32); a centre without points stays.
 * assign (device int32 [n]) receives the assignment to the final centres.  One CTA runs
 * every iteration (meant for camera sets, up to some 1e5 points).
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_CUDA. */
rs_status rs_kmeans(const float* points, int32_t n, float* centres, int32_t k, int32_t iterations,
                    int32_t* assign, void* stream);

/* rs_render_backward -- derivative of Eq. (render-gs) for the training loss of Sec. 3.2:
 * given dL/dimage (device, layout of rs_render's image) and the forward's T_final and
 * last, walks each pixel's list back to front from `last` (T_j recovered as
 * T_{j+1}/(1-alpha_j)), then chains through the projection to the parameters.
 * Gradients are ADDED into `grads` (zero them first), or with cfg->grad_overwrite written
 * over them (every row; for a visibility-list batch the call zeroes `grads` itself, then
 * adds); items of all views of the same Gaussian are summed.
 * ws: rs_workspace_size(RS_STAGE_BACKWARD, batch, 0) bytes.  It carries state from one call
 * to the next: a completed call marks it clean (the items it left no gradient for hold
 * zeros) and flags the items it did, so the next call with the same item count zeroes only
 * those; any other contents are zeroed whole.  Calls that share a workspace must not
 * overlap on the GPU.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_WORKSPACE, RS_ERR_UNSUPPORTED, RS_ERR_CUDA. */
rs_status rs_render_backward(const rs_gaussians* g, const rs_view_batch* batch,
                             const rs_config* cfg, const rs_projected* proj,
                             const rs_bins* bins, const float* T_final, const int32_t* last,
                             const float* dL_dimage, const rs_gaussian_grads* grads,
                             void* ws, size_t ws_bytes, void* stream);

/* Image-space gradients of every projected item (SURVEY A8's output, the derivative of
 * Eq. render-gs with respect to what rs_project produces), as rs_render_backward leaves
 * them in its workspace (device, FP32, [n_items] rows, summed over every pixel of the
 * item's view):
 *   g_xy_ab[n][4]   dL/dx, dL/dy of the image mean; dL/da, dL/db of the conic (a, b, c)
 *                   with power = -(a dx^2 + c dy^2)/2 - b dx dy
 *   g_c_o_rg[n][4]  dL/dc of the conic; dL/do of the opacity; dL/dr, dL/dg of the colour
 *   g_b[n]          dL/d(blue) of the colour
 * The colour gradient is taken at the clamped colour max(0, .) (zero where the clamp of
 * rs_project is active only after the chain to the SH); no gradient flows through alpha
 * where the 0.99 clamp is active. */
typedef struct rs_image_grads {
  const float* g_xy_ab;
  const float* g_c_o_rg;
  const float* g_b;
} rs_image_grads;

/* rs_backward_image_grads -- host helper (no device work): pointers into a backward
 * workspace `ws` of ws_bytes for `batch` (the ws a completed rs_render_backward of that
 * batch used) where the per-item image-space gradients above live.  They stay valid until
 * the workspace is reused.  Errors: RS_ERR_INVALID_ARG, RS_ERR_WORKSPACE (ws_bytes below
 * rs_workspace_size(RS_STAGE_BACKWARD, batch, 0)). */
rs_status rs_backward_image_grads(const rs_view_batch* batch, void* ws, size_t ws_bytes,
                                  rs_image_grads* out);

/* rs_l1_loss -- the L1 photometric loss used for the synthetic training step (a stand-in
 * for the radiance-field supervision of Sec. 3.2, whose teacher renders are not
 * available): loss = mean |image - target| over n values, and
 * dL_dimage = sign(image - target) / n (0 where they are equal).  image, target,
 * dL_dimage: device float [n]; loss: device double [1], overwritten.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_CUDA. */
rs_status rs_l1_loss(const float* image, const float* target, int64_t n, float* dL_dimage,
                     double* loss, void* stream);

/* rs_ssim_loss -- the training loss of Sec. 3.2,
 *   L = (1 - lambda) mean((x - y)^2) + lambda (1 - mean SSIM(x, y)),  lambda = 0.2 in the paper,
 * reading its SSIM term as the structural dissimilarity 1 - SSIM.  SSIM (Wang et al. 2004)
 * per plane and pixel with a normalised 11 x 11 Gaussian window (sigma 1.5) over the
 * zero-padded planes, C1 = 0.01^2, C2 = 0.03^2; means over all n = n_planes*H*W values.
 * image (x, rendered), target (y): device float [n_planes][height][width] (the planar
 * channels of one or more same-sized views).  dL_dimage: device float, same layout,
 * overwritten with dL/dx.  loss: device double [1], overwritten (may be NULL).
 * ws: rs_ssim_workspace_size(width, height, n_planes) bytes of device memory, 256-byte
 * aligned.  Errors: RS_ERR_INVALID_ARG (sizes, lambda outside [0, 1], height above
 * 1048560, n_planes above 65535), RS_ERR_WORKSPACE, RS_ERR_CUDA. */
rs_status rs_ssim_loss(const float* image, const float* target, int32_t width, int32_t height,
                       int32_t n_planes, float lambda, float* dL_dimage, double* loss, void* ws,
                       size_t ws_bytes, void* stream);
size_t rs_ssim_workspace_size(int32_t width, int32_t height, int32_t n_planes);

/* ---- optimisation step (Sec. 3.2 optimiser, Sec. 3.3 pruning) ----------------------- */

/* One parameter array of an Adam step (all device pointers, FP32, n elements). */
typedef struct rs_adam_group {
  float* param;          /* updated in place */
  const float* grad;
  float* m;              /* first moment, updated in place (zero before step 1) */
  float* v;              /* second moment, updated in place (zero before step 1) */
  int64_t n;
  float lr;              /* learning rate of this array */
  int32_t reserved;
} rs_adam_group;

/* rs_adam_step -- one step of Adam (Kingma & Ba, Algorithm 1), the optimiser 3D Gaussian
 * Splatting optimises phi with (Sec. 3.2), on up to 8 arrays in one launch:
 *   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
 *   p <- p - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps),
 * in FP32 with correctly rounded division and square root.  groups: HOST array of
 * n_groups (1..8) descriptors; step >= 1 counts the steps taken including this one.
 * Arrays of a group must not overlap.  Errors: RS_ERR_INVALID_ARG (counts, step, betas in
 * [0, 1), eps >= 0, null pointers with n > 0), RS_ERR_CUDA. */
rs_status rs_adam_step(const rs_adam_group* groups, int32_t n_groups, float beta1, float beta2,
                       float eps, int32_t step, void* stream);

/* One structure-of-arrays array to compact: rows x src_stride source, rows x dst_stride
 * destination (device, FP32, non-overlapping). */
typedef struct rs_gather_desc {
  const float* src;
  float* dst;
  int64_t rows;
  int64_t src_stride;    /* columns of src (the point count before pruning) */
  int64_t dst_stride;    /* columns of dst, >= max_count */
} rs_gather_desc;

/* rs_gather_columns -- removes pruned points from every parameter array (Sec. 3.3, "we
 * remove all Gaussians ... that have a mask value of one"): dst[r][k] = src[r][idx[k]] for
 * k < min(*count, max_count) and every row r of each of the n_desc (1..16) arrays.  idx and
 * count (device) are rs_filter's outputs for RS_PRUNE_KEEP: the survivors in ascending
 * order, so the points keep their relative order.  descs: HOST array.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_CUDA. */
rs_status rs_gather_columns(const rs_gather_desc* descs, int32_t n_desc, const uint32_t* idx,
                            const uint32_t* count, int64_t max_count, void* stream);

/* ---- view-sharded training over several GPUs ---------------------------------------- */

/* rs_touched_columns -- for a gradient matrix src (device float [rows][n], e.g. every
 * parameter gradient of n Gaussians stacked row by row), out[i] (device float [n]) = 1 if
 * some row of column i is non-zero, else 0: the Gaussians this rank's views gave a gradient.
 * Ranks that share views (the training loss of Sec. 3.2 is a sum over images) exchange only
 * the union of these columns (max over ranks of out, then rs_filter RS_KEEP_ABOVE 0.5, then
 * rs_gather_columns, a sum over ranks, and rs_scatter_columns), not all n.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_CUDA. */
rs_status rs_touched_columns(const float* src, int64_t rows, int64_t n, float* out, void* stream);

/* rs_scatter_columns -- the inverse placement of rs_gather_columns: dst[r][idx[k]] =
 * src[r][k] for k < min(*count, max_count) and every row r of each of the n_desc (1..16)
 * descriptors, here read as src = the packed rows x src_stride array (src_stride >=
 * max_count) and dst = the rows x dst_stride array it came from; columns not listed in idx
 * are left as they are.  idx (ascending, distinct) and count (device) as rs_filter writes
 * them.  descs: HOST array.  Errors: RS_ERR_INVALID_ARG, RS_ERR_CUDA. */
rs_status rs_scatter_columns(const rs_gather_desc* descs, int32_t n_desc, const uint32_t* idx,
                             const uint32_t* count, int64_t max_count, void* stream);

/* ---- batched execution: autotuner --------------------------------------------------- */

/* Choice of rs_autotune. */
typedef struct rs_tune_result {
  int32_t tile_w, tile_h;     /* tile shape: 16x16, 32x8 or 8x8 */
  int32_t smem_batch;         /* rs_config.batch: records staged per blend batch */
  int32_t views_per_launch;   /* views per launch (consecutive chunks of the view list) */
  float ms_per_view;          /* measured device time per view of the choice */
  int32_t cached;             /* 1: taken from the cache without measuring */
  int32_t n_candidates;       /* candidates measured by this call (0 if cached) */
  int32_t front_lists;        /* 1: bin with rs_bin_sort_front (RS_TUNE_FRONT and faster), 0: rs_bin_sort */
} rs_tune_result;

#define RS_TUNE_BACKWARD 1  /* time render_backward too (training), else the forward only */
#define RS_TUNE_FORCE 2     /* measure even when the workload is cached */
#define RS_TUNE_FRONT 4     /* bin with rs_bin_sort_front (else rs_bin_sort); the choice is
                               timed on whole lists too and the faster kept (front_lists) */

/* rs_autotune -- chooses the tile shape, the Gaussians staged per shared-memory batch of
 * the blend kernels and the views per launch for rendering the given views (the paper has
 * no counterpart: it serves the batched execution of many views, the training views of
 * Sec. 3.2 and the per-cluster view sets of Sec. 3.4).  It times the library's own
 * project -> bin_sort (rs_bin_sort_front with RS_TUNE_FRONT) -> render (with importance)
 * [-> render_backward] in two stages:
 * (1) every tile shape (16x16, 32x8, 8x8) x staging batch (1, 2, 4 records per thread),
 * all of the first min(n_views, 16) views in one launch per stage; (2) with the winner of
 * (1), views per launch 1, 2, 4, ... and n_views over the first min(n_views,
 * max(views per launch, 16)) views; (3) with RS_TUNE_FRONT, the choice of (2) once more on
 * whole lists (rs_bin_sort), keeping the faster binning (front_lists, also counted in
 * n_candidates).  Each candidate gets one untimed pass and three timed
 * passes (CUDA events on `stream`); the score is device milliseconds per view.  The choice
 * is cached under the workload (view sizes, n_items, g->n, sh_degree, subset use,
 * RS_TUNE_BACKWARD, RS_TUNE_FRONT, cfg apart from batch); a later call with the same
 * workload returns it without device work unless RS_TUNE_FORCE.
 * g, subset_idx (device, may be NULL) and n_items (host [n_views]) as in a batch of all the
 * views; cams: host [n_views]; cfg: its batch field is ignored; cand_ms (host, may be
 * NULL): rs_autotune_candidates(n_views) floats, device ms per view of each candidate in
 * the order of stage (1) (tile shape major, then 1, 2, 4 records per thread) followed by
 * stage (2) (ascending views per launch), -1 where a candidate was not measured.
 * Not a hot call: it allocates and frees device memory (cudaMalloc / cudaFree),
 * synchronises the stream, and must not run during stream capture.  The importance and
 * gradient buffers it renders into are its own.  Candidates needing 2^32 or more
 * instances, or more device memory than is free, are skipped.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_UNSUPPORTED (sh_degree), RS_ERR_CAPACITY (no
 * candidate fits), RS_ERR_CUDA, or a device status the pipeline reported. */
rs_status rs_autotune(const rs_gaussians* g, const rs_camera* cams, int32_t n_views,
                      const int64_t* n_items, const uint32_t* subset_idx, const rs_config* cfg,
                      int32_t flags, rs_tune_result* out, float* cand_ms, void* stream);

/* Number of candidates rs_autotune considers for n_views views (length of cand_ms). */
int32_t rs_autotune_candidates(int32_t n_views);

/* Empties the autotuner's cache (host state, guarded by a mutex). */
void rs_autotune_clear(void);

/* ---- peak probes -------------------------------------------------------------------- */

/* Kinds of rs_peak_probe. */
typedef enum rs_probe_kind {
  RS_PROBE_FFMA = 0,     /* FP32 fused multiply-add; work = FMA lane operations */
  RS_PROBE_FFMA2 = 1,    /* packed two-lane FP32 FMA (__ffma2_rn); work = FP32 lane operations */
  RS_PROBE_ALU = 2,      /* FP32 minimum / maximum (ALU pipe); work = lane operations */
  RS_PROBE_EX2 = 3,      /* ex2.approx (MUFU); work = lane operations */
  RS_PROBE_SMEM = 4,     /* conflict-free 16-byte shared-memory loads; work = bytes */
  RS_PROBE_L2 = 5        /* 16-byte loads of a 24 MB buffer held in L2 (the first 24 MB of
                            sink, read only); work = bytes */
} rs_probe_kind;

/* rs_peak_probe -- measures a peak the library's rooflines divide by (the paper has no
 * counterpart).  Launches one kernel of independent operations of the given kind on every
 * SM (8 CTAs of 256 threads per SM, `iters` iterations of 8 independent chains per thread,
 * or of passes over the L2 buffer) on `stream` and writes to *work (HOST) how many
 * operations (bytes for RS_PROBE_SMEM and RS_PROBE_L2) it performs; the caller times the
 * launch (CUDA events) and divides.  sink: device float
 * [sink_floats >= rs_peak_probe_sink_floats()], overwritten with meaningless values.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_CUDA. */
rs_status rs_peak_probe(int32_t kind, int32_t iters, float* sink, int64_t sink_floats, double* work,
                        void* stream);
int64_t rs_peak_probe_sink_floats(void);

/* ---- tracing ------------------------------------------------------------------------ */

/* Per-launch timing of the library's kernels (no counterpart in the paper; used to measure
 * each kernel against its roofline).  rs_profile_enable(1) clears the records and starts
 * bracketing every kernel launch of the library with two CUDA events on the launch's
 * stream (launches on a stream being captured into a CUDA graph are not recorded);
 * rs_profile_enable(0) clears and stops.  rs_profile_count() is the number of records;
 * rs_profile_read(i, &name, &ms) waits for record i and gives the kernel's name (static
 * string) and device time in milliseconds.  Host-side state, guarded by a mutex.
 * Errors: RS_ERR_INVALID_ARG (index or null pointer), RS_ERR_CUDA. */
rs_status rs_profile_enable(int32_t on);
int32_t rs_profile_count(void);
rs_status rs_profile_read(int32_t i, const char** name, float* ms);

#ifdef __cplusplus
}
#endif

#endif /* RADSPLAT_H */
