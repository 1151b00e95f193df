"""PyTorch-facing binding of the C ABI (include/radsplat.h).

Tensors provide device memory and the current CUDA stream; every computation runs in
the library's kernels.  Unsigned device arrays (uint32 item ids, uint16 rects, uint32
importance bits) are held in int32 / int16 tensors with the same bits.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _native as N

__all__ = ["Gaussians", "ViewBatch", "Projected", "Bins", "DeviceStatus", "Workspace", "config", "project",
           "bin_sort", "render", "importance", "filter", "nearest", "render_backward", "Rasterizer",
           "RadSplatFunction", "split_images", "importance_as_float", "autotune", "TILE_SHAPES", "blend_threads", "adam_step",
           "gather_columns", "scatter_columns", "touched_columns", "ssim_loss", "PAPER_LAMBDA", "kmeans", "nn_distance", "image_grads",
           "init_log_scales", "StepGraph"]

PAPER_LAMBDA = 0.2   # weight of the SSIM term in the loss of Sec. 3.2

TILE_SHAPES = ((16, 16), (32, 8), (8, 8))


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def config(eps2d: float = 0.3, near_plane: float = 0.2, bg=(0.0, 0.0, 0.0), batch: int = 0,
           grad_overwrite: bool = False) -> N.RsConfig:
    """rs_config; batch = Gaussian records staged per blend batch (0: default);
    grad_overwrite: render_backward writes the gradients instead of adding into them."""
    c = N.lib().rs_config_default()
    c.eps2d = eps2d
    c.near_plane = near_plane
    c.batch = int(batch)
    c.grad_overwrite = 1 if grad_overwrite else 0
    for i in range(3):
        c.bg[i] = float(bg[i])
    return c


class Gaussians:
    """FP32 structure-of-arrays parameters on the device (Sec. 3.2)."""

    def __init__(self, means, log_scales, quats, opacity_logit, sh, sh_degree: int):
        self.means, self.log_scales, self.quats = means, log_scales, quats
        self.opacity_logit, self.sh, self.sh_degree = opacity_logit, sh, int(sh_degree)
        for t in self.tensors():
            if t.dtype != torch.float32 or not t.is_contiguous():
                raise ValueError("Gaussian parameters must be contiguous float32 tensors")

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        return cls(*(torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device) for a in scene.arrays()),
                   scene.sh_degree)

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    def tensors(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logit, self.sh)

    def struct(self) -> N.RsGaussians:
        return N.RsGaussians(self.means.data_ptr(), self.log_scales.data_ptr(), self.quats.data_ptr(),
                             self.opacity_logit.data_ptr(), self.sh.data_ptr(), self.n, self.sh_degree, 0)


def _camera_struct(cam) -> N.RsCamera:
    c = N.RsCamera()
    vm = np.asarray(cam["viewmat"], dtype=np.float32).reshape(12)
    for i in range(12):
        c.viewmat[i] = float(vm[i])
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


class ViewBatch:
    """Views rendered together (rs_view_batch): descriptors on the device, optional
    per-view ascending visibility lists (Sec. 3.4)."""

    def __init__(self, cams: Sequence[dict], n_gaussians: int, subsets: Optional[Sequence] = None,
                 tile=(16, 16), device="cuda"):
        V = len(cams)
        if subsets is not None and len(subsets) != V:
            raise ValueError("one subset per view")
        n_items = np.array([(s.numel() if isinstance(s, torch.Tensor) else len(s)) for s in subsets]
                           if subsets is not None else [n_gaussians] * V, dtype=np.int64)
        cam_arr = (N.RsCamera * V)(*[_camera_struct(c) for c in cams])
        host = (N.RsView * V)()
        b = N.RsViewBatch()
        N.call("rs_views_prepare", cam_arr, V, n_items.ctypes.data_as(ctypes.c_void_p), int(tile[0]), int(tile[1]),
               host, N.ref(b))
        raw = np.frombuffer(bytes(host), dtype=np.uint8).copy()
        self.views_dev = torch.as_tensor(raw, device=device)
        self.views_host = host
        if subsets is not None and all(isinstance(s, torch.Tensor) for s in subsets):
            # device index lists (int32 bits of uint32 ids), e.g. rs_filter outputs: no host copy
            self.subset = torch.cat([s.to(device=device, dtype=torch.int32).reshape(-1) for s in subsets])
        elif subsets is not None:
            sub = np.concatenate([np.asarray(s, dtype=np.uint32) for s in subsets]).view(np.int32)
            self.subset = torch.as_tensor(sub, device=device)
        else:
            self.subset = None
        b.views = self.views_dev.data_ptr()
        b.subset_idx = self.subset.data_ptr() if self.subset is not None else None
        self.batch = b
        self.cams = list(cams)
        self.n_gaussians = int(n_gaussians)
        self.tile = (int(tile[0]), int(tile[1]))

    @property
    def n_views(self):
        return self.batch.n_views

    @property
    def n_items(self):
        return self.batch.n_items

    @property
    def n_tiles(self):
        return self.batch.n_tiles

    @property
    def n_pixels(self):
        return self.batch.n_pixels


@dataclass
class Projected:
    xy: torch.Tensor        # [M, 2] f32
    conic_o: torch.Tensor   # [M, 4] f32
    rgb_d: torch.Tensor     # [M, 4] f32
    rect: torch.Tensor      # [M, 4] int16 (uint16 bits)
    n_tiles: torch.Tensor   # [M] int32 (uint32 bits)

    @classmethod
    def empty(cls, m: int, device="cuda"):
        m = max(int(m), 1)
        return cls(torch.empty((m, 2), dtype=torch.float32, device=device),
                   torch.empty((m, 4), dtype=torch.float32, device=device),
                   torch.empty((m, 4), dtype=torch.float32, device=device),
                   torch.empty((m, 4), dtype=torch.int16, device=device),
                   torch.empty((m,), dtype=torch.int32, device=device))

    def struct(self) -> N.RsProjected:
        return N.RsProjected(self.xy.data_ptr(), self.conic_o.data_ptr(), self.rgb_d.data_ptr(),
                             self.rect.data_ptr(), self.n_tiles.data_ptr())


@dataclass
class Bins:
    vals: torch.Tensor                  # [capacity] int32 (uint32 item ids)
    ranges: torch.Tensor                # [n_tiles, 2] int32
    keys: Optional[torch.Tensor]        # [capacity] int64 (uint64 bits) or None
    capacity: int

    @classmethod
    def empty(cls, capacity: int, n_tiles: int, keys: bool = False, device="cuda"):
        capacity = max(int(capacity), 1)
        return cls(torch.empty(capacity, dtype=torch.int32, device=device),
                   torch.empty((max(n_tiles, 1), 2), dtype=torch.int32, device=device),
                   torch.empty(capacity, dtype=torch.int64, device=device) if keys else None, capacity)

    def struct(self) -> N.RsBins:
        return N.RsBins(self.keys.data_ptr() if self.keys is not None else None, self.vals.data_ptr(),
                        self.ranges.data_ptr(), self.capacity)


class DeviceStatus:
    """rs_device_status in device memory (32 bytes)."""

    def __init__(self, device="cuda"):
        self.t = torch.zeros(4, dtype=torch.int64, device=device)

    def ptr(self):
        return ctypes.c_void_p(self.t.data_ptr())

    def zero_(self):
        self.t.zero_()

    def read(self) -> dict:
        a = self.t.cpu().numpy()
        code_nonfinite = a[0:1].view(np.int32)
        return {"code": int(code_nonfinite[0]), "nonfinite": int(code_nonfinite[1]), "required": int(a[1]),
                "n_instances": int(a[2])}


class Workspace:
    """A byte buffer that grows on request (never shrinks)."""

    def __init__(self, device="cuda"):
        self.device = device
        self.t = None

    def get(self, nbytes: int) -> torch.Tensor:
        nbytes = max(int(nbytes), 256)
        if self.t is None or self.t.numel() < nbytes:
            self.t = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self.t


def project(g: Gaussians, vb: ViewBatch, cfg: Optional[N.RsConfig] = None, status: Optional[DeviceStatus] = None,
            out: Optional[Projected] = None, stream=None) -> Projected:
    cfg = cfg or config()
    out = out or Projected.empty(vb.n_items, g.means.device)
    N.call("rs_project", N.ref(g.struct()), N.ref(vb.batch), N.ref(cfg), N.ref(out.struct()),
           status.ptr() if status else None, _stream(stream))
    return out


def bin_sort(proj: Projected, vb: ViewBatch, bins: Bins, ws: Workspace, status: DeviceStatus, stream=None,
             front: bool = False) -> Bins:
    """rs_bin_sort (every tile's whole list), or with ``front`` rs_bin_sort_front (the part of
    every list in front of the depth where the tile's pixels provably saturate: the blend,
    importance and backward results are the same)."""
    nbytes = N.lib().rs_workspace_size(N.RS_STAGE_BIN_SORT, N.ref(vb.batch), bins.capacity)
    w = ws.get(nbytes)
    N.call("rs_bin_sort_front" if front else "rs_bin_sort", N.ref(proj.struct()), N.ref(vb.batch),
           N.ref(bins.struct()), _ptr(w), w.numel(), status.ptr(), _stream(stream))
    return bins


def render(proj: Projected, bins: Bins, vb: ViewBatch, cfg: Optional[N.RsConfig] = None, image=True,
           T_final=True, last=True, importance: Optional[torch.Tensor] = None, stream=None):
    """Returns (image [3*n_pixels] planar per view, T_final [n_pixels], last [n_pixels])."""
    cfg = cfg or config()
    dev = proj.xy.device
    img = torch.empty(3 * vb.n_pixels, dtype=torch.float32, device=dev) if image is True else image
    T = torch.empty(vb.n_pixels, dtype=torch.float32, device=dev) if T_final is True else T_final
    L = torch.empty(vb.n_pixels, dtype=torch.int32, device=dev) if last is True else last
    img = img if img is not False else None
    T = T if T is not False else None
    L = L if L is not False else None
    n_g = importance.numel() if importance is not None else 0
    N.call("rs_render", N.ref(proj.struct()), N.ref(bins.struct()), N.ref(vb.batch), N.ref(cfg), _ptr(img),
           _ptr(T), _ptr(L), _ptr(importance), n_g, _stream(stream))
    return img, T, L


def importance(proj: Projected, bins: Bins, vb: ViewBatch, h: torch.Tensor, cfg=None, stream=None) -> torch.Tensor:
    """Max-accumulates Eq. (importance-score) over the batch's views into h (int32 bits of float32)."""
    cfg = cfg or config()
    N.call("rs_importance", N.ref(proj.struct()), N.ref(bins.struct()), N.ref(vb.batch), N.ref(cfg), _ptr(h),
           h.numel(), _stream(stream))
    return h


def importance_as_float(h: torch.Tensor) -> torch.Tensor:
    return h.view(torch.float32)


def filter(h: torch.Tensor, t: float, mode: int, ws: Optional[Workspace] = None, mask=True, idx=True, stream=None):
    """Sec. 3.3 / Eq. (importance-score-vis): (mask uint8 [n], idx int32 [n], count int32 [1])."""
    n = h.numel()
    dev = h.device
    ws = ws or Workspace(dev)
    vb = N.RsViewBatch()
    vb.n_items = n
    nbytes = N.lib().rs_workspace_size(N.RS_STAGE_FILTER, N.ref(vb), 0)
    w = ws.get(nbytes)
    m = torch.empty(max(n, 1), dtype=torch.uint8, device=dev) if mask is True else (None if mask is False else mask)
    ix = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if idx is True else (None if idx is False else idx)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    hf = h.view(torch.float32) if h.dtype == torch.int32 else h
    N.call("rs_filter", _ptr(hf), n, float(t), int(mode), _ptr(m), _ptr(ix), _ptr(cnt), _ptr(w), w.numel(),
           _stream(stream))
    return m, ix, cnt


def nearest(centres: torch.Tensor, cam_centres: torch.Tensor, stream=None) -> torch.Tensor:
    """Sec. 3.4: index of the nearest cluster centre for each camera centre."""
    out = torch.empty(cam_centres.shape[0], dtype=torch.int32, device=cam_centres.device)
    N.call("rs_filter_nearest", _ptr(centres), centres.shape[0], _ptr(cam_centres), cam_centres.shape[0], _ptr(out),
           _stream(stream))
    return out


def nn_distance(means: torch.Tensor, ws: Optional[Workspace] = None, stream=None) -> torch.Tensor:
    """rs_nn_distance: distance from each point (means [3, n]) to its nearest other point."""
    m = means.to(torch.float32).contiguous()
    n = m.shape[1]
    d = torch.empty(n, dtype=torch.float32, device=m.device)
    ws = ws or Workspace(m.device)
    w = ws.get(N.lib().rs_nn_workspace_size(n))
    N.call("rs_nn_distance", _ptr(m), n, _ptr(d), _ptr(w), w.numel(), _stream(stream))
    return d


def init_log_scales(means: torch.Tensor, floor: float = 1e-7) -> torch.Tensor:
    """Sec. 3.2 initial scales: log of the nearest-neighbour distance (floored), on 3 rows."""
    d = nn_distance(means)
    return torch.log(torch.clamp(d, min=floor)).expand(3, -1).contiguous()


def kmeans(points: torch.Tensor, init: torch.Tensor, iterations: int = 50, stream=None):
    """Sec. 3.4 camera clustering (rs_kmeans): returns (centres [k, 3], assignment [n])."""
    pts = points.to(torch.float32).contiguous()
    centres = init.to(device=pts.device, dtype=torch.float32).clone().contiguous()
    assign = torch.empty(pts.shape[0], dtype=torch.int32, device=pts.device)
    N.call("rs_kmeans", _ptr(pts), pts.shape[0], _ptr(centres), centres.shape[0], int(iterations), _ptr(assign),
           _stream(stream))
    return centres, assign


def render_backward(g: Gaussians, vb: ViewBatch, proj: Projected, bins: Bins, T_final, last, dL_dimage,
                    grads: Sequence[torch.Tensor], ws: Workspace, cfg=None, stream=None):
    """Adds d(L)/d(params) into grads (means, log_scales, quats, opacity_logit, sh), or
    writes them over grads when cfg.grad_overwrite is set."""
    cfg = cfg or config()
    gs = N.RsGaussianGrads(*(t.data_ptr() for t in grads))
    nbytes = N.lib().rs_workspace_size(N.RS_STAGE_BACKWARD, N.ref(vb.batch), 0)
    w = ws.get(nbytes)
    N.call("rs_render_backward", N.ref(g.struct()), N.ref(vb.batch), N.ref(cfg), N.ref(proj.struct()),
           N.ref(bins.struct()), _ptr(T_final), _ptr(last), _ptr(dL_dimage), N.ref(gs), _ptr(w), w.numel(),
           _stream(stream))


def image_grads(vb: ViewBatch, ws: Workspace):
    """Per-item image-space gradients the last render_backward of `vb` left in `ws`
    (rs_backward_image_grads): (g_xy_ab [n_items, 4], g_c_o_rg [n_items, 4], g_b [n_items])
    float32 views of the workspace: dL/d(x, y, a, b), dL/d(c, o, r, g), dL/d(blue)."""
    out = N.RsImageGrads()
    w = ws.t
    if w is None:
        raise ValueError("no backward has run with this workspace")
    N.call("rs_backward_image_grads", N.ref(vb.batch), _ptr(w), w.numel(), N.ref(out))
    n = int(vb.n_items)
    base = w.data_ptr()
    f = w.view(torch.uint8)

    def at(ptr, count):
        off = ptr - base
        return f[off: off + 4 * count].view(torch.float32)

    return (at(out.g_xy_ab, 4 * n).view(n, 4), at(out.g_c_o_rg, 4 * n).view(n, 4), at(out.g_b, n))


def blend_threads(tile) -> int:
    """Threads of a blend CTA for a tile shape: one warp per tile (eight pixels per thread,
    two for 8x8), so rs_config.batch is 1, 2 or 4 x 32 for every shape."""
    return 32


def autotune(g: Gaussians, cams: Sequence[dict], subsets: Optional[Sequence] = None, cfg=None,
             backward: bool = True, force: bool = False, stream=None, front: bool = True) -> dict:
    """rs_autotune: tile shape, records staged per blend batch and views per launch for
    rendering `cams` (cached per workload); ``front`` times binning by rs_bin_sort_front
    (the Rasterizer's default), else by rs_bin_sort.

    Returns {"tile": (w, h), "smem_batch": rs_config.batch, "views_per_launch", "cached",
    "ms_per_view", "n_candidates", "front" (bin with front lists: ``front`` given and faster
    than whole lists for the choice), "stage1": {(w, h, records per thread): ms per view},
    "stage2": {views per launch: ms per view}}."""
    cfg = cfg or config()
    V = len(cams)
    if subsets is not None and len(subsets) != V:
        raise ValueError("one subset per view")
    n_items = np.array([len(x) for x in subsets] if subsets is not None else [g.n] * V, dtype=np.int64)
    sub = None
    if subsets is not None:
        sub = torch.as_tensor(np.concatenate([np.asarray(x, dtype=np.uint32) for x in subsets]).view(np.int32),
                              device=g.means.device)
    cam_arr = (N.RsCamera * V)(*[_camera_struct(c) for c in cams])
    res = N.RsTuneResult()
    nc = N.lib().rs_autotune_candidates(V)
    cand = (ctypes.c_float * nc)()
    flags = ((N.RS_TUNE_BACKWARD if backward else 0) | (N.RS_TUNE_FORCE if force else 0) |
             (N.RS_TUNE_FRONT if front else 0))
    N.call("rs_autotune", N.ref(g.struct()), cam_arr, V, n_items.ctypes.data_as(ctypes.c_void_p), _ptr(sub),
           N.ref(cfg), flags, N.ref(res), cand, _stream(stream))
    batches = []
    b = 1
    while b < V:
        batches.append(b)
        b *= 2
    batches.append(V)
    stage1, stage2 = {}, {}
    for si, (tw, th) in enumerate(TILE_SHAPES):
        for pi, m in enumerate((1, 2, 4)):
            ms = cand[si * 3 + pi]
            if ms >= 0:
                stage1[(tw, th, m)] = float(ms)
    for bi, bb in enumerate(batches):
        ms = cand[9 + bi]
        if ms >= 0:
            stage2[bb] = float(ms)
    return {"tile": (res.tile_w, res.tile_h), "smem_batch": res.smem_batch, "views_per_launch": res.views_per_launch,
            "cached": bool(res.cached), "ms_per_view": float(res.ms_per_view), "n_candidates": res.n_candidates,
            "front": bool(res.front_lists), "stage1": stage1, "stage2": stage2}


def ssim_loss(image: torch.Tensor, target: torch.Tensor, width: int, height: int, lam: float = 0.2,
              dL_dimage: Optional[torch.Tensor] = None, loss: Optional[torch.Tensor] = None,
              ws: Optional[Workspace] = None, stream=None):
    """rs_ssim_loss over planes [n_planes][height][width] (flat or shaped): the loss of
    Sec. 3.2, (1 - lam) MSE + lam (1 - SSIM), float64 [1], and dL/dimage."""
    n = image.numel()
    if n % (width * height) != 0 or target.numel() != n:
        raise ValueError("image and target must hold whole planes of width x height")
    planes = n // (width * height)
    g = torch.empty_like(image) if dL_dimage is None else dL_dimage
    l = torch.empty(1, dtype=torch.float64, device=image.device) if loss is None else loss
    ws = ws or Workspace(image.device)
    w = ws.get(N.lib().rs_ssim_workspace_size(width, height, planes))
    N.call("rs_ssim_loss", _ptr(image), _ptr(target), width, height, planes, float(lam), _ptr(g), _ptr(l), _ptr(w),
           w.numel(), _stream(stream))
    return l, g


def adam_step(groups: Sequence[tuple], step: int, betas=(0.9, 0.999), eps: float = 1e-15, stream=None):
    """rs_adam_step: groups of (param, grad, m, v, lr) float32 tensors updated in place."""
    arr = (N.RsAdamGroup * len(groups))()
    for i, (p, g, m, v, lr) in enumerate(groups):
        for t in (p, g, m, v):
            if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != p.numel():
                raise ValueError("Adam arrays must be contiguous float32 tensors of one size")
        arr[i] = N.RsAdamGroup(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), p.numel(), float(lr), 0)
    N.call("rs_adam_step", arr, len(groups), float(betas[0]), float(betas[1]), float(eps), int(step), _stream(stream))


def gather_columns(pairs: Sequence[tuple], idx: torch.Tensor, count: torch.Tensor, max_count: int, stream=None):
    """rs_gather_columns: for each (src [rows, n] or [n], dst [rows, >= max_count] or [>= max_count])
    float32 pair, dst[:, k] = src[:, idx[k]] for k < count (device)."""
    arr = (N.RsGatherDesc * len(pairs))()
    for i, (src, dst) in enumerate(pairs):
        if src.dtype != torch.float32 or dst.dtype != torch.float32 or not src.is_contiguous() \
                or not dst.is_contiguous():
            raise ValueError("gather arrays must be contiguous float32 tensors")
        rows = src.shape[0] if src.dim() == 2 else 1
        arr[i] = N.RsGatherDesc(src.data_ptr(), dst.data_ptr(), rows, src.shape[-1], dst.shape[-1])
    N.call("rs_gather_columns", arr, len(pairs), _ptr(idx), _ptr(count), int(max_count), _stream(stream))


def scatter_columns(pairs: Sequence[tuple], idx: torch.Tensor, count: torch.Tensor, max_count: int, stream=None):
    """rs_scatter_columns: for each (src [rows, >= max_count] packed, dst [rows, n]) float32
    pair, dst[:, idx[k]] = src[:, k] for k < count (device)."""
    arr = (N.RsGatherDesc * len(pairs))()
    for i, (src, dst) in enumerate(pairs):
        if src.dtype != torch.float32 or dst.dtype != torch.float32 or not src.is_contiguous() \
                or not dst.is_contiguous():
            raise ValueError("scatter arrays must be contiguous float32 tensors")
        rows = dst.shape[0] if dst.dim() == 2 else 1
        arr[i] = N.RsGatherDesc(src.data_ptr(), dst.data_ptr(), rows, src.shape[-1], dst.shape[-1])
    N.call("rs_scatter_columns", arr, len(pairs), _ptr(idx), _ptr(count), int(max_count), _stream(stream))


def touched_columns(src: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """rs_touched_columns: float32 [n], 1 where a column of src [rows, n] has a non-zero entry."""
    if src.dtype != torch.float32 or not src.is_contiguous() or src.dim() != 2:
        raise ValueError("src must be a contiguous float32 [rows, n] tensor")
    rows, n = src.shape
    out = torch.empty(n, dtype=torch.float32, device=src.device) if out is None else out
    N.call("rs_touched_columns", _ptr(src), rows, n, _ptr(out), _stream(stream))
    return out


class StepGraph:
    """A step repeated with fixed buffers, captured once as a CUDA graph: the host-to-device
    copies of its inputs from pinned host memory, the library calls `body` enqueues, and the
    device-to-host copies of its outputs; `run()` replays it (one graph launch) and waits.

    inputs: (pinned host tensor, device tensor) pairs copied in before the body;
    outputs: (device tensor, pinned host tensor) pairs copied out after it.  The body must
    not synchronise the host (every library hot call qualifies) and must use the current
    stream.  Capacity-dependent calls (bin_sort) need their capacity sized beforehand."""

    def __init__(self, body, inputs=(), outputs=(), warmup: int = 2, device=None):
        self.body, self.inputs, self.outputs = body, list(inputs), list(outputs)
        for h, d in self.inputs:
            if not h.is_pinned():
                raise ValueError("inputs must come from pinned host memory")
        for d, h in self.outputs:
            if not h.is_pinned():
                raise ValueError("outputs must go to pinned host memory")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        torch.cuda.synchronize(dev)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(max(warmup, 1)):   # allocations and lazy initialisation happen here
                self._enqueue()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._enqueue()
        torch.cuda.synchronize(dev)
        self.device = dev

    def _enqueue(self):
        for h, d in self.inputs:
            d.copy_(h, non_blocking=True)
        self.body()
        for d, h in self.outputs:
            h.copy_(d, non_blocking=True)

    def launch(self):
        """Enqueue one replay on the current stream without waiting (for callers that
        order it against their own streams, e.g. an input pipeline on a copy stream)."""
        self.graph.replay()

    def run(self):
        self.launch()
        torch.cuda.current_stream(self.device).synchronize()


def split_images(flat: torch.Tensor, vb: ViewBatch) -> List[torch.Tensor]:
    out = []
    for v in range(vb.n_views):
        hv = vb.views_host[v]
        base = 3 * hv.pixel_base
        out.append(flat[base: base + 3 * hv.width * hv.height].view(3, hv.height, hv.width))
    return out


class Rasterizer:
    """Owns workspaces and the instance capacity for repeated renders of view batches.

    The capacity grows on demand: rs_bin_sort reports the instance count it needed, and a
    render whose count exceeded the capacity is redone with a larger one (one host
    synchronisation per call on this path; fixed-capacity graph replay avoids it).
    ``front`` (default): bin with rs_bin_sort_front, which leaves out the entries behind the
    depth where every pixel of a tile has provably stopped; False keeps every list whole."""

    def __init__(self, cfg: Optional[N.RsConfig] = None, device="cuda", capacity: int = 0, keys: bool = False,
                 front: bool = True):
        self.cfg = cfg or config()
        self.device = device
        self.capacity = int(capacity)
        self.keys = keys
        self.front = front
        self.ws_sort = Workspace(device)
        self.ws_bwd = Workspace(device)
        self.status = DeviceStatus(device)
        self._bins = None

    def bins_for(self, vb: ViewBatch) -> Bins:
        if self._bins is None or self._bins.capacity < self.capacity or self._bins.ranges.shape[0] < vb.n_tiles \
                or (self.keys and self._bins.keys is None):
            self._bins = Bins.empty(self.capacity, vb.n_tiles, keys=self.keys, device=self.device)
        b = self._bins
        return Bins(b.vals, b.ranges[:max(vb.n_tiles, 1)], b.keys, b.capacity)

    def forward(self, g: Gaussians, vb: ViewBatch, importance: Optional[torch.Tensor] = None, image=True):
        if self.capacity <= 0:
            self.capacity = max(4 * vb.n_items, 1 << 16)
        self.status.zero_()
        proj = project(g, vb, self.cfg, self.status)
        while True:
            bins = self.bins_for(vb)
            bin_sort(proj, vb, bins, self.ws_sort, self.status, front=self.front)
            st = self.status.read()
            if st["required"] <= bins.capacity:
                break
            self.capacity = int(st["required"] * 1.25) + 1024
            self.status.zero_()
        img, T, L = render(proj, bins, vb, self.cfg, image=image, importance=importance)
        return {"image": img, "T_final": T, "last": L, "proj": proj, "bins": bins, "n_instances": st["n_instances"]}


class RadSplatFunction(torch.autograd.Function):
    """Differentiable render of a view batch: params -> flat planar images [3*n_pixels]."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, sh, vb: ViewBatch, rast: Rasterizer, sh_degree: int):
        g = Gaussians(means.detach(), log_scales.detach(), quats.detach(), opacity_logit.detach(), sh.detach(),
                      sh_degree)
        out = rast.forward(g, vb)
        ctx.g, ctx.vb, ctx.rast = g, vb, rast
        ctx.proj, ctx.bins = out["proj"], out["bins"]
        ctx.save_for_backward(out["T_final"], out["last"])
        return out["image"]

    @staticmethod
    def backward(ctx, dL_dimage):
        T_final, last = ctx.saved_tensors
        g = ctx.g
        grads = [torch.zeros_like(t) for t in g.tensors()]
        render_backward(g, ctx.vb, ctx.proj, ctx.bins, T_final, last, dL_dimage.contiguous(), grads,
                        ctx.rast.ws_bwd, ctx.rast.cfg)
        return (*grads, None, None, None)


def l1_loss(image: torch.Tensor, target: torch.Tensor, dL_dimage: Optional[torch.Tensor] = None,
            loss: Optional[torch.Tensor] = None, stream=None):
    """Mean |image - target| (float64 [1]) and its gradient (rs_l1_loss)."""
    n = image.numel()
    g = torch.empty_like(image) if dL_dimage is None else dL_dimage
    l = torch.empty(1, dtype=torch.float64, device=image.device) if loss is None else loss
    N.call("rs_l1_loss", _ptr(image), _ptr(target), n, _ptr(g), _ptr(l), _stream(stream))
    return l, g
