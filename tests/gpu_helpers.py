"""Shared helpers of the GPU parity tests: run the CUDA path through the binding and
compare with the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

import oracle

IMG_TOL = 2e-4          # max-abs per channel on unflagged pixels
FLIP_TOL = 0.02         # bound on a pixel whose skip/stop decision lies at its threshold


def u32(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def gpu_forward(scene, cams, tile=(16, 16), subsets=None, importance=True, keys=False, capacity=0):
    from paper_2403_13806_gb300 import api
    g = api.Gaussians.from_scene(scene)
    vb = api.ViewBatch(cams, scene.n, subsets=subsets, tile=tile)
    rast = api.Rasterizer(capacity=capacity, keys=keys)
    h = torch.zeros(scene.n, dtype=torch.int32, device="cuda") if importance else None
    out = rast.forward(g, vb, importance=h)
    torch.cuda.synchronize()
    out["h"] = h
    out["vb"] = vb
    out["g"] = g
    out["rast"] = rast
    return out


def check_view_against_oracle(out, scene, cam, view_index, pixels=None, mode="bucketed", subset=None):
    """Compares one view's image, T_final and last-contributor id with the oracle.

    Returns (max abs error over unflagged pixels, number of flagged pixels, oracle result)."""
    from paper_2403_13806_gb300 import api
    vb = out["vb"]
    hv = vb.views_host[view_index]
    W, H = hv.width, hv.height
    sc = scene if subset is None else scene.subset(np.asarray(subset, np.int64))
    proj = oracle.project(sc, cam, tile=vb.tile)
    ro = oracle.render(proj, pixels=pixels, mode=mode)
    img = api.split_images(out["image"], vb)[view_index].cpu().numpy()
    T = out["T_final"][hv.pixel_base: hv.pixel_base + W * H].cpu().numpy().reshape(H, W)
    last = out["last"][hv.pixel_base: hv.pixel_base + W * H].cpu().numpy().reshape(H, W)
    if pixels is None:
        vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        pix = np.stack([uu.ravel(), vv.ravel()], 1)
    else:
        pix = np.asarray(pixels).reshape(-1, 2)
    u, v = pix[:, 0], pix[:, 1]
    gi = img[:, v, u].T
    amb = ro["ambiguous"].astype(bool)
    err = np.abs(gi - ro["image"])
    errT = np.abs(T[v, u] - ro["T_final"])
    assert err[~amb].max(initial=0) <= IMG_TOL, err[~amb].max()
    assert errT[~amb].max(initial=0) <= IMG_TOL, errT[~amb].max()
    assert err[amb].max(initial=0) <= FLIP_TOL
    # last composited entry: position in the GPU tile list -> item -> Gaussian id
    vals = u32(out["bins"].vals)
    ranges = out["bins"].ranges.cpu().numpy().view(np.uint32)
    tw, th = vb.tile
    tiles = hv.tile_base + (v // th) * hv.tiles_x + (u // tw)
    L = last[v, u]
    gid = np.full(len(u), -1, np.int64)
    has = L > 0
    items = vals[ranges[tiles[has], 0] + L[has] - 1].astype(np.int64) - hv.item_base
    gid[has] = items if subset is None else np.arange(len(subset))[items]
    ok = ~amb
    assert np.array_equal(gid[ok], ro["last_id"][ok].astype(np.int64))
    return err[~amb].max(initial=0), int(amb.sum()), ro
