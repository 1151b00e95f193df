"""Shared helpers of the GPU parity tests: run the CUDA path through the binding and
compare with the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

import oracle

IMG_TOL = 2e-4          # max-abs per channel on unflagged pixels (the stated image tolerance)


def u32(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def gpu_forward(scene, cams, tile=(16, 16), subsets=None, importance=True, keys=False, capacity=0, front=True):
    from paper_2403_13806_gb300 import api
    g = api.Gaussians.from_scene(scene)
    vb = api.ViewBatch(cams, scene.n, subsets=subsets, tile=tile)
    rast = api.Rasterizer(capacity=capacity, keys=keys, front=front)
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
    # flagged pixels (reading C6): both renderings composite the same entries in front of the
    # first near-threshold decision and at most T_amb of colour <= c_amb behind it
    bound = ro["T_amb"] * ro["c_amb"] + IMG_TOL
    assert np.all(err[amb].max(1, initial=0) <= bound[amb])
    assert np.all(errT[amb] <= ro["T_amb"][amb] + IMG_TOL)
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


GRAD_KEYS = ("means", "log_scales", "quats", "opacity_logit", "sh")
IMG_GRAD_KEYS = ("g_xy", "g_conic", "g_opacity", "g_rgb")


def oracle_grads_two_means(args):
    """Worker (process pool, spawn): FP64 gradients of one view on sampled pixels at the FP64
    image means and camera centre (with the magnitude scales), and at the FP32 means and the
    FP32-rounded camera centre a single-precision renderer holds (reading C5), for the
    Gaussians that receive anything, as (ids, {name: values [..., ids]})."""
    import oracle.grad as og
    scene, cam, w, pix, threads = args
    torch.set_num_threads(threads)
    r64 = og.gradients(scene, cam, w, pixels=pix, scales=True)
    proj = oracle.project(scene, cam)
    shift = np.where(proj["valid"][:, None] == 1, oracle.mean2d_f32(scene, cam) - proj["xy"], 0.0)
    vm = np.asarray(cam["viewmat"], np.float32).astype(np.float64).reshape(3, 4)
    centre32 = (-(vm[:, :3].T @ vm[:, 3])).astype(np.float32)
    r32 = og.gradients(scene, cam, w, pixels=pix, mean_shift=shift, cam_centre=centre32)
    ids = np.nonzero((r64["scale_opacity"] > 0) | (r64["scale_rgb"] > 0).any(1))[0]
    out = {}
    for k in GRAD_KEYS:
        out[k] = r64[k][..., ids]
        out["scale_" + k] = r64["scale_" + k][..., ids]
        out["f32_" + k] = r32[k][..., ids]
    for k in IMG_GRAD_KEYS:
        out[k] = r64[k][ids]
        out["scale_" + k[2:]] = r64["scale_" + k[2:]][ids]
        out["f32_" + k] = r32[k][ids]
    return ids, out


def walk_tolerance(L_max: int) -> float:
    """Relative bound (of the magnitude scale) on the FP32 evaluation of a sum of per-pixel
    gradient terms when each pixel's list is walked back over at most L_max entries: every
    step recovers T by the hardware reciprocal (relative error < 2^-22) and one rounded
    product, and adds into rounded FP32 sums (2^-24 each), so a part of a term carries at
    most (L_max + 16) (2^-22 + 2^-23) relative error; 16 covers the per-term arithmetic
    outside the walk and the chain through the projection."""
    return (L_max + 16) * (2.0 ** -22 + 2.0 ** -23)


def check_gradient_elements(gpu, ref, scale, ref32, eps, floor, what):
    """|gpu - ref| <= eps * scale + 2 |ref - ref32| + floor, element by element; returns the
    largest ratio |gpu - ref| / bound."""
    gpu = np.asarray(gpu, np.float64)
    bound = eps * scale + 2.0 * np.abs(ref - ref32) + floor
    err = np.abs(gpu - ref)
    bad = err > bound
    if bad.any():
        where = np.argwhere(bad)[:8]
        detail = [(tuple(int(i) for i in w), float(gpu[tuple(w)]), float(ref[tuple(w)]), float(scale[tuple(w)]),
                   float(ref32[tuple(w)]), float(bound[tuple(w)])) for w in where]
        raise AssertionError(f"{what}: {int(bad.sum())} elements beyond the bound; "
                             f"(index, gpu, oracle, scale, oracle at FP32 means, bound): {detail}")
    return float((err / bound).max(initial=0.0))
