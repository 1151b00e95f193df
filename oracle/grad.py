"""FP64 gradient oracle (PyTorch autograd on the CPU) for the splatting hot path.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the benchmark).

The training step of Sec. 3.2 ("Radiance Field-based Supervision") differentiates the
rendered image of Eq. (render-gs) with respect to every point's position, scale,
rotation, opacity and SH coefficients.  This module restates the same forward as
``radsplat_oracle.c`` with differentiable FP64 tensor operations -- the projection
Sigma' = J M Sigma M^T J^T with Sigma = R S S^T R^T, sigmoid opacity, SH colour from the
associated-Legendre recurrence, and per-pixel front-to-back compositing -- and lets
autograd produce the exact derivative.  The discrete decisions (which entries are
skipped, where compositing stops, the front-to-back order, which points are culled)
are piecewise constant; they are taken from the FP64 values and held fixed, so the
gradient is that of the active branch.

The skip/stop rule and the order key are the same readings as in the C oracle
(alpha = min(0.99, o e^power); skip power > 0 or alpha < 1/255; stop before the entry
whose T(1-alpha) < 1e-4; order by the FP32 depth key, ties to the lower index).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import project as _c_project

ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4


def _assoc_legendre(l: int, m: int, x: torch.Tensor) -> torch.Tensor:
    """P_l^m(x) with the Condon-Shortley phase by the standard three-term recurrence."""
    somx2 = torch.sqrt(torch.clamp((1.0 - x) * (1.0 + x), min=0.0))
    pmm = torch.ones_like(x)
    fact = 1.0
    for _ in range(m):
        pmm = -pmm * fact * somx2
        fact += 2.0
    if l == m:
        return pmm
    pmmp1 = x * (2.0 * m + 1.0) * pmm
    if l == m + 1:
        return pmmp1
    for ll in range(m + 2, l + 1):
        pll = ((2.0 * ll - 1.0) * x * pmmp1 - (ll + m - 1.0) * pmm) / (ll - m)
        pmm, pmmp1 = pmmp1, pll
    return pmmp1


def sh_basis(degree: int, d: torch.Tensor) -> torch.Tensor:
    """Y_lm(d) for unit directions d [3, N] -> [(degree+1)^2, N] (index l*l + l + m)."""
    ct = torch.clamp(d[2], -1.0, 1.0)
    phi = torch.atan2(d[1], d[0])
    out = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            P = _assoc_legendre(l, am, ct)
            if m == 0:
                out.append(K * P)
            elif m > 0:
                out.append(math.sqrt(2.0) * K * torch.cos(m * phi) * P)
            else:
                out.append(math.sqrt(2.0) * K * torch.sin(am * phi) * P)
    return torch.stack(out)


def project_torch(params: dict, cam: dict, eps2d: float = 0.3, cam_centre=None):
    """Differentiable FP64 projection; returns xy [N,2], conic [N,3], opacity [N], rgb [N,3].
    cam_centre (optional, 3 floats): take the SH view direction from this camera centre
    instead of -M^T m (e.g. that centre rounded to FP32, as a single-precision renderer
    holds it)."""
    means, ls, q, lg, sh = (params[k] for k in ("means", "log_scales", "quats", "opacity_logit", "sh"))
    degree = params["sh_degree"]
    vm = torch.tensor(np.asarray(cam["viewmat"], dtype=np.float32).reshape(3, 4).astype(np.float64))
    M, m = vm[:, :3], vm[:, 3]
    fx, fy, cx, cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    W, H = cam["width"], cam["height"]
    lim_x, lim_y = 1.3 * (0.5 * W / fx), 1.3 * (0.5 * H / fy)

    qn = q / torch.linalg.norm(q, dim=0, keepdim=True)
    w, x, y, z = qn
    R = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)]),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)]),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]),
    ]).permute(2, 0, 1)                                             # [N,3,3]
    s2 = torch.exp(2.0 * ls).T                                      # [N,3]
    Sig = R @ torch.diag_embed(s2) @ R.transpose(1, 2)              # [N,3,3]
    t = (M @ means) + m[:, None]                                    # [3,N]
    tz = t[2]
    ux, uy = t[0] / tz, t[1] / tz
    uxc, uyc = torch.clamp(ux, -lim_x, lim_x), torch.clamp(uy, -lim_y, lim_y)
    zero = torch.zeros_like(tz)
    J = torch.stack([torch.stack([fx / tz, zero, -fx * uxc / tz]),
                     torch.stack([zero, fy / tz, -fy * uyc / tz])]).permute(2, 0, 1)   # [N,2,3]
    T = J @ M
    S2 = T @ Sig @ T.transpose(1, 2)
    a, b, c = S2[:, 0, 0] + eps2d, S2[:, 0, 1], S2[:, 1, 1] + eps2d
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], dim=1)
    xy = torch.stack([fx * ux + cx, fy * uy + cy], dim=1)
    o = torch.sigmoid(lg)
    cc = -(M.T @ m) if cam_centre is None else torch.as_tensor(np.asarray(cam_centre, dtype=np.float64))
    d = means - cc[:, None]
    d = d / torch.linalg.norm(d, dim=0, keepdim=True)
    Y = sh_basis(degree, d)                                         # [ncoef, N]
    ncoef = (degree + 1) ** 2
    shr = sh.reshape(ncoef, 3, -1)
    rgb = torch.clamp(0.5 + (shr * Y[:, None, :]).sum(0), min=0.0).T   # [N,3]
    return xy, conic, o, rgb


def composite_torch(xy, conic, o, rgb, order, pixels, bg=(0.0, 0.0, 0.0)):
    """Front-to-back compositing of the pixels [P,2] over Gaussians in ``order``.

    Returns image [P,3] and T_final [P]."""
    xy, conic, o, rgb = xy[order], conic[order], o[order], rgb[order]
    px = torch.as_tensor(pixels, dtype=torch.float64)
    dx = px[:, 0:1] - xy[None, :, 0]
    dy = px[:, 1:2] - xy[None, :, 1]
    power = -0.5 * (conic[None, :, 0] * dx * dx + conic[None, :, 2] * dy * dy) - conic[None, :, 1] * dx * dy
    alpha = torch.clamp(o[None, :] * torch.exp(power), max=ALPHA_MAX)
    with torch.no_grad():
        keep = (power <= 0.0) & (alpha >= ALPHA_MIN)
    a_eff = torch.where(keep, alpha, torch.zeros_like(alpha))
    one_minus = 1.0 - a_eff
    T_after = torch.cumprod(one_minus, dim=1)
    T_before = torch.cat([torch.ones_like(T_after[:, :1]), T_after[:, :-1]], dim=1)
    with torch.no_grad():
        stop_here = keep & (T_after < T_MIN)
        stopped = torch.cumsum(stop_here.to(torch.int32), dim=1) > 0   # the stop entry and all after
        incl = keep & ~stopped
    wgt = torch.where(incl, a_eff * T_before, torch.zeros_like(a_eff))
    img = wgt @ rgb
    T_final = torch.prod(torch.where(incl, one_minus, torch.ones_like(one_minus)), dim=1)
    bgt = torch.as_tensor(bg, dtype=torch.float64)
    return img + T_final[:, None] * bgt[None, :], T_final


def _fixed_decisions(scene, cam, eps2d, near):
    proj = _c_project(scene, cam, eps2d=eps2d, near=near)
    valid = np.nonzero(proj["valid"])[0]
    depth = proj["depth"][valid]
    order = valid[np.lexsort((valid, depth))]    # by FP32 depth, ties to the lower index
    return proj, order


def params_of(scene, requires_grad=True) -> dict:
    p = {k: torch.tensor(np.asarray(v, dtype=np.float64), requires_grad=requires_grad)
         for k, v in zip(("means", "log_scales", "quats", "opacity_logit", "sh"), scene.arrays())}
    p["sh_degree"] = scene.sh_degree
    return p


def render_torch(scene, cam, eps2d=0.3, near=0.2, bg=(0.0, 0.0, 0.0), pixels=None):
    """FP64 image [3,H,W] of one view by the differentiable restatement (no gradient)."""
    _, order = _fixed_decisions(scene, cam, eps2d, near)
    W, H = cam["width"], cam["height"]
    if pixels is None:
        vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        pixels = np.stack([uu.ravel(), vv.ravel()], axis=1)
    with torch.no_grad():
        p = params_of(scene, requires_grad=False)
        xy, conic, o, rgb = project_torch(p, cam, eps2d)
        img, T = composite_torch(xy, conic, o, rgb, torch.as_tensor(order), pixels, bg)
    return img.numpy(), T.numpy()


def _box_hits(pixels, xy, ext, width, height, cell=64):
    """For each pixel, the indices of the boxes |p - xy| <= ext (per axis) holding it.
    Each box is listed in the cell-grid cells it overlaps; a pixel tests only its cell's."""
    ncx, ncy = (width + cell - 1) // cell, (height + cell - 1) // cell
    x0 = np.floor((xy[:, 0] - ext[:, 0]) / cell)
    x1 = np.floor((xy[:, 0] + ext[:, 0]) / cell)
    y0 = np.floor((xy[:, 1] - ext[:, 1]) / cell)
    y1 = np.floor((xy[:, 1] + ext[:, 1]) / cell)
    on = (x1 >= 0) & (x0 <= ncx - 1) & (y1 >= 0) & (y0 <= ncy - 1)
    idx = np.nonzero(on)[0]
    cx0 = np.clip(x0[idx], 0, ncx - 1).astype(np.int64)
    cx1 = np.clip(x1[idx], 0, ncx - 1).astype(np.int64)
    cy0 = np.clip(y0[idx], 0, ncy - 1).astype(np.int64)
    cy1 = np.clip(y1[idx], 0, ncy - 1).astype(np.int64)
    nx = cx1 - cx0 + 1
    cnt = nx * (cy1 - cy0 + 1)
    gi = np.repeat(np.arange(len(idx)), cnt)
    k = np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    cells = (cy0[gi] + k // nx[gi]) * ncx + cx0[gi] + k % nx[gi]
    srt = np.argsort(cells, kind="stable")
    cs, gs = cells[srt], idx[gi[srt]]
    out = []
    for u, v in pixels:
        c = (int(v) // cell) * ncx + int(u) // cell
        lo, hi = np.searchsorted(cs, c, "left"), np.searchsorted(cs, c, "right")
        j = gs[lo:hi]
        out.append(j[(np.abs(xy[j, 0] - u) <= ext[j, 0]) & (np.abs(xy[j, 1] - v) <= ext[j, 1])])
    return out


def _pair_scales(xy, conic, o, rgb, pixel, w, bg):
    """Cancellation-free magnitudes of one pixel's contributions to the image-space
    gradients of the entries it composites (rows of the arguments, front to back).

    With C = sum_j c_j a_j T_j + T_final bg, dC/da_j = c_j T_j - B_j / (1 - a_j), B_j the
    colour composited behind j plus T_final bg.  Each part is kept by its magnitude:
    M_j = sum_ch |w_ch| (c_j T_j + B_j / (1 - a_j)) for dL/da_j; then, where the 0.99 clamp
    is inactive, M_j a_j for dL/dpower, M_j e^power for dL/do, and for the mean and conic
    M_j a_j times |a dx| + |b dy|, |b dx| + |c dy|, dx^2 / 2, |dx dy|, dy^2 / 2; a_j T_j |w_ch|
    for the colour.  Returns [n, 9] in the order x, y, a, b, c, o, r, g, b."""
    u, v = float(pixel[0]), float(pixel[1])
    dx, dy = u - xy[:, 0], v - xy[:, 1]
    A, B, Cc = conic[:, 0], conic[:, 1], conic[:, 2]
    power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy
    e = np.exp(power)
    araw = o * e
    alpha = np.minimum(araw, ALPHA_MAX)
    keep = (power <= 0.0) & (alpha >= ALPHA_MIN)
    n = len(o)
    out = np.zeros((n, 9))
    a_eff = np.where(keep, alpha, 0.0)
    T_after = np.cumprod(1.0 - a_eff)
    stops = np.nonzero(keep & (T_after < T_MIN))[0]
    end = stops[0] if len(stops) else n          # compositing stops before this entry
    idx = np.nonzero(keep[:end])[0]
    if len(idx) == 0:
        return out
    Tb_all = np.concatenate([[1.0], T_after[:-1]])
    Tb = Tb_all[idx]
    T = T_after[end - 1] if end > 0 else 1.0      # T_final
    aw = np.abs(np.asarray(w, dtype=np.float64))
    contrib = rgb[idx] * (alpha[idx] * Tb)[:, None]                      # [m, 3]
    behind = np.cumsum(contrib[::-1], axis=0)[::-1] - contrib + T * np.abs(np.asarray(bg))[None, :]
    M = ((rgb[idx] * Tb[:, None] + behind / (1.0 - alpha[idx])[:, None]) * aw[None, :]).sum(1)
    free = araw[idx] < ALPHA_MAX
    Mp = np.where(free, M * alpha[idx], 0.0)
    ddx, ddy = dx[idx], dy[idx]
    out[idx, 0] = Mp * (np.abs(A[idx] * ddx) + np.abs(B[idx] * ddy))
    out[idx, 1] = Mp * (np.abs(B[idx] * ddx) + np.abs(Cc[idx] * ddy))
    out[idx, 2] = Mp * 0.5 * ddx * ddx
    out[idx, 3] = Mp * np.abs(ddx * ddy)
    out[idx, 4] = Mp * 0.5 * ddy * ddy
    out[idx, 5] = np.where(free, M * e[idx], 0.0)
    out[idx, 6:9] = (alpha[idx] * Tb)[:, None] * aw[None, :]
    return out


def gradients(scene, cam, dL_dimage, eps2d=0.3, near=0.2, bg=(0.0, 0.0, 0.0), chunk=4096, pixels=None,
              mean_shift=None, scales=False, cam_centre=None):
    """d(sum dL_dimage * image)/d(params) in FP64 for one view.

    dL_dimage: [3,H,W], or [P,3] for the listed pixels [P,2] (u, v).  Returns a dict with
    the parameter gradients (same layouts as the scene arrays) and the image-space
    gradients per Gaussian: g_xy [N,2], g_conic [N,3] (w.r.t. (a, b, c) with
    power = -(a dx^2 + c dy^2)/2 - b dx dy), g_opacity [N], g_rgb [N,3].  Culled
    Gaussians get zeros.  With pixels given, each chunk of pixels composites only the
    Gaussians whose support box contains one of its pixels (every other Gaussian has
    alpha < 1/255 there and is skipped anyway), so the result is the same.

    mean_shift ([N,2], optional): evaluate everything with the image means moved by this
    much (the derivative chain through the mean unchanged), e.g. to the FP32 means a
    single-precision renderer uses; the decisions stay those of the unshifted means.
    cam_centre (optional): the camera centre the SH directions start from (project_torch).
    scales (pixels mode): also return scale_xy, scale_conic, scale_opacity, scale_rgb, the
    sum over pixels of the cancellation-free magnitudes of their contributions to the
    image-space gradients (_pair_scales), and scale_<parameter> = |J|^T of those per
    Gaussian (J the projection's Jacobian from the parameters to x, y, a, b, c, o, r, g, b):
    the scale against which the rounding of a single-precision evaluation of the same sums
    is measured."""
    proj, order = _fixed_decisions(scene, cam, eps2d, near)
    W, H = cam["width"], cam["height"]
    n = scene.n
    shift = None if mean_shift is None else np.asarray(mean_shift, dtype=np.float64).reshape(n, 2)
    ext_all = proj["ext"] * (1.0 + 1e-6) + 1e-6
    if shift is not None:
        ext_all = ext_all + np.abs(shift)
    if pixels is None:
        vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        pixels = np.stack([uu.ravel(), vv.ravel()], axis=1)
        g = torch.as_tensor(np.asarray(dL_dimage, dtype=np.float64).reshape(3, -1).T)   # [P,3]
        prune = False
        cand = np.arange(n)
    else:
        pixels = np.asarray(pixels).reshape(-1, 2)
        g = torch.as_tensor(np.asarray(dL_dimage, dtype=np.float64).reshape(-1, 3))
        prune = True
        # every Gaussian whose support box holds one of the pixels; the rest have alpha < 1/255
        # at all of them, get no gradient, and need not be projected
        per_pix = _box_hits(pixels, proj["xy"][order], ext_all[order], W, H)   # positions in `order`
        cand = np.sort(order[np.unique(np.concatenate(per_pix))]) if per_pix else np.zeros(0, np.int64)
    sub = scene.subset(cand) if len(cand) < n else scene
    p = params_of(sub)
    xy, conic, o, rgb = project_torch(p, cam, eps2d, cam_centre=cam_centre)
    if shift is not None:
        xy = xy + torch.as_tensor(shift[cand])
    leaves = [t.detach().clone().requires_grad_(True) for t in (xy, conic, o, rgb)]
    local = np.searchsorted(cand, order[np.isin(order, cand)])     # front-to-back order, local ids
    ordt = torch.as_tensor(local)
    if prune:
        # each pixel's entries as positions in the local front-to-back order
        rank_of_order_pos = np.full(len(order), -1, np.int64)
        rank_of_order_pos[np.nonzero(np.isin(order, cand))[0]] = np.arange(len(local))
    sc9 = np.zeros((len(cand), 9)) if scales else None
    if scales and not prune:
        raise ValueError("scales need sampled pixels")
    det = [t.detach().numpy() for t in leaves] if scales else None
    gnp = g.numpy()
    step = 1 if prune else chunk   # sparse pixels: one at a time is cheapest
    for s0 in range(0, pixels.shape[0], step):
        pc = pixels[s0:s0 + step]
        sel = ordt
        if prune:
            ranks = np.unique(np.concatenate([rank_of_order_pos[per_pix[s0 + q]] for q in range(len(pc))]))
            sel = ordt[torch.as_tensor(ranks)]
        img, _ = composite_torch(*leaves, sel, pc, bg)
        (img * g[s0:s0 + step]).sum().backward()
        if scales:
            ids = sel.numpy()
            if len(ids):
                sc9[ids] += _pair_scales(det[0][ids], det[1][ids], det[2][ids], det[3][ids], pc[0], gnp[s0], bg)
    grads2d = [lf.grad if lf.grad is not None else torch.zeros_like(lf) for lf in leaves]
    pkeys = ("means", "log_scales", "quats", "opacity_logit", "sh")
    pscale = None
    if scales:
        # |J|^T s per Gaussian: the projection acts on each Gaussian alone, so one backward
        # pass per image-space component with that component's unit seed on every Gaussian
        # gives that row of every Gaussian's Jacobian
        outs = (xy, conic, o, rgb)
        cols = [(0, 0), (0, 1), (1, 0), (1, 1), (1, 2), (2, None), (3, 0), (3, 1), (3, 2)]
        pscale = [np.zeros(p[k].shape) for k in pkeys]
        for ci, (oi, cj) in enumerate(cols):
            seeds = [torch.zeros_like(t) for t in outs]
            if cj is None:
                seeds[oi][:] = 1.0
            else:
                seeds[oi][:, cj] = 1.0
            rows = torch.autograd.grad(list(outs), [p[k] for k in pkeys], grad_outputs=seeds, retain_graph=True,
                                       allow_unused=True)
            for k, r in enumerate(rows):
                if r is not None:
                    pscale[k] += np.abs(r.numpy()) * sc9[:, ci]
    torch.autograd.backward([xy, conic, o, rgb], grads2d)

    out = {}
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        gk = p[k].grad.numpy()
        if len(cand) < n:
            z = np.zeros(gk.shape[:-1] + (n,))
            z[..., cand] = gk
            gk = z
        out[k] = gk.copy()
    for name, t in zip(("g_xy", "g_conic", "g_opacity", "g_rgb"), grads2d):
        a = t.numpy()
        if len(cand) < n:
            z = np.zeros((n,) + a.shape[1:])
            z[cand] = a
            a = z
        out[name] = a
    if scales:
        for k, a in zip(pkeys, pscale):
            if len(cand) < n:
                z = np.zeros(a.shape[:-1] + (n,))
                z[..., cand] = a
                a = z
            out["scale_" + k] = a
        for name, a in (("scale_xy", sc9[:, 0:2]), ("scale_conic", sc9[:, 2:5]), ("scale_opacity", sc9[:, 5]),
                        ("scale_rgb", sc9[:, 6:9])):
            if len(cand) < n:
                z = np.zeros((n,) + a.shape[1:])
                z[cand] = a
                a = z
            out[name] = a
    return out
