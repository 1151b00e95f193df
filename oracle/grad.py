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


def project_torch(params: dict, cam: dict, eps2d: float = 0.3):
    """Differentiable FP64 projection; returns xy [N,2], conic [N,3], opacity [N], rgb [N,3]."""
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
    cc = -(M.T @ m)
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


def gradients(scene, cam, dL_dimage, eps2d=0.3, near=0.2, bg=(0.0, 0.0, 0.0), chunk=4096, pixels=None):
    """d(sum dL_dimage * image)/d(params) in FP64 for one view.

    dL_dimage: [3,H,W], or [P,3] for the listed pixels [P,2] (u, v).  Returns a dict with
    the parameter gradients (same layouts as the scene arrays) and the image-space
    gradients per Gaussian: g_xy [N,2], g_conic [N,3] (w.r.t. (a, b, c) with
    power = -(a dx^2 + c dy^2)/2 - b dx dy), g_opacity [N], g_rgb [N,3].  Culled
    Gaussians get zeros.  With pixels given, each chunk of pixels composites only the
    Gaussians whose support box contains one of its pixels (every other Gaussian has
    alpha < 1/255 there and is skipped anyway), so the result is the same."""
    proj, order = _fixed_decisions(scene, cam, eps2d, near)
    W, H = cam["width"], cam["height"]
    p = params_of(scene)
    xy, conic, o, rgb = project_torch(p, cam, eps2d)
    leaves = [t.detach().clone().requires_grad_(True) for t in (xy, conic, o, rgb)]
    if pixels is None:
        vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        pixels = np.stack([uu.ravel(), vv.ravel()], axis=1)
        g = torch.as_tensor(np.asarray(dL_dimage, dtype=np.float64).reshape(3, -1).T)   # [P,3]
        prune = False
    else:
        pixels = np.asarray(pixels).reshape(-1, 2)
        g = torch.as_tensor(np.asarray(dL_dimage, dtype=np.float64).reshape(-1, 3))
        prune = True
    ordt = torch.as_tensor(order)
    if prune:
        oxy = proj["xy"][order]
        ext = proj["ext"][order] * (1.0 + 1e-6) + 1e-6
    for s in range(0, pixels.shape[0], chunk):
        pc = pixels[s:s + chunk]
        sel = ordt
        if prune:
            hit = np.zeros(len(order), dtype=bool)
            for u, v in pc:
                hit |= (np.abs(oxy[:, 0] - u) <= ext[:, 0]) & (np.abs(oxy[:, 1] - v) <= ext[:, 1])
            sel = ordt[torch.as_tensor(hit)]
        img, _ = composite_torch(*leaves, sel, pc, bg)
        (img * g[s:s + chunk]).sum().backward()
    grads2d = [lf.grad if lf.grad is not None else torch.zeros_like(lf) for lf in leaves]
    torch.autograd.backward([xy, conic, o, rgb], grads2d)
    out = {k: p[k].grad.numpy().copy() for k in ("means", "log_scales", "quats", "opacity_logit", "sh")}
    out.update(g_xy=grads2d[0].numpy(), g_conic=grads2d[1].numpy(), g_opacity=grads2d[2].numpy(),
               g_rgb=grads2d[3].numpy())
    return out
