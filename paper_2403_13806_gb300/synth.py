"""Seeded synthetic scenes and cameras for the splatting hot path.

This module only draws random numbers and builds camera poses. It holds none of
the rendering arithmetic, so both the CUDA path and the FP64 oracle read their
inputs from here without sharing any of the method's code.

The paper's scenes (mip-NeRF 360 and Zip-NeRF captures, Sec. 4) and its trained
point clouds are not available; the generators below stand in for them with the
shapes the paper works at: about 1M Gaussians after initialisation (Sec. 3.5),
degree-3 spherical harmonics (Sec. 3.2), object-centric 360-degree camera rings
and house-scale scenes whose cameras are grouped into spatial clusters (Sec. 3.4).

Layouts (all float32, structure of arrays):
  means        [3, N]
  log_scales   [3, N]
  quats        [4, N]   (w, x, y, z), not normalised
  opacity_logit[N]
  sh           [(D+1)^2 * 3, N]  row = coefficient * 3 + channel
Cameras are dicts with a row-major 3x4 world-to-camera matrix ``viewmat``
(OpenCV axes: x right, y down, z forward), ``fx, fy, cx, cy``, ``width``, ``height``.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Scene", "camera", "look_at", "ring_cameras", "config0", "config1", "config2",
    "config3", "config4", "fd_crop", "perturbed_copy", "random_unit_quats",
]


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    def subset(self, idx: np.ndarray) -> "Scene":
        return Scene(self.means[:, idx].copy(), self.log_scales[:, idx].copy(),
                     self.quats[:, idx].copy(), self.opacity_logit[idx].copy(),
                     self.sh[:, idx].copy(), self.sh_degree)

    def arrays(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logit, self.sh)


def camera(viewmat, fx, fy, cx, cy, width, height) -> dict:
    vm = np.asarray(viewmat, dtype=np.float32).reshape(3, 4)
    return {"viewmat": vm, "fx": float(np.float32(fx)), "fy": float(np.float32(fy)),
            "cx": float(np.float32(cx)), "cy": float(np.float32(cy)),
            "width": int(width), "height": int(height)}


def look_at(position, target, world_up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """World-to-camera [R|t] for a camera at ``position`` looking at ``target``.

    Rows of R are the camera's right, down and forward axes in world
    coordinates; ``world_up`` is the world direction that appears upward.
    """
    c = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(world_up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ c
    return np.concatenate([R, t[:, None]], axis=1).astype(np.float32)


def random_unit_quats(rng, n) -> np.ndarray:
    q = rng.normal(size=(4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return q.astype(np.float32)


def _sh_block(rng, n, degree, dc_sigma=0.3, rest_sigma=0.05) -> np.ndarray:
    ncoef = (degree + 1) ** 2
    sh = np.empty((ncoef * 3, n), dtype=np.float32)
    sh[:3] = rng.normal(0.0, dc_sigma, size=(3, n))
    if ncoef > 1:
        sh[3:] = rng.normal(0.0, rest_sigma, size=((ncoef - 1) * 3, n))
    return sh


def _params(rng, means, degree, log_scale_mu=-3.0, log_scale_sigma=0.5) -> Scene:
    n = means.shape[1]
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, size=(3, n)).astype(np.float32)
    quats = random_unit_quats(rng, n)
    logit = rng.normal(0.0, 1.0, size=n).astype(np.float32)
    sh = _sh_block(rng, n, degree)
    return Scene(np.ascontiguousarray(means, dtype=np.float32), log_scales, quats, logit, sh, degree)


def config0(seed: int = 0, n: int = 2000):
    """2k Gaussians in front of one 128x128 camera at the origin (f=120)."""
    rng = np.random.default_rng(seed)
    means = np.empty((3, n), dtype=np.float32)
    means[0] = rng.uniform(-1, 1, n)
    means[1] = rng.uniform(-1, 1, n)
    means[2] = rng.uniform(2, 6, n)
    scene = _params(rng, means, degree=0)
    cam = camera(np.eye(3, 4), 120.0, 120.0, 64.0, 64.0, 128, 128)
    return scene, [cam]


def fd_crop(seed: int = 3, n: int = 200):
    """200 Gaussians with the config-0 distribution in front of a 64x64 camera (f=60)."""
    rng = np.random.default_rng(seed)
    means = np.empty((3, n), dtype=np.float32)
    means[0] = rng.uniform(-1, 1, n)
    means[1] = rng.uniform(-1, 1, n)
    means[2] = rng.uniform(2, 6, n)
    scene = _params(rng, means, degree=3)
    cam = camera(np.eye(3, 4), 60.0, 60.0, 32.0, 32.0, 64, 64)
    return scene, [cam]


def _object_shell_means(rng, n, object_frac=0.7):
    n_obj = int(round(n * object_frac))
    n_shell = n - n_obj
    obj = rng.normal(0.0, 1.0, size=(3, n_obj))
    d = rng.normal(size=(3, n_shell))
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    r = rng.uniform(8.0, 20.0, size=n_shell)
    shell = d * r
    means = np.concatenate([obj, shell], axis=1)
    perm = rng.permutation(n)
    return means[:, perm].astype(np.float32)


def ring_cameras(n_views, radius=4.0, width=1280, height=832, f=1200.0):
    cams = []
    for k in range(n_views):
        th = 2.0 * np.pi * k / n_views
        pos = (radius * np.cos(th), 0.0, radius * np.sin(th))
        cams.append(camera(look_at(pos, (0.0, 0.0, 0.0)), f, f, width / 2, height / 2, width, height))
    return cams


def config1(seed: int = 1, n: int = 500_000, n_views: int = 32, width=1280, height=832):
    """360-degree capture: dense central object plus background shell, SH degree 3."""
    rng = np.random.default_rng(seed)
    scene = _params(rng, _object_shell_means(rng, n), degree=3)
    f = 1200.0 * width / 1280.0
    return scene, ring_cameras(n_views, width=width, height=height, f=f)


def config2(seed: int = 2, n: int = 1_000_000, n_views: int = 1, width=1280, height=832):
    """1M Gaussians shaped as config 1, viewed from the ring (first view at angle 0)."""
    rng = np.random.default_rng(seed)
    scene = _params(rng, _object_shell_means(rng, n), degree=3)
    f = 1200.0 * width / 1280.0
    return scene, ring_cameras(max(n_views, 1), width=width, height=height, f=f)[:n_views]


def perturbed_copy(scene: Scene, seed: int) -> Scene:
    """The scene a training target is rendered from: means, DC colour and opacity logits jittered."""
    rng = np.random.default_rng(seed)
    s = Scene(*(a.copy() for a in scene.arrays()), scene.sh_degree)
    s.means += rng.normal(0.0, 0.01, size=s.means.shape).astype(np.float32)
    s.sh[:3] += rng.normal(0.0, 0.05, size=(3, s.n)).astype(np.float32)
    s.opacity_logit += rng.normal(0.0, 0.2, size=s.n).astype(np.float32)
    return s


def _house_sites():
    xs = np.array([-6.0, -2.0, 2.0, 6.0])
    zs = np.array([-4.0, 4.0])
    return np.array([(x, 0.0, z) for z in zs for x in xs])


def _house_camera(rng, site, width, height):
    pos = site + rng.normal(0.0, 0.3, size=3)
    pos[1] = np.clip(pos[1], -1.2, 1.2)
    yaw = rng.uniform(0.0, 2.0 * np.pi)
    target = pos + np.array([np.sin(yaw), 0.0, np.cos(yaw)])
    f = 0.9375 * width
    return camera(look_at(pos, target), f, f, width / 2, height / 2, width, height), pos


def config3(seed: int = 4, n: int = 3_000_000, per_site: int = 8):
    """House-scale scene: uniform box 20x3x20 (y vertical), 64 cameras at 8 sites."""
    rng = np.random.default_rng(seed)
    means = np.empty((3, n), dtype=np.float32)
    means[0] = rng.uniform(-10, 10, n)
    means[1] = rng.uniform(-1.5, 1.5, n)
    means[2] = rng.uniform(-10, 10, n)
    scene = _params(rng, means, degree=3, log_scale_mu=-3.5)
    cams, sites = [], []
    for s, site in enumerate(_house_sites()):
        for _ in range(per_site):
            cam, pos = _house_camera(rng, site, 960, 544)
            cams.append(cam)
            sites.append(s)
    return scene, cams, np.array(sites)


def config4(scene: Scene, seed: int = 5, n_views: int = 256, min_subset=200_000, max_subset=2_000_000):
    """Uneven batch: 256 views of random resolution, each with its own ascending Gaussian subset."""
    rng = np.random.default_rng(seed)
    sites = _house_sites()
    cams, subsets = [], []
    for _ in range(n_views):
        w = int(rng.integers(320, 1921))
        h = int(rng.integers(240, 1081))
        cam, _ = _house_camera(rng, sites[rng.integers(0, len(sites))], w, h)
        cams.append(cam)
        k = int(rng.integers(min(min_subset, scene.n), min(max_subset, scene.n) + 1))
        subsets.append(np.sort(rng.choice(scene.n, size=k, replace=False)).astype(np.uint32))
    return cams, subsets
