"""Viewpoint-based visibility filtering (Sec. 3.4) on the library's kernels.

After optimisation: cluster the input camera locations with k-means (rs_kmeans), and for
every cluster render its assigned cameras plus random cameras near it (Sec. 3.4 adds random
camera samples for robustness to test views) to obtain the cluster importance
h_j = max alpha T (Eq. importance-score-vis, rs_importance) and the visibility indicator
m_j = 1(h_j > t_cluster) as an ascending index list (rs_filter, RS_KEEP_ABOVE).  A test view
is assigned to the nearest cluster centre (rs_filter_nearest) and rendered from that
cluster's list only.  The index lists stay on the device; this module orders the calls.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np
import torch

from . import api
from . import _native as N


def camera_centre(cam: dict) -> np.ndarray:
    """World position of a camera: -R^T t of its world-to-camera [R|t]."""
    vm = np.asarray(cam["viewmat"], np.float64).reshape(3, 4)
    return (-vm[:, :3].T @ vm[:, 3]).astype(np.float32)


def _yaw(theta: float) -> np.ndarray:
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, 0.0, -s], [0.0, 1.0, 0.0], [s, 0.0, c]])


def random_cameras_near(members: Sequence[dict], centre: np.ndarray, n: int, rng: np.random.Generator,
                        max_yaw_deg: float = 30.0) -> List[dict]:
    """n cameras near a cluster: the intrinsics and orientation of a random member camera,
    turned by a random yaw about its own vertical axis, placed at the centre plus Gaussian
    jitter with the spread of the members' positions."""
    out = []
    pos = np.stack([camera_centre(c) for c in members])
    sigma = float(max(pos.std(axis=0).mean(), 1e-3))
    for _ in range(n):
        tmpl = members[int(rng.integers(0, len(members)))]
        vm = np.asarray(tmpl["viewmat"], np.float64).reshape(3, 4)
        R = _yaw(np.deg2rad(rng.uniform(-max_yaw_deg, max_yaw_deg))) @ vm[:, :3]
        c = centre.astype(np.float64) + rng.normal(0.0, sigma, 3)
        cam = dict(tmpl)
        cam["viewmat"] = np.concatenate([R, (-R @ c)[:, None]], axis=1).astype(np.float32)
        out.append(cam)
    return out


class VisibilityFilter:
    """Per-cluster visibility lists for a set of Gaussians and input cameras (Sec. 3.4)."""

    def __init__(self, g: api.Gaussians, cams: Sequence[dict], k: int = 64, t_cluster: float = 0.001,
                 extra_per_cluster: int = 4, iterations: int = 50, seed: int = 0, tile=(16, 16), cfg=None):
        self.g = g
        self.cams = list(cams)
        self.k = min(int(k), len(self.cams))
        self.t_cluster = float(t_cluster)
        self.extra = int(extra_per_cluster)
        self.iterations = int(iterations)
        self.rng = np.random.default_rng(seed)
        self.tile = tuple(tile)
        self.cfg = cfg or api.config()
        self.rast = api.Rasterizer(cfg=self.cfg, device=g.means.device)
        self.centres: Optional[torch.Tensor] = None
        self.assign: Optional[np.ndarray] = None
        self.lists: List[torch.Tensor] = []
        self.importance: List[torch.Tensor] = []
        self.cluster_cams: List[List[dict]] = []

    def build(self):
        dev = self.g.means.device
        pos = np.stack([camera_centre(c) for c in self.cams])
        init = pos[np.sort(self.rng.choice(len(pos), size=self.k, replace=False))]
        self.centres, assign = api.kmeans(torch.as_tensor(pos, device=dev), torch.as_tensor(init, device=dev),
                                          self.iterations)
        self.assign = assign.cpu().numpy()
        centres = self.centres.cpu().numpy()
        self.lists, self.importance, self.cluster_cams = [], [], []
        for j in range(self.k):
            members = [c for c, a in zip(self.cams, self.assign) if a == j]
            views = members + (random_cameras_near(members, centres[j], self.extra, self.rng) if members else [])
            self.cluster_cams.append(views)
            h = torch.zeros(self.g.n, dtype=torch.int32, device=dev)
            for s0 in range(0, len(views), 8):
                vb = api.ViewBatch(views[s0:s0 + 8], self.g.n, tile=self.tile, device=dev)
                self.rast.forward(self.g, vb, importance=h, image=False)
            _, idx, cnt = api.filter(h, self.t_cluster, N.RS_KEEP_ABOVE, mask=False)
            self.importance.append(h)
            self.lists.append(idx[:int(cnt.item())])
        return self

    def cluster_of(self, cams: Sequence[dict]) -> np.ndarray:
        pos = torch.as_tensor(np.stack([camera_centre(c) for c in cams]), device=self.g.means.device)
        return api.nearest(self.centres, pos).cpu().numpy()

    def render(self, cams: Sequence[dict]):
        """Renders test views, each from the visibility list of its nearest cluster."""
        js = self.cluster_of(cams)
        vb = api.ViewBatch(list(cams), self.g.n, subsets=[self.lists[j] for j in js], tile=self.tile,
                           device=self.g.means.device)
        out = self.rast.forward(self.g, vb)
        out["vb"] = vb
        out["clusters"] = js
        return out
