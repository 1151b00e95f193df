"""Optimisation of the point parameters on synthetic targets with importance pruning.

Sec. 3.2 optimises phi = {(p, k, s, o, q)} with the loss (1 - lambda) L2 + lambda (1 - SSIM)
against target renders (here renders of a perturbed scene stand in for the radiance-field
teacher's renders; an L1 loss is available too), the
optimiser and learning rates of 3D Gaussian Splatting (Adam, eps 1e-15; SH rest at 1/20 of
the DC rate), one training view drawn uniformly per step; Sec. 3.3 prunes the points whose
importance h (Eq. importance-score, max over all training views) is below t_prune, twice
during optimisation (Sec. 3.5: after 16k and 24k steps).  Every step runs in the library's
kernels: render, loss, backward, rs_adam_step; pruning is rs_importance over the training
views, rs_filter (RS_PRUNE_KEEP) and rs_gather_columns over the parameters and both Adam
moments.  This module only orders the calls and owns the tensors.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import api
from . import _native as N

# learning rates of 3D Gaussian Splatting's optimiser, per parameter array
DEFAULT_LR = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "opacity_logit": 5e-2, "sh_dc": 2.5e-3,
              "sh_rest": 2.5e-3 / 20.0}


@dataclass
class PruneRecord:
    step: int
    n_before: int
    n_after: int
    t_prune: float


class Trainer:
    """Adam on the SoA parameters of `g` (modified in place and replaced at pruning)."""

    def __init__(self, g: api.Gaussians, cams: Sequence[dict], targets: Sequence[torch.Tensor],
                 prune_steps: Sequence[int] = (), t_prune: float = 0.01, lr: Optional[dict] = None,
                 extent: float = 1.0, betas=(0.9, 0.999), eps: float = 1e-15, seed: int = 0, tile=(16, 16),
                 cfg=None, loss: str = "paper", lam: float = api.PAPER_LAMBDA):
        if len(cams) != len(targets):
            raise ValueError("one target per camera")
        self.g = g
        self.cams = list(cams)
        self.targets = list(targets)
        self.prune_steps = set(int(s) for s in prune_steps)
        self.t_prune = float(t_prune)
        self.lr = dict(DEFAULT_LR, **(lr or {}))
        self.lr["means"] *= extent
        self.betas, self.eps = betas, eps
        self.rng = np.random.default_rng(seed)
        self.tile = tuple(tile)
        self.cfg = cfg or api.config()
        self.cfg_w = N.RsConfig.from_buffer_copy(self.cfg)   # backward writes the gradients
        self.cfg_w.grad_overwrite = 1
        self.rast = api.Rasterizer(cfg=self.cfg, device=g.means.device)
        if loss not in ("paper", "l1"):
            raise ValueError("loss is 'paper' ((1 - lam) MSE + lam (1 - SSIM)) or 'l1'")
        self.loss_kind, self.lam = loss, float(lam)
        self.ws_loss = api.Workspace(g.means.device)
        self.step_no = 0
        self.losses: List[float] = []
        self.prunes: List[PruneRecord] = []
        self.last_importance: Optional[torch.Tensor] = None
        self._alloc_state()

    def _alloc_state(self):
        self.m = [torch.zeros_like(t) for t in self.g.tensors()]
        self.v = [torch.zeros_like(t) for t in self.g.tensors()]
        self.grads = [torch.zeros_like(t) for t in self.g.tensors()]
        self._loss = torch.zeros(1, dtype=torch.float64, device=self.g.means.device)

    def _groups(self):
        names = ("means", "log_scales", "quats", "opacity_logit")
        out = [(p, gr, m, v, self.lr[k]) for k, p, gr, m, v in zip(names, self.g.tensors()[:4], self.grads[:4],
                                                                    self.m[:4], self.v[:4])]
        sh, gsh, msh, vsh = self.g.sh, self.grads[4], self.m[4], self.v[4]
        n = self.g.n
        out.append((sh[:3].reshape(-1), gsh[:3].reshape(-1), msh[:3].reshape(-1), vsh[:3].reshape(-1),
                    self.lr["sh_dc"]))
        if sh.shape[0] > 3:
            out.append((sh[3:].reshape(-1), gsh[3:].reshape(-1), msh[3:].reshape(-1), vsh[3:].reshape(-1),
                        self.lr["sh_rest"]))
        assert all(t.numel() % max(n, 1) == 0 for t in (sh,))
        return out

    def step(self) -> float:
        """One optimisation step on one uniformly drawn training view; returns its loss."""
        i = int(self.rng.integers(0, len(self.cams)))
        vb = api.ViewBatch([self.cams[i]], self.g.n, tile=self.tile, device=self.g.means.device)
        out = self.rast.forward(self.g, vb)
        if self.loss_kind == "paper":
            cam = self.cams[i]
            loss, dl = api.ssim_loss(out["image"], self.targets[i], cam["width"], cam["height"], self.lam,
                                     loss=self._loss, ws=self.ws_loss)
        else:
            loss, dl = api.l1_loss(out["image"], self.targets[i], loss=self._loss)
        api.render_backward(self.g, vb, out["proj"], out["bins"], out["T_final"], out["last"], dl, self.grads,
                            self.rast.ws_bwd, self.cfg_w)
        self.step_no += 1
        api.adam_step(self._groups(), self.step_no, self.betas, self.eps)
        lv = float(loss.item())
        self.losses.append(lv)
        if self.step_no in self.prune_steps:
            self.prune()
        return lv

    def importance(self) -> torch.Tensor:
        """Eq. (importance-score) over all training views (int32 bits of float32 h)."""
        h = torch.zeros(self.g.n, dtype=torch.int32, device=self.g.means.device)
        for s0 in range(0, len(self.cams), 8):
            vb = api.ViewBatch(self.cams[s0:s0 + 8], self.g.n, tile=self.tile, device=self.g.means.device)
            self.rast.forward(self.g, vb, importance=h, image=False)
        return h

    def prune(self) -> PruneRecord:
        """Sec. 3.3: removes the points with h < t_prune from the parameters and Adam moments."""
        h = self.importance()
        self.last_importance = h
        n = self.g.n
        _, idx, cnt = api.filter(h, self.t_prune, N.RS_PRUNE_KEEP, mask=False)
        k = int(cnt.item())   # the one host read of a pruning step: the new point count
        old = list(self.g.tensors()) + self.m + self.v
        new = [torch.empty(t.shape[:-1] + (k,), dtype=t.dtype, device=t.device) for t in old]
        if k > 0:
            pairs = list(zip(old, new))
            for s0 in range(0, len(pairs), 16):   # at most 16 arrays per launch
                api.gather_columns(pairs[s0:s0 + 16], idx, cnt, k)
        self.g = api.Gaussians(*new[:5], self.g.sh_degree)
        self.m, self.v = new[5:10], new[10:15]
        self.grads = [torch.zeros_like(t) for t in self.g.tensors()]
        rec = PruneRecord(self.step_no, n, k, self.t_prune)
        self.prunes.append(rec)
        return rec
