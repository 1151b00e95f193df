"""View-sharded data parallelism: one process per GPU, each rendering its own views of the
same Gaussians.

Every view's projection, binning, blend and backward are independent of the other views
(Sec. 3.2: the photometric loss is a sum over training images), so views shard across ranks
with no exchange inside the path.  Two results are reductions over views and need one
collective each per step:

* the importance score (Eq. importance-score) is a max over all images: an all-reduce MAX of
  h, held as the int32 bits of non-negative float32 values (their integer order is the float
  order, so the max of the bits is the bits of the max);
* the parameter gradient is a sum over images: an all-reduce SUM of one flat buffer that
  holds all parameter gradients, so the exchange is a single call.

Pruning (Sec. 3.3) then thresholds the reduced h identically on every rank.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch
import torch.distributed as dist

__all__ = ["shard", "GradBuffer", "allreduce_importance", "allreduce_grads"]


def shard(n_total: int, world: int, rank: int) -> Tuple[int, int]:
    """[start, stop) of rank's contiguous share of n_total views; the first n_total % world
    ranks take one extra view."""
    if world <= 0 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(n_total, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


class GradBuffer:
    """All parameter gradients in one contiguous float32 buffer (views shaped like the
    parameters, in the order means, log_scales, quats, opacity_logit, sh)."""

    def __init__(self, params: Sequence[torch.Tensor]):
        sizes = [p.numel() for p in params]
        dev = params[0].device
        self.flat = torch.zeros(sum(sizes), dtype=torch.float32, device=dev)
        self.views: List[torch.Tensor] = []
        off = 0
        for p, n in zip(params, sizes):
            self.views.append(self.flat[off:off + n].view(p.shape))
            off += n

    def zero_(self):
        self.flat.zero_()


def allreduce_importance(h: torch.Tensor, group=None) -> torch.Tensor:
    """Max of h over ranks, in place (h: int32 bits of non-negative float32)."""
    if h.dtype != torch.int32:
        raise TypeError("importance is held as int32 bits")
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(h, op=dist.ReduceOp.MAX, group=group)
    return h


def allreduce_grads(grads: GradBuffer, group=None) -> GradBuffer:
    """Sum of the gradient buffer over ranks, in place."""
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grads.flat, op=dist.ReduceOp.SUM, group=group)
    return grads
