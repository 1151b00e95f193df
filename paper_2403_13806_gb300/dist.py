"""View-sharded data parallelism: one process per GPU, each rendering its own views of the
same Gaussians.

Every view's projection, binning, blend and backward are independent of the other views
(Sec. 3.2: the photometric loss is a sum over training images), so views shard across ranks
with no exchange inside the path.  Two results are reductions over views and need one
collective each per step:

* the importance score (Eq. importance-score) is a max over all images: an all-reduce MAX of
  h, held as the int32 bits of non-negative float32 values (their integer order is the float
  order, so the max of the bits is the bits of the max);
* the parameter gradient is a sum over images.  In a deep scene only a small part of the
  Gaussians get a gradient from a step's views (the rest lie behind saturated pixels), so
  the sum is exchanged over the union of the columns (Gaussians) some rank touched: an
  all-reduce MAX of a per-Gaussian touched flag (4 B per Gaussian), its ascending index
  list, a gather of those columns of every gradient row into one packed buffer, an
  all-reduce SUM of that buffer, and a scatter back.  Columns outside the union are zero on
  every rank, so the result equals the dense sum element for element.  (The dense
  all-reduce of one flat buffer of all gradients is kept as allreduce_grads.)

Pruning (Sec. 3.3) then thresholds the reduced h identically on every rank.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch
import torch.distributed as dist

__all__ = ["shard", "GradBuffer", "allreduce_importance", "allreduce_grads", "SparseGradExchange", "LibraryOps"]


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


class LibraryOps:
    """The device steps of SparseGradExchange, all in the library's kernels."""

    def touched(self, mat: torch.Tensor) -> torch.Tensor:
        from . import api
        return api.touched_columns(mat)

    def compact(self, flag: torch.Tensor):
        from . import _native as N
        from . import api
        _, idx, cnt = api.filter(flag, 0.5, N.RS_KEEP_ABOVE, mask=False)
        return idx, cnt

    def gather(self, mat: torch.Tensor, idx: torch.Tensor, cnt: torch.Tensor, k: int) -> torch.Tensor:
        from . import api
        packed = torch.empty((mat.shape[0], max(k, 1)), dtype=mat.dtype, device=mat.device)
        api.gather_columns([(mat, packed)], idx, cnt, k)
        return packed

    def scatter(self, packed: torch.Tensor, mat: torch.Tensor, idx: torch.Tensor, cnt: torch.Tensor, k: int):
        from . import api
        api.scatter_columns([(packed, mat)], idx, cnt, k)


class SparseGradExchange:
    """Sum over ranks of the parameter gradients, exchanging only the columns some rank has
    a gradient for (see the module notes).  grads: the GradBuffer whose flat storage is the
    [rows, n] matrix of every gradient row of n Gaussians (means 3, log-scales 3,
    quaternions 4, opacity logit 1, SH (D+1)^2 * 3 rows).  One host read per step: the size
    of the union, which the packed all-reduce needs."""

    def __init__(self, grads: GradBuffer, n: int, ops=None):
        if grads.flat.numel() % n:
            raise ValueError("the gradient buffer is not a whole number of rows of n")
        self.grads = grads
        self.n = int(n)
        self.mat = grads.flat.view(-1, self.n)
        self.ops = ops if ops is not None else LibraryOps()
        self.last = {}

    def allreduce(self, group=None) -> GradBuffer:
        if not (dist.is_initialized() and dist.get_world_size(group) > 1):
            return self.grads
        flag = self.ops.touched(self.mat)
        dist.all_reduce(flag, op=dist.ReduceOp.MAX, group=group)
        idx, cnt = self.ops.compact(flag)
        k = int(cnt.item())
        if k:
            packed = self.ops.gather(self.mat, idx, cnt, k)
            dist.all_reduce(packed, op=dist.ReduceOp.SUM, group=group)
            self.ops.scatter(packed, self.mat, idx, cnt, k)
        self.last = {"columns": k, "bytes_exchanged": 4 * self.n + 4 * k * self.mat.shape[0],
                     "dense_bytes": 4 * self.mat.numel()}
        return self.grads
