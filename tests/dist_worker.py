"""Rank body of the two-process CPU test of the view-sharded reductions (gloo backend)."""
import os

import numpy as np
import torch
import torch.distributed as dist

import oracle
import oracle.grad as og
from paper_2403_13806_gb300 import dist as rd


def views_and_scene():
    from paper_2403_13806_gb300 import synth
    scene, (cam,) = synth.fd_crop()
    cams = []
    for k in range(5):
        vm = np.eye(3, 4, dtype=np.float32)
        vm[0, 3] = 0.15 * (k - 2)
        vm[1, 3] = 0.05 * k
        c = dict(cam)
        c["viewmat"] = vm
        cams.append(c)
    return scene, cams


def dL_for(cam, k):
    rng = np.random.default_rng(100 + k)
    return rng.normal(size=(3, cam["height"], cam["width"]))


def local_terms(scene, cams, views):
    """This rank's importance (FP64 max over its views, then float32 bits) and gradient
    (FP64 sum over its views, then float32)."""
    h = np.zeros(scene.n)
    g = [np.zeros(a.shape) for a in scene.arrays()]
    for k in views:
        hk, _ = oracle.importance(scene, [cams[k]])
        h = np.maximum(h, hk)
        gk = og.gradients(scene, cams[k], dL_for(cams[k], k))
        for i, name in enumerate(("means", "log_scales", "quats", "opacity_logit", "sh")):
            g[i] += gk[name]
    return h.astype(np.float32), [a.astype(np.float32) for a in g]


def run(rank, world, port, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        scene, cams = views_and_scene()
        a, b = rd.shard(len(cams), world, rank)
        h32, g32 = local_terms(scene, cams, range(a, b))
        h = torch.from_numpy(h32.view(np.int32).copy())
        gb = rd.GradBuffer([torch.from_numpy(x) for x in g32])
        for v, x in zip(gb.views, g32):
            v.copy_(torch.from_numpy(x))
        rd.allreduce_importance(h)
        rd.allreduce_grads(gb)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), h=h.numpy(), flat=gb.flat.numpy(),
                 local_h=h32, local_flat=np.concatenate([x.ravel() for x in g32]))
    finally:
        dist.destroy_process_group()


class TorchCpuOps:
    """The device steps of the sparse exchange restated with plain tensor indexing on the CPU
    (the library's kernels need a GPU; their own parity is tested there)."""

    def touched(self, mat):
        return (mat != 0).any(0).to(torch.float32)

    def compact(self, flag):
        idx = torch.nonzero(flag > 0.5).flatten().to(torch.int32)
        return idx, torch.tensor([idx.numel()], dtype=torch.int32)

    def gather(self, mat, idx, cnt, k):
        return mat[:, idx[:k].long()].contiguous()

    def scatter(self, packed, mat, idx, cnt, k):
        mat[:, idx[:k].long()] = packed


def sparse_grads(rank, n=1000, rows=59):
    """Seeded gradient rows with a few hundred touched columns per rank, overlapping."""
    rng = np.random.default_rng(500 + rank)
    g = np.zeros((rows, n), np.float32)
    cols = rng.choice(n, size=150, replace=False)
    g[:, cols] = rng.normal(size=(rows, len(cols))).astype(np.float32)
    g[rng.integers(0, rows, 40), cols[:40]] = 0.0    # touched columns with some zero rows
    return g


def run_sparse(rank, world, port, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        g = sparse_grads(rank)
        params = [torch.zeros(3, 1000), torch.zeros(3, 1000), torch.zeros(4, 1000), torch.zeros(1000),
                  torch.zeros(48, 1000)]
        dense = rd.GradBuffer(params)
        sparse = rd.GradBuffer(params)
        dense.flat.copy_(torch.from_numpy(g.ravel()))
        sparse.flat.copy_(torch.from_numpy(g.ravel()))
        rd.allreduce_grads(dense)
        ex = rd.SparseGradExchange(sparse, 1000, ops=TorchCpuOps())
        ex.allreduce()
        np.savez(os.path.join(out_dir, f"sparse{rank}.npz"), dense=dense.flat.numpy(), sparse=sparse.flat.numpy(),
                 columns=ex.last["columns"], sent=ex.last["bytes_exchanged"], full=ex.last["dense_bytes"])
    finally:
        dist.destroy_process_group()
