"""The device steps of the view-sharded gradient exchange (rs_touched_columns, the filter's
index list, rs_gather_columns, rs_scatter_columns) against plain indexing of the same seeded
sparse gradient matrix; the protocol itself runs on two gloo ranks in test_dist_cpu.py."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_touched_gather_scatter_roundtrip():
    from paper_2403_13806_gb300 import build
    build.build()
    from paper_2403_13806_gb300 import dist as rd
    rng = np.random.default_rng(61)
    rows, n = 59, 1_000_003
    g = np.zeros((rows, n), np.float32)
    cols = rng.choice(n, size=20_000, replace=False)
    g[:, cols] = rng.normal(size=(rows, len(cols))).astype(np.float32)
    g[rng.integers(0, rows, 5000), cols[:5000]] = 0.0
    g[:, cols[-3:]] = 0.0
    g[7, cols[-3:]] = -0.0                     # a column holding only a negative zero is not touched
    mat = torch.as_tensor(g, device="cuda")
    ops = rd.LibraryOps()
    flag = ops.touched(mat)
    want = (g != 0).any(0)
    assert np.array_equal(flag.cpu().numpy(), want.astype(np.float32))
    idx, cnt = ops.compact(flag)
    k = int(cnt.item())
    assert np.array_equal(idx[:k].cpu().numpy(), np.nonzero(want)[0].astype(np.int32))
    packed = ops.gather(mat, idx, cnt, k)
    assert np.array_equal(packed.cpu().numpy(), g[:, want])
    out = torch.zeros_like(mat)
    ops.scatter(packed * 2.0, out, idx, cnt, k)
    assert np.array_equal(out.cpu().numpy(), 2.0 * g)
    # one rank: the exchange leaves the gradients as they are
    params = [torch.zeros(3, n, device="cuda"), torch.zeros(3, n, device="cuda"), torch.zeros(4, n, device="cuda"),
              torch.zeros(n, device="cuda"), torch.zeros(48, n, device="cuda")]
    gb = rd.GradBuffer(params)
    gb.flat.copy_(mat.view(-1))
    rd.SparseGradExchange(gb, n).allreduce()
    assert torch.equal(gb.flat, mat.view(-1))
