"""View sharding and its two reductions (importance MAX, gradient SUM) across two gloo ranks on
the CPU, against the oracle's single-process results over all views."""
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2403_13806_gb300 import dist as rd


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def test_shard_partitions_views():
    for n in range(0, 13):
        for world in range(1, 6):
            spans = [rd.shard(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        rd.shard(4, 2, 2)


def test_grad_buffer_views_alias_flat():
    params = [torch.zeros(3, 5), torch.zeros(4, 5), torch.zeros(5), torch.zeros(48, 5)]
    gb = rd.GradBuffer(params)
    assert gb.flat.numel() == sum(p.numel() for p in params)
    for i, v in enumerate(gb.views):
        assert v.shape == params[i].shape
        v.fill_(i + 1)
    off = 0
    for i, p in enumerate(params):
        assert torch.all(gb.flat[off:off + p.numel()] == i + 1)
        off += p.numel()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_reductions_match_single_process(tmp_path):
    import dist_worker as w
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=w.run, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    # both ranks hold the same reduced values
    assert np.array_equal(res[0]["h"], res[1]["h"])
    assert np.array_equal(res[0]["flat"], res[1]["flat"])
    # importance: max over all views, the bits of float32 values (rounding is monotone, so
    # the max of the rounded per-rank maxima is the rounded global max)
    scene, cams = w.views_and_scene()
    h_all, _ = oracle.importance(scene, cams)
    assert np.array_equal(res[0]["h"].view(np.float32), h_all.astype(np.float32))
    assert h_all.max() > 0.1
    # gradient: the sum of the two ranks' partial sums, exactly as the two operands add
    expect = res[0]["local_flat"] + res[1]["local_flat"]
    assert np.array_equal(res[0]["flat"], expect)
    # and the FP64 single-process sum over all views, up to the float32 roundings
    import oracle.grad as og
    tot = None
    for k, cam in enumerate(cams):
        gk = og.gradients(scene, cam, w.dL_for(cam, k))
        flat = np.concatenate([gk[n].ravel() for n in ("means", "log_scales", "quats", "opacity_logit", "sh")])
        tot = flat if tot is None else tot + flat
    assert np.max(np.abs(res[0]["flat"] - tot)) <= 1e-6 * max(1.0, np.abs(tot).max())


def test_two_rank_sparse_gradient_exchange_equals_dense_sum(tmp_path):
    """The exchange over the union of touched columns gives the dense all-reduce SUM bit for
    bit, and moves the union's columns only."""
    import dist_worker as w
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=w.run_sparse, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = [np.load(tmp_path / f"sparse{r}.npz") for r in range(2)]
    for r in res:
        assert np.array_equal(r["dense"], r["sparse"])
    expect = w.sparse_grads(0).ravel() + w.sparse_grads(1).ravel()
    assert np.array_equal(res[0]["sparse"], expect)
    union = ((w.sparse_grads(0) != 0).any(0) | (w.sparse_grads(1) != 0).any(0)).sum()
    assert int(res[0]["columns"]) == int(union) and 150 < union < 300
    assert int(res[0]["sent"]) == 4 * 1000 + 4 * 59 * int(union) < int(res[0]["full"])
