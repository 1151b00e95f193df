"""rs_filter_noalloc: the pruning / visibility filter for callers that cannot allocate device
memory (hosts that own all device memory and forbid cudaMalloc after start-up).  Its scratch
lives in a fixed array inside the library; its results must equal those of rs_filter, which
takes a caller-allocated workspace.  Called through the C ABI directly.

This file is collected last on purpose, and must pass both alone in a fresh process and after
every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _opt(t):
    return None if t is None else _p(t)


def run_both(L, N, h, t, mode, with_mask=True, with_idx=True):
    dev = h.device
    n = h.numel()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # existing entry point with a caller workspace
    b = N.RsViewBatch()
    b.n_items = n
    ws = torch.empty(max(L.rs_workspace_size(N.RS_STAGE_FILTER, ctypes.byref(b), 0), 256), dtype=torch.uint8, device=dev)
    m1 = torch.full((max(n, 1),), 7, dtype=torch.uint8, device=dev) if with_mask else None
    i1 = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev) if with_idx else None
    c1 = torch.full((1,), -1, dtype=torch.int32, device=dev)
    hp = _p(h) if n > 0 else None
    assert L.rs_filter(hp, n, t, mode, _opt(m1), _opt(i1), _p(c1), _p(ws), ws.numel(), stream) == 0
    # the entry point that allocates nothing
    m2 = torch.full((max(n, 1),), 9, dtype=torch.uint8, device=dev) if with_mask else None
    i2 = torch.full((max(n, 1),), -2, dtype=torch.int32, device=dev) if with_idx else None
    c2 = torch.full((1,), -2, dtype=torch.int32, device=dev)
    assert L.rs_filter_noalloc(hp, n, t, mode, _opt(m2), _opt(i2), _p(c2), stream) == 0
    torch.cuda.synchronize()
    k = int(c1.item())
    assert int(c2.item()) == k
    if with_mask:
        assert torch.equal(m1[:n], m2[:n])
    if with_idx:
        assert torch.equal(i1[:k], i2[:k])
    return k


def test_noalloc_filter_matches_workspace_filter_twice():
    from paper_2403_13806_gb300 import build, _native as N
    build.build()
    L = N.lib()
    rng = np.random.default_rng(41)
    # call 1: a large prune (many blocks); call 2: a smaller keep-above, so any state left in
    # the shared scratch by call 1 would show up in call 2
    h1 = torch.as_tensor((rng.random(3_000_017) ** 3 * 0.05).astype(np.float32), device="cuda")
    k1 = run_both(L, N, h1, 0.01, N.RS_PRUNE_BELOW)
    h2 = torch.as_tensor((rng.random(70_001) * 0.004).astype(np.float32), device="cuda")
    k2 = run_both(L, N, h2, 0.001, N.RS_KEEP_ABOVE)
    assert 0 < k1 < h1.numel() and 0 < k2 < h2.numel()


def test_noalloc_filter_rejects_oversized_input():
    from paper_2403_13806_gb300 import build, _native as N
    build.build()
    L = N.lib()
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    # rejected on the host before anything is launched or dereferenced
    rc = L.rs_filter_noalloc(ctypes.c_void_p(16), N.RS_FILTER_NOALLOC_MAX_N + 1, 0.01, 0, None, None, _p(cnt), None)
    assert rc == N.RS_ERR_INVALID_ARG


def test_noalloc_filter_at_the_size_limit_and_degenerate_calls():
    """n = RS_FILTER_NOALLOC_MAX_N uses every word of the fixed array; n = 0, no mask, no index
    list and the survivors mode (RS_PRUNE_KEEP) give what rs_filter gives too."""
    from paper_2403_13806_gb300 import build, _native as N
    build.build()
    L = N.lib()
    g = torch.Generator(device="cuda").manual_seed(43)
    h = torch.rand(N.RS_FILTER_NOALLOC_MAX_N, device="cuda", generator=g) * 0.02
    k = run_both(L, N, h, 0.01, N.RS_PRUNE_KEEP)
    assert 0 < k < h.numel()
    del h
    empty = torch.zeros(0, device="cuda")
    assert run_both(L, N, empty, 0.01, N.RS_PRUNE_BELOW) == 0
    h = torch.rand(100_003, device="cuda", generator=g) * 0.02
    k1 = run_both(L, N, h, 0.01, N.RS_PRUNE_BELOW, with_mask=False)
    k2 = run_both(L, N, h, 0.01, N.RS_PRUNE_BELOW, with_idx=False)
    assert k1 == k2 and 0 < k1 < h.numel()
