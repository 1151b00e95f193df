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


def run_both(L, N, h, t, mode):
    dev = h.device
    n = h.numel()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # existing entry point with a caller workspace
    b = N.RsViewBatch()
    b.n_items = n
    ws = torch.empty(max(L.rs_workspace_size(N.RS_STAGE_FILTER, ctypes.byref(b), 0), 256), dtype=torch.uint8, device=dev)
    m1 = torch.full((n,), 7, dtype=torch.uint8, device=dev)
    i1 = torch.full((n,), -1, dtype=torch.int32, device=dev)
    c1 = torch.full((1,), -1, dtype=torch.int32, device=dev)
    assert L.rs_filter(_p(h), n, t, mode, _p(m1), _p(i1), _p(c1), _p(ws), ws.numel(), stream) == 0
    # the entry point that allocates nothing
    m2 = torch.full((n,), 9, dtype=torch.uint8, device=dev)
    i2 = torch.full((n,), -2, dtype=torch.int32, device=dev)
    c2 = torch.full((1,), -2, dtype=torch.int32, device=dev)
    assert L.rs_filter_noalloc(_p(h), n, t, mode, _p(m2), _p(i2), _p(c2), stream) == 0
    torch.cuda.synchronize()
    k = int(c1.item())
    assert int(c2.item()) == k
    assert torch.equal(m1, m2)
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
