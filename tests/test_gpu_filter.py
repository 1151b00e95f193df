"""GPU rs_filter / rs_filter_nearest against the oracle's mask, compaction and nearest
centre: bit-exact (the FP32 decisions are taken the same way on both sides)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_13806_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("n", [0, 1, 17, 4096, 3 * 4096 + 17, 1_000_003])
@pytest.mark.parametrize("mode", [0, 1])
def test_filter_bit_exact(n, mode):
    from paper_2403_13806_gb300 import api
    c = json.load(open(GOLDEN))
    t = c["t_prune_default_360"]["value"] if mode == 0 else c["t_cluster"]["value"]
    rng = np.random.default_rng(n + mode)
    h = (rng.random(n) ** 3 * 0.05).astype(np.float32)
    if n > 10:
        h[:5] = np.float32(t)                       # ties with the threshold
        h[5:8] = np.nextafter(np.float32(t), np.float32(1))
    m_o, idx_o = oracle.filter_mask(h, t, mode)
    m, idx, cnt = api.filter(torch.as_tensor(h, device="cuda"), t, mode)
    torch.cuda.synchronize()
    k = int(cnt.item())
    assert k == len(idx_o)
    if n:
        assert np.array_equal(m.cpu().numpy()[:n], m_o)
        assert np.array_equal(idx.cpu().numpy()[:k].view(np.uint32), idx_o)


def test_nearest_bit_exact():
    from paper_2403_13806_gb300 import api
    rng = np.random.default_rng(3)
    centres = rng.normal(size=(64, 3)).astype(np.float32)
    centres[10] = centres[3]                         # duplicate centre: ties go to 3
    cams = rng.normal(size=(5000, 3)).astype(np.float32)
    cams[:4] = centres[[3, 10, 0, 63]]
    out = api.nearest(torch.as_tensor(centres, device="cuda"), torch.as_tensor(cams, device="cuda"))
    torch.cuda.synchronize()
    ref = oracle.nearest(centres, cams)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert list(ref[:4]) == [3, 3, 0, 63]
