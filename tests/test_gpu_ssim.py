"""GPU parity of rs_ssim_loss (the loss of Sec. 3.2) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle.ssim as os_
from paper_2403_13806_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_13806_gb300 import build
    build.build()


def images(rng, planes, H, W):
    x = rng.random((planes, H, W)).astype(np.float32)
    # a related target: a smoothed, shifted, noisy copy (SSIM well inside (0, 1))
    y = 0.6 * x + 0.4 * np.roll(x, (1, 2), axis=(1, 2)) + 0.05 * rng.normal(size=x.shape)
    return x, np.clip(y, 0, 1).astype(np.float32)


@pytest.mark.parametrize("planes,H,W,lam", [(3, 45, 67, 0.2), (2, 16, 32, 0.2), (1, 7, 5, 0.2), (3, 45, 67, 0.0),
                                            (1, 40, 40, 1.0), (2, 48, 100, 0.2)])
def test_ssim_loss_matches_oracle(planes, H, W, lam):
    rng = np.random.default_rng(planes * 1000 + H + W)
    x, y = images(rng, planes, H, W)
    L_o, g_o = os_.loss_and_grad(x, y, lam)
    L, g = api.ssim_loss(torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda"), W, H, lam)
    torch.cuda.synchronize()
    L = float(L.item())
    g = g.cpu().numpy().astype(np.float64)
    # FP32 window sums of 121 terms per moment: ~1e-6 relative on SSIM, ~1e-6 of n on sums
    assert abs(L - L_o) <= 2e-6 * max(abs(L_o), 1e-3), (L, L_o)
    scale = np.abs(g_o).max()
    assert np.abs(g - g_o).max() <= 2e-4 * scale, (np.abs(g - g_o).max(), scale)
    assert np.linalg.norm(g - g_o) <= 2e-5 * np.linalg.norm(g_o)


def test_identical_images():
    rng = np.random.default_rng(7)
    x, _ = images(rng, 3, 33, 70)
    xd = torch.as_tensor(x, device="cuda")
    L, g = api.ssim_loss(xd, xd.clone(), 70, 33, 0.2)
    torch.cuda.synchronize()
    assert abs(float(L.item())) < 1e-6
    assert g.abs().max().item() < 1e-7


def test_full_view_size():
    """One 1280x832 RGB view (the benchmark resolution) against the oracle."""
    rng = np.random.default_rng(8)
    x, y = images(rng, 3, 832, 1280)
    L_o, g_o = os_.loss_and_grad(x, y, 0.2)
    L, g = api.ssim_loss(torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda"), 1280, 832, 0.2)
    torch.cuda.synchronize()
    assert abs(float(L.item()) - L_o) <= 2e-6 * abs(L_o)
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_o) <= 2e-5 * np.linalg.norm(g_o)


def test_rejects_bad_arguments():
    t = torch.zeros(12, device="cuda")
    with pytest.raises(ValueError):
        api.ssim_loss(t, t, 5, 2)             # not whole planes
    with pytest.raises(api.N.RadsplatError):
        api.ssim_loss(t, t, 3, 2, lam=1.5)    # lambda outside [0, 1]
