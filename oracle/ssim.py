"""FP64 statement of the training loss of Sec. 3.2 (TEST INFRASTRUCTURE ONLY).

The paper trains with L = (1 - lambda) ||I_f - I_phi||_2^2 + lambda SSIM(I_f, I_phi),
lambda = 0.2.  Readings: the squared norm is the mean over all values of (x - y)^2, and
the SSIM term is the structural dissimilarity 1 - SSIM (a loss that decreases as the
images agree).  SSIM (Wang, Bovik, Sheikh, Simoncelli 2004) per channel and pixel p, with
a normalised 11 x 11 Gaussian window w (sigma 1.5) centred on p over the zero-padded image:
  mu_x = sum w x, mu_y = sum w y, s_xx = sum w x^2 - mu_x^2, s_yy = sum w y^2 - mu_y^2,
  s_xy = sum w x y - mu_x mu_y,
  SSIM_p = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1), averaged over every pixel and channel.

Everything is direct sums over the 121 window offsets in numpy FP64 (no FFT, no library
convolution); the gradient with respect to the rendered image x follows from the chain rule
through (mu_x, E[x^2], E[xy]) at every pixel p whose window covers x(q):
  dSSIM_p/dx(q) = w(p - q) (a(p) + b(p) x(q) + c(p) y(q)),
  a = dS/dmu_x - 2 mu_x dS/ds_xx - mu_y dS/ds_xy,  b = 2 dS/ds_xx,  c = dS/ds_xy.
Pins: tests/test_oracle_ssim.py.
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
RADIUS = 5
SIGMA = 1.5
LAMBDA = 0.2


def window() -> np.ndarray:
    """Normalised 11 x 11 Gaussian window (outer product of the normalised 1D Gaussian)."""
    k = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-k * k / (2.0 * SIGMA * SIGMA))
    g /= g.sum()
    return np.outer(g, g)


def _filt(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum over offsets (dy, dx) of w[dy, dx] * img[y + dy - R, x + dx - R], zero outside."""
    H, W = img.shape
    R = RADIUS
    pad = np.zeros((H + 2 * R, W + 2 * R))
    pad[R:R + H, R:R + W] = img
    out = np.zeros((H, W))
    for dy in range(2 * R + 1):
        for dx in range(2 * R + 1):
            out += w[dy, dx] * pad[dy:dy + H, dx:dx + W]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray):
    """Per-pixel SSIM of two planes and the maps (a, b, c) of the gradient."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = window()
    mx, my = _filt(x, w), _filt(y, w)
    exx, eyy, exy = _filt(x * x, w), _filt(y * y, w), _filt(x * y, w)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    ln, ld = 2 * mx * my + C1, mx * mx + my * my + C1
    cn, cd = 2 * sxy + C2, sxx + syy + C2
    s = ln * cn / (ld * cd)
    d_mx = s * (2 * my / ln - 2 * mx / ld)
    d_sxx = -s / cd
    d_sxy = 2 * s / cn
    a = d_mx - 2 * mx * d_sxx - my * d_sxy
    b = 2 * d_sxx
    c = d_sxy
    return s, (a, b, c)


def loss_and_grad(x: np.ndarray, y: np.ndarray, lam: float = LAMBDA):
    """L = (1 - lam) mean((x - y)^2) + lam (1 - mean SSIM) over planes [P, H, W], and dL/dx."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    w = window()
    ssum = 0.0
    grad = np.empty_like(x)
    for i in range(x.shape[0]):
        s, (a, b, c) = ssim_map(x[i], y[i])
        ssum += s.sum()
        # the window is symmetric, so the transposed filter is the same filter
        gs = _filt(a, w) + x[i] * _filt(b, w) + y[i] * _filt(c, w)
        grad[i] = (1 - lam) * 2 * (x[i] - y[i]) / n - lam * gs / n
    loss = (1 - lam) * np.mean((x - y) ** 2) + lam * (1 - ssum / n)
    return loss, grad
