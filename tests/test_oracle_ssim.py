"""Pins of the oracle's SSIM loss: closed forms, invariants and finite differences."""
import numpy as np

import oracle.ssim as os_


def test_window_is_a_normalised_gaussian():
    w = os_.window()
    assert w.shape == (11, 11) and abs(w.sum() - 1) < 1e-15
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    # ratio of neighbouring taps of a Gaussian with sigma 1.5: exp(-(2k+1)/(2 sigma^2))
    assert abs(w[5, 6] / w[5, 5] - np.exp(-1 / 4.5)) < 1e-14
    assert abs(w[5, 8] / w[5, 7] - np.exp(-5 / 4.5)) < 1e-14


def test_identical_images_give_ssim_one_and_zero_gradient():
    rng = np.random.default_rng(0)
    x = rng.random((2, 20, 23))
    L, g = os_.loss_and_grad(x, x)
    assert abs(L) < 1e-14 and np.abs(g).max() < 1e-12


def test_constant_images_interior_closed_form():
    a, b = 0.3, 0.7
    x = np.full((31, 31), a)
    y = np.full((31, 31), b)
    s, _ = os_.ssim_map(x, y)
    # away from the zero padding: mu = the constants, all variances 0
    expect = (2 * a * b + os_.C1) / (a * a + b * b + os_.C1)
    assert abs(s[15, 15] - expect) < 1e-12   # sums of 121 FP64 terms
    # within 5 pixels of the border the zero padding lowers mu (not the closed form)
    assert abs(s[0, 0] - expect) > 1e-3


def test_delta_image_closed_form():
    x = np.zeros((21, 21))
    x[10, 10] = 1.0
    y = np.zeros((21, 21))
    s, _ = os_.ssim_map(x, y)
    w00 = os_.window()[5, 5]
    # at the delta: mu_x = w00, E[x^2] = w00, mu_y = E[y^2] = E[xy] = 0
    expect = (os_.C1 / (w00 ** 2 + os_.C1)) * (os_.C2 / (w00 - w00 ** 2 + os_.C2))
    assert abs(s[10, 10] - expect) < 1e-14


def test_ssim_is_symmetric():
    rng = np.random.default_rng(1)
    x, y = rng.random((2, 17, 19))
    assert np.allclose(os_.ssim_map(x, y)[0], os_.ssim_map(y, x)[0], rtol=0, atol=1e-14)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    x = rng.random((2, 14, 16))
    y = rng.random((2, 14, 16))
    L, g = os_.loss_and_grad(x, y)
    h = 1e-6
    for _ in range(40):
        i, r, c = rng.integers(0, 2), rng.integers(0, 14), rng.integers(0, 16)
        xp, xm = x.copy(), x.copy()
        xp[i, r, c] += h
        xm[i, r, c] -= h
        fd = (os_.loss_and_grad(xp, y)[0] - os_.loss_and_grad(xm, y)[0]) / (2 * h)
        assert abs(fd - g[i, r, c]) <= 1e-7 * max(1.0, abs(fd)) + 1e-10, (i, r, c, fd, g[i, r, c])


def test_lambda_zero_is_the_mean_squared_error():
    rng = np.random.default_rng(3)
    x, y = rng.random((2, 1, 9, 9))
    L, g = os_.loss_and_grad(x, y, lam=0.0)
    assert abs(L - np.mean((x - y) ** 2)) < 1e-15
    assert np.allclose(g, 2 * (x - y) / x.size, rtol=0, atol=1e-17)
