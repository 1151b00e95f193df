"""Pins of the FP64 gradient oracle: central finite differences of the C forward and
the single-Gaussian closed form d(centre pixel)/d(opacity logit) = o (1 - o) c."""
import math

import numpy as np
import pytest

import oracle
import oracle.grad as og
from paper_2403_13806_gb300 import synth

KEYS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def loss_c(scene, cam, w):
    p = oracle.project(scene, cam)
    r = oracle.render(p, mode="brute")
    return float((r["image_chw"] * w).sum())


def test_autograd_matches_central_differences(oracle_lib):
    scene, cams = synth.fd_crop()
    cam = cams[0]
    scene = synth.Scene(*(a.astype(np.float64) for a in scene.arrays()), scene.sh_degree)
    rng = np.random.default_rng(11)
    w = rng.normal(size=(3, cam["height"], cam["width"]))
    G = og.gradients(scene, cam, w)
    checked = 0
    for key in KEYS:
        arr_all = dict(zip(KEYS, scene.arrays()))
        arr = arr_all[key]
        gmax = np.abs(G[key]).max()
        for _ in range(12):
            idx = tuple(int(rng.integers(0, s)) for s in arr.shape)
            x0 = arr[idx]
            h = 1e-6 * max(1.0, abs(x0))
            arr[idx] = x0 + h; lp = loss_c(scene, cam, w)
            arr[idx] = x0 - h; lm = loss_c(scene, cam, w)
            arr[idx] = x0; l0 = loss_c(scene, cam, w)
            fwd, bwd = (lp - l0) / h, (l0 - lm) / h
            if abs(fwd - bwd) > 1e-4 * max(1.0, abs(fwd)):
                continue           # the bracket crosses a skip/stop/clamp decision
            fd = (lp - lm) / (2 * h)
            assert G[key][idx] == pytest.approx(fd, rel=1e-6, abs=1e-7 * max(gmax, 1e-3)), (key, idx)
            checked += 1
    assert checked >= 50


def test_single_gaussian_logit_closed_form(oracle_lib):
    z, s, f = 3.0, 0.05, 50.0
    for logit in (-1.0, 0.5, 2.0):
        k = (0.7 - 0.5) * 2.0 * math.sqrt(math.pi)
        sc = synth.Scene(np.array([[0.0], [0.0], [z]]), np.full((3, 1), math.log(s)), np.array([[1.0], [0], [0], [0]]),
                         np.array([logit]), np.array([[k], [k], [k]]), 0)
        cam = synth.camera(np.eye(3, 4), f, f, 32.0, 32.0, 64, 64)
        w = np.zeros((3, 64, 64))
        w[1, 32, 32] = 1.0
        G = og.gradients(sc, cam, w)
        o = 1 / (1 + math.exp(-logit))
        assert G["opacity_logit"][0] == pytest.approx(o * (1 - o) * 0.7, rel=1e-12)
        assert G["g_opacity"][0] == pytest.approx(0.7, rel=1e-12)
        np.testing.assert_allclose(G["g_rgb"][0], [0.0, o, 0.0], rtol=1e-12, atol=1e-15)
        # the centre pixel sits at the maximum: no gradient to the mean
        np.testing.assert_allclose(G["means"][:, 0], 0.0, atol=1e-12)


def test_sampled_pixel_mode_equals_dense_mode(oracle_lib):
    """The sampled-pixel path (only Gaussians whose support box holds a listed pixel are
    projected and composited) gives the dense path's gradient for a dL/dimage that is zero
    off those pixels; the magnitude scales bound each gradient; a zero mean shift changes
    nothing."""
    scene, cams = synth.config1(n=3000, n_views=1, width=160, height=104)
    cam = cams[0]
    scene = synth.Scene(*(a.astype(np.float64) for a in scene.arrays()), scene.sh_degree)
    rng = np.random.default_rng(12)
    W, H = cam["width"], cam["height"]
    flat = np.unique(rng.integers(0, W * H, 40))
    pix = np.stack([flat % W, flat // W], 1)
    w = rng.normal(size=(len(pix), 3))
    dense = np.zeros((3, H, W))
    dense[:, pix[:, 1], pix[:, 0]] = w.T
    G = og.gradients(scene, cam, dense)
    S = og.gradients(scene, cam, w, pixels=pix, scales=True)
    Z = og.gradients(scene, cam, w, pixels=pix, mean_shift=np.zeros((scene.n, 2)))
    for k in KEYS + ("g_xy", "g_conic", "g_opacity", "g_rgb"):
        scale = max(np.abs(G[k]).max(), 1e-300)
        np.testing.assert_allclose(S[k], G[k], rtol=1e-10, atol=1e-12 * scale, err_msg=k)
        np.testing.assert_array_equal(Z[k], S[k], err_msg=k)
    pairs = [("g_xy", "scale_xy"), ("g_conic", "scale_conic"), ("g_opacity", "scale_opacity"), ("g_rgb", "scale_rgb")]
    pairs += [(k, "scale_" + k) for k in KEYS]
    for g, a in pairs:
        assert np.all(np.abs(S[g]) <= S[a] * (1 + 1e-10) + 1e-300), g
        assert np.all((S[a] == 0) <= (S[g] == 0)), g      # no scale where there is a gradient
    assert (np.abs(S["g_opacity"]) > 0).sum() > 10


def test_scales_of_a_lone_gaussian_are_the_gradient_magnitudes(oracle_lib):
    """One Gaussian, one pixel, weights of one sign: no term can cancel, so every
    image-space scale equals the gradient's magnitude (dC/da = c T with nothing behind)."""
    z, s, f = 3.0, 0.08, 50.0
    k = (0.7 - 0.5) * 2.0 * math.sqrt(math.pi)
    sc = synth.Scene(np.array([[0.1], [-0.05], [z]]), np.full((3, 1), math.log(s)),
                     np.array([[0.9], [0.1], [0.3], [0.2]]), np.array([0.3]), np.array([[k], [k], [k]]), 0)
    cam = synth.camera(np.eye(3, 4), f, f, 32.0, 32.0, 64, 64)
    for px in ([33, 32], [31, 33]):
        G = og.gradients(sc, cam, np.array([[1.0, 0.5, 0.25]]), pixels=np.array([px]), scales=True)
        for g, a in (("g_opacity", "scale_opacity"), ("g_rgb", "scale_rgb"), ("g_conic", "scale_conic")):
            np.testing.assert_allclose(G[a], np.abs(G[g]), rtol=1e-12, err_msg=g)
        # the mean: |a dx + b dy| <= |a dx| + |b dy|, equal when the two parts share a sign
        assert np.all(G["scale_xy"] >= np.abs(G["g_xy"]) * (1 - 1e-12))
        assert G["scale_opacity"][0] > 0


def test_mean_shift_moves_the_evaluation_point(oracle_lib):
    """A lone isotropic Gaussian on the optical axis (image mean (32, 32), conic I/var,
    colour 0.7): with its mean shifted by delta, the pixel (u, v) contributes
    dL/dx = (sum_ch w_ch) 0.7 o exp(-((u - 32 - delta)^2 + (v - 32)^2) / (2 var)) (u - 32 - delta) / var."""
    z, s, f, eps = 3.0, 0.08, 50.0, 0.3
    k = (0.7 - 0.5) * 2.0 * math.sqrt(math.pi)
    sc = synth.Scene(np.array([[0.0], [0.0], [z]]), np.full((3, 1), math.log(s)), np.array([[1.0], [0], [0], [0]]),
                     np.array([0.3]), np.array([[k], [k], [k]]), 0)
    cam = synth.camera(np.eye(3, 4), f, f, 32.0, 32.0, 64, 64)
    o = 1 / (1 + math.exp(-0.3))
    var = (f * s / z) ** 2 + eps
    pix = np.array([[33, 32]])
    w = np.array([[1.0, 0.5, -0.25]])
    for delta in (0.0, 0.3, -0.45):
        G = og.gradients(sc, cam, w, pixels=pix, mean_shift=np.array([[delta, 0.0]]))
        dx = 33 - 32 - delta
        expect = w.sum() * 0.7 * o * math.exp(-dx * dx / (2 * var)) * dx / var
        assert G["g_xy"][0, 0] == pytest.approx(expect, rel=1e-12)
        assert G["g_xy"][0, 1] == pytest.approx(0.0, abs=1e-15)
