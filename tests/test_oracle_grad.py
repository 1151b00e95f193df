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
