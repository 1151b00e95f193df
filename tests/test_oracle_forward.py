"""Pins of the FP64 oracle's forward path against closed forms, invariants and brute force.

Each test fixes a value the mathematics determines independently of the oracle's
code path, so that a dropped term, a wrong sign or index, or a transposed operand in
the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.grad as og
from paper_2403_13806_gb300 import synth

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


def one_scene(means, log_scales, quats, logits, sh, degree=0):
    return synth.Scene(np.asarray(means, np.float64).reshape(3, -1), np.asarray(log_scales, np.float64).reshape(3, -1),
                       np.asarray(quats, np.float64).reshape(4, -1), np.asarray(logits, np.float64).reshape(-1),
                       np.asarray(sh, np.float64).reshape((degree + 1) ** 2 * 3, -1), degree)


def cam_at_origin(W=64, H=64, f=50.0, cx=None, cy=None):
    return synth.camera(np.eye(3, 4), f, f, W / 2 if cx is None else cx, H / 2 if cy is None else cy, W, H)


def rgb_dc(c):
    """DC coefficient giving colour c (SH degree 0): 0.5 + Y00 k = c."""
    return (c - 0.5) / Y00


# ---------------------------------------------------------------- projection

@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_isotropic_on_axis_closed_form(oracle_lib, eps):
    """Sec. 3.2: Sigma' = J M Sigma M^T J^T; on the optical axis J M = diag(f/z, f/z, *)."""
    z, s, f = 4.0, 0.05, 50.0
    sc = one_scene([0, 0, z], [math.log(s)] * 3, [1, 0, 0, 0], [0.7], [rgb_dc(0.6)] * 3)
    cam = cam_at_origin(f=f)
    p = oracle.project(sc, cam, eps2d=eps)
    var = (f * s / z) ** 2 + eps
    assert p["valid"][0] == 1
    np.testing.assert_allclose(p["cov2d"][0], [var, 0.0, var], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(p["conic"][0], [1 / var, 0.0, 1 / var], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(p["xy"][0], [32.0, 32.0], rtol=0, atol=1e-12)
    o = 1.0 / (1.0 + math.exp(-0.7))
    assert p["opacity"][0] == pytest.approx(o, rel=1e-15)
    np.testing.assert_allclose(p["rgb"][0], [0.6] * 3, rtol=1e-14)
    # support half extent: alpha >= 1/255  <=>  r^2/var <= 2 ln(255 o)
    ext = math.sqrt(2 * math.log(255 * o) * var)
    np.testing.assert_allclose(p["ext"][0], [ext, ext], rtol=1e-13)


def test_isotropic_falloff_matches_gaussian(oracle_lib):
    """Centre pixel = min(0.99, o) c exactly; neighbours follow o c exp(-d^T Sigma'^-1 d / 2)."""
    z, s, f, eps = 3.0, 0.06, 50.0, 0.3
    for logit in (0.7, 6.0):     # o below and above the 0.99 clamp
        sc = one_scene([0, 0, z], [math.log(s)] * 3, [1, 0, 0, 0], [logit], [rgb_dc(0.8)] * 3)
        cam = cam_at_origin(f=f)
        p = oracle.project(sc, cam, eps2d=eps)
        r = oracle.render(p, mode="brute")
        img = r["image_chw"]
        o = 1 / (1 + math.exp(-logit))
        var = (f * s / z) ** 2 + eps
        assert img[0, 32, 32] == pytest.approx(min(0.99, o) * 0.8, rel=1e-14)
        for du, dv in [(1, 0), (2, 1), (0, 3), (-3, -2)]:
            a = min(0.99, o * math.exp(-0.5 * (du * du + dv * dv) / var))
            expect = a * 0.8 if a >= 1 / 255 else 0.0
            assert img[1, 32 + dv, 32 + du] == pytest.approx(expect, rel=1e-12, abs=1e-15)
        assert r["T_final"].reshape(64, 64)[32, 32] == pytest.approx(1 - min(0.99, o), rel=1e-13)


def test_offaxis_projection_and_world_transform(oracle_lib):
    """Isotropic Sigma: Sigma' = s^2 J J^T + eps I depends only on the camera-space position."""
    f, s, eps = 40.0, 0.1, 0.3
    xc, yc, zc = 0.4, -0.3, 2.5                      # camera-space position
    # a camera rotated 30 degrees about y and translated; place the point so that M p + m = (xc, yc, zc)
    th = math.radians(30)
    R = np.array([[math.cos(th), 0, -math.sin(th)], [0, 1, 0], [math.sin(th), 0, math.cos(th)]], np.float32)
    m = np.array([0.5, -0.2, 1.0], np.float32)
    vm = np.concatenate([R, m[:, None]], 1)
    pw = np.linalg.solve(R.astype(np.float64), np.array([xc, yc, zc]) - m.astype(np.float64))
    sc = one_scene(pw, [math.log(s)] * 3, [1, 0, 0, 0], [2.0], [rgb_dc(0.5)] * 3)
    cam = synth.camera(vm, f, f, 30.0, 20.0, 60, 40)
    p = oracle.project(sc, cam, eps2d=eps)
    J = np.array([[f / zc, 0, -f * xc / zc ** 2], [0, f / zc, -f * yc / zc ** 2]])
    S = s * s * J @ J.T + eps * np.eye(2)
    np.testing.assert_allclose(p["cov2d"][0], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-6)
    np.testing.assert_allclose(p["xy"][0], [f * xc / zc + 30.0, f * yc / zc + 20.0], rtol=1e-6)


def test_jacobian_clamp_applies_to_J_only(oracle_lib):
    """x/z beyond 1.3 * (W/2)/f is clamped inside J, not in the projected mean."""
    f, s, eps, W, H = 40.0, 0.1, 0.0, 60, 40
    xc, yc, zc = 3.0, 0.0, 2.0                        # x/z = 1.5 > 1.3*30/40 = 0.975
    sc = one_scene([xc, yc, zc], [math.log(s)] * 3, [1, 0, 0, 0], [2.0], [rgb_dc(0.5)] * 3)
    cam = synth.camera(np.eye(3, 4), f, f, 30.0, 20.0, W, H)
    p = oracle.project(sc, cam, eps2d=eps)
    lim = 1.3 * 30.0 / 40.0
    J = np.array([[f / zc, 0, -f * lim / zc], [0, f / zc, 0.0]])
    S = s * s * J @ J.T
    np.testing.assert_allclose(p["cov2d"][0], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-12, atol=1e-14)
    assert p["xy"][0][0] == pytest.approx(f * xc / zc + 30.0, rel=1e-14)


def test_quaternion_rotation_swaps_axes(oracle_lib):
    """q = identity gives Sigma = diag(s^2); 90 degrees about z swaps the x and y scales."""
    f, z, eps = 50.0, 4.0, 0.0
    s = np.array([0.02, 0.09, 0.05])
    cam = cam_at_origin(f=f)
    for q, expect in [((1, 0, 0, 0), (s[0], s[1])),
                      ((math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)), (s[1], s[0])),
                      ((3.0, 0, 0, 0), (s[0], s[1]))]:         # unnormalised identity
        sc = one_scene([0, 0, z], np.log(s), q, [1.0], [rgb_dc(0.5)] * 3)
        p = oracle.project(sc, cam, eps2d=eps)
        k = (f / z) ** 2
        np.testing.assert_allclose(p["cov2d"][0], [k * expect[0] ** 2, 0.0, k * expect[1] ** 2], rtol=1e-12, atol=1e-14)
    # 90 degrees about x maps the z scale onto image y
    sc = one_scene([0, 0, z], np.log(s), (math.cos(math.pi / 4), math.sin(math.pi / 4), 0, 0), [1.0], [rgb_dc(0.5)] * 3)
    p = oracle.project(sc, cam, eps2d=eps)
    np.testing.assert_allclose(p["cov2d"][0], [(f / z) ** 2 * s[0] ** 2, 0.0, (f / z) ** 2 * s[2] ** 2], rtol=1e-12, atol=1e-14)


def test_culling_rules(oracle_lib):
    """Near plane (FP32 depth <= 0.2), opacity below 1/255, non-finite input, zero quaternion."""
    means = np.array([[0, 0, 0.2], [0, 0, 0.21], [0, 0, 3.0], [0, 0, 3.0], [0, 0, 3.0], [0, 0, 3.0]]).T
    logits = [0.0, 0.0, -math.log(300.0), 0.0, 0.0, 0.0]    # o = 1/301 < 1/255
    quats = np.array([[1, 0, 0, 0]] * 6, float).T
    quats[:, 4] = 0.0
    ls = np.full((3, 6), -3.0)
    ls[0, 5] = np.nan
    sc = one_scene(means, ls, quats, logits, np.zeros((3, 6)))
    p = oracle.project(sc, cam_at_origin())
    assert list(p["valid"]) == [0, 1, 0, 1, 0, 0]


# ---------------------------------------------------------------- compositing

def proj_dict(xy, conic, opacity, rgb, depth, W=8, H=8):
    n = len(opacity)
    return {"xy": np.asarray(xy, float).reshape(n, 2), "conic": np.asarray(conic, float).reshape(n, 3),
            "opacity": np.asarray(opacity, float), "rgb": np.asarray(rgb, float).reshape(n, 3),
            "depth": np.asarray(depth, np.float32), "valid": np.ones(n, np.int32),
            "ext": np.full((n, 2), 100.0), "width": W, "height": H}


def test_two_coincident_gaussians_order_and_weights(oracle_lib):
    """Eq. (render-gs): c = c1 a1 + c2 a2 (1 - a1); importance (Eq. importance-score) = a1, a2(1-a1)."""
    a1, a2 = 0.6, 0.3
    # index 0 lies behind index 1: the front one is the one with the smaller depth
    p = proj_dict([[4, 4], [4, 4]], [[0.01, 0, 0.01]] * 2, [a2, a1], [[0, 0, 1], [1, 0, 0]], [5.0, 2.0])
    r = oracle.render(p, pixels=[[4, 4]], mode="brute")
    np.testing.assert_allclose(r["image"][0], [a1, 0.0, a2 * (1 - a1)], rtol=1e-15)
    assert r["T_final"][0] == pytest.approx((1 - a1) * (1 - a2), rel=1e-15)
    assert r["last_id"][0] == 0 and r["n_contrib"][0] == 2
    np.testing.assert_allclose(r["h"], [a2 * (1 - a1), a1], rtol=1e-15)


def test_depth_tie_goes_to_lower_index(oracle_lib):
    p = proj_dict([[4, 4], [4, 4]], [[0.01, 0, 0.01]] * 2, [0.5, 0.5], [[1, 0, 0], [0, 1, 0]], [3.0, 3.0])
    r = oracle.render(p, pixels=[[4, 4]], mode="brute")
    np.testing.assert_allclose(r["image"][0], [0.5, 0.25, 0.0], rtol=1e-15)
    assert r["last_id"][0] == 1


def test_stack_of_half_alpha_stops_after_13(oracle_lib):
    """T' = 0.5^14 < 1e-4 <= 0.5^13: compositing stops before entry 14."""
    n = 20
    p = proj_dict([[4, 4]] * n, [[0.01, 0, 0.01]] * n, [0.5] * n, [[1, 1, 1]] * n, np.arange(1, n + 1))
    r = oracle.render(p, pixels=[[4, 4]], mode="brute")
    assert r["n_contrib"][0] == 13
    assert r["T_final"][0] == 0.5 ** 13
    assert r["image"][0][0] == pytest.approx(1 - 0.5 ** 13, rel=1e-15)
    assert r["last_id"][0] == 12
    np.testing.assert_allclose(r["h"][:13], 0.5 ** np.arange(1, 14), rtol=1e-15)
    assert np.all(r["h"][13:] == 0.0)


def test_alpha_threshold_is_inclusive(oracle_lib):
    """alpha == 1/255 is composited, alpha just below is skipped; the 0.99 clamp applies."""
    p = proj_dict([[4, 4], [4, 4], [4, 4]], [[0.01, 0, 0.01]] * 3,
                  [1.0 / 255.0, (1.0 / 255.0) * (1 - 1e-12), 1.0], [[1, 0, 0], [0, 1, 0], [0, 0, 1]], [1.0, 2.0, 3.0])
    r = oracle.render(p, pixels=[[4, 4]], mode="brute", amb_rel=0.0)
    assert r["n_contrib"][0] == 2
    np.testing.assert_allclose(r["image"][0], [1 / 255, 0.0, 0.99 * (1 - 1 / 255)], rtol=1e-15)


def test_unit_colour_image_is_one_minus_T(oracle_lib):
    """Telescoping: sum_j a_j tau_j = 1 - T_final, and T_final >= 1e-4 by the stop rule."""
    scene, cams = synth.config0()
    scene.sh[:] = 0.0
    scene.sh[:3] = rgb_dc(1.0)
    p = oracle.project(scene, cams[0])
    r = oracle.render(p, mode="brute")
    np.testing.assert_allclose(r["image"][:, 0], 1.0 - r["T_final"], atol=1e-12)
    assert r["T_final"].min() >= 1e-4
    assert r["h"].max() <= 0.99


def test_bucketed_equals_brute(oracle_lib):
    for scene, cams in (synth.config0(), synth.fd_crop()):
        p = oracle.project(scene, cams[0])
        a = oracle.render(p, mode="brute")
        b = oracle.render(p, mode="bucketed")
        for k in ("image", "T_final", "last_id", "n_contrib", "ambiguous", "h", "h_amb"):
            assert np.array_equal(a[k], b[k]), k


def test_c_and_torch_restatements_agree(oracle_lib):
    """The differentiable FP64 restatement (grad.py) renders the same image as the C oracle."""
    scene, cams = synth.fd_crop()
    p = oracle.project(scene, cams[0])
    r = oracle.render(p, mode="brute", bg=(0.1, 0.2, 0.3))
    img, T = og.render_torch(scene, cams[0], bg=(0.1, 0.2, 0.3))
    np.testing.assert_allclose(r["image"], img, atol=1e-13)
    np.testing.assert_allclose(r["T_final"], T, atol=1e-13)


def test_importance_is_max_of_composited_contributions(oracle_lib):
    """Eq. (importance-score): h_i = max over pixels of a_i tau_i, from the restatement's weights."""
    import torch
    scene, cams = synth.fd_crop()
    cam = cams[0]
    p = oracle.project(scene, cam)
    r = oracle.render(p, mode="brute", amb_rel=0.0, alt_mean=False)
    _, order = og._fixed_decisions(scene, cam, 0.3, 0.2)
    with torch.no_grad():
        prm = og.params_of(scene, requires_grad=False)
        xy, conic, o, rgb = og.project_torch(prm, cam)
        vv, uu = np.meshgrid(np.arange(64), np.arange(64), indexing="ij")
        pix = np.stack([uu.ravel(), vv.ravel()], 1)
        # weights per (pixel, entry): recover them by rendering unit colour per Gaussian
        h = np.zeros(scene.n)
        for k, gid in enumerate(order):
            onehot = torch.zeros_like(rgb)
            onehot[gid, 0] = 1.0
            img, _ = og.composite_torch(xy, conic, o, onehot, torch.as_tensor(order), pix)
            h[gid] = img[:, 0].max().item()
    np.testing.assert_allclose(r["h"], h, rtol=1e-12, atol=1e-15)


def test_rect_is_superset_of_support(oracle_lib):
    """Every pixel with alpha >= 1/255 lies in a tile of the Gaussian's rect (all tile shapes)."""
    for scene, cams in (synth.config0(), synth.fd_crop()):
        cam = cams[0]
        W, H = cam["width"], cam["height"]
        vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        for tw, th in ((16, 16), (32, 8), (8, 8)):
            p = oracle.project(scene, cam, tile=(tw, th))
            for i in np.nonzero(p["valid"])[0]:
                a, b, c = p["conic"][i]
                dx, dy = uu - p["xy"][i, 0], vv - p["xy"][i, 1]
                power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
                on = p["opacity"][i] * np.exp(power) >= (1 / 255) * (1 + 1e-9)
                if not on.any():
                    continue
                x0, y0, x1, y1 = p["rect"][i]
                tx, ty = uu[on] // tw, vv[on] // th
                assert (tx >= x0).all() and (tx < x1).all() and (ty >= y0).all() and (ty < y1).all()


# ---------------------------------------------------------------- SH basis

def test_sh_orthonormal_by_quadrature(oracle_lib):
    """Gauss-Legendre in cos(theta) x uniform phi integrates Y_i Y_j to the identity."""
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phis = 2 * np.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            y = oracle.sh_basis(3, [st * math.cos(ph), st * math.sin(ph), ct])
            G += w * (2 * np.pi / nphi) * np.outer(y, y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_known_values_and_symmetries(oracle_lib):
    rng = np.random.default_rng(7)
    c1 = math.sqrt(3 / (4 * math.pi))
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        y = oracle.sh_basis(3, d)
        assert y[0] == pytest.approx(Y00, rel=1e-15)
        np.testing.assert_allclose(y[1:4], [-c1 * d[1], c1 * d[2], -c1 * d[0]], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(y[6], math.sqrt(5 / (16 * math.pi)) * (3 * d[2] ** 2 - 1), rtol=1e-12, atol=1e-14)
        for l in range(4):   # addition theorem
            assert np.sum(y[l * l:(l + 1) ** 2] ** 2) == pytest.approx((2 * l + 1) / (4 * math.pi), rel=1e-12)
        ym = oracle.sh_basis(3, -d)
        for l in range(4):   # parity
            np.testing.assert_allclose(ym[l * l:(l + 1) ** 2], (-1) ** l * y[l * l:(l + 1) ** 2], atol=1e-14)


def test_torch_sh_matches_c_sh(oracle_lib):
    import torch
    rng = np.random.default_rng(8)
    d = rng.normal(size=(3, 50))
    d /= np.linalg.norm(d, axis=0)
    yt = og.sh_basis(3, torch.tensor(d)).numpy()
    for k in range(50):
        np.testing.assert_allclose(yt[:, k], oracle.sh_basis(3, d[:, k]), atol=1e-14)


def test_degree0_colour_closed_form(oracle_lib):
    for k in (-3.0, -0.5, 0.0, 0.9):
        sc = one_scene([0, 0, 3.0], [-3.0] * 3, [1, 0, 0, 0], [0.0], [k, 2 * k, -k])
        p = oracle.project(sc, cam_at_origin())
        np.testing.assert_allclose(p["rgb"][0], np.maximum(0.0, 0.5 + Y00 * np.array([k, 2 * k, -k])), rtol=1e-15)


def test_rotated_anisotropic_falloff(oracle_lib):
    """Rotation by +30 degrees about z of diag(s1^2, s2^2): the off-diagonal of Sigma' and the
    sign of the cross term in the exponent are fixed by the closed form."""
    f, z, eps, th = 50.0, 3.0, 0.3, math.radians(30)
    s1, s2, s3 = 0.12, 0.03, 0.05
    q = (math.cos(th / 2), 0.0, 0.0, math.sin(th / 2))
    sc = one_scene([0, 0, z], np.log([s1, s2, s3]), q, [3.0], [rgb_dc(0.9)] * 3)
    cam = cam_at_origin(f=f)
    p = oracle.project(sc, cam, eps2d=eps)
    c, s = math.cos(th), math.sin(th)
    k = (f / z) ** 2
    S = k * np.array([[c * c * s1 ** 2 + s * s * s2 ** 2, c * s * (s1 ** 2 - s2 ** 2)],
                      [c * s * (s1 ** 2 - s2 ** 2), s * s * s1 ** 2 + c * c * s2 ** 2]]) + eps * np.eye(2)
    np.testing.assert_allclose(p["cov2d"][0], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-12)
    Si = np.linalg.inv(S)
    r = oracle.render(p, mode="brute")
    img = r["image_chw"]
    o = 1 / (1 + math.exp(-3.0))
    for du, dv in [(2, 1), (2, -1), (-2, 1), (3, 2), (1, -3)]:
        d = np.array([du, dv], float)
        a = min(0.99, o * math.exp(-0.5 * d @ Si @ d))
        expect = a * 0.9 if a >= 1 / 255 else 0.0
        assert img[2, 32 + dv, 32 + du] == pytest.approx(expect, rel=1e-12, abs=1e-15)
    assert img[0, 33, 34] != pytest.approx(img[0, 31, 34], rel=1e-3)     # the cross term matters


# ---------------------------------------------------------------- FP32 image mean (reading C5)

def _round_f32(q):
    """Exact rational q rounded to the nearest float32, ties to even (IEEE 754 default)."""
    from fractions import Fraction
    x = np.float32(float(q))
    cands = [x, np.nextafter(x, np.float32(np.inf)), np.nextafter(x, np.float32(-np.inf))]
    best = None
    for c in cands:
        d = abs(Fraction(float(c)) - q)
        if best is None or d < best[0] or (d == best[0] and (int(np.array(c).view(np.uint32)) & 1) == 0):
            best = (d, c)
    return best[1]


def _mean_f32_exact(p, vm, intr):
    """The FP32 mean by exact rational arithmetic with one explicit rounding per fma and per
    division (an fma rounds a*b + c once)."""
    from fractions import Fraction as F
    fma = lambda a, b, c: _round_f32(F(float(a)) * F(float(b)) + F(float(c)))
    t = [fma(vm[4 * r], p[0], fma(vm[4 * r + 1], p[1], fma(vm[4 * r + 2], p[2], vm[4 * r + 3]))) for r in range(3)]
    u = _round_f32(F(float(t[0])) / F(float(t[2])))
    v = _round_f32(F(float(t[1])) / F(float(t[2])))
    return fma(intr[0], u, intr[2]), fma(intr[1], v, intr[3])


def test_fp32_mean_exact_cases(oracle_lib):
    """Inputs whose every operation is exact: identity and axis-permutation views."""
    sc = one_scene([0.5, -0.25, 2.0], [0.0] * 3, [1, 0, 0, 0], [0.0], [0.0] * 3)
    cam = synth.camera(np.eye(3, 4), 64.0, 64.0, 32.0, 16.0, 64, 32)
    np.testing.assert_array_equal(oracle.mean2d_f32(sc, cam)[0], np.float32([48.0, 8.0]))
    # camera looking down -x: x_c = y, y_c = z, z_c = -x + 3
    vm = np.array([[0, 1, 0, 0], [0, 0, 1, 0], [-1, 0, 0, 3]], np.float64)
    sc = one_scene([1.0, 0.5, -1.0], [0.0] * 3, [1, 0, 0, 0], [0.0], [0.0] * 3)
    cam = synth.camera(vm, 100.0, 50.0, 10.0, 20.0, 64, 64)
    np.testing.assert_array_equal(oracle.mean2d_f32(sc, cam)[0], np.float32([100 * 0.25 + 10, 50 * -0.5 + 20]))


def test_fp32_mean_is_correctly_rounded_chain(oracle_lib):
    """Random poses and points: bit-equal to the same chain in exact rational arithmetic."""
    rng = np.random.default_rng(11)
    for trial in range(6):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        vm = np.concatenate([R, rng.normal(size=(3, 1)) + np.array([[0], [0], [6.0]])], 1).astype(np.float32)
        n = 40
        means = rng.normal(size=(3, n)).astype(np.float32)
        sc = synth.Scene(means.astype(np.float64), np.zeros((3, n)), np.tile([[1.0], [0], [0], [0]], n),
                         np.zeros(n), np.zeros((3, n)), 0)
        cam = synth.camera(vm.astype(np.float64), 1200.0, 1100.0, 640.0, 416.0, 1280, 832)
        got = oracle.mean2d_f32(sc, cam)
        vmf = np.asarray(cam["viewmat"], np.float32).reshape(12)
        intr = np.float32([cam["fx"], cam["fy"], cam["cx"], cam["cy"]])
        for i in range(n):
            ex = _mean_f32_exact(means[:, i], vmf, intr)
            assert got[i, 0] == ex[0] and got[i, 1] == ex[1], (trial, i)


# ---------------------------------------------------------------- ambiguity flags (reading C6)

def _one_gaussian_at(d, o, xy32_shift=0.0):
    """One isotropic Gaussian (conic = I) at (4, 4); the pixel (4 + d, 4) sees alpha = o e^(-d^2/2)."""
    p = proj_dict([[4.0, 4.0]], [[1.0, 0.0, 1.0]], [o], [[0.5, 0.25, 0.75]], [1.0], W=16, H=8)
    p["xy32"] = p["xy"] + np.array([[xy32_shift, 0.0]])
    return p


def _d_for_alpha(alpha, o):
    return math.sqrt(2.0 * math.log(o / alpha))


def test_flag_band_is_relative_1e5(oracle_lib):
    """A skip decision within a relative 1e-5 of 1/255 flags the pixel; 3e-5 away does not."""
    o = 0.8
    for rel, flagged in ((0.5e-5, 1), (-0.5e-5, 1), (3e-5, 0), (-3e-5, 0)):
        d = _d_for_alpha((1 + rel) / 255.0, o)
        p = _one_gaussian_at(d, o)
        p["xy"] = np.array([[8.0 - d, 4.0]])     # pixel (8, 4) at distance d
        p["xy32"] = p["xy"].copy()
        r = oracle.render(p, pixels=[[8, 4], [15, 0]], mode="brute")
        assert r["ambiguous"][0] == flagged, rel
        assert r["ambiguous"][1] == 0             # far away: alpha << 1/255
        if flagged:
            assert r["T_amb"][0] == 1.0 and r["c_amb"][0] == 0.75
        else:
            assert r["T_amb"][0] == 0.0 and r["c_amb"][0] == 0.0


def test_flag_where_the_fp32_mean_decides_otherwise(oracle_lib):
    """alpha is 1e-3 above 1/255 at the FP64 mean and below it at the FP32 one: flagged,
    although both lie far outside the 1e-5 band; with equal means it is not."""
    o = 0.8
    d = _d_for_alpha(1.001 / 255.0, o)
    x0 = 10.0 - d                         # pixel (10, 4) at distance d from the FP64 mean
    for shift, flagged in ((0.0, 0), (-2e-3 / d, 1)):
        p = _one_gaussian_at(d, o)
        p["xy"] = np.array([[x0, 4.0]])
        p["xy32"] = np.array([[x0 + shift, 4.0]])
        r = oracle.render(p, pixels=[[10, 4]], mode="brute")
        assert r["ambiguous"][0] == flagged
        assert r["n_contrib"][0] == 1     # the compositing follows the FP64 mean
        r2 = oracle.render(p, pixels=[[10, 4]], mode="brute", alt_mean=False)
        assert r2["ambiguous"][0] == 0


def test_flagged_pixel_bound_covers_both_outcomes(oracle_lib):
    """Behind the first flagged decision the image can change by at most T_amb * c_amb: the
    two outcomes of a flagged skip decision (compositing it or not) stay within it."""
    o = 0.8
    d = _d_for_alpha(1.000002 / 255.0, o)
    front = 0.4
    p = proj_dict([[4.0, 4.0], [10.0 - d, 4.0], [10.0, 4.0]], [[0.01, 0, 0.01], [1.0, 0, 1.0], [0.01, 0, 0.01]],
                  [front, o, 0.5], [[0.2, 0.2, 0.2], [0.9, 0.1, 0.3], [0.6, 0.7, 0.1]], [1.0, 2.0, 3.0], W=16, H=8)
    p["ext"][:] = 100.0
    r = oracle.render(p, pixels=[[10, 4]], mode="brute")
    assert r["ambiguous"][0] == 1
    T_front = 1.0 - front * math.exp(-0.5 * 0.01 * 36.0)
    assert r["T_amb"][0] == pytest.approx(T_front, rel=1e-14)
    assert r["c_amb"][0] == 0.9
    # the other outcome: the middle Gaussian skipped
    q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    q["opacity"][1] = 0.0
    q["valid"][1] = 0
    r_skip = oracle.render(q, pixels=[[10, 4]], mode="brute")
    assert np.abs(r_skip["image"][0] - r["image"][0]).max() <= r["T_amb"][0] * r["c_amb"][0]
