"""rs_bin_sort_front against rs_bin_sort on the same projected items: every tile list of the
front binning is the first part of the whole list, and the blend (image, T_final, last
composited entry), the importance and the backward come out the same on both.

The forward results and the importance are compared bit for bit.  The parameter gradients
are sums that the backward accumulates with floating-point atomics, whose order differs from
run to run even on identical lists (over a million Gaussians, the largest element difference
between two runs on the same lists varies tenfold from one pair of runs to the next); they are
compared per parameter group within 2^-12 of the group's largest magnitude element by element
and 2^-12 of its L2 norm, plus four times the largest difference among three runs of the
backward on whole lists (a single pair can understate that spread several times over).  Since the forward's `last` is bit-identical and lies inside every front list,
the backward reads the same entries on either lists, and nothing but the order of the
additions can differ.  Every other GPU
test that renders through api.Rasterizer runs on front lists (its default) and checks them
against the FP64 oracle, the backward element by element at full size."""
import numpy as np
import pytest
import torch

from gpu_helpers import u32
from paper_2403_13806_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_13806_gb300 import build
    build.build()


def both(scene, cams, tile=(16, 16), subsets=None):
    from paper_2403_13806_gb300 import api
    g = api.Gaussians.from_scene(scene)
    vb = api.ViewBatch(cams, scene.n, subsets=subsets, tile=tile)
    gen = torch.Generator(device="cuda").manual_seed(5)
    dL = torch.randn(3 * vb.n_pixels, generator=gen, device="cuda")
    res = {}
    for front in (False, True):
        rast = api.Rasterizer(front=front)
        h = torch.zeros(scene.n, dtype=torch.int32, device="cuda")
        out = rast.forward(g, vb, importance=h)
        runs = []
        for _ in range(1 if front else 3):   # whole lists: three runs, for the atomics' run-to-run noise
            grads = [torch.zeros_like(t) for t in g.tensors()]
            api.render_backward(g, vb, out["proj"], out["bins"], out["T_final"], out["last"], dL, grads,
                                rast.ws_bwd, rast.cfg)
            torch.cuda.synchronize()
            runs.append([t.cpu().numpy().astype(np.float64) for t in grads])
        res[front] = (out, h, runs)
    return vb, res


def check_grads_at_noise_level(whole_runs, front_grads):
    """Front-list gradients against the first whole-list run, at the level by which the
    whole-list runs differ among themselves (the atomics' order; the largest of the three
    pairs)."""
    (w1, w2, w3), f = whole_runs, front_grads
    for k, (a, b, b2, c) in enumerate(zip(w1, w2, w3, f)):
        amax, anorm = np.abs(a).max(initial=0), np.linalg.norm(a)
        pairs = ((a, b), (a, b2), (b, b2))
        noise_max = max(np.abs(x - y).max(initial=0) for x, y in pairs)
        noise_l2 = max(np.linalg.norm(x - y) for x, y in pairs)
        diff_max, diff_l2 = np.abs(a - c).max(initial=0), np.linalg.norm(a - c)
        print(f"group {k}: max |a| {amax:.3e} L2 {anorm:.3e}  run-to-run max {noise_max:.3e} "
              f"L2 {noise_l2:.3e}  front max {diff_max:.3e} L2 {diff_l2:.3e}")
        assert diff_max <= 2.0 ** -12 * amax + 4 * noise_max, (k, diff_max, noise_max, amax)
        assert diff_l2 <= 2.0 ** -12 * anorm + 4 * noise_l2, (k, diff_l2, noise_l2, anorm)


def check_same(vb, res):
    """Returns (whole-list instances, front-list instances)."""
    (wo, wh, wg), (fo, fh, fg) = res[False], res[True]
    assert torch.equal(wo["image"], fo["image"])
    assert torch.equal(wo["T_final"], fo["T_final"])
    assert torch.equal(wo["last"], fo["last"])
    assert torch.equal(wh, fh)
    check_grads_at_noise_level(wg, fg[0])
    # every front list is the first part of the whole list of its tile
    rw = wo["bins"].ranges.cpu().numpy().view(np.uint32).astype(np.int64)[:vb.n_tiles]
    rf = fo["bins"].ranges.cpu().numpy().view(np.uint32).astype(np.int64)[:vb.n_tiles]
    lw, lf = rw[:, 1] - rw[:, 0], rf[:, 1] - rf[:, 0]
    assert np.all(lf <= lw)
    Kw, Kf = int(wo["n_instances"]), int(fo["n_instances"])
    assert lw.sum() == Kw and lf.sum() == Kf
    vw, vf = u32(wo["bins"].vals[:max(Kw, 1)]), u32(fo["bins"].vals[:max(Kf, 1)])
    off = np.arange(Kf) - np.repeat(np.cumsum(lf) - lf, lf)
    tile_of = np.repeat(np.arange(vb.n_tiles), lf)
    assert np.array_equal(vf[rf[tile_of, 0] + off], vw[rw[tile_of, 0] + off])
    # the last composited entry of every pixel lies inside its tile's front list
    last = fo["last"].cpu().numpy().astype(np.int64)
    tw, th = vb.tile
    for v in range(vb.n_views):
        hv = vb.views_host[v]
        W, H = hv.width, hv.height
        vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        t = hv.tile_base + (vv // th) * hv.tiles_x + uu // tw
        assert np.all(last[hv.pixel_base: hv.pixel_base + W * H].reshape(H, W) <= lf[t])
    return Kw, Kf


def test_bench_batch_four_ring_views():
    """The benchmark's batch: 1M Gaussians, 4 ring views of 1280x832 in one launch per stage;
    the deep scene saturates every tile near its front, so the lists shrink many times."""
    scene, _ = synth.config2(n_views=1)
    vb, res = both(scene, synth.ring_cameras(4))
    Kw, Kf = check_same(vb, res)
    assert Kf < 0.1 * Kw, (Kw, Kf)


def test_over_65536_tiles_32_bit_super_keys():
    """8x8 tiles over 4 views of 1280x832 (66560 tiles): super-tile ids need 32-bit keys."""
    scene, _ = synth.config2(n_views=1)
    vb, res = both(scene, synth.ring_cameras(4), tile=(8, 8))
    assert vb.n_tiles > 65536
    Kw, Kf = check_same(vb, res)
    assert Kf < Kw


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 8)])
def test_config0_tile_shapes(tile):
    """20k Gaussians of the config-0 distribution in front of a 128x128 camera (at least 32
    items per tile for every shape, so the cut runs): some tiles saturate, the rest keep
    their whole lists."""
    scene, cams = synth.config0(n=20_000)
    vb, res = both(scene, cams, tile=tile)
    check_same(vb, res)


def test_sparse_batch_bins_whole_lists():
    """config 0 itself: 2k Gaussians over 64 tiles of 16x16, 31 items per tile, fewer than
    32: the call bins whole lists, as rs_bin_sort does."""
    scene, cams = synth.config0()
    vb, res = both(scene, cams)
    Kw, Kf = check_same(vb, res)
    assert Kf == Kw


def test_occluders_cut_every_list_short():
    """8k Gaussians of the config-0 distribution behind five large, nearly opaque Gaussians
    covering the image (alpha > 0.9 at every pixel): every tile saturates within the first
    few depth ranks, so each front list holds the occluders and at most a couple of other
    entries."""
    scene, cams = synth.config0(n=8000)
    scene.means[:, :5] = np.array([[0.0, 0.3, -0.3, 0.0, 0.0], [0.0, 0.0, 0.0, 0.3, -0.3], [1.0] * 5], np.float32)
    scene.log_scales[:, :5] = 1.0
    scene.opacity_logit[:5] = 6.0
    vb, res = both(scene, cams)
    Kw, Kf = check_same(vb, res)
    rf = res[True][0]["bins"].ranges.cpu().numpy().view(np.uint32).astype(np.int64)[:vb.n_tiles]
    assert (rf[:, 1] - rf[:, 0]).max() <= 8 and Kf < 0.2 * Kw, (Kw, Kf)


def test_transparent_scene_keeps_whole_lists():
    """Opacities just above 1/255 (8k Gaussians): no tile can saturate, so nothing is cut."""
    scene, cams = synth.config0(n=8000)
    scene.opacity_logit[:] = -5.0
    vb, res = both(scene, cams)
    Kw, Kf = check_same(vb, res)
    assert Kf == Kw


def test_uneven_views_with_subsets():
    """Views of different resolutions in one batch, each over its own subset of a 500k scene."""
    scene, _ = synth.config1(n_views=1)
    rng = np.random.default_rng(7)
    cams = [synth.ring_cameras(8, width=w, height=h, f=1200.0 * w / 1280)[k]
            for k, (w, h) in enumerate([(640, 480), (1280, 832), (333, 251)])]
    subsets = [np.sort(rng.choice(scene.n, size=m, replace=False)).astype(np.uint32)
               for m in (200_000, 400_000, 50_000)]
    vb, res = both(scene, cams, subsets=subsets)
    Kw, Kf = check_same(vb, res)
    assert Kf < Kw
