"""The autotuner (rs_autotune): candidates measured, the fastest chosen and cached, and the
chosen tile shape and views per launch render the same images as the default batch."""
import numpy as np
import pytest
import torch

from paper_2403_13806_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_13806_gb300 import build
    build.build()


def three_views():
    scene, (cam,) = synth.config0()
    cams = []
    for k in range(3):
        vm = np.eye(3, 4, dtype=np.float32)
        vm[0, 3] = 0.2 * (k - 1)
        c = dict(cam)
        c["viewmat"] = vm
        cams.append(c)
    return scene, cams


def render_chunks(g, cams, tile, batch, subsets=None, smem_batch=0):
    imgs = []
    cfg = api.config(batch=smem_batch)
    for s0 in range(0, len(cams), batch):
        sub = subsets[s0:s0 + batch] if subsets is not None else None
        vb = api.ViewBatch(cams[s0:s0 + batch], g.n, subsets=sub, tile=tile)
        out = api.Rasterizer(cfg=cfg).forward(g, vb)
        imgs += [x.cpu().numpy() for x in api.split_images(out["image"], vb)]
    return imgs


def check_choice(r, n_views, front=True):
    n_batches = len(r["stage2"])
    assert len(r["stage1"]) == 9 and all(ms > 0 for ms in r["stage1"].values())
    # stage 3 (front lists offered) times the choice once more on whole lists
    assert r["n_candidates"] == 9 + n_batches + (1 if front else 0)
    # stage 1 picks the fastest tile shape and staging batch, stage 2 the fastest views per launch
    tw, th, m = min(r["stage1"], key=r["stage1"].get)
    assert r["tile"] == (tw, th) and r["smem_batch"] == m * api.blend_threads((tw, th))
    assert r["views_per_launch"] == min(r["stage2"], key=r["stage2"].get)
    best2 = min(r["stage2"].values())
    if r["front"]:   # front lists kept: stage 2's time
        assert front and r["ms_per_view"] == pytest.approx(best2, rel=1e-6)
    else:            # whole lists: not offered, or faster than stage 2's front-list time
        assert r["ms_per_view"] == pytest.approx(best2, rel=1e-6) if not front else r["ms_per_view"] < best2
    assert set(r["stage2"]) <= set([1, 2, 4, 8, 16, 32, 64, 128, n_views])


def test_autotune_measures_chooses_and_caches():
    scene, cams = three_views()
    g = api.Gaussians.from_scene(scene)
    api.N.lib().rs_autotune_clear()
    r = api.autotune(g, cams, backward=True)
    assert not r["cached"]
    check_choice(r, 3)
    assert sorted(r["stage2"]) == [1, 2, 3]
    again = api.autotune(g, cams, backward=True)
    assert again["cached"] and again["n_candidates"] == 0
    assert (again["tile"], again["smem_batch"], again["views_per_launch"]) == \
        (r["tile"], r["smem_batch"], r["views_per_launch"])
    # the forward-only workload is a different cache entry; forcing re-measures
    fwd = api.autotune(g, cams, backward=False)
    assert not fwd["cached"]
    forced = api.autotune(g, cams, backward=True, force=True)
    assert not forced["cached"] and forced["n_candidates"] == 13
    # whole lists only: no third stage, and a cache entry of its own
    whole = api.autotune(g, cams, backward=True, front=False)
    assert not whole["cached"] and not whole["front"]
    check_choice(whole, 3, front=False)
    # the choice renders the same images as one 16x16 batch of all views
    ref = render_chunks(g, cams, (16, 16), 3)
    got = render_chunks(g, cams, r["tile"], r["views_per_launch"], smem_batch=r["smem_batch"])
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_autotune_with_visibility_lists():
    scene, cams = three_views()
    g = api.Gaussians.from_scene(scene)
    rng = np.random.default_rng(5)
    subsets = [np.sort(rng.choice(scene.n, size=n, replace=False)).astype(np.uint32) for n in (500, 1200, 800)]
    r = api.autotune(g, cams, subsets=subsets, backward=True, force=True)
    check_choice(r, 3)
    ref = render_chunks(g, cams, (16, 16), 3, subsets)
    got = render_chunks(g, cams, r["tile"], r["views_per_launch"], subsets, smem_batch=r["smem_batch"])
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_autotune_rejects_bad_arguments():
    import ctypes
    scene, cams = three_views()
    g = api.Gaussians.from_scene(scene)
    with pytest.raises(ValueError):
        api.autotune(g, cams, subsets=[np.arange(10, dtype=np.uint32)] * 2)   # subsets != views
    # without visibility lists every view must list all Gaussians
    cam_arr = (api.N.RsCamera * 3)(*[api._camera_struct(c) for c in cams])
    n_items = np.array([5, 5, 5], dtype=np.int64)
    res = api.N.RsTuneResult()
    rc = api.N.lib().rs_autotune(api.N.ref(g.struct()), cam_arr, 3, n_items.ctypes.data_as(ctypes.c_void_p), None,
                                 api.N.ref(api.config()), 0, api.N.ref(res), None, None)
    assert rc == api.N.RS_ERR_INVALID_ARG
