"""GPU parity of the forward hot path (rs_project, rs_bin_sort, rs_render, rs_importance)
against the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import IMG_TOL, check_view_against_oracle, gpu_forward, u32
from paper_2403_13806_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_13806_gb300 import build
    build.build()
    oracle.build()


def test_projection_matches_oracle():
    from paper_2403_13806_gb300 import api
    for scene, cams in (synth.config0(), synth.fd_crop(), synth.config1(n=4000, n_views=2, width=320, height=208)):
        for cam_i, cam in enumerate(cams):
            g = api.Gaussians.from_scene(scene)
            vb = api.ViewBatch([cam], scene.n)
            st = api.DeviceStatus()
            p = api.project(g, vb, status=st)
            torch.cuda.synchronize()
            o = oracle.project(scene, cam)
            valid = o["valid"].astype(bool)
            n_t = u32(p.n_tiles)
            # the FP32 order key is bit-exact
            assert np.array_equal(p.rgb_d[:, 3].cpu().numpy().view(np.uint32), o["depth"].view(np.uint32))
            vis = valid & (o["n_tiles"] > 0)
            assert np.all(n_t[~valid] == 0)
            xy = p.xy.cpu().numpy()
            co = p.conic_o.cpu().numpy()
            rgb = p.rgb_d[:, :3].cpu().numpy()
            # the image mean is the FP32 mirror's bit for bit (reading C5), close to the FP64 one
            assert np.array_equal(xy[vis], o["xy32"][vis])
            np.testing.assert_allclose(xy[vis], o["xy"][vis], rtol=1e-5, atol=2e-3)
            np.testing.assert_allclose(co[vis, 3], o["opacity"][vis], rtol=1e-5)
            np.testing.assert_allclose(rgb[vis], o["rgb"][vis], atol=2e-5)
            cscale = np.abs(o["conic"][vis]).max(1, keepdims=True)
            assert np.all(np.abs(co[vis, :3] - o["conic"][vis]) <= 2e-4 * cscale + 1e-7)
            # rects: contain the exact rect, inside a slightly widened one
            rect = p.rect.cpu().numpy().view(np.uint16).astype(np.int64)
            orect = o["rect"].astype(np.int64)
            assert np.all(rect[vis, 0] <= orect[vis, 0]) and np.all(rect[vis, 1] <= orect[vis, 1])
            assert np.all(rect[vis, 2] >= orect[vis, 2]) and np.all(rect[vis, 3] >= orect[vis, 3])
            W, H = cam["width"], cam["height"]
            ex = o["ext"] * (1 + 1e-3) + 1e-2
            u0 = np.clip(np.ceil(o["xy"][:, 0] - ex[:, 0]), 0, W - 1) // 16
            u1 = np.clip(np.floor(o["xy"][:, 0] + ex[:, 0]), 0, W - 1) // 16 + 1
            v0 = np.clip(np.ceil(o["xy"][:, 1] - ex[:, 1]), 0, H - 1) // 16
            v1 = np.clip(np.floor(o["xy"][:, 1] + ex[:, 1]), 0, H - 1) // 16 + 1
            g_on = n_t > 0
            assert np.all(rect[g_on, 0] >= u0[g_on]) and np.all(rect[g_on, 2] <= u1[g_on])
            assert np.all(rect[g_on, 1] >= v0[g_on]) and np.all(rect[g_on, 3] <= v1[g_on])
            assert np.all(n_t == (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1]))


def synthetic_projected(rng, views, m_per_view, span=5):
    """Seeded projected items (depth with ties, random rects up to span-1 tiles a side) for
    the integer stages."""
    depth, rect = [], []
    for (tx, ty), m in zip(views, m_per_view):
        d = rng.choice(np.array([0.5, 1.25, 2.0, 3.5, 9.0], np.float32), m)
        cont = rng.random(m) < 0.5
        d[cont] = rng.uniform(0.3, 50.0, int(cont.sum())).astype(np.float32)
        x0 = rng.integers(0, tx, m); y0 = rng.integers(0, ty, m)
        x1 = np.minimum(tx, x0 + rng.integers(0, span, m)); y1 = np.minimum(ty, y0 + rng.integers(0, span, m))
        depth.append(d.astype(np.float32))
        rect.append(np.stack([x0, y0, x1, y1], 1).astype(np.uint16))
    return np.concatenate(depth), np.concatenate(rect)


def check_ranges(ranges, ranges_o, K):
    """Tile ranges bit for bit, empty tiles included (reading C5: an empty tile's range is
    the empty one at the place its list would start)."""
    assert np.array_equal(ranges, ranges_o)
    assert ranges_o[-1, 1] == K


@pytest.mark.parametrize("views,m,span", [([(8, 8)], [5000], 5), ([(80, 52)], [60000], 5),
                                         ([(5, 3), (12, 9), (1, 1)], [700, 3000, 5], 5),
                                         ([(8, 8)], [200003], 5), ([(30, 21), (7, 9)], [90001, 40000], 12),
                                         ([(80, 52)] * 20, [3000] * 20, 5)])
def test_bin_sort_bit_exact(views, m, span):
    """Keys, values and ranges equal the oracle's stable sort of the duplicated keys, also
    where the per-super-tile lists span many 256-entry chunks with a ragged last chunk, and
    beyond 65536 tiles (32-bit super-tile keys, three sort passes whose digit widths the
    device narrows to the super-tiles present)."""
    from paper_2403_13806_gb300 import api, _native as N
    rng = np.random.default_rng(len(m) * 7 + m[0])
    depth, rect = synthetic_projected(rng, views, m, span)
    M = len(depth)
    item_view = np.repeat(np.arange(len(views)), m).astype(np.int32)
    tiles_x = np.array([v[0] for v in views], np.int32)
    tile_base = np.concatenate([[0], np.cumsum([a * b for a, b in views])[:-1]]).astype(np.int32)
    keys_o, vals_o = oracle.bin_sort(depth, rect, item_view, tiles_x, tile_base)
    n_tiles = int(sum(a * b for a, b in views))
    ranges_o = oracle.tile_ranges(keys_o, n_tiles)
    cams = [synth.camera(np.eye(3, 4), 100.0, 100.0, 0.0, 0.0, tx * 16, ty * 16) for tx, ty in views]
    vb = api.ViewBatch(cams, 0, subsets=[np.zeros(k, np.uint32) for k in m])
    proj = api.Projected.empty(M)
    proj.rgb_d[:, 3] = torch.as_tensor(depth, device="cuda")
    proj.rect.copy_(torch.as_tensor(rect.view(np.int16), device="cuda"))
    nt = (rect[:, 2].astype(np.int64) - rect[:, 0]) * (rect[:, 3].astype(np.int64) - rect[:, 1])
    proj.n_tiles.copy_(torch.as_tensor(nt.astype(np.int32), device="cuda"))
    for cap in (len(keys_o) + 17, len(keys_o)):
        bins = api.Bins.empty(cap, n_tiles, keys=True)
        st = api.DeviceStatus()
        api.bin_sort(proj, vb, bins, api.Workspace(), st)
        torch.cuda.synchronize()
        s = st.read()
        assert s["code"] == 0 and s["required"] == len(keys_o) and s["n_instances"] == len(keys_o)
        K = len(keys_o)
        assert np.array_equal(bins.keys[:K].cpu().numpy().view(np.uint64), keys_o)
        assert np.array_equal(u32(bins.vals[:K]), vals_o)
        check_ranges(bins.ranges.cpu().numpy().view(np.uint32), ranges_o, K)
    # capacity overflow is reported, nothing is written out of bounds
    bins = api.Bins.empty(len(keys_o) // 2, n_tiles)
    st = api.DeviceStatus()
    api.bin_sort(proj, vb, bins, api.Workspace(), st)
    torch.cuda.synchronize()
    s = st.read()
    assert s["code"] == N.RS_ERR_CAPACITY and s["required"] == len(keys_o) and s["n_instances"] == len(keys_o) // 2


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 8)])
def test_render_config0_matches_brute_oracle(tile):
    scene, cams = synth.config0()
    out = gpu_forward(scene, cams, tile=tile)
    err, namb, ro = check_view_against_oracle(out, scene, cams[0], 0, mode="brute")
    assert namb < 1e-4 * 128 * 128          # reading C6: flagged pixels below 1e-4 of the image


def test_images_identical_across_tile_shapes():
    scene, cams = synth.fd_crop()
    imgs = [gpu_forward(scene, cams, tile=t)["image"].cpu().numpy() for t in ((16, 16), (32, 8), (8, 8))]
    assert np.array_equal(imgs[0], imgs[1]) and np.array_equal(imgs[0], imgs[2])


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 8)])
def test_staging_batch_changes_nothing(tile):
    """rs_config.batch (records staged per blend batch) leaves image, T_final, last and
    importance bit-identical; values that are not 1, 2 or 4 per thread are rejected."""
    from paper_2403_13806_gb300 import api, _native as N
    scene, cams = synth.config1(n=20000, n_views=2, width=320, height=208)
    g = api.Gaussians.from_scene(scene)
    vb = api.ViewBatch(cams, scene.n, tile=tile)
    nt = api.blend_threads(tile)
    outs = []
    for m in (1, 2, 4):
        h = torch.zeros(scene.n, dtype=torch.int32, device="cuda")
        out = api.Rasterizer(cfg=api.config(batch=m * nt)).forward(g, vb, importance=h)
        torch.cuda.synchronize()
        outs.append([out["image"].cpu().numpy(), out["T_final"].cpu().numpy(), out["last"].cpu().numpy(),
                     h.cpu().numpy()])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)
    rast = api.Rasterizer()
    out = rast.forward(g, vb)
    with pytest.raises(N.RadsplatError) as e:
        api.render(out["proj"], out["bins"], vb, api.config(batch=3 * nt))
    assert e.value.code == N.RS_ERR_UNSUPPORTED


def check_importance(h_gpu, h, h_amb, min_strict=0.999):
    """h: max alpha*T over entries no near-threshold decision precedes; h_amb: over the
    others.  Flipping an alpha decision rescales later T by at most 1/(1 - 1/255), and a
    stop flip adds or removes the stopping entry (included in h_amb), so
    h - tol <= h_gpu <= max(h, FLIP h_amb) + tol; where FLIP h_amb <= h + tol the two
    bounds meet and the check is |h_gpu - h| <= tol."""
    flip = 1.0 + 1.0 / 254.0 + 1e-4
    upper = np.maximum(h, flip * h_amb)
    assert np.all(h_gpu >= h - IMG_TOL)
    assert np.all(h_gpu <= upper + IMG_TOL)
    strict = flip * h_amb <= h + IMG_TOL
    assert np.abs(h_gpu[strict] - h[strict]).max() <= IMG_TOL
    assert strict.mean() >= min_strict, strict.mean()
    assert h_gpu.max() <= 0.99
    return strict.mean()


def test_importance_matches_oracle():
    scene, cams = synth.config1(n=20000, n_views=4, width=320, height=208)
    out = gpu_forward(scene, cams)
    h_gpu = out["h"].view(torch.float32).cpu().numpy().astype(np.float64)
    h, h_amb = oracle.importance(scene, cams)
    check_importance(h_gpu, h, h_amb)


def test_importance_entry_point_equals_render_importance():
    """rs_importance (no image, T_final or last outputs) accumulates exactly the maxima the
    render with importance does, also on top of values already in h (Eq. importance-score
    over several calls)."""
    from paper_2403_13806_gb300 import api
    scene, cams = synth.config1(n=20000, n_views=3, width=320, height=208)
    out = gpu_forward(scene, cams)
    h_ref = out["h"]
    h = torch.zeros_like(h_ref)
    api.importance(out["proj"], out["bins"], out["vb"], h)
    torch.cuda.synchronize()
    assert torch.equal(h, h_ref)
    # accumulation: a second call over the same views changes nothing; seeded larger values stay
    seed = torch.where(torch.arange(h.numel(), device="cuda") % 7 == 0, torch.full_like(h, 0x3f700000), h)
    h2 = seed.clone()
    api.importance(out["proj"], out["bins"], out["vb"], h2)
    torch.cuda.synchronize()
    assert torch.equal(h2, torch.maximum(seed, h_ref))


def test_multiview_batch_with_subsets():
    scene, cams = synth.config1(n=20000, n_views=3, width=256, height=160)
    rng = np.random.default_rng(5)
    subsets = [np.sort(rng.choice(scene.n, size=k, replace=False)).astype(np.uint32) for k in (15000, 4000, 9000)]
    cams = [cams[0], dict(cams[1], width=200, height=120, cx=100.0, cy=60.0), cams[2]]
    out = gpu_forward(scene, cams, subsets=subsets, tile=(16, 16))
    for v in range(3):
        check_view_against_oracle(out, scene, cams[v], v, subset=subsets[v])
    # importance accumulated over the batch equals the max over views of the per-view oracle
    h_gpu = out["h"].view(torch.float32).cpu().numpy().astype(np.float64)
    h = np.zeros(scene.n)
    h_amb = np.zeros(scene.n)
    for v in range(3):
        hv, ha = oracle.importance(scene.subset(subsets[v].astype(np.int64)), [cams[v]])
        np.maximum.at(h, subsets[v].astype(np.int64), hv)
        np.maximum.at(h_amb, subsets[v].astype(np.int64), ha)
    check_importance(h_gpu, h, h_amb)


def test_empty_and_degenerate_inputs():
    """All Gaussians behind the camera: empty lists, background image, T = 1, last = 0."""
    from paper_2403_13806_gb300 import api
    scene, cams = synth.config0(n=300)
    scene.means[2] = -1.0
    out = gpu_forward(scene, cams)
    assert out["n_instances"] == 0
    assert torch.all(out["image"] == 0) and torch.all(out["T_final"] == 1) and torch.all(out["last"] == 0)
    assert torch.all(out["h"] == 0)
    # non-finite parameters are culled and counted
    scene, cams = synth.config0(n=300)
    scene.log_scales[0, :10] = np.nan
    g = api.Gaussians.from_scene(scene)
    vb = api.ViewBatch(cams, scene.n)
    st = api.DeviceStatus()
    p = api.project(g, vb, status=st)
    torch.cuda.synchronize()
    assert st.read()["nonfinite"] == 10
    assert np.all(u32(p.n_tiles)[:10] == 0)


def test_bin_sort_rejects_a_batch_with_too_few_tiles():
    """A hand-built batch whose n_tiles is below its views' tile count is reported through the
    device status (RS_ERR_INVALID_ARG) and binned to empty lists, not out of bounds."""
    from paper_2403_13806_gb300 import api, _native as N
    scene, cams = synth.config1(n=4000, n_views=2, width=320, height=208)
    g = api.Gaussians.from_scene(scene)
    vb = api.ViewBatch(cams, scene.n)
    proj = api.project(g, vb)
    real = vb.batch.n_tiles               # 2 views x 20 x 13 tiles (2 x 20 super-tiles)
    vb.batch.n_tiles = real // 4          # 130 tiles declared: enough for the super-tiles, not the tiles
    bins = api.Bins.empty(4 * vb.n_items + 65536, vb.batch.n_tiles)
    st = api.DeviceStatus()
    api.bin_sort(proj, vb, bins, api.Workspace(), st)
    torch.cuda.synchronize()
    s = st.read()
    assert s["code"] == N.RS_ERR_INVALID_ARG and s["n_instances"] == 0
    r = bins.ranges.cpu().numpy()
    assert np.all(r[:, 0] == r[:, 1])
    # the same projection with the true tile count bins normally
    vb.batch.n_tiles = real
    out = gpu_forward(scene, cams)
    assert out["n_instances"] > 0
