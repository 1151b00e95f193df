"""GPU parity of the visibility-filtering pipeline of Sec. 3.4: rs_kmeans against the
oracle's Lloyd iterations, per-cluster lists against the FP64 importance, and rendering of
test views from their nearest cluster's list."""
import numpy as np
import pytest
import torch

import oracle
import oracle.kmeans as ok
from paper_2403_13806_gb300 import api, synth
from paper_2403_13806_gb300.visibility import VisibilityFilter, camera_centre

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_13806_gb300 import build
    build.build()
    oracle.build()


def near_ties(points, centres, rel=1e-5):
    """Points whose two nearest centres are within rel of each other (FP32 rounding decides)."""
    d = ((points[:, None, :].astype(np.float64) - centres[None].astype(np.float64)) ** 2).sum(-1)
    s = np.sort(d, axis=1)
    return (s[:, 1] - s[:, 0]) <= rel * np.maximum(s[:, 0], 1e-12)


@pytest.mark.parametrize("n,k,iters", [(64, 8, 50), (2000, 64, 30), (5, 5, 3), (300, 17, 0)])
def test_kmeans_matches_oracle(n, k, iters):
    rng = np.random.default_rng(n + k)
    if n == 64:
        _, cams, _ = synth.config3(n=10)
        pts = np.stack([camera_centre(c) for c in cams])
    else:
        pts = rng.normal(0, 3, (n, 3)).astype(np.float32)
    init = pts[rng.choice(n, k, replace=False)]
    c_o, a_o = ok.kmeans(pts, init, iters)
    c_g, a_g = api.kmeans(torch.as_tensor(pts, device="cuda"), torch.as_tensor(init, device="cuda"), iters)
    torch.cuda.synchronize()
    c_g, a_g = c_g.cpu().numpy(), a_g.cpu().numpy()
    # FP64 sums in another order: centres within 2 ulp; assignments equal off near-ties
    assert np.allclose(c_g, c_o, rtol=3e-7, atol=1e-7)
    tie = near_ties(pts, c_o)
    assert np.array_equal(a_g[~tie], a_o[~tie])
    assert tie.mean() < 0.01


def test_kmeans_rejects_bad_arguments():
    p = torch.zeros((4, 3), device="cuda")
    with pytest.raises(api.N.RadsplatError):
        api.kmeans(p, torch.zeros((300, 3), device="cuda"))    # k above 256


def test_visibility_filter_pipeline():
    """A 40k-Gaussian house-like scene, 16 cameras at 4 sites, k = 4 clusters."""
    rng = np.random.default_rng(11)
    scene, cams, site = synth.config3(n=40000, per_site=4)
    keep_sites = [0, 3, 4, 7]
    cams = [c for c, s in zip(cams, site) if s in keep_sites]
    cams = [dict(c, width=240, height=136, fx=225.0, fy=225.0, cx=120.0, cy=68.0) for c in cams]
    g = api.Gaussians.from_scene(scene)
    vf = VisibilityFilter(g, cams, k=4, t_cluster=0.001, extra_per_cluster=2, iterations=30, seed=1).build()
    assert len(vf.lists) == 4 and sum(len(c) for c in vf.cluster_cams) == 16 + 4 * 2
    # each cluster's list: {i : h_j(i) > t}, h_j the oracle's FP64 importance over the cluster's
    # views; mismatches only where |h - t| is within the importance tolerance (2e-4)
    for j in range(4):
        h_o, h_amb = oracle.importance(scene, vf.cluster_cams[j])
        got = np.zeros(scene.n, bool)
        got[vf.lists[j].cpu().numpy().view(np.uint32)] = True
        want = h_o > 0.001
        bad = got != want
        assert np.all(np.abs(h_o[bad] - 0.001) <= 2e-4 + np.maximum(h_amb[bad] - h_o[bad], 0)), j
        assert np.array_equal(np.sort(vf.lists[j].cpu().numpy().view(np.uint32)),
                              vf.lists[j].cpu().numpy().view(np.uint32))   # ascending
    # test views near the sites: nearest cluster = the oracle's nearest centre; the filtered
    # render differs from the full one only by what the dropped points contribute
    test = [dict(c) for c in cams[::3]]
    js = vf.cluster_of(test)
    assert np.array_equal(js, oracle.nearest(vf.centres.cpu().numpy(), np.stack([camera_centre(c) for c in test])))
    out = vf.render(test)
    full = api.Rasterizer().forward(g, api.ViewBatch(test, scene.n))
    a = out["image"].cpu().numpy()
    b = full["image"].cpu().numpy()
    assert np.mean(np.abs(a - b)) < 0.02
