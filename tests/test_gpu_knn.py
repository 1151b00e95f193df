"""GPU parity of rs_nn_distance (the scale initialisation of Sec. 3.2) against the oracle's
nearest-neighbour distances: all pairs on small sets, the k-d tree on the 1M-point scene."""
import numpy as np
import pytest
import torch

import oracle.knn as ok
from paper_2403_13806_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_13806_gb300 import build
    build.build()


def gpu_nn(p):
    return api.nn_distance(torch.as_tensor(np.ascontiguousarray(p.T), device="cuda")).cpu().numpy()


@pytest.mark.parametrize("case", ["blob_shell", "lattice", "duplicates", "plane", "two", "line"])
def test_nn_distance_small(case):
    rng = np.random.default_rng(len(case))
    if case == "blob_shell":
        p = np.concatenate([rng.normal(0, 0.05, (3000, 3)), rng.uniform(-20, 20, (1000, 3))])
    elif case == "lattice":
        p = np.stack(np.meshgrid(*[np.arange(12)] * 3, indexing="ij"), -1).reshape(-1, 3) * 0.25 + 1.0
    elif case == "duplicates":
        p = rng.normal(size=(1500, 3))
        p[500:700] = p[:200]
    elif case == "plane":
        p = np.concatenate([rng.uniform(-1, 1, (2000, 2)), np.zeros((2000, 1))], 1)
    elif case == "two":
        p = np.array([[0, 0, 0], [3, 4, 12]], float)
    else:
        p = np.concatenate([np.linspace(0, 1, 777)[:, None], np.zeros((777, 2))], 1)
    p = p.astype(np.float32)
    d_o = ok.nn_distance_brute(p)
    d_g = gpu_nn(p)
    # FP32 distances of FP32 coordinates: relative 1e-6 of the coordinate scale
    scale = np.abs(p).max()
    assert np.all(np.abs(d_g - d_o) <= 2e-6 * np.maximum(d_o, 1e-3 * scale) + 1e-12), case
    if case == "duplicates":
        assert np.all(d_g[:200] == 0) and np.all(d_g[500:700] == 0)


def test_nn_distance_one_million_point_scene():
    """The headline scene's 1M means (dense object + sparse shell) against the k-d tree."""
    pytest.importorskip("scipy")
    scene, _ = synth.config2()
    p = scene.means.T.astype(np.float32)
    d_o = ok.nn_distance_tree(p)
    d_g = gpu_nn(p)
    assert np.all(np.abs(d_g - d_o) <= 2e-6 * np.maximum(d_o, 1e-4) + 1e-9)
    ls = api.init_log_scales(torch.as_tensor(scene.means, device="cuda")).cpu().numpy()
    assert np.allclose(ls, ok.init_log_scales(d_o), rtol=0, atol=1e-5)


def test_nn_distance_rejects_bad_arguments():
    with pytest.raises(api.N.RadsplatError):
        api.nn_distance(torch.zeros((3, 1), device="cuda"))
