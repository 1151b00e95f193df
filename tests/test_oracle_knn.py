"""Pins of the oracle's nearest-neighbour distances."""
import numpy as np
import pytest

import oracle.knn as ok


def test_lattice_spacing():
    a = 0.37
    g = np.stack(np.meshgrid(np.arange(6), np.arange(5), np.arange(4), indexing="ij"), -1).reshape(-1, 3) * a
    assert np.allclose(ok.nn_distance_brute(g), a, rtol=1e-13)


def test_two_points_and_duplicates():
    p = np.array([[0, 0, 0], [3, 4, 0]], float)
    assert np.allclose(ok.nn_distance_brute(p), [5, 5])
    q = np.array([[1, 2, 3], [1, 2, 3], [10, 0, 0]], float)
    d = ok.nn_distance_brute(q)
    assert d[0] == 0 and d[1] == 0 and abs(d[2] - np.linalg.norm([9, -2, -3])) < 1e-12
    ls = ok.init_log_scales(d)
    assert ls.shape == (3, 3) and np.all(np.isfinite(ls)) and ls[0, 0] == np.log(1e-7)


def test_tree_equals_brute_force():
    pytest.importorskip("scipy")
    rng = np.random.default_rng(0)
    p = np.concatenate([rng.normal(size=(1500, 3)), rng.uniform(-20, 20, (500, 3))]).astype(np.float32)
    assert np.allclose(ok.nn_distance_tree(p), ok.nn_distance_brute(p), rtol=1e-12, atol=0)


def test_far_point_sees_its_cluster():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.01, (100, 3))
    p[0] = [5, 0, 0]
    d = ok.nn_distance_brute(p)
    assert abs(d[0] - np.min(np.linalg.norm(p[1:] - p[0], axis=1))) < 1e-12 and d[0] > 4.9
