"""Pins of the oracle's k-means against invariants and known partitions."""
import numpy as np

import oracle
import oracle.kmeans as ok


def test_assignment_equals_the_nearest_centre_oracle():
    oracle.build()
    rng = np.random.default_rng(0)
    p = rng.normal(size=(500, 3)).astype(np.float32)
    c = rng.normal(size=(7, 3)).astype(np.float32)
    c[3] = c[1]                       # duplicated centre: ties go to the lower index
    a = ok.assign(p, c)
    assert np.array_equal(a, oracle.nearest(c, p))
    assert not np.any(a == 3)


def test_separated_blobs_converge_to_their_means():
    rng = np.random.default_rng(1)
    truth = np.array([[0, 0, 0], [10, 0, 0], [0, 10, 0], [0, 0, 10]], np.float32)
    lab = rng.integers(0, 4, 400)
    p = (truth[lab] + rng.normal(0, 0.5, (400, 3))).astype(np.float32)
    init = (truth + np.float32(2.0)).astype(np.float32)
    c, a = ok.kmeans(p, init, 10)
    assert np.array_equal(a, lab)
    for j in range(4):
        assert np.allclose(c[j], p[lab == j].astype(np.float64).mean(0), rtol=0, atol=1e-6)


def test_fixed_point_invariants():
    rng = np.random.default_rng(2)
    p = rng.uniform(-5, 5, (300, 3)).astype(np.float32)
    c, a = ok.kmeans(p, p[:6], 50)
    # a Lloyd fixed point: every centre is the mean of its points, every point at its nearest centre
    for j in range(6):
        if np.any(a == j):
            assert np.allclose(c[j], p[a == j].astype(np.float64).mean(0), atol=1e-6)
    d = ((p[:, None, :].astype(np.float64) - c[None].astype(np.float64)) ** 2).sum(-1)
    assert np.all(d[np.arange(300), a] <= d.min(1) + 1e-5)


def test_empty_cluster_keeps_its_centre():
    p = np.array([[0, 0, 0], [1, 0, 0]], np.float32)
    init = np.array([[0.5, 0, 0], [100, 100, 100]], np.float32)
    c, a = ok.kmeans(p, init, 3)
    assert np.array_equal(c[1], init[1]) and np.array_equal(a, [0, 0])
    assert np.array_equal(c[0], np.array([0.5, 0, 0], np.float32))
