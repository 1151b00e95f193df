"""Pins of the oracle's Adam step and pruning compaction against closed forms."""
import numpy as np

import oracle
import oracle.optim as oo


def test_adam_first_step_is_lr_times_sign():
    # t = 1: m_hat = g and v_hat = g^2, so the step is lr g / (|g| + eps)
    rng = np.random.default_rng(0)
    g = rng.normal(size=100)
    p0 = rng.normal(size=100)
    p, m, v = oo.adam(p0, g, np.zeros(100), np.zeros(100), lr=0.01, step=1, eps=1e-15)
    assert np.allclose(p0 - p, 0.01 * g / (np.abs(g) + 1e-15), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g, rtol=1e-15) and np.allclose(v, 0.001 * g * g, rtol=1e-15)


def test_adam_constant_gradient_moves_lr_per_step():
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step (bias correction)
    g = np.array([0.5, -2.0, 1e-3])
    p = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 21):
        p, m, v = oo.adam(p, g, m, v, lr=0.1, step=t, eps=0.0)
    assert np.allclose(p, -20 * 0.1 * np.sign(g), rtol=1e-12)


def test_adam_two_steps_by_hand():
    b1, b2, eps, lr = 0.9, 0.999, 1e-8, 0.01
    g1, g2 = 0.3, -0.1
    m1 = (1 - b1) * g1
    v1 = (1 - b2) * g1 ** 2
    p1 = 1.0 - lr * (m1 / (1 - b1)) / (np.sqrt(v1 / (1 - b2)) + eps)
    m2 = b1 * m1 + (1 - b1) * g2
    v2 = b2 * v1 + (1 - b2) * g2 ** 2
    p2 = p1 - lr * (m2 / (1 - b1 ** 2)) / (np.sqrt(v2 / (1 - b2 ** 2)) + eps)
    p, m, v = oo.adam(np.array([1.0]), np.array([g1]), np.zeros(1), np.zeros(1), lr, 1, b1, b2, eps)
    p, m, v = oo.adam(p, np.array([g2]), m, v, lr, 2, b1, b2, eps)
    assert abs(p[0] - p2) < 1e-15 and abs(m[0] - m2) < 1e-16 and abs(v[0] - v2) < 1e-18


def test_adam_zero_gradient_and_zero_moments_leaves_parameters():
    p, m, v = oo.adam(np.ones(4), np.zeros(4), np.zeros(4), np.zeros(4), lr=1.0, step=3, eps=1e-15)
    assert np.array_equal(p, np.ones(4)) and not m.any() and not v.any()


def test_prune_keeps_complement_of_the_pruning_mask():
    oracle.build()
    rng = np.random.default_rng(1)
    h = rng.random(1000).astype(np.float32) * 0.02
    h[:5] = np.float32(0.01)           # equality: h == t is kept (the mask is h < t)
    keep = oo.survivors(h, 0.01)
    mask, pruned = oracle.filter_mask(h, 0.01, oracle.PRUNE_BELOW)
    assert np.array_equal(np.sort(np.concatenate([keep, pruned])), np.arange(1000, dtype=np.uint32))
    assert len(np.intersect1d(keep, pruned)) == 0
    assert set(range(5)) <= set(keep.tolist())
    mk, kept = oracle.filter_mask(h, 0.01, oracle.PRUNE_KEEP)
    assert np.array_equal(kept, keep) and np.array_equal(mk, 1 - mask)
    arrays = {"means": rng.normal(size=(3, 1000)), "opacity_logit": rng.normal(size=1000)}
    k2, out = oo.prune(arrays, h, 0.01)
    assert np.array_equal(k2, keep)
    for name, a in arrays.items():
        assert out[name].shape[-1] == len(keep)
        for j, i in enumerate(keep[:50]):
            assert np.array_equal(out[name][..., j], a[..., i])
