"""GPU parity of the optimisation step: rs_adam_step against the FP64 Adam oracle,
rs_gather_columns and the RS_PRUNE_KEEP filter bit-exact against the oracle's pruning, and
the Trainer's loop (loss decreases, pruning keeps exactly the points with h >= t, their
parameters and moments unchanged)."""
import numpy as np
import pytest
import torch

import oracle
import oracle.optim as oo
from paper_2403_13806_gb300 import api, synth
from paper_2403_13806_gb300 import _native as N

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_13806_gb300 import build
    build.build()
    oracle.build()


def test_adam_matches_fp64_oracle():
    rng = np.random.default_rng(0)
    sizes = [1, 3, 4, 4097, 100003]
    lrs = [1e-3, 5e-2, 1.6e-4, 2.5e-3, 1e-2]
    # one buffer per array, the last one offset by one float so it is not 16-byte aligned
    host = []
    dev = []
    for i, n in enumerate(sizes):
        arrs = [rng.normal(size=n).astype(np.float32) for _ in range(2)]   # p, then a gradient seed
        off = 1 if i == len(sizes) - 1 else 0
        bufs = [torch.zeros(n + off, device="cuda") for _ in range(4)]
        views = [b[off:] for b in bufs]
        views[0].copy_(torch.from_numpy(arrs[0]))
        host.append([arrs[0].astype(np.float64), np.zeros(n), np.zeros(n), np.zeros(n)])
        dev.append(views)
    for step in range(1, 6):
        groups = []
        for i, n in enumerate(sizes):
            g = rng.normal(size=n).astype(np.float32) * (10.0 ** rng.integers(-3, 2))
            dev[i][1].copy_(torch.from_numpy(g))
            p, m, v = oo.adam(host[i][0], g.astype(np.float64), host[i][1], host[i][2], lrs[i], step,
                              0.9, 0.999, 1e-15)
            mabs = 0.9 * host[i][3] + 0.1 * np.abs(g.astype(np.float64))   # scale of m's rounding
            host[i] = [p, m, v, mabs]
            groups.append((dev[i][0], dev[i][1], dev[i][2], dev[i][3], lrs[i]))
        api.adam_step(groups, step, (0.9, 0.999), 1e-15)
    torch.cuda.synchronize()
    for i, n in enumerate(sizes):
        p = dev[i][0].cpu().numpy().astype(np.float64)
        # FP32 against FP64 over five steps: parameters within a few ulps plus 1e-5 of the lr
        assert np.all(np.abs(p - host[i][0]) <= 1e-6 * np.abs(host[i][0]) + 1e-5 * lrs[i]), i
        m = dev[i][2].cpu().numpy().astype(np.float64)
        # m is a sum of terms of both signs: FP32 rounding is relative to the terms' magnitude
        assert np.all(np.abs(m - host[i][1]) <= 1e-6 * host[i][3]), i


def test_adam_rejects_bad_arguments():
    t = torch.zeros(4, device="cuda")
    with pytest.raises(N.RadsplatError):
        api.adam_step([(t, t.clone(), t.clone(), t.clone(), 1e-3)], 0)            # step must be >= 1
    with pytest.raises(N.RadsplatError):
        api.adam_step([(t, t.clone(), t.clone(), t.clone(), 1e-3)] * 9, 1)        # at most 8 groups


def test_prune_filter_and_gather_bit_exact():
    rng = np.random.default_rng(1)
    n = 300001
    h = (rng.random(n) * 0.03).astype(np.float32)
    h[::97] = np.float32(0.01)   # equality is kept
    keep = oo.survivors(h, 0.01)
    hd = torch.as_tensor(h, device="cuda")
    m, idx, cnt = api.filter(hd, 0.01, N.RS_PRUNE_KEEP)
    torch.cuda.synchronize()
    k = int(cnt.item())
    assert k == len(keep)
    assert np.array_equal(idx[:k].cpu().numpy().view(np.uint32), keep)
    mo, _ = oracle.filter_mask(h, 0.01, oracle.PRUNE_KEEP)
    assert np.array_equal(m.cpu().numpy(), mo)
    arrays = {"means": rng.normal(size=(3, n)).astype(np.float32), "sh": rng.normal(size=(48, n)).astype(np.float32),
              "opacity_logit": rng.normal(size=n).astype(np.float32)}
    _, expect = oo.prune(arrays, h, 0.01)
    pairs = []
    for name, a in arrays.items():
        src = torch.as_tensor(a, device="cuda")
        pairs.append((src, torch.full(a.shape[:-1] + (k,), np.nan, device="cuda")))
    api.gather_columns(pairs, idx, cnt, k)
    torch.cuda.synchronize()
    for (name, a), (_, dst) in zip(arrays.items(), pairs):
        assert np.array_equal(dst.cpu().numpy(), expect[name])


@pytest.mark.parametrize("loss", ["paper", "l1"])
def test_trainer_loss_decreases_and_pruning_keeps_h_at_least_t(loss):
    from paper_2403_13806_gb300.train import Trainer
    scene, (cam,) = synth.config0()
    cams = []
    for k in range(4):
        vm = np.eye(3, 4, dtype=np.float32)
        vm[0, 3] = 0.25 * (k - 1.5)
        c = dict(cam)
        c["viewmat"] = vm
        cams.append(c)
    target_scene = synth.perturbed_copy(scene, 7)
    tg = api.Gaussians.from_scene(target_scene)
    targets = []
    for c in cams:
        vb = api.ViewBatch([c], scene.n)
        targets.append(api.Rasterizer().forward(tg, vb)["image"].clone())
    g = api.Gaussians.from_scene(scene)
    tr = Trainer(g, cams, targets, prune_steps=(), t_prune=0.01, extent=3.0, seed=3, loss=loss)
    for _ in range(50):
        tr.step()
    before = [t.clone() for t in tr.g.tensors()] + [t.clone() for t in tr.m] + [t.clone() for t in tr.v]
    rec = tr.prune()
    torch.cuda.synchronize()
    h = tr.last_importance.view(torch.float32).cpu().numpy()
    keep = oo.survivors(h, 0.01)
    assert rec.n_before == scene.n and rec.n_after == len(keep) and 0 < len(keep) < scene.n
    after = list(tr.g.tensors()) + tr.m + tr.v
    for b, a in zip(before, after):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy()[..., keep.astype(np.int64)])
    # pruning at the paper's threshold removes only points that contribute little: the loss
    # right after it stays close to the loss before it
    for _ in range(70):
        tr.step()
    first, last = np.mean(tr.losses[:10]), np.mean(tr.losses[-10:])
    assert last < 0.9 * first, (first, last)
    assert all(np.isfinite(tr.losses))
