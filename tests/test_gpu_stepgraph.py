"""api.StepGraph: a captured step with host copies in and out gives the eager results, and
each replay reads the pinned host inputs as they are at that moment."""
import numpy as np
import pytest
import torch

from paper_2403_13806_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_13806_gb300 import build
    build.build()


def test_step_graph_matches_eager_and_rereads_inputs():
    scene, cams = synth.config0()
    host = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory() for a in scene.arrays()]
    dev = [torch.empty_like(t, device="cuda") for t in host]
    g = api.Gaussians(*dev, scene.sh_degree)
    vb = api.ViewBatch(cams, scene.n)
    rast = api.Rasterizer()
    for d, h in zip(dev, host):
        d.copy_(h)
    rast.forward(g, vb)   # sizes the instance capacity
    bins = rast.bins_for(vb)
    st = api.DeviceStatus()
    proj = api.Projected.empty(vb.n_items)
    img = torch.empty(3 * vb.n_pixels, device="cuda")
    out_h = torch.empty(3 * vb.n_pixels).pin_memory()

    def body():
        api.project(g, vb, rast.cfg, st, out=proj)
        api.bin_sort(proj, vb, bins, rast.ws_sort, st)
        api.render(proj, bins, vb, rast.cfg, image=img, T_final=False, last=False)

    sg = api.StepGraph(body, inputs=list(zip(host, dev)), outputs=[(img, out_h)])
    sg.run()
    eager = rast.forward(g, vb)["image"].cpu()
    assert torch.equal(out_h, eager)
    # change the host inputs: the next replay copies the new values in
    host[3].add_(1.0)   # opacity logits
    sg.run()
    for d, h in zip(dev, host):
        d.copy_(h)
    eager2 = rast.forward(g, vb)["image"].cpu()
    assert torch.equal(out_h, eager2) and not torch.equal(eager, eager2)


def test_step_graph_requires_pinned_memory():
    with pytest.raises(ValueError):
        api.StepGraph(lambda: None, inputs=[(torch.zeros(4), torch.zeros(4, device="cuda"))])


def test_step_graph_launch_with_copy_stream_pipeline():
    """Two graphs on two device buffer sets, their inputs copied on a side stream behind the
    other set's compute (the input pipeline of the end-to-end step): each replay renders the
    host inputs it was given."""
    scene, cams = synth.config0()
    hosts = []
    for k in range(3):
        hs = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory() for a in scene.arrays()]
        hs[3].add_(0.5 * k)
        hosts.append(hs)
    vb = api.ViewBatch(cams, scene.n)
    rast = api.Rasterizer()
    refs = []
    for hs in hosts:
        g = api.Gaussians(*[h.cuda() for h in hs], scene.sh_degree)
        refs.append(rast.forward(g, vb)["image"].cpu())
    bins = rast.bins_for(vb)
    st = api.DeviceStatus()
    proj = api.Projected.empty(vb.n_items)
    sets = []
    for _ in range(2):
        dev = [torch.empty_like(t, device="cuda") for t in hosts[0]]
        for d, h in zip(dev, hosts[0]):
            d.copy_(h)
        g = api.Gaussians(*dev, scene.sh_degree)
        img = torch.empty(3 * vb.n_pixels, device="cuda")
        out_h = torch.empty(3 * vb.n_pixels).pin_memory()

        def body(g=g, img=img):
            api.project(g, vb, rast.cfg, st, out=proj)
            api.bin_sort(proj, vb, bins, rast.ws_sort, st)
            api.render(proj, bins, vb, rast.cfg, image=img, T_final=False, last=False)

        sets.append((dev, api.StepGraph(body, outputs=[(img, out_h)]), out_h))
    cs = torch.cuda.Stream()
    comp = torch.cuda.current_stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]

    def copy_in(k):
        dev = sets[k % 2][0]
        with torch.cuda.stream(cs):
            cs.wait_event(used[k % 2])
            for d, h in zip(dev, hosts[k % 3]):
                d.copy_(h, non_blocking=True)
            copied[k % 2].record(cs)

    copy_in(0)
    for k in range(6):
        copy_in(k + 1)
        comp.wait_event(copied[k % 2])
        sets[k % 2][1].launch()
        used[k % 2].record(comp)
        comp.synchronize()
        assert torch.equal(sets[k % 2][2], refs[k % 3]), k
