"""Benchmark of the splatting hot path on GB300.

Workload: 1M Gaussians shaped as a 360-degree capture (dense central object plus
background shell, SH degree 3), views of 1280x832 on a ring around it.  One step is one
pass of the whole hot path over a batch of views, one launch per stage, replayed as a
CUDA graph: projection -> tile binning (keys + radix sort) -> blend with the importance
max -> L1 loss against a synthetic target -> backward (blend + projection) -> pruning
filter on the importance.  The metric is fwd+bwd milliseconds per view (lower is
better); the same views looped one at a time through plain launches ("plain") and the
forward-only FPS of one view are reported beside it.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload.
Under torchrun every rank renders its own views of the same Gaussians (weak scaling); the
step then ends with the two reductions over views: an all-reduce MAX of the importance and
an all-reduce SUM of the parameter gradients (NCCL), before the pruning filter.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FPS and fwd+bwd ms/view at 1M Gaussians, 1280×832; batched vs plain on one GB300"
N_GAUSSIANS = 1_000_000
FRONT_ALLOWED = True   # --lists front: the autotuner may choose front lists (rs_bin_sort_front)
FRONT = True           # the lists the step bins: the autotuner's choice, else FRONT_ALLOWED
WIDTH, HEIGHT = 1280, 832


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--views", type=int, default=4, help="views per rank per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--smem-batch", type=int, default=0,
                    help="with a fixed --tile: Gaussian records staged per blend batch (rs_config.batch, 0: default)")
    ap.add_argument("--no-legs", action="store_true", help="skip the filtered-rendering and importance legs")
    ap.add_argument("--uneven-views", type=int, default=256,
                    help="views of the uneven-batch leg (house-scale 3M scene, random resolutions, per-view "
                         "visibility lists); 0 skips it")
    ap.add_argument("--step-only", action="store_true",
                    help="time the step and stop (no per-stage pass, plain loop, end-to-end or optimiser "
                         "measurements): the command for profiling the step's launches")
    ap.add_argument("--loss", default="paper", choices=["paper", "l1"],
                    help="paper: (1 - 0.2) MSE + 0.2 (1 - SSIM) of Sec. 3.2; l1: mean absolute error")
    ap.add_argument("--tile", default="auto", help="tile shape WxH with all views in one launch, or 'auto' "
                                                   "(autotuner: tile shape, staging batch, views per launch)")
    ap.add_argument("--sample-pixels", type=int, default=0, help="reference arm: pixels per step (0: auto)")
    ap.add_argument("--lists", default="front", choices=["front", "whole"],
                    help="tile lists: the part in front of each tile's provable saturation depth "
                         "(rs_bin_sort_front) or whole (rs_bin_sort); the rendered results are the same")
    ap.add_argument("--probes", action="store_true", help="only run the peak probe kernels and print their rates")
    ap.add_argument("--cpu-report", action="store_true",
                    help="only time the FP64 C oracle on the host cores (config 0 full image, config 2 full view)")
    return ap.parse_args()


def make_loss(api, kind, width, height, dev):
    """The step's photometric loss: 'paper' = (1 - 0.2) MSE + 0.2 (1 - SSIM) (Sec. 3.2), or L1."""
    ws = api.Workspace(dev)

    def loss_fn(img, target, dL=None, loss=None):
        if kind == "paper":
            return api.ssim_loss(img, target, width, height, api.PAPER_LAMBDA, dL_dimage=dL, loss=loss, ws=ws)
        return api.l1_loss(img, target, dL, loss)
    return loss_fn


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(views, world, tile=(16, 16), per_launch=None, loss="paper"):
    return {"workload": "360-capture synthetic scene, 1M Gaussians SH3, 1280x832 ring views, "
                        "project+bin/sort+blend+importance+loss+backward+prune",
            "loss": "0.8 MSE + 0.2 (1 - SSIM)" if loss == "paper" else "L1",
            "gaussians": N_GAUSSIANS, "width": WIDTH, "height": HEIGHT, "views_per_step": views * world,
            "views_per_rank": views, "views_per_launch": per_launch or views, "sh_degree": 3,
            "tile": f"{tile[0]}x{tile[1]}", "seed": 2,
            "l2": "inputs larger than L2 (236 MB of parameters, ~0.5 GB of instances per view)"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 8:
                for nm, v in zip(names, r[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured", d
    return 6800.0, "fallback", {}


# ------------------------------------------------------------------ our arm

def run_ours(args):
    global FRONT
    import torch
    import torch.distributed as dist
    from paper_2403_13806_gb300 import api, synth, _native as N
    from paper_2403_13806_gb300 import dist as rd

    world, rank, local = dist_env()
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    V = args.views

    scene, _ = synth.config2(n=N_GAUSSIANS, n_views=1)
    all_cams = synth.ring_cameras(V * world, width=WIDTH, height=HEIGHT, f=1200.0)
    cams = all_cams[rank * V:(rank + 1) * V]
    g = api.Gaussians.from_scene(scene, device=dev)
    vb1 = [api.ViewBatch([c], scene.n, device=dev) for c in cams]
    cfg = api.config()
    loss_fn = make_loss(api, args.loss, WIDTH, HEIGHT, dev)

    # tile shape and views per launch from the autotuner (setup, untimed; cached per workload)
    if args.tile == "auto":
        tune = api.autotune(g, cams, cfg=cfg, backward=True, front=FRONT_ALLOWED)
        FRONT = tune["front"]
        tile, B = tune["tile"], tune["views_per_launch"]
        cfg = api.config(batch=tune["smem_batch"])
    else:
        tune = None
        tile, B = tuple(int(x) for x in args.tile.split("x")), V
        cfg = api.config(batch=args.smem_batch)
    vbs = [api.ViewBatch(cams[i:i + B], scene.n, tile=tile, device=dev) for i in range(0, V, B)]

    # synthetic targets: renders of a perturbed copy (setup, untimed)
    tscene = synth.perturbed_copy(scene, 12)
    tg = api.Gaussians.from_scene(tscene, device=dev)
    trast = api.Rasterizer(device=dev, front=FRONT)
    targets = [trast.forward(tg, vb)["image"].clone() for vb in vbs]
    del trast, tg

    # capacity from a first (plain) forward of every chunk
    rast = api.Rasterizer(device=dev, front=FRONT)
    K_max = 0
    for vb in vbs:
        rast.forward(g, vb)
        K_max = max(K_max, rast.status.read()["required"])
    del rast
    cap = int(K_max * 1.05) + 4096
    M = max(vb.n_items for vb in vbs)
    P = max(vb.n_pixels for vb in vbs)
    NTI = max(vb.n_tiles for vb in vbs)
    st = api.DeviceStatus(dev)
    proj = api.Projected.empty(M, dev)
    bins_all = api.Bins.empty(cap, NTI, device=dev)
    bins_of = [api.Bins(bins_all.vals, bins_all.ranges[:vb.n_tiles], None, cap) for vb in vbs]
    ws_sort, ws_bwd, ws_f = api.Workspace(dev), api.Workspace(dev), api.Workspace(dev)
    img_all = torch.empty(3 * P, device=dev)
    T_all = torch.empty(P, device=dev)
    L_all = torch.empty(P, dtype=torch.int32, device=dev)
    dL_all = torch.empty_like(img_all)
    bufs = [(img_all[:3 * vb.n_pixels], T_all[:vb.n_pixels], L_all[:vb.n_pixels], dL_all[:3 * vb.n_pixels])
            for vb in vbs]
    h = torch.zeros(scene.n, dtype=torch.int32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    gbuf = rd.GradBuffer(g.tensors())
    grads = gbuf.views
    mask = torch.empty(scene.n, dtype=torch.uint8, device=dev)
    idx = torch.empty(scene.n, dtype=torch.int32, device=dev)
    chunks = list(zip(vbs, bins_of, bufs, targets))
    cfg_w = overwrite_cfg(N, cfg)

    def prune():
        api.filter(h, 0.01, N.RS_PRUNE_BELOW, ws_f, mask=mask, idx=idx)

    # N = 1: the prune filter needs only the importance, complete after the last chunk's
    # render, so it runs on a side stream beside that chunk's loss and backward (the graph
    # captures the fork and the join)
    side = torch.cuda.Stream(device=dev)
    imp_done, prune_done = torch.cuda.Event(), torch.cuda.Event()

    def views_part(overlap_prune=False):
        h.zero_()
        for k, (vb, bins, (img, T, L, dL), target) in enumerate(chunks):
            api.project(g, vb, cfg, st, out=proj)
            api.bin_sort(proj, vb, bins, ws_sort, st, front=FRONT)
            api.render(proj, bins, vb, cfg, image=img, T_final=T, last=L, importance=h)
            if overlap_prune and k == len(chunks) - 1:
                imp_done.record()
                with torch.cuda.stream(side):
                    side.wait_event(imp_done)
                    prune()
                    prune_done.record(side)
            loss_fn(img, target, dL, loss)
            # the first launch writes the gradients, later ones add theirs
            api.render_backward(g, vb, proj, bins, T, L, dL, grads, ws_bwd, cfg_w if k == 0 else cfg)
        if overlap_prune:
            torch.cuda.current_stream().wait_event(prune_done)

    # N = 1: the whole step is one graph.  N > 1: the per-view part is the graph, then the
    # reductions over views (NCCL) and the filter on the reduced importance.
    def step_body():
        views_part(overlap_prune=(world == 1))

    # capture the batched step in a CUDA graph
    torch.cuda.synchronize()
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            step_body()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_body()
    torch.cuda.synchronize()

    exchange = rd.SparseGradExchange(gbuf, scene.n)

    def run_step():
        graph.replay()
        if world > 1:
            rd.allreduce_importance(h)
            exchange.allreduce()
            prune()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        run_step()
    st.zero_()
    barrier()
    with ClockSampler(local) as clk:
        # keep the GPU busy for ~1 s before the timed region so the clock sampler (100 ms
        # period) sees the clocks under this load; then time exactly `steps` replays
        t_end = time.perf_counter() + 1.0
        while time.perf_counter() < t_end:
            for _ in range(8):
                run_step()
            torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            run_step()
        e1.record()
        barrier()
    ms = e0.elapsed_time(e1)
    sres = st.read()
    if sres["code"] != 0:
        raise RuntimeError(f"device status {sres}")
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    views_total = V * world
    value = ms_per_step / views_total   # whole job: all ranks' views in the max-over-ranks step time

    if args.step_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 5), "unit": "ms/view (fwd+bwd)",
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": round(ms_per_step, 5), "higher_is_better": False, "step_only": True,
                              "config": dict(workload_config(V, world, tile, B, args.loss))}))
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # per-stage times of the same batched step (plain launches, events on this stream), and
    # the work counts of each launch (pairs walked, super-tile instances)
    stage_ms, kernel_ms, work_counts = stage_times(api, N, torch, g, chunks, cfg, st, proj, h, gbuf, loss, ws_sort,
                                                   ws_bwd, ws_f, mask, idx, reps=max(3, min(args.steps, 10)),
                                                   loss_fn=loss_fn)
    pairs, n_super, touched = work_counts["pairs"], work_counts["super_instances"], work_counts["touched"]

    # plain: the same views one at a time, no graph, the library's default configuration;
    # then the gain split: the autotuned configuration one view at a time, the autotuned
    # views per launch without the graph, and the graph (the value)
    plain = None
    fps = None
    gain = None
    if not args.no_plain:
        rp = max(3, min(args.steps, 10))
        plain, fps = plain_loop(api, N, torch, g, vb1, api.config(), torch.cat(targets), cams, reps=rp, dev=dev,
                                loss_fn=loss_fn)
        vb1t = [api.ViewBatch([c], scene.n, tile=tile, device=dev) for c in cams]
        plain_t, _ = plain_loop(api, N, torch, g, vb1t, cfg, torch.cat(targets), cams, reps=rp, dev=dev,
                                loss_fn=loss_fn)
        step_body()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(rp):
            step_body()
        e1.record()
        torch.cuda.synchronize()
        nograph = e0.elapsed_time(e1) / (rp * V)
        gain = {"plain_default_ms_per_view": round(plain, 5), "plain_autotuned_ms_per_view": round(plain_t, 5),
                "batched_no_graph_ms_per_view": round(nograph, 5), "batched_graph_ms_per_view": round(value, 5),
                "note": "every variant does the same work per step: project, bin/sort, blend with importance, loss "
                        "and backward per view, one prune filter per step"}

    # end to end through the public API: host parameters and targets in pinned memory
    e2e = e2e_run(api, N, torch, scene, vbs, cfg, targets, cap, reps=max(3, args.steps), dev=dev, world=world,
                  loss_fn=loss_fn)

    # roofline of the dominant kernel
    hbm, peak_kind, pk = peaks()
    optim = optimizer_bench(api, N, torch, g, gbuf, h, hbm, reps=10)
    uneven = uneven_bench(api, N, torch, dev, args.uneven_views, reps=2) if args.uneven_views > 0 else None
    filtered = filtered_bench(api, N, torch, dev, reps=5) if not args.no_legs else None
    imp_leg = importance_bench(api, N, torch, dev, reps=5) if not args.no_legs else None
    small = small_scene_bench(api, N, torch, dev, reps=50) if not args.no_legs else None
    work = kernel_work(vbs, sres, pairs, n_super, touched, work_counts["kept_items"], work_counts["touched_items"])
    probes = probe_peaks(N, torch, dev)
    roof = roofline(kernel_ms, work, hbm, peak_kind, B, probes)
    per_kernel = {k: kernel_frac(k, kernel_ms[k], work, hbm, probes) for k in kernel_ms if k in work}
    launches = int(round(sum(v["launches_per_step"] for v in kernel_ms.values()))) * args.steps

    if rank == 0:
        cpu = None if args.no_cpu else cpu_baseline(args)
        line = {
            "metric": METRIC, "value": round(value, 5), "unit": "ms/view (fwd+bwd)", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded 360-capture scene; target = render of a perturbed copy)",
            "config": dict(workload_config(V, world, tile, B, args.loss),
                           parallelism=(f"views sharded over {world} GPUs; all-reduce MAX of importance and SUM "
                                        f"of the gradient columns some rank touched per step" if world > 1
                                        else "1 GPU, no collective")),
            "gradient_exchange": exchange.last if world > 1 else None,
            "tile_lists": ("front: each tile's list up to the depth where its pixels provably stop "
                           "(rs_bin_sort_front; same results)" if FRONT else "whole (rs_bin_sort)"),
            "batched_ms_per_view": round(value, 5),
            "plain_ms_per_view": round(plain, 5) if plain else None,
            "batched_over_plain_speedup": round(plain / value, 3) if plain else None,
            "gain_split": gain,
            "fps_forward_single_view": round(fps, 1) if fps else None,
            "instances_per_view": int(sres["n_instances"] / B),
            "gaussians_with_gradient": touched,
            "items_with_gradient_per_launch": work_counts["touched_items"],
            "super_instances_per_view": int(n_super / V),
            "pairs_per_pixel": round(pairs / sum(vb.n_pixels for vb in vbs), 2),
            "tile_list_fraction_walked": round(work_counts["walked"] / max(1, sres["n_instances"] * len(vbs)), 4),
            "blends_per_s_forward": round(pairs / (kernel_ms["k_render_importance"]["ms_per_step"] / 1e3), 0)
            if "k_render_importance" in kernel_ms else None,
            "autotune": None if tune is None else {
                "tile": f"{tile[0]}x{tile[1]}", "smem_batch": tune["smem_batch"], "views_per_launch": B,
                "ms_per_view": round(tune["ms_per_view"], 5), "front_lists": tune["front"],
                "stage1_ms_per_view": {f"{a}x{b}/{m}": round(v, 5) for (a, b, m), v in tune["stage1"].items()},
                "stage2_ms_per_view": {str(k): round(v, 5) for k, v in tune["stage2"].items()}},
            "stage_ms_per_step": {k: round(v, 5) for k, v in stage_ms.items()},
            "kernel_ms_per_step": {k: round(v["ms_per_step"], 5) for k, v in
                                   sorted(kernel_ms.items(), key=lambda kv: -kv[1]["ms_per_step"])},
            "e2e": e2e, "roofline": roof, "roofline_per_kernel": per_kernel, "probes": probes, "optimizer": optim,
            "uneven_batch": uneven, "visibility_filtered_64_views": filtered, "importance_32_views": imp_leg,
            "config0_forward": small,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "gpu_launches": launches,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def stage_times(api, N, torch, g, chunks, cfg, st, proj, h, gbuf, loss, ws_sort, ws_bwd, ws_f, mask, idx, reps,
                loss_fn):
    """Per-stage times (CUDA events around each C-ABI call, summed over the launches of a
    step) and per-kernel times (the library's own launch events, rs_profile_*) of the same
    step with plain launches; then, in an untimed pass, the work counts: pairs walked by the
    backward (sum of `last` over pixels) and super-tile instances (4 x 4 tiles) of every
    launch."""
    names = ["project", "bin_sort", "render_importance", "loss", "backward", "filter"]
    acc = {k: 0.0 for k in names}
    kern = {}
    cfg_w = overwrite_cfg(N, cfg)
    for r in range(reps + 1):
        h.zero_()
        if r == 1:
            N.profile_enable(True)
        evs = []
        for k, (vb, bins, (img, T, L, dL), target) in enumerate(chunks):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            ev[0].record()
            api.project(g, vb, cfg, st, out=proj); ev[1].record()
            api.bin_sort(proj, vb, bins, ws_sort, st, front=FRONT); ev[2].record()
            api.render(proj, bins, vb, cfg, image=img, T_final=T, last=L, importance=h); ev[3].record()
            loss_fn(img, target, dL, loss); ev[4].record()
            api.render_backward(g, vb, proj, bins, T, L, dL, gbuf.views, ws_bwd, cfg_w if k == 0 else cfg)
            ev[5].record()
            evs.append(ev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        api.filter(h, 0.01, N.RS_PRUNE_BELOW, ws_f, mask=mask, idx=idx)
        f1.record()
        torch.cuda.synchronize()
        if r == 0:
            continue   # warm-up pass
        for ev in evs:
            for i, k in enumerate(names[:5]):
                acc[k] += ev[i].elapsed_time(ev[i + 1]) / reps
        acc["filter"] += f0.elapsed_time(f1) / reps
    for name, ms in N.profile_records():
        c = kern.setdefault(name, [0, 0.0])
        c[0] += 1
        c[1] += ms
    N.profile_enable(False)
    kernels = {k: {"launches_per_step": v[0] / reps, "ms_per_step": v[1] / reps, "ms_per_launch": v[1] / v[0]}
               for k, v in kern.items()}
    pairs, n_super, walked, kept_items = 0, 0, 0, 0
    for vb, bins, (img, T, L, dL), target in chunks:
        api.project(g, vb, cfg, st, out=proj)
        api.bin_sort(proj, vb, bins, ws_sort, st, front=FRONT)
        api.render(proj, bins, vb, cfg, image=img, T_final=T, last=L)
        pairs += int(L.to(torch.int64).sum().item())
        # entries a tile's blend reads: up to the largest `last` of its pixels
        tw, th = vb.tile
        for v in range(vb.n_views):
            hv = vb.views_host[v]
            Lv = L[hv.pixel_base: hv.pixel_base + hv.width * hv.height].view(hv.height, hv.width)
            Lp = torch.nn.functional.pad(Lv, (0, hv.tiles_x * tw - hv.width, 0, hv.tiles_y * th - hv.height))
            walked += int(Lp.view(hv.tiles_y, th, hv.tiles_x, tw).amax(dim=(1, 3)).to(torch.int64).sum().item())
        kept_items += int((proj.n_tiles[:vb.n_items] != 0).sum().item())
        if FRONT:
            # super instances the emission wrote: distinct (super-tile, item) pairs of the lists
            K = int(st.read()["n_instances"])
            rg = bins.ranges[:vb.n_tiles].to(torch.int64).view(-1, 2)
            t_of = torch.repeat_interleave(torch.arange(vb.n_tiles, device=rg.device), rg[:, 1] - rg[:, 0])
            sid = torch.zeros(vb.n_tiles, dtype=torch.int64, device=rg.device)
            for v in range(vb.n_views):
                hv = vb.views_host[v]
                loc = torch.arange(hv.tiles_x * hv.tiles_y, device=rg.device)
                sid[hv.tile_base: hv.tile_base + loc.numel()] = \
                    ((v * 4096 + (loc // hv.tiles_x) // 4) * 4096 + (loc % hv.tiles_x) // 4)
            items = bins.vals[:K].to(torch.int64) & 0xffffffff
            n_super += int(torch.unique(sid[t_of] * (1 << 32) + items).numel())
            del rg, t_of, sid, items
        else:
            r = proj.rect[:vb.n_items].to(torch.int64) & 0xffff
            nonempty = (r[:, 2] > r[:, 0]) & (r[:, 3] > r[:, 1])
            zero = torch.zeros_like(r[:, 0])
            sw = torch.where(nonempty, (r[:, 2] - 1) // 4 - r[:, 0] // 4 + 1, zero)
            sh = torch.where(nonempty, (r[:, 3] - 1) // 4 - r[:, 1] // 4 + 1, zero)
            n_super += int((sw * sh).sum().item())
            del r, nonempty, zero, sw, sh
    # Gaussians some view gives a gradient (the last timed step's gradients): only their
    # parameters are read by the projection backward
    gm = gbuf.views[0].reshape(3, -1)
    touched = int(((gm != 0).any(dim=0) | (gbuf.views[3].reshape(-1) != 0)).sum().item())
    # items the last launch's backward gave an image-space gradient (per launch: chunks alike)
    ga, gb, gc = api.image_grads(chunks[-1][0], ws_bwd)
    touched_items = int(((ga != 0).any(dim=1) | (gb != 0).any(dim=1) | (gc != 0)).sum().item())
    torch.cuda.synchronize()
    return acc, kernels, {"pairs": pairs, "super_instances": n_super, "touched": touched, "walked": walked,
                          "kept_items": kept_items, "touched_items": touched_items}


def uneven_bench(api, N, torch, dev, n_views, reps):
    """Uneven batch (config 4): views of random resolution (320-1920 x 240-1080) of the
    3M-Gaussian house-scale scene, each with its own ascending visibility list of 0.2M-2M
    Gaussians (the first n_views of the 256-view set).  fwd+bwd ms/view (L1 loss per view,
    gradients summed over views) with the autotuner's tile shape, staging batch and views per
    launch, processed in chunks of that many views, against a loop of plain single-view
    launches.  Each side reuses one Rasterizer (instance capacity grown to the largest
    chunk), so device memory stays bounded by one chunk.  Includes every stage of the step
    but the pruning filter."""
    from paper_2403_13806_gb300 import synth
    scene, _, _ = synth.config3()
    cams, subsets = synth.config4(scene, n_views=n_views)   # the first n_views of the 256-view set
    g = api.Gaussians.from_scene(scene, device=dev)
    grads = [torch.zeros_like(t) for t in g.tensors()]
    tune = api.autotune(g, cams[:32], subsets=subsets[:32], backward=True, front=FRONT_ALLOWED)
    B = tune["views_per_launch"]
    cfg = api.config(batch=tune["smem_batch"])

    def make(chunks, tile, cfg_, front):
        r = api.Rasterizer(cfg=cfg_, device=dev, front=front)
        vbs = [api.ViewBatch(cams[i:i + chunks], scene.n, subsets=subsets[i:i + chunks], tile=tile, device=dev)
               for i in range(0, len(cams), chunks)]
        for vb in vbs:
            r.forward(g, vb)   # grows the capacity to the largest chunk
        return r, vbs

    def run(plan):
        r, vbs = plan
        for vb in vbs:
            o = r.forward(g, vb)
            loss, dl = api.l1_loss(o["image"], torch.zeros_like(o["image"]))
            api.render_backward(g, vb, o["proj"], o["bins"], o["T_final"], o["last"], dl, grads, r.ws_bwd, r.cfg)

    def timed(plan):
        run(plan)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run(plan)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / (reps * len(cams))

    plan = make(B, tune["tile"], cfg, tune["front"])
    batched = timed(plan)
    del plan
    plan = make(1, (16, 16), api.config(), FRONT_ALLOWED)
    plain = timed(plan)
    del plan
    torch.cuda.empty_cache()
    return {"views": len(cams), "pixels": int(sum(c["width"] * c["height"] for c in cams)),
            "items": int(sum(len(s) for s in subsets)), "tile": f"{tune['tile'][0]}x{tune['tile'][1]}",
            "smem_batch": tune["smem_batch"], "views_per_launch": B, "front_lists": tune["front"],
            "batched_ms_per_view": round(batched, 4), "plain_ms_per_view": round(plain, 4),
            "batched_over_plain_speedup": round(plain / batched, 3),
            "note": "autotuned on the first 32 views; Rasterizer calls (one host read of the instance count per "
                    "launch) on both sides"}


def _graph_of(torch, body):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        body()
        body()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr):
        body()
    torch.cuda.synchronize()
    return gr


def _replay_ms(torch, gr, reps):
    gr.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        gr.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _forward_plan(api, torch, g, vb, cfg, dev, importance=None, image=True):
    """Buffers and a body for one forward (project -> bin_sort -> render) of a batch with the
    instance capacity sized by a first render."""
    r = api.Rasterizer(cfg=cfg, device=dev, front=FRONT)
    r.forward(g, vb)
    cap = int(r.status.read()["required"] * 1.02) + 4096
    st = api.DeviceStatus(dev)
    proj = api.Projected.empty(vb.n_items, dev)
    bins = api.Bins.empty(cap, vb.n_tiles, device=dev)
    ws = api.Workspace(dev)
    img = torch.empty(3 * vb.n_pixels, device=dev) if image else False
    T = torch.empty(vb.n_pixels, device=dev) if image else False
    L = torch.empty(vb.n_pixels, dtype=torch.int32, device=dev) if image else False
    del r

    def body():
        api.project(g, vb, cfg, st, out=proj)
        api.bin_sort(proj, vb, bins, ws, st, front=FRONT)
        api.render(proj, bins, vb, cfg, image=img, T_final=T, last=L, importance=importance)

    return body, st, cap


def filtered_bench(api, N, torch, dev, reps):
    """Visibility-filtered rendering (config 3, Sec. 3.4): the 3M-Gaussian house-scale scene,
    64 views of 960x544 at 8 camera clusters.  Setup (untimed): per cluster, the importance of
    Eq. importance-score-vis over the cluster's views and its list h > 0.005.  Timed: the
    forward of all 64 views in one launch per stage, replayed as a CUDA graph, once with every
    view on its cluster's list and once on all 3M Gaussians; FPS = views / time."""
    from paper_2403_13806_gb300 import synth
    scene, cams, site = synth.config3()
    g = api.Gaussians.from_scene(scene, device=dev)
    cfg = api.config()
    lists = {}
    rast = api.Rasterizer(device=dev, front=FRONT)
    for s in range(int(site.max()) + 1):
        vb = api.ViewBatch([c for c, k in zip(cams, site) if k == s], scene.n, device=dev)
        h = torch.zeros(scene.n, dtype=torch.int32, device=dev)
        rast.forward(g, vb, importance=h, image=False)
        m, idx, cnt = api.filter(h, 0.005, N.RS_KEEP_ABOVE)
        lists[s] = idx[:int(cnt.item())].clone()
    del rast
    out = {"views": len(cams), "width": 960, "height": 544, "gaussians": scene.n, "t_cluster": 0.005,
           "mean_list_fraction": round(float(np.mean([lists[int(k)].numel() for k in site])) / scene.n, 4)}
    for name, subsets in (("filtered", [lists[int(k)] for k in site]), ("unfiltered", None)):
        vb = api.ViewBatch(cams, scene.n, subsets=subsets, device=dev)
        body, st, cap = _forward_plan(api, torch, g, vb, cfg, dev)
        gr = _graph_of(torch, body)
        ms = _replay_ms(torch, gr, reps)
        if st.read()["code"] != 0:
            raise RuntimeError(f"device status {st.read()}")
        out[name] = {"ms_per_batch": round(ms, 3), "fps": round(len(cams) / (ms / 1e3), 1),
                     "items": int(vb.n_items), "instances": int(st.read()["n_instances"])}
        del gr, body, vb
        torch.cuda.empty_cache()
    out["fps_gain"] = round(out["filtered"]["fps"] / out["unfiltered"]["fps"], 3)
    return out


def small_scene_bench(api, N, torch, dev, reps):
    """Config 0 (2000 Gaussians, one 128x128 view, SH degree 0): the plain forward (project ->
    bin_sort -> render) replayed as a CUDA graph; launch-bound at this size."""
    from paper_2403_13806_gb300 import synth
    scene, cams = synth.config0()
    g = api.Gaussians.from_scene(scene, device=dev)
    vb = api.ViewBatch(cams, scene.n, device=dev)
    body, st, cap = _forward_plan(api, torch, g, vb, api.config(), dev)
    gr = _graph_of(torch, body)
    ms = _replay_ms(torch, gr, reps)
    return {"gaussians": scene.n, "width": 128, "height": 128, "ms_forward": round(ms, 4),
            "fps": round(1000.0 / ms, 1), "instances": int(st.read()["n_instances"])}


def importance_bench(api, N, torch, dev, reps):
    """Importance scoring (config 1, Sec. 3.3): 500k Gaussians, 32 views of 1280x832 in one
    launch per stage (project -> bin_sort -> rs_importance, no image outputs), replayed as a
    CUDA graph, then the prune filter h < 0.01 with its index list."""
    from paper_2403_13806_gb300 import synth
    scene, cams = synth.config1()
    g = api.Gaussians.from_scene(scene, device=dev)
    cfg = api.config()
    vb = api.ViewBatch(cams, scene.n, device=dev)
    h = torch.zeros(scene.n, dtype=torch.int32, device=dev)
    body, st, cap = _forward_plan(api, torch, g, vb, cfg, dev, importance=h, image=False)

    def imp():
        h.zero_()
        body()

    gr = _graph_of(torch, imp)
    ms = _replay_ms(torch, gr, reps)
    ws = api.Workspace(dev)
    mask = torch.empty(scene.n, dtype=torch.uint8, device=dev)
    idx = torch.empty(scene.n, dtype=torch.int32, device=dev)
    cnt_holder = {}

    def filt():
        cnt_holder["c"] = api.filter(h, 0.01, N.RS_PRUNE_BELOW, ws, mask=mask, idx=idx)[2]

    grf = _graph_of(torch, filt)
    ms_f = _replay_ms(torch, grf, max(reps, 10))
    pruned = int(cnt_holder["c"].item())
    return {"views": len(cams), "gaussians": scene.n, "ms_importance_32_views": round(ms, 3),
            "ms_per_view": round(ms / len(cams), 4), "ms_filter": round(ms_f, 4),
            "pruned_at_t_0.01": pruned, "kept": scene.n - pruned, "instances": int(st.read()["n_instances"])}


def optimizer_bench(api, N, torch, g, gbuf, h, hbm, reps):
    """The optimisation step around the path on the 1M-Gaussian parameters: one Adam step over
    all 59 floats per Gaussian (28 B moved per float: p, g, m, v read, p, m, v written), and
    the pruning compaction at threshold 0 (every point survives: the largest compaction a
    pruning step can do; at the paper's t_prune = 0.01 this synthetic scene, whose front
    layer occludes most points, keeps well under 1 %, reported beside it) -- the survivors'
    columns of the parameters and both moments:
    2 x 4 B per float moved, plus 4 B of index per survivor."""
    m = [torch.zeros_like(t) for t in g.tensors()]
    v = [torch.zeros_like(t) for t in g.tensors()]
    groups = [(p, gr, mm, vv, 1e-3) for p, gr, mm, vv in zip(g.tensors(), gbuf.views, m, v)]
    n_float = sum(t.numel() for t in g.tensors())
    api.adam_step(groups, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for k in range(reps):
        api.adam_step(groups, 2 + k)
    e1.record()
    torch.cuda.synchronize()
    ms_adam = e0.elapsed_time(e1) / reps
    gbs = 28.0 * n_float / (ms_adam / 1e3) / 1e9
    _, _, cnt_paper = api.filter(h, 0.01, N.RS_PRUNE_KEEP, mask=False)
    kept_paper = int(cnt_paper.item())
    t_med = 0.0   # every point survives: the largest compaction a pruning step can do
    _, idx, cnt = api.filter(h, t_med, N.RS_PRUNE_KEEP, mask=False)
    kept = int(cnt.item())
    src = list(g.tensors()) + m + v
    dst = [torch.empty(t.shape[:-1] + (max(kept, 1),), device=t.device) for t in src]
    pairs = list(zip(src, dst))
    api.gather_columns(pairs, idx, cnt, max(kept, 1))
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        api.gather_columns(pairs, idx, cnt, max(kept, 1))
    e1.record()
    torch.cuda.synchronize()
    ms_g = e0.elapsed_time(e1) / reps
    moved = kept * (3 * (n_float // g.n) * 8 + 4)
    ggbs = moved / (ms_g / 1e3) / 1e9
    del m, v, dst, pairs
    # the scale initialisation of Sec. 3.2: nearest-neighbour distance of every mean
    api.nn_distance(g.means)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(3):
        api.nn_distance(g.means)
    e1.record()
    torch.cuda.synchronize()
    ms_nn = e0.elapsed_time(e1) / 3
    return {"adam": {"floats": int(n_float), "ms": round(ms_adam, 4), "achieved_gbs": round(gbs, 1),
                     "frac": round(gbs / hbm, 4)},
            "nn_init": {"points": int(g.n), "ms": round(ms_nn, 4), "points_per_s": round(g.n / (ms_nn / 1e3), 0)},
            "prune_gather": {"t": t_med, "kept": kept, "kept_at_paper_t_prune": kept_paper, "of": int(g.n),
                             "arrays": 15, "ms": round(ms_g, 4),
                             "achieved_gbs": round(ggbs, 1), "frac": round(ggbs / hbm, 4)}}


def plain_loop(api, N, torch, g, vb1, cfg, target, cams, reps, dev, loss_fn):
    """The same views one at a time with plain launches (no graph), the step's work per view
    (project, bin/sort, blend with importance, loss, backward) and its one prune filter per
    step: fwd+bwd ms/view, and forward-only FPS of one view (project + bin/sort + blend).
    cfg and the views' tile shape are the caller's (defaults, or the autotuned ones)."""
    rasts = []
    for vb in vb1:
        r = api.Rasterizer(cfg=cfg, device=dev, front=FRONT)
        r.forward(g, vb)
        cap = int(r.status.read()["required"] * 1.05) + 4096
        rasts.append((r, api.Bins.empty(cap, vb.n_tiles, device=dev)))
    V = len(vb1)
    per = vb1[0].n_pixels * 3
    tg = [target[i * per:(i + 1) * per] for i in range(V)]
    grads = [torch.zeros_like(t) for t in g.tensors()]
    h = torch.zeros(g.n, dtype=torch.int32, device=dev)
    st = api.DeviceStatus(dev)
    ws_f = api.Workspace(dev)

    def one(i):
        vb = vb1[i]
        r, bins = rasts[i]
        proj = api.project(g, vb, r.cfg, st)
        api.bin_sort(proj, vb, bins, r.ws_sort, st, front=FRONT)
        img, T, L = api.render(proj, bins, vb, r.cfg, importance=h)
        l, dl = loss_fn(img, tg[i])
        # a step's first view writes the gradients and the others add theirs, as in the
        # batched step
        api.render_backward(g, vb, proj, bins, T, L, dl, grads, r.ws_bwd,
                            overwrite_cfg(N, r.cfg) if i == 0 else r.cfg)
        if i == V - 1:
            api.filter(h, 0.01, N.RS_PRUNE_BELOW, ws_f)

    for i in range(V):
        one(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        for i in range(V):
            one(i)
    e1.record()
    torch.cuda.synchronize()
    plain = e0.elapsed_time(e1) / (reps * V)
    # forward-only FPS, view 0
    vb = vb1[0]
    r, bins = rasts[0]
    proj = api.project(g, vb, r.cfg, st)
    img = torch.empty(3 * vb.n_pixels, device=dev)
    fr = max(reps, 10)
    for _ in range(3):
        api.project(g, vb, r.cfg, st, out=proj)
        api.bin_sort(proj, vb, bins, r.ws_sort, st, front=FRONT)
        api.render(proj, bins, vb, r.cfg, image=img, T_final=False, last=False)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(fr):
        api.project(g, vb, r.cfg, st, out=proj)
        api.bin_sort(proj, vb, bins, r.ws_sort, st, front=FRONT)
        api.render(proj, bins, vb, r.cfg, image=img, T_final=False, last=False)
    e1.record()
    torch.cuda.synchronize()
    fps = 1000.0 / (e0.elapsed_time(e1) / fr)
    return plain, fps


def overwrite_cfg(N, cfg):
    """A copy of cfg whose render_backward writes the gradients (the first launch of a step)."""
    c = N.RsConfig.from_buffer_copy(cfg)
    c.grad_overwrite = 1
    return c


def e2e_run(api, N, torch, scene, vbs, cfg, targets, cap, reps, dev, world=1, loss_fn=None):
    """Same batched step through the public API (an api.StepGraph per input buffer set):
    every step copies its parameters and targets from pinned host memory and reads its loss
    back to the host.  The copies of step k+1 run on a copy stream while step k computes
    (two device buffer sets, events order each buffer's reuse), as a training loop's input
    pipeline would, and the host reads step k's loss once step k+1 is queued (a logging
    loop that never leaves the GPU idle); the last step's loss is read inside the timed
    region too.  With world > 1 the reductions over ranks follow each graph."""
    from paper_2403_13806_gb300 import dist as rd
    host = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory() for a in scene.arrays()]
    tgt_h = [t.cpu().pin_memory() for t in targets]
    st = api.DeviceStatus(dev)
    proj = api.Projected.empty(max(vb.n_items for vb in vbs), dev)
    bins_all = api.Bins.empty(cap, max(vb.n_tiles for vb in vbs), device=dev)
    ws_sort, ws_bwd, ws_f = api.Workspace(dev), api.Workspace(dev), api.Workspace(dev)
    h = torch.zeros(scene.n, dtype=torch.int32, device=dev)
    loss_d = torch.zeros(len(vbs), dtype=torch.float64, device=dev)
    img_buf = [torch.empty(3 * vb.n_pixels, device=dev) for vb in vbs]
    T_buf = [torch.empty(vb.n_pixels, device=dev) for vb in vbs]
    L_buf = [torch.empty(vb.n_pixels, dtype=torch.int32, device=dev) for vb in vbs]
    dl_buf = [torch.empty(3 * vb.n_pixels, device=dev) for vb in vbs]
    mask = torch.empty(scene.n, dtype=torch.uint8, device=dev)
    idx = torch.empty(scene.n, dtype=torch.int32, device=dev)
    cfg_w = overwrite_cfg(N, cfg)

    def make_set():
        dev_p = [torch.empty_like(t, device=dev) for t in host]
        tgt_d = [torch.empty_like(t) for t in targets]
        for d, s_ in zip(dev_p, host):
            d.copy_(s_)
        for d, s_ in zip(tgt_d, tgt_h):
            d.copy_(s_)
        g = api.Gaussians(*dev_p, scene.sh_degree)
        gbuf = rd.GradBuffer(dev_p)
        loss_h = torch.zeros(len(vbs), dtype=torch.float64).pin_memory()   # this set's step loss

        def prune():
            api.filter(h, 0.01, N.RS_PRUNE_BELOW, ws_f, mask=mask, idx=idx)

        side = torch.cuda.Stream(device=dev)
        imp_done, prune_done = torch.cuda.Event(), torch.cuda.Event()

        def views_part(overlap_prune=False):
            h.zero_()
            for i, vb in enumerate(vbs):
                bins = api.Bins(bins_all.vals, bins_all.ranges[:vb.n_tiles], None, cap)
                api.project(g, vb, cfg, st, out=proj)
                api.bin_sort(proj, vb, bins, ws_sort, st, front=FRONT)
                img, T, L = api.render(proj, bins, vb, cfg, image=img_buf[i], T_final=T_buf[i], last=L_buf[i],
                                       importance=h)
                if overlap_prune and i == len(vbs) - 1:   # the filter beside the last loss and backward
                    imp_done.record()
                    with torch.cuda.stream(side):
                        side.wait_event(imp_done)
                        prune()
                        prune_done.record(side)
                loss, dl = loss_fn(img, tgt_d[i], dL=dl_buf[i], loss=loss_d[i:i + 1])
                api.render_backward(g, vb, proj, bins, T, L, dl, gbuf.views, ws_bwd, cfg_w if i == 0 else cfg)
            if overlap_prune:
                torch.cuda.current_stream().wait_event(prune_done)

        if world == 1:
            sg = api.StepGraph(lambda: views_part(overlap_prune=True), outputs=[(loss_d, loss_h)], device=dev)
        else:
            sg = api.StepGraph(views_part, device=dev)
        return {"p": dev_p, "t": tgt_d, "sg": sg, "gbuf": gbuf, "prune": prune, "loss_h": loss_h,
                "done": torch.cuda.Event()}

    sets = [make_set(), make_set()]
    copy_stream = torch.cuda.Stream(device=dev)
    comp = torch.cuda.current_stream(dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]

    def copy_in(k):
        b = sets[k % 2]
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(used[k % 2])   # the previous step on this buffer set is done
            for d, s_ in zip(b["p"], host):
                d.copy_(s_, non_blocking=True)
            for d, s_ in zip(b["t"], tgt_h):
                d.copy_(s_, non_blocking=True)
            copied[k % 2].record(copy_stream)

    def step(k):
        """Queues step k, then reads step k-1's loss on the host."""
        b = sets[k % 2]
        copy_in(k + 1)                 # the next step's inputs, behind this step's compute
        comp.wait_event(copied[k % 2])
        b["sg"].launch()
        if world > 1:
            rd.allreduce_importance(h)
            rd.allreduce_grads(b["gbuf"])
            b["prune"]()
            b["loss_h"].copy_(loss_d, non_blocking=True)
        used[k % 2].record(comp)
        b["done"].record(comp)
        return read_loss(k - 1) if k > 0 else None

    def read_loss(k):
        b = sets[k % 2]
        b["done"].synchronize()
        return float(b["loss_h"].mean())

    copy_in(0)
    for k in range(2):
        step(k)
    read_loss(1)
    t0 = time.perf_counter()
    for k in range(2, 2 + reps):
        step(k)
    read_loss(1 + reps)
    dt = (time.perf_counter() - t0) / reps * 1000.0
    torch.cuda.synchronize()
    h2d = sum(t.numel() * 4 for t in host) + sum(t.numel() * 4 for t in targets)
    n_views = sum(vb.n_views for vb in vbs)
    return {"value": round(dt / n_views, 4), "unit": "ms/view (fwd+bwd)", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": 8 * len(vbs),
            "input_pipeline": "step k+1's copies overlap step k's compute (two device buffer sets); "
                              "step k's loss is read on the host once step k+1 is queued"}


# Algorithmic work per evaluated (pixel, Gaussian) pair of the blend kernels, as the
# method's arithmetic counts it (an FMA is one operation): the forward blend (A5) needs about
# 15 FP32 operations and one ex2, the importance maximum (A6) one more operation; the
# backward blend (A8) about 40 FP32 operations and one ex2.
FP32_OPS_PER_PAIR = {"k_render_importance": 16, "k_render": 15, "k_render_bwd": 40}
EX2_PER_PAIR = 1
# The FP32 operations the kernels as written execute per pair (counted from their source:
# forward 18 = offsets 1.25, quadratic form 2.75 (its column terms shared by a thread's
# eight pixels), warp pre-test 0.6, exp2 and saturated scale 2, alpha factor and product 2,
# transmittance and stop test 3, weight 1, colour 3, last-entry test and select 2,
# importance max 0.5; backward 43), reported beside the algorithmic figure.
INSTR_OPS_PER_PAIR = {"k_render_importance": 18, "k_render": 18, "k_render_bwd": 43}
L2_BYTES = 126 * 2 ** 20     # the working set below which a kernel's bytes stay in L2

# Probe kernels (rs_peak_probe): name, kind, iterations per launch (about 1-3 ms each).
PROBES = (("ffma", 0, 20000), ("ffma2", 1, 10000), ("alu", 2, 12000), ("ex2", 3, 2500), ("smem", 4, 3000),
          ("l2", 5, 300))


def probe_peaks(N, torch, dev, reps=5):
    """Measured peaks (rates per second) of the probe kernels on this GPU: best of `reps`
    launches after two untimed ones, CUDA events on the launching stream, SM clocks sampled
    meanwhile.  FP32/ALU/ex2 in lane operations per second, smem and L2 in bytes per second."""
    import ctypes
    L = N.lib()
    sink = torch.zeros(int(L.rs_peak_probe_sink_floats()), device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    rates = {}
    with ClockSampler(dev.index or 0) as clk:
        for name, kind, iters in PROBES:
            work = ctypes.c_double()
            best = 0.0
            for r in range(2 + reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                N.call("rs_peak_probe", kind, iters, ctypes.c_void_p(sink.data_ptr()), sink.numel(),
                       ctypes.byref(work), sp)
                e1.record(stream)
                e1.synchronize()
                if r >= 2:
                    best = max(best, work.value / (e0.elapsed_time(e1) / 1e3))
            rates[name] = best
    c = clk.summary()
    mhz = c["sm_mhz"] or 2070.0
    per = 152 * mhz * 1e6
    return {
        "ffma_tops": round(rates["ffma"] / 1e12, 2), "ffma2_tops": round(rates["ffma2"] / 1e12, 2),
        "alu_tops": round(rates["alu"] / 1e12, 2), "ex2_tops": round(rates["ex2"] / 1e12, 3),
        "smem_tbs": round(rates["smem"] / 1e12, 2), "l2_tbs": round(rates["l2"] / 1e12, 2),
        "per_sm_per_clock": {"ffma": round(rates["ffma"] / per, 1), "ffma2": round(rates["ffma2"] / per, 1),
                             "alu": round(rates["alu"] / per, 1), "ex2": round(rates["ex2"] / per, 1),
                             "smem_bytes": round(rates["smem"] / per, 1), "l2_bytes": round(rates["l2"] / per, 1)},
        "fp32_peak_tops": round(max(rates["ffma"], rates["ffma2"]) / 1e12, 2),
        "clocks": c,
        "how": "rs_peak_probe kernels (8 CTAs x 256 threads per SM, 8 independent chains per thread), best of "
               f"{reps} launches, CUDA events; FP32 peak = the larger of the FFMA and packed-FFMA2 lane-op rates",
    }


# DRAM bytes (read + write) per launch of a kernel, per view of the benchmark workload, from
# one ncu capture of a one-view run (command and figures under profiles/), with the hashes
# of the sources the kernel was built from.  A capture stays valid only while those sources
# are unchanged; otherwise the roofline reports traffic as null.
NCU_TRAFFIC = {
    "k_render_bwd": {"bytes_per_view": 25188352, "files": ['render_bwd.cu', 'blend.cuh', 'rs_common.cuh'], "sha": "a467508de8517e80",
                "profile": "k_render_bwd_1M_1view.md"},
    "k_render_importance": {"bytes_per_view": 4438016, "files": ['render.cu', 'blend.cuh', 'rs_common.cuh'], "sha": "178210ccb9e97d95",
                "profile": "k_render_1M_1view.md"},
    "k_fine_scatter": {"bytes_per_view": 20112128, "files": ['binsort.cu', 'rs_common.cuh'], "sha": "4cffedcde21798e1",
                "profile": "k_fine_scatter_1M_1view.md"},
    "k_ssim_stats": {"bytes_per_view": 25871360, "files": ['ssim.cu', 'rs_common.cuh'], "sha": "77368fb65aa91f37",
                "profile": "k_ssim_stats_1view.md"},
}


def _src_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2403_13806_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(name, views):
    rec = NCU_TRAFFIC.get(name)
    if not rec or _src_hash(rec["files"]) != rec["sha"]:
        return None
    return int(rec["bytes_per_view"] * views)


class _PerLaunch:
    """Averages of a step's launches (all launches of a step cover equal view chunks)."""

    def __init__(self, vbs):
        c = len(vbs)
        self.n_items = sum(vb.n_items for vb in vbs) / c
        self.n_pixels = sum(vb.n_pixels for vb in vbs) / c
        self.n_tiles = max(vb.n_tiles for vb in vbs)
        self.n_gaussians = vbs[0].n_gaussians
        self.launches = c


def kernel_work(vbs, sres, pairs, n_super, touched, kept_items, touched_items):
    """Algorithmic work per launch of each library kernel: DRAM bytes the method must move
    (bound "hbm") or FP32 lane operations (bound "alu").

    Items M (view, Gaussian) pairs, instances K, super-tile instances Ks, pixels P:
    projection reads 236 B of parameters per Gaussian (per item for visibility lists) and
    writes 52 B per item; the occlusion cut of front lists reads 36 B per item of the
    nearest 1/32 and 64 B of bound sums per tile, and the emission then reads only the items
    ranked before the largest cut (counted as the window); the depth sort moves
    8 B per item and pass (read key+value, write key+value = 16 B in the scatter, 4 B read in
    the count); the super-tile sort moves 2 x (2 + 4 + 1) B per super instance and pass
    (count: 2 B); the fine partition reads the 1 B cover byte per super instance (count),
    then 4 B item + 1 B cover byte per super instance and writes 4 B per instance (scatter);
    the projection backward writes 236 B of gradients per Gaussian (written, not
    accumulated), reads a 1 B flag per item and 36 B of image-space gradients per flagged
    item, and reads the 236 B of
    parameters and the 16 B colour rows only for the `touched` Gaussians some view gives a
    gradient (most of a dense scene is hidden behind saturated pixels); for the blend kernels
    the work is the (pixel, Gaussian) pairs evaluated per launch."""
    vb = _PerLaunch(vbs)
    c = vb.launches
    M, K, Ks, P = vb.n_items, sres["n_instances"], n_super / c, vb.n_pixels
    Wc = -(-(kept_items / c) // 32)    # the occlusion cut's window (ranks) per launch
    Mr = Wc if FRONT else M            # items the super-instance emission reads
    pairs = pairs / c
    kb = 2 if vb.n_tiles <= 65536 else 4
    hbm = {
        # dense batches read each Gaussian's parameters once for all its views
        "k_project": (vb.n_gaussians * 236 + M * 52) if (vbs[0].subset is None and vbs[0].n_views > 1)
        else M * (236 + 52),
        "k_depth_keys": M * (4 + 8),
        # front lists: only the items ranked before the largest cut (at most the window) are read
        "k_count_blocks": Mr * (4 + 8),
        "k_emit": Mr * (4 + 8) + Ks * (kb + 4 + 1),
        "k_depth_sort_hist": M * 4,
        "k_depth_sort": M * 16,
        # occlusion cut (front lists): the nearest 1/32 of the items with instances, their order
        # entry, mean, conic and rect; then 16 bound sums per tile
        "k_cut_accumulate": Wc * (4 + 8 + 16 + 8),
        "k_cut_tiles": vb.n_tiles * 16 * 4,
        "k_super_sort_hist": Ks * kb,
        "k_super_sort": Ks * 2 * (kb + 4 + 1),
        "k_ranges": Ks * kb,
        "k_fine_count": Ks * 1,
        "k_fine_scatter": Ks * (4 + 1) + K * 4,
        "k_l1": P * 3 * 4 * 3,
        "k_ssim_stats": P * 3 * (8 + 12),
        "k_ssim_grad": P * 3 * (12 + 8 + 4),
        # gradients written once per Gaussian (all views summed in registers); a 1 B flag read
        # per item, 36 B of image-space gradients per flagged item; parameters and colour rows
        # of the Gaussians with a gradient
        "k_project_bwd": vb.n_gaussians * 236 + M * 1 + touched_items * 36 + touched * (236 + 16 * M / vb.n_gaussians),
        # the previous call's flagged items: flags read, their gradients and flags zeroed
        "k_bwd_prepare": M * 1 + touched_items * (36 + 1),
        "k_filter_count": vb.n_gaussians * 4,
        "k_filter_scatter": vb.n_gaussians * (4 + 1) + vb.n_gaussians * 4,
    }
    out = {k: ("hbm", v) for k, v in hbm.items()}
    for k in FP32_OPS_PER_PAIR:
        out[k] = ("alu", pairs)     # pairs evaluated per launch
    return out


def kernel_frac(name, rec, work, hbm_peak, probes):
    """Achieved rate of one kernel against its bound.  Byte-bound kernels: GB/s of their
    algorithmic bytes against the measured HBM copy bandwidth, and against the probed L2
    bandwidth; the bound is "l2" when the bytes of one launch fit in L2 (they are then
    served from it), else "hbm".  Blend kernels: FP32 lane operations per second of the
    method's count per pair against the probed FP32 peak, with the ex2 rate against MUFU."""
    kind, w = work[name]
    t = rec["ms_per_launch"] / 1000.0
    if kind == "hbm":
        a = w / t / 1e9
        l2 = probes["l2_tbs"] * 1e3
        bound = "l2" if w <= L2_BYTES else "hbm"
        out = {"bound": bound, "achieved_gbs": round(a, 1), "frac_hbm": round(a / hbm_peak, 4),
               "frac_l2": round(a / l2, 4)}
        out["frac"] = out["frac_l2"] if bound == "l2" else out["frac_hbm"]
        return out
    pairs = w
    a = pairs * FP32_OPS_PER_PAIR[name] / t / 1e12
    ex2 = pairs * EX2_PER_PAIR / t / 1e12
    return {"bound": "alu", "achieved_tops": round(a, 2), "frac": round(a / probes["fp32_peak_tops"], 4),
            "ex2_frac": round(ex2 / probes["ex2_tops"], 4),
            "instr_tops": round(pairs * INSTR_OPS_PER_PAIR[name] / t / 1e12, 2),
            "instr_frac": round(pairs * INSTR_OPS_PER_PAIR[name] / t / 1e12 / probes["fp32_peak_tops"], 4)}


def roofline(kernel_ms, work, hbm, peak_kind, views, probes):
    """Roofline of the kernel with the largest share of the step (library launch events)."""
    name, rec = max(kernel_ms.items(), key=lambda kv: kv[1]["ms_per_step"])
    t = rec["ms_per_launch"] / 1000.0
    kind, w = work.get(name, ("hbm", 0))
    traffic = ncu_traffic(name, views)
    if kind == "hbm":
        a = w / t / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": round(a, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(a / hbm, 4), "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "work_per_launch": int(w), "ms_per_launch": round(rec["ms_per_launch"], 5)}
    f = kernel_frac(name, rec, work, hbm, probes)
    ops = w * FP32_OPS_PER_PAIR[name]
    return {"kernel": name, "bound": "alu", "achieved": f["achieved_tops"], "peak": probes["fp32_peak_tops"],
            "unit": "TOP/s (FP32 lane ops)", "frac": f["frac"], "traffic": traffic,
            "peak_source": "measured: rs_peak_probe FFMA / FFMA2 probe kernels on this GPU during this run "
                           f"(SM clock {probes['clocks']['sm_mhz']} MHz)",
            "work_per_launch": int(ops),
            "work": f"{int(w)} (pixel, Gaussian) pairs x {FP32_OPS_PER_PAIR[name]} FP32 ops (+{EX2_PER_PAIR} ex2)",
            "ex2_frac": f["ex2_frac"], "instr_frac": f["instr_frac"],
            "ms_per_launch": round(rec["ms_per_launch"], 5)}


# ------------------------------------------------------------------ CPU oracle

def _oracle_pass(scene, cam, pix, threads):
    import oracle
    import oracle.grad as og
    t0 = time.perf_counter()
    proj = oracle.project(scene, cam)
    r = oracle.render(proj, pixels=pix, mode="bucketed", threads=threads)
    w = np.sign(r["image"] - 0.5) / (3.0 * WIDTH * HEIGHT)
    og.gradients(scene, cam, w, pixels=pix, chunk=64)
    return time.perf_counter() - t0


def oracle_sample_time(n_small: int, n_big: int, threads: int, seed: int = 0):
    """Times the FP64 oracle on a bounded sample of the workload (view 0): the FP64
    projection of all 1M Gaussians, front-to-back compositing of seeded random pixels
    (bucketed candidates) and the FP64 autograd gradient of an L1 loss on them, once with
    n_small and once with n_big pixels.  The per-view cost is extrapolated as
    fixed + per-pixel x (1280*832): fixed = t_small - n_small * per-pixel,
    per-pixel = (t_big - t_small) / (n_big - n_small).  Returns (seconds spent, ms/view)."""
    import torch
    from paper_2403_13806_gb300 import synth
    torch.set_num_threads(threads)
    scene, cams = synth.config2(n=N_GAUSSIANS, n_views=1)
    cam = cams[0]
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, WIDTH, n_big), rng.integers(0, HEIGHT, n_big)], 1).astype(np.int32)
    t_small = _oracle_pass(scene, cam, pix[:n_small], threads)
    t_big = _oracle_pass(scene, cam, pix, threads)
    per_pixel = max(t_big - t_small, 0.0) / (n_big - n_small)
    fixed = max(t_small - n_small * per_pixel, 0.0)
    return t_small + t_big, (fixed + per_pixel * WIDTH * HEIGHT) * 1000.0


def cpu_baseline(args):
    threads = os.cpu_count() or 1
    n_small, n_big = 64, 960
    try:
        dt, ms_view = oracle_sample_time(n_small, n_big, threads)
    except Exception as e:  # the baseline is reported, not required
        return {"value": None, "unit": "ms/view (fwd+bwd)", "cores": threads, "kind": "oracle", "error": str(e)[:200]}
    return {"value": round(ms_view, 1), "unit": "ms/view (fwd+bwd)", "cores": threads, "kind": "oracle",
            "sample": f"view 0: FP64 projection of all 1M Gaussians + compositing and autograd gradient of "
                      f"{n_small} and {n_big} seeded pixels ({dt:.1f} s), per-view cost extrapolated as "
                      f"fixed + per-pixel x 1280*832"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    for w in range(args.warmup):
        oracle_sample_time(8, 16, threads, seed=100 + w)
    times, spent = [], 0.0
    for k in range(args.steps):
        dt, ms_view = oracle_sample_time(32, 96, threads, seed=k)
        times.append(ms_view)
        spent += dt
    value = float(np.mean(times))
    cpu = {"value": round(value, 1), "unit": "ms/view (fwd+bwd)", "cores": threads, "kind": "oracle",
           "sample": "per step, view 0: FP64 projection of all 1M Gaussians + compositing and autograd gradient of "
                     "32 and 96 seeded pixels, per-view cost extrapolated as fixed + per-pixel x 1280*832"}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms/view (fwd+bwd)",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(spent / max(args.steps, 1) * 1000.0, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded 360-capture scene)", "config": workload_config(args.views, world),
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 1), "unit": "ms/view (fwd+bwd)", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_report(full_view: bool = True):
    """The FP64 C oracle timed alone on the host cores (wall clock): config 0 forward in
    brute mode over its full 128x128 image, single thread and all cores, best of 3; config 2
    (1M Gaussians, one 1280x832 view) forward in bucketed mode over the full view on all cores
    (once), and single-thread on 4096 seeded pixels (best of 3, scaled to the view); the FP64
    autograd gradient on 512 seeded pixels (scaled to the view, labelled as autograd)."""
    import oracle
    import oracle.grad as og
    import torch
    from paper_2403_13806_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    torch.set_num_threads(cores)
    rep = {"nproc": cores, "cpu_model": _cpu_model(), "how": "wall clock (time.perf_counter), best of 3 unless noted"}

    def best(f, k=3):
        return min(f() for _ in range(k))

    def timed(f):
        t = time.perf_counter()
        f()
        return time.perf_counter() - t

    scene0, cams0 = synth.config0()
    p0 = oracle.project(scene0, cams0[0])
    rep["config0_forward_brute_full_image_s"] = {
        "threads_1": round(best(lambda: timed(lambda: oracle.render(p0, mode="brute", threads=1))), 4),
        f"threads_{cores}": round(best(lambda: timed(lambda: oracle.render(p0, mode="brute", threads=cores))), 4)}
    scene, cams = synth.config2(n=N_GAUSSIANS, n_views=1)
    cam = cams[0]
    tproj = best(lambda: timed(lambda: oracle.project(scene, cam)))
    p = oracle.project(scene, cam)
    P = WIDTH * HEIGHT
    rng = np.random.default_rng(7)
    pix = np.stack([rng.integers(0, WIDTH, 4096), rng.integers(0, HEIGHT, 4096)], 1).astype(np.int32)
    t1 = best(lambda: timed(lambda: oracle.render(p, pixels=pix, mode="bucketed", threads=1)))
    c2 = {"projection_1M_s": round(tproj, 3), "threads_1_per_view_s_scaled_from_4096_pixels": round(tproj + t1 / 4096 * P, 1)}
    if full_view:
        tf = timed(lambda: oracle.render(p, mode="bucketed", threads=cores))
        c2[f"threads_{cores}_full_view_s"] = round(tproj + tf, 1)
    rep["config2_forward_bucketed"] = c2
    pg = pix[:512]
    w = rng.normal(size=(512, 3))
    tg = timed(lambda: og.gradients(scene, cam, w, pixels=pg))
    rep["config2_gradient_autograd"] = {"pixels": 512, "s": round(tg, 2),
                                        "per_view_s_scaled": round(tg / 512 * P, 1),
                                        "note": "FP64 PyTorch autograd restatement, one pixel at a time"}
    fwd = c2.get(f"threads_{cores}_full_view_s")
    if fwd is not None:
        rep["fwd_plus_bwd_ms_per_view"] = round((fwd + tg / 512 * P) * 1000.0, 0)
    return rep


def run_probes():
    import torch
    from paper_2403_13806_gb300 import _native as N
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    print(json.dumps({"probes": probe_peaks(N, torch, dev)}))


def main():
    global FRONT, FRONT_ALLOWED
    args = parse()
    FRONT = FRONT_ALLOWED = args.lists == "front"
    if args.probes:
        run_probes()
    elif args.cpu_report:
        print(json.dumps({"cpu_report": cpu_report()}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
