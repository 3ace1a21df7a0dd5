"""Throughput of one multi-view training step of EWA splatting on GB300.

A step is one pass of the whole hot path over one batch of V views of a
resident scene: participation + projection + colour, (view, tile, depth)
binning and sort, front-to-back blending, 0.8 L1 + 0.2 D-SSIM loss and its
gradient, back-to-front blend backward, reduction of the gradients across
views onto the 3D Gaussians, and the multi-view densification statistics.

The headline workload is 3M SH-3 Gaussians seen by 8 views of mixed
resolutions (800x600 to 1920x1080) in one persistent launch per stage, with
the autotuned tile; `secondary_workload` repeats the batched step and the
per-view loop on 500k Gaussians and 4 views of 1264x832.

Prints one JSON line.  `value` is views per second of the batched path
(inputs resident in HBM), `e2e` the same through the C ABI with the scene and
the targets copied from pinned host memory and the loss copied back every
step.  `--impl reference` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "uneven_3m_8views"
SECONDARY_WORKLOAD = "multiview_500k_4x1264x832"
LAMBDA = 0.2
METRIC = "fwd+bwd views/s (batched multi-view vs per-view loop) at oracle tol; serve p50/p99"
FP32_LANES_PER_SM = 128
# Algorithmic FP32 work of the blend kernels, counted only on the (pixel,
# Gaussian) pairs Eq. 1 actually blends (so it does not depend on the tile
# size or on how many list entries an implementation inspects): evaluating
# the pair (offsets, quadratic form, exponent, opacity product and clamp:
# 14 FLOP, plus one ex2), then blending it in the forward (transmittance,
# weight, three colour FMAs: 8 FLOP) or differentiating it in the backward
# (transmittance recovery, colour, alpha, exponent, mean2d, conic, opacity and
# E1 terms: 50 FLOP, counted from the chain rule of Eq. 1).
FWD_FLOP_PER_BLENDED = 14 + 8
BWD_FLOP_PER_BLENDED = 14 + 50


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--tile", default="auto", help="WxH, or auto (timed choice before the measured steps)")
    ap.add_argument("--ppt", type=int, default=0, help="blend pixels per thread (0 = automatic)")
    ap.add_argument("--smem-batch", type=int, default=0, help="Gaussians per shared-memory batch (0 = automatic)")
    ap.add_argument("--no-loop", action="store_true", help="skip the per-view launch loop")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph measurements")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrivals per second")
    ap.add_argument("--profile-once", action="store_true",
                    help="size the buffers by the participation pre-count, run exactly one training step and exit "
                         "(one launch of each kernel, in order: for profilers)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary workload (500k Gaussians, 4 views of 1264x832)")
    ap.add_argument("--no-partial", action="store_true",
                    help="skip the partial-rendering comparison (full / masked / thread-efficient)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # nvidia-smi takes a while to start: wait for its first sample so the
        # ones that follow cover the timed steps
        t0 = time.time()
        while not self.lines and self.proc.poll() is None and time.time() - t0 < 5.0:
            time.sleep(0.01)
        self.lines.clear()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    from paper_2506_12727_gb300 import build as lib_build
    lib_build.build()
    from paper_2506_12727_gb300 import mvgs, shard

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    scene, cams, extra = synth.workload(args.workload)
    sharder = None
    if world > 1:
        # weak scaling: a global batch of world x V views (the workload's
        # resolutions again, new poses; its first V views are the workload's
        # own), split between the ranks by pixels; one all-reduce per step
        res = [(int(w), int(h)) for w, h in zip(cams.width, cams.height)] * world
        cams_g = synth.make_cameras(res, radius=4.0)
        sharder = shard.ViewShardedStep(rank, world)
        own, grad_scale = sharder.views([int(p) for p in cams_g.pixels()])
        cams = cams_g.subset(own)
    V, n = cams.V, scene.n
    V_total = V if sharder is None else cams_g.V  # views of all ranks per step
    if sharder is not None:
        # the other legs measure single-GPU paths: at N > 1 only the sharded step runs
        args.no_graph = args.no_loop = args.no_partial = args.no_serve = args.no_secondary = True
    targets = synth.make_targets(cams)
    hw = np.stack([cams.height, cams.width], 1).astype(np.int32)
    dev = "cuda"
    params = {k: torch.tensor(getattr(scene, k), device=dev).contiguous() for k in
              ("means", "log_scales", "quats", "opacity_logits", "sh")}
    tgt = torch.tensor(synth.pack_images(targets), device=dev)
    sc = mvgs.make_scene(params, scene.sh_degree)
    tuning = None
    if args.tile == "auto":
        from paper_2506_12727_gb300.autotune import autotune
        tile, ppt, tuning, wb = autotune(sc, cams, params)
        args.ppt = ppt
        args.smem_batch = wb
        args.tile = f"{tile[0]}x{tile[1]}"
    tile = tuple(int(x) for x in args.tile.split("x"))
    rz = mvgs.Rasterizer(cams, tile=tile, pixels_per_thread=args.ppt, smem_batch=args.smem_batch)
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    dssim_ws = torch.empty(mvgs.dssim_workspace_size(hw), dtype=torch.uint8, device=dev)
    loss = torch.empty(V, device=dev)
    dimg = torch.empty_like(tgt)
    acc = [torch.zeros(n, device=dev) for _ in range(3)]
    incr = [torch.zeros(n, device=dev) for _ in range(3)] if sharder else None
    gm2d = None
    e1 = None
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def step(rast, scene_c, target, hw_, loss_, dimg_, ws_):
        nonlocal gm2d, e1
        img = rast.forward(scene_c)
        mvgs.dssim_loss(img, target, hw_, LAMBDA, loss_, dimg_, ws_)
        R = int(rast.needed.records)
        if gm2d is None or gm2d.shape[0] < R:
            gm2d = torch.empty(int(R * 1.2) + 16, 2, device=dev)
            e1 = torch.empty(int(R * 1.2) + 16, device=dev)
        if sharder is None or rast is not rz:
            rast.backward(scene_c, dimg_, grads, gm2d, e1)
            mvgs.adc_accumulate(rast.state, n, gm2d, e1, *acc)
            return
        # view-sharded step: this rank's share of the batch-mean loss
        # gradient, this step's statistic increments, one all-reduce of the
        # bucket, then the increments join the running statistics
        dimg_.mul_(grad_scale)
        rast.backward(scene_c, dimg_, grads, gm2d, e1)
        for t_ in incr:
            t_.zero_()
        mvgs.adc_accumulate(rast.state, n, gm2d, e1, *incr)
        sharder.exchange(grads, incr, loss_.sum().reshape(1))
        for a_, d_ in zip(acc, incr):
            a_.add_(d_)

    if args.profile_once:
        rz.reserve_for(sc)
        step(rz, sc, tgt, hw, loss, dimg, dssim_ws)
        torch.cuda.synchronize()
        return {"profile_once": True, "workload": args.workload, "tile": args.tile,
                "records": int(rz.needed.records), "keys": int(rz.needed.keys)}

    def timed(fn, steps, warmup, profile=False):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        if profile:
            mvgs.profile_read()
            mvgs.profile_enable(True)
        ms = []
        s = torch.cuda.current_stream()
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            ms.append((a, b))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        stages = None
        if profile:
            mvgs.profile_enable(False)
            stages = mvgs.profile_read()
        total = sum(a.elapsed_time(b) for a, b in ms)
        return total / steps, stages

    # ---- batched multi-view step (the headline) ----
    clocks = ClockSampler(local)
    launches0 = mvgs.launch_count()
    clocks.start()
    ms_batched, stages = timed(lambda: step(rz, sc, tgt, hw, loss, dimg, dssim_ws), args.steps, args.warmup,
                               profile=True)
    clk = clocks.stop()
    launches = (mvgs.launch_count() - launches0)
    launches_per_step = launches / float(args.steps + args.warmup)
    if dist:
        t = torch.tensor([ms_batched], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_batched = float(t.item())
    needed = (int(rz.needed.records), int(rz.needed.keys))
    # blended (pixel, Gaussian) pairs of the step, the unit of the blend
    # kernels' work: counted by one more forward with the per-pixel statistics
    # (off in the timed steps), outside the timed region
    rz.forward(sc, stats=True)
    blended = int(rz.records()["pixel_stats"].to(torch.int64)[:, 1].sum().item())

    # ---- the same step captured in a CUDA graph (capturable mode) ----
    def graphed(rasterizers, tgts, hws, losses, dimgs, wss, rec_caps):
        """Captures one step over the given rasterizers (one per call) in a
        CUDA graph; returns (graph, fits) where fits() checks the counts."""
        bufs = []
        for rz_, rc in zip(rasterizers, rec_caps):
            bufs.append((torch.empty(3 * rz_.pixels, device=dev), torch.empty(rc, 2, device=dev),
                         torch.empty(rc, device=dev)))
        acc_grads = {k: torch.zeros_like(v) for k, v in params.items()}
        many = len(rasterizers) > 1

        def gstep():
            if many:
                for g_ in acc_grads.values():
                    g_.zero_()
            for rz_, t_, h_, l_, d_, w_, (im_, gm_, e_) in zip(rasterizers, tgts, hws, losses, dimgs, wss, bufs):
                rz_.forward(sc, images=im_)
                mvgs.dssim_loss(im_, t_, h_, LAMBDA, l_, d_, w_)
                rz_.backward(sc, d_, grads, gm_, e_)
                mvgs.adc_accumulate(rz_.state, n, gm_, e_, *acc)
                if many:
                    for k in acc_grads:
                        acc_grads[k].add_(grads[k])
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            gstep()
        torch.cuda.current_stream().wait_stream(side)
        graph_ = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_):
            gstep()
        return graph_, (lambda: all(r.fits() for r in rasterizers))

    graph = None
    if not args.no_graph:
        rzg = mvgs.Rasterizer(cams, tile=tile, pixels_per_thread=args.ppt, smem_batch=args.smem_batch, capturable=True, headroom=1.02)
        rzg.reserve(n, needed[0], needed[1])
        g_b, fits_b = graphed([rzg], [tgt], [hw], [loss], [dimg], [dssim_ws], [rzg.cap.records])
        ms_graph, _ = timed(lambda: g_b.replay(), args.steps, args.warmup)
        graph = {"views_per_s": V / (ms_graph / 1e3), "ms_per_step": ms_graph, "counts_fit": fits_b(),
                 "launches_per_step": None}
        del g_b

    # ---- per-view launch loop: the same library, V = 1, V times ----
    loop = None
    if not args.no_loop:
        singles = []
        for v in range(V):
            cv = cams.subset([v])
            hv = hw[v:v + 1]
            off = synth.view_offsets(cams)
            singles.append((mvgs.Rasterizer(cv, tile=tile, pixels_per_thread=args.ppt, smem_batch=args.smem_batch),
                            tgt[off[v]:off[v + 1]].contiguous(), hv,
                            torch.empty(1, device=dev), torch.empty(int(off[v + 1] - off[v]), device=dev),
                            torch.empty(mvgs.dssim_workspace_size(hv), dtype=torch.uint8, device=dev)))

        acc_grads = {k: torch.zeros_like(v) for k, v in params.items()}

        def loop_step():
            # a per-view training step sums the views' parameter gradients
            for g in acc_grads.values():
                g.zero_()
            for rv, tv, hv, lv, dv, wv in singles:
                step(rv, sc, tv, hv, lv, dv, wv)
                for k in acc_grads:
                    acc_grads[k].add_(grads[k])
        ms_loop, _ = timed(loop_step, max(3, args.steps // 2), 2)
        loop = {"views_per_s": V / (ms_loop / 1e3), "ms_per_step": ms_loop,
                "speedup_batched_over_loop": ms_loop / ms_batched}
        if not args.no_graph:
            # the loop captured in one CUDA graph as well (V capturable calls)
            rzs = []
            for v, (rv, tv, hv, lv, dv, wv) in enumerate(singles):
                rg = mvgs.Rasterizer(cams.subset([v]), tile=tile, pixels_per_thread=args.ppt, smem_batch=args.smem_batch, capturable=True,
                                     headroom=1.02)
                rv.forward(sc)
                rg.reserve(n, int(rv.needed.records), int(rv.needed.keys))
                rzs.append(rg)
            g_l, fits_l = graphed(rzs, [x[1] for x in singles], [x[2] for x in singles], [x[3] for x in singles],
                                  [x[4] for x in singles], [x[5] for x in singles], [r.cap.records for r in rzs])
            ms_gloop, _ = timed(lambda: g_l.replay(), max(3, args.steps // 2), 2)
            loop["graphed"] = {"views_per_s": V / (ms_gloop / 1e3), "ms_per_step": ms_gloop,
                               "counts_fit": fits_l()}
            if graph:
                loop["speedup_graphed_batched_over_graphed_loop"] = ms_gloop / graph["ms_per_step"]
            del g_l, rzs

    # ---- partial rendering (Sec. 5.1.1): one image's worth of pixels over the V views ----
    partial = None
    if not args.no_partial:
        ss = rz.sample_set(V, seed=11)
        ss_strip = rz.sample_set(V, seed=11, cell="strip")

        def render_step(samples=None, masked=False):
            rz.forward(sc, samples=samples, masked=masked)
            rz.backward(sc, dimg, grads, samples=samples, masked=masked)

        modes = {}
        for name, kw in (("full", {}), ("masked_partial", {"samples": ss, "masked": True}),
                         ("thread_efficient", {"samples": ss}),
                         ("thread_efficient_strip_cells", {"samples": ss_strip})):
            ms_m, st_m = timed(lambda: render_step(**kw), max(3, args.steps // 2), 2, profile=True)
            nst = max(3, args.steps // 2)
            modes[name] = {"render_fwd_bwd_ms": round(ms_m, 4),
                           "blend_forward_ms": round(st_m.get("blend_forward", (0, 0))[0] / nst, 4),
                           "blend_backward_ms": round(st_m.get("blend_backward", (0, 0))[0] / nst, 4)}
        # the whole partial training step of Sec. 5.1 (one merged image per
        # iteration): sampled render with depth, merge, 3D distance-aware
        # D-SSIM + L1, split, sampled backward, ADC
        if (cams.width == cams.width[0]).all() and (cams.height == cams.height[0]).all():
            H0, W0 = int(cams.height[0]), int(cams.width[0])
            mimg = torch.empty(3 * H0 * W0, device=dev)
            mtgt, pts = torch.empty_like(mimg), torch.empty_like(mimg)
            sig = torch.empty(H0 * W0, device=dev)
            mhw = np.array([[H0, W0]], np.int32)
            mloss = torch.empty(1, device=dev)
            dm = torch.empty_like(mimg)
            ws3 = torch.empty(mvgs.dssim3d_workspace_size(mhw), dtype=torch.uint8, device=dev)
            pimg = torch.zeros(3 * rz.pixels, device=dev)
            pd = torch.empty_like(pimg)
            cell = rz.strip_cell()

            def partial_train_step():
                rz.forward(sc, images=pimg, samples=ss_strip, depth=True)
                rec = rz.records()
                mvgs.merge_views(rz.cams_c, V, 11, pimg, tgt, rec["depth_acc"], rec["final_T"], mimg, mtgt, pts,
                                 sig, cell=cell)
                mvgs.dssim3d_loss(mimg, mtgt, pts, sig, mhw, LAMBDA, mloss, dm, ws3)
                mvgs.split_merged_grad(rz.cams_c, V, 11, dm, pd, cell=cell)
                R = int(rz.needed.records)
                gm_p = torch.empty(max(R, 1), 2, device=dev)
                e1_p = torch.empty(max(R, 1), device=dev)
                rz.backward(sc, pd, grads, gm_p, e1_p, samples=ss_strip)
                mvgs.adc_accumulate(rz.state, n, gm_p, e1_p, *acc)

            ms_pt, st_pt = timed(partial_train_step, max(3, args.steps // 2), 2, profile=True)
            nst = max(3, args.steps // 2)
            modes["train_step_partial_3d_dssim"] = {
                "ms": round(ms_pt, 4), "merged_images_per_s": 1e3 / ms_pt,
                "stages_ms": {k: round(v[0] / nst, 4) for k, v in st_pt.items() if v[1]}}
        partial = {"group": V, "sampled_pixels": int(ss.offsets[-1].item()), "pixels": rz.pixels,
                   "sampling": "per pixel (1x1 cells); strip cells: %dx%d" % rz.strip_cell(),
                   "modes": modes,
                   "blend_speedup_thread_efficient_over_masked":
                       (modes["masked_partial"]["blend_forward_ms"] + modes["masked_partial"]["blend_backward_ms"]) /
                       max(1e-9, modes["thread_efficient"]["blend_forward_ms"] +
                           modes["thread_efficient"]["blend_backward_ms"])}

    # ---- training-loop kernels: Adam over every parameter, one densification step ----
    training = None
    if not args.no_partial:
        m_st = {k: torch.zeros_like(v) for k, v in params.items()}
        v_st = {k: torch.zeros_like(v) for k, v in params.items()}
        p_copy = {k: v.clone() for k, v in params.items()}
        t_adam = [0]

        def adam_all():
            t_adam[0] += 1
            for k in p_copy:
                mvgs.adam_step(p_copy[k], grads[k], m_st[k], v_st[k], 1e-3, t_adam[0])
        ms_adam, _ = timed(adam_all, max(3, args.steps // 2), 2)
        elems = sum(v.numel() for v in params.values())
        adam_bytes = 28 * elems  # read p, g, m, v; write p, m, v (float32)
        z = torch.randn(n, 2, 3, device=dev)
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record()
        new_p, _, _, _ = mvgs.densify(p_copy, scene.sh_degree, acc[0], acc[1], acc[2], z, 2e-4, 2e-4,
                                      float(np.log(0.02 / 0.98)), float(np.log(0.01)))
        t1e.record()
        torch.cuda.synchronize()
        peaks, _ = _peaks()
        hbm = peaks.get("hbm_gbs", 6800.0)
        training = {"adam_ms": round(ms_adam, 4),
                    "adam_roofline": {"bound": "hbm", "achieved": round(adam_bytes / (ms_adam / 1e3) / 1e9, 1),
                                      "peak": hbm, "unit": "GB/s",
                                      "frac": round(adam_bytes / (ms_adam / 1e3) / 1e9 / hbm, 4),
                                      "algorithmic": f"28 B x {elems} parameters"},
                    "densify_ms": round(t0e.elapsed_time(t1e), 3),
                    "densify_gaussians": [n, int(new_p["means"].shape[0])],
                    "densify_note": "includes one count read-back and the allocation of the outputs"}
        del m_st, v_st, p_copy, new_p

    # ---- the secondary workload: batched step and per-view loop ----
    secondary = None
    memory = None
    if not args.no_secondary and args.workload != SECONDARY_WORKLOAD:
        secondary = run_secondary(args, torch, mvgs, timed)
        memory = run_memory(torch, mvgs)

    # ---- serving loop: resident 2M SH-3 scene, Poisson arrivals ----
    serving = None
    if not args.no_serve and rank == 0:
        serving = run_serving(args, torch, mvgs)

    # ---- end to end through the C ABI with host buffers ----
    host = {k: v.cpu().pin_memory() for k, v in params.items()}
    host_tgt = tgt.cpu().pin_memory()
    host_loss = torch.empty(V, pin_memory=True)
    h2d = sum(t.numel() * 4 for t in host.values()) + host_tgt.numel() * 4
    d2h = host_loss.numel() * 4

    # Two device copies of the step's inputs: while step i computes on one,
    # the other receives step i + 1's inputs on a copy stream (each copy waits
    # until the step that last used its buffer has finished); every timed step
    # still moves its whole input from pinned host memory and reads its loss
    # back.
    params2 = {k: torch.empty_like(v) for k, v in params.items()}
    bufs = [(params, tgt, sc), (params2, torch.empty_like(tgt), mvgs.make_scene(params2, scene.sh_degree))]
    copy_stream = torch.cuda.Stream()
    used = [torch.cuda.Event(), torch.cuda.Event()]
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    e2e_i = [0]

    def issue_copy(b):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(used[b])
            for k in bufs[b][0]:
                bufs[b][0][k].copy_(host[k], non_blocking=True)
            bufs[b][1].copy_(host_tgt, non_blocking=True)
            ready[b].record(copy_stream)

    def e2e_step():
        i = e2e_i[0]
        b = i % 2
        if i == 0:
            issue_copy(0)
        issue_copy(1 - b)  # the next step's inputs, overlapped with this step
        cur = torch.cuda.current_stream()
        cur.wait_event(ready[b])
        step(rz, bufs[b][2], bufs[b][1], hw, loss, dimg, dssim_ws)
        used[b].record(cur)
        host_loss.copy_(loss, non_blocking=True)
        e2e_i[0] += 1
    ms_e2e = None if args.no_e2e else timed(e2e_step, max(3, args.steps // 2), 2)[0]
    torch.cuda.synchronize()
    del params2, bufs

    # ---- roofline of the dominant kernel ----
    roof, per_stage = roofline(stages, args, needed, rz, clk, V, rz.pixels, blended)

    out = {
        "metric": METRIC, "value": V_total / (ms_batched / 1e3), "unit": "views/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batched, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "gaussians": n, "sh_degree": scene.sh_degree, "views": V,
                   "resolutions": sorted({f"{w}x{h}" for w, h in zip(cams.width, cams.height)}),
                   "loss": "0.8 L1 + 0.2 D-SSIM (11x11, sigma 1.5)", "adc": True, "tile": args.tile,
                   "pixels_per_thread": args.ppt or "auto", "smem_batch": args.smem_batch or "auto",
                   "autotune_ms": tuning,
                   "records": needed[0], "keys": needed[1],
                   "l2": "512 MB buffer written between timed steps (L2 is 129 MB); per-step working set > 1 GB",
                   "parallelism": (f"dp{world}: a global batch of {V_total} views split between the ranks by "
                                   "pixels, one all-reduce per step of the gradients and the statistic increments"
                                   if world > 1 else "single")},
        "e2e": None if ms_e2e is None else {"value": V_total / (ms_e2e / 1e3), "unit": "views/s",
                                            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                                            "copies": "next step's inputs copied on a second stream during the "
                                                      "current step (two device buffers)"},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "per_view_loop": loop,
        "cuda_graph": graph,
        "partial_rendering": partial,
        "training_kernels": training,
        "serving": serving,
        "secondary_workload": secondary,
        "memory_at_differentiation_scale": memory,
        "stages_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in (stages or {}).items() if v[1]},
        "roofline": roof,
        "stage_roofline": per_stage,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    if dist:
        dist.destroy_process_group()
    return out


def run_secondary(args, torch, mvgs, timed):
    """Views/s of the training step on the 500k-Gaussian, 4 x 1264x832
    workload (batched, and the per-view launch loop), autotuned tile."""
    from paper_2506_12727_gb300.autotune import autotune
    dev = "cuda"
    scene, cams, _ = synth.workload(SECONDARY_WORKLOAD)
    V, n = cams.V, scene.n
    params = {k: torch.tensor(getattr(scene, k), device=dev).contiguous() for k in
              ("means", "log_scales", "quats", "opacity_logits", "sh")}
    sc = mvgs.make_scene(params, scene.sh_degree)
    tile, ppt, _, wb = autotune(sc, cams, params)
    tgt = torch.tensor(synth.pack_images(synth.make_targets(cams)), device=dev)
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    acc = [torch.zeros(n, device=dev) for _ in range(3)]

    def prepare(c, t):
        h = np.stack([c.height, c.width], 1).astype(np.int32)
        return dict(rz=mvgs.Rasterizer(c, tile=tile, pixels_per_thread=ppt, smem_batch=wb), tgt=t, hw=h,
                    loss=torch.empty(c.V, device=dev), dimg=torch.empty_like(t), gm=None, e1=None,
                    ws=torch.empty(mvgs.dssim_workspace_size(h), dtype=torch.uint8, device=dev))

    def step(d):
        img = d["rz"].forward(sc)
        mvgs.dssim_loss(img, d["tgt"], d["hw"], LAMBDA, d["loss"], d["dimg"], d["ws"])
        R = int(d["rz"].needed.records)
        if d["gm"] is None or d["gm"].shape[0] < R:
            d["gm"] = torch.empty(int(R * 1.2) + 16, 2, device=dev)
            d["e1"] = torch.empty(int(R * 1.2) + 16, device=dev)
        d["rz"].backward(sc, d["dimg"], grads, d["gm"], d["e1"])
        mvgs.adc_accumulate(d["rz"].state, n, d["gm"], d["e1"], *acc)

    batch = prepare(cams, tgt)
    steps = max(10, args.steps // 2)
    ms_b, _ = timed(lambda: step(batch), steps, max(3, args.warmup))
    off = synth.view_offsets(cams)
    singles = [prepare(cams.subset([v]), tgt[off[v]:off[v + 1]].contiguous()) for v in range(V)]
    acc_grads = {k: torch.zeros_like(v) for k, v in params.items()}

    def loop():
        for g in acc_grads.values():
            g.zero_()
        for d in singles:
            step(d)
            for k in acc_grads:
                acc_grads[k].add_(grads[k])
    ms_l, _ = timed(loop, steps, 3)
    out = {"workload": SECONDARY_WORKLOAD, "tile": f"{tile[0]}x{tile[1]}", "pixels_per_thread": ppt or "auto",
           "smem_batch": wb or "auto", "views_per_s": V / (ms_b / 1e3), "ms_per_step": ms_b,
           "per_view_loop": {"views_per_s": V / (ms_l / 1e3), "ms_per_step": ms_l,
                             "speedup_batched_over_loop": ms_l / ms_b}, "steps": steps}
    del batch, singles, params, grads, acc, acc_grads
    torch.cuda.empty_cache()
    return out


def run_memory(torch, mvgs):
    """Device memory of one differentiable step at the differentiation scale
    (1M SH-3 Gaussians, 16 views of 1024x768) against a 20 GB activation
    budget: the blend state kept from the forward for the backward (sorted
    lists, final transmittance and last contributor per pixel: the backward
    recomputes each pixel's transmittances from them instead of storing
    per-pixel lists), the workspace, and the torch allocator's peak over a
    forward + backward through the autograd function (parameters and their
    gradients included)."""
    from paper_2506_12727_gb300 import autograd
    dev = "cuda"
    scene, cams, _ = synth.workload("diff_1m_16x1024x768")
    params = {k: torch.tensor(getattr(scene, k), device=dev).contiguous() for k in
              ("means", "log_scales", "quats", "opacity_logits", "sh")}
    rz = mvgs.Rasterizer(cams, tile=(16, 64))
    need = rz.reserve_for(mvgs.make_scene(params, scene.sh_degree))
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    ps = {k: v.clone().requires_grad_(True) for k, v in params.items()}
    img = autograd.render(rz, ps, scene.sh_degree)
    img.sum().backward()
    torch.cuda.synchronize()
    peak = torch.cuda.max_memory_allocated() - base
    L = rz.layout
    # what storing each blended pair's state would cost instead (4 bytes of
    # transmittance per pair), from the pixels' blend statistics
    rz.forward(mvgs.make_scene(params, scene.sh_degree), stats=True)
    blended = int(rz.records()["pixel_stats"].to(torch.int64)[:, 1].sum().item())
    out = {"workload": "diff_1m_16x1024x768", "records": int(need.records), "keys": int(need.keys),
           "state_bytes": int(L.state_bytes), "workspace_bytes": int(L.workspace_bytes),
           "step_peak_bytes": int(peak), "budget_bytes": 20 * 10**9,
           "stored_per_pair_state_bytes": 4 * blended,
           "reading": "the backward recomputes the transmittances from the final T and the last contributor; "
                      "state + workspace and the step's peak are the bytes against the 20 GB budget"}
    del ps, img, rz, params
    torch.cuda.empty_cache()
    return out


def run_serving(args, torch, mvgs):
    """Continuous-batching serving of Poisson requests (1-16 views each, 640x480
    / 1280x720 / 1920x1080, poses on a radius 3..5 shell) against a resident
    scene of 2M SH-3 Gaussians; latency from arrival to the completion of the
    request's batch on the device.

    First the closed-loop capacity (requests/s with the queue always full),
    then two Poisson traces of about 10 s of work each: at the configured rate
    (200 req/s, far above one GPU's capacity for this scene: the queue grows
    and latency measures the backlog) and at 70% of the measured capacity."""
    from paper_2506_12727_gb300 import serve
    import time as _time
    scene = synth.make_scene(2_000_000, 3, seed=synth.SEED_SCENE)
    params = {k: torch.tensor(getattr(scene, k), device="cuda").contiguous() for k in
              ("means", "log_scales", "quats", "opacity_logits", "sh")}
    pool = synth.poisson_requests(400, rate_hz=args.serve_rate)
    cams = [synth.make_cameras(r["resolutions"], radius=(3.0, 5.0), seed=r["cam_seed"]) for r in pool]

    def server(coalesce_ms=0.0, coalesce_views=0):
        return serve.Server(params, 3, tile=(16, 64), slots=2, max_views=32, max_pixels=40_000_000,
                            memory_budget=96 << 30, coalesce_ms=coalesce_ms, coalesce_views=coalesce_views)

    out = {"scene": "2M SH-3 resident", "tile": "16x64", "slots": 2,
           "latency": "arrival to completion of the request's batch on the device; images stay on the device"}
    # warm-up and closed-loop capacity
    srv = server()
    serve.run_trace(srv, [serve.Request(i, cams[i]) for i in range(6)], [0.0] * 6, realtime=False, timeout_s=120)
    cap_reqs = [serve.Request(i, cams[i]) for i in range(6, 30)]
    wall = serve.run_trace(srv, cap_reqs, [0.0] * len(cap_reqs), realtime=False, timeout_s=120)
    done = [r for r in cap_reqs if r.error is None]
    cap_rps = len(done) / wall
    out["capacity"] = {"requests_per_s": cap_rps, "views_per_s": sum(r.views for r in done) / wall,
                       "requests": len(cap_reqs), "failed": len(cap_reqs) - len(done)}
    srv.close()
    traces = {}
    # (name, offered rate, coalescing window ms, coalescing target views)
    runs = (("configured_rate", args.serve_rate, 0.0, 0), ("at_70pct_capacity", 0.7 * cap_rps, 0.0, 0),
            ("at_70pct_capacity_coalesced", 0.7 * cap_rps, 40.0, 24))
    for name, rate, cms, cviews in runs:
        n = int(min(len(pool) - 30, max(8, cap_rps * 10.0)))  # about 10 s of work
        rng = np.random.default_rng(3)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
        reqs = [serve.Request(30 + i, cams[30 + i]) for i in range(n)]
        srv = server(cms, cviews)
        wall = serve.run_trace(srv, reqs, list(arrivals - arrivals[0]), realtime=True, timeout_s=60)
        srv.close()
        st = serve.latency_summary(reqs)
        log = srv.batch_log
        st.update({"offered_requests_per_s": rate, "wall_s": wall, "views_per_s": st["views"] / wall,
                   "coalesce_ms": cms, "coalesce_views": cviews, "batches": len(log),
                   "mean_requests_per_batch": float(np.mean([b[3] for b in log])) if log else 0,
                   "mean_views_per_batch": float(np.mean([b[1] for b in log])) if log else 0,
                   # per batch: device time of the render call (CUDA events on the
                   # worker's stream) and host time from taking the batch to its
                   # completion (adds the two count read-backs' waits, launches and
                   # the Python around the call)
                   "batch_device_ms_mean": float(np.mean([b[4] for b in log])) if log else 0,
                   "batch_host_ms_mean": float(np.mean([b[5] for b in log])) if log else 0})
        traces[name] = st
    out["traces"] = traces
    main = traces["configured_rate"]
    out.update({"p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"], "views_per_s": main["views_per_s"]})
    del params
    torch.cuda.empty_cache()
    return out


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def stage_work(rz, needed, V, pixels, blended):
    """Algorithmic work of each stage for one step: (bound, amount, unit).
    Bytes are what the stage must read and write in HBM (each array once);
    FLOPs are counted on blended pairs only (see FWD_/BWD_FLOP_PER_BLENDED)."""
    R, K = needed
    n = rz.n
    tiles = int(rz.layout.tiles)
    bits = max(1, int(np.ceil(np.log2(max(tiles, 2)))))
    passes = max(1, (bits + 7) // 8)
    vb = max(1, int(R - 1).bit_length())  # record-id bits
    if passes == 2 and (bits - 8) + vb <= 32:
        # packed two-pass tile sort: duplication writes a 16-bit tile id and a
        # record id, pass 0 reads them and writes one word, pass 1 reads it
        # twice (histogram, scatter) and writes the record id; the duplication
        # reads each record's id, descriptor and entry offset
        tile_sort_bytes = 28.0 * K + 20.0 * R
    else:
        tile_sort_bytes = 8.0 * K + passes * 16.0 * K - 4.0 * K + 20.0 * R
    return {
        "count_visible": ("hbm", 44.0 * n + 4.0 * n + n * V, "B"),
        "scan_records": ("hbm", 12.0 * n, "B"),
        "preprocess": ("hbm", 236.0 * n + n * V + 8.0 * n + 76.0 * R, "B"),
        "depth_sort": ("hbm", 4 * 16.0 * R, "B"),
        "scan_tiles": ("hbm", 12.0 * R, "B"),
        "tile_sort": ("hbm", tile_sort_bytes, "B"),
        "ranges": ("hbm", 8.0 * R + 24.0 * tiles, "B"),
        "blend_forward": ("alu", FWD_FLOP_PER_BLENDED * blended, "FLOP"),
        "zero_grads": ("hbm", 56.0 * R, "B"),  # 8 float and 3 double slots per record
        "blend_backward": ("alu", BWD_FLOP_PER_BLENDED * blended, "FLOP"),
        "preprocess_backward": ("hbm", 472.0 * n + 76.0 * R, "B"),
        "dssim": ("hbm", 44.0 * 3 * pixels, "B"),
        "adc": ("hbm", 12.0 * R + 32.0 * n, "B"),
    }, blended


# DRAM bytes (read + write) per launch of the blend kernels, from the ncu
# launch list of one headline step (dram__bytes_read.sum +
# dram__bytes_write.sum).  Valid only for that workload and launch
# configuration and for the blend sources it was taken on (their hash is
# kept with it); otherwise the line reports no traffic.
BLEND_TRAFFIC = {
    "workload": "uneven_3m_8views", "tile": "32x64", "smem_batch": 64, "blended": 2118024889,
    "blend_forward": 3720.0e6 + 170.8e6,
    "blend_backward": 7450.7e6 + 419.6e6,
    "capture": "profiles/launches_uneven_3m_8views.md",
    "sources_sha256": "a114b24ee0915ba63bfb74ce3df782c2859888aed9232cb2cd9b4c1a09a8e591",
}


def blend_sources_hash():
    """SHA-256 of the blend sources' code: comments and blank lines left out,
    so that a comment edit does not invalidate a capture."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("blend.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2506_12727_gb300", "csrc", f)) as fh:
            for line in fh:
                code = re.sub(r"//.*$", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def roofline(stages, args, needed, rz, clk, V, pixels, blended):
    """Per-stage achieved / peak, and the dominant stage's entry."""
    if not stages:
        return None, None
    import torch
    peaks, src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1455.0)
    alu_peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    work, blended = stage_work(rz, needed, V, pixels, blended)
    table = {}
    for name, (ms_total, launches) in stages.items():
        if not launches or name not in work:
            continue
        bound, amount, unit = work[name]
        ms = ms_total / args.steps  # per step (a stage may launch several kernels)
        if bound == "alu":
            ach = amount / (ms / 1e3) / 1e12
            table[name] = {"bound": "alu", "ms": round(ms, 4), "achieved": round(ach, 3), "peak": round(alu_peak, 2),
                           "unit": "TFLOP/s", "frac": round(ach / alu_peak, 4)}
        else:
            ach = amount / (ms / 1e3) / 1e9
            table[name] = {"bound": "hbm", "ms": round(ms, 4), "achieved": round(ach, 1), "peak": hbm,
                           "unit": "GB/s", "frac": round(ach / hbm, 4)}
    dom = max(table, key=lambda k: table[k]["ms"])
    d = dict(table[dom])
    d.pop("ms")
    d["kernel"] = dom
    d["traffic"] = None
    if dom in ("blend_forward", "blend_backward") and blended:
        same_launch = (args.workload == BLEND_TRAFFIC["workload"] and
                       f"{rz.cfg.tile_w}x{rz.cfg.tile_h}" == BLEND_TRAFFIC["tile"] and
                       rz.cfg.smem_batch == BLEND_TRAFFIC["smem_batch"] and blended == BLEND_TRAFFIC["blended"])
        if not same_launch:
            d["traffic_source"] = "null: no ncu capture of this workload and launch configuration"
        elif BLEND_TRAFFIC["sources_sha256"] != blend_sources_hash():
            d["traffic_source"] = "null: no ncu capture of the current blend sources"
        else:
            d["traffic"] = int(BLEND_TRAFFIC[dom])
            d["traffic_source"] = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel's launch "
                                   f"in {BLEND_TRAFFIC['capture']} (same workload, tile, batch and sources)")
    if d["bound"] == "alu":
        per = FWD_FLOP_PER_BLENDED if dom == "blend_forward" else BWD_FLOP_PER_BLENDED
        d["algorithmic"] = f"{per} FLOP x {blended} blended (pixel, Gaussian) pairs per launch"
        d["peak_source"] = f"{sms} SMs x 128 FP32 lanes x 2 FLOP x {mhz:.0f} MHz (sampled SM clock)"
    else:
        d["peak_source"] = f"MEASURED_PEAKS.json hbm_gbs ({src})"
    return d, table


# ---------------------------------------------------------------------------
# the CPU oracle
# ---------------------------------------------------------------------------
ORACLE_TILE = (16, 16)  # the oracle's own binning tile (its images do not depend on it)
_ORACLE_INPUTS = {}


def _oracle_threads():
    return max(1, min(64, os.cpu_count() or 1))


def _oracle_inputs(workload, threads):
    """The seeded scene, cameras and targets of a workload, and the scene cut
    into one contiguous chunk of Gaussians per host thread (generated once per
    process: generation is not part of a sample)."""
    key = (workload, threads)
    if key not in _ORACLE_INPUTS:
        scene, cams, _ = synth.workload(workload)
        chunks = np.array_split(np.arange(scene.n), threads)
        _ORACLE_INPUTS[key] = (scene, cams, synth.make_targets(cams), [(c, scene.subset(c)) for c in chunks])
    return _ORACLE_INPUTS[key]


def oracle_sample(workload, view=0, window=None, threads=None):
    """One bounded sample of the workload on the oracle: projection, sort,
    blend, loss and backward of one view, or of a pixel window of it, with
    the host threads sharing the work (ctypes releases the GIL while the
    oracle's C routines run): projection and 3D gradients over chunks of
    Gaussians, sort, blend and blend backward over row bands of the window,
    each band with the loss of its own pixels.  Returns (seconds, fraction of
    a full view covered, threads used)."""
    import concurrent.futures as cf
    import oracle
    nt = threads or _oracle_threads()
    scene, cams, targets, chunks = _oracle_inputs(workload, nt)
    c1 = cams.subset([view])
    H, W = int(c1.height[0]), int(c1.width[0])
    x0, y0, x1, y1 = window if window is not None else (0, 0, W, H)
    tg = targets[view]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(nt) as ex:
        parts = list(ex.map(lambda c: oracle.project(c[1], c1, ORACLE_TILE), chunks))
        P = {k: np.concatenate([p[k] for p in parts]) for k in parts[0] if isinstance(parts[0][k], np.ndarray)}
        P["N"], P["V"], P["tile"] = scene.n, 1, ORACLE_TILE
        rows = np.array_split(np.arange(y0, y1), max(1, min(nt, (y1 - y0) // 16)))

        def band(r):
            win = np.array([[x0, int(r[0]), x1, int(r[-1]) + 1]], np.int32)
            S = oracle.sort_keys(c1, ORACLE_TILE, P["valid"], P["rect"], P["depth"].astype(np.float32), win)
            img, _, _, _ = oracle.render(c1, P, S, (0.0, 0.0, 0.0), win)
            ya, yb = int(r[0]), int(r[-1]) + 1
            sub = img.reshape(3, H, W)[:, ya:yb, x0:x1]
            _, _, g = oracle.dssim_l1_loss([sub], [tg[:, ya:yb, x0:x1]], LAMBDA)
            d = np.zeros((3, H, W))
            d[:, ya:yb, x0:x1] = g[0]
            g2d, _ = oracle.render_backward(c1, P, S, d.reshape(-1), (0.0, 0.0, 0.0), win)
            return g2d
        g2d = None
        for part in ex.map(band, rows):
            g2d = part if g2d is None else g2d + part
        list(ex.map(lambda c: oracle.project_backward(c[1], c1, ORACLE_TILE, g2d[c[0]]), chunks))
    dt = time.perf_counter() - t0
    return dt, ((x1 - x0) * (y1 - y0)) / float(H * W), nt


def cpu_baseline(workload, views=2):
    """The oracle on the host's cores over the first `views` views of the
    workload at full resolution (forward + loss + backward of each)."""
    _, cams, _, _ = _oracle_inputs(workload, _oracle_threads())
    views = min(views, cams.V)
    secs, frac, nt = 0.0, 0.0, 1
    for v in range(views):
        dt, f, nt = oracle_sample(workload, view=v)
        secs += dt
        frac += f
    return {"value": frac / secs, "unit": "views/s", "cores": nt, "kind": "oracle",
            "sample": f"views 0-{views - 1} of {workload} at full resolution (the first {views} of the batch), "
                      f"forward + loss + backward, {nt} host threads (projection and 3D gradients by chunks of "
                      "Gaussians, blend and its backward by row bands with each band's own loss)",
            "seconds": secs}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    nt = _oracle_threads()
    scene, cams, _, _ = _oracle_inputs(args.workload, nt)
    # each step is one square window at the centre of one view (views in
    # turn), sized so that the whole run stays within about two and a half
    # minutes: the projection and 3D gradients of the whole scene are a
    # fixed cost per step, the window's pixels the rest
    t_fixed, _, _ = oracle_sample(args.workload, view=0, window=(0, 0, 8, 8))
    t_64, _, _ = oracle_sample(args.workload, view=0, window=(0, 0, 64, 64))
    per_px = max(t_64 - t_fixed, 1e-3) / 4096.0
    per_step = 150.0 / max(1, args.steps + args.warmup)
    side = 32
    for s in (512, 384, 256, 192, 128, 96, 64, 48):
        if t_fixed + s * s * per_px <= per_step:
            side = s
            break

    def win(v):
        W, H = int(cams.width[v]), int(cams.height[v])
        sd = min(side, W, H)
        return (W // 2 - sd // 2, H // 2 - sd // 2, W // 2 - sd // 2 + sd, H // 2 - sd // 2 + sd)
    for i in range(args.warmup):
        oracle_sample(args.workload, view=i % cams.V, window=win(i % cams.V))
    times, fracs = [], []
    for i in range(args.steps):
        dt, frac, _ = oracle_sample(args.workload, view=i % cams.V, window=win(i % cams.V))
        times.append(dt)
        fracs.append(frac)
    ms = 1e3 * sum(times) / len(times)
    value = sum(fracs) / sum(times)
    sample = (f"a {side}x{side} window at the centre of one view of {args.workload} per step (views in turn), "
              f"forward + loss + backward, {nt} host threads")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "gaussians": scene.n, "views": cams.V,
                       "tile": f"{ORACLE_TILE[0]}x{ORACLE_TILE[1]}"},
            "cpu_baseline": {"value": value, "unit": "views/s", "cores": nt, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    out = run_reference(args, rank, world) if args.impl == "reference" else run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
