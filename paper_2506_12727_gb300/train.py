"""Multi-view training loop (Sec. 5) on top of the library's calls.

Each iteration takes `views_per_iter` cameras and either
  - renders them fully and uses (1 - lambda) L1 + lambda D-SSIM per view
    (mvgs_render_views, mvgs_dssim_loss), or
  - (partial=True) renders one image's worth of pixels spread over them with
    thread-efficient partial rendering (Alg. 3, group = views_per_iter, a new
    seeded sample set per iteration) and uses the same loss with the 3D
    distance-aware D-SSIM on the merged image (Sec. 5.1.2; mvgs_render_views_
    sampled with the depth output, mvgs_merge_views, mvgs_dssim3d_loss,
    mvgs_split_merged_grad);
then back-propagates (mvgs_render_views[_sampled]_backward), adds the ADC
statistics E_1 / E_2 (mvgs_adc_accumulate) and takes an Adam step per
parameter group (mvgs_adam_step).  With a process group (one process per
GPU, full renders only), the iteration's views are split between the ranks
and one all-reduce per step sums the gradients and the statistics'
increments (shard.ViewShardedStep), so every rank holds the same Gaussians.
Every `densify_every` iterations the multi-view densification step (mvgs_densify: split by mean E_1, clone by mean
E_2, prune with the opacity threshold times the views per iteration, as the
supplement prescribes) replaces the Gaussians; the Adam moments follow them
(mvgs_densify_carry) and the statistics restart.

Every step of the computation runs in the library's kernels; this module
moves tensors between the calls.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import mvgs
from .serve import CameraBatch, _subset
from .shard import ViewShardedStep

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")
DEFAULT_LR = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, opacity_logits=5e-2, sh=2.5e-3)


class MultiViewTrainer:
    def __init__(self, params: dict, sh_degree: int, cams, targets, views_per_iter=4, tile=(16, 16),
                 partial=False, lam=0.2, lr=None, densify_every=0, split_threshold=2e-4, clone_threshold=2e-4,
                 prune_opacity=0.005, dense_extent=0.01, seed=0, device="cuda", cell=(1, 1), process_group=None):
        """`cams`: all training cameras (numpy camera set); `targets`: list of
        [3, H, W] device tensors, one per camera.  Thresholds are in the units
        of the statistics (pixel-space gradient norms, averaged over views).
        `process_group`: a torch.distributed group over which each
        iteration's views are sharded (every rank must pass the same seed,
        cameras and parameters); None trains in this process alone."""
        self.p = {k: params[k].detach().clone().contiguous() for k in PARAMS}
        self.sh_degree = sh_degree
        self.cams = cams
        self.targets = targets
        self.V = views_per_iter
        self.tile = tuple(tile)
        self.partial = partial
        self.cell = cell  # partial sampling cell: (1, 1) pixel by pixel, "strip" one warp strip
        self.lam = lam
        self.lr = dict(DEFAULT_LR, **(lr or {}))
        self.densify_every = densify_every
        self.thresholds = (split_threshold, clone_threshold,
                           math.log(prune_opacity * views_per_iter / (1.0 - prune_opacity * views_per_iter)),
                           math.log(dense_extent))
        self.rng = np.random.default_rng(seed)
        self.device = device
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.t = 0
        self.rz = None
        rank, world = 0, 1
        if process_group is not None:
            import torch.distributed as dist
            rank, world = dist.get_rank(process_group), dist.get_world_size(process_group)
        if partial and world > 1:
            raise ValueError("partial rendering merges the views of an iteration: it is not sharded over ranks")
        self.shard = ViewShardedStep(rank, world, process_group)
        self._reset_stats()

    def _reset_stats(self):
        n = self.p["means"].shape[0]
        self.acc = [torch.zeros(n, device=self.device) for _ in range(3)]

    @property
    def n(self) -> int:
        return int(self.p["means"].shape[0])

    def _views(self, ids):
        cams = CameraBatch([_subset(self.cams, list(ids))])
        if self.rz is None:
            self.rz = mvgs.Rasterizer(cams, tile=self.tile, device=self.device)
        else:
            self.rz.set_cameras(cams)
        tgt = torch.cat([self.targets[i].reshape(-1) for i in ids]).contiguous()
        return cams, tgt

    def step(self, ids=None) -> float:
        """One iteration on the views `ids` (default: a random draw).  Returns
        the mean loss over the views (or merged images)."""
        if ids is None:
            ids = self.rng.choice(self.cams.V, size=self.V, replace=False)
        ids = [int(i) for i in ids]
        pixels = [int(self.cams.width[i]) * int(self.cams.height[i]) for i in ids]
        grads, incr, loss_sum = self.shard.run(pixels, lambda own, scale: self._local_step(ids, own, scale))
        for a, d in zip(self.acc, incr):
            a.add_(d)
        self.t += 1
        for k in PARAMS:
            mvgs.adam_step(self.p[k], grads[k], self.m[k], self.v[k], self.lr[k], self.t)
        if self.densify_every and self.t % self.densify_every == 0:
            self.densify()
        return float(loss_sum.item()) / (1 if self.partial else len(ids))

    def _local_step(self, ids, own, scale):
        """This process's share of an iteration: render, loss and backward of
        the views ids[own]; returns the gradients of scale x their mean loss,
        this step's ADC increments and the sum of their losses."""
        grads = {k: torch.zeros_like(v) for k, v in self.p.items()}
        incr = [torch.zeros(self.n, device=self.device) for _ in range(3)]
        if not own:
            return grads, incr, torch.zeros(1, device=self.device)
        cams, tgt = self._views([ids[i] for i in own])
        rz = self.rz
        sc = mvgs.make_scene(self.p, self.sh_degree)
        hw = np.stack([cams.height, cams.width], 1).astype(np.int32)
        if not self.partial:
            img = rz.forward(sc)
            loss = torch.empty(cams.V, device=self.device)
            dimg = torch.empty_like(img)
            ws = torch.empty(mvgs.dssim_workspace_size(hw), dtype=torch.uint8, device=self.device)
            mvgs.dssim_loss(img, tgt, hw, self.lam, loss, dimg, ws)
            if scale != 1.0:
                dimg.mul_(scale)
            samples = None
        else:
            if not (cams.width == cams.width[0]).all() or not (cams.height == cams.height[0]).all():
                raise ValueError("partial rendering merges views of one resolution")
            samples = rz.sample_set(cams.V, seed=int(self.t), cell=self.cell)
            cell = rz.strip_cell() if self.cell == "strip" else self.cell
            img = torch.zeros(3 * rz.pixels, device=self.device)
            rz.forward(sc, images=img, samples=samples, depth=True)
            rec = rz.records()
            H, W = int(cams.height[0]), int(cams.width[0])
            mimg = torch.empty(3 * H * W, device=self.device)
            mtgt = torch.empty_like(mimg)
            pts = torch.empty_like(mimg)
            sig = torch.empty(H * W, device=self.device)
            mvgs.merge_views(rz.cams_c, cams.V, int(self.t), img, tgt, rec["depth_acc"], rec["final_T"], mimg, mtgt,
                             pts, sig, cell=cell)
            mhw = np.array([[H, W]], np.int32)
            loss = torch.empty(1, device=self.device)
            dm = torch.empty_like(mimg)
            ws = torch.empty(mvgs.dssim3d_workspace_size(mhw), dtype=torch.uint8, device=self.device)
            mvgs.dssim3d_loss(mimg, mtgt, pts, sig, mhw, self.lam, loss, dm, ws)
            dimg = torch.empty_like(img)
            mvgs.split_merged_grad(rz.cams_c, cams.V, int(self.t), dm, dimg, cell=cell)
        R = int(rz.needed.records)
        gm2d = torch.empty(max(R, 1), 2, device=self.device)
        e1 = torch.empty(max(R, 1), device=self.device)
        rz.backward(sc, dimg, grads, gm2d, e1, samples=samples)
        mvgs.adc_accumulate(rz.state, self.n, gm2d, e1, *incr)
        return grads, incr, loss.sum().reshape(1)

    def densify(self):
        """The multi-view densification step on the statistics gathered since
        the last one."""
        z = torch.tensor(self.rng.standard_normal((self.n, 2, 3)), dtype=torch.float32, device=self.device)
        carry = [self.m[k] for k in PARAMS] + [self.v[k] for k in PARAMS]
        new, src, kind, moved = mvgs.densify(self.p, self.sh_degree, self.acc[0], self.acc[1], self.acc[2], z,
                                             *self.thresholds, carry=carry)
        self.p = new
        self.m = dict(zip(PARAMS, moved[:5]))
        self.v = dict(zip(PARAMS, moved[5:]))
        self._reset_stats()
        return src, kind
