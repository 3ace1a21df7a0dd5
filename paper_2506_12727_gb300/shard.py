"""View-sharded data parallelism: one process per GPU, each holding a replica
of the Gaussians.

A batch of V views is split between the ranks (balanced by pixel count, the
unit the blend kernels' work follows); every rank renders and back-propagates
its own views with the single-GPU library, then one all-reduce (sum) of the
3D parameter gradients and of the densification accumulators makes every
rank's state identical, so each takes the same optimiser step.  E_1 and E_2
(Sec. 5.2.2) are sums of per-view norms, so summing them over ranks keeps the
per-view separation; the visible-view counts add likewise.  A loss averaged
over all V views needs each rank to scale its views' gradient by 1/V (not by
its own view count) before the sum.
"""
from __future__ import annotations

import torch


def shard_views(pixels, rank: int, world: int) -> list[int]:
    """The views of `rank`: the largest views first, each to the rank with the
    fewest pixels so far (ties to the lowest rank); deterministic, so every
    rank computes the same split."""
    load = [0] * world
    owner = {}
    for v in sorted(range(len(pixels)), key=lambda i: (-int(pixels[i]), i)):
        r = min(range(world), key=lambda j: (load[j], j))
        owner[v] = r
        load[r] += int(pixels[v])
    return [v for v in range(len(pixels)) if owner[v] == rank]


def allreduce_sum_(tensors, group=None):
    """Sums each tensor over the ranks, in place (one collective per tensor,
    issued in a fixed order on every rank)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def reduce_step(grads: dict, accumulators=(), group=None):
    """The per-iteration exchange of a view-sharded step: gradients of every
    parameter tensor and the ADC accumulators, summed over the ranks."""
    keys = sorted(grads)
    allreduce_sum_([grads[k] for k in keys] + list(accumulators), group)
    return grads
