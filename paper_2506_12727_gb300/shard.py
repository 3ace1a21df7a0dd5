"""View-sharded data parallelism: one process per GPU, each holding a replica
of the Gaussians.

A global batch of V views is split between the ranks (balanced by pixel
count, the unit the blend kernels' work follows); every rank renders and
back-propagates its own views with the single-GPU library, then ONE
all-reduce (sum) of a flat bucket makes every rank's step identical.  The
bucket holds
  - the 3D parameter gradients of this step, each rank's taken for the loss
    of the whole batch: the batch loss is the mean of the V per-view losses,
    so a rank holding V_r views scales the gradient of its own views' mean
    loss by V_r / V before the sum;
  - this step's INCREMENTS of the densification statistics -- E_1 and E_2
    (Sec. 5.2.2: sums over views of per-view norms) and the visible-view
    counts -- never the running accumulators: per-view terms add across
    ranks, so the sum of the increments is the single-process increment,
    while summing running accumulators would multiply every earlier step's
    statistics by the number of ranks;
  - the sum of the rank's per-view losses (for reporting).
Every rank then adds the reduced increments to its own accumulators and takes
the same optimiser step and the same densification decisions.
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


class Bucket:
    """A flat buffer holding a fixed list of tensors of one dtype back to
    back, exchanged with one collective.  The buffer is kept between steps
    (it is re-made only when the total size, dtype or device changes)."""

    def __init__(self):
        self.flat = None

    def allreduce_sum_(self, tensors, group=None):
        import torch.distributed as dist
        n = sum(t.numel() for t in tensors)
        dev, dt = tensors[0].device, tensors[0].dtype
        if self.flat is None or self.flat.numel() != n or self.flat.device != dev or self.flat.dtype != dt:
            self.flat = torch.empty(n, dtype=dt, device=dev)
        off = 0
        for t in tensors:
            assert t.dtype == dt and t.is_contiguous()
            self.flat[off:off + t.numel()].copy_(t.reshape(-1))
            off += t.numel()
        dist.all_reduce(self.flat, op=dist.ReduceOp.SUM, group=group)
        off = 0
        for t in tensors:
            t.reshape(-1).copy_(self.flat[off:off + t.numel()])
            off += t.numel()
        return tensors


class ViewShardedStep:
    """The host side of one view-sharded training step.

    `local_step(views, grad_scale)` does this rank's device work for the
    batch views `views` (indices into the global batch; possibly none) and
    returns (grads, increments, loss_sum): the parameter gradients of
    grad_scale x the mean loss over `views` (a dict of tensors), this
    step's ADC increments [E_1, E_2, visible-view count] (three [N]
    tensors) and the sum of the per-view losses (a one-element tensor), all
    of one dtype (float32 from the library).  run() exchanges them and returns the reduced values,
    identical on every rank."""

    def __init__(self, rank: int = 0, world: int = 1, group=None):
        self.rank, self.world, self.group = rank, world, group
        self.bucket = Bucket()

    def views(self, pixels) -> tuple[list[int], float]:
        """This rank's views of a batch with these per-view pixel counts,
        and the scale of their mean-loss gradient (own views / batch views)."""
        own = shard_views(pixels, self.rank, self.world) if self.world > 1 else list(range(len(pixels)))
        return own, len(own) / float(len(pixels))

    def exchange(self, grads, incr, loss_sum):
        """Sums this rank's gradients, statistic increments and loss sum
        over the ranks, in place, with one collective."""
        if self.world > 1:
            keys = sorted(grads)
            self.bucket.allreduce_sum_([grads[k] for k in keys] + list(incr) + [loss_sum], self.group)
        return grads, incr, loss_sum

    def run(self, pixels, local_step):
        own, scale = self.views(pixels)
        return self.exchange(*local_step(own, scale))
