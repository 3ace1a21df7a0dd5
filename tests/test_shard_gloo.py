"""View-sharded data parallelism on CPU ranks (gloo): the product's exchange
logic (shard.ViewShardedStep: view split, gradient scale, one flat bucket of
gradients and per-step statistic increments) with the oracle standing in
for each rank's GPU.  Over several steps -- parameters updated from the
reduced gradients, statistics accumulated from the reduced increments, then
a densification decision -- two ranks reproduce the single-rank run over the
same global batches."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from oracle import densify as odensify

# the sharding helpers need no GPU; import the module file directly so the
# CUDA binding (which needs the built library) is not loaded here
import importlib.util

_HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location(
    "shard", os.path.join(os.path.dirname(_HERE), "paper_2506_12727_gb300", "shard.py"))
shard = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(shard)

TILE = (16, 16)
STEPS = 3
LR = 2e-3
FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _case():
    scene = synth.make_scene(300, 3, seed=51)
    scene.log_scales += np.float32(0.5)
    cams = synth.make_cameras([(48, 40), (64, 32), (40, 40), (56, 24), (32, 48), (40, 56), (24, 24)], radius=3.0,
                              seed=52)
    # the global batch of each step (view indices into `cams`) and the weights
    # of a loss linear in each view's image
    rng = np.random.default_rng(53)
    batches = [list(rng.choice(cams.V, size=5, replace=False)) for _ in range(STEPS)]
    _, _, _, pix_base = oracle.layout(cams, TILE)
    w = [rng.normal(size=3 * int(cams.pixels()[v])) for v in range(cams.V)]
    return scene, cams, batches, w


def _local_step(scene, cams, w, batch, own, scale):
    """One rank's share, by the oracle: gradients of scale x the mean over
    `own` of the per-view losses L_v = w_v . image_v, the ADC increments and
    the loss sum (float64 tensors)."""
    n = scene.n
    grads = {k: torch.zeros(getattr(scene, k).shape, dtype=torch.float64) for k in FIELDS}
    incr = [torch.zeros(n, dtype=torch.float64) for _ in range(3)]
    if not own:
        return grads, incr, torch.zeros(1, dtype=torch.float64)
    views = [batch[i] for i in own]
    sub = cams.subset(views)
    ref = oracle.forward(scene, sub, TILE)
    _, _, _, spb = oracle.layout(sub, TILE)
    loss = sum(float(w[v] @ ref["img"][3 * spb[i]:3 * spb[i + 1]]) for i, v in enumerate(views))
    d = np.concatenate([w[v] for v in views]) * (scale / len(views))
    g, g2d, e1 = oracle.backward(scene, sub, ref, d, TILE)
    E1, E2, _, denom = oracle.adc_statistics(g2d, e1, ref["P"]["valid"], len(views))
    for k in FIELDS:
        grads[k] = torch.tensor(g[k].reshape(grads[k].shape))
    incr = [torch.tensor(E1), torch.tensor(E2), torch.tensor(denom.astype(np.float64))]
    return grads, incr, torch.tensor([loss], dtype=torch.float64)


def _train(rank, world, group=None):
    """STEPS sharded steps (SGD on the reduced gradients, statistics from the
    reduced increments), then the densification decision."""
    scene, cams, batches, w = _case()
    step = shard.ViewShardedStep(rank, world, group)
    acc = [torch.zeros(scene.n, dtype=torch.float64) for _ in range(3)]
    losses, owned = [], []
    for batch in batches:
        pixels = [int(cams.pixels()[v]) for v in batch]
        owned.append(step.views(pixels)[0])
        grads, incr, loss_sum = step.run(pixels, lambda own, scale: _local_step(scene, cams, w, batch, own, scale))
        for a, d in zip(acc, incr):
            a += d
        losses.append(float(loss_sum) / len(batch))
        for k in FIELDS:
            arr = getattr(scene, k)
            arr[...] = (arr.astype(np.float64) - LR * grads[k].numpy()).astype(np.float32)
    acc = [a.numpy() for a in acc]
    m1 = acc[0] / np.maximum(acc[2], 1)
    m2 = acc[1] / np.maximum(acc[2], 1)
    dec = odensify.decide(scene.log_scales, scene.opacity_logits, acc[0], acc[1], acc[2],
                          float(np.median(m1[acc[2] > 0])), float(np.median(m2[acc[2] > 0])),
                          float(np.log(0.05 / 0.95)), float(np.median(scene.log_scales.max(1))))
    return dict(params={k: getattr(scene, k).copy() for k in FIELDS}, acc=acc, losses=losses, owned=owned,
                decisions={k: dec[k] for k in ("pruned", "split", "cloned")})


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    out[rank] = _train(rank, world, None)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_views_balances_and_partitions():
    pixels = [1920 * 1080, 1264 * 832, 800 * 600, 1600 * 1067, 1920 * 1080, 800 * 600, 1264 * 832, 1600 * 1067]
    for world in (1, 2, 3, 4, 8):
        parts = [shard.shard_views(pixels, r, world) for r in range(world)]
        assert sorted(v for p in parts for v in p) == list(range(len(pixels)))
        loads = [sum(pixels[v] for v in p) for p in parts]
        assert max(loads) - min(loads) <= max(pixels)


def test_views_and_gradient_scale():
    step = shard.ViewShardedStep(1, 3)
    own, scale = step.views([100, 90, 80, 70, 60])
    assert own == [1, 4] and scale == 2 / 5
    own, scale = shard.ViewShardedStep(0, 1).views([5, 5])
    assert own == [0, 1] and scale == 1.0
    # more ranks than views: a rank may hold none
    own, scale = shard.ViewShardedStep(3, 4).views([5, 5])
    assert own == [] and scale == 0.0


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_steps_reproduce_the_single_rank_run(world):
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    single = _train(0, 1)
    runs = [out[r] for r in range(world)]
    for s in range(STEPS):
        views = sorted(v for r in runs for v in r["owned"][s])
        assert views == list(range(5)) and all(len(r["owned"][s]) for r in runs)
    for r in runs:
        for k in FIELDS:
            # parameters after three updates: equal up to the order of the
            # float64 sums, then identical float32 roundings on every rank
            np.testing.assert_allclose(r["params"][k], single["params"][k], rtol=1e-6, atol=1e-7)
            np.testing.assert_array_equal(r["params"][k], runs[0]["params"][k])
        for a, b in zip(r["acc"], single["acc"]):
            np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)
        np.testing.assert_array_equal(r["acc"][2], single["acc"][2])  # visible-view counts, exact
        np.testing.assert_allclose(r["losses"], single["losses"], rtol=1e-9)
        for k in ("pruned", "split", "cloned"):
            np.testing.assert_array_equal(r["decisions"][k], single["decisions"][k])
    # the statistics accumulated over the steps (not multiplied by the ranks)
    assert single["acc"][2].max() >= STEPS
    assert single["decisions"]["split"].sum() > 0 and single["decisions"]["cloned"].sum() > 0
