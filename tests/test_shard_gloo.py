"""View-sharded data parallelism on CPU ranks (gloo, world size 2): each rank
computes the gradients and ADC statistics of its share of the views (with the
oracle standing in for its GPU), one all-reduce sums them, and the result
equals the single-rank computation over all views."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth

# the sharding helpers need no GPU; import the module file directly so the
# CUDA binding (which needs the built library) is not loaded here
import importlib.util

_HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location(
    "shard", os.path.join(os.path.dirname(_HERE), "paper_2506_12727_gb300", "shard.py"))
shard = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(shard)

TILE = (16, 16)


def _case():
    scene = synth.make_scene(300, 3, seed=51)
    cams = synth.make_cameras([(48, 40), (64, 32), (40, 40), (56, 24), (32, 48)], radius=3.0, seed=52)
    rng = np.random.default_rng(53)
    _, _, _, pix_base = oracle.layout(cams, TILE)
    w = rng.normal(size=3 * int(pix_base[-1]))
    return scene, cams, w


def _grads_for(scene, cams, w, views):
    """Oracle gradients and ADC statistics of the views `views` (weights w)."""
    sub = cams.subset(views)
    _, _, _, pb = oracle.layout(cams, TILE)
    ws = np.concatenate([w[3 * pb[v]:3 * pb[v + 1]] for v in views])
    ref = oracle.forward(scene, sub, TILE)
    amb = ref["amb"] != 0
    _, _, _, spb = oracle.layout(sub, TILE)
    amb3 = np.concatenate([np.tile(amb[spb[i]:spb[i + 1]], 3) for i in range(len(views))])
    ws = np.where(amb3, 0.0, ws)
    grads, g2d, e1 = oracle.backward(scene, sub, ref, ws, TILE)
    E1, E2, _, denom = oracle.adc_statistics(g2d, e1, ref["P"]["valid"], len(views))
    return grads, np.stack([E1, E2, denom])


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    scene, cams, w = _case()
    views = shard.shard_views(cams.pixels(), rank, world)
    grads, adc = _grads_for(scene, cams, w, views)
    g = {k: torch.tensor(v) for k, v in grads.items()}
    acc = [torch.tensor(adc)]
    shard.reduce_step(g, acc)
    out[rank] = ({k: v.numpy() for k, v in g.items()}, acc[0].numpy(), views)
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


def test_two_ranks_sum_to_the_single_rank_result():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    scene, cams, w = _case()
    full, adc_full = _grads_for(scene, cams, w, list(range(cams.V)))
    (g0, a0, v0), (g1, a1, v1) = out[0], out[1]
    assert sorted(v0 + v1) == list(range(cams.V)) and v0 and v1
    for k in full:
        np.testing.assert_allclose(g0[k], full[k], rtol=1e-12, atol=1e-12 * np.abs(full[k]).max())
        np.testing.assert_array_equal(g0[k], g1[k])  # every rank holds the same reduced gradient
    np.testing.assert_allclose(a0, adc_full, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(a0, a1)
