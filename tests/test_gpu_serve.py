"""Serving loop (continuous batching) on the GPU: every request's images are
the same alone and in a mixed batch; admission by memory splits batches
instead of failing them; a request that cannot fit alone fails cleanly."""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import scene_to_device

pytestmark = pytest.mark.gpu

RES = [(64, 48), (160, 120), (200, 90), (33, 77)]


@pytest.fixture(scope="module")
def world(cuda_lib):
    from paper_2506_12727_gb300 import serve
    scene = synth.make_scene(60_000, 3, seed=21)
    params = scene_to_device(scene)
    rng = np.random.default_rng(22)
    reqs = []
    for i in range(10):
        nv = int(rng.integers(1, 5))
        res = [RES[j] for j in rng.integers(0, len(RES), size=nv)]
        reqs.append(synth.make_cameras(res, radius=(3.0, 5.0), seed=100 + i))
    return dict(serve=serve, scene=scene, params=params, cams=reqs)


def _alone(world, tile=(16, 16)):
    serve = world["serve"]
    srv = serve.Server(world["params"], world["scene"].sh_degree, tile=tile, slots=1)
    out = []
    for i, c in enumerate(world["cams"]):
        r = srv.submit(serve.Request(i, c))
        r.done.wait()
        assert r.error is None
        out.append(r.images.clone())
    srv.close()
    return out


def test_results_are_the_same_alone_and_in_the_mix(world):
    serve = world["serve"]
    alone = _alone(world)
    srv = serve.Server(world["params"], world["scene"].sh_degree, slots=2, max_views=12)
    reqs = [serve.Request(i, c) for i, c in enumerate(world["cams"])]
    for r in reqs:  # all at once: the two workers batch them
        srv.submit(r)
    for r in reqs:
        r.done.wait()
    srv.close()
    torch.cuda.synchronize()
    sizes = [b[3] for b in srv.batch_log]
    assert max(sizes) > 1, "no request was batched with another"
    for r, a in zip(reqs, alone):
        assert r.error is None
        assert torch.equal(r.images, a), r.rid
    s = serve.latency_summary(reqs)
    assert s["failed"] == 0 and s["p99_ms"] >= s["p50_ms"] > 0


def test_memory_admission_splits_batches(world):
    serve = world["serve"]
    alone = _alone(world)
    from paper_2506_12727_gb300 import mvgs
    # budget: enough for the largest single request, far too small for all of them together
    need = []
    for c in world["cams"]:
        rz = mvgs.Rasterizer(c, tile=(16, 16), headroom=1.0)
        rz.forward(mvgs.make_scene(world["params"], 3))
        need.append(rz.held_bytes())
    budget = int(max(need) * 1.5)
    srv = serve.Server(world["params"], world["scene"].sh_degree, slots=1, memory_budget=budget, max_views=64)
    reqs = [serve.Request(i, c) for i, c in enumerate(world["cams"])]
    for r in reqs:
        srv.submit(r)
    for r in reqs:
        r.done.wait()
    srv.close()
    assert all(r.error is None for r in reqs)
    assert len(srv.batch_log) > 1
    for r, a in zip(reqs, alone):
        assert torch.equal(r.images, a), r.rid
    # a request larger than the whole budget fails without stopping the server
    srv = serve.Server(world["params"], world["scene"].sh_degree, slots=1, memory_budget=1 << 20)
    big = srv.submit(serve.Request(99, world["cams"][0]))
    big.done.wait()
    ok = srv.submit(serve.Request(100, synth.make_cameras([(8, 8)], radius=4.0, seed=3)))
    ok.done.wait()
    srv.close()
    assert big.error is not None and "budget" in big.error
    assert ok.error is None or "budget" in ok.error
