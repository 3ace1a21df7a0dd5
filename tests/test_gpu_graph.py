"""Capturable mode (MVGS_FLAG_CAPTURABLE) and CUDA-graph capture of the whole
batched step (render, loss, backward, ADC).

  - with enough capacity, the capturable forward gives the same images,
    sorted lists and ranges as the counting forward, bit for bit;
  - with too little capacity it stays in bounds and the counts block reports
    the needed counts (fits() is False);
  - a captured step replayed after the parameters changed in place equals an
    uncaptured step on the new parameters (images bit-exact, gradients within
    the atomic-order tolerance).
"""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import PARAMS, assert_close_frac, grads_like, scene_to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world(cuda_lib):
    scene = synth.make_scene(20_000, 3, seed=41)
    cams = synth.make_cameras([(160, 120), (96, 130), (201, 45)], radius=4.0, seed=42)
    params = scene_to_device(scene)
    ref = cuda_lib.Rasterizer(cams, tile=(16, 32))
    sc = cuda_lib.make_scene(params, 3)
    img = ref.forward(sc).clone()
    return dict(scene=scene, cams=cams, params=params, ref=ref, img=img)


def test_capturable_forward_equals_counting_forward(world, cuda_lib):
    cams, params, ref = world["cams"], world["params"], world["ref"]
    R, K = int(ref.needed.records), int(ref.needed.keys)
    rz = cuda_lib.Rasterizer(cams, tile=(16, 32), capturable=True)
    rz.reserve(params["means"].shape[0], R + 100, K + 1000)
    sc = cuda_lib.make_scene(params, 3)
    img = rz.forward(sc)
    torch.cuda.synchronize()
    assert torch.equal(img, world["img"])
    c = rz.counts()
    assert (c["records"], c["keys"], c["records_needed"], c["keys_needed"]) == (R, K, R, K)
    assert rz.fits()
    a, b = rz.records(), ref.records()
    assert torch.equal(a["sorted"][:K], b["sorted"][:K])
    assert torch.equal(a["ranges"], b["ranges"])


@pytest.mark.parametrize("short", ["records", "keys"])
def test_capturable_forward_reports_overflow(world, cuda_lib, short):
    cams, params, ref = world["cams"], world["params"], world["ref"]
    R, K = int(ref.needed.records), int(ref.needed.keys)
    rz = cuda_lib.Rasterizer(cams, tile=(16, 32), capturable=True)
    if short == "records":
        rz.reserve(params["means"].shape[0], R // 2, K + 1000)
    else:
        rz.reserve(params["means"].shape[0], R + 100, K // 3)
    sc = cuda_lib.make_scene(params, 3)
    img = rz.forward(sc)
    gg = grads_like(params)
    rz.backward(sc, torch.ones_like(img), gg)
    torch.cuda.synchronize()
    c = rz.counts()
    assert not rz.fits()
    if short == "records":
        assert c["records_needed"] == R and c["records"] == rz.cap.records < R
    else:
        assert c["keys_needed"] == K and c["keys"] == rz.cap.keys < K
    assert torch.isfinite(img).all()


def test_captured_step_replays_on_new_parameters(world, cuda_lib):
    cams, params = world["cams"], world["params"]
    n = params["means"].shape[0]
    ref = world["ref"]
    R, K = int(ref.needed.records), int(ref.needed.keys)
    hw = np.stack([cams.height, cams.width], 1).astype(np.int32)
    tgt = torch.tensor(synth.pack_images(synth.make_targets(cams)), device="cuda")
    p = {k: v.clone() for k, v in params.items()}
    sc = cuda_lib.make_scene(p, 3)
    rz = cuda_lib.Rasterizer(cams, tile=(16, 32), capturable=True)
    rz.reserve(n, int(R * 1.3) + 1000, int(K * 1.3) + 10_000)
    img = torch.empty(3 * rz.pixels, device="cuda")
    loss = torch.empty(cams.V, device="cuda")
    dimg = torch.empty_like(img)
    ws = torch.empty(cuda_lib.dssim_workspace_size(hw), dtype=torch.uint8, device="cuda")
    gm = torch.empty(rz.cap.records, 2, device="cuda")
    e1 = torch.empty(rz.cap.records, device="cuda")
    gg = grads_like(p)
    acc = [torch.zeros(n, device="cuda") for _ in range(3)]

    def step():
        rz.forward(sc, images=img)
        cuda_lib.dssim_loss(img, tgt, hw, 0.2, loss, dimg, ws)
        rz.backward(sc, dimg, gg, gm, e1)
        cuda_lib.adc_accumulate(rz.state, n, gm, e1, *acc)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    # new parameters, same buffers
    gen = torch.Generator("cuda").manual_seed(5)
    p["means"] += 0.01 * torch.randn(p["means"].shape, device="cuda", generator=gen)
    p["sh"][:, 0] += 0.1 * torch.randn(p["sh"][:, 0].shape, device="cuda", generator=gen)
    g.replay()
    torch.cuda.synchronize()
    assert rz.fits()
    got_img, got_loss = img.clone(), loss.clone()
    got_g = {k: v.clone() for k, v in gg.items()}
    # uncaptured reference on the new parameters
    rz2 = cuda_lib.Rasterizer(cams, tile=(16, 32))
    sc2 = cuda_lib.make_scene(p, 3)
    img2 = rz2.forward(sc2)
    loss2 = torch.empty_like(loss)
    d2 = torch.empty_like(img2)
    cuda_lib.dssim_loss(img2, tgt, hw, 0.2, loss2, d2, ws)
    g2 = grads_like(p)
    rz2.backward(sc2, d2, g2)
    torch.cuda.synchronize()
    assert torch.equal(got_img, img2)
    assert torch.equal(got_loss, loss2)
    for k in PARAMS:
        e = g2[k].cpu().numpy()
        assert_close_frac(got_g[k].cpu().numpy(), e, 1e-3, 1e-5 * np.abs(e).max(), k)


@pytest.mark.parametrize("tile", [(16, 16), (16, 64), (8, 8)])
def test_precount_equals_render_counts(world, cuda_lib, tile):
    cams, params = world["cams"], world["params"]
    sc = cuda_lib.make_scene(params, 3)
    rz = cuda_lib.Rasterizer(cams, tile=tile)
    need = cuda_lib.count_views(sc, rz.cams_c, rz.cfg)
    rz.forward(sc)
    torch.cuda.synchronize()
    assert (need.records, need.keys) == (int(rz.needed.records), int(rz.needed.keys))
    # a capturable rasterizer sized from the pre-count fits
    rc = cuda_lib.Rasterizer(cams, tile=tile, capturable=True, headroom=1.0)
    rc.reserve_for(sc)
    rc.forward(sc)
    torch.cuda.synchronize()
    assert rc.fits()
