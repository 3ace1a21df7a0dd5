"""GPU parity: the sm_103a path through the C ABI against the CPU oracle on the
same seeded inputs.

Tolerances (float32 kernels against a float64 oracle):
  images         1e-4 absolute (per pixel and channel), on pixels where no
                 discrete decision of the blend lies within the oracle's
                 ambiguity margin of its threshold (those pixels are counted
                 and must stay rare);
  gradients      1e-3 relative with an absolute floor of 1e-6 x the
                 tensor's largest entry (_grad_floor), on a loss that puts no
                 weight on ambiguous pixels and on Gaussians with no
                 ambiguous record;
  sort           bit-exact on identical projected inputs.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import PARAMS, assert_close_frac, dense_records, gpu_forward, grads_like, scene_to_device

pytestmark = pytest.mark.gpu

AMB_FWD = oracle.PA_FORWARD
AMB_ALL = 0xFF


def _large_gaussians():
    # few Gaussians of about 0.2 units (radii of 40-150 px): gradients that
    # sum many pixels at large offsets from the mean
    rng = np.random.default_rng(3)
    sc = synth.make_scene(40, 3, seed=11)
    sc.log_scales[:] = rng.normal(-1.5, 0.3, size=sc.log_scales.shape)
    sc.opacity_logits[:] = rng.normal(0.5, 0.5, size=sc.opacity_logits.shape)
    return sc, synth.make_cameras([(196, 160), (160, 196)], radius=4.0, seed=5)


def _small_cases():
    # several tiles in each direction and ragged image edges
    return {
        "large_gaussians_sh3": _large_gaussians(),
        "single_view_10k_sh0": (synth.make_scene(10_000, 0), synth.make_cameras([(128, 128)], radius=3.0)),
        "multiview_sh3_ragged": (synth.make_scene(6_000, 3, seed=5),
                                 synth.make_cameras([(150, 97), (64, 130), (201, 45)], radius=4.0, seed=6)),
        # half of the Gaussians beyond the guard band of the projection
        # Jacobian (1.4-1.9x the half-FOV tangent), large enough to reach
        # into the image: records whose covariance uses the clamped J
        "off_axis_guard_band_sh3": synth.off_axis_scene(300, 300, sh_degree=3, W=96, H=72, seed=45),
    }


CASES = _small_cases()


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, cuda_lib):
    name = request.param
    scene, cams = CASES[name]
    bg = (0.1, 0.2, 0.3) if "ragged" in name else (0.0, 0.0, 0.0)
    ref = oracle.forward(scene, cams, (16, 16), bg=bg)
    rz, sc, params, img = gpu_forward(cuda_lib, scene, cams, (16, 16), bg, None)
    return dict(name=name, scene=scene, cams=cams, bg=bg, ref=ref, rz=rz, sc=sc, params=params,
                img=img.cpu().numpy().astype(np.float64))


def test_records_match_oracle(case):
    scene, cams, ref = case["scene"], case["cams"], case["ref"]
    P = ref["P"]
    D = dense_records(case["rz"], scene.n, cams.V)
    amb = P["amb"] != 0
    ok = ~amb
    np.testing.assert_array_equal(D["valid"][ok], P["valid"][ok])
    vis = ok & (P["valid"] != 0)
    assert vis.sum() > 0.5 * scene.n
    assert_close_frac(D["xy"][vis], P["xy"][vis], 0, 2e-3, "mean2d")
    assert_close_frac(D["conic"][vis], P["conic"][vis], 2e-4, 1e-7 * np.abs(P["conic"]).max(), "conic")
    assert_close_frac(D["opac"][vis], P["opac"][vis], 1e-5, 1e-7, "opacity")
    assert_close_frac(D["rgb"][vis], P["rgb"][vis], 1e-5, 1e-6, "rgb")
    assert_close_frac(D["depth"][vis], P["depth"][vis], 1e-6, 0, "depth")
    np.testing.assert_array_equal(D["radius"][vis], P["radius"][vis])
    np.testing.assert_array_equal(D["clamp"][vis], P["clampmask"][vis])
    # rects may differ only by float rounding of the tile boundary test
    assert (D["rect"][vis] != P["rect"][vis]).any(axis=1).mean() < 1e-3


def _assert_same_ranges(got, exp):
    """Non-empty tile ranges are unique and must match exactly; an empty
    tile may be reported as [p, p) for any p."""
    got = np.asarray(got)
    exp = np.asarray(exp)
    ne = exp[:, 1] > exp[:, 0]
    np.testing.assert_array_equal(got[ne], exp[ne])
    assert np.all(got[~ne, 1] == got[~ne, 0])


def test_sort_is_bitexact_on_gpu_projected_inputs(case):
    """The oracle sort (std ordering of (tile, view, depth, Gaussian)) on the
    GPU's own projected records reproduces the GPU list exactly."""
    scene, cams = case["scene"], case["cams"]
    D = dense_records(case["rz"], scene.n, cams.V)
    depth32 = np.zeros(scene.n * cams.V, np.float32)
    depth32[D["valid"] != 0] = D["raw"]["depth"][D["rec_index"][D["valid"] != 0]]
    keys, recs, ranges = oracle.sort_keys(cams, (16, 16), D["valid"], D["rect"], depth32)
    gsorted = D["raw"]["sorted"].astype(np.int64)
    gdense = D["raw"]["v"][gsorted].astype(np.int64) * scene.n + D["raw"]["g"][gsorted]
    assert len(gdense) == len(recs) > 0
    np.testing.assert_array_equal(gdense, recs)
    _assert_same_ranges(D["raw"]["ranges"], ranges)


def test_forward_image_matches_oracle(case):
    ref, img = case["ref"], case["img"]
    amb = (ref["amb"] & AMB_FWD) != 0
    _, _, _, pix_base = oracle.layout(case["cams"], (16, 16))
    amb3 = np.concatenate([np.tile(amb[pix_base[v]:pix_base[v + 1]], 3) for v in range(case["cams"].V)])
    frac = amb.mean()
    print(f"[{case['name']}] ambiguous pixels {frac:.4%}; max |err| unflagged "
          f"{np.abs(img - ref['img'])[~amb3].max():.3e}; flagged {np.abs(img - ref['img'])[amb3].max(initial=0):.3e}")
    assert frac < 0.03
    assert_close_frac(img[~amb3], ref["img"][~amb3], 0, 1e-4, "image")
    rec = case["rz"].records()
    T = rec["final_T"].cpu().numpy()
    assert_close_frac(T[~amb], ref["T"][~amb], 0, 1e-4, "final T")
    nc = rec["n_contrib"].cpu().numpy()
    np.testing.assert_array_equal(nc[~amb], ref["last"][~amb])


def _grad_floor(ref):
    return 1e-6 * max(np.abs(ref).max(), 1e-30)


def test_backward_matches_oracle(case):
    cuda = case
    scene, cams, ref, bg = case["scene"], case["cams"], case["ref"], case["bg"]
    rng = np.random.default_rng(31)
    dimg = rng.normal(size=ref["img"].shape).astype(np.float32)
    amb = ref["amb"] != 0
    _, _, _, pix_base = oracle.layout(cams, (16, 16))
    amb3 = np.concatenate([np.tile(amb[pix_base[v]:pix_base[v + 1]], 3) for v in range(cams.V)])
    dimg[amb3] = 0.0
    grads, g2d, e1 = oracle.backward(scene, cams, ref, dimg.astype(np.float64), (16, 16), bg)
    rz = cuda["rz"]
    gg = grads_like(cuda["params"])
    R = int(rz.needed.records)
    gm2d = torch.zeros(R, 2, device="cuda")
    ge1 = torch.zeros(R, device="cuda")
    rz.backward(cuda["sc"], torch.tensor(dimg, device="cuda"), gg, gm2d, ge1)
    torch.cuda.synchronize()
    # Gaussians whose records carry an ambiguous clamp or radius decision
    bad_g = np.zeros(scene.n, bool)
    bad_g[np.nonzero(ref["P"]["amb"])[0] % scene.n] = True
    D = dense_records(rz, scene.n, cams.V)
    vis = (D["valid"] != 0) & (ref["P"]["valid"] != 0) & ~bad_g[np.arange(scene.n * cams.V) % scene.n]
    gm = np.zeros((scene.n * cams.V, 2))
    gm[D["valid"] != 0] = gm2d.cpu().numpy()[D["rec_index"][D["valid"] != 0]]
    ge = np.zeros(scene.n * cams.V)
    ge[D["valid"] != 0] = ge1.cpu().numpy()[D["rec_index"][D["valid"] != 0]]
    for name, got, exp in (("mean2d", gm[vis], g2d[vis, :2]), ("e1", ge[vis], e1[vis])):
        err = np.abs(got - exp) / (np.abs(exp) + _grad_floor(exp))
        print(f"[{case['name']}] {name}: max rel err {err.max():.3e}, p99 {np.quantile(err, 0.99):.3e}")
        assert_close_frac(got, exp, 1e-3, _grad_floor(exp), name)
    for k in PARAMS:
        got = gg[k].cpu().numpy().astype(np.float64)[~bad_g]
        exp = grads[k][~bad_g]
        err = np.abs(got - exp) / (np.abs(exp) + _grad_floor(exp))
        print(f"[{case['name']}] d{k}: max rel err {err.max():.3e}, p99 {np.quantile(err, 0.99):.3e}, "
              f"excluded Gaussians {bad_g.sum()}")
        assert_close_frac(got, exp, 1e-3, _grad_floor(exp), "d" + k)


def test_image_is_independent_of_tile_size(cuda_lib):
    scene, cams = CASES["multiview_sh3_ragged"]
    imgs = []
    for tile in ((8, 8), (16, 16), (16, 32), (32, 16), (8, 16), (32, 8), (8, 32), (16, 8), (32, 32), (16, 64),
                 (32, 64)):
        _, _, _, img = gpu_forward(cuda_lib, scene, cams, tile, (0.3, 0.3, 0.3))
        imgs.append(img.cpu().numpy())
    for im in imgs[1:]:
        np.testing.assert_array_equal(im, imgs[0])


def test_dssim_loss_matches_oracle(cuda_lib):
    rng = np.random.default_rng(41)
    shapes = [(37, 52), (16, 16), (100, 7), (64, 81)]
    imgs = [rng.uniform(size=(3, h, w)).astype(np.float32) for h, w in shapes]
    tgts = [np.clip(i + rng.normal(0, 0.15, size=i.shape), 0, 1).astype(np.float32) for i in imgs]
    hw = np.array(shapes, np.int32)
    lam = 0.2
    per, total, grads = oracle.dssim_l1_loss(imgs, tgts, lam)
    I = torch.tensor(synth.pack_images(imgs), device="cuda")
    Tt = torch.tensor(synth.pack_images(tgts), device="cuda")
    ws = torch.empty(cuda_lib.dssim_workspace_size(hw), dtype=torch.uint8, device="cuda")
    loss = torch.empty(len(shapes), device="cuda")
    dimg = torch.empty_like(I)
    cuda_lib.dssim_loss(I, Tt, hw, lam, loss, dimg, ws)
    torch.cuda.synchronize()
    np.testing.assert_allclose(loss.cpu().numpy(), per, rtol=2e-5, atol=1e-6)
    g = synth.pack_images([x.astype(np.float32) for x in grads]).astype(np.float64)
    got = dimg.cpu().numpy().astype(np.float64)
    scale = np.abs(g).max()
    print(f"dssim grad max abs err {np.abs(got - g).max():.3e} (scale {scale:.3e})")
    assert_close_frac(got, g, 1e-3, 1e-4 * scale, "dL/dimage")


def test_adc_statistics_match_oracle(case, cuda_lib):
    scene, cams, ref, bg = case["scene"], case["cams"], case["ref"], case["bg"]
    rng = np.random.default_rng(43)
    dimg = rng.normal(size=ref["img"].shape).astype(np.float32)
    amb = ref["amb"] != 0
    _, _, _, pix_base = oracle.layout(cams, (16, 16))
    amb3 = np.concatenate([np.tile(amb[pix_base[v]:pix_base[v + 1]], 3) for v in range(cams.V)])
    dimg[amb3] = 0.0
    _, g2d, e1 = oracle.backward(scene, cams, ref, dimg.astype(np.float64), (16, 16), bg)
    E1, E2, Eold, denom = oracle.adc_statistics(g2d, e1, ref["P"]["valid"], cams.V)
    rz = case["rz"]
    R = int(rz.needed.records)
    gm2d = torch.zeros(R, 2, device="cuda")
    ge1 = torch.zeros(R, device="cuda")
    rz.backward(case["sc"], torch.tensor(dimg, device="cuda"), grads_like(case["params"]), gm2d, ge1)
    acc = [torch.zeros(scene.n, device="cuda") for _ in range(3)]
    for _ in range(2):  # accumulates across calls
        cuda_lib.adc_accumulate(rz.state, scene.n, gm2d, ge1, *acc)
    torch.cuda.synchronize()
    bad_g = np.zeros(scene.n, bool)
    bad_g[np.nonzero(ref["P"]["amb"])[0] % scene.n] = True
    ok = ~bad_g
    np.testing.assert_array_equal(acc[2].cpu().numpy()[ok], 2 * denom[ok])
    assert_close_frac(acc[0].cpu().numpy()[ok], 2 * E1[ok], 1e-3, _grad_floor(E1), "E1")
    assert_close_frac(acc[1].cpu().numpy()[ok], 2 * E2[ok], 1e-3, _grad_floor(E2), "E2")
    assert (E1[ok] >= E2[ok] - 1e-9).all()


def test_empty_scene_and_views_without_gaussians(cuda_lib):
    scene = synth.make_scene(50, 1, seed=3)
    cams = synth.make_cameras([(40, 33), (17, 70)], radius=3.0)
    # every Gaussian behind the first camera's near plane: move the means far behind camera 0
    sc0 = scene.subset(np.arange(0))
    _, _, _, img = gpu_forward(cuda_lib, sc0, cams, (16, 16), (0.25, 0.5, 0.75))
    im = img.cpu().numpy()
    _, _, _, pix_base = oracle.layout(cams, (16, 16))
    for v in range(cams.V):
        block = im[3 * pix_base[v]:3 * pix_base[v + 1]].reshape(3, -1)
        np.testing.assert_array_equal(block, np.array([[0.25], [0.5], [0.75]], np.float32) * np.ones_like(block))
    # a camera looking away from all Gaussians renders the background
    away = synth.Cameras(cams.width[:1], cams.height[:1], cams.fx[:1], cams.fy[:1], cams.cx[:1], cams.cy[:1],
                         synth.look_at(np.array([0, 0, 5.0]), target=(0, 0, 10.0))[None].astype(np.float32),
                         np.array([[0, 0, 5.0]], np.float32), cams.near[:1])
    rz, _, _, img = gpu_forward(cuda_lib, scene, away, (16, 16), (0.1, 0.1, 0.1))
    assert int(rz.needed.records) == 0
    np.testing.assert_array_equal(img.cpu().numpy(), np.float32(0.1))


def test_huge_gaussian_and_tiny_images(cuda_lib):
    """One Gaussian covering the whole image, 1x1 and 7x5 images."""
    sc = synth.make_scene(3, 0, seed=2)
    sc.log_scales[:] = np.float32(math.log(2.0))
    sc.means[:] = 0.0
    cams = synth.make_cameras([(1, 1), (7, 5), (120, 90)], radius=3.0)
    ref = oracle.forward(sc, cams, (16, 16), bg=(0.2, 0.2, 0.2))
    _, _, _, img = gpu_forward(cuda_lib, sc, cams, (16, 16), (0.2, 0.2, 0.2))
    amb = ref["amb"] != 0
    _, _, _, pix_base = oracle.layout(cams, (16, 16))
    amb3 = np.concatenate([np.tile(amb[pix_base[v]:pix_base[v + 1]], 3) for v in range(cams.V)])
    assert_close_frac(img.cpu().numpy()[~amb3], ref["img"][~amb3], 0, 1e-4, "image")


def _plane_scene(n, z, seed):
    """Gaussians on the plane z = const in front of an axis-aligned camera:
    every record has the same float32 depth, so the sort order inside a tile
    rests entirely on the tie-break by Gaussian index."""
    rng = np.random.default_rng(seed)
    sc = synth.make_scene(n, 1, seed=seed)
    sc.means[:, 0] = rng.uniform(-1.2, 1.2, n).astype(np.float32)
    sc.means[:, 1] = rng.uniform(-0.9, 0.9, n).astype(np.float32)
    sc.means[:, 2] = np.float32(z)
    return sc


def _axis_cams(resolutions, f=300.0):
    V = len(resolutions)
    vm = np.zeros((V, 3, 4), np.float32)
    vm[:, :, :3] = np.eye(3, dtype=np.float32)
    vm[:, 0, 3] = np.linspace(-0.3, 0.3, V)  # small shifts keep the depth and change the image
    W = np.array([r[0] for r in resolutions], np.int32)
    H = np.array([r[1] for r in resolutions], np.int32)
    return synth.Cameras(W, H, np.full(V, f, np.float32), np.full(V, f, np.float32), (W / 2).astype(np.float32),
                         (H / 2).astype(np.float32), vm, np.zeros((V, 3), np.float32), np.full(V, 0.2, np.float32))


@pytest.mark.parametrize("tile,nviews", [((16, 16), 3), ((8, 8), 3), ((8, 8), 22)])
def test_sort_bitexact_with_exact_depth_ties_and_many_tiles(cuda_lib, tile, nviews):
    """Exact depth ties everywhere.  The global tile id takes 12 bits (3 views
    of 16x16 tiles), 14 bits (3 views of 8x8 tiles: two radix passes, packed,
    the second over 6 bits) or 17 bits (22 views of 8x8 tiles: three passes)."""
    scene = _plane_scene(3000, 2.0, seed=17)
    cams = _axis_cams([(640, 480)] * nviews)
    rz, _, _, _ = gpu_forward(cuda_lib, scene, cams, tile)
    if nviews == 22:
        assert int(rz.layout.tiles) > 65536
    D = dense_records(rz, scene.n, cams.V)
    vis = D["valid"] != 0
    depth32 = np.zeros(scene.n * cams.V, np.float32)
    depth32[vis] = D["raw"]["depth"][D["rec_index"][vis]]
    assert len(np.unique(depth32[vis])) == 1
    keys, recs, ranges = oracle.sort_keys(cams, tile, D["valid"], D["rect"], depth32)
    gsorted = D["raw"]["sorted"].astype(np.int64)
    gdense = D["raw"]["v"][gsorted].astype(np.int64) * scene.n + D["raw"]["g"][gsorted]
    np.testing.assert_array_equal(gdense, recs)
    _assert_same_ranges(D["raw"]["ranges"], ranges)


def test_results_do_not_depend_on_the_batch_size(cuda_lib):
    # the shared-memory batch only changes how many records a warp stages at a
    # time: images must agree bit for bit, gradients up to atomic order
    scene, cams = CASES["multiview_sh3_ragged"]
    params = scene_to_device(scene)
    sc = cuda_lib.make_scene(params, scene.sh_degree)
    dimg = None
    imgs, grads = [], []
    for wb in (64, 128, 192):
        rz = cuda_lib.Rasterizer(cams, tile=(16, 32), smem_batch=wb)
        img = rz.forward(sc).clone()
        if dimg is None:
            dimg = torch.randn(img.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(9))
        gg = grads_like(params)
        rz.backward(sc, dimg, gg)
        torch.cuda.synchronize()
        imgs.append(img)
        grads.append({k: v.cpu().numpy() for k, v in gg.items()})
    for im in imgs[1:]:
        assert torch.equal(im, imgs[0])
    for g in grads[1:]:
        for k in PARAMS:
            assert_close_frac(g[k], grads[0][k], 1e-3, 1e-6 * np.abs(grads[0][k]).max(), k)


def test_optional_outputs_do_not_change_the_render(cuda_lib):
    # the depth and statistics outputs are separate kernel variants: the image,
    # final T and last contributors must not depend on which one runs
    scene, cams = CASES["multiview_sh3_ragged"]
    params = scene_to_device(scene)
    sc = cuda_lib.make_scene(params, scene.sh_degree)
    rz = cuda_lib.Rasterizer(cams, tile=(16, 32), bg=(0.1, 0.2, 0.3))
    runs = []
    for depth, stats in ((False, False), (True, False), (False, True), (True, True)):
        img = rz.forward(sc, depth=depth, stats=stats).clone()
        rec = rz.records()
        runs.append((img, rec["final_T"].clone(), rec["n_contrib"].clone(),
                     rec["pixel_stats"].clone() if stats else None))
    for img, T, last, _ in runs[1:]:
        assert torch.equal(img, runs[0][0])
        assert torch.equal(T, runs[0][1])
        assert torch.equal(last, runs[0][2])
    # the statistics agree between the two variants that write them, and the
    # blended count never exceeds the list position of the last contributor
    assert torch.equal(runs[2][3], runs[3][3])
    st = runs[2][3].to(torch.int64)
    assert bool((st[:, 1] <= runs[2][2].to(torch.int64)).all())
    assert bool((runs[2][2].to(torch.int64) <= st[:, 0]).all())


def test_backward_with_an_exact_odd_record_capacity(cuda_lib):
    """Capacities exactly the records and keys needed, with an odd record
    count: the per-record gradient slots (8 floats and 3 doubles per record)
    are zeroed to their last byte before the backward's atomics, whatever the
    workspace held (filled with NaN bytes here).  The pre-count runs on 6000
    Gaussians and fewer, where its scan scratch is not a multiple of 16 bytes
    (the camera table behind it must still be aligned)."""
    scene, cams = CASES["multiview_sh3_ragged"]
    params = scene_to_device(scene)
    cams_c = cuda_lib.make_cameras(cams)
    cfg = cuda_lib.make_config((16, 16))
    # the first Gaussian count (from all of them down) with an odd record count
    for n in range(scene.n, scene.n - 32, -1):
        keep = {k: v[:n].contiguous() for k, v in params.items()}
        sck = cuda_lib.make_scene(keep, scene.sh_degree)
        need = cuda_lib.count_views(sck, cams_c, cfg)
        if int(need.records) % 2 == 1:
            break
    else:
        pytest.skip("no odd record count")
    cap = cuda_lib.Capacity(int(need.records), int(need.keys))
    L = cuda_lib.render_layout(n, cams_c, cfg, cap)
    state = torch.empty(L.state_bytes, dtype=torch.uint8, device="cuda")
    ws = torch.full((L.workspace_bytes,), 0xFF, dtype=torch.uint8, device="cuda")
    probe = cuda_lib.Rasterizer(cams, tile=(16, 16))
    img = probe.forward(sck)
    dimg = torch.randn(img.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    exp = grads_like(keep)
    probe.backward(sck, dimg, exp)
    img2 = torch.empty_like(img)
    cuda_lib.render_views(sck, cams_c, cfg, cap, img2, state, ws)
    got = grads_like(keep)
    cuda_lib.render_views_backward(sck, cams_c, cfg, cap, dimg, state, ws, got)
    torch.cuda.synchronize()
    assert torch.equal(img2, img)
    for k in got:
        assert torch.isfinite(got[k]).all(), k
        torch.testing.assert_close(got[k], exp[k], rtol=1e-4, atol=1e-6 * float(exp[k].abs().max()))
