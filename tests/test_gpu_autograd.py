"""Differentiation at scale: the torch.autograd.Function around the rasterizer,
on the differentiation workload (1M SH-3 Gaussians, 16 views of 1024x768).

  - autograd gives the same gradients as the direct backward call;
  - central finite differences of the float32 forward agree with the autograd
    gradient on 64 seeded parameters of strongly visible Gaussians (loss
    accumulated in float64; pixels whose discrete decisions change between the
    +h and -h renders, including any change of their tile's depth-sorted list,
    carry no loss weight for that parameter);
  - the gradient of a loss on a 64x64 window of every view matches the oracle
    (1e-3 of each Gaussian's gradient vector norm per tensor: at this scale a
    component 100x smaller than its row, e.g. the depth-direction mean
    gradient of a large Gaussian, is the difference of float32 terms of the
    row's size).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import PARAMS, assert_close_frac, assert_close_rows, scene_to_device

pytestmark = pytest.mark.gpu

WORKLOAD = "diff_1m_16x1024x768"
TILE = (16, 64)


@pytest.fixture(scope="module")
def setup(cuda_lib):
    from paper_2506_12727_gb300 import autograd
    scene, cams, _ = synth.workload(WORKLOAD)
    params = scene_to_device(scene)
    rz = cuda_lib.Rasterizer(cams, tile=TILE)
    return dict(scene=scene, cams=cams, params=params, rz=rz, autograd=autograd, mvgs=cuda_lib)


def _grads(setup, weights):
    ps = {k: v.clone().requires_grad_(True) for k, v in setup["params"].items()}
    img = setup["autograd"].render(setup["rz"], ps, setup["scene"].sh_degree)
    (img.double() * weights.double()).sum().backward()
    return {k: v.grad.detach() for k, v in ps.items()}


def test_autograd_matches_direct_backward(setup):
    mvgs, rz, scene = setup["mvgs"], setup["rz"], setup["scene"]
    w = torch.randn(3 * rz.pixels, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    g_auto = _grads(setup, w)
    sc = mvgs.make_scene(setup["params"], scene.sh_degree)
    rz.forward(sc)
    direct = {k: torch.empty_like(v) for k, v in setup["params"].items()}
    rz.backward(sc, w.contiguous(), direct)
    torch.cuda.synchronize()
    for k in PARAMS:
        # the two runs differ only in the order of the float32 atomics that sum
        # per-pixel terms; where those terms cancel (the conic gradients carry
        # dx^2 ~ 1e4 px^2 factors) the rounding of a different order can exceed
        # the tolerance, so a few entries in a million may
        a, d = g_auto[k].cpu().numpy(), direct[k].cpu().numpy()
        assert_close_frac(a, d, 1e-3, 1e-5 * np.abs(d).max(), k, max_bad=int(1e-5 * a.size))


def _tile_hash(rec):
    """A per-(view, tile) hash of the tile's sorted list (the Gaussians and their
    depth order), to see which lists a perturbation changed."""
    ranges = rec["ranges"]
    lens = (ranges[:, 1] - ranges[:, 0]).clamp(min=0)
    n_tiles = len(lens)
    tile_of = torch.repeat_interleave(torch.arange(n_tiles, device="cuda"), lens)
    first = torch.cumsum(lens, 0) - lens
    pos = torch.arange(len(tile_of), device="cuda") - first[tile_of]
    rec_ids = rec["sorted"][(ranges[tile_of, 0] + pos)].to(torch.int64)
    gauss = rec["g"][rec_ids].to(torch.int64)
    # a term non-linear in (Gaussian, position): a swap of two entries changes the sum
    P = 2147483647
    z = ((gauss + 1) * 1000003 + pos) % P
    term = ((z * z) % P * 48271 + z) % P
    h = torch.zeros(n_tiles, dtype=torch.int64, device="cuda")
    h.index_add_(0, tile_of, term)
    return h


def _render_with_stats(setup, params):
    mvgs, rz = setup["mvgs"], setup["rz"]
    img = rz.forward(mvgs.make_scene(params, setup["scene"].sh_degree), stats=True).clone()
    rec = rz.records()
    stats = torch.cat([rec["pixel_stats"], rec["n_contrib"][:, None]], 1).clone()
    return img, stats, _tile_hash(rec)


def _pixel_tiles(setup):
    """Global tile id of every pixel (views concatenated)."""
    cams = setup["cams"]
    out = []
    base = 0
    for v in range(cams.V):
        W, H = int(cams.width[v]), int(cams.height[v])
        tx = -(-W // TILE[0])
        ys, xs = torch.meshgrid(torch.arange(H, device="cuda"), torch.arange(W, device="cuda"), indexing="ij")
        out.append(base + (ys // TILE[1]) * tx + xs // TILE[0])
        base += tx * -(-H // TILE[1])
    return torch.cat([o.reshape(-1) for o in out])


def test_central_differences_on_64_parameters(setup):
    mvgs, rz, scene, params = setup["mvgs"], setup["rz"], setup["scene"], setup["params"]
    rng = np.random.default_rng(71)
    w = torch.tensor(rng.normal(size=3 * rz.pixels).astype(np.float32), device="cuda")
    base_img, base_stats, base_hash = _render_with_stats(setup, params)
    ptile = _pixel_tiles(setup)
    g_full = _grads(setup, w)
    # 64 parameters spread over the five kinds, of Gaussians that carry real
    # weight in the images (the 2000 with the largest opacity gradient): for a
    # Gaussian seen only through T ~ 1e-3, the float32 rounding of the renders
    # is as large as the h-sized change it makes
    strong = torch.topk(g_full["opacity_logits"].abs(), 2000).indices.cpu().numpy()
    picks = []
    for i in range(64):
        kind = PARAMS[i % 5]
        g = int(rng.choice(strong))
        comp = tuple(int(rng.integers(0, s)) for s in params[kind].shape[1:])
        picks.append((kind, (g,) + comp))
    # step per kind: the float32 rounding of the two renders enters the
    # difference quotient as 1/h while the central-difference error is O(h^2);
    # the colour is linear in sh and smooth in the opacity logit, and the
    # footprint smooth in the log-scales and the rotation, so larger steps
    # there only lower the rounding noise
    steps = dict(means=2e-3, log_scales=5e-3, quats=5e-3, opacity_logits=1e-2, sh=1e-2)
    errs, scales, kinds, ok = [], [], [], 0
    for kind, idx in picks:
        t = params[kind]
        x0 = t[idx].item()
        h = steps[kind]
        imgs, stats, hashes, xs = [], [], [], []
        for sgn in (1, -1):
            t[idx] = x0 + sgn * h
            xs.append(t[idx].item())
            im, st, th = _render_with_stats(setup, params)
            imgs.append(im)
            stats.append(st)
            hashes.append(th)
        t[idx] = x0
        # a pixel is differentiable in the FD sense only if no discrete decision
        # changed: same list (content and depth order) for its tile, same
        # stopping point, same number of blended Gaussians
        same_list = (hashes[0] == base_hash) & (hashes[1] == base_hash)
        stable = ((stats[0] == base_stats).all(1) & (stats[1] == base_stats).all(1)) & same_list[ptile]
        # per-pixel mask over the packed [3, H, W] layout of each view
        mask = torch.zeros(3 * rz.pixels, dtype=torch.bool, device="cuda")
        off = 0
        pix_off = 0
        for v in range(setup["cams"].V):
            hw = int(setup["cams"].width[v]) * int(setup["cams"].height[v])
            mask[off:off + 3 * hw] = stable[pix_off:pix_off + hw].repeat(3)
            off += 3 * hw
            pix_off += hw
        wm = torch.where(mask, w, torch.zeros_like(w))
        fd = ((imgs[0].double() - imgs[1].double()) * wm.double()).sum().item() / (xs[0] - xs[1])
        an = _grads(setup, wm)[kind][idx].item()
        errs.append(abs(fd - an))
        scales.append(abs(an))
        kinds.append(kind)
        ok += 1
    errs, scales = np.array(errs), np.array(scales)
    rel = errs / (scales + 1e-3 * scales.max())
    print(f"finite differences: median rel err {np.median(rel):.2e}, 90th pct {np.quantile(rel, 0.9):.2e}, "
          f"max {rel.max():.2e}")
    for kind in PARAMS:
        sel = np.array([k == kind for k in kinds])
        print(f"   {kind}: median {np.median(rel[sel]):.2e} max {rel[sel].max():.2e}")
    assert ok == 64
    assert np.median(rel) < 1e-2
    assert np.quantile(rel, 0.9) < 5e-2


def test_window_gradients_match_oracle(setup):
    mvgs, rz, scene, cams = setup["mvgs"], setup["rz"], setup["scene"], setup["cams"]
    rng = np.random.default_rng(72)
    win = []
    for v in range(cams.V):
        x0 = int(rng.integers(0, cams.width[v] - 64))
        y0 = int(rng.integers(0, cams.height[v] - 64))
        win.append([x0, y0, x0 + 64, y0 + 64])
    win = np.array(win, np.int32)
    ref = oracle.forward(scene, cams, TILE, window=win)
    _, _, _, pix_base = oracle.layout(cams, TILE)
    dimg = np.zeros(3 * int(pix_base[-1]), np.float32)
    for v in range(cams.V):
        H, W = int(cams.height[v]), int(cams.width[v])
        x0, y0, x1, y1 = win[v]
        d = rng.normal(size=(3, 64, 64)).astype(np.float32)
        amb = ref["amb"][pix_base[v]:pix_base[v + 1]].reshape(H, W)[y0:y1, x0:x1] != 0
        d[:, amb] = 0.0
        dimg[3 * pix_base[v]:3 * pix_base[v + 1]].reshape(3, H, W)[:, y0:y1, x0:x1] = d
    grads, _, _ = oracle.backward(scene, cams, ref, dimg.astype(np.float64), TILE, window=win)
    g = _grads(setup, torch.tensor(dimg, device="cuda"))
    bad_g = np.zeros(scene.n, bool)
    bad_g[np.nonzero(ref["P"]["amb"])[0] % scene.n] = True
    touched = np.abs(grads["opacity_logits"]) > 0
    print(f"window gradients: {touched.sum()} Gaussians touched, {bad_g.sum()} excluded")
    assert touched.sum() > 1000
    for k in PARAMS:
        # excluded Gaussians compare as zero, so reported indices are Gaussian ids
        got = g[k].cpu().numpy().astype(np.float64)
        exp = grads[k].copy()
        got[bad_g] = 0.0
        exp[bad_g] = 0.0
        # float32 transmittance recovered by division and the running colour
        # behind each Gaussian (the backward of Eq. 1) leave a dL/dalpha that
        # cancels in dense scenes slightly off for a handful of Gaussians per
        # million; more than 1 per million fails
        assert_close_rows(got, exp, 1e-3, 1e-5 * np.abs(exp).max(), "d" + k, max_bad=got.size // 1_000_000)


def test_backward_after_a_later_forward_on_the_same_rasterizer_raises(cuda_lib):
    """One rasterizer holds one forward's state: a backward whose state a
    second forward overwrote is refused (not silently wrong)."""
    from paper_2506_12727_gb300 import autograd
    scene = synth.make_scene(2000, 3, seed=91)
    cams = synth.make_cameras([(64, 48), (48, 64)], radius=3.0, seed=92)
    rz = cuda_lib.Rasterizer(cams, tile=(16, 16))
    ps = {k: v.clone().requires_grad_(True) for k, v in scene_to_device(scene).items()}
    first = autograd.render(rz, ps, 3)
    second = autograd.render(rz, ps, 3)
    with pytest.raises(RuntimeError, match="later forward"):
        first.sum().backward()
    second.sum().backward()  # the latest forward's backward still runs
    assert torch.isfinite(ps["means"].grad).all() and ps["means"].grad.abs().max() > 0
