"""Thread-efficient partial rendering (Sec. 5.1.1, Alg. 3) on the GPU.

  - the sample sets the library generates are exactly the oracle's selection
    (integer hashing: bit-exact);
  - a sampled pixel gets bit for bit the value of the full render, for the
    packed runs (Alg. 3) and the masked strips (Fig. 3b), over tile sizes and
    pixels per lane; unsampled pixels are left untouched;
  - against the oracle: images at the sampled pixels within 1e-4, and the
    sampled backward equals the oracle's full backward with dL/dimage zero
    off the samples (gradient tolerance of the parity suite);
  - edge cases: group 1 (every pixel), more views than the group, a group
    larger than the views, an empty scene.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import PARAMS, assert_close_frac, grads_like, scene_to_device
from oracle import partial

pytestmark = pytest.mark.gpu


def _masks_from_samples(ss, cams, tile):
    """Packed boolean pixel mask of a GPU sample set (and a check that each
    tile's samples are distinct and in raster order)."""
    tw, th = tile
    off = ss.offsets.cpu().numpy()
    pix = ss.pixel_index().cpu().numpy()
    out = []
    t = 0
    for v in range(cams.V):
        W, H = int(cams.width[v]), int(cams.height[v])
        tx, ty = -(-W // tw), -(-H // th)
        m = np.zeros((H, W), bool)
        for j in range(ty):
            for i in range(tx):
                s = pix[off[t]:off[t + 1]]
                assert np.all(np.diff(s) > 0)
                lx, ly = s % tw, s // tw
                assert np.all(ly < th)
                m[j * th + ly, i * tw + lx] = True
                t += 1
        out.append(m.reshape(-1))
    assert t == len(off) - 1
    return np.concatenate(out)


def _packed3(mask_px, cams):
    """Pixel mask -> mask over the packed [3, H, W] image layout."""
    out, p = [], 0
    for v in range(cams.V):
        hw = int(cams.width[v]) * int(cams.height[v])
        out.append(np.tile(mask_px[p:p + hw], 3))
        p += hw
    return np.concatenate(out)


CASES = {
    "ragged_3views": (synth.make_scene(6_000, 3, seed=5),
                      synth.make_cameras([(150, 97), (64, 130), (201, 45)], radius=4.0, seed=6)),
    "same_res_4views": (synth.make_scene(8_000, 3, seed=7), synth.make_cameras([(160, 120)] * 4, radius=4.0,
                                                                               seed=8)),
}


@pytest.mark.parametrize("cell", [(1, 1), (16, 8), (3, 5)])
@pytest.mark.parametrize("group", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16), (16, 64)])
def test_samples_match_oracle_selection(cuda_lib, tile, group, cell):
    _, cams = CASES["ragged_3views"]
    rz = cuda_lib.Rasterizer(cams, tile=tile)
    ss = rz.sample_set(group, seed=1234, cell=cell)
    got = _masks_from_samples(ss, cams, tile)
    np.testing.assert_array_equal(got, partial.packed_mask(cams, group, 1234, cell))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("tile,ppt", [((16, 16), 0), ((16, 16), 1), ((8, 8), 2), ((32, 32), 0), ((16, 64), 0),
                                      ((16, 64), 8)])
def test_sampled_pixels_equal_full_render(cuda_lib, case, tile, ppt):
    scene, cams = CASES[case]
    params = scene_to_device(scene)
    sc = cuda_lib.make_scene(params, scene.sh_degree)
    rz = cuda_lib.Rasterizer(cams, tile=tile, bg=(0.1, 0.2, 0.3), pixels_per_thread=ppt)
    full = rz.forward(sc).clone()
    fT = rz.records()["final_T"].clone()
    fN = rz.records()["n_contrib"].clone()
    for group, cell in ((2, (1, 1)), (3, (1, 1)), (4, "strip")):
        ss = rz.sample_set(group, seed=77 + group, cell=cell)
        m = _masks_from_samples(ss, cams, tile)
        m3 = torch.tensor(_packed3(m, cams), device="cuda")
        mt = torch.tensor(m, device="cuda")
        for masked in (False, True):
            img = torch.full_like(full, float("nan"))
            rz.records()["final_T"].fill_(-1.0)
            rz.forward(sc, images=img, samples=ss, masked=masked)
            torch.cuda.synchronize()
            assert torch.equal(img[m3], full[m3]), (group, masked)
            assert torch.isnan(img[~m3]).all()
            rec = rz.records()
            assert torch.equal(rec["final_T"][mt], fT[mt])
            assert torch.equal(rec["n_contrib"][mt], fN[mt])
            assert (rec["final_T"][~mt] == -1.0).all()


@pytest.mark.parametrize("case", sorted(CASES))
def test_sampled_forward_and_backward_match_oracle(cuda_lib, case):
    scene, cams = CASES[case]
    tile, bg, group, seed = (16, 16), (0.1, 0.2, 0.3), 3, 5
    ref = oracle.forward(scene, cams, tile, bg=bg)
    m = partial.packed_mask(cams, group, seed)
    m3 = _packed3(m, cams)
    amb = ref["amb"] != 0
    ok3 = _packed3(m & ~amb, cams)
    params = scene_to_device(scene)
    sc = cuda_lib.make_scene(params, scene.sh_degree)
    rz = cuda_lib.Rasterizer(cams, tile=tile, bg=bg)
    ss = rz.sample_set(group, seed)
    img = torch.zeros(3 * rz.pixels, device="cuda")
    rz.forward(sc, images=img, samples=ss)
    got = img.cpu().numpy().astype(np.float64)
    assert ok3.sum() > 0.3 * m3.sum()
    np.testing.assert_allclose(got[ok3], ref["img"][ok3], rtol=0, atol=1e-4)

    rng = np.random.default_rng(17)
    dimg = rng.normal(size=ref["img"].shape).astype(np.float32)
    dimg[~ok3] = 0.0  # off the samples and on ambiguous pixels
    grads, g2d, e1 = oracle.backward(scene, cams, ref, dimg.astype(np.float64), tile, bg)
    # the sampled backward reads only sampled pixels: garbage elsewhere must not matter
    d_dev = torch.tensor(dimg, device="cuda")
    d_dev[torch.tensor(~m3, device="cuda")] = 1e6
    gg = grads_like(params)
    rz.backward(sc, d_dev, gg, samples=ss)
    torch.cuda.synchronize()
    bad_g = np.zeros(scene.n, bool)
    bad_g[np.nonzero(ref["P"]["amb"])[0] % scene.n] = True
    touched = np.abs(grads["opacity_logits"]) > 0
    assert touched.sum() > 500
    for k in PARAMS:
        g = gg[k].cpu().numpy().astype(np.float64)[~bad_g]
        e = grads[k][~bad_g]
        assert_close_frac(g, e, 1e-3, 1e-6 * np.abs(e).max(), "d" + k)


def test_sampled_backward_equals_masked_full_backward(cuda_lib):
    scene, cams = CASES["same_res_4views"]
    tile = (16, 32)
    params = scene_to_device(scene)
    sc = cuda_lib.make_scene(params, scene.sh_degree)
    rz = cuda_lib.Rasterizer(cams, tile=tile)
    ss = rz.sample_set(4, seed=3)
    m3 = torch.tensor(_packed3(_masks_from_samples(ss, cams, tile), cams), device="cuda")
    gen = torch.Generator("cuda").manual_seed(4)
    d = torch.randn(3 * rz.pixels, device="cuda", generator=gen)
    dm = torch.where(m3, d, torch.zeros_like(d))
    rz.forward(sc)
    full = grads_like(params)
    rz.backward(sc, dm, full)
    out = {}
    for masked in (False, True):
        rz.forward(sc, samples=ss, masked=masked)
        gs = grads_like(params)
        rz.backward(sc, d, gs, samples=ss, masked=masked)
        out[masked] = gs
    torch.cuda.synchronize()
    for k in PARAMS:
        f = full[k].cpu().numpy()
        for masked in (False, True):
            assert_close_frac(out[masked][k].cpu().numpy(), f, 1e-3, 1e-5 * np.abs(f).max(), f"{k}/{masked}")


def test_group_one_is_the_full_render_and_empty_scene(cuda_lib):
    scene, cams = CASES["ragged_3views"]
    params = scene_to_device(scene)
    sc = cuda_lib.make_scene(params, scene.sh_degree)
    rz = cuda_lib.Rasterizer(cams, tile=(16, 16))
    full = rz.forward(sc).clone()
    ss = rz.sample_set(1, seed=0)
    assert int(ss.offsets[-1]) == rz.pixels
    img = torch.full_like(full, float("nan"))
    rz.forward(sc, images=img, samples=ss)
    assert torch.equal(img, full)
    empty = synth.make_scene(0, 3)
    pe = scene_to_device(empty)
    sce = cuda_lib.make_scene(pe, 3)
    rz2 = cuda_lib.Rasterizer(cams, tile=(16, 16), bg=(0.25, 0.5, 0.75))
    ss2 = rz2.sample_set(2, seed=1)
    img = torch.full((3 * rz2.pixels,), float("nan"), device="cuda")
    rz2.forward(sce, images=img, samples=ss2)
    m3 = torch.tensor(_packed3(_masks_from_samples(ss2, cams, (16, 16)), cams), device="cuda")
    bgv = torch.tensor(np.concatenate([np.repeat([0.25, 0.5, 0.75], int(w) * int(h))
                                       for w, h in zip(cams.width, cams.height)]), dtype=torch.float32,
                       device="cuda")
    assert torch.equal(img[m3], bgv[m3])
    assert torch.isnan(img[~m3]).all()
