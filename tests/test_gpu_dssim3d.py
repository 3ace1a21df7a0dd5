"""3D distance-aware D-SSIM (Sec. 5.1.2) and the merged images of a partial
render, on the GPU against the oracle (oracle/dssim3d.py).

  - the expected depth the forward writes with MVGS_FLAG_DEPTH matches the
    oracle's blend of camera depths (1e-4 relative, unambiguous pixels);
  - mvgs_merge_views: merged colour bit-exact with the owner view's pixel,
    surface points and kernel widths against the oracle's lift;
  - mvgs_dssim3d_loss: loss and gradient against the oracle on random images
    with rough surfaces, ragged sizes and pixels without a surface point;
  - mvgs_split_merged_grad sends each merged gradient to its owner view only.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import assert_close_frac, scene_to_device
from oracle import dssim3d, partial

pytestmark = pytest.mark.gpu


def _cam(cams, v):
    vm = np.asarray(cams.viewmat[v], np.float64)
    return dict(W=int(cams.width[v]), H=int(cams.height[v]), fx=float(cams.fx[v]), fy=float(cams.fy[v]),
                cx=float(cams.cx[v]), cy=float(cams.cy[v]), R=vm[:, :3], t=vm[:, 3])


@pytest.fixture(scope="module")
def rendered(cuda_lib):
    scene = synth.make_scene(8_000, 3, seed=7)
    cams = synth.make_cameras([(160, 120)] * 4, radius=4.0, seed=8)
    tile, group, seed = (16, 16), 2, 31
    ref = oracle.forward(scene, cams, tile)
    params = scene_to_device(scene)
    sc = cuda_lib.make_scene(params, 3)
    rz = cuda_lib.Rasterizer(cams, tile=tile)
    ss = rz.sample_set(group, seed)
    img = torch.zeros(3 * rz.pixels, device="cuda")
    rz.forward(sc, images=img, samples=ss, depth=True)
    rec = rz.records()
    return dict(scene=scene, cams=cams, tile=tile, group=group, seed=seed, ref=ref, rz=rz, img=img,
                depth=rec["depth_acc"].clone(), T=rec["final_T"].clone(), mask=partial.packed_mask(cams, group, seed))


def test_expected_depth_matches_oracle(rendered):
    ref, m = rendered["ref"], rendered["mask"]
    ok = m & (ref["amb"] == 0)
    got = rendered["depth"].cpu().numpy().astype(np.float64)
    assert ok.sum() > 0.3 * m.sum()
    assert_close_frac(got[ok], ref["depth"][ok], 1e-4, 1e-5, "expected depth")


def test_merge_matches_oracle(rendered, cuda_lib):
    cams, group, seed, ref = rendered["cams"], rendered["group"], rendered["seed"], rendered["ref"]
    rz = rendered["rz"]
    tgt = torch.tensor(synth.pack_images(synth.make_targets(cams)), device="cuda")
    M = cams.V // group
    H, W = int(cams.height[0]), int(cams.width[0])
    mimg = torch.full((M * 3 * H * W,), float("nan"), device="cuda")
    mtgt = torch.full_like(mimg, float("nan"))
    pts = torch.full_like(mimg, float("nan"))
    sig = torch.full((M * H * W,), float("nan"), device="cuda")
    cuda_lib.merge_views(rz.cams_c, group, seed, rendered["img"], tgt, rendered["depth"], rendered["T"], mimg, mtgt,
                         pts, sig)
    torch.cuda.synchronize()
    img_v = rendered["img"].cpu().numpy().reshape(cams.V, 3, H, W)
    tgt_v = tgt.cpu().numpy().reshape(cams.V, 3, H, W)
    dep_v = ref["depth"].reshape(cams.V, H, W)
    T_v = ref["T"].reshape(cams.V, H, W)
    amb_v = ref["amb"].reshape(cams.V, H, W) != 0
    for mi in range(M):
        views = range(mi * group, mi * group + group)
        exp_img, owner = dssim3d.merge_views([img_v[v] for v in range(cams.V)], None, group, seed, first=mi * group)
        exp_tgt, _ = dssim3d.merge_views([tgt_v[v] for v in range(cams.V)], None, group, seed, first=mi * group)
        got = mimg.cpu().numpy().reshape(M, 3, H, W)[mi]
        np.testing.assert_array_equal(got, exp_img)
        np.testing.assert_array_equal(mtgt.cpu().numpy().reshape(M, 3, H, W)[mi], exp_tgt)
        # the oracle's surface points from its own depth and T, per owner view
        X = np.zeros((3, H, W))
        S = np.zeros((H, W))
        amb = np.zeros((H, W), bool)
        opac = np.zeros((H, W))
        for v in views:
            Xv, Sv = dssim3d.lift(dep_v[v], T_v[v], _cam(cams, v))
            sel = owner == v
            X[:, sel] = Xv[:, sel]
            S[sel] = Sv[sel]
            amb |= sel & amb_v[v]
            opac[sel] = 1.0 - T_v[v][sel]
        gp = pts.cpu().numpy().reshape(M, 3, H, W)[mi]
        gs = sig.cpu().numpy().reshape(M, H, W)[mi]
        # z = D / (1 - T): compared where the accumulated opacity is not small
        # (float32 T near 1 makes the quotient ill-conditioned)
        ok = ~amb & (opac > 0.05)
        assert ok.sum() > 0.5 * H * W
        assert np.all((gs > 0) == (opac >= 1e-3) | (np.abs(opac - 1e-3) < 1e-5))
        assert_close_frac(gs[ok], S[ok], 2e-4, 1e-6, "sigma")
        assert_close_frac(gp[:, ok].T, X[:, ok].T, 2e-4, 2e-4, "points")


def _rough(W, H, rng, f=60.0):
    cam = dict(W=W, H=H, fx=f, fy=f, cx=W / 2, cy=H / 2, R=np.eye(3), t=np.zeros(3))
    depth = 2.0 + 0.3 * rng.uniform(size=(H, W)) + np.linspace(0, 1, W)[None, :]
    T = np.where(rng.uniform(size=(H, W)) < 0.05, 1.0 - 1e-5, rng.uniform(0, 0.5, size=(H, W)))
    return dssim3d.lift(depth * (1 - T), T, cam)


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_dssim3d_matches_oracle(cuda_lib, lam):
    rng = np.random.default_rng(11)
    shapes = [(37, 23), (16, 16), (50, 41)]
    I1s, I2s, Xs, Ss = [], [], [], []
    for W, H in shapes:
        X, S = _rough(W, H, rng)
        I1 = rng.uniform(size=(3, H, W))
        I1s.append(I1)
        I2s.append(np.clip(I1 + rng.normal(0, 0.2, size=I1.shape), 0, 1))
        Xs.append(X)
        Ss.append(S)
    hw = np.array([[H, W] for W, H in shapes], np.int32)
    pack = lambda arrs: torch.tensor(np.concatenate([a.reshape(-1) for a in arrs]).astype(np.float32), device="cuda")
    # the oracle runs on the float32-rounded inputs the GPU sees
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    ws = torch.empty(cuda_lib.dssim3d_workspace_size(hw), dtype=torch.uint8, device="cuda")
    loss = torch.empty(len(shapes), device="cuda")
    d = torch.empty(sum(3 * W * H for W, H in shapes), device="cuda")
    cuda_lib.dssim3d_loss(pack(I1s), pack(I2s), pack(Xs), pack(Ss), hw, lam, loss, d, ws)
    torch.cuda.synchronize()
    off = 0
    for i, (W, H) in enumerate(shapes):
        L, g, _ = dssim3d.dssim3d_loss(r32(I1s[i]), r32(I2s[i]), r32(Xs[i]), r32(Ss[i]), lam)
        assert abs(loss[i].item() - L) < 2e-6, (i, loss[i].item(), L)
        got = d[off:off + 3 * W * H].cpu().numpy().reshape(3, H, W) * len(shapes)
        assert_close_frac(got, g, 1e-3, 1e-4 * np.abs(g).max(), f"dL/dI image {i}")
        off += 3 * W * H


def test_split_sends_gradient_to_owner(rendered, cuda_lib):
    cams, group, seed = rendered["cams"], rendered["group"], rendered["seed"]
    rz = rendered["rz"]
    H, W = int(cams.height[0]), int(cams.width[0])
    M = cams.V // group
    dm = torch.randn(M * 3 * H * W, device="cuda")
    dv = torch.full((3 * rz.pixels,), float("nan"), device="cuda")
    cuda_lib.split_merged_grad(rz.cams_c, group, seed, dm, dv)
    torch.cuda.synchronize()
    dmn = dm.cpu().numpy().reshape(M, 3, H, W)
    dvn = dv.cpu().numpy().reshape(cams.V, 3, H, W)
    slot = partial.slot_image(seed, W, H, group)
    for v in range(cams.V):
        own = slot == v % group
        np.testing.assert_array_equal(dvn[v][:, own], dmn[v // group][:, own])
        assert (dvn[v][:, ~own] == 0).all()
