"""Pins the CPU oracle to facts outside itself (no GPU).

Each test ties one part of the oracle to something it does not compute
itself: a library routine for a textbook definition (scipy spherical
harmonics and rotations, torch conv2d), a closed form, a Monte-Carlo
estimate, a brute-force ordering, finite differences, or the paper's worked
example (tests/golden/opposite_cameras.json).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cams(W, H, f, R, t, pos, cx=None, cy=None, near=0.2):
    V = len(R)
    vm = np.zeros((V, 3, 4), np.float32)
    for v in range(V):
        vm[v, :, :3] = R[v]
        vm[v, :, 3] = t[v]
    return synth.Cameras(np.full(V, W, np.int32), np.full(V, H, np.int32), np.full(V, f, np.float32),
                         np.full(V, f, np.float32), np.full(V, W / 2 if cx is None else cx, np.float32),
                         np.full(V, H / 2 if cy is None else cy, np.float32), vm, np.asarray(pos, np.float32),
                         np.full(V, near, np.float32))


def _one_gaussian(mu, log_s, q, logit, rgb, deg=0):
    k = (deg + 1) ** 2
    sh = np.zeros((1, k, 3), np.float32)
    sh[0, 0] = (np.asarray(rgb) - 0.5) / (0.5 / math.sqrt(math.pi))
    return synth.Scene(np.asarray([mu], np.float32), np.asarray([log_s], np.float32), np.asarray([q], np.float32),
                       np.asarray([logit], np.float32), sh, deg)


# ---------------------------------------------------------------------------
# spherical harmonics and rotations against scipy
# ---------------------------------------------------------------------------
def test_sh_basis_matches_scipy_with_condon_shortley_phase():
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(5)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    got = oracle.sh_basis(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            Yc = sph_harm_y(l, abs(m), theta, phi)  # complex, Condon-Shortley phase included
            if m > 0:
                real = math.sqrt(2) * (-1) ** m * Yc.real
            elif m < 0:
                real = math.sqrt(2) * (-1) ** m * Yc.imag
            else:
                real = Yc.real
            expect = (-1) ** m * real  # the basis keeps the Condon-Shortley sign
            np.testing.assert_allclose(got[:, l * l + l + m], expect, rtol=0, atol=1e-12, err_msg=f"l={l} m={m}")


def test_quaternion_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(6)
    q = rng.normal(size=(50, 4)) * rng.uniform(0.2, 3.0, size=(50, 1))
    got = oracle.quat_to_rotation(q)
    exp = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()  # scipy is scalar-last
    np.testing.assert_allclose(got, exp, atol=1e-12)


# ---------------------------------------------------------------------------
# projection
# ---------------------------------------------------------------------------
def test_isotropic_on_axis_closed_form():
    f, W, H, z, s = 200.0, 64, 48, 2.5, 0.05
    cams = _cams(W, H, f, [np.eye(3)], [np.zeros(3)], [np.zeros(3)])
    sc = _one_gaussian([0, 0, z], [math.log(s)] * 3, [1, 0, 0, 0], 0.3, [0.2, 0.5, 0.9])
    P = oracle.project(sc, cams, (16, 16))
    sig2 = (f * s / z) ** 2
    vv = sig2 + 0.3
    np.testing.assert_allclose(P["cov"][0], [vv, 0.0, vv], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(P["conic"][0], [1 / vv, 0.0, 1 / vv], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(P["xy"][0], [W / 2, H / 2], atol=1e-9)
    np.testing.assert_allclose(P["depth"][0], z, rtol=1e-6)
    # equal eigenvalues: the discriminant is floored at 0.1
    assert P["radius"][0] == math.ceil(3 * math.sqrt(vv + math.sqrt(0.1)))
    np.testing.assert_allclose(P["rgb"][0], [0.2, 0.5, 0.9], atol=1e-6)
    np.testing.assert_allclose(P["opac"][0], 1 / (1 + math.exp(-0.3)), rtol=1e-6)


def test_projection_matches_monte_carlo_of_the_perspective_map():
    """EWA's local affine approximation: for a Gaussian small against its
    depth, the empirical mean and covariance of perspectively projected 3D
    samples match (mu', Sigma' - dilation I)."""
    rng = np.random.default_rng(7)
    cams = synth.make_cameras([(320, 240), (200, 260)], radius=4.0, seed=11)
    for trial in range(4):
        mu = rng.uniform(-0.6, 0.6, size=3)
        ls = rng.normal(-4.0, 0.4, size=3)
        q = rng.normal(size=4)
        sc = _one_gaussian(mu, ls, q, 0.0, [0.5, 0.5, 0.5])
        P = oracle.project(sc, cams, (16, 16))
        mu32 = sc.means[0].astype(np.float64)
        s = np.exp(sc.log_scales[0].astype(np.float64))
        from scipy.spatial.transform import Rotation
        qq = sc.quats[0].astype(np.float64)
        Rg = Rotation.from_quat(qq[[1, 2, 3, 0]] / np.linalg.norm(qq)).as_matrix()
        Sig = Rg @ np.diag(s ** 2) @ Rg.T
        X = rng.multivariate_normal(mu32, Sig, size=400_000)
        for v in range(cams.V):
            Rc = cams.viewmat[v, :, :3].astype(np.float64)
            tc = cams.viewmat[v, :, 3].astype(np.float64)
            Y = X @ Rc.T + tc
            u = cams.fx[v] * Y[:, 0] / Y[:, 2] + cams.cx[v]
            w = cams.fy[v] * Y[:, 1] / Y[:, 2] + cams.cy[v]
            emp = np.cov(np.stack([u, w]))
            a, b, c = P["cov"][v]
            model = np.array([[a - 0.3, b], [b, c - 0.3]])
            scale = np.sqrt(np.trace(model))
            assert np.abs(emp - model).max() < 0.03 * scale ** 2, (trial, v, emp, model)
            np.testing.assert_allclose([u.mean(), w.mean()], P["xy"][v], atol=0.02 * scale)


def test_quaternion_sign_and_scale_invariance():
    sc = synth.make_scene(200, 3, seed=3)
    cams = synth.make_cameras([(96, 80)] * 2, radius=3.0)
    P1 = oracle.project(sc, cams)
    sc2 = sc.subset(np.arange(sc.n))
    sc2.quats = (-2.0 * sc2.quats).astype(np.float32)  # exact in float32
    P2 = oracle.project(sc2, cams)
    for k in ("cov", "conic", "xy"):
        np.testing.assert_allclose(P1[k], P2[k], rtol=1e-6, atol=1e-9)
    np.testing.assert_array_equal(P1["radius"], P2["radius"])


# ---------------------------------------------------------------------------
# blending
# ---------------------------------------------------------------------------
def test_single_isotropic_gaussian_image_closed_form():
    f, W, H, z, s = 120.0, 40, 36, 2.0, 0.08
    cx, cy = float(np.float32(17.3)), float(np.float32(19.6))
    cams = _cams(W, H, f, [np.eye(3)], [np.zeros(3)], [np.zeros(3)], cx=cx, cy=cy)
    bg = np.array([0.2, 0.3, 0.7])
    for logit in (-1.0, 1.5, 6.0):  # the last one hits the 0.99 clamp
        sc = _one_gaussian([0, 0, z], [math.log(s)] * 3, [1, 0, 0, 0], logit, [0.9, 0.4, 0.1])
        f_ = oracle.forward(sc, cams, (16, 16), bg=bg)
        # the inputs as the oracle sees them (float32, widened exactly)
        rgb = 0.5 / math.sqrt(math.pi) * sc.sh[0, 0].astype(np.float64) + 0.5
        o = 1 / (1 + math.exp(-float(sc.opacity_logits[0])))
        s32 = math.exp(float(sc.log_scales[0, 0]))
        vv = (f * s32 / z) ** 2 + 0.3
        r = math.ceil(3 * math.sqrt(vv + math.sqrt(0.1)))
        img = f_["img"].reshape(3, H, W)
        ys, xs = np.mgrid[0:H, 0:W]
        dx, dy = xs + 0.5 - cx, ys + 0.5 - cy
        alpha = np.minimum(0.99, o * np.exp(-(dx * dx + dy * dy) / (2 * vv)))
        inside = (np.abs(dx) <= r) & (np.abs(dy) <= r) & (alpha >= 1 / 255)
        alpha = np.where(inside, alpha, 0.0)
        exp = rgb[:, None, None] * alpha + (1 - alpha) * bg[:, None, None]
        np.testing.assert_allclose(img, exp, rtol=0, atol=1e-12)
        np.testing.assert_allclose(f_["T"].reshape(H, W), 1 - alpha, rtol=0, atol=1e-12)
        assert inside.sum() > 20


def test_white_gaussians_on_black_give_one_minus_transmittance():
    """With every colour 1 and a black background Eq. 1 telescopes:
    sum_i alpha_i T_i = 1 - T_final; on a white background C = 1."""
    sc = synth.make_scene(300, 0, seed=9)
    sc.sh[:, 0, :] = 0.5 / (0.5 / math.sqrt(math.pi))
    cams = synth.make_cameras([(64, 48), (50, 70)], radius=3.0)
    f0 = oracle.forward(sc, cams, (16, 16), bg=(0, 0, 0))
    C = np.concatenate([f0["img"][3 * a:3 * b].reshape(3, -1) for a, b in
                        zip(*(lambda pb: (pb[:-1], pb[1:]))(oracle.layout(cams, (16, 16))[3]))], axis=1)
    np.testing.assert_allclose(C, np.broadcast_to(1 - f0["T"], C.shape), atol=1e-12)
    f1 = oracle.forward(sc, cams, (16, 16), bg=(1, 1, 1))
    np.testing.assert_allclose(f1["img"], 1.0, atol=1e-12)
    assert f0["T"].min() >= 1e-4 and f0["T"].max() <= 1.0
    assert (f0["T"] < 0.5).mean() > 0.2  # the scene is not trivially transparent


def test_tiled_lists_equal_per_pixel_bruteforce_and_tile_size_invariance():
    sc = synth.make_scene(64, 3, seed=4)
    sc.log_scales += np.float32(0.8)
    cams = synth.make_cameras([(32, 32), (40, 24)], radius=3.0, seed=8)
    bg = (0.1, 0.2, 0.3)
    ref = None
    for tile in ((8, 8), (16, 16), (16, 32), (32, 8)):
        f = oracle.forward(sc, cams, tile, bg=bg)
        if ref is None:
            ref = f
        else:
            np.testing.assert_array_equal(f["img"], ref["img"])
            np.testing.assert_array_equal(f["T"], ref["T"])
    P = ref["P"]
    _, _, _, pix_base = oracle.layout(cams, (8, 8))
    pix = []
    for v in range(cams.V):
        ys, xs = np.mgrid[0:cams.height[v], 0:cams.width[v]]
        pix.append(np.stack([np.full(xs.size, v), xs.ravel(), ys.ravel()], 1))
    pix = np.concatenate(pix)
    C, T, nc, amb = oracle.render_pixels_bruteforce(cams, P, pix, bg=bg)
    img = ref["img"]
    for v in range(cams.V):
        sel = pix[:, 0] == v
        H, W = cams.height[v], cams.width[v]
        got = img[3 * pix_base[v]:3 * pix_base[v + 1]].reshape(3, H * W).T
        np.testing.assert_array_equal(got, C[sel])
        np.testing.assert_array_equal(ref["T"][pix_base[v]:pix_base[v + 1]], T[sel])
    assert nc.max() > 3


def test_sort_invariants():
    sc = synth.make_scene(3000, 1, seed=2)
    cams = synth.make_cameras([(200, 120), (64, 64), (130, 90)], radius=3.0)
    P = oracle.project(sc, cams, (16, 16))
    keys, recs, ranges = oracle.sort_keys(cams, (16, 16), P["valid"], P["rect"], P["depth"].astype(np.float32))
    area = (P["rect"][:, 2] - P["rect"][:, 0]) * (P["rect"][:, 3] - P["rect"][:, 1]) * (P["valid"] != 0)
    assert len(keys) == area.sum()
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) and np.all(keys[1:] >= keys[:-1])
    np.testing.assert_array_equal(np.bincount(recs, minlength=len(area)), area)
    # ranges partition [0, K) in global tile order
    nz = ranges[:, 1] > ranges[:, 0]
    r = ranges[nz]
    assert r[0, 0] == 0 and r[-1, 1] == len(keys) and np.all(r[1:, 0] == r[:-1, 1])
    # inside a tile: depth then Gaussian index, matches numpy's lexsort
    N = sc.n
    g = recs % N
    order = np.lexsort((g, keys))
    np.testing.assert_array_equal(order, np.arange(len(keys)))
    # the tile of each key is one its record's rectangle covers
    _, _, tile_base, _ = oracle.layout(cams, (16, 16))
    tiles_x = oracle.layout(cams, (16, 16))[0]
    gt = (keys >> np.uint64(32)).astype(np.int64)
    v = recs // N
    local = gt - tile_base[v]
    tx, ty = local % tiles_x[v], local // tiles_x[v]
    rc = P["rect"][recs]
    assert np.all((tx >= rc[:, 0]) & (tx < rc[:, 2]) & (ty >= rc[:, 1]) & (ty < rc[:, 3]))


# ---------------------------------------------------------------------------
# derivatives
# ---------------------------------------------------------------------------
def _fd_setup():
    sc = synth.make_scene(40, 3, seed=12)
    sc.log_scales += np.float32(0.9)
    cams = synth.make_cameras([(48, 40), (40, 32)], radius=3.0, seed=13)
    return sc, cams


def test_backward_matches_central_differences():
    sc, cams = _fd_setup()
    tile, bg = (16, 16), (0.3, 0.1, 0.2)
    base = oracle.forward(sc, cams, tile, bg=bg)
    rng = np.random.default_rng(14)
    w = rng.normal(size=base["img"].shape)
    grads, g2d, e1 = oracle.backward(sc, cams, base, w, tile, bg)
    fields = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    # parameters of Gaussians that actually contribute
    contributing = np.unique(base["S"][1] % sc.n)
    checked = {f: 0 for f in fields}
    for field in fields:
        arr = getattr(sc, field)
        tries = 0
        while checked[field] < 8 and tries < 80:
            tries += 1
            g = int(rng.choice(contributing))
            idx = (g,) + tuple(int(rng.integers(0, s)) for s in arr.shape[1:])
            x0 = float(arr[idx])
            h = 1e-4 * max(1.0, abs(x0))
            vals = []
            hashes = []
            xs = []
            for sgn in (1, -1):
                arr[idx] = np.float32(x0 + sgn * h)
                xs.append(float(arr[idx]))
                f = oracle.forward(sc, cams, tile, bg=bg)
                vals.append(float((w * f["img"]).sum()))
                hashes.append((f["chash"].copy(), f["P"]["radius"].copy(), f["P"]["clampmask"].copy()))
            arr[idx] = np.float32(x0)
            same = all(np.array_equal(a, b) for a, b in zip(hashes[0], hashes[1])) and \
                np.array_equal(hashes[0][0], base["chash"])
            if not same:
                continue
            fd = (vals[0] - vals[1]) / (xs[0] - xs[1])
            an = grads[field][idx]
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)) + 1e-6, (field, idx, fd, an)
            checked[field] += 1
        assert checked[field] >= 5, (field, checked)


def test_single_gaussian_colour_and_opacity_gradients():
    """dC/drgb = alpha and dC/do = G (rgb - bg) below the clamp."""
    f, W, H, z, s = 100.0, 24, 24, 2.0, 0.1
    cx, cy = float(np.float32(11.2)), float(np.float32(12.7))
    cams = _cams(W, H, f, [np.eye(3)], [np.zeros(3)], [np.zeros(3)], cx=cx, cy=cy)
    bg = np.array([0.1, 0.5, 0.3])
    sc = _one_gaussian([0, 0, z], [math.log(s)] * 3, [1, 0, 0, 0], 0.2, [0.7, 0.2, 0.4])
    rgb = 0.5 / math.sqrt(math.pi) * sc.sh[0, 0].astype(np.float64) + 0.5
    o = 1 / (1 + math.exp(-float(sc.opacity_logits[0])))
    s32 = math.exp(float(sc.log_scales[0, 0]))
    fw = oracle.forward(sc, cams, (16, 16), bg=bg)
    x, y = 13, 9
    for ch in range(3):
        d = np.zeros_like(fw["img"])
        d[ch * H * W + y * W + x] = 1.0
        g2d, _ = oracle.render_backward(cams, fw["P"], fw["S"], d, bg)
        vv = (f * s32 / z) ** 2 + 0.3
        G = math.exp(-((x + 0.5 - cx) ** 2 + (y + 0.5 - cy) ** 2) / (2 * vv))
        np.testing.assert_allclose(g2d[0, 6 + ch], o * G, rtol=1e-10)
        np.testing.assert_allclose(g2d[0, 5], G * (rgb[ch] - bg[ch]), rtol=1e-10)


# ---------------------------------------------------------------------------
# densification statistics: the supplement's worked example and invariants
# ---------------------------------------------------------------------------
def test_opposite_cameras_nullify_summed_2d_gradients():
    gold = json.load(open(os.path.join(GOLDEN, "opposite_cameras.json")))
    W = H = 32
    R = [np.array(gold["camera_1"]["R"], float), np.array(gold["camera_2"]["R"], float)]
    t = [np.array(gold["camera_1"]["t"], float), np.array(gold["camera_2"]["t"], float)]
    pos = [gold["camera_1"]["centre"], gold["camera_2"]["centre"]]
    cams = _cams(W, H, 40.0, R, t, pos)
    sc = _one_gaussian([0, 0, 0], [math.log(0.05), math.log(0.08), math.log(0.06)], [1, 0, 0, 0], 0.0,
                       [0.6, 0.6, 0.6])
    fw = oracle.forward(sc, cams, (16, 16))
    # a loss whose 3D positional gradient is along world +x (grad_3d) in both
    # views: world +x is image +x in camera 1 and image -x in camera 2
    xs = np.arange(W) + 0.5 - W / 2
    d1 = np.broadcast_to(xs[None, None, :], (3, H, W)).ravel()
    d = np.concatenate([d1, -d1])
    grads, g2d, e1 = oracle.backward(sc, cams, fw, d)
    gx1, gy1 = g2d[0, :2]
    gx2, gy2 = g2d[1, :2]
    exp = gold["expected"]
    assert np.sign(gx1) == exp["x_sign_camera_1"] and np.sign(gx2) == exp["x_sign_camera_2"]
    assert abs(gy1) < 1e-12 * abs(gx1) and abs(gy2) < 1e-12 * abs(gx1)
    E1, E2, Eold, denom = oracle.adc_statistics(g2d, e1, fw["P"]["valid"], 2)
    assert Eold[0] < 1e-12 * E2[0]
    np.testing.assert_allclose(E2[0], 2 * abs(gx1), rtol=1e-12)
    assert E1[0] >= E2[0] and denom[0] == 2
    # the 3D gradient itself points along world +x, as in the example
    gm = grads["means"][0]
    assert gm[0] > 0 and abs(gm[1]) < 1e-9 * abs(gm[0]) and abs(gm[2]) < 1e-9 * abs(gm[0])


def test_adc_invariants_and_single_pixel_equality():
    sc = synth.make_scene(400, 1, seed=21)
    cams = synth.make_cameras([(48, 48)] * 3, radius=3.0, seed=22)
    fw = oracle.forward(sc, cams, (16, 16))
    rng = np.random.default_rng(23)
    d = rng.normal(size=fw["img"].shape)
    _, g2d, e1 = oracle.backward(sc, cams, fw, d)
    E1, E2, Eold, _ = oracle.adc_statistics(g2d, e1, fw["P"]["valid"], 3)
    assert np.all(E1 >= E2 - 1e-12) and np.all(E2 >= Eold - 1e-12)
    assert (E1 > E2 * (1 + 1e-6)).sum() > 50
    # one pixel of one view carries the loss: the three metrics coincide
    d1 = np.zeros_like(d)
    _, _, _, pix_base = oracle.layout(cams, (16, 16))
    d1[3 * pix_base[1] + 20 * 48 + 17] = 1.0
    _, g2d, e1 = oracle.backward(sc, cams, fw, d1)
    E1, E2, Eold, _ = oracle.adc_statistics(g2d, e1, fw["P"]["valid"], 3)
    assert E1.max() > 0
    np.testing.assert_allclose(E1, E2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(E2, Eold, rtol=1e-12, atol=1e-15)


def test_tile_rect_covers_every_pixel_a_gaussian_can_reach():
    """The tile rectangle (bounding box of the alpha >= 1/255 ellipse inside
    the support square) holds every pixel where the Gaussian passes the
    support rule and the 1/255 test, checked pixel by pixel."""
    sc = synth.make_scene(400, 0, seed=31)
    sc.opacity_logits[:] = np.random.default_rng(1).normal(0, 2.5, sc.n).astype(np.float32)
    cams = synth.make_cameras([(160, 120), (90, 70)], radius=3.0, seed=32)
    for tile in ((8, 8), (16, 16), (32, 16)):
        P = oracle.project(sc, cams, tile)
        for v in range(cams.V):
            W, H = int(cams.width[v]), int(cams.height[v])
            ys, xs = np.mgrid[0:H, 0:W]
            for g in range(sc.n):
                r = v * sc.n + g
                dx = xs + 0.5 - P["xy"][r, 0]
                dy = ys + 0.5 - P["xy"][r, 1]
                A, B, C = P["conic"][r]
                power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
                alpha = np.minimum(0.99, P["opac"][r] * np.exp(power))
                rad = P["radius"][r]
                hit = (np.abs(dx) <= rad) & (np.abs(dy) <= rad) & (alpha >= 1 / 255)
                if not P["valid"][r]:
                    assert not hit.any() or P["opac"][r] <= 1 / 255 or rad == 0
                    continue
                x0, y0, x1, y1 = P["rect"][r]
                tx, ty = xs[hit] // tile[0], ys[hit] // tile[1]
                assert np.all((tx >= x0) & (tx < x1) & (ty >= y0) & (ty < y1)), (v, g)


# ---------------------------------------------------------------------------
# the projection far off the optical axis (guard band of the Jacobian)
# ---------------------------------------------------------------------------
def _camera_space(sc, cams, v):
    vm = cams.viewmat[v].astype(np.float64)
    return sc.means.astype(np.float64) @ vm[:, :3].T + vm[:, 3]


def _band(cams, v):
    """The guard band of the 3DGS projection: 1.3 x the half-FOV tangents."""
    return (1.3 * 0.5 * float(cams.width[v]) / float(cams.fx[v]),
            1.3 * 0.5 * float(cams.height[v]) / float(cams.fy[v]))


def test_guard_band_covariance_is_the_projection_at_the_band_edge():
    """Beyond 1.3 x the half-FOV tangent the EWA Jacobian is taken at the
    band's edge (3DGS reading): the projected covariance of a Gaussian out
    there equals that of the same Gaussian moved, at the same depth, onto the
    edge -- where it is the plain perspective map, checked against Monte
    Carlo samples pushed through it -- while its projected mean is the
    pinhole projection of the unmoved mean."""
    sc, cams = synth.off_axis_scene(24, 0, sh_degree=0, seed=41)
    sc.log_scales[:] = np.random.default_rng(42).normal(-4.0, 0.3, size=sc.log_scales.shape).astype(np.float32)
    N = sc.n
    P = oracle.project(sc, cams, (16, 16))
    t = _camera_space(sc, cams, 0)  # the first camera is the identity: world = camera
    limx, limy = _band(cams, 0)
    ux, uy = t[:, 0] / t[:, 2], t[:, 1] / t[:, 2]
    out_x, out_y = np.abs(ux) > limx, np.abs(uy) > limy
    assert (out_x & (ux > 0)).any() and (out_x & (ux < 0)).any() and (out_y & (uy > 0)).any() \
        and (out_y & (uy < 0)).any() and (out_x & out_y).any()
    edge = sc.subset(np.arange(N))
    ex = np.clip(ux, -limx, limx) * t[:, 2]
    ey = np.clip(uy, -limy, limy) * t[:, 2]
    # float32 rounding keeps the moved means on (not beyond) the edge
    ex = np.where(np.abs(ex) > limx * t[:, 2], np.nextafter(ex.astype(np.float32), np.float32(0)), ex)
    ey = np.where(np.abs(ey) > limy * t[:, 2], np.nextafter(ey.astype(np.float32), np.float32(0)), ey)
    edge.means = np.stack([ex, ey, t[:, 2]], 1).astype(np.float32)
    Pe = oracle.project(edge, cams, (16, 16))
    np.testing.assert_allclose(P["cov"][:N], Pe["cov"][:N], rtol=1e-6, atol=1e-9)
    # projected means: K [R | t] applied to the homogeneous (unmoved) mean
    K = np.array([[cams.fx[0], 0, cams.cx[0]], [0, cams.fy[0], cams.cy[0]], [0, 0, 1]], np.float64)
    h = (K @ np.concatenate([cams.viewmat[0].astype(np.float64)], 0) @
         np.concatenate([sc.means.astype(np.float64), np.ones((N, 1))], 1).T).T
    np.testing.assert_allclose(P["xy"][:N], h[:, :2] / h[:, 2:], rtol=0, atol=1e-9)
    assert np.abs(P["xy"][:N, 0] - Pe["xy"][:N, 0])[out_x].min() > 1.0  # the mean itself is not moved
    # the covariance at the edge is the perspective map's (Monte Carlo)
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(43)
    for g in np.flatnonzero(out_x | out_y)[:6]:
        s = np.exp(edge.log_scales[g].astype(np.float64))
        qq = edge.quats[g].astype(np.float64)
        Rg = Rotation.from_quat(qq[[1, 2, 3, 0]] / np.linalg.norm(qq)).as_matrix()
        X = rng.multivariate_normal(edge.means[g].astype(np.float64), Rg @ np.diag(s ** 2) @ Rg.T, size=300_000)
        u = cams.fx[0] * X[:, 0] / X[:, 2] + cams.cx[0]
        w = cams.fy[0] * X[:, 1] / X[:, 2] + cams.cy[0]
        emp = np.cov(np.stack([u, w]))
        a, b, c = P["cov"][g]
        model = np.array([[a - 0.3, b], [b, c - 0.3]])
        assert np.abs(emp - model).max() < 0.03 * np.trace(model), (g, emp, model)


def test_backward_through_the_guard_band_matches_central_differences():
    """Central differences of the whole forward w.r.t. the parameters of
    Gaussians beyond the guard band (on both sides, on both axes) agree
    with the oracle's reverse mode, which holds the band's edge fixed in
    view-angle tangent (so it moves with the depth)."""
    sc, cams = synth.off_axis_scene(30, 10, sh_degree=1, seed=40)
    tile, bg = (16, 16), (0.2, 0.1, 0.3)
    N = sc.n
    base = oracle.forward(sc, cams, tile, bg=bg)
    rng = np.random.default_rng(44)
    w = rng.normal(size=base["img"].shape)
    grads, g2d, e1 = oracle.backward(sc, cams, base, w, tile, bg)
    far = np.zeros(N, bool)
    for v in range(cams.V):
        t = _camera_space(sc, cams, v)
        limx, limy = _band(cams, v)
        # well beyond the edge: no step below moves a Gaussian across it
        far |= (np.abs(t[:, 0] / t[:, 2]) > 1.05 * limx) | (np.abs(t[:, 1] / t[:, 2]) > 1.05 * limy)
    contributing = np.intersect1d(np.unique(base["S"][1] % N), np.flatnonzero(far))
    assert len(contributing) >= 15
    checked = {}
    for field in ("means", "log_scales", "quats", "opacity_logits"):
        arr = getattr(sc, field)
        checked[field] = 0
        tries = 0
        while checked[field] < 10 and tries < 120:
            tries += 1
            g = int(rng.choice(contributing))
            idx = (g,) + tuple(int(rng.integers(0, s)) for s in arr.shape[1:])
            if field == "means" and checked[field] < 4:
                idx = (g, 2)  # depth: the band's edge moves with it
            x0 = float(arr[idx])
            h = 1e-4 * max(1.0, abs(x0))
            vals, states, xs = [], [], []
            for sgn in (1, -1):
                arr[idx] = np.float32(x0 + sgn * h)
                xs.append(float(arr[idx]))
                f = oracle.forward(sc, cams, tile, bg=bg)
                vals.append(float((w * f["img"]).sum()))
                states.append((f["chash"].copy(), f["P"]["radius"].copy(), f["P"]["clampmask"].copy()))
            arr[idx] = np.float32(x0)
            if not (all(np.array_equal(a, b) for a, b in zip(*states)) and
                    np.array_equal(states[0][0], base["chash"])):
                continue
            fd = (vals[0] - vals[1]) / (xs[0] - xs[1])
            an = grads[field][idx]
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)) + 1e-6, (field, idx, fd, an)
            checked[field] += 1
        assert checked[field] >= 6, checked


# ---------------------------------------------------------------------------
# expected depth (the surface the 3D distance-aware D-SSIM lifts pixels to)
# ---------------------------------------------------------------------------
def test_expected_depth_of_one_gaussian_is_depth_times_alpha():
    f, W, H, z, s = 120.0, 40, 36, 2.5, 0.08
    cx, cy = float(np.float32(18.3)), float(np.float32(16.6))
    cams = _cams(W, H, f, [np.eye(3)], [np.zeros(3)], [np.zeros(3)], cx=cx, cy=cy)
    for logit in (-0.5, 6.0):  # below and at the 0.99 clamp
        sc = _one_gaussian([0, 0, z], [math.log(s)] * 3, [1, 0, 0, 0], logit, [0.3, 0.6, 0.9])
        fw = oracle.forward(sc, cams, (16, 16))
        o = 1 / (1 + math.exp(-float(sc.opacity_logits[0])))
        vv = (f * math.exp(float(sc.log_scales[0, 0])) / z) ** 2 + 0.3
        r = math.ceil(3 * math.sqrt(vv + math.sqrt(0.1)))
        ys, xs = np.mgrid[0:H, 0:W]
        dx, dy = xs + 0.5 - cx, ys + 0.5 - cy
        alpha = np.minimum(0.99, o * np.exp(-(dx * dx + dy * dy) / (2 * vv)))
        alpha = np.where((np.abs(dx) <= r) & (np.abs(dy) <= r) & (alpha >= 1 / 255), alpha, 0.0)
        np.testing.assert_allclose(fw["depth"].reshape(H, W), z * alpha, rtol=0, atol=1e-12)
        assert (alpha > 0).sum() > 20


def test_expected_depth_weights_each_gaussian_by_its_blend_weight():
    """Three overlapping Gaussians at three depths with pure red, green and
    blue colours on black: the colour channels are the blend weights
    alpha_i T_i (Eq. 1), so the expected depth is sum_i z_i C_i; with all
    at one depth, D / (1 - T_final) is that depth."""
    f, W, H = 80.0, 32, 32
    cams = _cams(W, H, f, [np.eye(3)], [np.zeros(3)], [np.zeros(3)])
    rgb = np.eye(3)
    for depths in ((1.5, 2.0, 2.6), (2.2, 2.2, 2.2)):
        means = [[0.05 * (i - 1) * z, 0.03 * (1 - i) * z, z] for i, z in enumerate(depths)]
        sh = ((rgb - 0.5) / (0.5 / math.sqrt(math.pi)))[:, None, :].astype(np.float32)
        sc = synth.Scene(np.asarray(means, np.float32), np.full((3, 3), math.log(0.12), np.float32),
                         np.tile(np.float32([1, 0, 0, 0]), (3, 1)), np.float32([0.5, 1.0, 2.0]), sh, 0)
        fw = oracle.forward(sc, cams, (16, 16))
        C = fw["img"].reshape(3, H * W)
        z32 = sc.means[:, 2].astype(np.float64)
        # the colours are 1 and 0 up to the float32 rounding of the SH coefficient
        np.testing.assert_allclose(fw["P"]["rgb"], rgb, atol=1e-7)
        np.testing.assert_allclose(fw["depth"], (z32[:, None] * C).sum(0), rtol=1e-6, atol=1e-12)
        covered = (1 - fw["T"]) > 1e-3
        assert covered.sum() > 50 and (C > 1e-3).sum(1).min() > 20
        if len(set(depths)) == 1:
            np.testing.assert_allclose(fw["depth"][covered] / (1 - fw["T"][covered]), z32[0], rtol=1e-12)
        else:
            assert np.abs(fw["depth"][covered] / (1 - fw["T"][covered]) - z32[0]).max() > 0.1
