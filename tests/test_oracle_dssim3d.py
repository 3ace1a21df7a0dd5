"""Pins of the 3D distance-aware D-SSIM oracle (oracle/dssim3d.py)."""
import numpy as np

from oracle import dssim3d, losses, partial


def _plane_cam(W, H, f=40.0):
    return dict(W=W, H=H, fx=f, fy=f, cx=W / 2, cy=H / 2, R=np.eye(3), t=np.zeros(3))


def test_lift_round_trips_through_the_camera():
    rng = np.random.default_rng(1)
    W, H = 9, 7
    R = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    R *= np.sign(np.linalg.det(R))
    cam = dict(W=W, H=H, fx=30.0, fy=25.0, cx=4.1, cy=3.3, R=R, t=rng.normal(size=3))
    z = rng.uniform(1, 3, size=(H, W))
    T = rng.uniform(0.0, 0.5, size=(H, W))
    X, sig = dssim3d.lift(z * (1 - T), T, cam)
    pc = np.einsum("ij,jhw->ihw", R, X) + cam["t"][:, None, None]
    ys, xs = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    np.testing.assert_allclose(pc[2], z, rtol=1e-12)
    np.testing.assert_allclose(cam["fx"] * pc[0] / pc[2] + cam["cx"], xs, atol=1e-9)
    np.testing.assert_allclose(cam["fy"] * pc[1] / pc[2] + cam["cy"], ys, atol=1e-9)
    np.testing.assert_allclose(sig, 1.5 * z / cam["fx"], rtol=1e-12)
    # no surface point below the opacity floor
    X2, sig2 = dssim3d.lift(z, np.full((H, W), 1 - 1e-4), cam)
    assert (sig2 == 0).all()


def test_fronto_parallel_plane_gives_the_2d_ssim_inside():
    # one camera, every pixel at depth 2: K* is the 11x11 sigma-1.5 window, so
    # away from the border the SSIM map is the 2D one of the (pinned) 2D oracle
    rng = np.random.default_rng(2)
    H, W = 24, 27
    cam = _plane_cam(W, H)
    X, sig = dssim3d.lift(np.full((H, W), 2.0), np.zeros((H, W)), cam)
    I1 = rng.uniform(size=(3, H, W))
    I2 = np.clip(I1 + rng.normal(0, 0.1, size=I1.shape), 0, 1)
    _, _, S3 = dssim3d.dssim3d_loss(I1, I2, X, sig)
    S2 = losses.ssim_map(I1, I2, losses.gaussian_window())[0]
    np.testing.assert_allclose(S3[:, 5:-5, 5:-5], S2[:, 5:-5, 5:-5], rtol=0, atol=1e-12)


def test_identical_images_and_isolated_points():
    rng = np.random.default_rng(3)
    H, W = 12, 13
    I = rng.uniform(size=(3, H, W))
    X = rng.normal(size=(3, H, W)) * 100.0  # far apart: each window is its centre alone
    sig = np.full((H, W), 1e-3)
    loss, g, S = dssim3d.dssim3d_loss(I, I, X, sig, lam=1.0)
    assert abs(loss) < 1e-12 and np.abs(g).max() < 1e-12
    I2 = rng.uniform(size=(3, H, W))
    _, _, S = dssim3d.dssim3d_loss(I, I2, X, sig)
    closed = (2 * I * I2 + dssim3d.C1) / (I ** 2 + I2 ** 2 + dssim3d.C1)  # sigma terms are C2 / C2
    np.testing.assert_allclose(S, closed, rtol=1e-12)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    H, W = 9, 11
    cam = _plane_cam(W, H, f=8.0)
    depth = rng.uniform(1.5, 2.5, size=(H, W))  # a rough surface: weights vary
    X, sig = dssim3d.lift(depth, np.zeros((H, W)), cam)
    I1 = rng.uniform(0.1, 0.9, size=(3, H, W))
    I2 = rng.uniform(0.1, 0.9, size=(3, H, W))
    wts = dssim3d.window_weights(X, sig)
    loss, g, _ = dssim3d.dssim3d_loss(I1, I2, X, sig, lam=0.6, weights=wts)
    h = 1e-6
    for _ in range(25):
        c, y, x = rng.integers(0, 3), rng.integers(0, H), rng.integers(0, W)
        a, b = I1.copy(), I1.copy()
        a[c, y, x] += h
        b[c, y, x] -= h
        fd = (dssim3d.dssim3d_loss(a, I2, X, sig, 0.6, wts)[0] - dssim3d.dssim3d_loss(b, I2, X, sig, 0.6, wts)[0]) / (2 * h)
        assert abs(fd - g[c, y, x]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (c, y, x, fd, g[c, y, x])


def test_merged_image_takes_each_pixel_from_its_slot_view():
    rng = np.random.default_rng(5)
    imgs = [rng.uniform(size=(3, 10, 14)) for _ in range(6)]
    merged, owner = dssim3d.merge_views(imgs, None, 3, seed=7, first=3)
    slot = partial.slot_image(7, 14, 10, 3)
    np.testing.assert_array_equal(owner, 3 + slot)
    for y in range(10):
        for x in range(14):
            np.testing.assert_array_equal(merged[:, y, x], imgs[owner[y, x]][:, y, x])
