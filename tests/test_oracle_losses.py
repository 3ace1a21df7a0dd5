"""Pins the oracle's L1 + D-SSIM loss (SSIM equations of Sec. 5.1.2) to
torch's conv2d, to closed forms and to finite differences (no GPU)."""
import numpy as np
import torch

import oracle
from oracle import losses


def _ssim_torch(i1, i2, size=11, sigma=1.5):
    """The same definition evaluated with a library 2D convolution (grouped,
    zero padded, float64)."""
    x = np.arange(size) - (size - 1) / 2
    g = np.exp(-x ** 2 / (2 * sigma ** 2))
    g /= g.sum()
    k2 = torch.tensor(np.outer(g, g), dtype=torch.float64)
    C = i1.shape[0]
    w = k2.expand(C, 1, size, size).contiguous()
    a = torch.tensor(i1, dtype=torch.float64)[None]
    b = torch.tensor(i2, dtype=torch.float64)[None]
    conv = lambda t: torch.nn.functional.conv2d(t, w, padding=size // 2, groups=C)  # noqa: E731
    m1, m2 = conv(a), conv(b)
    s11 = conv(a * a) - m1 * m1
    s22 = conv(b * b) - m2 * m2
    s12 = conv(a * b) - m1 * m2
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    S = (2 * m1 * m2 + c1) * (2 * s12 + c2) / ((m1 * m1 + m2 * m2 + c1) * (s11 + s22 + c2))
    return S[0].numpy()


def test_ssim_map_matches_torch_conv2d():
    rng = np.random.default_rng(1)
    i1 = rng.uniform(size=(3, 37, 52))
    i2 = np.clip(i1 + rng.normal(0, 0.2, size=i1.shape), 0, 1)
    S, _ = losses.ssim_map(i1, i2, losses.gaussian_window())
    np.testing.assert_allclose(S, _ssim_torch(i1, i2), atol=1e-12)


def test_identical_images_have_zero_dssim_and_zero_gradient():
    rng = np.random.default_rng(2)
    img = [rng.uniform(size=(3, 20, 30)), rng.uniform(size=(3, 15, 9))]
    per, total, grads = losses.dssim_l1_loss(img, img, lam=1.0)
    np.testing.assert_allclose(per, 0.0, atol=1e-14)
    for g in grads:
        np.testing.assert_allclose(g, 0.0, atol=1e-14)


def test_constant_images_interior_closed_form():
    a, b = 0.3, 0.7
    i1 = np.full((3, 40, 40), a)
    i2 = np.full((3, 40, 40), b)
    S, _ = losses.ssim_map(i1, i2, losses.gaussian_window())
    inner = S[:, 5:-5, 5:-5]
    c1 = 0.01 ** 2
    np.testing.assert_allclose(inner, (2 * a * b + c1) / (a * a + b * b + c1), rtol=1e-12)
    # zero padding darkens the border means, so the border differs
    assert abs(S[0, 0, 0] - inner[0, 0, 0]) > 1e-3


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    imgs = [rng.uniform(size=(3, 14, 17)), rng.uniform(size=(3, 9, 12))]
    tg = [rng.uniform(size=i.shape) for i in imgs]
    _, L0, grads = losses.dssim_l1_loss(imgs, tg, lam=0.2)
    for v in range(2):
        for _ in range(25):
            idx = tuple(int(rng.integers(0, s)) for s in imgs[v].shape)
            h = 1e-6
            x0 = imgs[v][idx]
            imgs[v][idx] = x0 + h
            Lp = losses.dssim_l1_loss(imgs, tg, 0.2, want_grad=False)[1]
            imgs[v][idx] = x0 - h
            Lm = losses.dssim_l1_loss(imgs, tg, 0.2, want_grad=False)[1]
            imgs[v][idx] = x0
            fd = (Lp - Lm) / (2 * h)
            np.testing.assert_allclose(grads[v][idx], fd, rtol=1e-5, atol=1e-10)


def test_l1_weight_and_view_mean():
    """lambda = 0 is the plain mean absolute error, averaged over views."""
    rng = np.random.default_rng(4)
    imgs = [rng.uniform(size=(3, 8, 8)), rng.uniform(size=(3, 5, 6))]
    tg = [rng.uniform(size=i.shape) for i in imgs]
    per, total, _ = oracle.dssim_l1_loss(imgs, tg, lam=0.0)
    np.testing.assert_allclose(per, [np.abs(a - b).mean() for a, b in zip(imgs, tg)], rtol=1e-14)
    np.testing.assert_allclose(total, per.mean(), rtol=1e-14)
