"""Oracle of the 3D distance-aware D-SSIM loss (Sec. 5.1.2) and of the merged
image it is computed on -- TEST INFRASTRUCTURE ONLY.

Readings of the paper (it leaves these open):
  - surface point of a pixel: the expected camera depth of the blend,
    z = sum_i alpha_i T_i z_i / (1 - T_final), lifted through the pixel
    centre: X = R^T (z K^-1 (x + 0.5, y + 0.5, 1)^T - t).  A pixel whose
    accumulated opacity 1 - T_final is below 1e-3 has no surface point;
  - the kernel K*(p, q) = exp(-|X_q - X_p|^2 / (2 s_p^2)) over the 11 x 11
    pixel window around the centre p, with s_p = 1.5 z_p / f_x: the 2D
    window's sigma of 1.5 pixels carried to the centre's depth, so that on a
    fronto-parallel plane seen by one camera K* is the usual Gaussian window.
    The 1 / (2 pi s^2) factor cancels: the weights are normalised to sum 1
    over the window (neighbours outside the image, or without a surface
    point, take no part; a centre without a surface point keeps only itself);
  - the weights are constants of the loss (no gradient flows into depth);
  - the loss of one merged image is (1 - lambda) mean |I - I*| + lambda (1 -
    mean SSIM*), SSIM* the usual SSIM formula with K* in place of the 2D
    window, C1 = 0.01^2, C2 = 0.03^2, averaged over pixels and channels.
The merged image of a group of `group` views of one resolution takes every
pixel from the view its partial-render sample slot names (oracle.partial).
"""
from __future__ import annotations

import numpy as np

from .partial import slot_image

C1 = 0.01 ** 2
C2 = 0.03 ** 2
HALF = 5          # 11 x 11 window
SIGMA_PX = 1.5
MIN_OPACITY = 1e-3


def lift(depth_acc, final_T, cam, sigma_px=SIGMA_PX):
    """Surface points [3, H, W], kernel sigmas [H, W] (0 where the pixel has
    no surface point) of one view from its accumulated depth and final T.
    `cam`: dict with W, H, fx, fy, cx, cy, R [3, 3], t [3]."""
    H, W = cam["H"], cam["W"]
    depth_acc = np.asarray(depth_acc, np.float64).reshape(H, W)
    opac = 1.0 - np.asarray(final_T, np.float64).reshape(H, W)
    ok = opac >= MIN_OPACITY
    z = np.where(ok, depth_acc / np.where(ok, opac, 1.0), 0.0)
    ys, xs = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    pc = np.stack([z * (xs - cam["cx"]) / cam["fx"], z * (ys - cam["cy"]) / cam["fy"], z])  # camera frame
    R, t = np.asarray(cam["R"], np.float64), np.asarray(cam["t"], np.float64)
    X = np.einsum("ji,jhw->ihw", R, pc - t[:, None, None])  # R^T (pc - t)
    sig = np.where(ok, sigma_px * z / cam["fx"], 0.0)
    return np.where(ok[None], X, 0.0), sig


def window_weights(X, sig):
    """Unnormalised weights w[k, y, x] of the 121 window offsets k = (du, dv)
    around each centre (y, x), and the offsets."""
    H, W = sig.shape
    offs = [(du, dv) for dv in range(-HALF, HALF + 1) for du in range(-HALF, HALF + 1)]
    w = np.zeros((len(offs), H, W))
    valid = sig > 0
    for k, (du, dv) in enumerate(offs):
        for y in range(H):
            qy = y + dv
            if qy < 0 or qy >= H:
                continue
            for x in range(W):
                qx = x + du
                if qx < 0 or qx >= W:
                    continue
                if du == 0 and dv == 0:
                    w[k, y, x] = 1.0
                elif valid[y, x] and valid[qy, qx]:
                    d2 = np.sum((X[:, qy, qx] - X[:, y, x]) ** 2)
                    w[k, y, x] = np.exp(-d2 / (2.0 * sig[y, x] ** 2))
    return w, offs


def _shift(a, du, dv):
    """b[..., y, x] = a[..., y + dv, x + du], zero outside."""
    H, W = a.shape[-2:]
    b = np.zeros_like(a)
    ys0, ys1 = max(0, -dv), min(H, H - dv)
    xs0, xs1 = max(0, -du), min(W, W - du)
    if ys1 > ys0 and xs1 > xs0:
        b[..., ys0:ys1, xs0:xs1] = a[..., ys0 + dv:ys1 + dv, xs0 + du:xs1 + du]
    return b


def dssim3d_loss(I1, I2, X, sig, lam=0.2, weights=None):
    """Loss of one image [3, H, W] and its gradient w.r.t. I1 (weights held
    constant).  Returns (loss, dL/dI1, ssim_map)."""
    I1 = np.asarray(I1, np.float64)
    I2 = np.asarray(I2, np.float64)
    if weights is None:
        weights = window_weights(X, sig)
    w, offs = weights
    wn = w / w.sum(0, keepdims=True)
    mu1 = np.zeros_like(I1)
    mu2 = np.zeros_like(I1)
    e11 = np.zeros_like(I1)
    e22 = np.zeros_like(I1)
    e12 = np.zeros_like(I1)
    for k, (du, dv) in enumerate(offs):
        a, b = _shift(I1, du, dv), _shift(I2, du, dv)
        mu1 += wn[k] * a
        mu2 += wn[k] * b
        e11 += wn[k] * a * a
        e22 += wn[k] * b * b
        e12 += wn[k] * a * b
    s11, s22, s12 = e11 - mu1 ** 2, e22 - mu2 ** 2, e12 - mu1 * mu2
    num1, num2 = 2 * mu1 * mu2 + C1, 2 * s12 + C2
    den1, den2 = mu1 ** 2 + mu2 ** 2 + C1, s11 + s22 + C2
    S = num1 * num2 / (den1 * den2)
    n = S.size
    loss = (1 - lam) * np.abs(I1 - I2).mean() + lam * (1.0 - S.mean())
    # dS/d(mu1, s11, s12) at each centre
    dS_dmu1 = (2 * mu2 * num2) / (den1 * den2) - S * 2 * mu1 / den1
    dS_ds11 = -S / den2
    dS_ds12 = 2 * num1 / (den1 * den2)
    # d mu1 / dI1(q) = wn, d s11 / dI1(q) = 2 wn (I1(q) - mu1), d s12 / dI1(q) = wn (I2(q) - mu2)
    A = dS_dmu1 - 2 * mu1 * dS_ds11 - mu2 * dS_ds12
    B = dS_ds11
    Cc = dS_ds12
    g = np.zeros_like(I1)
    for k, (du, dv) in enumerate(offs):
        # centre p = q - (du, dv) sends wn[k, p] (A + 2 B I1(q) + C I2(q)) to q
        wA = _shift(wn[k] * A, -du, -dv)
        wB = _shift(wn[k] * B, -du, -dv)
        wC = _shift(wn[k] * Cc, -du, -dv)
        g += wA + 2 * wB * I1 + wC * I2
    grad = (1 - lam) * np.sign(I1 - I2) / n - lam * g / n
    return loss, grad, S


def merge_views(imgs, cams_list, group, seed, first=0):
    """Merged image of views first .. first + group - 1 (one resolution):
    pixel (x, y) from view first + slot(x, y).  `imgs` is a list of arrays
    [C, H, W] per view; returns ([C, H, W], owner view [H, W])."""
    H, W = imgs[first].shape[-2:]
    slot = slot_image(seed, W, H, group)
    out = np.zeros_like(imgs[first])
    for k in range(group):
        m = slot == k
        out[..., m] = imgs[first + k][..., m]
    return out, first + slot
