"""Oracle for the photometric loss and the densification statistics --
TEST INFRASTRUCTURE ONLY (numpy float64, no GPU, never called by the product).

D-SSIM (Sec. 5.1.2, SSIM equations): SSIM = (2 mu1 mu2 + C1)(2 tau12 + C2) /
((mu1^2 + mu2^2 + C1)(tau1^2 + tau2^2 + C2)) with local moments taken against
a Gaussian kernel K_sigma; D-SSIM = 1 - SSIM.  Readings used here (the paper
leaves them open): 11x11 window, sigma = 1.5, discrete kernel normalised to
sum 1, zero padding, single scale, C1 = 0.01^2 and C2 = 0.03^2 for unit-range
images, SSIM averaged over channels and pixels of a view.

Loss per view v: L_v = (1 - lambda) mean|I - I*| + lambda (1 - SSIM_v)
(photometric l1 plus D-SSIM, Sec. 3); batch loss = mean over views.

Densification statistics (Sec. 5.2.2): for each Gaussian,
  E_old = || sum_views sum_pixels dL/dp ||,
  E_1   = sum_views sum_pixels || dL/dp ||,
  E_2   = sum_views || sum_pixels dL/dp ||,
with dL/dp the gradient of the loss with respect to the Gaussian's projected
2D mean in the view's pixel units.
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    """1D Gaussian taps, normalised to sum 1; the 2D window is their outer product."""
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    w = np.exp(-(x * x) / (2.0 * sigma * sigma))
    return w / w.sum()


def _filter_axis(a: np.ndarray, w: np.ndarray, axis: int) -> np.ndarray:
    """'same'-size correlation along one axis with zero padding."""
    h = len(w) // 2
    n = a.shape[axis]
    pad = [(0, 0)] * a.ndim
    pad[axis] = (h, h)
    ap = np.pad(a, pad)
    out = np.zeros_like(a, dtype=np.float64)
    for k in range(len(w)):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(k, k + n)
        out += w[k] * ap[tuple(sl)]
    return out


def blur(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Local weighted mean over the last two axes (H, W)."""
    return _filter_axis(_filter_axis(a, w, a.ndim - 1), w, a.ndim - 2)


def ssim_map(i1: np.ndarray, i2: np.ndarray, w: np.ndarray):
    """SSIM map and the local moments of one [C, H, W] image pair."""
    m1, m2 = blur(i1, w), blur(i2, w)
    m11, m22, m12 = blur(i1 * i1, w), blur(i2 * i2, w), blur(i1 * i2, w)
    t11 = m11 - m1 * m1
    t22 = m22 - m2 * m2
    t12 = m12 - m1 * m2
    a1 = 2.0 * m1 * m2 + C1
    a2 = 2.0 * t12 + C2
    b1 = m1 * m1 + m2 * m2 + C1
    b2 = t11 + t22 + C2
    S = (a1 * a2) / (b1 * b2)
    return S, dict(m1=m1, m2=m2, a1=a1, a2=a2, b1=b1, b2=b2)


def dssim_l1_loss(imgs, targets, lam: float = 0.2, window: int = 11, sigma: float = 1.5,
                  want_grad: bool = True):
    """Per-view losses [V], batch loss and dLoss/dimage (list of [C,H,W]) for
    Loss = mean_v [(1 - lam) mean|I_v - I*_v| + lam (1 - SSIM(I_v, I*_v))].

    Gradient of the mean SSIM with respect to I1 at pixel p (chain rule through
    the blurred moments m1 = K*I1, m11 = K*I1^2, m12 = K*(I1 I2); the adjoint of
    the zero-padded correlation with a symmetric kernel is the same filter):
      dS/dm1  = S (2 m2/a1 - 2 m2/a2 - 2 m1/b1 + 2 m1/b2)
      dS/dm11 = -S / b2
      dS/dm12 = 2 S / a2
      dmeanS/dI1 = [K*(dS/dm1) + 2 I1 K*(dS/dm11) + I2 K*(dS/dm12)] / (C H W)
    """
    w = gaussian_window(window, sigma)
    V = len(imgs)
    losses = np.zeros(V)
    grads = []
    for v in range(V):
        i1 = np.asarray(imgs[v], dtype=np.float64)
        i2 = np.asarray(targets[v], dtype=np.float64)
        n = i1.size
        S, m = ssim_map(i1, i2, w)
        l1 = np.abs(i1 - i2).mean()
        losses[v] = (1.0 - lam) * l1 + lam * (1.0 - S.mean())
        if want_grad:
            dS_dm1 = S * (2.0 * m["m2"] / m["a1"] - 2.0 * m["m2"] / m["a2"] - 2.0 * m["m1"] / m["b1"]
                          + 2.0 * m["m1"] / m["b2"])
            dS_dm11 = -S / m["b2"]
            dS_dm12 = 2.0 * S / m["a2"]
            dmean = (blur(dS_dm1, w) + 2.0 * i1 * blur(dS_dm11, w) + i2 * blur(dS_dm12, w)) / n
            g = (1.0 - lam) * np.sign(i1 - i2) / n - lam * dmean
            grads.append(g / V)
    return losses, losses.mean(), grads


def adc_statistics(g2d: np.ndarray, e1: np.ndarray, valid: np.ndarray, V: int):
    """Per-Gaussian E_1, E_2, E_old and the visible-view count from dense
    per-record arrays ([V*N, >=2] positional gradients in columns 0..1,
    [V*N] E_1 terms, [V*N] visibility)."""
    N = valid.shape[0] // V
    gxy = np.asarray(g2d, dtype=np.float64)[:, :2].reshape(V, N, 2)
    vis = np.asarray(valid).reshape(V, N) != 0
    E1 = np.asarray(e1, dtype=np.float64).reshape(V, N).sum(axis=0)
    E2 = np.sqrt((gxy ** 2).sum(axis=2)).sum(axis=0)
    Eold = np.sqrt((gxy.sum(axis=0) ** 2).sum(axis=1))
    denom = vis.sum(axis=0).astype(np.float64)
    return E1, E2, Eold, denom
