"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the splatting method itself: it only draws
Gaussian parameters, pinhole cameras and target images from fixed seeds, with
the distributions of the workloads the paper trains on (Sec. 6, Table 4: scenes
seen by several cameras per iteration).  Both sides receive the same float32
arrays; the oracle widens them to float64 exactly.

Distributions (stand-ins for the MipNeRF-360 / OMMO / Deep Blending / Tanks &
Temples scenes, which are not available here):
  means            ~ U[-1, 1]^3
  log-scales       ~ N(-3, 0.5)
  rotations        ~ normalised N(0, I_4), stored as (w, x, y, z)
  opacity logits   ~ N(0, 1)
  SH degree 0      DC coefficient chosen so that the DC colour is U[0, 1]
  SH degree >= 1   DC ~ U[0, 1] (as a coefficient), higher bands ~ N(0, 0.05)
  cameras          look at the origin from a uniform random direction on a
                   sphere (or a shell of radii), horizontal FOV 60 degrees,
                   square pixels, principal point at the image centre,
                   OpenCV axes (+x right, +y down, +z forward), near plane 0.2
  targets          U[0, 1] per pixel and channel
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_SCENE = 0
SEED_CAMERAS = 1
SEED_TARGETS = 2
SEED_REQUESTS = 3


@dataclass
class Scene:
    means: np.ndarray           # [n, 3] float32
    log_scales: np.ndarray      # [n, 3] float32
    quats: np.ndarray           # [n, 4] float32, (w, x, y, z)
    opacity_logits: np.ndarray  # [n] float32
    sh: np.ndarray              # [n, (d+1)^2, 3] float32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity_logits[idx].copy(),
                     self.sh[idx].copy(), self.sh_degree)


@dataclass
class Cameras:
    width: np.ndarray    # [V] int32
    height: np.ndarray   # [V] int32
    fx: np.ndarray       # [V] float32
    fy: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    viewmat: np.ndarray  # [V, 3, 4] float32, world -> camera [R | t]
    campos: np.ndarray   # [V, 3] float32, camera centre in world space
    near: np.ndarray     # [V] float32

    @property
    def V(self) -> int:
        return int(self.width.shape[0])

    def subset(self, idx) -> "Cameras":
        idx = np.atleast_1d(np.asarray(idx))
        return Cameras(*(getattr(self, f)[idx].copy() for f in
                         ("width", "height", "fx", "fy", "cx", "cy", "viewmat", "campos", "near")))

    def pixels(self) -> np.ndarray:
        return (self.width.astype(np.int64) * self.height.astype(np.int64))


def make_scene(n: int, sh_degree: int, seed: int = SEED_SCENE) -> Scene:
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    log_scales = rng.normal(-3.0, 0.5, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(0.0, 1.0, size=(n,))
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    if sh_degree == 0:
        # DC basis value is 1 / (2 sqrt(pi)); the colour is that times the
        # coefficient plus 0.5, so this draws the colour itself from U[0, 1].
        sh[:, 0, :] = (rng.uniform(0.0, 1.0, size=(n, 3)) - 0.5) * (2.0 * math.sqrt(math.pi))
    else:
        sh[:, 0, :] = rng.uniform(0.0, 1.0, size=(n, 3))
        sh[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, k - 1, 3))
    f32 = np.float32
    return Scene(means.astype(f32), log_scales.astype(f32), q.astype(f32),
                 logits.astype(f32), sh.astype(f32), sh_degree)


def look_at(eye: np.ndarray, target=(0.0, 0.0, 0.0)) -> np.ndarray:
    """World->camera [R|t] (3x4) for a camera at `eye` looking at `target`,
    OpenCV axes; world +y is 'up' unless the view is within 1 degree of it."""
    eye = np.asarray(eye, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - eye
    z /= np.linalg.norm(z)
    up = np.array([0.0, 1.0, 0.0])
    if abs(float(z @ up)) > math.cos(math.radians(1.0)):
        up = np.array([0.0, 0.0, 1.0])
    x = np.cross(z, up)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=0)
    t = -R @ eye
    return np.concatenate([R, t[:, None]], axis=1)


def make_cameras(resolutions, radius=4.0, seed: int = SEED_CAMERAS,
                 fov_deg: float = 60.0, near: float = 0.2) -> Cameras:
    """One camera per (W, H) in `resolutions`.  `radius` is a float (sphere)
    or a (lo, hi) pair (uniform shell)."""
    rng = np.random.default_rng(seed)
    V = len(resolutions)
    W = np.array([r[0] for r in resolutions], dtype=np.int32)
    H = np.array([r[1] for r in resolutions], dtype=np.int32)
    f = (W.astype(np.float64) / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    vm = np.zeros((V, 3, 4))
    pos = np.zeros((V, 3))
    for v in range(V):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        r = radius if np.isscalar(radius) else rng.uniform(radius[0], radius[1])
        pos[v] = d * r
        vm[v] = look_at(pos[v])
    f32 = np.float32
    return Cameras(W, H, f.astype(f32), f.astype(f32), (W / 2.0).astype(f32), (H / 2.0).astype(f32),
                   vm.astype(f32), pos.astype(f32), np.full(V, near, dtype=f32))


def make_targets(cams: Cameras, seed: int = SEED_TARGETS) -> list:
    """U[0,1] target images, one [3, H, W] float32 array per view."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.0, 1.0, size=(3, int(h), int(w))).astype(np.float32)
            for w, h in zip(cams.width, cams.height)]


def pack_images(imgs) -> np.ndarray:
    """Concatenate per-view [3, H, W] images into the packed layout used by
    both sides: view v occupies [off[v], off[v+1]) with off[v+1]-off[v] = 3 H W."""
    return np.concatenate([np.ascontiguousarray(i, dtype=np.float32).reshape(-1) for i in imgs])


def view_offsets(cams: Cameras) -> np.ndarray:
    off = np.zeros(cams.V + 1, dtype=np.int64)
    off[1:] = np.cumsum(3 * cams.pixels())
    return off


# ---------------------------------------------------------------------------
# The five workloads (scene sizes, view batches, resolutions).
# ---------------------------------------------------------------------------
MIXED_RES = [(800, 600), (1264, 832), (1600, 1067), (1920, 1080)]
SERVE_RES = [(640, 480), (1280, 720), (1920, 1080)]


def workload(name: str):
    """Returns (scene, cameras, extras) for a named workload."""
    if name == "single_view_10k":
        return make_scene(10_000, 0), make_cameras([(128, 128)], radius=3.0), {"loss": "l1"}
    if name == "multiview_500k_1x1264x832":  # one view of the batch below (profiling-sized)
        return (make_scene(500_000, 3), make_cameras([(1264, 832)], radius=4.0),
                {"loss": "l1_dssim", "lambda_dssim": 0.2})
    if name == "multiview_500k_4x1264x832":
        return (make_scene(500_000, 3), make_cameras([(1264, 832)] * 4, radius=4.0),
                {"loss": "l1_dssim", "lambda_dssim": 0.2})
    if name == "uneven_3m_8views":
        rng = np.random.default_rng(SEED_CAMERAS + 100)
        res = [MIXED_RES[i] for i in rng.integers(0, len(MIXED_RES), size=8)]
        return make_scene(3_000_000, 3), make_cameras(res, radius=4.0), {"loss": "l1_dssim", "lambda_dssim": 0.2}
    if name == "diff_1m_16x1024x768":
        return make_scene(1_000_000, 3), make_cameras([(1024, 768)] * 16, radius=4.0), {"loss": "l1"}
    raise KeyError(name)


def poisson_requests(n_requests: int, rate_hz: float = 200.0, seed: int = SEED_REQUESTS):
    """Serving requests: arrival time, view count 1..16, a resolution per
    view from SERVE_RES and a pose on the radius 3..5 shell."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    reqs = []
    for i in range(n_requests):
        nv = int(rng.integers(1, 17))
        res = [SERVE_RES[j] for j in rng.integers(0, len(SERVE_RES), size=nv)]
        reqs.append({"t": float(t[i]), "resolutions": res, "cam_seed": int(rng.integers(0, 2**31 - 1))})
    return reqs


def off_axis_scene(n_out: int, n_in: int, sh_degree: int = 1, W: int = 64, H: int = 48, fov_deg: float = 60.0,
                   seed: int = 40):
    """Gaussians seen at steep angles, for the projection's behaviour far
    off the optical axis: two cameras facing each other (the first at the
    origin looking down +z, the second at z = 6 looking down -z), `n_out`
    Gaussians whose view-angle tangents in the first camera are 1.4 to 1.9
    times the half-FOV tangent on one or both axes (so their centres project
    outside the image), with scales large enough that they still reach
    into it, and `n_in` ordinary Gaussians inside the view.  Depths 1.8 to
    4.2 in both cameras."""
    rng = np.random.default_rng(seed)
    f = (W / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    Lx, Ly = (W / 2.0) / f, (H / 2.0) / f
    n = n_out + n_in
    z = rng.uniform(1.8, 4.2, size=n)
    ux = rng.uniform(-0.6, 0.6, size=n) * Lx
    uy = rng.uniform(-0.6, 0.6, size=n) * Ly
    # which axes are far out: x only, y only, or both, with either sign
    kind = rng.integers(0, 3, size=n_out)
    sx = rng.choice([-1.0, 1.0], size=n_out)
    sy = rng.choice([-1.0, 1.0], size=n_out)
    far_x = rng.uniform(1.4, 1.9, size=n_out) * Lx * sx
    far_y = rng.uniform(1.4, 1.9, size=n_out) * Ly * sy
    ux[:n_out] = np.where(kind != 1, far_x, ux[:n_out])
    uy[:n_out] = np.where(kind != 0, far_y, uy[:n_out])
    means = np.stack([ux * z, uy * z, z], 1)
    log_scales = np.empty((n, 3))
    log_scales[:n_out] = rng.normal(np.log(0.6), 0.2, size=(n_out, 3)) + np.log(z[:n_out, None] / 3.0)
    log_scales[n_out:] = rng.normal(-2.5, 0.4, size=(n_in, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(0.5, 1.0, size=n)
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = rng.uniform(0.0, 1.0, size=(n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, k - 1, 3))
    f32 = np.float32
    scene = Scene(means.astype(f32), log_scales.astype(f32), q.astype(f32), logits.astype(f32), sh.astype(f32),
                  sh_degree)
    vm = np.zeros((2, 3, 4))
    vm[0, :, :3] = np.eye(3)
    vm[1, :, :3] = np.diag([-1.0, 1.0, -1.0])
    vm[1, :, 3] = [0.0, 0.0, 6.0]
    # the second camera's far Gaussians: depth 6 - z must stay in 1.8 .. 4.2
    cams = Cameras(np.full(2, W, np.int32), np.full(2, H, np.int32), np.full(2, f, f32), np.full(2, f, f32),
                   np.full(2, W / 2.0, f32), np.full(2, H / 2.0, f32), vm.astype(f32),
                   np.array([[0, 0, 0], [0, 0, 6]], f32), np.full(2, 0.2, f32))
    return scene, cams
