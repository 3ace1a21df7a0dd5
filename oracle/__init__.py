"""CPU oracle for multi-view EWA splatting -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product library never calls it and
shares no code with it; it exists to say what the CUDA path must compute.

`mvgs_oracle.c` holds the splatting arithmetic (projection, sort, blend and
their derivatives) in double precision; `losses.py` holds the D-SSIM loss and
the densification statistics in numpy float64.  This module builds the C file
with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .losses import dssim_l1_loss, adc_statistics, gaussian_window  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mvgs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmvgs_oracle.so")
_lock = threading.Lock()
_lib = None

CAM_STRIDE = 22
# record-level ambiguity bits (see mvgs_oracle.c)
RA_RADIUS, RA_RGB_CLAMP, RA_J_CLAMP, RA_NEAR = 1, 2, 4, 8
# pixel-level ambiguity bits
PA_SUPPORT, PA_ALPHA_MIN, PA_T_MIN, PA_ALPHA_MAX, PA_RADIUS = 1, 2, 4, 16, 32
PA_FORWARD = PA_SUPPORT | PA_ALPHA_MIN | PA_T_MIN | PA_RADIUS


def build(force: bool = False) -> str:
    """Compiles the oracle shared library (plain C, no GPU)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_count_keys.restype = ctypes.c_int64
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def cams_array(cams) -> np.ndarray:
    """Packs a synth.Cameras into the oracle's [V, 22] float64 layout."""
    V = cams.V
    out = np.zeros((V, CAM_STRIDE), dtype=np.float64)
    out[:, 0] = cams.width
    out[:, 1] = cams.height
    out[:, 2] = cams.fx
    out[:, 3] = cams.fy
    out[:, 4] = cams.cx
    out[:, 5] = cams.cy
    out[:, 6:15] = cams.viewmat[:, :, :3].astype(np.float64).reshape(V, 9)
    out[:, 15:18] = cams.viewmat[:, :, 3]
    out[:, 18:21] = cams.campos
    out[:, 21] = cams.near
    return out


def layout(cams, tile):
    tw, th = tile
    tiles_x = -(-cams.width.astype(np.int64) // tw)
    tiles_y = -(-cams.height.astype(np.int64) // th)
    tile_base = np.zeros(cams.V + 1, dtype=np.int64)
    tile_base[1:] = np.cumsum(tiles_x * tiles_y)
    pix_base = np.zeros(cams.V + 1, dtype=np.int64)
    pix_base[1:] = np.cumsum(cams.pixels())
    return tiles_x, tiles_y, tile_base, pix_base


def project(scene, cams, tile=(16, 16)) -> dict:
    """Dense projection of every (view, Gaussian) pair; arrays are [V*N, ...]."""
    lib = _load()
    N, V = scene.n, cams.V
    R = N * V
    out = dict(valid=np.zeros(R, np.int32), xy=np.zeros((R, 2)), conic=np.zeros((R, 3)), cov=np.zeros((R, 3)),
               opac=np.zeros(R), rgb=np.zeros((R, 3)), clampmask=np.zeros(R, np.int32), depth=np.zeros(R),
               radius=np.zeros(R, np.int32), rect=np.zeros((R, 4), np.int32), amb=np.zeros(R, np.int32))
    keep = [_c(scene.means, np.float32), _c(scene.log_scales, np.float32), _c(scene.quats, np.float32),
            _c(scene.opacity_logits, np.float32), _c(scene.sh, np.float32), cams_array(cams)]
    lib.orc_project(ctypes.c_int(N), ctypes.c_int(scene.sh_degree), *[_p(k) for k in keep[:5]], ctypes.c_int(V),
                    _p(keep[5]), ctypes.c_int(tile[0]), ctypes.c_int(tile[1]),
                    *[_p(out[k]) for k in ("valid", "xy", "conic", "cov", "opac", "rgb", "clampmask", "depth",
                                           "radius", "rect", "amb")])
    out["N"], out["V"], out["tile"] = N, V, tuple(tile)
    return out


def sort_keys(cams, tile, valid, rect, depth32, window=None):
    """Keys (global tile << 32 | float32 depth bits) sorted by (key, Gaussian
    index); returns (keys uint64 [K], records int32 [K] = v*N+g, ranges int64
    [tiles, 2]).  With `window` ([V, 4] pixel boxes) only the tiles that
    intersect the boxes get keys."""
    lib = _load()
    valid = _c(valid, np.int32)
    rect = _c(rect, np.int32)
    depth32 = _c(depth32, np.float32)
    V = cams.V
    N = valid.shape[0] // V
    win = _window_arg(cams, window)
    K = int(lib.orc_count_keys(ctypes.c_int(N), ctypes.c_int(V), ctypes.c_int(tile[0]), ctypes.c_int(tile[1]),
                               _p(valid), _p(rect), _p(win)))
    _, _, tile_base, _ = layout(cams, tile)
    keys = np.zeros(max(K, 1), np.uint64)
    recs = np.zeros(max(K, 1), np.int32)
    ranges = np.zeros((int(tile_base[-1]), 2), np.int64)
    ca = cams_array(cams)
    lib.orc_sort(ctypes.c_int(N), ctypes.c_int(V), _p(ca), ctypes.c_int(tile[0]), ctypes.c_int(tile[1]),
                 _p(valid), _p(rect), _p(depth32), _p(win), ctypes.c_int64(K), _p(keys), _p(recs), _p(ranges))
    return keys[:K], recs[:K], ranges


def _rec_args(P):
    return [_c(P["xy"], np.float64), _c(P["conic"], np.float64), _c(P["opac"], np.float64),
            _c(P["rgb"], np.float64), _c(P["depth"], np.float64), _c(P["radius"], np.int32),
            _c(P["amb"], np.int32)]


def _window_arg(cams, window):
    if window is None:
        return None
    w = np.asarray(window, dtype=np.int32).reshape(cams.V, 4)
    return _c(w, np.int32)


def render(cams, P, S, bg=(0.0, 0.0, 0.0), window=None, want_hash=False):
    """Front-to-back blending (Eq. 1) of every pixel (or a window per view).
    `S` is the (keys, recs, ranges) triple from sort_keys.  Returns packed
    image [sum 3HW], final T [sum HW], list position one past the last
    contributor [sum HW] and pixel ambiguity bits [sum HW] (and, if asked,
    a per-pixel hash of the contributor ids)."""
    lib = _load()
    _, _, _, pix_base = layout(cams, P["tile"])
    npx = int(pix_base[-1])
    img = np.zeros(3 * npx)
    T = np.zeros(npx)
    last = np.zeros(npx, np.int64)
    amb = np.zeros(npx, np.int32)
    chash = np.zeros(npx, np.uint64)
    depth = np.zeros(npx)
    ca = cams_array(cams)
    bgv = np.asarray(bg, dtype=np.float64)
    ra = _rec_args(P)
    ranges = _c(S[2], np.int64)
    recs = _c(S[1], np.int32)
    win = _window_arg(cams, window)
    lib.orc_render(ctypes.c_int(P["N"]), ctypes.c_int(cams.V), _p(ca), ctypes.c_int(P["tile"][0]),
                   ctypes.c_int(P["tile"][1]), _p(bgv), *[_p(a) for a in ra], _p(ranges), _p(recs), _p(win),
                   _p(img), _p(T), _p(last), _p(amb), _p(chash), _p(depth))
    if want_hash:
        return img, T, last, amb, chash, depth
    return img, T, last, amb


def render_pixels_bruteforce(cams, P, pixels, bg=(0.0, 0.0, 0.0)):
    """Tile-free reference for individual pixels: `pixels` is [n, 3] of (v, x, y)."""
    lib = _load()
    pix = _c(pixels, np.int32)
    n = pix.shape[0]
    C = np.zeros((n, 3))
    T = np.zeros(n)
    nc = np.zeros(n, np.int32)
    amb = np.zeros(n, np.int32)
    ca = cams_array(cams)
    bgv = np.asarray(bg, dtype=np.float64)
    ra = _rec_args(P)
    valid = _c(P["valid"], np.int32)
    lib.orc_render_pixels_bruteforce(ctypes.c_int(P["N"]), ctypes.c_int(cams.V), _p(ca), _p(bgv), _p(valid),
                                     *[_p(a) for a in ra], ctypes.c_int(n), _p(pix), _p(C), _p(T), _p(nc), _p(amb))
    return C, T, nc, amb


def render_backward(cams, P, S, dimg, bg=(0.0, 0.0, 0.0), window=None):
    """Per-record 2D gradients [V*N, 9] = (dmean2d x, y, dconic A, B, C,
    dopacity, drgb r, g, b) and E1 terms [V*N] from dL/dimage (packed)."""
    lib = _load()
    R = P["N"] * cams.V
    g2d = np.zeros((R, 9))
    e1 = np.zeros(R)
    ca = cams_array(cams)
    bgv = np.asarray(bg, dtype=np.float64)
    ra = _rec_args(P)
    d = _c(dimg, np.float64)
    win = _window_arg(cams, window)
    lib.orc_render_backward(ctypes.c_int(P["N"]), ctypes.c_int(cams.V), _p(ca), ctypes.c_int(P["tile"][0]),
                            ctypes.c_int(P["tile"][1]), _p(bgv), *[_p(a) for a in ra], _p(_c(S[2], np.int64)),
                            _p(_c(S[1], np.int32)), _p(win), _p(d), _p(g2d), _p(e1))
    return g2d, e1


def project_backward(scene, cams, tile, g2d):
    """3D parameter gradients from per-record 2D gradients, summed over views."""
    lib = _load()
    N, k = scene.n, (scene.sh_degree + 1) ** 2
    out = dict(means=np.zeros((N, 3)), log_scales=np.zeros((N, 3)), quats=np.zeros((N, 4)),
               opacity_logits=np.zeros(N), sh=np.zeros((N, k, 3)))
    keep = [_c(scene.means, np.float32), _c(scene.log_scales, np.float32), _c(scene.quats, np.float32),
            _c(scene.opacity_logits, np.float32), _c(scene.sh, np.float32)]
    ca = cams_array(cams)
    lib.orc_project_backward(ctypes.c_int(N), ctypes.c_int(scene.sh_degree), *[_p(a) for a in keep],
                             ctypes.c_int(cams.V), _p(ca), ctypes.c_int(tile[0]), ctypes.c_int(tile[1]),
                             _p(_c(g2d, np.float64)),
                             *[_p(out[n]) for n in ("means", "log_scales", "quats", "opacity_logits", "sh")])
    return out


def sh_basis(deg, dirs):
    lib = _load()
    d = _c(dirs, np.float64).reshape(-1, 3)
    out = np.zeros((d.shape[0], (deg + 1) ** 2))
    lib.orc_sh_basis(ctypes.c_int(deg), ctypes.c_int(d.shape[0]), _p(d), _p(out))
    return out


def quat_to_rotation(q):
    lib = _load()
    qq = _c(q, np.float64).reshape(-1, 4)
    out = np.zeros((qq.shape[0], 3, 3))
    lib.orc_quat_to_rotation(ctypes.c_int(qq.shape[0]), _p(qq), _p(out))
    return out


def forward(scene, cams, tile=(16, 16), bg=(0.0, 0.0, 0.0), window=None):
    """Projection, sort and blend of all views; returns a dict with the
    projected records `P`, the sorted lists `S` and the render outputs."""
    P = project(scene, cams, tile)
    S = sort_keys(cams, tile, P["valid"], P["rect"], P["depth"].astype(np.float32), window)
    img, T, last, amb, chash, depth = render(cams, P, S, bg, window, want_hash=True)
    return dict(P=P, S=S, img=img, T=T, last=last, amb=amb, chash=chash, depth=depth)


def backward(scene, cams, fwd, dimg, tile=(16, 16), bg=(0.0, 0.0, 0.0), window=None):
    g2d, e1 = render_backward(cams, fwd["P"], fwd["S"], dimg, bg, window)
    grads = project_backward(scene, cams, tile, g2d)
    return grads, g2d, e1
