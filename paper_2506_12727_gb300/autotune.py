"""Tile-size / pixels-per-thread / shared-memory-batch autotuner for the
rasterizer.

The tile size decides how many (Gaussian, tile) entries are sorted; the strip
shape decides how the blend kernels spread a tile over warps; the batch is how
many Gaussians a warp stages in shared memory at a time.  None of them
changes the rendered image.  `autotune` times one forward + backward of each candidate
on the caller's scene and cameras (CUDA events, after one warm-up) and returns
the fastest; results are cached per (Gaussians, view resolutions) signature.
"""
from __future__ import annotations

import torch

from . import mvgs

# (tile, pixels per lane (0: automatic), Gaussians per shared-memory batch (0: automatic))
CANDIDATES = (
    ((16, 16), 0, 0), ((16, 32), 0, 0), ((16, 32), 2, 0), ((32, 32), 0, 0), ((16, 64), 0, 0), ((16, 64), 2, 0),
    ((16, 64), 0, 64), ((16, 64), 0, 192), ((32, 64), 0, 0), ((32, 64), 0, 64), ((32, 64), 0, 192), ((32, 16), 0, 0),
)

_cache: dict = {}


def _signature(n, cams):
    return (int(n), tuple((int(w), int(h)) for w, h in zip(cams.width, cams.height)))


def _time_config(scene_c, cams, tile, ppt, wb, grads, reps):
    rz = mvgs.Rasterizer(cams, tile=tile, pixels_per_thread=ppt, smem_batch=wb)
    img = rz.forward(scene_c)
    dimg = torch.full_like(img, 1e-3)
    rz.backward(scene_c, dimg, grads)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        rz.forward(scene_c, images=img)
        rz.backward(scene_c, dimg, grads)
    b.record(s)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    keys = int(rz.needed.keys)
    del rz
    return ms, keys


def autotune(scene_c, cams, params, candidates=CANDIDATES, reps=2, key_budget=None):
    """Returns ((tile_w, tile_h), pixels_per_thread, {candidate: ms}, smem_batch).
    `params` are the scene's device tensors (for gradient buffers);
    candidates needing more than `key_budget` keys are skipped."""
    sig = _signature(scene_c.n, cams)
    if sig in _cache:
        return _cache[sig]
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    timings = {}
    best = None
    for tile, ppt, wb in candidates:
        try:
            ms, keys = _time_config(scene_c, cams, tile, ppt, wb, grads, reps)
        except mvgs.MvgsError:
            continue
        if key_budget is not None and keys > key_budget:
            continue
        timings[f"{tile[0]}x{tile[1]}/ppt{ppt or 'auto'}/batch{wb or 'auto'}"] = round(ms, 3)
        if best is None or ms < best[0]:
            best = (ms, tile, ppt, wb)
        torch.cuda.empty_cache()
    if best is None:
        raise RuntimeError("no tile configuration ran")
    result = (best[1], best[2], timings, best[3])
    _cache[sig] = result
    return result
