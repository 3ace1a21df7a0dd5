"""Oracle of the pixel selection for thread-efficient partial rendering
(Sec. 5.1.1, Alg. 3) -- TEST INFRASTRUCTURE ONLY.

The paper renders, per tile and viewpoint, a sub-sample of the pixels given
as an index array, and leaves the sampling rule open.  The rule adopted:
view v renders pixel (x, y) when its cell (cx, cy) = (x // cell_w, y // cell_h)
has

    floor(group * (h >> 32) / 2^32) == v mod group,

h the SplitMix64 output number c + 1, c = 2^32 cy + cx, of the stream seeded
with `seed` (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output number k is mix(seed + k * gamma) with
gamma = 0x9e3779b97f4a7c15 and mix the published 64-bit finalizer.  Written
here with Python integers (exact 64-bit wrap-around by masking), one pixel at
a time for small cases and vectorised over numpy uint64 for whole images.

A partially rendered pixel takes exactly the value the full render gives it,
so the oracle of the partial render is the full oracle at the sampled pixels,
and the oracle of its backward is the full backward with dL/dimage zero at
every unsampled pixel.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1


def splitmix64_mix(z: int) -> int:
    """The SplitMix64 output finalizer on one 64-bit integer."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def splitmix64_stream(seed: int, count: int) -> list[int]:
    """The first `count` outputs of SplitMix64 seeded with `seed`."""
    return [splitmix64_mix(seed + (k + 1) * GAMMA) for k in range(count)]


def pixel_slot(seed: int, x: int, y: int, group: int) -> int:
    """The view slot (0 .. group - 1) of pixel (x, y), one pixel at a time."""
    h = splitmix64_mix(seed + (((y << 32) | x) + 1) * GAMMA)
    return ((h >> 32) * group) >> 32


def slot_image(seed: int, width: int, height: int, group: int, cell=(1, 1)) -> np.ndarray:
    """The slot of every pixel of an image [height, width] (its cell's
    pixel_slot), vectorised in uint64."""
    with np.errstate(over="ignore"):
        ys, xs = np.meshgrid(np.arange(height, dtype=np.uint64) // np.uint64(cell[1]),
                             np.arange(width, dtype=np.uint64) // np.uint64(cell[0]), indexing="ij")
        c = (ys << np.uint64(32)) | xs
        z = np.uint64(seed & MASK64) + (c + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        h = z ^ (z >> np.uint64(31))
        return (((h >> np.uint64(32)) * np.uint64(group)) >> np.uint64(32)).astype(np.int64)


def sample_masks(cams, group: int, seed: int, cell=(1, 1)) -> list[np.ndarray]:
    """Per view, the boolean [H, W] mask of the pixels it renders."""
    out = []
    for v in range(cams.V):
        W, H = int(cams.width[v]), int(cams.height[v])
        out.append(slot_image(seed, W, H, group, cell) == (v % group))
    return out


def packed_mask(cams, group: int, seed: int, cell=(1, 1)) -> np.ndarray:
    """The sample masks flattened in the packed per-view pixel order."""
    return np.concatenate([m.reshape(-1) for m in sample_masks(cams, group, seed, cell)])
