"""Pins of the partial-render pixel selection (oracle/partial.py)."""
import numpy as np

import synth
from oracle import partial


def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 seeded with 0, as printed by the
    # reference implementation of the generator
    assert partial.splitmix64_stream(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_vectorised_slots_match_scalar_definition():
    rng = np.random.default_rng(5)
    for seed in (0, 1, 0xDEADBEEF12345678):
        for group in (1, 2, 3, 4, 7, 16):
            img = partial.slot_image(seed, 37, 23, group)
            for _ in range(40):
                x, y = int(rng.integers(0, 37)), int(rng.integers(0, 23))
                assert img[y, x] == partial.pixel_slot(seed, x, y, group)
            assert img.min() >= 0 and img.max() < group


def test_cells_share_one_slot():
    img = partial.slot_image(7, 40, 30, 4, cell=(16, 8))
    for cy in range(0, 30, 8):
        for cx in range(0, 40, 16):
            blk = img[cy:cy + 8, cx:cx + 16]
            assert (blk == partial.pixel_slot(7, cx // 16, cy // 8, 4)).all()


def test_views_of_a_group_partition_the_pixels():
    cams = synth.make_cameras([(64, 48)] * 4, seed=1)
    for group in (1, 2, 4):
        masks = partial.sample_masks(cams, group, seed=9)
        for first in range(0, 4, group):
            cover = sum(m.astype(int) for m in masks[first:first + group])
            assert (cover == 1).all()
    # views v and v + group take the same pixels
    masks = partial.sample_masks(cams, 2, seed=9)
    assert (masks[0] == masks[2]).all() and (masks[1] == masks[3]).all()


def test_sampled_fraction_is_one_over_group():
    # binomial(n, 1/group): within 5 standard deviations
    n = 1264 * 832
    for group in (2, 4, 8):
        frac = (partial.slot_image(3, 1264, 832, group) == 1).mean()
        sd = np.sqrt((1 / group) * (1 - 1 / group) / n)
        assert abs(frac - 1 / group) < 5 * sd
