"""The C ABI library on a machine without a GPU: it loads, exports every
symbol include/mvgs.h declares, and its host-only calls (layout and argument
checks) behave.  No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_12727_gb300 import build
    build.build()
    from paper_2506_12727_gb300 import mvgs
    return mvgs


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mvgs_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert {"mvgs_render_views", "mvgs_render_views_backward", "mvgs_dssim_loss", "mvgs_adc_accumulate"} <= declared
    so = ctypes.CDLL(lib.load_library.__globals__["_build"].LIB)
    for name in sorted(declared):
        assert hasattr(so, name), name
    assert declared == set(lib.EXPORTS)


def test_struct_sizes_match_header(lib):
    assert ctypes.sizeof(lib.Camera) == 88
    assert ctypes.sizeof(lib.Config) == 32
    assert ctypes.sizeof(lib.Scene) == 56


def test_layout_is_aligned_and_consistent(lib):
    cams = synth.make_cameras([(1264, 832), (800, 600), (17, 5)])
    cfg = lib.make_config((16, 16))
    L = lib.render_layout(1000, lib.make_cameras(cams), cfg, lib.Capacity(3000, 100_000))
    offs = [getattr(L, f) for f in lib._LAYOUT_FIELDS[2:]]
    assert all(o % 256 == 0 for o in offs)
    assert offs == sorted(offs) and L.state_bytes >= offs[-1]
    assert L.tiles == 79 * 52 + 50 * 38 + 2 * 1
    assert L.pixels == 1264 * 832 + 800 * 600 + 17 * 5
    assert L.off_rec_offsets == 256  # fixed: mvgs_adc_accumulate finds the record map there
    # the workspace grows with the capacities
    L2 = lib.render_layout(1000, lib.make_cameras(cams), cfg, lib.Capacity(6000, 200_000))
    assert L2.workspace_bytes > L.workspace_bytes and L2.state_bytes > L.state_bytes


@pytest.mark.parametrize("tile,ok", [((16, 16), True), ((8, 8), True), ((16, 32), True), ((32, 16), True),
                                     ((8, 32), True), ((32, 32), True), ((16, 64), True), ((32, 64), True),
                                     ((12, 16), False), ((4, 16), False), ((64, 32), False), ((8, 4), False),
                                     ((24, 8), False), ((16, 128), False)])
def test_tile_validation(lib, tile, ok):
    cams = lib.make_cameras(synth.make_cameras([(64, 64)]))
    if ok:
        lib.render_layout(10, cams, lib.make_config(tile), lib.Capacity(10, 10))
    else:
        with pytest.raises(lib.MvgsError) as e:
            lib.render_layout(10, cams, lib.make_config(tile), lib.Capacity(10, 10))
        assert e.value.status == lib.EINVAL


def test_bad_arguments_are_rejected(lib):
    cams = synth.make_cameras([(64, 64)])
    cc = lib.make_cameras(cams)
    cfg = lib.make_config()
    with pytest.raises(lib.MvgsError) as e:
        lib.render_layout(10, cc, cfg, lib.Capacity(2 ** 31, 10))
    assert e.value.status == lib.EOVERFLOW
    with pytest.raises(lib.MvgsError) as e:
        lib.render_layout(10, cc, cfg, lib.Capacity(10, 2 ** 32))
    assert e.value.status == lib.EOVERFLOW
    with pytest.raises(lib.MvgsError) as e:
        lib.render_layout(-1, cc, cfg, lib.Capacity(10, 10))
    assert e.value.status == lib.EINVAL
    bad = lib.make_cameras(synth.make_cameras([(0, 64)]))
    with pytest.raises(lib.MvgsError) as e:
        lib.render_layout(10, bad, cfg, lib.Capacity(10, 10))
    assert e.value.status == lib.EINVAL
    assert "empty image" in lib.last_error()
    # tile coordinates travel in 12-bit fields: at most 4095 tiles along an axis of a view
    wide = lib.make_cameras(synth.make_cameras([(8 * 4095, 64)]))
    lib.render_layout(10, wide, lib.make_config((8, 8)), lib.Capacity(10, 10))
    wider = lib.make_cameras(synth.make_cameras([(8 * 4095 + 1, 64)]))
    with pytest.raises(lib.MvgsError) as e:
        lib.render_layout(10, wider, lib.make_config((8, 8)), lib.Capacity(10, 10))
    assert e.value.status == lib.EOVERFLOW
    assert "4095 tiles per axis" in lib.last_error()
    cfg.flags = 16  # only bits 1, 2, 4 and 8 (masked partial, depth, capturable, pixel stats) are defined
    with pytest.raises(lib.MvgsError):
        lib.render_layout(10, cc, cfg, lib.Capacity(10, 10))
    cfg.flags = lib.FLAG_MASKED_PARTIAL
    lib.render_layout(10, cc, cfg, lib.Capacity(10, 10))


def test_dssim_workspace_size(lib):
    hw = np.array([[832, 1264], [5, 7]], np.int32)
    n = lib.dssim_workspace_size(hw)
    P = 832 * 1264 + 35
    assert n >= 3 * 3 * P * 4


def test_flag_constants_match_header(lib):
    src = open(os.path.join(ROOT, "include", "mvgs.h")).read()
    flags = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define MVGS_(FLAG_[A-Z_]+)\s+(\d+)u", src)}
    assert flags == {"FLAG_MASKED_PARTIAL": 1, "FLAG_DEPTH": 2, "FLAG_CAPTURABLE": 4, "FLAG_PIXEL_STATS": 8}
    for name, value in flags.items():
        assert getattr(lib, name) == value, name
